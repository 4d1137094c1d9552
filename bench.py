"""Benchmark: decoded Gaussians/s (and p50/p99 scene-decode latency) of the B300 decode path.

A step is one whole scene decode (octree geometry -> positions, attribute tokens -> fp32
structure of arrays) of a synthetic paper-shaped scene already resident in HBM.  Default
workload: 1,000,000 Gaussians (900,000 after pruning), depth-16 octree, channel-wise
fixed-length attributes with per-channel widths drawn from 4..10 bits.  Other workloads:
--workload static (same scene, channel-wise static rANS, 151,552 lanes), learned (same scene,
learned context model, 4,096 lanes), small (20,000 Gaussians, depth 12, static rANS, 32 lanes).

With no --workload the run decodes the default scene in every coding mode: the fixed-length
decode is the headline line, and static rANS (4,096 and 151,552 lanes), the learned model
(4,096 lanes), the position-aware model and the small plain-method scene are sub-objects
("modes") with the same measurements, all but the small one on the same scene.

Prints one JSON line.  --impl reference times the CPU oracle on the headline workload instead.
Multi-GPU (torchrun): scenes are independent, so each rank decodes its own replica with no
collective; value = Gaussians decoded by all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "fixed": dict(n=1_000_000, seed=1000, depth=16, mode=0, geo_mode=0, lanes=0,
                  desc="fixed-length scene decode: N=1,000,000 Gaussians (900,000 after pruning), "
                       "depth-16 octree (raw tokens), 56 channels at 4..10 bits"),
    "static": dict(n=1_000_000, seed=1000, depth=16, mode=1, geo_mode=1, lanes=151552, geo_w=32,
                   desc="channel-wise static rANS scene decode: N=1,000,000 (900,000 kept), depth 16, "
                        "8-bit tokens, 151,552 lanes (one 32-warp CTA per SM), rANS-coded octree levels "
                        "at about 32 tokens per geometry lane"),
    "learned": dict(n=1_000_000, seed=1000, depth=16, mode=2, geo_mode=1, lanes=4096,
                    desc="learned-model scene decode: N=1,000,000 (900,000 kept), depth 16, 8-bit "
                         "tokens, 4,096 lanes, context MLP 4->64->64->256 trained 2,000 steps x 65,536 "
                         "tokens on the scene's own tokens"),
    "learned_pe": dict(n=1_000_000, seed=1000, depth=16, mode=3, geo_mode=1, lanes=28125,
                       desc="position-aware learned scene decode: N=1,000,000 (900,000 kept), depth 16, "
                            "8-bit tokens, 28,125 lanes (W = 32 rows per lane, the paper's fast group size), "
                            "context MLP over 4 previous tokens + Fourier positional embedding of the decoded "
                            "voxel (12 bands, 75 -> 32), Laplace head"),
    "learned_geo": dict(n=1_000_000, seed=1000, depth=16, mode=1, geo_mode=2, lanes=151552,
                        desc="learned geometry decode: N=1,000,000 (900,000 kept), depth 16, every octree level "
                             "of 4,096 or more nodes coded with the context MLP 4->64->64->256 conditioned on "
                             "the level above (contexts 8 b + k), about 128 tokens per geometry lane; static "
                             "channel-wise attributes at 151,552 lanes.  The geometry model is the architecture "
                             "with random-init weights frozen on the scene's own occupancy samples (no trainer "
                             "for explicit samples on the device): it times the decode, its bits are not a "
                             "trained model's"),
    "small": dict(n=20_000, seed=0, depth=12, mode=1, geo_mode=1, lanes=32,
                  desc="small static scene decode: N=20,000 (18,000 kept), depth 12, 32 lanes"),
}
METRIC = "decoded Gaussians/s"
WORKLOADS_DEFAULT = None  # the default workload's dict, set in main()

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one k_fixed launch on the
# default workload, from an ncu --set full capture of the present kernel: 43.95 MB read +
# 142.94 MB written (part of the 201.6 MB of output is still in L2 when the kernel ends).
K_FIXED_TRAFFIC = 43_947_776 + 142_937_344
# The same for one k_rans_attr launch of the static workload (151,552 lanes): 85.51 MB read +
# 192.59 MB written; and one k_learned_decode launch of the learned workload (4,096 lanes):
# 190.74 MB read + 297.41 MB written (the consumer's 4-byte stores, 32 lanes far apart).
K_RANS_ATTR_TRAFFIC = {151552: 85_508_096 + 192_589_312}
K_LEARNED_TRAFFIC = {4096: 190_743_040 + 297_414_144}


from paper_2607_12656_b300.workloads import BATCH, SERVE  # noqa: E402


def batch_specs(n_scenes: int, w_learned: int = 220, w_static: int = 32) -> list:
    from paper_2607_12656_b300 import workloads
    return workloads.batch_specs(n_scenes, w_learned, w_static)


def serve_specs(per_mode: int) -> list:
    from paper_2607_12656_b300 import workloads
    return workloads.serve_specs(per_mode)


TUNED = {}  # rows per lane chosen by the tuner for the batched workload, per coding mode


def build_batch(n_scenes: int, train_steps: int, specs=None, tune: bool = False):
    """All bitstreams of a multi-scene workload, generated, trained (every learned scene its
    own model, on its own tokens) and encoded by a pool of spawned workers.  With `tune`, the
    rows per lane of each coding mode are first chosen by the lane tuner (sgs_autotune: the
    fastest decode over W in 16..256) on that mode's median-size scene (a learned one with
    its own model), and every scene of the mode is encoded at that W."""
    from paper_2607_12656_b300 import workloads
    specs = batch_specs(n_scenes) if specs is None else specs
    if tune:
        from paper_2607_12656_b300 import learned, sgs
        from paper_2607_12656_b300.scenegen import make_scene
        from paper_2607_12656_b300.tune import LaneTuner
        tuner = LaneTuner()
        ctx = sgs.Context(0, 0)
        w_of = {}
        for mode in sorted({s[4] for s in specs if s[4] != 0}):
            mine = sorted((s for s in specs if s[4] == mode), key=lambda s: s[1])
            j, n, seed, depth, _, lanes = mine[len(mine) // 2]
            sc = make_scene(n, seed)
            model = (learned.train_and_freeze(ctx, sc, depth, lanes, steps=train_steps, batch=65536, seed=seed)
                     if mode == 2 else None)
            lanes = tuner.choose_lanes(ctx, sc.pos, sc.attr, mode=mode, depth=depth, reps=3, model=model)
            w_of[mode] = -(-(n - n // 10) // lanes)
        ctx.close()
        TUNED.update({{1: "static", 2: "learned"}[m]: w for m, w in w_of.items()})
        specs = [(j, n, seed, depth, mode, workloads.lanes_for(n, w_of[mode]) if mode in w_of else lanes)
                 for j, n, seed, depth, mode, lanes in specs]
    return specs, workloads.build(specs, train_steps)


def peaks() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """Samples SM clocks and throttle reasons with a streaming nvidia-smi (every 100 ms) while
    the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.samples = []
        self.proc = None
        self._t = None

    def _read(self):
        for line in self.proc.stdout:
            vals = [v.strip() for v in line.strip().split(",")]
            if len(vals) >= 6:
                self.samples.append(vals)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            time.sleep(0.3)  # first sample before the timed region
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self._t.join(timeout=5)

    def summary(self) -> dict:
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        num = lambda v: v.replace(".", "", 1).isdigit()
        sm = [float(s[0]) for s in self.samples if num(s[0])]
        mx = [float(s[1]) for s in self.samples if num(s[1])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if s[2 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def make_bitstream(w: dict, ctx=None, sc=None):
    """The workload's scene (or the given one, when it is the same scene) and its bitstream;
    learned modes train their model on the scene's own tokens on the device first."""
    from paper_2607_12656_b300 import sgs
    from paper_2607_12656_b300.scenegen import fixed_bits, make_scene
    if sc is None:
        sc = make_scene(w["n"], w["seed"])
    kw = dict(mode=w["mode"], depth=w["depth"], geo_mode=w["geo_mode"])
    if w["mode"] == 0:
        kw["bits"] = fixed_bits(w["seed"])
    else:
        kw["lanes"] = w["lanes"]
    if w.get("geo_w"):  # geometry lanes for throughput: about geo_w coded tokens per lane
        kw["geo_lanes"] = geo_lanes_for(sc, w)
    if w["geo_mode"] == 2:
        from paper_2607_12656_b300.scenegen import kaiming_init
        u, chan, _ = sgs.scene_geo_samples(sc.pos, sc.attr, w["depth"])
        kw["geo_model"] = sgs.sgs_freeze_samples(sgs.pack_weights(kaiming_init(7)), u, chan, 1)
    model = None
    if w["mode"] in (2, 3):
        from paper_2607_12656_b300 import learned
        train = learned.train_and_freeze if w["mode"] == 2 else learned.train_and_freeze_pe
        model = train(ctx, sc, w["depth"], w["lanes"], steps=w.get("train_steps", 2000), batch=65536, seed=1)
        kw["model"] = model
        kw["ctx"] = ctx
    return sc, sgs.scene_encode(sc.pos, sc.attr, **kw)


def geo_lanes_for(sc, w) -> int:
    """Geometry lanes giving about w["geo_w"] rANS-coded octree tokens per lane (a multiple
    of 32): the coded token count is read back from a first encode's header."""
    from paper_2607_12656_b300 import sgs
    probe = sgs.scene_encode(sc.pos, sc.attr, mode=0, depth=w["depth"], bits=4, geo_mode=1)
    n_coded = int(sgs.scene_query(probe).n_geo_coded)
    per = w["geo_w"] * 32
    return max(32, -(-n_coded // per) * 32)


SMS = 148  # B300: 2 dies x 74 SMs


def attr_roofline(mode: int, n: int, attr_bytes: int, attr_ms: float, pk: dict, lanes: int = 0) -> dict:
    """Roofline of the attribute decoder of a coded mode over its stage time (CUDA events on the
    attribute stream).  Algorithmic work per decoded symbol (56 per Gaussian):
      static rANS: the coded attribute section read once + 4 B written (HBM);
      learned: the integer softmax and cumulative table, 10 integer operations for each of the
        256 entries (ALU; peak = 148 SMs x 4 warp instructions x 32 lanes per clock at the
        maximum SM clock), with the 20,480 tensor-core MACs of layers 2-3 beside it;
      position-aware: 4 x 64 + 64 x 64 + 2 x 64 MACs per symbol and 75 x 64 per row (tensor)."""
    sec = attr_ms / 1e3
    syms = 56 * n
    bf16 = pk.get("bf16_tflops")
    bf16_src = "MEASURED_PEAKS.json bf16_tflops (measured, burst)" if bf16 else "fallback 1800"
    bf16 = bf16 or 1800.0
    if mode == 1:
        hbm = pk.get("hbm_gbs")
        src = "MEASURED_PEAKS.json hbm_gbs (measured)" if hbm else "fallback 6400"
        hbm = hbm or 6400.0
        alg = attr_bytes + 4 * syms
        ach = alg / sec / 1e9
        return {"kernel": "k_rans_attr (static rANS + dequant + SoA store)", "bound": "hbm", "achieved": ach,
                "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "peak_source": src, "algorithmic_bytes": alg,
                "traffic": K_RANS_ATTR_TRAFFIC.get(lanes) if n == 900_000 else None,
                "note": "issue-bound in practice: a dependent integer chain per symbol"}
    if mode == 2:
        mhz = pk.get("sm_max_mhz") or 2032.0
        peak = SMS * 4 * 32 * mhz * 1e6 / 1e9
        ops = 10 * 256 * syms
        ach = ops / sec / 1e9
        tf = 2 * 20480 * syms / sec / 1e12
        return {"kernel": "k_learned_decode (context MLP + integer softmax + rANS)", "bound": "alu",
                "achieved": ach, "peak": peak, "unit": "Gop/s", "frac": ach / peak,
                "peak_source": "derived: 148 SMs x 4 warp instructions x 32 lanes per clock at %.0f MHz" % mhz,
                "algorithmic_ops": ops, "traffic": K_LEARNED_TRAFFIC.get(lanes) if n == 900_000 else None,
                "tensor": {"achieved": tf, "peak": bf16, "unit": "TFLOP/s", "frac": tf / bf16,
                           "peak_source": bf16_src}}
    flops = 2 * (4 * 64 + 64 * 64 + 2 * 64) * syms + 2 * 75 * 64 * n
    ach = flops / sec / 1e12
    return {"kernel": "k_learned_pe (position-aware context MLP + Laplace CDF search + rANS)", "bound": "tensor",
            "achieved": ach, "peak": bf16, "unit": "TFLOP/s", "frac": ach / bf16, "peak_source": bf16_src,
            "algorithmic_flops": flops, "traffic": None,
            "note": "latency-bound in practice: dependent mma and requantisation chains per row step"}


def fixed_algorithmic_bytes(info, bits_np) -> int:
    n = info.n_rows
    read = sum(4 * ((n * int(b) + 31) // 32) for b in bits_np)
    return read + 4 * 56 * n


def measure(args, w, ctx, sc=None, cpu: bool = True, headline: bool = False) -> dict:
    """One coding mode of one scene: the timed decode (bitstream resident in HBM, L2 flushed
    before every step, CUDA events on the caller's stream), latency percentiles, stage split,
    CUDA-graph replay, the attribute kernel's roofline, the end-to-end figure through the
    public API (bitstream from pinned host memory, outputs read back), the CPU oracle on the
    same bitstream, and bits per Gaussian."""
    import torch
    from paper_2607_12656_b300 import sgs
    from paper_2607_12656_b300 import replicas
    rank, world, local = replicas.rank_info()
    sc, buf = make_bitstream(w, ctx, sc)
    train = None
    if w["mode"] in (2, 3):
        from paper_2607_12656_b300 import learned
        train = dict(learned.LAST_TRAIN)
    info = sgs.scene_query(buf)
    ctx.reserve(info.scratch_bytes)
    n = info.n_rows
    dev = torch.device("cuda", local)
    host_bits = torch.frombuffer(bytearray(buf), dtype=torch.uint8).pin_memory()
    bits = host_bits.to(dev)
    attr = torch.empty((56, n), device=dev)
    pos = torch.empty((3, n), device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # 256 MiB > 126 MB L2
    stream = torch.cuda.current_stream()

    def step():
        sgs.scene_decode(ctx, bits, info, attr, pos, None, None, stream)

    for _ in range(args.warmup):
        step()
    st = ctx.sync(stream)
    if st != sgs.OK:
        raise RuntimeError("decode status %s" % sgs.lib().sgs_strerror(st).decode())
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = ctx.launch_count()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
            stream.synchronize()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    launches = ctx.launch_count() - launches0
    # stage split from separate decodes with the context's stage events on (they add calls)
    ctx.profile(True)
    stage = []
    for k in range(min(args.steps, 100)):
        flush.zero_()
        step()
        stream.synchronize()
        stage.append(ctx.profile_read())
    ctx.profile(False)
    st = ctx.sync(stream)
    if st != sgs.OK:
        raise RuntimeError("decode status %s" % sgs.lib().sgs_strerror(st).decode())
    times = [a.elapsed_time(b) for a, b in ev]  # ms
    # the same decode captured once in a CUDA graph and replayed (no per-kernel launch cost)
    graph_times = []
    try:
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream()
        cap.wait_stream(stream)
        with torch.cuda.stream(cap):
            sgs.scene_decode(ctx, bits, info, attr, pos, None, None, cap)
            cap.synchronize()
            with torch.cuda.graph(g, stream=cap):
                sgs.scene_decode(ctx, bits, info, attr, pos, None, None, cap)
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.replay()
            b.record(stream)
            stream.synchronize()
            graph_times.append(a.elapsed_time(b))
        if ctx.sync(stream) != sgs.OK:
            graph_times = []
        del g
    except Exception as exc:  # graph capture unavailable: report eager numbers only
        print("graph capture failed: %s" % exc, file=sys.stderr)
        graph_times = []
    total_ms = replicas.max_over_ranks(sum(times), dev)  # the slowest replica sets the time
    ms_per_step = total_ms / args.steps
    value = n * world * args.steps / (total_ms / 1e3)

    # end to end through the public API: pinned host bitstream -> device, decode, outputs -> host
    host_attr = torch.empty((56, n), dtype=torch.float32).pin_memory()
    host_pos = torch.empty((3, n), dtype=torch.float32).pin_memory()
    reps = max(3, min(args.steps, 50 if w["mode"] < 2 else 10))
    e2e_times = []
    for k in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        bits.copy_(host_bits, non_blocking=True)
        step()
        host_attr.copy_(attr, non_blocking=True)
        host_pos.copy_(pos, non_blocking=True)
        b.record(stream)
        stream.synchronize()
        e2e_times.append(a.elapsed_time(b))
    # the same with the outputs left on the device for a renderer: upload, decode, status read
    dev_times = []
    for k in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        bits.copy_(host_bits, non_blocking=True)
        step()
        st_k = ctx.sync(stream)  # reads the 4-byte status word back
        b.record(stream)
        stream.synchronize()
        if st_k != sgs.OK:
            raise RuntimeError("decode status %d" % st_k)
        dev_times.append(a.elapsed_time(b))

    pk = peaks()
    hbm = pk.get("hbm_gbs")
    line = {"value": value, "unit": "Gaussians/s", "ms_per_step": ms_per_step,
            "config": {"workload": w["desc"], "n_rows": n, "bitstream_bytes": len(buf),
                       "bits_per_gaussian": 8.0 * len(buf) / n if n else None,
                       "l2": "flushed (256 MiB write) before every timed step",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "latency_ms": {"p50": float(np.percentile(times, 50)), "p99": float(np.percentile(times, 99)),
                           "min": min(times), "max": max(times)},
            "stage_ms": {"geometry_tokens": float(np.mean([s[0] for s in stage])),
                         "octree_positions": float(np.mean([s[1] for s in stage])),
                         "attributes": float(np.mean([s[2] for s in stage])),
                         "whole_decode": float(np.mean([s[3] for s in stage])),
                         "note": "attributes run on their own stream, concurrent with geometry (the "
                                 "position-aware model after it); separate decodes with stage events recorded"},
            "wall_s": wall}
    if graph_times:
        gms = float(np.mean(graph_times))
        line["graph"] = {"ms_per_step": gms, "value": n * world / (gms / 1e3),
                         "p50_ms": float(np.percentile(graph_times, 50)),
                         "p99_ms": float(np.percentile(graph_times, 99)),
                         "note": "same decode captured in one CUDA graph and replayed"}
    if w["mode"] == 0:
        from paper_2607_12656_b300.scenegen import fixed_bits
        alg = fixed_algorithmic_bytes(info, fixed_bits(w["seed"]))
        att_ms = line["stage_ms"]["attributes"]
        ach = alg / (att_ms / 1e3) / 1e9
        line["roofline"] = {"kernel": "k_fixed (fixed-length unpack + dequant + SoA store)", "bound": "hbm",
                            "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm if hbm else None,
                            "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if hbm else "fallback 6400",
                            "algorithmic_bytes": alg,
                            "traffic": args.traffic if args.traffic is not None else
                            (K_FIXED_TRAFFIC if headline else None)}
        geo_alg = info.n_geo + 12 * n
        line["roofline_octree"] = {"bound": "hbm", "algorithmic_bytes": geo_alg,
                                   "achieved": geo_alg / (line["stage_ms"]["octree_positions"] / 1e3) / 1e9,
                                   "unit": "GB/s"}
    else:
        line["config"]["attr_bits_per_gaussian"] = 8.0 * (info.total_len - info.off[7]) / n
        rl = attr_roofline(w["mode"], n, info.total_len - info.off[7], line["stage_ms"]["attributes"], pk, w.get("lanes", 0))
        line["roofline"] = rl
    if train is not None:
        line["training"] = {"steps": train["steps"], "batch": train["batch"], "device_ms": train["ms"],
                            "tokens_per_s": train["steps"] * train["batch"] / (train["ms"] / 1e3),
                            "final_loss_bits_per_token": train["final_bits"],
                            "note": "context-model training on the GPU before the timed decodes (not timed in value)"}
    line["e2e"] = {"value": n * len(e2e_times) / (sum(e2e_times) / 1e3), "unit": "Gaussians/s",
                   "h2d_bytes_per_step": len(buf), "d2h_bytes_per_step": 4 * 59 * n,
                   "ms_per_step": sum(e2e_times) / len(e2e_times),
                   "note": "bitstream uploaded from pinned memory, every decoded fp32 array read back"}
    line["e2e_outputs_on_device"] = {"value": n * len(dev_times) / (sum(dev_times) / 1e3), "unit": "Gaussians/s",
                                     "h2d_bytes_per_step": len(buf), "d2h_bytes_per_step": 4,
                                     "ms_per_step": sum(dev_times) / len(dev_times),
                                     "note": "bitstream uploaded, outputs kept on the device, status word read"}
    line["gpu_launches"] = launches
    line["clocks"] = clk.summary()
    if cpu and rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, buf, args.cpu_budget)
    return sc, line


def _contract(line: dict, args, world: int) -> dict:
    """The benchmark contract's keys around a measured line."""
    out = {"metric": METRIC, "value": line["value"], "unit": "Gaussians/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": line["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u32->f32", "data": "synthetic"}
    out.update({k: v for k, v in line.items() if k not in out})
    return out


def run_ours(args, w):
    """One workload: its measured line."""
    import torch
    import torch.distributed as dist
    from paper_2607_12656_b300 import sgs
    from paper_2607_12656_b300 import replicas
    rank, world, local = replicas.rank_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    ctx = sgs.Context(local, 0)
    _, line = measure(args, w, ctx, headline=w is WORKLOADS_DEFAULT)
    if rank == 0:
        print(json.dumps(_contract(line, args, world)), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


# The default run: the 1M-Gaussian scene of the fixed-length workload (seed 1000, depth 16)
# decoded in every coding mode -- the metric's comparison of learned and channel-wise coding on
# the same scene -- plus the small static scene of the plain method.  The fixed-length decode
# is the headline (value); the others are sub-objects with the same measurements.
DEFAULT_MODES = (("static", "static_4096"), ("static", "static"), ("learned", "learned"),
                 ("learned_pe", "learned_pe"), ("learned_geo", "learned_geo"), ("small", "small"))


def run_default(args):
    import torch
    import torch.distributed as dist
    from paper_2607_12656_b300 import sgs
    from paper_2607_12656_b300 import replicas
    rank, world, local = replicas.rank_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    ctx = sgs.Context(local, 0)
    w = WORKLOADS_DEFAULT
    sc, head = measure(args, w, ctx, headline=True)
    modes = {}
    for key, name in DEFAULT_MODES:
        wm = dict(WORKLOADS[key])
        if name == "static_4096":
            wm.update(lanes=4096, geo_w=None,
                      desc="channel-wise static rANS scene decode of the same scene: N=1,000,000 (900,000 kept), "
                           "depth 16, 8-bit tokens, 4,096 lanes (the learned workload's lanes and W = 220 rows "
                           "per lane), rANS-coded octree levels at the default 128 tokens per geometry lane")
        same = wm["n"] == w["n"] and wm["seed"] == w["seed"]
        _, line = measure(args, wm, ctx, sc if same else None)
        modes[name] = line
        torch.cuda.empty_cache()
    head["modes"] = modes
    head["modes_note"] = ("every mode but 'small' decodes the same 1M-Gaussian scene (seed 1000, depth 16, "
                          "900,000 rows kept): fixed-length (the headline), channel-wise static rANS at "
                          "4,096 lanes and at 151,552 lanes, the learned context model at 4,096 lanes "
                          "(trained 2,000 x 65,536 tokens on the device), the position-aware model at "
                          "28,125 lanes, and the learned geometry coder (static attributes); 'small' is "
                          "the 20,000-Gaussian plain-method scene (seed 0, "
                          "depth 12, 32 lanes)")
    if rank == 0:
        print(json.dumps(_contract(head, args, world)), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def scene_latency(samples: list, modes: list) -> dict:
    """p50/p99 of the per-scene completion times of the timed batch runs, overall and per
    coding mode (completion flags: the device's global timer from the run's first kernel to
    the end of the scene's last work item)."""
    names = {0: "fixed", 1: "static", 2: "learned"}
    out = {"note": "per-scene completion time inside a batch run (completion flags, device global timer)"}
    groups = {"all": [v for run in samples for v in run if v >= 0]}
    for m in sorted(set(modes)):
        groups[names.get(m, str(m))] = [run[j] for run in samples for j in range(len(run)) if modes[j] == m and run[j] >= 0]
    for k, v in groups.items():
        if v:
            out[k] = {"p50": float(np.percentile(v, 50)), "p99": float(np.percentile(v, 99)), "max": float(max(v)),
                      "samples": len(v)}
    return out


def run_batch(args):
    """The batched workload: every scene's bitstream resident in HBM, one plan run per step."""
    import torch
    import torch.distributed as dist
    from paper_2607_12656_b300 import sgs

    from paper_2607_12656_b300 import replicas
    rank, world, local = replicas.rank_info()
    # scenes are independent: rank r decodes its share of the batch, no exchange
    all_specs = batch_specs(args.scenes)
    specs, bufs = build_batch(args.scenes, args.train_steps or 300,
                              [all_specs[i] for i in replicas.shard(len(all_specs), rank, world)], tune=True)
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    ctx = sgs.Context(local, 0)
    infos = [sgs.scene_query(b) for b in bufs]
    rows = sum(int(i.n_rows) for i in infos)
    host_bits = [torch.frombuffer(bytearray(b), dtype=torch.uint8).pin_memory() for b in bufs]
    dev_bits = [h.to(dev) for h in host_bits]
    outs = [(torch.empty((56, i.n_rows), device=dev), torch.empty((3, i.n_rows), device=dev)) for i in infos]
    items = [(dev_bits[j], infos[j], outs[j][0], outs[j][1]) for j in range(len(infos))]
    plan = sgs.BatchPlan(ctx, items)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        plan.run(stream)
    if ctx.sync(stream) != sgs.OK or plan.status() != [sgs.OK] * len(items):
        raise RuntimeError("batch decode status %s" % plan.status())
    launches0 = ctx.launch_count()
    times, scene_ms = [], []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plan.run(stream)
            b.record(stream)
            stream.synchronize()
            times.append(a.elapsed_time(b))
            scene_ms.append(plan.times_ms())  # read after the step's stop event
        torch.cuda.synchronize()
    launches = ctx.launch_count() - launches0
    if ctx.sync(stream) != sgs.OK:
        raise RuntimeError("batch decode failed")
    total_ms = replicas.max_over_ranks(sum(times), dev)
    rows_all = int(replicas.sum_over_ranks(rows, dev))  # Gaussians decoded by all ranks per step
    ms = total_ms / args.steps
    # the same scenes decoded one after another (one scene_decode call each)
    ctx.reserve(max(int(i.scratch_bytes) for i in infos))
    seq = []
    for k in range(min(args.steps, 10)):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for j in range(len(items)):
            sgs.scene_decode(ctx, dev_bits[j], infos[j], outs[j][0], outs[j][1], None, None, stream)
        b.record(stream)
        stream.synchronize()
        seq.append(a.elapsed_time(b))
    # one plan run captured in a CUDA graph and replayed
    graph = []
    try:
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream()
        cap.wait_stream(stream)
        with torch.cuda.graph(g, stream=cap):
            plan.run(cap)
        torch.cuda.synchronize()
        for k in range(min(args.steps, 20)):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.replay()
            b.record(stream)
            stream.synchronize()
            graph.append(a.elapsed_time(b))
    except Exception as exc:
        print("graph capture failed: %s" % exc, file=sys.stderr)
    # end to end: bitstreams from pinned host memory, decode, outputs back to pinned host memory
    host_out = [(torch.empty(o[0].shape, pin_memory=True), torch.empty(o[1].shape, pin_memory=True)) for o in outs]
    e2e = []
    for k in range(min(args.steps, 5)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for h, d in zip(host_bits, dev_bits):
            d.copy_(h, non_blocking=True)
        plan.run(stream)
        for (ha, hp), (da, dp) in zip(host_out, outs):
            ha.copy_(da, non_blocking=True)
            hp.copy_(dp, non_blocking=True)
        b.record(stream)
        stream.synchronize()
        e2e.append(a.elapsed_time(b))
    if ctx.sync(stream) != sgs.OK:
        raise RuntimeError("batch decode failed")
    pk = peaks()
    hbm = pk.get("hbm_gbs")
    in_bytes = sum(len(b) for b in bufs)
    out_bytes = 4 * 59 * rows
    learned_rows = sum(int(i.n_rows) for i, s in zip(infos, specs) if s[4] == 2)
    line = {"metric": METRIC, "value": rows_all / (ms / 1e3), "unit": "Gaussians/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "u32->f32",
            "data": "synthetic",
            "config": {"workload": BATCH["desc"] + " [%d scenes, split by scene over %d GPU(s)]" % (args.scenes, world),
                       "n_rows": rows_all,
                       "scenes": len(items), "learned_scenes": sum(1 for s in specs if s[4] == 2),
                       "rows_per_lane": dict(TUNED), "tuning": "lane tuner (sgs_autotune, fastest decode over W "
                                                               "in 16..256) on each mode's median scene",
                       "bitstream_bytes": in_bytes, "output_bytes": out_bytes,
                       "l2": "flushed (256 MiB write) before every timed step; outputs exceed L2",
                       "parallelism": "scenes split across GPUs" if world > 1 else "single GPU"},
            "latency_ms": {"p50": float(np.percentile(times, 50)), "p99": float(np.percentile(times, 99)),
                           "min": min(times), "max": max(times), "note": "whole-batch makespan per step"},
            "scene_latency_ms": scene_latency(scene_ms, [s[4] for s in specs]),
            "sequential": {"ms_per_step": float(np.mean(seq)), "value": rows / (np.mean(seq) / 1e3),
                           "note": "same scenes, one scene_decode call after another"},
            "gpu_launches": launches // args.steps,
            "roofline": dict(attr_roofline(2, learned_rows, 0, ms, pk),
                             kernel="k_learned_multi: the batch's learned scenes over the whole-batch makespan "
                                    "(the learned decoder dominates it)"),
            "roofline_hbm": {"kernel": "whole batch", "bound": "hbm",
                         "achieved": (in_bytes + out_bytes) / (ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": (in_bytes + out_bytes) / (ms / 1e3) / 1e9 / hbm if hbm else None,
                         "traffic": None,
                         "note": "compressed bytes read + fp32 outputs written over the makespan"},
            "e2e": {"value": rows / (np.mean(e2e) / 1e3), "unit": "Gaussians/s", "h2d_bytes_per_step": in_bytes,
                    "d2h_bytes_per_step": out_bytes, "ms_per_step": float(np.mean(e2e))},
            "clocks": clk.summary()}
    if graph:
        line["graph"] = {"ms_per_step": float(np.mean(graph)), "value": rows / (np.mean(graph) / 1e3),
                         "note": "one plan run captured in a CUDA graph and replayed"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def run_render(args):
    """Decode to first frame: the default fixed-length 1M scene's bitstream resident in HBM,
    decoded, then splatted at 1920 x 1080 (sgs_render) from a camera 1.2 units in front of
    the scene's centre; per step the whole chain is timed with CUDA events (L2 flushed
    before), and decode and render separately."""
    import torch
    from paper_2607_12656_b300 import sgs
    from paper_2607_12656_b300.replicas import rank_info
    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    w = dict(WORKLOADS["fixed"])
    ctx = sgs.Context(local, 0)
    sc, buf = make_bitstream(w, ctx)
    info = sgs.scene_query(buf)
    ctx.reserve(info.scratch_bytes)
    dev = torch.device("cuda", local)
    bits = torch.frombuffer(bytearray(buf), dtype=torch.uint8).to(dev)
    n = int(info.n_rows)
    attr = torch.empty((56, n), device=dev)
    pos = torch.empty((3, n), device=dev)
    W, H = 1920, 1080
    cam = sgs.look_at([0.5, 0.5, -0.7], [0.5, 0.5, 0.5], [0, -1, 0], W, H, 50.0)
    img = torch.empty((3, H, W), device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        sgs.scene_decode(ctx, bits, info, attr, pos, stream=stream)
        sgs.render(ctx, attr, pos, n, cam, img, stream)
    if ctx.sync(stream) != sgs.OK:
        raise RuntimeError("decode failed")
    first, dec, ren = [], [], []
    launches0 = ctx.launch_count()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            sgs.scene_decode(ctx, bits, info, attr, pos, stream=stream)
            e[1].record(stream)
            sgs.render(ctx, attr, pos, n, cam, img, stream)
            e[2].record(stream)
            torch.cuda.synchronize()
            first.append(e[0].elapsed_time(e[2]))
            dec.append(e[0].elapsed_time(e[1]))
            ren.append(e[1].elapsed_time(e[2]))
    launches = (ctx.launch_count() - launches0) // args.steps
    if ctx.sync(stream) != sgs.OK:
        raise RuntimeError("decode failed")
    ms = float(np.median(first))
    line = {"metric": METRIC, "value": n / (ms / 1e3), "unit": "Gaussians/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32->f32", "data": "synthetic",
            "config": {"workload": w["desc"] + ", decoded then splatted at %d x %d (decode to first frame)" % (W, H),
                       "n_rows": n, "image": [W, H],
                       "l2": "flushed (256 MiB write) before every timed step"},
            "first_frame_ms": {"p50": ms, "min": float(min(first)), "max": float(max(first))},
            "decode_ms": float(np.median(dec)), "render_ms": float(np.median(ren)),
            "render_fps": 1e3 / float(np.median(ren)),
            "note": "value = Gaussians decoded and rendered per second of the decode-to-first-frame chain; the "
                    "render synchronises once to size its sort",
            "gpu_launches": launches, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def run_serve(args):
    """Serving: Poisson request streams at several rates against the decode server."""
    import torch
    from paper_2607_12656_b300 import serve, sgs

    local = int(os.environ.get("LOCAL_RANK", "0"))
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    c = SERVE
    specs = serve_specs(args.pool_per_mode or c["pool_per_mode"])
    specs, bufs = build_batch(len(specs), args.train_steps or 300, specs)
    torch.cuda.set_device(local)
    scenes = [serve.Scene(b) for b in bufs]
    modes = {name: [s[0] for s in specs if s[4] == m] for m, name in enumerate(("fixed", "static", "learned"))}
    srv = serve.DecodeServer(scenes, slots=c["slots"], hbm_budget=c["budget"], device=local)
    # warm-up: every scene once
    warm = srv.run([(0.0, j) for j in range(len(scenes))] * max(1, args.warmup // 3))
    if any(r.status != sgs.OK for r in warm):
        raise RuntimeError("serving warm-up failed")
    rates = [float(r) for r in (args.rates.split(",") if args.rates else c["rates"])]
    per_rate = []
    with ClockSampler(local) as clk:
        for k, lam in enumerate(rates):
            reqs = serve.poisson_arrivals_modes(lam, args.requests or c["requests"], modes,
                                                seed=c["arrival_seed"] + k)
            res = srv.run(reqs)
            summ = serve.summarize(res, scenes, modes)
            summ["rate_req_s"] = lam
            per_rate.append(summ)
    srv.close()
    best = max(per_rate, key=lambda d: d["gaussians_per_s"])
    line = {"metric": METRIC, "value": best["gaussians_per_s"] * world, "unit": "Gaussians/s", "n_gpus": world,
            "steps": len(rates), "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32->f32", "data": "synthetic",
            "config": {"workload": c["desc"], "requests_per_rate": args.requests or c["requests"],
                       "rates_req_s": rates, "pool_scenes": len(scenes),
                       "pool_gaussians": int(sum(s.n_rows for s in scenes)),
                       "l2": "not flushed: serving traffic (bitstream upload + outputs) far exceeds L2",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "latency_ms": {"p50": best["p50_ms"], "p99": best["p99_ms"],
                           "note": "arrival to completion, at the rate with the highest throughput"},
            "per_rate": per_rate,
            "e2e": {"value": best["gaussians_per_s"] * world, "unit": "Gaussians/s",
                    "h2d_bytes_per_step": None, "d2h_bytes_per_step": 0,
                    "note": "every request uploads its bitstream from pinned host memory inside its latency"},
            "gpu_launches": None, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_sweep(args):
    """Group-size sweep: for W (rows per lane, the paper's complexity knob) in 16..256, the
    bitstream size and the decode time of the 1M-Gaussian scene, static and both learned modes,
    measured by sgs_autotune (encode at each W, median of timed decodes)."""
    import torch
    from paper_2607_12656_b300 import learned, sgs
    from paper_2607_12656_b300.scenegen import make_scene
    from paper_2607_12656_b300.replicas import rank_info
    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    ctx = sgs.Context(local, 0)
    ws = [16, 32, 64, 128, 256]
    curves = {}
    encode_s = {}
    for mode, name, seed in ((1, "static", 1000), (2, "learned", 1000), (3, "learned_pe", 1000)):
        sc = make_scene(1_000_000, seed)
        model = None
        if mode == 2:
            model = learned.train_and_freeze(ctx, sc, 16, 4096, steps=args.train_steps or 2000, batch=65536, seed=1)
        if mode == 3:  # trained at W = 32, the paper's fast group size
            model = learned.train_and_freeze_pe(ctx, sc, 16, 28125, steps=args.train_steps or 2000, batch=65536,
                                                seed=1)
        r = sgs.autotune(ctx, sc.pos, sc.attr, mode=mode, depth=16, rows_per_lane=ws, reps=5 if mode == 1 else 3,
                         model=model)
        # whole scene_encode at W = 32, with a context (device preparation and coding) and without
        lanes = -(-900_000 // 32)
        for where, c in (("device", ctx), ("host", None)):
            if mode != 1 and c is None:
                continue  # learned coding needs the device for the model's frequencies
            t0 = time.perf_counter()
            sgs.scene_encode(sc.pos, sc.attr, mode=mode, depth=16, lanes=lanes, model=model, ctx=c)
            encode_s["%s_%s" % (name, where)] = time.perf_counter() - t0
        kept = 900_000
        curves[name] = [{"rows_per_lane": w, "lanes": l, "bytes": b, "bits_per_gaussian": 8.0 * b / kept,
                         "decode_ms": ms, "gaussians_per_s": kept / (ms / 1e3)}
                        for w, l, b, ms in zip(r["rows_per_lane"], r["lanes"], r["bytes"], r["ms"])]
    ctx.close()
    best = max((c for v in curves.values() for c in v), key=lambda c: c["gaussians_per_s"])
    line = {"metric": METRIC, "value": best["gaussians_per_s"], "unit": "Gaussians/s", "n_gpus": 1,
            "steps": 5, "warmup": 1, "ms_per_step": best["decode_ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32->f32", "data": "synthetic",
            "config": {"workload": "group-size sweep: 1M-Gaussian scene (900,000 kept), depth 16, W = rows per "
                                   "lane in 16..256, static, learned and position-aware learned attribute coding; decode median of timed runs "
                                   "(sgs_autotune), L2 not flushed", "rows_per_lane": ws},
            "curves": curves,
            "encode": {"seconds": encode_s, "gaussians": 1_000_000, "threads": os.cpu_count(),
                       "note": "whole scene_encode of the 1M scene at W = 32: with a context (device) the scene "
                               "is prepared (prune, Morton sort, octree, quantize) and its attributes coded on "
                               "the GPU, the geometry streams on the host; without one (host) everything runs "
                               "on the host cores"}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_seconds(buf: bytes, groups) -> tuple:
    """Seconds of one oracle decode of buf: the whole decode, or (learned modes, groups = k)
    the geometry and dequantisation plus the attribute lanes of the first k groups of 32,
    returned as (base seconds, seconds with k groups)."""
    from oracle import scene as S
    if groups is None:
        t0 = time.perf_counter()
        S.decode(buf)
        return time.perf_counter() - t0, None
    t0 = time.perf_counter()
    S.decode(buf, attr_groups=0)
    t1 = time.perf_counter()
    S.decode(buf, attr_groups=groups)
    return t1 - t0, time.perf_counter() - t1


def _oracle_worker(path: str, groups):
    with open(path, "rb") as f:
        buf = f.read()
    return _oracle_seconds(buf, groups)


def cpu_baseline(w: dict, buf: bytes, budget_s: float) -> dict:
    """The CPU oracle, as it stands, decoding the same bitstream (or a bounded part of it):
    one host thread, then the same sample on every available core at once (one oracle
    process per core, each decoding its own copy: the throughput of the host's cores on
    independent scenes)."""
    from oracle import scene as S
    h = S.parse_header(buf)
    rows = h["n_rows"]
    G = (h["lanes"] + 31) // 32 if h["mode"] in (S.MODE_LEARNED, S.MODE_LEARNED_PE) else 0
    if G <= 2:
        dt, _ = _oracle_seconds(buf, None)
        k, est = None, dt
        sample = "one full decode of the same bitstream (%d rows) by the numpy + C oracle, %.2f s" % (rows, dt)
    else:
        # learned models: the oracle's attribute decode costs about a minute per million tokens,
        # so it decodes the full geometry and the first k of the G equal groups of lanes, and the
        # attribute time is scaled by G / k
        t_base, t_one = _oracle_seconds(buf, 1)
        t_one = max(1e-3, t_one - t_base)
        k = int(min(G, max(1, (budget_s - t_base) / t_one)))
        t_base, t_k = _oracle_seconds(buf, k)
        t_k = max(1e-6, t_k - t_base)
        est = t_base + t_k * G / k
        sample = ("the numpy + C oracle on the same bitstream (%d rows): full geometry and dequantisation "
                  "(%.2f s) plus the attribute decode of %d of the %d groups of 32 lanes (%.2f s), scaled to "
                  "all groups: %.1f s per decode" % (rows, t_base, k, G, t_k, est))
    out = {"value": rows / est, "unit": "Gaussians/s", "cores": 1, "kind": "oracle", "sample": sample,
           "cpu_model": cpu_model(), "nproc": host_cores()}
    out["all_cores"] = cpu_baseline_all_cores(buf, k, G, rows)
    return out


def cpu_baseline_all_cores(buf: bytes, k, G: int, rows: int) -> dict:
    """Every usable core runs the single-thread sample at once, in its own spawned oracle
    process (numpy and BLAS limited to one thread each); value = decodes completed per second
    over the slowest process, times the rows of a decode."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import tempfile
    cores = host_cores()
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        avail = 0
    # each oracle decode of a 1M-Gaussian scene holds a few GB of numpy temporaries
    per = max(1 << 30, 60 * len(buf))
    n = max(1, min(cores, int(avail // per) if avail else cores))
    env = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    with tempfile.NamedTemporaryFile(suffix=".sgs", delete=False) as f:
        f.write(buf)
        path = f.name
    try:
        for v in env:
            os.environ[v] = "1"
        t0 = time.perf_counter()
        with cf.ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn")) as pool:
            res = [f.result() for f in [pool.submit(_oracle_worker, path, k) for _ in range(n)]]
        wall = time.perf_counter() - t0
    finally:
        for v, old in env.items():
            if old is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = old
        os.unlink(path)
    if k is None:
        est = max(r[0] for r in res)
    else:
        est = max(b + max(1e-6, t - b) * G / k for b, t in res)
    return {"value": n * rows / est, "unit": "Gaussians/s", "cores": n, "kind": "oracle",
            "sample": "%d oracle processes at once, each decoding the single-thread sample of its own copy "
                      "(slowest %.1f s per full decode, %.1f s wall with process start-up)" % (n, est, wall)}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import scene as S
    from paper_2607_12656_b300.scenegen import fixed_bits, make_scene
    # each step decodes a bounded sample of the workload: a scene of the same recipe (seed,
    # depth, coding, rows per lane) with fewer Gaussians, so that the whole run stays within
    # about two minutes of host time at the oracle's measured rate per coding mode (Gaussians/s
    # on one core: fixed-length 3.3e5, static 1.4e5, learned 1.8e3, position-aware 3.2e3)
    budget_s = 120.0
    rate = {0: 3.3e5, 1: 1.4e5, 2: 1.8e3, 3: 3.2e3}[w["mode"]]
    floor = 20_000 if w["mode"] < 2 else 256
    n = int(min(w["n"], max(floor, budget_s * rate / max(1, args.steps + args.warmup))))
    frac = n / w["n"]
    sc = make_scene(n, w["seed"])
    kw = dict(mode=w["mode"], depth=w["depth"], geo_mode=w["geo_mode"])
    if w["mode"] == 0:
        kw["bits"] = fixed_bits(w["seed"])
    else:
        kw["lanes"] = max(1, int(round(w["lanes"] * frac)))  # the same rows per lane
    P = S.prepare(sc.pos, sc.attr, w["depth"], kw.get("bits", 8))
    if w.get("geo_w"):  # the same geometry lanes as the GPU arm
        coded = S.geo_plan(P.levels, w["geo_mode"])
        n_coded = sum(len(P.levels[l]) for l in range(w["depth"]) if coded[l])
        kw["geo_lanes"] = max(32, -(-n_coded // (w["geo_w"] * 32)) * 32)
    note = ""
    if w["mode"] in (2, 3):
        # a model from a short oracle training run: the decode's work per token does not
        # depend on the weights
        from paper_2607_12656_b300.scenegen import kaiming_init, kaiming_init_pe
        q = P.q.astype(np.uint8)
        lr = S.lane_bounds(P.n_rows, kw["lanes"])
        if w["mode"] == 2:
            from oracle import model as M
            p, _ = M.train(kaiming_init(1), q, lr, 30, 4096, seed=1, lr=3e-3)
            kw["model"] = M.freeze({k: v.astype(np.float32) for k, v in p.items()}, q, lr, seed=1)
        else:
            from oracle import model_pe as E
            p, _ = E.train(kaiming_init_pe(1), q, lr, P.coord, w["depth"], 30, 4096, seed=1, lr=3e-3)
            kw["model"] = E.freeze({k: v.astype(np.float32) for k, v in p.items()}, q, lr, P.coord, w["depth"],
                                   seed=1)
        note = "; model from 30 oracle training steps of 4,096 tokens"
    buf = S.encode(sc.pos, sc.attr, prep=P, **kw)
    for _ in range(args.warmup):
        S.decode(buf)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        S.decode(buf)
        times.append(time.perf_counter() - t0)
    rows = S.parse_header(buf)["n_rows"]
    value = rows * len(times) / sum(times)
    sample = ("one oracle decode per step of a %d-Gaussian scene (%d rows) of the workload's recipe "
              "(%s), single thread%s" % (n, rows, "full size" if n == w["n"] else "bounded sample", note))
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": "Gaussians/s",
                      "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32->f32",
                      "data": "synthetic", "config": {"workload": w["desc"], "n_rows": rows},
                      "cpu_baseline": {"value": value, "unit": "Gaussians/s", "cores": 1, "kind": "oracle",
                                       "sample": sample},
                      "e2e": {"value": value, "unit": "Gaussians/s", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="default",
                    choices=["default"] + sorted(WORKLOADS) + ["batch", "serve", "sweep", "render"])
    ap.add_argument("--scenes", type=int, default=BATCH["n_scenes"], help="scenes of the batch workload")
    ap.add_argument("--rates", default=None, help="serve workload: comma-separated request rates (req/s)")
    ap.add_argument("--requests", type=int, default=None, help="serve workload: requests per rate")
    ap.add_argument("--pool-per-mode", type=int, default=None, help="serve workload: pool scenes per coding mode")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=30.0)
    ap.add_argument("--traffic", type=float, default=None,
                    help="dram bytes per launch of the dominant kernel from an ncu capture")
    ap.add_argument("--n", type=int, default=None, help="override the workload's Gaussian count")
    ap.add_argument("--lanes", type=int, default=None, help="override the workload's rANS lanes")
    ap.add_argument("--train-steps", type=int, default=None, help="override the learned model's steps")
    args = ap.parse_args()
    if args.workload in ("batch", "serve", "sweep", "render"):
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the %s workload is timed on the GPU only; "
                              "the oracle arm runs the single-scene workloads" % args.workload}))
            return
        {"batch": run_batch, "serve": run_serve, "sweep": run_sweep, "render": run_render}[args.workload](args)
        return
    global WORKLOADS_DEFAULT
    if args.workload == "default":
        WORKLOADS_DEFAULT = dict(WORKLOADS["fixed"])
        if args.impl == "reference":
            run_reference(args, WORKLOADS_DEFAULT)
        else:
            run_default(args)
        return
    w = dict(WORKLOADS[args.workload])
    if args.workload == "fixed" and args.n is None:
        WORKLOADS_DEFAULT = w
    if args.n is not None:
        w["n"] = args.n
        w["desc"] += " [resized: N=%d]" % args.n
    if args.lanes is not None:
        w["lanes"] = args.lanes
        w["desc"] += " [lanes=%d]" % args.lanes
    if args.train_steps is not None:
        w["train_steps"] = args.train_steps
        w["desc"] = w["desc"].replace("trained 2,000 steps", "trained %s steps" % f"{args.train_steps:,}")
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
