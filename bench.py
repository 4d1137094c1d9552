"""Benchmark: decoded Gaussians/s (and p50/p99 scene-decode latency) of the B300 decode path.

A step is one whole scene decode (octree geometry -> positions, attribute tokens -> fp32
structure of arrays) of a synthetic paper-shaped scene already resident in HBM.  Default
workload: 1,000,000 Gaussians (900,000 after pruning), depth-16 octree, channel-wise
fixed-length attributes with per-channel widths drawn from 4..10 bits.  Other workloads:
--workload static (same scene, channel-wise static rANS, 151,552 lanes), learned (same scene,
learned context model, 4,096 lanes), small (20,000 Gaussians, depth 12, static rANS, 32 lanes).

Prints one JSON line.  --impl reference times the CPU oracle on the same workload instead.
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
    "static": dict(n=1_000_000, seed=1000, depth=16, mode=1, geo_mode=1, lanes=151552,
                   desc="channel-wise static rANS scene decode: N=1,000,000 (900,000 kept), depth 16, "
                        "8-bit tokens, 151,552 lanes (one 32-warp CTA per SM), rANS-coded octree levels"),
    "learned": dict(n=1_000_000, seed=2000, depth=16, mode=2, geo_mode=1, lanes=4096,
                    desc="learned-model scene decode: N=1,000,000 (900,000 kept), depth 16, 8-bit "
                         "tokens, 4,096 lanes, context MLP 4->64->64->256"),
    "small": dict(n=20_000, seed=0, depth=12, mode=1, geo_mode=1, lanes=32,
                  desc="small static scene decode: N=20,000 (18,000 kept), depth 12, 32 lanes"),
}
METRIC = "decoded Gaussians/s"


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


def make_bitstream(w: dict, ctx=None):
    from paper_2607_12656_b300 import sgs
    from paper_2607_12656_b300.scenegen import fixed_bits, make_scene
    sc = make_scene(w["n"], w["seed"])
    kw = dict(mode=w["mode"], depth=w["depth"], geo_mode=w["geo_mode"])
    if w["mode"] == 0:
        kw["bits"] = fixed_bits(w["seed"])
    else:
        kw["lanes"] = w["lanes"]
    model = None
    if w["mode"] == 2:
        from paper_2607_12656_b300 import learned
        model = learned.train_and_freeze(ctx, sc, w["depth"], w["lanes"], steps=w.get("train_steps", 2000),
                                         batch=65536, seed=1)
        kw["model"] = model
        kw["ctx"] = ctx
    return sc, sgs.scene_encode(sc.pos, sc.attr, **kw)


def fixed_algorithmic_bytes(info, bits_np) -> int:
    n = info.n_rows
    read = sum(4 * ((n * int(b) + 31) // 32) for b in bits_np)
    return read + 4 * 56 * n


def run_ours(args, w):
    import torch
    import torch.distributed as dist
    from paper_2607_12656_b300 import sgs

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    ctx = sgs.Context(local, 0)
    sc, buf = make_bitstream(w, ctx)
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
    ctx.profile(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stage = []
    launches0 = ctx.launch_count()
    if world > 1:
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
            stage.append(ctx.profile_read())
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    launches = ctx.launch_count() - launches0
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
    except Exception as exc:  # graph capture unavailable: report eager numbers only
        print("graph capture failed: %s" % exc, file=sys.stderr)
        graph_times = []
    total_ms = sum(times)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = n * world * args.steps / (total_ms / 1e3)

    # end to end through the public API: pinned host bitstream -> device, decode, outputs -> host
    host_attr = torch.empty((56, n), dtype=torch.float32).pin_memory()
    host_pos = torch.empty((3, n), dtype=torch.float32).pin_memory()
    e2e_times = []
    for k in range(min(args.steps, 50)):
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
    e2e_ms = sum(e2e_times) / len(e2e_times)

    pk = peaks()
    hbm = pk.get("hbm_gbs")
    line = {"metric": METRIC, "value": value, "unit": "Gaussians/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32->f32", "data": "synthetic",
            "config": {"workload": w["desc"], "n_rows": n, "bitstream_bytes": len(buf),
                       "l2": "flushed (256 MiB write) before every timed step",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "latency_ms": {"p50": float(np.percentile(times, 50)), "p99": float(np.percentile(times, 99)),
                           "min": min(times), "max": max(times)},
            "stage_ms": {"geometry_tokens": float(np.mean([s[0] for s in stage])),
                         "octree_positions": float(np.mean([s[1] for s in stage])),
                         "attributes": float(np.mean([s[2] for s in stage])),
                         "whole_decode": float(np.mean([s[3] for s in stage])),
                         "note": "attributes run on their own stream, concurrent with geometry"},
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
                            "algorithmic_bytes": alg, "traffic": args.traffic}
        geo_alg = info.n_geo + 12 * n
        line["roofline_octree"] = {"bound": "hbm", "algorithmic_bytes": geo_alg,
                                   "achieved": geo_alg / (line["stage_ms"]["octree_positions"] / 1e3) / 1e9,
                                   "unit": "GB/s"}
    line["e2e"] = {"value": n * len(e2e_times) / (sum(e2e_times) / 1e3), "unit": "Gaussians/s",
                   "h2d_bytes_per_step": len(buf), "d2h_bytes_per_step": 4 * 59 * n, "ms_per_step": e2e_ms}
    line["gpu_launches"] = launches
    line["clocks"] = clk.summary()
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, buf, args.cpu_budget)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def cpu_baseline(w: dict, buf: bytes, budget_s: float) -> dict:
    """The CPU oracle, as it stands, decoding the same bitstream (or a bounded part of it)."""
    from oracle import scene as S
    h = S.parse_header(buf)
    t0 = time.perf_counter()
    d = S.decode(buf)
    dt = time.perf_counter() - t0
    return {"value": h["n_rows"] / dt, "unit": "Gaussians/s", "cores": 1, "kind": "oracle",
            "sample": "one full decode of the same bitstream (%d rows) by the numpy + C oracle, "
                      "single thread, %.2f s" % (h["n_rows"], dt)}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2607_12656_b300 import sgs
    from oracle import scene as S
    from paper_2607_12656_b300.scenegen import fixed_bits, make_scene
    sc = make_scene(w["n"], w["seed"])
    kw = dict(mode=w["mode"], depth=w["depth"], geo_mode=w["geo_mode"])
    if w["mode"] == 0:
        kw["bits"] = fixed_bits(w["seed"])
    else:
        kw["lanes"] = w["lanes"]
    buf = S.encode(sc.pos, sc.attr, **kw)
    for _ in range(args.warmup):
        S.decode(buf)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        S.decode(buf)
        times.append(time.perf_counter() - t0)
    n = S.parse_header(buf)["n_rows"]
    value = n * len(times) / sum(times)
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": "Gaussians/s",
                      "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32->f32",
                      "data": "synthetic", "config": {"workload": w["desc"], "n_rows": n},
                      "cpu_baseline": {"value": value, "unit": "Gaussians/s", "cores": 1, "kind": "oracle",
                                       "sample": "full decode of the workload's bitstream per step"},
                      "e2e": {"value": value, "unit": "Gaussians/s", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fixed", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=30.0)
    ap.add_argument("--traffic", type=float, default=None,
                    help="dram bytes per launch of the dominant kernel from an ncu capture")
    ap.add_argument("--n", type=int, default=None, help="override the workload's Gaussian count")
    ap.add_argument("--lanes", type=int, default=None, help="override the workload's rANS lanes")
    ap.add_argument("--train-steps", type=int, default=None, help="override the learned model's steps")
    args = ap.parse_args()
    w = dict(WORKLOADS[args.workload])
    if args.n is not None:
        w["n"] = args.n
        w["desc"] += " [resized: N=%d]" % args.n
    if args.lanes is not None:
        w["lanes"] = args.lanes
        w["desc"] += " [lanes=%d]" % args.lanes
    if args.train_steps is not None:
        w["train_steps"] = args.train_steps
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
