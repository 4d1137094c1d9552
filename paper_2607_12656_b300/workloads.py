"""The multi-scene workloads: the batched decode (64 scenes) and the serving pool.

Recipes (sizes, depths, seeds, coding modes, rows per lane) and a builder that generates,
trains and encodes their scenes in a pool of spawned worker processes.  Every learned scene
gets its own context model, trained on the device on that scene's own tokens (Sec. 3.4.2:
the model is fitted to the scene it codes) and frozen to the integer model, then the scene is
encoded with it.  Only orchestration lives here: generation is scenegen's, training,
freezing and encoding are the library's.
"""
from __future__ import annotations

import os

import numpy as np

# Batched decode: 64 scenes, N log-uniform in [50k, 3M] (seed 3000), depth uniform in
# {14..17} (seed 3001), even scenes learned-model rANS, odd scenes channel-wise static rANS.
BATCH = dict(n_scenes=64, lo=50_000, hi=3_000_000, size_seed=3000, depth_lo=14, depth_hi=17,
             desc="batched decode of 64 scenes: N log-uniform 50k..3M (seeded), depth U{14..17}, "
                  "even scenes learned-model rANS (each with its own model trained on its own tokens), "
                  "odd scenes channel-wise static rANS, rows per lane per mode chosen by the lane tuner, "
                  "rANS-coded octree levels; one persistent launch per stage over all scenes")

# Serving: a pool of 3 modes x per_mode scenes, N log-uniform in [100k, 6M] (seed 4000),
# depth 16; requests draw a mode, then a scene of that mode, uniformly.
SERVE = dict(pool_per_mode=40, lo=100_000, hi=6_000_000, size_seed=4000, depth=16, rates=(20, 50, 100, 200, 400),
             requests=2000, arrival_seed=4999, budget=120 << 30, slots=8,
             desc="continuous-batching decode server: a pool of 3 modes x 40 scenes (N log-uniform "
                  "100k..6M, depth 16; learned scenes each with their own model), requests draw a mode then "
                  "a scene uniformly, Poisson arrivals, admission by HBM footprint within 120 GB, 8 concurrent "
                  "decode slots")

# A spec is (index, N, seed, depth, mode, lanes).


def lanes_for(n: int, rows_per_lane: int) -> int:
    kept = n - n // 10
    return max(32, -(-kept // rows_per_lane))


def batch_specs(n_scenes: int = 64, w_learned: int = 220, w_static: int = 32) -> list:
    from .scenegen import loguniform_sizes
    b = BATCH
    sizes = loguniform_sizes(b["size_seed"], n_scenes, b["lo"], b["hi"])
    rng = np.random.Generator(np.random.PCG64(b["size_seed"] + 1))
    depths = rng.integers(b["depth_lo"], b["depth_hi"] + 1, size=n_scenes)
    out = []
    for j in range(n_scenes):
        n = int(sizes[j])
        learned = j % 2 == 0
        out.append((j, n, 3000 + j, int(depths[j]), 2 if learned else 1,
                    lanes_for(n, w_learned if learned else w_static)))
    return out


def serve_specs(per_mode: int = 40) -> list:
    """Pool scenes, fixed-length first, then static, then learned."""
    from .scenegen import loguniform_sizes
    c = SERVE
    sizes = loguniform_sizes(c["size_seed"], 3 * per_mode, c["lo"], c["hi"])
    out = []
    for j in range(3 * per_mode):
        mode = j // per_mode
        n = int(sizes[j])
        lanes = 0 if mode == 0 else lanes_for(n, 220 if mode == 2 else 32)
        out.append((j, n, 4000 + j, c["depth"], mode, lanes))
    return out


_ctx = None


def encode_spec(spec, train_steps: int = 300, scene=None) -> bytes:
    """Generates (or takes) one scene and encodes it; a learned scene first gets its own
    model, trained train_steps x 65,536 of its tokens on the device (this process's context)
    and frozen."""
    global _ctx
    from . import sgs
    from .scenegen import fixed_bits, make_scene
    j, n, seed, depth, mode, lanes = spec
    sc = make_scene(n, seed) if scene is None else scene
    if mode == 0:
        return sgs.scene_encode(sc.pos, sc.attr, mode=0, depth=depth, bits=fixed_bits(seed), geo_mode=0)
    kw = dict(mode=mode, depth=depth, lanes=lanes, geo_mode=1)
    if mode in (2, 3):
        from . import learned
        if _ctx is None:
            _ctx = sgs.Context(0, 0)
        train = learned.train_and_freeze if mode == 2 else learned.train_and_freeze_pe
        kw.update(model=train(_ctx, sc, depth, lanes, steps=train_steps, batch=65536, seed=seed), ctx=_ctx)
    return sgs.scene_encode(sc.pos, sc.attr, **kw)


def pool_workers(max_workers: int = 32, per_worker_bytes: int = 6 << 30) -> int:
    """Worker processes for building scenes: the host's cores, bounded by its free memory."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        avail = 0
    n = min(max_workers, cores)
    if avail:
        n = min(n, max(1, int(avail // per_worker_bytes)))
    return max(1, n)


def build(specs: list, train_steps: int = 300, fn=None, workers: int | None = None) -> list:
    """fn(spec, train_steps) (default encode_spec) for every spec in a pool of spawned
    processes (each with its own CUDA context when it trains); results in spec order."""
    import concurrent.futures as cf
    import multiprocessing as mp
    fn = fn or encode_spec
    workers = workers or pool_workers()
    env = os.environ.get("OMP_NUM_THREADS")
    os.environ["OMP_NUM_THREADS"] = str(max(1, (os.cpu_count() or 1) // workers))
    try:
        out = [None] * len(specs)
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as pool:
            futs = {pool.submit(fn, s, train_steps): k for k, s in enumerate(specs)}
            for f in cf.as_completed(futs):
                out[futs[f]] = f.result()
        return out
    finally:
        if env is None:
            os.environ.pop("OMP_NUM_THREADS", None)
        else:
            os.environ["OMP_NUM_THREADS"] = env
