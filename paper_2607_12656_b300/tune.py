"""Autotuner: picks the rANS lane count (the paper's group size W = N'/L, Sec. 3.4.2, its
complexity knob) per coding mode and scene-size bucket by timing real decodes on this GPU.

More lanes mean more parallel decoders but more per-lane overhead (4-byte initial state,
final flush) and, for the learned model, shorter contexts; the tuner measures decode time
and coded size for each candidate and keeps the fastest candidate whose size is within
`max_size_growth` of the smallest.  Results are cached in a JSON file keyed by GPU name, SM
count, mode and log2 size bucket.
"""
from __future__ import annotations

import json
import math
import os

from . import sgs

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.json")
CANDIDATES = {sgs.MODE_STATIC: [4096, 16384, 32768, 65536, 131072, 262144],
              sgs.MODE_LEARNED: [1024, 2048, 4096, 8192, 16384]}


def _key(mode: int, n: int) -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return "%s|%d|mode%d|n2^%d" % (p.name, p.multi_processor_count, mode, int(math.log2(max(n, 2))))


def load_cache() -> dict:
    try:
        return json.load(open(CACHE))
    except Exception:
        return {}


def lookup(mode: int, n: int) -> int | None:
    return load_cache().get(_key(mode, n), {}).get("lanes")


def time_decode(ctx: sgs.Context, buf: bytes, reps: int = 5) -> float:
    import torch
    info = sgs.scene_query(buf)
    ctx.reserve(info.scratch_bytes)
    bits = torch.frombuffer(bytearray(buf), dtype=torch.uint8).cuda()
    attr = torch.empty((56, max(info.n_rows, 1)), device="cuda")
    pos = torch.empty((3, max(info.n_rows, 1)), device="cuda")
    sgs.scene_decode(ctx, bits, info, attr, pos)
    if ctx.sync() != sgs.OK:
        raise RuntimeError("decode failed while tuning")
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        sgs.scene_decode(ctx, bits, info, attr, pos)
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    return sorted(times)[len(times) // 2]


def tune(ctx: sgs.Context, scene, depth: int, mode: int, model: bytes | None = None,
         candidates: list[int] | None = None, max_size_growth: float = 0.01, save: bool = True) -> dict:
    cands = candidates or CANDIDATES[mode]
    rows = []
    for L in cands:
        kw = dict(mode=mode, depth=depth, lanes=L, geo_mode=sgs.GEO_RANS)
        if mode == sgs.MODE_LEARNED:
            kw.update(model=model, ctx=ctx)
        buf = sgs.scene_encode(scene.pos, scene.attr, **kw)
        rows.append({"lanes": L, "bytes": len(buf), "ms": time_decode(ctx, buf)})
    smallest = min(r["bytes"] for r in rows)
    ok = [r for r in rows if r["bytes"] <= smallest * (1 + max_size_growth)] or rows
    best = min(ok, key=lambda r: r["ms"])
    out = {"lanes": best["lanes"], "ms": best["ms"], "bytes": best["bytes"], "candidates": rows}
    if save:
        cache = load_cache()
        cache[_key(mode, scene.n)] = out
        json.dump(cache, open(CACHE, "w"), indent=1)
    return out
