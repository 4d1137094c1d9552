"""Lane-count and launch-shape choice per (GPU, mode, scene size), cached as JSON.

The decode's parallelism is set at encode time by the group size W (rows per lane), the
paper's complexity knob (Sec. 4, implementation details), and at decode time by the
attribute decoder's launch shape (warps per CTA; fixed-length and static modes).
``choose`` returns the lane count and the shape for a scene and sets the shape on the
context: from the cache when the same GPU model and SM count have already tuned this mode at
this size bucket (power of two of N), else by running ``sgs_autotune`` on the scene (every W
at every shape) and recording the choice.
"""
from __future__ import annotations

import json
import math
import os

from . import sgs

DEFAULT_W = (16, 32, 64, 128, 256)
# candidate warps per CTA of the attribute decoder, per coding mode that has a tunable shape
DEFAULT_SHAPES = {sgs.MODE_FIXED: (2, 4, 8), sgs.MODE_STATIC: (8, 16, 32)}


def _device_key(device: int) -> str:
    import torch
    p = torch.cuda.get_device_properties(device)
    return "%s/%dsm" % (p.name, p.multi_processor_count)


def bucket(n: int) -> int:
    return int(round(math.log2(max(n, 1))))


class LaneTuner:
    def __init__(self, path: str | None = None):
        self.path = path
        self.table = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.table = json.load(f)

    def key(self, ctx: sgs.Context, mode: int, n: int, max_ms: float) -> str:
        return "%s|mode%d|n2^%d|max%.3g" % (_device_key(ctx.device), mode, bucket(n), max_ms)

    def choose(self, ctx: sgs.Context, pos, attr, *, mode: int, depth: int, max_ms: float = 0.0,
               candidates=DEFAULT_W, model: bytes | None = None, reps: int = 5, shapes=None,
               geo_mode: int = sgs.GEO_RANS) -> tuple[int, int]:
        """(lanes, warps per CTA) for the scene; the shape is set on the context.  Fixed-length
        scenes have no lanes (0): only their shape is tuned."""
        n = pos.shape[1]
        kept = n - n // 10
        k = self.key(ctx, mode, n, max_ms)
        if k not in self.table:
            shapes = DEFAULT_SHAPES.get(mode, ()) if shapes is None else tuple(shapes)
            ws = (1,) if mode == sgs.MODE_FIXED else tuple(candidates)
            r = sgs.autotune(ctx, pos, attr, mode=mode, depth=depth, rows_per_lane=ws, max_ms=max_ms,
                             reps=reps, model=model, warps_per_cta=shapes, geo_mode=geo_mode)
            b = r["best"]
            self.table[k] = {"rows_per_lane": r["rows_per_lane"][b], "ms": r["ms"][b], "bytes": r["bytes"][b],
                             "warps": r.get("best_warps", 0),
                             "sweep": {str(w): [ms, by] for w, ms, by in zip(r["rows_per_lane"], r["ms"], r["bytes"])}}
            if self.path:  # written whole, then renamed: a reader never sees half a file
                tmp = self.path + ".tmp"
                with open(tmp, "w") as f:
                    json.dump(self.table, f, indent=1, sort_keys=True)
                os.replace(tmp, self.path)
        e = self.table[k]
        warps = int(e.get("warps", 0))
        if mode in DEFAULT_SHAPES and hasattr(ctx, "set_launch_shape"):
            ctx.set_launch_shape(mode, warps)
        lanes = 0 if mode == sgs.MODE_FIXED else max(1, -(-kept // e["rows_per_lane"]))
        return lanes, warps

    def choose_lanes(self, ctx: sgs.Context, pos, attr, *, mode: int, depth: int, max_ms: float = 0.0,
                     candidates=DEFAULT_W, model: bytes | None = None, reps: int = 5) -> int:
        return self.choose(ctx, pos, attr, mode=mode, depth=depth, max_ms=max_ms, candidates=candidates,
                           model=model, reps=reps)[0]
