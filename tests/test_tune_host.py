"""Host logic of the lane tuner: one autotune per (GPU, mode, size bucket, latency cap), the
choice cached in memory and on disk, the lane count derived from the kept rows.  The GPU
measurement (sgs.autotune) is replaced by a stub that records its calls."""
import types

import numpy as np

from paper_2607_12656_b300 import sgs, tune


def _stub(monkeypatch, best_w):
    calls = []

    def autotune(ctx, pos, attr, *, mode, depth, rows_per_lane, max_ms, reps, model, warps_per_cta=(), geo_mode=1):
        calls.append((mode, pos.shape[1], max_ms, tuple(warps_per_cta)))
        ws = list(rows_per_lane)
        best = ws.index(best_w) if best_w in ws else 0
        return {"best": best, "rows_per_lane": ws, "ms": [1.0 + w for w in ws],
                "bytes": [1000 - w for w in ws], "warps": [16] * len(ws), "best_warps": 16 if warps_per_cta else 0}

    monkeypatch.setattr(sgs, "autotune", autotune)
    monkeypatch.setattr(tune, "_device_key", lambda device: "FakeGPU/148sm")
    return calls


def test_one_autotune_per_key_and_lanes_from_kept_rows(monkeypatch, tmp_path):
    calls = _stub(monkeypatch, 32)
    ctx = types.SimpleNamespace(device=0)
    path = str(tmp_path / "lanes.json")
    t = tune.LaneTuner(path)
    pos = np.zeros((3, 10_000), np.float32)
    L = t.choose_lanes(ctx, pos, None, mode=2, depth=12)
    assert L == -(-(10_000 - 1_000) // 32) and len(calls) == 1
    # same mode and size bucket (2^13..2^14 rounds to 13 for 10,000 and 9,000): cached
    assert t.choose_lanes(ctx, np.zeros((3, 9_000)), None, mode=2, depth=12) == -(-8_100 // 32)
    assert len(calls) == 1
    # another mode, another bucket or another latency cap: tuned again
    t.choose_lanes(ctx, pos, None, mode=1, depth=12)
    t.choose_lanes(ctx, np.zeros((3, 40_000)), None, mode=2, depth=12)
    t.choose_lanes(ctx, pos, None, mode=2, depth=12, max_ms=5.0)
    assert len(calls) == 4
    # a new tuner reads the file and tunes nothing
    t2 = tune.LaneTuner(path)
    assert t2.choose_lanes(ctx, pos, None, mode=2, depth=12) == L and len(calls) == 4
    key = t2.key(ctx, 2, 10_000, 0.0)
    assert key.startswith("FakeGPU/148sm|mode2|") and t2.table[key]["sweep"]["32"] == [33.0, 968]


def test_tiny_scene_gets_one_lane(monkeypatch):
    _stub(monkeypatch, 256)
    t = tune.LaneTuner()
    assert t.choose_lanes(types.SimpleNamespace(device=0), np.zeros((3, 5)), None, mode=1, depth=4) == 1


class _ShapeCtx(types.SimpleNamespace):
    def set_launch_shape(self, mode, warps):
        self.shapes[mode] = warps


def test_launch_shape_is_tuned_cached_and_set_on_the_context(monkeypatch, tmp_path):
    """Static and fixed-length scenes tune their attribute decoder's warps per CTA with W (the
    fixed-length mode has no lanes), and the choice reaches the context on a cache hit too."""
    calls = _stub(monkeypatch, 32)
    path = str(tmp_path / "lanes.json")
    ctx = _ShapeCtx(device=0, shapes={})
    pos = np.zeros((3, 10_000), np.float32)
    lanes, warps = tune.LaneTuner(path).choose(ctx, pos, None, mode=sgs.MODE_STATIC, depth=12)
    assert lanes == -(-9_000 // 32) and warps == 16 and ctx.shapes == {sgs.MODE_STATIC: 16}
    assert calls[-1][3] == tune.DEFAULT_SHAPES[sgs.MODE_STATIC]
    lanes, warps = tune.LaneTuner(path).choose(ctx, pos, None, mode=sgs.MODE_FIXED, depth=12)
    assert lanes == 0 and warps == 16 and calls[-1][3] == tune.DEFAULT_SHAPES[sgs.MODE_FIXED]
    n_calls = len(calls)
    ctx2 = _ShapeCtx(device=0, shapes={})
    assert tune.LaneTuner(path).choose(ctx2, pos, None, mode=sgs.MODE_STATIC, depth=12) == (-(-9_000 // 32), 16)
    assert len(calls) == n_calls and ctx2.shapes == {sgs.MODE_STATIC: 16}
    # learned modes have no tunable shape
    assert tune.LaneTuner().choose(ctx2, pos, None, mode=sgs.MODE_LEARNED, depth=12)[1] == 0
    assert calls[-1][3] == ()
