"""Host logic of the lane tuner: one autotune per (GPU, mode, size bucket, latency cap), the
choice cached in memory and on disk, the lane count derived from the kept rows.  The GPU
measurement (sgs.autotune) is replaced by a stub that records its calls."""
import types

import numpy as np

from paper_2607_12656_b300 import sgs, tune


def _stub(monkeypatch, best_w):
    calls = []

    def autotune(ctx, pos, attr, *, mode, depth, rows_per_lane, max_ms, reps, model):
        calls.append((mode, pos.shape[1], max_ms))
        ws = list(rows_per_lane)
        return {"best": ws.index(best_w), "rows_per_lane": ws, "ms": [1.0 + w for w in ws],
                "bytes": [1000 - w for w in ws]}

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
