"""The multi-scene workloads at their full recipes, bit for bit against the oracle.

Batched: 64 scenes, N log-uniform in [50k, 3M], depths 14..17, half learned (each with its
own model, trained on the device on its own tokens), half channel-wise static, decoded in
one plan run (one persistent launch per stage) and again from a CUDA graph replay; every
scene's attributes and positions equal the oracle's (0 ULP, compared through SHA-256 of the
fp32 bytes).  Serving: a continuous-batching mix with one scene of every coding mode at
several million Gaussians among smaller ones; every request's output equals the oracle's."""
import numpy as np
import pytest

from paper_2607_12656_b300 import sgs, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from scene_workers import build_with_oracle, digests  # noqa: E402


def _device_items(bufs):
    items = []
    for b in bufs:
        info = sgs.scene_query(b)
        bits = torch.frombuffer(bytearray(b), dtype=torch.uint8).cuda()
        attr = torch.full((56, info.n_rows), float("nan"), device="cuda")
        pos = torch.full((3, info.n_rows), float("nan"), device="cuda")
        items.append((bits, info, attr, pos))
    return items


def _check(items, want, specs):
    bad = []
    for (bits, info, attr, pos), d, sp in zip(items, want, specs):
        if digests(attr.cpu().numpy(), pos.cpu().numpy()) != d:
            bad.append(sp)
    assert not bad, "scenes differing from the oracle: %s" % bad


def _reset(items):
    for it in items:
        it[2].fill_(float("nan"))
        it[3].fill_(float("nan"))


@pytest.mark.timeout(3600)
def test_batch_full_recipe_matches_oracle():
    specs = workloads.batch_specs(64, w_learned=220, w_static=32)
    built = workloads.build(specs, 200, fn=build_with_oracle)
    bufs, want = [b for b, _ in built], [d for _, d in built]
    assert sum(s[4] == 2 for s in specs) == 32
    rows = sum(int(sgs.scene_query(b).n_rows) for b in bufs)
    assert rows > 30_000_000  # about 41 M Gaussians kept of the 64 scenes
    items = _device_items(bufs)
    c = sgs.Context(0, 0)
    plan = sgs.BatchPlan(c, items)
    plan.run()
    assert c.sync() == sgs.OK and plan.status() == [sgs.OK] * len(items)
    _check(items, want, specs)
    _reset(items)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(s)
    g.replay()
    torch.cuda.synchronize()
    assert c.sync() == sgs.OK and plan.status() == [sgs.OK] * len(items)
    _check(items, want, specs)
    del g
    plan.close()
    c.close()


@pytest.mark.timeout(3600)
def test_serving_mix_with_multi_million_scenes_matches_oracle():
    from paper_2607_12656_b300 import serve
    big = [(0, 3_000_000, 4100, 16, 0, 0), (1, 4_000_000, 4101, 16, 1, workloads.lanes_for(4_000_000, 32)),
           (2, 2_500_000, 4102, 16, 2, workloads.lanes_for(2_500_000, 220))]
    small = [(3, 150_000, 4103, 16, 0, 0), (4, 300_000, 4104, 16, 1, workloads.lanes_for(300_000, 32)),
             (5, 200_000, 4105, 16, 2, workloads.lanes_for(200_000, 220))]
    specs = big + small
    built = workloads.build(specs, 200, fn=build_with_oracle)
    scenes = [serve.Scene(b) for b, _ in built]
    assert all(scenes[j].n_rows >= 2_000_000 for j in range(3))
    srv = serve.DecodeServer(scenes, slots=4, hbm_budget=120 << 30, keep_outputs="digest")
    reqs = serve.poisson_arrivals(400.0, 30, len(scenes), seed=11)
    res = srv.run(reqs)
    srv.close()
    assert len(res) == 30 and all(r.status == sgs.OK for r in res)
    overlapped = sum(1 for r in res if any(o is not r and o.admitted < r.done and r.admitted < o.done for o in res))
    assert overlapped > 5
    assert {r.scene for r in res} >= {0, 1, 2}  # every big scene was served
    for r in res:
        assert r.digest == built[r.scene][1], (r.req, specs[r.scene])
