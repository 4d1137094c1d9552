"""Batched multi-scene decode and the continuous-batching server: every scene's decoded output
is identical alone, in a batch, and in the serving mix (and equal to the oracle's values)."""
import numpy as np
import pytest

from oracle import scene as S
from paper_2607_12656_b300 import sgs
from paper_2607_12656_b300.scenegen import fixed_bits, loguniform_sizes, make_scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_gpu_decode import gpu_decode, same_bits  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = sgs.Context(0, 1 << 20)
    yield c
    c.close()


@pytest.fixture(scope="module")
def pool(ctx):
    """Mixed-mode scenes of uneven sizes (the batched and serving workloads, scaled down)."""
    from paper_2607_12656_b300 import learned
    sizes = loguniform_sizes(3000, 9, 5_000, 120_000)
    out = []
    for j, n in enumerate(sizes):
        sc = make_scene(int(n), 3000 + j)
        depth = 12 + j % 4
        mode = j % 3
        if mode == sgs.MODE_FIXED:
            buf = sgs.scene_encode(sc.pos, sc.attr, mode=mode, depth=depth, bits=fixed_bits(j), geo_mode=sgs.GEO_RAW)
            P = S.prepare(sc.pos, sc.attr, depth, fixed_bits(j))
        elif mode == sgs.MODE_STATIC:
            buf = sgs.scene_encode(sc.pos, sc.attr, mode=mode, depth=depth, lanes=256 + 32 * j)
            P = S.prepare(sc.pos, sc.attr, depth, 8)
        else:
            lanes = 128 + 64 * j
            model = learned.train_and_freeze(ctx, sc, depth, lanes, steps=60, batch=8192, seed=j)
            buf = sgs.scene_encode(sc.pos, sc.attr, mode=mode, depth=depth, lanes=lanes, model=model, ctx=ctx)
            P = S.prepare(sc.pos, sc.attr, depth, 8)
        out.append((buf, P))
    return out


def test_pool_alone_matches_oracle(ctx, pool):
    for buf, P in pool:
        st, attr, pos, _, _ = gpu_decode(ctx, buf)
        assert st == sgs.OK and same_bits(attr, P.attr) and same_bits(pos, P.pos)


def test_batch_decode_matches_alone(pool):
    infos = [sgs.scene_query(b) for b, _ in pool]
    need = sum((i.scratch_bytes + 255) // 256 * 256 for i in infos)
    c = sgs.Context(0, need)
    items, outs = [], []
    for (buf, P), info in zip(pool, infos):
        bits = torch.frombuffer(bytearray(buf), dtype=torch.uint8).cuda()
        attr = torch.full((56, info.n_rows), float("nan"), device="cuda")
        pos = torch.full((3, info.n_rows), float("nan"), device="cuda")
        items.append((bits, info, attr, pos))
        outs.append((attr, pos, P))
    sgs.scene_decode_batch(c, items)
    assert c.sync() == sgs.OK
    for attr, pos, P in outs:
        assert same_bits(attr.cpu().numpy(), P.attr) and same_bits(pos.cpu().numpy(), P.pos)
    c.close()


def test_server_mix_equals_alone(pool):
    from paper_2607_12656_b300 import serve
    scenes = [serve.Scene(b) for b, _ in pool]
    srv = serve.DecodeServer(scenes, slots=4, hbm_budget=2 << 30, keep_outputs=True)
    reqs = serve.poisson_arrivals(3000.0, 40, len(scenes), seed=7)
    res = srv.run(reqs)
    srv.close()
    assert len(res) == 40 and all(r.status == sgs.OK for r in res)
    overlapped = sum(1 for r in res if any(o is not r and o.admitted < r.done and r.admitted < o.done for o in res))
    assert overlapped > 10  # requests really shared the device
    for r in res:
        P = pool[r.scene][1]
        assert same_bits(r.attr.numpy(), P.attr) and same_bits(r.pos.numpy(), P.pos)
    s = serve.summarize(res, scenes)
    assert s["p99_ms"] >= s["p50_ms"] > 0 and s["bad_status"] == 0


def test_server_respects_hbm_budget(pool):
    from paper_2607_12656_b300 import serve
    scenes = [serve.Scene(b) for b, _ in pool]
    biggest = max(s.footprint() for s in scenes)
    srv = serve.DecodeServer(scenes, slots=4, hbm_budget=biggest)  # one request at a time
    res = srv.run(serve.poisson_arrivals(5000.0, 12, len(scenes), seed=8))
    srv.close()
    res = sorted(res, key=lambda r: r.admitted)
    for a, b in zip(res, res[1:]):
        assert b.admitted >= a.done - 1e-3 or scenes[a.scene].footprint() + scenes[b.scene].footprint() <= biggest
