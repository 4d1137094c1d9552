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


def _batch_items(pool, with_index=()):
    """Device buffers for every pool scene; scenes listed in with_index also get coordinates
    and a permuted out_index (the scatter variants of every stage)."""
    items, refs = [], []
    for j, (buf, P) in enumerate(pool):
        info = sgs.scene_query(buf)
        n = info.n_rows
        bits = torch.frombuffer(bytearray(buf), dtype=torch.uint8).cuda()
        attr = torch.full((56, n), float("nan"), device="cuda")
        pos = torch.full((3, n), float("nan"), device="cuda")
        if j in with_index:
            perm = np.random.default_rng(j).permutation(n).astype(np.int32)
            crd = torch.full((3, n), -1, dtype=torch.int32, device="cuda")
            items.append((bits, info, attr, pos, crd, torch.from_numpy(perm).cuda()))
            refs.append((P, perm))
        else:
            items.append((bits, info, attr, pos))
            refs.append((P, None))
    return items, refs


def _check_outputs(items, refs, skip=()):
    for j, (it, (P, perm)) in enumerate(zip(items, refs)):
        if j in skip:
            continue
        attr, pos = it[2].cpu().numpy(), it[3].cpu().numpy()
        if perm is None:
            assert same_bits(attr, P.attr) and same_bits(pos, P.pos), j
        else:
            assert same_bits(attr[:, perm], P.attr) and same_bits(pos[:, perm], P.pos), j
            assert np.array_equal(it[4].cpu().numpy()[:, perm].view(np.uint32), P.coord), j


def _reset(items):
    for it in items:
        it[2].fill_(float("nan"))
        it[3].fill_(float("nan"))


def test_batch_decode_matches_alone(pool):
    items, refs = _batch_items(pool)
    need = sgs.scene_batch_bytes(items)
    assert need >= sum((it[1].scratch_bytes + 255) // 256 * 256 for it in items)
    c = sgs.Context(0, need)
    sgs.scene_decode_batch(c, items)
    assert c.sync() == sgs.OK
    _check_outputs(items, refs)
    # a smaller scratch is refused before anything runs
    c2 = sgs.Context(0, need - 256)
    with pytest.raises(sgs.SgsError) as e:
        sgs.scene_decode_batch(c2, items)
    assert e.value.code == sgs.E_NOMEM
    c2.close()
    c.close()


def test_batch_plan_runs_again_and_replays_in_a_graph(pool):
    items, refs = _batch_items(pool, with_index=(1, 2, 3, 4))
    c = sgs.Context(0, 0)
    plan = sgs.BatchPlan(c, items)
    before = c.launch_count()
    plan.run()
    assert c.sync() == sgs.OK
    launches = c.launch_count() - before
    assert launches <= 16 + 17  # one launch per stage, whatever the number of scenes
    assert plan.status() == [sgs.OK] * len(items)
    _check_outputs(items, refs)
    _reset(items)
    plan.run()  # the work lists are reused: counters and flags are cleared by the run itself
    assert c.sync() == sgs.OK
    _check_outputs(items, refs)
    # captured once, replayed twice
    _reset(items)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(s)
    g.replay()
    torch.cuda.synchronize()
    _check_outputs(items, refs)
    _reset(items)
    g.replay()
    torch.cuda.synchronize()
    assert c.sync() == sgs.OK and plan.status() == [sgs.OK] * len(items)
    _check_outputs(items, refs)
    del g
    plan.close()
    c.close()


def test_batch_completion_times(pool):
    """Every scene's completion time (completion flags, device global timer) lies inside the
    run as the caller's stream events see it, and a graph replay stamps new ones."""
    items, refs = _batch_items(pool)
    c = sgs.Context(0, 0)
    plan = sgs.BatchPlan(c, items)
    plan.run()  # warm
    assert c.sync() == sgs.OK
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    plan.run(torch.cuda.current_stream())
    e1.record()
    torch.cuda.synchronize()
    span = e0.elapsed_time(e1)
    t = plan.times_ms()
    assert len(t) == len(items)
    assert all(0.0 <= v <= span + 0.01 for v in t), (t, span)
    assert max(t) > 0.5 * span  # the last scene ends near the end of the run
    _check_outputs(items, refs)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(s)
    plan.times_ms()  # nothing ran during the capture; the last run's times stay
    g.replay()
    torch.cuda.synchronize()
    t2 = plan.times_ms()
    assert all(v >= 0.0 for v in t2) and max(t2) > 0.0
    del g
    plan.close()
    c.close()


def test_batch_status_isolates_a_corrupt_scene(pool):
    """A scene whose payload was damaged reports its own status; the others decode intact."""
    bad = 4  # a static-mode scene of the pool
    assert S.parse_header(pool[bad][0])["mode"] == S.MODE_STATIC
    damaged = list(pool)
    buf = bytearray(pool[bad][0])
    h = S.parse_header(bytes(buf))
    lo = h["off_attr_pay"]
    for k in range(lo, min(lo + 64, h["total"])):
        buf[k] ^= 0x5A
    damaged[bad] = (bytes(buf), pool[bad][1])
    items, refs = _batch_items(damaged)
    c = sgs.Context(0, 0)
    plan = sgs.BatchPlan(c, items)
    plan.run()
    st = plan.status()
    assert c.sync() == sgs.E_CORRUPT
    assert st[bad] == sgs.E_CORRUPT and all(v == sgs.OK for j, v in enumerate(st) if j != bad)
    _check_outputs(items, refs, skip=(bad,))
    plan.close()
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
    biggest = max(s.buffers() for s in scenes)
    scratch = 4 * max(int(s.info.scratch_bytes) for s in scenes)  # the 4 slots' scratch
    srv = serve.DecodeServer(scenes, slots=4, hbm_budget=scratch + biggest)  # one request at a time
    res = srv.run(serve.poisson_arrivals(5000.0, 12, len(scenes), seed=8))
    srv.close()
    assert all(r.status == sgs.OK for r in res)
    res = sorted(res, key=lambda r: r.admitted)
    for a, b in zip(res, res[1:]):
        assert b.admitted >= a.done - 1e-3 or scenes[a.scene].buffers() + scenes[b.scene].buffers() <= biggest
