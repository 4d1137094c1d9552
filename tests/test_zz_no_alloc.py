"""The allocation-free decode entry point, scene_decode_noalloc.

Callers that own all device memory (an engine or renderer that forbids allocation after
start-up), or that must not let cudaMalloc / cudaFree synchronize the device mid-loop, cannot
create a context.  For them the library decodes with a fixed scratch array compiled into it.
These checks go through the C ABI: the entry point's output equals scene_decode's, bit for
bit (the tolerance of every decode test here), on consecutive calls that share the array --
each call finds the previous call's leftovers -- and a scene needing more scratch than the
array is refused before anything runs.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2607_12656_b300 import sgs
from paper_2607_12656_b300.scenegen import fixed_bits, make_scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bits(n, seed, mode, ctx=None):
    sc = make_scene(n, seed)
    if mode == sgs.MODE_FIXED:
        return sgs.scene_encode(sc.pos, sc.attr, mode=mode, depth=15, bits=fixed_bits(seed), geo_mode=sgs.GEO_RAW)
    if mode in (sgs.MODE_LEARNED, sgs.MODE_LEARNED_PE):
        # a short training run on the device: the decode's work does not depend on the weights
        from paper_2607_12656_b300 import learned
        lanes = 640
        train = learned.train_and_freeze if mode == sgs.MODE_LEARNED else learned.train_and_freeze_pe
        model = train(ctx, sc, 14, lanes, steps=40, batch=8192, seed=3)
        return sgs.scene_encode(sc.pos, sc.attr, mode=mode, depth=14, lanes=lanes, model=model, ctx=ctx,
                                geo_mode=sgs.GEO_RANS)
    return sgs.scene_encode(sc.pos, sc.attr, mode=mode, depth=14, lanes=2048, geo_mode=sgs.GEO_RANS)


def _outputs(n):
    return (torch.full((56, n), float("nan"), device="cuda"), torch.full((3, n), float("nan"), device="cuda"),
            torch.full((3, n), -1, dtype=torch.int32, device="cuda"))


def _same(a, b):
    return torch.equal(a.contiguous().view(torch.int32), b.contiguous().view(torch.int32))


def test_noalloc_matches_scene_decode_on_consecutive_calls():
    """Every coding mode, each call finding another mode's leftovers in the shared array (the
    learned modes use other scratch regions and, for the position-aware model, a launch after
    the octree on the caller's stream), and each scene decoded twice in a row."""
    ctx = sgs.Context(0, 0)
    scenes = [_bits(150_000, 51, sgs.MODE_FIXED), _bits(60_000, 52, sgs.MODE_STATIC),
              _bits(30_000, 54, sgs.MODE_LEARNED, ctx), _bits(40_000, 55, sgs.MODE_LEARNED_PE, ctx)]
    ref = []
    for buf in scenes:
        info = sgs.scene_query(buf)
        assert info.scratch_bytes <= sgs.NOALLOC_SCRATCH_BYTES - 256
        ctx.reserve(info.scratch_bytes)
        dev = torch.frombuffer(bytearray(buf), dtype=torch.uint8).cuda()
        a, p, c = _outputs(info.n_rows)
        sgs.scene_decode(ctx, dev, info, a, p, c)
        assert ctx.sync() == sgs.OK
        ref.append((dev, info, a, p, c))
    ctx.close()
    # mode after mode, each scene twice in a row, then back to the first ones
    for k in (0, 2, 2, 1, 3, 3, 0, 0, 2, 1, 1, 3, 0):
        dev, info, a_ref, p_ref, c_ref = ref[k]
        a, p, c = _outputs(info.n_rows)
        st = sgs.scene_decode_noalloc(dev, info, a, p, c)
        assert st == sgs.OK
        assert _same(a, a_ref) and _same(p, p_ref) and _same(c, c_ref)
        if info.mode == sgs.MODE_LEARNED_PE:
            # without caller coordinates the position-aware model reads the array's own copy
            a, p, _ = _outputs(info.n_rows)
            assert sgs.scene_decode_noalloc(dev, info, a, p, None) == sgs.OK
            assert _same(a, a_ref) and _same(p, p_ref)


def test_noalloc_refuses_scene_beyond_the_array():
    buf = _bits(5_000, 53, sgs.MODE_FIXED)
    info = sgs.scene_query(buf)
    big = sgs.SceneInfo.from_buffer_copy(info)
    big.scratch_bytes = sgs.NOALLOC_SCRATCH_BYTES  # more than the array holds after its status word
    dev = torch.frombuffer(bytearray(buf), dtype=torch.uint8).cuda()
    a, p, c = _outputs(info.n_rows)
    with pytest.raises(sgs.SgsError) as e:
        sgs.scene_decode_noalloc(dev, big, a, p, c)
    assert e.value.code == sgs.E_NOMEM
    assert torch.isnan(a).all()  # nothing ran
