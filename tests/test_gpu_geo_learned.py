"""GPU parity of the learned geometry decoder (SGS_GEO_LEARNED; Sec. 3.4 "Geometry Occupancy
Coding", Eq. 8: each octree level coded conditioned on the level above it): bitstreams written
by the oracle's encoder decode on the device, through the C ABI, to the oracle's values bit for
bit -- positions and voxel coordinates exactly, attributes as fp32 bit patterns -- for arbitrary
valid integer models and for models trained and frozen by the oracle, at depths 12 to 17."""
import numpy as np
import pytest

from oracle import model as M
from oracle import scene as S
from paper_2607_12656_b300 import sgs
from paper_2607_12656_b300.scenegen import fixed_bits, kaiming_init, make_scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_gpu_decode import gpu_decode, same_bits  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = sgs.Context(0, 1 << 20)
    yield c
    c.close()


def _random_model(seed):
    rng = np.random.default_rng(seed)
    return dict(w1=rng.integers(-127, 128, (64, 4)), b1=rng.integers(-3000, 3000, (56, 64)),
                w2=rng.integers(-127, 128, (64, 64)), b2=rng.integers(-20000, 20000, 64),
                w3=rng.integers(-127, 128, (256, 64)), b3=rng.integers(-(1 << 22), 1 << 22, 256),
                m1=int(rng.integers(1, 1 << 30)), sh1=int(rng.integers(20, 32)),
                m2=int(rng.integers(1, 1 << 30)), sh2=int(rng.integers(24, 36)),
                ms=int(rng.integers(1, 1 << 20)), ss=16)


def _trained_model(P, steps=60):
    U, C, Sy = S.geo_samples(P.levels)
    p, _ = M.train_ctx(kaiming_init(2), U, C, Sy, steps, 4096, seed=4, lr=3e-3)
    return M.freeze_ctx({k: v.astype(np.float32) for k, v in p.items()}, U, C, seed=4)


def _check(ctx, P, buf):
    st, attr, pos, crd, info = gpu_decode(ctx, buf)
    assert info.geo_mode == sgs.GEO_LEARNED and info.n_geo_coded > 0
    assert st == sgs.OK, sgs.lib().sgs_strerror(st)
    assert same_bits(pos, P.pos) and np.array_equal(crd, P.coord)
    assert same_bits(attr, P.attr)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_models_static_attributes(ctx, seed):
    sc = make_scene(20000, 6)
    P = S.prepare(sc.pos, sc.attr, 12, 8)
    buf = S.encode(None, None, mode=S.MODE_STATIC, depth=12, lanes=40, prep=P, geo_mode=S.GEO_LEARNED,
                   geo_model=_random_model(seed))
    _check(ctx, P, buf)


@pytest.mark.parametrize("n,depth", [(60_000, 14), (150_000, 16), (120_000, 17)])
def test_trained_models_fixed_length(ctx, n, depth):
    sc = make_scene(n, 900 + depth)
    P = S.prepare(sc.pos, sc.attr, depth, fixed_bits(depth))
    assert sum(S.geo_plan(P.levels, S.GEO_LEARNED)) >= 3  # several coded levels
    buf = S.encode(None, None, mode=S.MODE_FIXED, depth=depth, bits=fixed_bits(depth), prep=P,
                   geo_mode=S.GEO_LEARNED, geo_model=_trained_model(P))
    _check(ctx, P, buf)


def test_library_encoded_scene_and_learned_attributes(ctx):
    """The library's encoder (a random geometry model) with the learned attribute model on the
    device: both learned coders in one stream decode to the oracle's values."""
    from paper_2607_12656_b300 import learned
    sc = make_scene(40_000, 77)
    P = S.prepare(sc.pos, sc.attr, 14, 8)
    amodel = learned.train_and_freeze(ctx, sc, 14, 1024, steps=40, batch=8192, seed=3)
    buf = sgs.scene_encode(sc.pos, sc.attr, mode=sgs.MODE_LEARNED, depth=14, lanes=1024, model=amodel, ctx=ctx,
                           geo_mode=sgs.GEO_LEARNED, geo_model=S.model_bytes(_random_model(5)))
    _check(ctx, P, buf)


def test_corrupt_geometry_model_flagged(ctx):
    sc = make_scene(20000, 6)
    P = S.prepare(sc.pos, sc.attr, 12, 8)
    buf = bytearray(S.encode(None, None, mode=S.MODE_STATIC, depth=12, lanes=40, prep=P, geo_mode=S.GEO_LEARNED,
                             geo_model=_random_model(0)))
    h = S.parse_header(bytes(buf))
    buf[h["off_geo_tab"] + 4:h["off_geo_tab"] + 8] = (60).to_bytes(4, "little")  # sh1 out of range
    st, _, _, _, _ = gpu_decode(ctx, bytes(buf))
    assert st == sgs.E_CORRUPT


def test_noalloc_and_batch_refusal(ctx):
    """The allocation-free entry point decodes the stream too; a batch plan refuses it."""
    sc = make_scene(20000, 8)
    P = S.prepare(sc.pos, sc.attr, 12, 8)
    buf = S.encode(None, None, mode=S.MODE_STATIC, depth=12, lanes=40, prep=P, geo_mode=S.GEO_LEARNED,
                   geo_model=_random_model(3))
    info = sgs.scene_query(buf)
    bits = torch.frombuffer(bytearray(buf), dtype=torch.uint8).cuda()
    attr = torch.full((56, info.n_rows), float("nan"), device="cuda")
    pos = torch.full((3, info.n_rows), float("nan"), device="cuda")
    assert sgs.scene_decode_noalloc(bits, info, attr, pos) == sgs.OK
    assert same_bits(attr.cpu().numpy(), P.attr) and same_bits(pos.cpu().numpy(), P.pos)
    with pytest.raises(sgs.SgsError) as e:
        sgs.scene_batch_bytes([(bits, info, attr, pos)])
    assert e.value.code == sgs.E_UNSUPPORTED
