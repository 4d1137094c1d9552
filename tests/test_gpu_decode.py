"""GPU parity: the CUDA decode path (through the C ABI) against the CPU oracle, bit for bit.

Decoded values must be identical: fp32 attributes compared as bit patterns (0 ULP), positions
and voxel coordinates exactly.  Outputs are poisoned (NaN / 0xFFFFFFFF) before each decode so
an unwritten row fails the comparison."""
import numpy as np
import pytest

from oracle import scene as S
from paper_2607_12656_b300 import sgs
from paper_2607_12656_b300.scenegen import fixed_bits, make_scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = sgs.Context(0, 1 << 20)
    yield c
    c.close()


def gpu_decode(ctx, buf, out_index=None):
    info = sgs.scene_query(buf)
    ctx.reserve(info.scratch_bytes)
    bits = torch.frombuffer(bytearray(buf), dtype=torch.uint8).cuda()
    n = info.n_rows
    attr = torch.full((56, max(n, 1)), float("nan"), device="cuda")
    pos = torch.full((3, max(n, 1)), float("nan"), device="cuda")
    crd = torch.full((3, max(n, 1)), -1, dtype=torch.int32, device="cuda")
    oi = None if out_index is None else torch.from_numpy(out_index.astype(np.int32)).cuda()
    sgs.scene_decode(ctx, bits, info, attr, pos, crd, oi)
    st = ctx.sync()
    return (st, attr.cpu().numpy()[:, :n], pos.cpu().numpy()[:, :n],
            crd.cpu().numpy()[:, :n].view(np.uint32), info)


def same_bits(a, b):
    return a.shape == b.shape and np.array_equal(np.ascontiguousarray(a).view(np.uint32),
                                                 np.ascontiguousarray(b).view(np.uint32))


def check(ctx, sc, depth, **kw):
    mode = kw["mode"]
    bits = kw.pop("bits", 8)
    P = S.prepare(sc.pos, sc.attr, depth, bits)
    buf = S.encode(sc.pos, sc.attr, depth=depth, bits=bits, prep=P, **kw)
    st, attr, pos, crd, info = gpu_decode(ctx, buf)
    assert st == sgs.OK, sgs.lib().sgs_strerror(st)
    assert same_bits(attr, P.attr), "attributes differ"
    assert same_bits(pos, P.pos), "positions differ"
    assert np.array_equal(crd, P.coord), "coordinates differ"
    return P, buf


SIZES = [(0, 3), (1, 1), (2, 5), (7, 2), (33, 4), (1000, 12), (20000, 12), (60000, 14)]


@pytest.mark.parametrize("n,depth", SIZES)
@pytest.mark.parametrize("geo", [S.GEO_RAW, S.GEO_RANS])
def test_fixed_parity(ctx, n, depth, geo):
    check(ctx, make_scene(n, 11 + n), depth, mode=S.MODE_FIXED, bits=fixed_bits(n), geo_mode=geo)


@pytest.mark.parametrize("n,depth", SIZES)
@pytest.mark.parametrize("lanes", [1, 31, 33, 100])
def test_static_parity(ctx, n, depth, lanes):
    check(ctx, make_scene(n, 13 + n), depth, mode=S.MODE_STATIC, lanes=lanes, geo_mode=S.GEO_RANS)


def test_fixed_all_widths(ctx):
    sc = make_scene(5000, 3)
    for b in (1, 2, 3, 7, 9, 11, 12, 13, 15, 16):
        check(ctx, sc, 10, mode=S.MODE_FIXED, bits=b, geo_mode=S.GEO_RAW)


def test_duplicates(ctx):
    """Coarse grid: many Gaussians share a voxel; one position per voxel plus counts."""
    sc = make_scene(4000, 5)
    P, _ = check(ctx, sc, 3, mode=S.MODE_STATIC, lanes=40, geo_mode=S.GEO_RAW)
    assert len(P.dups) > 10
    check(ctx, sc, 2, mode=S.MODE_FIXED, bits=fixed_bits(2), geo_mode=S.GEO_RAW)


def test_geometry_lane_counts(ctx, small_scene):
    for gl in (1, 32, 33, 200, 4000):
        check(ctx, small_scene, 12, mode=S.MODE_STATIC, lanes=64, geo_mode=S.GEO_RANS, geo_lanes=gl)


def test_out_index_scatter(ctx, small_scene):
    P = S.prepare(small_scene.pos, small_scene.attr, 12, 8)
    buf = S.encode(None, None, mode=S.MODE_STATIC, depth=12, lanes=64, prep=P)
    perm = np.random.default_rng(0).permutation(P.n_rows)
    st, attr, pos, crd, _ = gpu_decode(ctx, buf, out_index=perm)
    assert st == sgs.OK
    want_attr = np.empty_like(P.attr)
    want_attr[:, perm] = P.attr
    want_pos = np.empty_like(P.pos)
    want_pos[:, perm] = P.pos
    assert same_bits(attr, want_attr) and same_bits(pos, want_pos)


def test_library_encoder_roundtrip_on_gpu(ctx, small_scene):
    """The library's own encoder -> GPU decode equals the oracle's decoded values."""
    P = S.prepare(small_scene.pos, small_scene.attr, 12, 8)
    buf = sgs.scene_encode(small_scene.pos, small_scene.attr, mode=sgs.MODE_STATIC, depth=12, lanes=96)
    st, attr, pos, _, _ = gpu_decode(ctx, buf)
    assert st == sgs.OK and same_bits(attr, P.attr) and same_bits(pos, P.pos)


def test_scratch_too_small_is_refused():
    c = sgs.Context(0, 0)
    sc = make_scene(1000, 1)
    buf = S.encode(sc.pos, sc.attr, mode=S.MODE_FIXED, depth=10, bits=fixed_bits(1))
    info = sgs.scene_query(buf)
    bits = torch.frombuffer(bytearray(buf), dtype=torch.uint8).cuda()
    attr = torch.zeros((56, info.n_rows), device="cuda")
    pos = torch.zeros((3, info.n_rows), device="cuda")
    with pytest.raises(sgs.SgsError) as e:
        sgs.scene_decode(c, bits, info, attr, pos)
    assert e.value.code == sgs.E_NOMEM
    c.close()


def test_corrupt_payload_detected(ctx, small_scene):
    """Bit flips in the coded payloads: the decoder reports CORRUPT or decodes different
    tokens; it never reads or writes out of bounds (all accesses are checked)."""
    P = S.prepare(small_scene.pos, small_scene.attr, 12, 8)
    buf = S.encode(None, None, mode=S.MODE_STATIC, depth=12, lanes=64, prep=P)
    h = S.parse_header(buf)
    rng = np.random.default_rng(1)
    flagged = 0
    for trial in range(12):
        b = bytearray(buf)
        sec = ("attr_pay", "geo_pay")[trial % 2]
        lo = h["off_" + sec]
        hi = h["total"] if sec == "attr_pay" else h["off_attr_tab"]
        k = int(rng.integers(lo, hi))
        b[k] ^= 1 << int(rng.integers(0, 8))
        st, attr, pos, _, _ = gpu_decode(ctx, bytes(b))
        if st == sgs.E_CORRUPT:
            flagged += 1
        else:
            assert st == sgs.OK and not (same_bits(attr, P.attr) and same_bits(pos, P.pos))
    assert flagged >= 6


@pytest.fixture(scope="module")
def fixed_1m():
    sc = make_scene(1_000_000, 1000)
    bits = fixed_bits(1000)
    P = S.prepare(sc.pos, sc.attr, 16, bits)
    return sc, P, bits


def test_full_size_fixed_length_scene(ctx, fixed_1m):
    """The 1M-Gaussian fixed-length workload, every output compared."""
    sc, P, bits = fixed_1m
    buf = sgs.scene_encode(sc.pos, sc.attr, mode=sgs.MODE_FIXED, depth=16, bits=bits, geo_mode=sgs.GEO_RAW)
    assert buf == S.encode(None, None, mode=S.MODE_FIXED, depth=16, bits=bits, geo_mode=S.GEO_RAW, prep=P)
    st, attr, pos, crd, _ = gpu_decode(ctx, buf)
    assert st == sgs.OK and same_bits(attr, P.attr) and same_bits(pos, P.pos)
    assert np.array_equal(crd, P.coord)


def test_full_size_static_scene(ctx, fixed_1m):
    sc, _, _ = fixed_1m
    P = S.prepare(sc.pos, sc.attr, 16, 8)
    for lanes in (4096, 65536):
        buf = sgs.scene_encode(sc.pos, sc.attr, mode=sgs.MODE_STATIC, depth=16, lanes=lanes, geo_mode=sgs.GEO_RANS)
        st, attr, pos, _, _ = gpu_decode(ctx, buf)
        assert st == sgs.OK and same_bits(attr, P.attr) and same_bits(pos, P.pos)


def test_autotune_sweeps_group_sizes(ctx, small_scene):
    """The tuner measures every candidate W: smaller groups mean more lanes and a larger
    bitstream, and every trial decode succeeded; the choice honours the target."""
    from paper_2607_12656_b300.tune import LaneTuner
    sc = small_scene
    r = sgs.autotune(ctx, sc.pos, sc.attr, mode=sgs.MODE_STATIC, depth=12, rows_per_lane=[8, 32, 128], reps=3)
    assert r["lanes"][0] > r["lanes"][1] > r["lanes"][2]
    assert r["bytes"][0] > r["bytes"][1] > r["bytes"][2]
    assert all(ms > 0 for ms in r["ms"])
    assert r["ms"][r["best"]] == min(r["ms"])
    loose = sgs.autotune(ctx, sc.pos, sc.attr, mode=sgs.MODE_STATIC, depth=12, rows_per_lane=[8, 32, 128],
                         reps=3, max_ms=1e3)
    assert loose["best"] == 2  # every candidate meets the target: the smallest bitstream wins
    t = LaneTuner()
    lanes = t.choose_lanes(ctx, sc.pos, sc.attr, mode=sgs.MODE_STATIC, depth=12, candidates=(16, 64), reps=2)
    assert lanes >= 1 and len(t.table) == 1
    with pytest.raises(sgs.SgsError):  # fixed-length scenes have no lanes: one candidate only
        sgs.autotune(ctx, sc.pos, sc.attr, mode=sgs.MODE_FIXED, depth=12, rows_per_lane=[32, 64])


@pytest.mark.parametrize("mode,shapes", [(S.MODE_FIXED, [1, 3, 8]), (S.MODE_STATIC, [1, 5, 32])])
def test_launch_shapes_decode_bit_exact(ctx, mode, shapes):
    """The attribute decoder's launch shape (warps per CTA, the autotuner's second knob) does
    not change a bit of the result: fixed-length items and static groups land in other CTAs,
    ragged last CTAs included."""
    sc = make_scene(60_000, 91)
    kw = dict(mode=mode, bits=fixed_bits(14), geo_mode=S.GEO_RAW) if mode == S.MODE_FIXED else \
        dict(mode=mode, lanes=700, geo_mode=S.GEO_RANS)
    try:
        for w in shapes:
            ctx.set_launch_shape(mode, w)
            check(ctx, sc, 14, **dict(kw))
    finally:
        ctx.set_launch_shape(mode, 0)
    for bad_mode, bad_w in ((mode, 9 if mode == S.MODE_FIXED else 33), (S.MODE_LEARNED, 4)):
        with pytest.raises(sgs.SgsError):
            ctx.set_launch_shape(bad_mode, bad_w)


def test_autotune_chooses_launch_shapes(ctx, small_scene):
    """Every W is decoded at every candidate shape and keeps its fastest; fixed-length scenes
    tune the shape alone; the tuner sets its choice on the context, whose decodes stay exact."""
    from paper_2607_12656_b300.tune import LaneTuner
    sc = small_scene
    r = sgs.autotune(ctx, sc.pos, sc.attr, mode=sgs.MODE_STATIC, depth=12, rows_per_lane=[16, 64], reps=2,
                     warps_per_cta=[4, 32])
    assert all(w in (4, 32) for w in r["warps"]) and r["best_warps"] == r["warps"][r["best"]]
    f = sgs.autotune(ctx, sc.pos, sc.attr, mode=sgs.MODE_FIXED, depth=12, rows_per_lane=[1], reps=2,
                     warps_per_cta=[2, 8], geo_mode=sgs.GEO_RAW)
    assert f["lanes"] == [0] and f["best_warps"] in (2, 8)
    try:
        lanes, warps = LaneTuner().choose(ctx, sc.pos, sc.attr, mode=sgs.MODE_FIXED, depth=12, reps=2,
                                          geo_mode=sgs.GEO_RAW)
        assert lanes == 0 and warps in (2, 4, 8)
        check(ctx, sc, 12, mode=S.MODE_FIXED, bits=fixed_bits(12), geo_mode=S.GEO_RAW)
    finally:
        ctx.set_launch_shape(sgs.MODE_FIXED, 0)


@pytest.mark.parametrize("n,lanes", [(20_000, 40), (60_000, 2048), (30_000, 33), (5_000, 1)])
def test_device_static_encoder_matches_oracle_and_host(ctx, n, lanes):
    """The attribute rANS coding on the device (with a context) writes the oracle's bytes, and
    the host coding (no context) the same; lane counts include ragged last groups."""
    sc = make_scene(n, 71)
    P = S.prepare(sc.pos, sc.attr, 13, 8)
    want = S.encode(None, None, mode=S.MODE_STATIC, depth=13, lanes=lanes, prep=P)
    dev = sgs.scene_encode(sc.pos, sc.attr, mode=sgs.MODE_STATIC, depth=13, lanes=lanes, ctx=ctx)
    host = sgs.scene_encode(sc.pos, sc.attr, mode=sgs.MODE_STATIC, depth=13, lanes=lanes)
    assert dev == want and host == want


@pytest.mark.parametrize("n,depth", [(1, 21), (3, 21), (5000, 21), (5000, 20), (20000, 17)])
def test_deep_octrees(ctx, n, depth):
    """Deep trees (up to the 21-bit coordinate limit): every leaf walks depth levels up to the
    root; a single Gaussian is one chain of 21 nodes."""
    sc = make_scene(n, 300 + depth)
    check(ctx, sc, depth, mode=S.MODE_FIXED, bits=fixed_bits(depth), geo_mode=S.GEO_RAW)
    check(ctx, sc, depth, mode=S.MODE_STATIC, lanes=7, geo_mode=S.GEO_RANS)


def _scene_at(codes, depth, seed):
    """A scene with one Gaussian at the centre of each voxel of Morton codes `codes` (plus
    duplicates on a few of them), attributes from the generator."""
    from paper_2607_12656_b300.scenegen import make_scene as mk
    coord = S.demorton(np.asarray(codes, np.uint64), depth).astype(np.float64)  # [3][n]
    rng = np.random.default_rng(seed)
    extra = rng.integers(0, coord.shape[1], size=max(1, coord.shape[1] // 50))
    coord = np.concatenate([coord, coord[:, extra]], axis=1)
    pos = ((coord + 0.5) / float(1 << depth)).astype(np.float32)
    sc = mk(pos.shape[1], seed)
    sc.pos = np.ascontiguousarray(pos)
    return sc


def test_octree_dense_cluster_subtree(ctx):
    """A dense cluster of 60,000 voxels under one node of the split level among 6,000 scattered
    ones (depth 16): that node's subtree is wider than a CTA's shared memory, so its CTA falls
    back to parent entries and a climb to the split level; every position still matches."""
    rng = np.random.default_rng(0)
    D = 16
    sparse = rng.integers(0, 8 ** D, size=6000, dtype=np.uint64)
    base = np.uint64(rng.integers(0, 8 ** 5)) << np.uint64(3 * (D - 5))
    dense = base + rng.integers(0, 8 ** (D - 5), size=60000, dtype=np.uint64)
    sc = _scene_at(np.unique(np.concatenate([sparse, dense])), D, 41)
    check(ctx, sc, D, mode=S.MODE_FIXED, bits=fixed_bits(41), geo_mode=S.GEO_RAW)
    check(ctx, sc, D, mode=S.MODE_STATIC, lanes=300, geo_mode=S.GEO_RANS)


def test_octree_fan_and_chain(ctx):
    """Depth 21: 40,000 voxels fanning out at level 7 and one isolated 21-level chain; a slab
    boundary falls between very unequal subtrees."""
    rng = np.random.default_rng(1)
    D = 21
    codes = np.unique(np.concatenate([rng.integers(0, 8 ** 7, size=40000, dtype=np.uint64) << np.uint64(3 * 14),
                                      np.array([8 ** 21 - 1], np.uint64)]))
    sc = _scene_at(codes, D, 42)
    check(ctx, sc, D, mode=S.MODE_FIXED, bits=fixed_bits(42), geo_mode=S.GEO_RAW)


def test_duplicates_with_scatter_and_coords(ctx):
    """Many Gaussians per voxel at a shallow depth, rows scattered by out_index, with voxel
    coordinates: each leaf writes all its rows."""
    sc = make_scene(9000, 6)
    P = S.prepare(sc.pos, sc.attr, 4, 8)
    assert len(P.dups) > 20
    buf = S.encode(None, None, mode=S.MODE_STATIC, depth=4, lanes=50, geo_mode=S.GEO_RAW, prep=P)
    perm = np.random.default_rng(6).permutation(P.n_rows)
    st, attr, pos, crd, _ = gpu_decode(ctx, buf, out_index=perm)
    assert st == sgs.OK
    assert same_bits(attr[:, perm], P.attr) and same_bits(pos[:, perm], P.pos)
    assert np.array_equal(crd[:, perm], P.coord)


def test_corrupt_raw_geometry_detected(ctx, small_scene):
    """Flipped bits in raw occupancy tokens (fixed-length scene): the level counts no longer
    match the tokens, and the decoder reports CORRUPT (or decodes other positions) without
    reading or writing out of bounds."""
    P = S.prepare(small_scene.pos, small_scene.attr, 12, fixed_bits(4))
    buf = S.encode(None, None, mode=S.MODE_FIXED, depth=12, bits=fixed_bits(4), geo_mode=S.GEO_RAW, prep=P)
    h = S.parse_header(buf)
    rng = np.random.default_rng(3)
    flagged = 0
    for trial in range(12):
        b = bytearray(buf)
        k = int(rng.integers(h["off_geo_raw"], h["off_geo_raw"] + h["n_geo"]))
        b[k] ^= 1 << int(rng.integers(0, 8))
        st, attr, pos, _, _ = gpu_decode(ctx, bytes(b))
        if st == sgs.E_CORRUPT:
            flagged += 1
        else:
            assert st == sgs.OK and not same_bits(pos, P.pos)
    assert flagged >= 10


def _crowded_scene(n, seed):
    """Eight channels whose values sit mostly at two levels and otherwise on ~250 rare ones,
    each seen a few times: their static tables pack many small-frequency symbols into single
    64-slot buckets, so the decoder's bucket search must step past several symbol starts."""
    sc = make_scene(n, seed)
    attr = sc.attr.copy()
    rng = np.random.default_rng(seed)
    for c in range(8):
        common = rng.choice(np.array([0.0, 1.0]), n)
        rare = rng.integers(2, 255, n) / 255.0
        v = np.where(rng.random(n) < 0.97, common, rare).astype(np.float32)
        v[:2] = (0.0, 1.0)
        attr[c] = v
    return type("Scene", (), {"pos": sc.pos, "attr": attr})()


@pytest.mark.parametrize("lanes", [33, 100, 1000])
def test_static_crowded_buckets(ctx, lanes):
    sc = _crowded_scene(20_000, 71 + lanes)
    P = S.prepare(sc.pos, sc.attr, 12, 8)
    crowded = 0
    for c in range(8):
        f = S.normalize_freq(np.bincount(P.q[:, c], minlength=256))
        starts = np.cumsum(f)[:-1][f[1:] > 0]  # first slot of every present symbol after the first
        crowded = max(crowded, int(np.bincount(starts >> 6, minlength=1024).max()))
    assert crowded >= 3, "the scene must put several symbol starts into one bucket"
    check(ctx, sc, 12, mode=S.MODE_STATIC, lanes=lanes, geo_mode=S.GEO_RANS)
