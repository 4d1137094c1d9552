"""Pins of the oracle's learned geometry coder (Sec. 3.4, "Geometry Occupancy Coding": each
octree level is coded conditioned on the level above it, Eq. 8): context derivation, the
explicit-sample trainer and freeze, the coding round trip and the conditional-entropy bound;
and the library's host encoder for the same coder against the oracle's bytes."""
import numpy as np
import pytest

from oracle import model as M
from oracle import scene as S


def _levels(depth, n, seed):
    rng = np.random.default_rng(seed)
    coord = rng.integers(0, 1 << depth, size=(3, n)).astype(np.int64)
    leaf = np.unique(S.morton(coord, depth))
    return S.octree_levels(leaf, depth), leaf


def test_contexts_against_morton_codes():
    """The node order of a level and each node's (parent byte, child index), derived
    independently from the leaves' Morton codes."""
    D = 6
    levels, leaf = _levels(D, 300, 1)
    for l in range(1, D):
        nodes = np.unique(leaf >> (3 * (D - l)))  # level l nodes in order
        parents = np.unique(leaf >> (3 * (D - l + 1)))
        want_b = np.array([levels[l - 1][np.searchsorted(parents, x >> 3)] for x in nodes])
        want_k = nodes & 7
        ctx = S.geo_children_ctx(levels[l - 1])
        assert np.array_equal(ctx >> 3, want_b) and np.array_equal(ctx & 7, want_k)


def test_context_inputs_hand_case():
    b, k = 0b10110000, 5  # set bits 4, 5, 7: child 5 has one sibling below it
    u = S.geo_ctx_inputs(np.array([8 * b + k]))[0]
    assert u.tolist() == [b - 128, 32 * 5 - 112, 16 * 3 - 64, 32 * 1 - 112]
    all_u = S.geo_ctx_inputs(np.arange(2048))
    assert all_u.min() >= -128 and all_u.max() <= 127


def _token_dataset(q, lr):
    """Every token position p = 56 row + c, in order, as an explicit sample set."""
    pos = np.arange(q.shape[0] * 56)
    u, c, s, _, _ = M.contexts(q, lr, pos)
    return u, c, s


def test_explicit_trainer_and_freeze_reduce_to_the_token_ones():
    """Fed every token position in order, the explicit-sample trainer and freeze draw the
    same samples as the pinned token-based ones and give identical results."""
    from paper_2607_12656_b300.scenegen import kaiming_init, make_scene
    sc = make_scene(1500, 3)
    P = S.prepare(sc.pos, sc.attr, 9, 8)
    q = P.q.astype(np.uint8)
    lr = S.lane_bounds(P.n_rows, 6)
    U, C, Sy = _token_dataset(q, lr)
    p1, l1 = M.train(kaiming_init(4), q, lr, 3, 512, seed=5, lr=1e-3)
    p2, l2 = M.train_ctx(kaiming_init(4), U, C, Sy, 3, 512, seed=5, lr=1e-3)
    assert l1 == l2 and all(np.array_equal(p1[k], p2[k]) for k in M.PARAMS)
    w = {k: v.astype(np.float32) for k, v in p1.items()}
    assert S.model_bytes(M.freeze(w, q, lr, seed=7)) == S.model_bytes(M.freeze_ctx(w, U, C, seed=7))


def _random_model(seed):
    rng = np.random.default_rng(seed)
    return dict(w1=rng.integers(-127, 128, (64, 4)), b1=rng.integers(-3000, 3000, (56, 64)),
                w2=rng.integers(-127, 128, (64, 64)), b2=rng.integers(-20000, 20000, 64),
                w3=rng.integers(-127, 128, (256, 64)), b3=rng.integers(-(1 << 22), 1 << 22, 256),
                m1=int(rng.integers(1, 1 << 30)), sh1=int(rng.integers(20, 32)),
                m2=int(rng.integers(1, 1 << 30)), sh2=int(rng.integers(24, 36)),
                ms=int(rng.integers(1, 1 << 20)), ss=16)


@pytest.fixture(scope="module")
def geo_scene():
    from paper_2607_12656_b300.scenegen import make_scene
    sc = make_scene(20000, 6)
    P = S.prepare(sc.pos, sc.attr, 12, 8)
    assert sum(S.geo_plan(P.levels, S.GEO_LEARNED)) >= 2  # at least two coded levels
    return sc, P


@pytest.mark.parametrize("seed", [0, 1])
def test_round_trip_random_models(geo_scene, seed):
    sc, P = geo_scene
    buf = S.encode(None, None, mode=S.MODE_STATIC, depth=12, lanes=40, prep=P, geo_mode=S.GEO_LEARNED,
                   geo_model=_random_model(seed))
    d = S.decode(buf)
    assert np.array_equal(d["q"], P.q) and np.array_equal(d["pos"], P.pos) and np.array_equal(d["coord"], P.coord)


def _entropy_bits(counts):
    p = counts[counts > 0] / counts.sum()
    return float(-(p * np.log2(p)).sum() * counts.sum())


def test_trained_model_codes_above_the_conditional_entropy(geo_scene):
    """A trained geometry model codes the levels losslessly (fixed-length attributes) and
    never below the empirical conditional entropy of the tokens given (parent byte, child
    index), the bound of any coder using that context; it stays within 25% of it."""
    from paper_2607_12656_b300.scenegen import fixed_bits, kaiming_init
    sc, _ = geo_scene
    P = S.prepare(sc.pos, sc.attr, 12, fixed_bits(1))
    U, C, Sy = S.geo_samples(P.levels)
    p, losses = M.train_ctx(kaiming_init(2), U, C, Sy, 200, 4096, seed=4, lr=3e-3)
    m = M.freeze_ctx({k: v.astype(np.float32) for k, v in p.items()}, U, C, seed=4)
    learned = S.encode(None, None, mode=S.MODE_FIXED, depth=12, bits=fixed_bits(1), prep=P, geo_mode=S.GEO_LEARNED,
                       geo_model=m)
    static = S.encode(None, None, mode=S.MODE_FIXED, depth=12, bits=fixed_bits(1), prep=P, geo_mode=S.GEO_RANS)
    hl, hs = S.parse_header(learned), S.parse_header(static)
    pay_l = hl["off_attr_tab"] - hl["off_geo_pay"]
    pay_s = hs["off_attr_tab"] - hs["off_geo_pay"]
    bound = 0.0
    for l in range(1, 12):
        if S.geo_plan(P.levels, S.GEO_LEARNED)[l]:
            ctx = S.geo_children_ctx(P.levels[l - 1])
            joint = np.bincount(ctx * 256 + P.levels[l], minlength=2048 * 256).reshape(2048, 256).astype(float)
            bound += sum(_entropy_bits(r) for r in joint if r.sum() > 0) / 8.0
    assert bound < pay_l < 1.25 * bound, (bound, pay_l, pay_s)
    d = S.decode(learned)
    assert np.array_equal(d["attr"], P.attr) and np.array_equal(d["coord"], P.coord)


@pytest.mark.parametrize("seed", [0, 1])
def test_library_encoder_bytes_equal_oracle(geo_scene, seed):
    """The library's host encoder writes the oracle's bytes for learned geometry (any valid
    integer model; fixed-length and static attributes), and scene_query reads the stream's
    header facts (its coded levels and their lanes) for the device decoder."""
    from paper_2607_12656_b300 import sgs
    from paper_2607_12656_b300.scenegen import fixed_bits
    sc, P = geo_scene
    m = _random_model(seed)
    want = S.encode(None, None, mode=S.MODE_STATIC, depth=12, lanes=40, prep=P, geo_mode=S.GEO_LEARNED, geo_model=m)
    got = sgs.scene_encode(sc.pos, sc.attr, mode=sgs.MODE_STATIC, depth=12, lanes=40, geo_mode=sgs.GEO_LEARNED,
                           geo_model=S.model_bytes(m))
    assert got == want
    Pf = S.prepare(sc.pos, sc.attr, 12, fixed_bits(2))
    want = S.encode(None, None, mode=S.MODE_FIXED, depth=12, bits=fixed_bits(2), prep=Pf, geo_mode=S.GEO_LEARNED,
                    geo_model=m)
    got = sgs.scene_encode(sc.pos, sc.attr, mode=sgs.MODE_FIXED, depth=12, bits=fixed_bits(2),
                           geo_mode=sgs.GEO_LEARNED, geo_model=S.model_bytes(m))
    assert got == want
    info = sgs.scene_query(got)
    h = S.parse_header(got)
    assert info.geo_mode == sgs.GEO_LEARNED and info.n_geo_coded == h["n_geo_coded"] > 0
    assert info.geo_lanes == sum(S.geo_lanes_for_level(len(b)) for b, c in
                                 zip(Pf.levels, S.geo_plan(Pf.levels, S.GEO_LEARNED)) if c)


def test_library_encoder_trained_geometry_model(geo_scene):
    """A geometry model trained and frozen by the oracle: the library's bytes equal the
    oracle's; a missing or invalid model is refused."""
    from paper_2607_12656_b300 import sgs
    from paper_2607_12656_b300.scenegen import kaiming_init
    sc, P = geo_scene
    U, C, Sy = S.geo_samples(P.levels)
    p, _ = M.train_ctx(kaiming_init(2), U, C, Sy, 40, 2048, seed=4, lr=3e-3)
    m = M.freeze_ctx({k: v.astype(np.float32) for k, v in p.items()}, U, C, seed=4)
    want = S.encode(None, None, mode=S.MODE_STATIC, depth=12, lanes=40, prep=P, geo_mode=S.GEO_LEARNED, geo_model=m)
    got = sgs.scene_encode(sc.pos, sc.attr, mode=sgs.MODE_STATIC, depth=12, lanes=40, geo_mode=sgs.GEO_LEARNED,
                           geo_model=S.model_bytes(m))
    assert got == want
    with pytest.raises(sgs.SgsError):
        sgs.scene_encode(sc.pos, sc.attr, mode=sgs.MODE_STATIC, depth=12, lanes=40, geo_mode=sgs.GEO_LEARNED)
    bad = bytearray(S.model_bytes(m))
    bad[4:8] = (0).to_bytes(4, "little")  # sh1 = 0 is outside the model's range
    with pytest.raises(sgs.SgsError):
        sgs.scene_encode(sc.pos, sc.attr, mode=sgs.MODE_STATIC, depth=12, lanes=40, geo_mode=sgs.GEO_LEARNED,
                         geo_model=bytes(bad))


def test_library_freeze_over_samples_equals_oracle(geo_scene):
    """sgs_freeze_samples writes the oracle's freeze_ctx model byte for byte (same weights,
    samples and seed); it refuses inputs out of range."""
    from paper_2607_12656_b300 import sgs
    from paper_2607_12656_b300.scenegen import kaiming_init
    sc, P = geo_scene
    U, C, Sy = S.geo_samples(P.levels)
    p, _ = M.train_ctx(kaiming_init(3), U, C, Sy, 20, 2048, seed=6, lr=3e-3)
    w = {k: v.astype(np.float32) for k, v in p.items()}
    for seed in (6, 9):
        want = S.model_bytes(M.freeze_ctx(w, U, C, seed=seed))
        got = sgs.sgs_freeze_samples(sgs.pack_weights(w), U, C, seed)
        assert got == want
    with pytest.raises(sgs.SgsError):
        sgs.sgs_freeze_samples(sgs.pack_weights(w), U + 200, C, 6)
    with pytest.raises(sgs.SgsError):
        sgs.sgs_freeze_samples(sgs.pack_weights(w), U, C + 56, 6)


def test_library_geometry_samples_equal_oracle(geo_scene):
    """scene_geo_samples gives the oracle's training samples (inputs, level, token) in order;
    a scene with no coded level has none."""
    from paper_2607_12656_b300 import sgs
    sc, P = geo_scene
    U, C, Sy = S.geo_samples(P.levels)
    u, c, s = sgs.scene_geo_samples(sc.pos, sc.attr, 12)
    assert np.array_equal(u, U) and np.array_equal(c, C) and np.array_equal(s, Sy)
    from paper_2607_12656_b300.scenegen import make_scene
    small = make_scene(300, 2)
    u, c, s = sgs.scene_geo_samples(small.pos, small.attr, 8)
    assert len(u) == len(c) == len(s) == 0
