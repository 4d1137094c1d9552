"""Pins of the oracle's position-aware learned model (Sec. 3.4.2 Fourier positional embedding,
Sec. 3.2 conditional Laplace): sine table, embedding phases, integer Laplace CDF, fp64
gradients, freeze and the coding round trip."""
import ctypes
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import model as M
from oracle import model_pe as E
from oracle import native
from oracle import scene as S
from oracle.exp2q import exp2q_table


def test_sin8_special_values_and_symmetries():
    T = E.sin8_table()
    assert T[0] == 0 and T[64] == 127 and T[128] == 0 and T[192] == -127
    assert T[32] == 90  # 127 / sqrt(2) = 89.80
    for j in range(1, 256):
        assert T[256 - j] == -T[j]              # sin(-x) = -sin(x)
    for j in range(0, 129):
        assert T[(128 - j) % 256] == T[j]       # sin(pi - x) = sin(x)
    # sin^2 + cos^2 = 1 within the rounding of both entries (each off by at most 1/2:
    # |2 a e_a + 2 b e_b| + 1/2 <= 127 sqrt(2) + 1/2)
    for j in range(256):
        assert abs(int(T[j]) ** 2 + int(T[(j + 64) % 256]) ** 2 - 127 ** 2) <= 180


def test_phi_phases_against_exact_fractions():
    """theta = floor(256 frac(2^k mu)), mu = (v + 1/2) / 2^D, and the linear part
    floor(128 mu), checked with exact rationals; C and numpy agree."""
    rng = np.random.default_rng(0)
    T = E.sin8_table()
    L = native.lib()
    s8 = T.astype(np.int8)
    for D in (1, 5, 10, 16, 21):
        v = rng.integers(0, 1 << D, size=(3, 40)).astype(np.int64)
        phi = E.phi_q(v, D)
        for i in range(v.shape[1]):
            for a in range(3):
                mu = Fraction(2 * int(v[a, i]) + 1, 2 ** (D + 1))
                assert phi[i, a] == math.floor(128 * mu)
                for k in range(E.BANDS):
                    fr = (2 ** k * mu) % 1
                    th = math.floor(256 * fr)
                    assert phi[i, 3 + 3 * k + a] == T[th]
                    assert phi[i, 3 + 3 * E.BANDS + 3 * k + a] == T[(th + 64) % 256]
            out = np.zeros(75, np.int32)
            vv = np.ascontiguousarray(v[:, i], np.uint32)
            L.or_pe_phi(native.ptr(vv), D, native.ptr(s8), native.ptr(out))
            assert np.array_equal(out, phi[i])


def _rand_params(rng, n):
    return rng.integers(0, 65281, n), rng.integers(2048, 5633, n)


def test_laplace_cdf_is_a_valid_coding_table():
    """cdf(0) = 0, cdf(256) = 2^16, every count >= 1, over the whole parameter range."""
    rng = np.random.default_rng(1)
    mu8, n = _rand_params(rng, 3000)
    mu8 = np.concatenate([mu8, [0, 65280, 32640, 0, 65280]])
    n = np.concatenate([n, [2048, 2048, 5632, 5632, 5632]])
    s = np.arange(257)
    cdf = E.pe_cdf(mu8[:, None], n[:, None], s[None, :])
    assert np.all(cdf[:, 0] == 0) and np.all(cdf[:, 256] == 65536)
    assert np.all(np.diff(cdf, axis=1) >= 1)


def test_laplace_cdf_tracks_the_closed_form():
    """Against the Laplace CDF F(x) = 2^(-r (m - x)) / 2 (x < m), 1 - 2^(-r (x - m)) / 2,
    at the mean m = mu8 / 256 and rate r = 2^(n/256 - 16): EXP2Q's 1/256 exponent steps
    bound the error by 2^(1/256) - 1 of F, about 90 counts; a wrong sign or offset costs
    thousands."""
    rng = np.random.default_rng(2)
    mu8, n = _rand_params(rng, 400)
    s = np.arange(1, 256)
    cdf = E.pe_cdf(mu8[:, None], n[:, None], s[None, :]).astype(np.float64)
    m = mu8[:, None] / 256.0
    r = 2.0 ** (n[:, None] / 256.0 - 16.0)
    x = s[None, :] - 0.5
    below = 0.5 * 2.0 ** (-r * np.maximum(m - x, 0.0))
    above = 1.0 - 0.5 * 2.0 ** (-r * np.maximum(x - m, 0.0))
    F = np.where(x < m, below, above)
    want = s[None, :] + 65280.0 * F
    assert np.max(np.abs(cdf - want)) < 100.0


def test_laplace_cdf_c_matches_numpy():
    rng = np.random.default_rng(3)
    L = native.lib()
    ex = np.array(exp2q_table(), np.uint32)
    mu8, n = _rand_params(rng, 50)
    for a, b in zip(mu8, n):
        for s in range(0, 257, 5):
            assert L.or_pe_cdf(int(a), int(b), s, native.ptr(ex)) == int(E.pe_cdf(a, b, s))


def test_float_head_is_a_distribution():
    """sum over s of p(s) = 1 for any head output, and the two tails absorb the mass beyond
    the token range."""
    rng = np.random.default_rng(4)
    for _ in range(50):
        z = rng.normal(0, 3, size=2)
        bits, _ = E._head(np.tile(z, (256, 1)), np.arange(256, dtype=np.float64))
        assert abs(np.sum(2.0 ** (-bits)) - 1.0) < 1e-12


def _toy(n=3000, seed=1, rho=0.8, lanes=8, depth=10):
    from paper_2607_12656_b300.scenegen import make_scene
    sc = make_scene(n, seed, rho)
    P = S.prepare(sc.pos, sc.attr, depth, 8)
    return sc, P, P.q.astype(np.uint8), S.lane_bounds(P.n_rows, lanes)


def test_fp64_gradients_match_central_differences():
    from paper_2607_12656_b300.scenegen import kaiming_init_pe
    _, P, q, lr = _toy()
    p = {k: np.asarray(v, np.float64) for k, v in kaiming_init_pe(3).items()}
    p["w3"] = p["w3"] * 10.0  # heads away from the initial point: means and rates spread
    phi_rows = E.phi_q(P.coord, 10)
    pos = M.sample_positions(9, 0, 64, q.shape[0] * 56)
    u, c, phi, s = E.batch(q, lr, phi_rows, pos)
    loss, g = E.forward_backward(p, u, c, phi, s)
    rng = np.random.default_rng(0)
    h = 1e-6
    for k in E.PARAMS:
        for _ in range(6):
            idx = tuple(rng.integers(0, d) for d in p[k].shape)
            if k == "emb":
                idx = (int(c[rng.integers(0, len(c))]), int(rng.integers(0, 16)))
            pp = {kk: vv.copy() for kk, vv in p.items()}
            pp[k][idx] += h
            lp = E.loss_only(pp, u, c, phi, s)
            pp[k][idx] -= 2 * h
            lm = E.loss_only(pp, u, c, phi, s)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k][idx]) <= 1e-5 * max(1.0, abs(fd)) + 1e-8, (k, idx, fd, g[k][idx])


def _random_model(seed):
    rng = np.random.default_rng(seed)
    return dict(w1=rng.integers(-127, 128, (64, 80)), b1=rng.integers(-(1 << 22), 1 << 22, (56, 64)),
                s1=np.float32(rng.uniform(1e-6, 1e-3)), w2=rng.integers(-127, 128, (64, 64)),
                b2=rng.integers(-(1 << 20), 1 << 20, 64), s2=np.float32(rng.uniform(1e-5, 1e-3)),
                w3=rng.integers(-127, 128, (2, 64)), b3=rng.integers(-(1 << 20), 1 << 20, 2),
                smu=np.float32(rng.uniform(1e-4, 0.1)), slr=np.float32(rng.uniform(1e-5, 0.01)))


def test_integer_head_brute_force_and_c_agree():
    """The vectorised integer forward, plain nested sums, and the C loop give the same head."""
    m = _random_model(5)
    rng = np.random.default_rng(6)
    u = rng.integers(-128, 128, (8, 4))
    c = rng.integers(0, 56, 8)
    phi = E.phi_q(rng.integers(0, 1 << 12, (3, 8)), 12)
    mu8, n = E.forward_int(m, u, c, phi)
    L = native.lib()
    ms = native.pe_model_struct(m)
    for i in range(8):
        x = list(u[i]) + list(phi[i]) + [0]
        h1 = []
        for o in range(64):
            acc = int(m["b1"][c[i], o]) + sum(int(m["w1"][o, k]) * int(x[k]) for k in range(80))
            h1.append(min(max(int(np.rint(np.float32(acc) * m["s1"])), 0), 127))
        h2 = []
        for o in range(64):
            acc = int(m["b2"][o]) + sum(int(m["w2"][o, k]) * h1[k] for k in range(64))
            h2.append(min(max(int(np.rint(np.float32(acc) * m["s2"])), 0), 127))
        z = [int(m["b3"][o]) + sum(int(m["w3"][o, k]) * h2[k] for k in range(64)) for o in range(2)]
        vm = min(max(float(np.rint(np.float32(z[0]) * m["smu"])), -32640.0), 32640.0)
        vl = min(max(float(np.rint(np.float32(z[1]) * m["slr"])), -2048.0), 1536.0)
        assert (mu8[i], n[i]) == (32640 + int(vm), 4096 + int(vl))
        a, b = ctypes.c_int32(), ctypes.c_int32()
        uu = np.ascontiguousarray(u[i], np.int32)
        pp = np.ascontiguousarray(phi[i], np.int32)
        L.or_pe_head(ctypes.byref(ms), native.ptr(uu), int(c[i]), native.ptr(pp), ctypes.byref(a), ctypes.byref(b))
        assert (a.value, b.value) == (mu8[i], n[i])


@pytest.mark.parametrize("seed", [0, 1])
def test_random_integer_models_round_trip(seed):
    """Arbitrary valid integer models (saturated activations, extreme means and rates)
    encode and decode losslessly; the decoder is the C loop, the encoder numpy."""
    _, P, q, _ = _toy(800, 7 + seed, lanes=3)
    m = _random_model(seed)
    buf = S.encode(None, None, mode=S.MODE_LEARNED_PE, depth=10, lanes=37, model=m, prep=P)
    d = S.decode(buf)
    assert np.array_equal(d["q"], P.q) and np.array_equal(d["attr"], P.attr)


@pytest.fixture(scope="module")
def trained_toy():
    from paper_2607_12656_b300.scenegen import kaiming_init_pe
    sc, P, q, lr = _toy(6000, 2, 0.8, 16)
    p, losses = E.train(kaiming_init_pe(1), q, lr, P.coord, 10, 150, 2048, seed=3, lr=3e-3)
    return sc, P, q, lr, p, losses


def test_training_reduces_code_length(trained_toy):
    *_, losses = trained_toy
    assert np.mean(losses[-10:]) < np.mean(losses[:5]) - 0.5


def test_freeze_integer_model_tracks_float(trained_toy):
    """Code length of the frozen integer model ~ the float model's."""
    sc, P, q, lr, p, _ = trained_toy
    m = E.freeze({k: v.astype(np.float32) for k, v in p.items()}, q, lr, P.coord, 10, seed=3)
    f, _ = E.token_fc(m, q, lr, P.coord, 10)
    int_bits = float(-np.log2(f / 65536.0).mean())
    pos = np.arange(q.shape[0] * 56)
    u, c, phi, s = E.batch(q, lr, E.phi_q(P.coord, 10), pos)
    float_bits = E.loss_only(p, u, c, phi, s)
    assert abs(int_bits - float_bits) < 0.15, (int_bits, float_bits)


def test_learned_pe_round_trip(trained_toy):
    sc, P, q, lr, p, _ = trained_toy
    m = E.freeze({k: v.astype(np.float32) for k, v in p.items()}, q, lr, P.coord, 10, seed=3)
    buf = S.encode(None, None, mode=S.MODE_LEARNED_PE, depth=10, lanes=16, model=m, prep=P)
    h = S.parse_header(buf)
    assert h["mode"] == S.MODE_LEARNED_PE and h["off_attr_grp"] - h["off_attr_tab"] == E.MODEL_PE_BYTES
    d = S.decode(buf)
    assert np.array_equal(d["q"], P.q) and np.array_equal(d["attr"], P.attr)
    assert np.array_equal(d["pos"], P.pos)
    # the model bytes survive a parse
    assert E.model_bytes(E.parse_model(buf, h["off_attr_tab"])) == E.model_bytes(m)


def test_sampled_decode_is_the_full_decode_on_its_groups(trained_toy):
    """decode(attr_groups=k) decodes the rows of the first k groups of 32 lanes exactly as the
    full decode does and leaves every other row 0."""
    sc, P, q, lr, p, _ = trained_toy
    m = E.freeze({k: v.astype(np.float32) for k, v in p.items()}, q, lr, P.coord, 10, seed=3)
    L = 70
    buf = S.encode(None, None, mode=S.MODE_LEARNED_PE, depth=10, lanes=L, model=m, prep=P)
    rows = S.lane_bounds(P.n_rows, L)
    for k in (0, 1, 3):
        d = S.decode(buf, attr_groups=k)
        cut = int(rows[min(L, 32 * k)])
        assert np.array_equal(d["q"][:cut], P.q[:cut]) and not d["q"][cut:].any()
