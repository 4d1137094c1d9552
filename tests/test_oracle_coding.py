"""Pins of the oracle's quantizer and coders: closed forms, hand-worked examples, code-length
bounds, brute force, round trips."""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import scene as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- quantizer

def test_quantize_hand_example_ties_to_even():
    v = np.array([0.0, 0.5, 1.5, 2.5, 3.0], np.float32)
    q, step, off = S.quantize(v, 2)
    assert step == np.float32(1.0) and off == np.float32(0.0)
    assert q.tolist() == [0, 0, 2, 2, 3]
    assert S.dequantize(q, step, off).tolist() == [0.0, 0.0, 2.0, 2.0, 3.0]


@pytest.mark.parametrize("bits", [4, 7, 8, 10])
def test_quantize_error_bound(bits):
    rng = np.random.default_rng(bits)
    v = (rng.standard_normal(10000) * 3 + 1).astype(np.float32)
    q, step, off = S.quantize(v, bits)
    r = S.dequantize(q, step, off)
    err = np.abs(r.astype(np.float64) - v.astype(np.float64))
    ulp = np.spacing(np.maximum(np.abs(v), np.abs(r))).astype(np.float64)
    assert np.all(err <= float(step) / 2 + 2 * ulp)
    assert q.max() <= (1 << bits) - 1 and q.min() == 0 and q.max() == (1 << bits) - 1
    assert r.min() >= v.min() - np.spacing(abs(v.min())) and r.max() <= v.max() + 2 * np.spacing(abs(v.max()))


def test_quantize_constant_channel():
    v = np.full(7, -2.25, np.float32)
    q, step, off = S.quantize(v, 8)
    assert step == 0 and np.all(q == 0) and np.all(S.dequantize(q, step, off) == v)


@pytest.mark.parametrize("first", [0.0, -0.0])
def test_quantize_zero_extremum_keeps_the_first_sign(first):
    """-0.0 and +0.0 tie as the minimum (and as the maximum): the offset, whose bits the bitstream
    stores, is the first one in row order.  Long vectors, so that a SIMD reduction order would
    show."""
    second = -first
    lo = np.full(4099, 3.0, np.float32)
    lo[[17, 700, 2048, 4098]] = [first, second, first, second]
    q, step, off = S.quantize(lo, 8)
    assert math.copysign(1.0, off) == math.copysign(1.0, first)
    assert q[17] == 0 and q[0] == 255
    hi = np.full(4099, -3.0, np.float32)
    hi[[5, 3000]] = [first, second]
    _, step, off = S.quantize(hi, 8)
    assert off == np.float32(-3.0) and step == np.float32(3.0 / 255)


def test_dequantize_two_roundings_not_fused():
    # q * step rounds to fp32 before the add: choose values where a fused form differs
    step, off = np.float32(0.1), np.float32(-0.30000001)
    q = np.arange(256, dtype=np.uint32)
    want = np.array([np.float32(np.float32(np.float32(i) * step) + off) for i in range(256)], np.float32)
    assert np.array_equal(S.dequantize(q, step, off), want)
    fused = (q.astype(np.float64) * np.float64(step) + np.float64(off)).astype(np.float32)
    assert not np.array_equal(fused, want)


# --------------------------------------------------------------------------- tables

def test_normalize_freq_properties():
    rng = np.random.default_rng(0)
    for trial in range(200):
        h = rng.integers(0, 1000, 256) * (rng.random(256) < rng.random())
        if h.sum() == 0:
            h[3] = 1
        f = S.normalize_freq(h)
        assert int(f.sum()) == 65536
        assert np.all((f > 0) == (h > 0))
    f = S.normalize_freq(np.eye(256, dtype=np.int64)[17] * 9)
    assert f[17] == 65536 and f.sum() == 65536
    # remainder to the most frequent symbol, lowest index on ties
    h = np.zeros(256, np.int64); h[[5, 9]] = 3
    f = S.normalize_freq(h)
    assert f[5] == 32768 and f[9] == 32768 - 0 or f[5] >= f[9]


def test_table_bytes_round_trip():
    rng = np.random.default_rng(2)
    h = rng.integers(0, 50, 256) * (rng.random(256) < 0.6)
    h[0] = 1
    f = S.normalize_freq(h)
    buf = S.table_bytes(f)
    assert len(buf) % 16 == 0
    tabs, end = S.parse_tables(buf, 0, 1)
    assert np.array_equal(tabs[0], f) and end == len(buf)


# --------------------------------------------------------------------------- rANS

def _golden_rans():
    cases = []
    for line in open(os.path.join(GOLD, "rans_single_lane.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        name, freq, syms, words = [t.strip() for t in line.split("|")]
        f = np.zeros(256, np.uint32)
        for kv in freq.split(","):
            k, v = kv.split(":")
            f[int(k)] = int(v)
        cases.append((name, f, [int(t) for t in syms.split()], [int(w, 16) for w in words.split()]))
    return cases


@pytest.mark.parametrize("case", _golden_rans(), ids=lambda c: c[0])
def test_rans_golden(case):
    _, f, syms, words = case
    cum = S.cum_of(f)
    s = np.array(syms)
    pay, goff, gw = S.rans_encode(np.array([0, len(s)]), f[s], cum[s])
    got = np.frombuffer(pay, "<u2")[: int(gw[0])].tolist()
    assert got == words
    assert len(pay) % 16 == 0 and set(pay[2 * int(gw[0]):]) <= {0}
    dec = S.rans_decode_static(np.array([0, len(s)]), np.zeros(len(s), np.uint8), [f], pay, goff, gw)
    assert dec.tolist() == syms


def _random_tables(rng, n):
    return [S.normalize_freq(rng.integers(0, 100, 256) ** 2 * (rng.random(256) < 0.7) + (np.arange(256) == 0))
            for _ in range(n)]


@pytest.mark.parametrize("lanes", [1, 2, 31, 32, 33, 100])
def test_rans_round_trip_uneven_lanes_and_bound(lanes):
    rng = np.random.default_rng(lanes)
    tabs = _random_tables(rng, 5)
    counts = rng.integers(0, 300, lanes)
    counts[0] = 0 if lanes > 3 else counts[0]
    ls = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    n = int(ls[-1])
    tab_id = rng.integers(0, 5, n).astype(np.uint8)
    syms = np.empty(n, np.uint8)
    for i in range(n):  # draw each symbol from its own table's distribution
        f = tabs[tab_id[i]]
        syms[i] = rng.choice(256, p=f / 65536.0)
    f, c = S.static_fc(syms, tab_id, tabs)
    pay, goff, gw = S.rans_encode(ls, f, c)
    assert np.array_equal(S.rans_decode_static(ls, tab_id, tabs, pay, goff, gw), syms)
    ideal_bits = float(-np.log2(f / 65536.0).sum())
    assert 2 * int(gw.sum()) <= 1.005 * ideal_bits / 8 + 64 * lanes


def test_rans_uniform_closed_form():
    """f = 256 for every symbol: one word every second symbol, plus the 4-byte final state."""
    rng = np.random.default_rng(7)
    for n in range(0, 40):
        s = rng.integers(0, 256, n)
        pay, goff, gw = S.rans_encode(np.array([0, n]), np.full(n, 256, np.uint32), (s * 256).astype(np.uint32))
        assert 2 * int(gw[0]) == 2 * (n // 2) + 4


def test_rans_certain_symbol_costs_nothing():
    n = 1000
    pay, goff, gw = S.rans_encode(np.array([0, n]), np.full(n, 65536, np.uint32), np.zeros(n, np.uint32))
    assert int(gw[0]) == 2


def test_rans_brute_force_injective():
    """All 4^8 sequences over a 4-symbol table round-trip and give distinct streams."""
    f = np.zeros(256, np.uint32)
    f[:4] = [30000, 20000, 10000, 5536]
    cum = S.cum_of(f)
    seen = set()
    for seq in itertools.product(range(4), repeat=8):
        s = np.array(seq)
        pay, goff, gw = S.rans_encode(np.array([0, 8]), f[s], cum[s])
        assert S.rans_decode_static(np.array([0, 8]), np.zeros(8, np.uint8), [f], pay, goff, gw).tolist() == list(seq)
        seen.add(pay[: 2 * int(gw[0])])
    assert len(seen) == 4 ** 8


def test_rans_corruption_detected_or_differs():
    rng = np.random.default_rng(11)
    tabs = _random_tables(rng, 1)
    ls = np.array([0, 500, 1000, 1400], np.int64)
    syms = rng.choice(256, 1400, p=tabs[0] / 65536.0).astype(np.uint8)
    tid = np.zeros(1400, np.uint8)
    f, c = S.static_fc(syms, tid, tabs)
    pay, goff, gw = S.rans_encode(ls, f, c)
    flagged = 0
    for trial in range(60):
        b = bytearray(pay)
        k = int(rng.integers(0, 2 * int(gw[0])))
        b[k] ^= 1 << int(rng.integers(0, 8))
        try:
            out = S.rans_decode_static(ls, tid, tabs, bytes(b), goff, gw)
            assert not np.array_equal(out, syms)
        except ValueError:
            flagged += 1
    assert flagged > 30


# --------------------------------------------------------------------------- fixed length

@pytest.mark.parametrize("b", [1, 4, 5, 7, 10, 16, 31])
def test_fixed_pack_layout(b):
    rng = np.random.default_rng(b)
    n = 101
    q = rng.integers(0, 1 << b, n).astype(np.uint32)
    buf = S.pack_fixed(q, b)
    assert len(buf) % 16 == 0 and len(buf) >= 4 * ((n * b + 31) // 32)
    words = np.frombuffer(buf, "<u4")
    big = sum(int(w) << (32 * i) for i, w in enumerate(words))  # LSB-first bit stream
    for i in range(n):
        assert (big >> (i * b)) & ((1 << b) - 1) == q[i]
    assert np.array_equal(S.unpack_fixed(buf, 0, n, b), q)


# --------------------------------------------------------------------------- whole scene

@pytest.mark.parametrize("n,depth", [(0, 3), (1, 1), (2, 5), (7, 2), (8, 3), (33, 4), (1000, 12), (4000, 6)])
@pytest.mark.parametrize("mode", [S.MODE_FIXED, S.MODE_STATIC])
def test_scene_round_trip(n, depth, mode):
    from paper_2607_12656_b300.scenegen import make_scene, fixed_bits
    sc = make_scene(n, 100 + n)
    bits = fixed_bits(n) if mode == S.MODE_FIXED else 8
    P = S.prepare(sc.pos, sc.attr, depth, bits)
    for geo in (S.GEO_RAW, S.GEO_RANS):
        buf = S.encode(sc.pos, sc.attr, mode=mode, depth=depth, bits=bits, lanes=33, geo_mode=geo, prep=P)
        d = S.decode(buf)
        assert np.array_equal(d["attr"], P.attr)
        assert np.array_equal(d["pos"], P.pos)
        assert np.array_equal(d["q"], P.q)


def test_scene_geometry_rans_levels(small_scene):
    P = S.prepare(small_scene.pos, small_scene.attr, 12, 8)
    buf = S.encode(None, None, mode=S.MODE_STATIC, depth=12, lanes=32, prep=P)
    h = S.parse_header(buf)
    coded = [len(b) for b in P.levels if len(b) >= S.GEO_RANS_MIN_LEVEL]
    assert h["n_geo_coded"] == sum(coded) > 0
    d = S.decode(buf)
    assert np.array_equal(d["attr"], P.attr) and np.array_equal(d["pos"], P.pos)
