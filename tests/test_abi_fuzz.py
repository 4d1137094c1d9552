"""scene_query, the host-side parser of untrusted bitstreams, on seeded random corruptions of
valid bitstreams of every coding mode: each call either accepts the buffer or refuses it with
one of the library's error codes, and never crashes or reads outside the buffer (a crash fails
the whole run).  The encoder refuses non-finite inputs."""
import numpy as np
import pytest

from oracle import scene as S
from paper_2607_12656_b300 import sgs
from paper_2607_12656_b300.scenegen import fixed_bits, make_scene

CODES = {sgs.E_INVALID, sgs.E_CORRUPT, sgs.E_UNSUPPORTED}


def _random_model(seed):
    rng = np.random.default_rng(seed)
    return dict(w1=rng.integers(-127, 128, (64, 4)), b1=rng.integers(-3000, 3000, (56, 64)),
                w2=rng.integers(-127, 128, (64, 64)), b2=rng.integers(-20000, 20000, 64),
                w3=rng.integers(-127, 128, (256, 64)), b3=rng.integers(-(1 << 20), 1 << 20, 256),
                m1=int(rng.integers(1, 1 << 30)), sh1=28, m2=int(rng.integers(1, 1 << 30)), sh2=30,
                ms=int(rng.integers(1, 1 << 20)), ss=16)


@pytest.fixture(scope="module")
def streams():
    sc = make_scene(3000, 21)
    P8 = S.prepare(sc.pos, sc.attr, 12, 8)
    out = {
        "fixed": S.encode(sc.pos, sc.attr, mode=S.MODE_FIXED, depth=12, bits=fixed_bits(3), geo_mode=S.GEO_RAW),
        "static": S.encode(None, None, mode=S.MODE_STATIC, depth=12, lanes=40, prep=P8, geo_mode=S.GEO_RANS,
                           geo_lanes=64),
        "learned": S.encode(None, None, mode=S.MODE_LEARNED, depth=12, lanes=40, prep=P8, model=_random_model(1)),
    }
    for b in out.values():
        sgs.scene_query(b)  # the unmodified streams are accepted
    return out


@pytest.mark.parametrize("name", ["fixed", "static", "learned"])
def test_corrupted_headers_and_tables(streams, name):
    buf = streams[name]
    rng = np.random.default_rng({"fixed": 1, "static": 2, "learned": 3}[name])
    head = min(len(buf), 4096)
    accepted = refused = 0
    for trial in range(3000):
        b = bytearray(buf)
        kind = trial % 4
        if kind == 0:    # one random byte in the header
            b[int(rng.integers(0, 256))] = int(rng.integers(0, 256))
        elif kind == 1:  # a random 32-bit word in the header: counts, offsets, lanes
            o = 4 * int(rng.integers(0, 64))
            b[o:o + 4] = int(rng.integers(0, 1 << 32)).to_bytes(4, "little")
        elif kind == 2:  # a few bytes anywhere in the first 4 KB (levels, tables, group table)
            for o in rng.integers(0, head, size=4):
                b[int(o)] ^= 1 << int(rng.integers(0, 8))
        else:            # truncated or extended
            cut = int(rng.integers(0, len(buf) + 64))
            b = b[:cut] if cut <= len(buf) else b + bytes(cut - len(buf))
        try:
            info = sgs.scene_query(bytes(b))
            accepted += 1
            # an accepted buffer's sections lie inside it, in order, 16-byte aligned, and its
            # tables inside their sections: the device decode relies on these
            off = [int(x) for x in info.off]
            assert info.total_len == len(b) and off[10] == len(b)
            assert all(0 <= x <= y for x, y in zip(off, off[1:])) and all(x % 16 == 0 for x in off)
            assert all(off[4] <= int(info.table_off[t]) < off[10] for t in range(info.n_tables))
        except sgs.SgsError as e:
            refused += 1
            assert e.code in CODES, e.code
    assert refused > 1000  # most corruptions of the header are caught before any decode


def test_encoder_refuses_non_finite_inputs():
    sc = make_scene(500, 3)
    for bad in (np.nan, np.inf, -np.inf):
        attr = sc.attr.copy()
        attr[7, 11] = bad
        with pytest.raises(sgs.SgsError) as e:
            sgs.scene_encode(sc.pos, attr, mode=sgs.MODE_STATIC, depth=10, lanes=8)
        assert e.value.code == sgs.E_INVALID
    pos = sc.pos.copy()
    pos[1, 3] = np.nan
    with pytest.raises(sgs.SgsError):
        sgs.scene_encode(pos, sc.attr, mode=sgs.MODE_FIXED, depth=10, bits=8)
