"""Host-side checks of the C-ABI library (no GPU needed): every declared symbol is exported,
the library's encoder emits the oracle's bytes, scene_query agrees with the oracle's header
parse and rejects malformed headers."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import scene as S
from paper_2607_12656_b300 import sgs
from paper_2607_12656_b300.scenegen import fixed_bits, make_scene

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = sgs.lib()
    names = _declared_functions()
    assert "scene_decode" in names and "scene_encode" in names and len(names) >= 12
    for n in names:
        assert hasattr(L, n), n
        assert ctypes.cast(getattr(L, n), ctypes.c_void_p).value


CASES = [(0, 3, 8), (1, 1, 8), (5, 2, 8), (33, 4, 8), (1500, 7, 8), (6000, 12, 8)]


@pytest.mark.parametrize("n,depth,lanes", CASES)
@pytest.mark.parametrize("mode", [S.MODE_FIXED, S.MODE_STATIC])
@pytest.mark.parametrize("geo", [S.GEO_RAW, S.GEO_RANS])
def test_encoder_bytes_match_oracle(n, depth, lanes, mode, geo):
    sc = make_scene(n, 7 + n)
    bits = fixed_bits(n) if mode == S.MODE_FIXED else 8
    want = S.encode(sc.pos, sc.attr, mode=mode, depth=depth, bits=bits, lanes=lanes + 25, geo_mode=geo)
    got = sgs.scene_encode(sc.pos, sc.attr, mode=mode, depth=depth, bits=bits, lanes=lanes + 25, geo_mode=geo)
    assert got == want


def test_encoder_bytes_match_oracle_geometry_coded(small_scene):
    for geo_lanes in (0, 33, 96):
        want = S.encode(small_scene.pos, small_scene.attr, mode=S.MODE_STATIC, depth=12, lanes=32,
                        geo_mode=S.GEO_RANS, geo_lanes=geo_lanes)
        got = sgs.scene_encode(small_scene.pos, small_scene.attr, mode=sgs.MODE_STATIC, depth=12, lanes=32,
                               geo_mode=sgs.GEO_RANS, geo_lanes=geo_lanes)
        assert got == want


def test_tokens_match_oracle(small_scene):
    P = S.prepare(small_scene.pos, small_scene.attr, 12, 8)
    assert np.array_equal(sgs.scene_tokens(small_scene.pos, small_scene.attr, 12), P.q.astype(np.uint8))


def test_query_matches_oracle_header(small_scene):
    buf = S.encode(small_scene.pos, small_scene.attr, mode=S.MODE_STATIC, depth=12, lanes=32)
    h = S.parse_header(buf)
    info = sgs.scene_query(buf)
    for k in ("mode", "geo_mode", "n_rows", "depth", "n_leaves", "n_dup", "lanes", "geo_lanes", "n_geo",
              "n_geo_coded"):
        assert getattr(info, k) == h[k], k
    assert info.total_len == len(buf) and info.scratch_bytes > 0
    P = S.prepare(small_scene.pos, small_scene.attr, 12, 8)
    assert [info.n_level[l] for l in range(12)] == [len(b) for b in P.levels]


def test_query_rejects_malformed(small_scene):
    buf = bytearray(S.encode(small_scene.pos, small_scene.attr, mode=S.MODE_FIXED, depth=12,
                             bits=fixed_bits(1)))
    for off, val in [(0, 0), (4, 9), (8, 7), (24, 0), (24, 40), (36, 55), (64, 255)]:
        b = bytearray(buf)
        b[off:off + 4] = int(val).to_bytes(4, "little")
        with pytest.raises(sgs.SgsError):
            sgs.scene_query(bytes(b))
    with pytest.raises(sgs.SgsError):
        sgs.scene_query(bytes(buf[:-16]))  # total length mismatch
    with pytest.raises(sgs.SgsError):
        sgs.scene_query(bytes(buf[:100]))


def test_library_exp2q_table_matches_oracle():
    from oracle.exp2q import exp2q_table
    text = open(os.path.join(ROOT, "paper_2607_12656_b300", "csrc", "exp2q_table.h")).read()
    vals = [int(v) for v in re.findall(r"(\d+)u", text)]
    assert vals == list(exp2q_table())


def test_freeze_matches_oracle(small_scene):
    """Given the same fp32 weights and tokens, the library's freeze emits the oracle's model."""
    from oracle import model as M
    from paper_2607_12656_b300.scenegen import kaiming_init
    P = S.prepare(small_scene.pos, small_scene.attr, 12, 8)
    q = P.q.astype(np.uint8)
    for lanes, seed, wseed in ((32, 3, 1), (7, 11, 2), (4096, 5, 3)):
        w = kaiming_init(wseed)
        rng = np.random.default_rng(wseed)
        w = {k: (v + 0.05 * rng.standard_normal(v.shape)).astype(np.float32) for k, v in w.items()}
        want = S.model_bytes(M.freeze(w, q, S.lane_bounds(P.n_rows, lanes), seed))
        got = sgs.sgs_freeze(sgs.pack_weights(w), q, lanes, seed)
        assert got == want


def test_scene_rows_match_oracle(small_scene):
    """Tokens and voxel coordinates of the rows, as the oracle prepares them."""
    P = S.prepare(small_scene.pos, small_scene.attr, 12, 8)
    tok, crd = sgs.scene_rows(small_scene.pos, small_scene.attr, 12)
    assert np.array_equal(tok, P.q.astype(np.uint8)) and np.array_equal(crd, P.coord)


def test_freeze_pe_matches_oracle(small_scene):
    """Given the same fp32 weights, rows and voxels, the library's freeze of the
    position-aware model emits the oracle's model byte for byte."""
    from oracle import model_pe as E
    from paper_2607_12656_b300.scenegen import kaiming_init_pe
    for depth, lanes, seed, wseed in ((12, 32, 3, 1), (9, 7, 11, 2), (16, 4096, 5, 3)):
        P = S.prepare(small_scene.pos, small_scene.attr, depth, 8)
        q = P.q.astype(np.uint8)
        w = kaiming_init_pe(wseed)
        rng = np.random.default_rng(wseed)
        w = {k: (v + 0.05 * rng.standard_normal(v.shape)).astype(np.float32) for k, v in w.items()}
        want = E.model_bytes(E.freeze(w, q, S.lane_bounds(P.n_rows, lanes), P.coord, depth, seed))
        got = sgs.sgs_freeze_pe(sgs.pack_weights_pe(w), q, P.coord, depth, lanes, seed)
        assert got == want


def test_batch_bytes_host_side(small_scene):
    """scene_batch_bytes lays a batch out on the host only: it covers every scene's scratch,
    grows with the batch, and refuses infos that scene_query did not produce or misaligned
    bitstreams (the pointers are never dereferenced here)."""
    bufs = [S.encode(small_scene.pos, small_scene.attr, mode=m, depth=12, lanes=64, bits=8)
            for m in (S.MODE_FIXED, S.MODE_STATIC)]
    infos = [sgs.scene_query(b) for b in bufs]
    fake = 1 << 24  # 16-byte aligned stand-ins for device addresses

    def items(k):
        return [(fake, infos[j % 2], fake, fake) for j in range(k)]

    one, four = sgs.scene_batch_bytes(items(1)), sgs.scene_batch_bytes(items(4))
    assert one >= (infos[0].scratch_bytes + 255) // 256 * 256
    assert four > 2 * one
    assert sgs.scene_batch_bytes([]) >= 0
    bad = sgs.SceneInfo.from_buffer_copy(infos[0])
    bad.scratch_bytes += 16
    with pytest.raises(sgs.SgsError) as e:
        sgs.scene_batch_bytes([(fake, bad, fake, fake)])
    assert e.value.code == sgs.E_INVALID
    with pytest.raises(sgs.SgsError) as e:
        sgs.scene_batch_bytes([(fake + 8, infos[0], fake, fake)])
    assert e.value.code == sgs.E_INVALID


def test_look_at_camera():
    """The binding's camera: an orthonormal world-to-camera rotation whose z axis points at
    the target, which projects to the image centre; the focal length gives the field of view."""
    import math
    cam = sgs.look_at([0.2, -0.4, -1.0], [0.5, 0.5, 0.5], [0, -1, 0], 640, 480, 60.0)
    R = np.array(cam.rot[:], np.float64).reshape(3, 3)
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-6)
    t = R @ (np.array([0.5, 0.5, 0.5]) - np.array(cam.origin[:]))
    assert abs(t[0]) < 1e-5 and abs(t[1]) < 1e-5 and t[2] > 0
    assert abs(cam.fy - 240.0 / math.tan(math.radians(30.0))) < 1e-3 and cam.cx == 320.0 and cam.cy == 240.0
