"""CPU oracle for scene encode/decode.  TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use this
package; the library (``paper_2607_12656_b300``) never imports it and it imports nothing from
the library.  Plain numpy (fp64 where the method computes in floating point) plus the C loops
of ``oracle.c``.  Each step cites the passage of the paper it follows.

Steps (the decoded values are fixed by steps 1-5 alone: the coders change only the bytes):
  1. prune: drop floor(N/10) Gaussians of lowest opacity (stand-in for the learned masks of
     Sec. 3.3; ties drop the lower original index first);
  2. voxelize to a depth-D grid and sort by (Morton code, original index) (Sec. 3.4,
     "Autoregressive Attribute Coding": Morton ordering gives the 1D token sequence);
  3. serialize the sparse octree level by level as 8-bit occupancy tokens (Sec. 3.4,
     "Geometry Occupancy Coding"), one position per voxel plus duplicate counts as metadata;
  4. per-channel uniform quantization (Sec. 3.3 learned steps, replaced by min/max steps at a
     given bit width; Sec. 3.4.1 fixed-length precision per channel);
  5. dequantize: v' = fl32(fl32(q * step) + offset), two roundings, no fused multiply-add;
  6. code the tokens: channel-wise fixed-length (Sec. 3.4.1, "UltraFast"), channel-wise
     static-frequency rANS, or rANS driven by the learned local autoregressive model
     (Sec. 3.4.2, groups of W Gaussians decoded in parallel = rANS lanes), either the plain
     model (softmax over 256 symbols) or the position-aware one (Fourier positional
     embedding of the decoded voxel and a Laplace head, oracle/model_pe.py).
"""
from __future__ import annotations

import struct
from dataclasses import dataclass, field

import numpy as np

from . import model_pe, native
from .exp2q import exp2q_table

MAGIC = 0x31534753  # "SGS1"
VERSION = 1
MODE_FIXED, MODE_STATIC, MODE_LEARNED, MODE_LEARNED_PE = 0, 1, 2, 3
GEO_RAW, GEO_RANS, GEO_LEARNED = 0, 1, 2
NCHAN = 56
NSYM = 256
GEO_RANS_MIN_LEVEL = 4096   # octree levels with fewer nodes are stored raw
PROB_BITS = 16
HEADER_BYTES = 256
MODEL_BYTES = 36384


def _align16(n: int) -> int:
    return (n + 15) & ~15


# ----------------------------------------------------------------------------- steps 1-3

def prune(attr: np.ndarray) -> np.ndarray:
    """Indices (ascending) kept after dropping floor(N/10) of lowest opacity (channel 48)."""
    n = attr.shape[1]
    k = n // 10
    order = np.lexsort((np.arange(n), attr[48]))  # opacity, then index
    return np.sort(order[k:])


def voxelize(pos: np.ndarray, depth: int) -> np.ndarray:
    """v = min(floor(p * 2^D), 2^D - 1) per axis -> uint32 [3, n]."""
    v = np.floor(pos.astype(np.float64) * float(1 << depth))
    v = np.minimum(v, float((1 << depth) - 1))
    return v.astype(np.uint32)


def morton(coord: np.ndarray, depth: int) -> np.ndarray:
    """Interleave the bits of (x, y, z), x most significant within each 3-bit digit."""
    x, y, z = (coord[k].astype(np.uint64) for k in range(3))
    m = np.zeros(coord.shape[1], dtype=np.uint64)
    for b in range(depth):
        bb = np.uint64(b)
        m |= ((x >> bb) & np.uint64(1)) << np.uint64(3 * b + 2)
        m |= ((y >> bb) & np.uint64(1)) << np.uint64(3 * b + 1)
        m |= ((z >> bb) & np.uint64(1)) << np.uint64(3 * b)
    return m


def demorton(m: np.ndarray, depth: int) -> np.ndarray:
    coord = np.zeros((3, m.shape[0]), dtype=np.uint64)
    for b in range(depth):
        for k in range(3):
            coord[k] |= ((m >> np.uint64(3 * b + 2 - k)) & np.uint64(1)) << np.uint64(b)
    return coord.astype(np.uint32)


def octree_levels(leaf_codes: np.ndarray, depth: int) -> list[np.ndarray]:
    """Occupancy bytes per level 0..D-1 from sorted unique leaf Morton codes.  A node's byte
    has bit k set iff its child k = (bx<<2 | by<<1 | bz) is occupied; nodes of each level in
    increasing Morton order (breadth-first, children in increasing k)."""
    levels = []
    for l in range(depth):
        node = leaf_codes >> np.uint64(3 * (depth - l))
        child = (leaf_codes >> np.uint64(3 * (depth - l - 1))) & np.uint64(7)
        uniq, inv = np.unique(node, return_inverse=True)
        b = np.zeros(len(uniq), dtype=np.uint8)
        np.bitwise_or.at(b, inv, (np.uint8(1) << child.astype(np.uint8)))
        levels.append(b)
    return levels


def octree_expand(levels: list[np.ndarray], depth: int) -> np.ndarray:
    """Inverse of octree_levels: leaf Morton codes in order.  Raises on inconsistent counts."""
    codes = np.zeros(1, dtype=np.uint64) if depth > 0 else np.zeros(0, np.uint64)
    if len(levels) == 0 or len(levels[0]) == 0:
        return np.zeros(0, dtype=np.uint64)
    for l in range(depth):
        b = levels[l]
        if len(b) != len(codes):
            raise ValueError("corrupt octree: level %d has %d bytes for %d nodes" % (l, len(b), len(codes)))
        bits = np.unpackbits(b[:, None], axis=1, bitorder="little")
        node, k = np.nonzero(bits)
        codes = (codes[node] << np.uint64(3)) | k.astype(np.uint64)
    return codes


def position(coord: np.ndarray, depth: int) -> np.ndarray:
    """pos = coord * 2^-D + 2^-(D+1) (voxel centre; exact in fp32 for D <= 23)."""
    c = coord.astype(np.float32)
    return (c * np.float32(2.0 ** -depth) + np.float32(2.0 ** -(depth + 1))).astype(np.float32)


# ----------------------------------------------------------------------------- steps 4-5

def quantize(v: np.ndarray, bits: int):
    """Per-channel uniform quantizer: offset = min, step = fl32((max - min) / (2^b - 1)),
    q = clamp(rint((v - offset) / step), 0, 2^b - 1) in fp64 (ties to even); step 0 -> q 0.
    The minimum and maximum are the first values in row order that attain them, so a zero
    extremum keeps the sign of its first occurrence (-0.0 and +0.0 compare equal)."""
    if v.size == 0:
        return np.zeros(0, np.uint32), np.float32(0), np.float32(0)
    mn, mx = v[np.argmin(v)], v[np.argmax(v)]
    top = (1 << bits) - 1
    step = np.float32(0.0) if mx == mn else np.float32((np.float64(mx) - np.float64(mn)) / top)
    offset = np.float32(mn)
    if step == 0:
        return np.zeros(v.shape, np.uint32), step, offset
    q = np.rint((v.astype(np.float64) - np.float64(offset)) / np.float64(step))
    q = np.clip(q, 0, top).astype(np.uint32)
    return q, step, offset


def dequantize(q: np.ndarray, step, offset) -> np.ndarray:
    """v' = fl32(fl32(q * step) + offset): two separate fp32 roundings."""
    prod = (q.astype(np.float32) * np.float32(step)).astype(np.float32)
    return (prod + np.float32(offset)).astype(np.float32)


# ----------------------------------------------------------------------------- tables

def normalize_freq(hist: np.ndarray) -> np.ndarray:
    """Static 16-bit table: f_s = 1 + floor(h_s (2^16 - K) / sum h) for h_s > 0 (K symbols
    present), else 0; the remainder goes to the most frequent symbol (lowest s on ties)."""
    h = hist.astype(np.int64)
    tot = int(h.sum())
    f = np.zeros(NSYM, dtype=np.uint32)
    if tot == 0:
        return f
    K = int((h > 0).sum())
    present = h > 0
    f[present] = (1 + (h[present] * ((1 << PROB_BITS) - K)) // tot).astype(np.uint32)
    f[int(np.argmax(h))] += np.uint32((1 << PROB_BITS) - int(f.sum()))
    return f


def cum_of(f: np.ndarray) -> np.ndarray:
    c = np.zeros(NSYM, dtype=np.uint32)
    c[1:] = np.cumsum(f[:-1], dtype=np.uint64).astype(np.uint32)
    return c


def table_bytes(f: np.ndarray) -> bytes:
    """32-byte presence mask, then (f - 1) as uint16 for present symbols in order, padded."""
    mask = np.packbits((f > 0).astype(np.uint8), bitorder="little").tobytes()
    body = (f[f > 0].astype(np.int64) - 1).astype("<u2").tobytes()
    raw = mask + body
    return raw + b"\0" * (_align16(len(raw)) - len(raw))


def parse_tables(buf: bytes, off: int, count: int):
    tabs = []
    for _ in range(count):
        mask = np.unpackbits(np.frombuffer(buf, np.uint8, 32, off), bitorder="little").astype(bool)
        k = int(mask.sum())
        body = np.frombuffer(buf, "<u2", k, off + 32).astype(np.uint32) + 1
        f = np.zeros(NSYM, np.uint32)
        f[mask] = body
        if int(f.sum(dtype=np.uint64)) not in (0, 1 << PROB_BITS):  # 0: channel of an empty scene
            raise ValueError("corrupt table")
        tabs.append(f)
        off += _align16(32 + 2 * k)
    return tabs, off


# ----------------------------------------------------------------------------- lanes + rANS

def lane_bounds(n: int, lanes: int) -> np.ndarray:
    """Lane j owns items [floor(j n / L), floor((j+1) n / L)) (groups of W, Sec. 3.4.2)."""
    j = np.arange(lanes + 1, dtype=np.int64)
    return (j * n) // lanes


def static_row_order(n: int, lanes: int) -> tuple[np.ndarray, np.ndarray]:
    """Item order of static-table coding (attribute rows, or octree tokens) and its lane
    boundaries.

    Group g of 32 lanes owns the items that its lanes would own as contiguous chunks
    (items [floor(32 g n / L), floor(min(32 g + 32, L) n / L))), and deals them round robin to
    its n_g lanes: lane j of the group codes items R_g + j, R_g + j + n_g, ...  Static coding
    has no context between items, so this changes no code length; it only makes the 32 lanes
    of a group hold 32 consecutive items at every step.  Returns (perm, lane_start): the items
    in lane-major coding order and the offsets of each lane's items in perm."""
    perm = np.empty(n, np.int64)
    lane_start = np.zeros(lanes + 1, np.int64)
    lb = lane_bounds(n, lanes)
    pos = 0
    for g in range((lanes + 31) // 32):
        j0, j1 = 32 * g, min(lanes, 32 * g + 32)
        nl = j1 - j0
        R0, R1 = int(lb[j0]), int(lb[j1])
        for jj in range(nl):
            rows = np.arange(R0 + jj, R1, nl, dtype=np.int64)
            perm[pos:pos + len(rows)] = rows
            pos += len(rows)
            lane_start[j0 + jj + 1] = pos
    return perm, lane_start


def rans_encode(lane_start: np.ndarray, f: np.ndarray, c: np.ndarray, lane_lo: int = 0,
                lane_hi: int | None = None):
    """Interleaved rANS of lanes [lane_lo, lane_hi); f, c indexed by absolute position."""
    L = native.lib()
    n_lanes = len(lane_start) - 1
    if lane_hi is None:
        lane_hi = n_lanes
    G = (lane_hi - lane_lo + 31) // 32
    ls = np.ascontiguousarray(lane_start, dtype=np.int64)
    f = np.ascontiguousarray(f, dtype=np.uint32)
    c = np.ascontiguousarray(c, dtype=np.uint32)
    nsym = int(ls[lane_hi] - ls[lane_lo])
    cap = 2 * nsym + 160 * G + 64
    out = np.zeros(cap, np.uint8)
    goff = np.zeros(G + 1, np.uint64)
    gw = np.zeros(max(G, 1), np.uint32)
    n = L.or_rans_encode(lane_lo, lane_hi, native.ptr(ls), native.ptr(f), native.ptr(c),
                         native.ptr(out), cap, native.ptr(goff), native.ptr(gw))
    if n < 0:
        raise RuntimeError("rans encode failed (%d)" % n)
    return out[:n].tobytes(), goff, gw[:G]


def rans_decode_static(lane_start, tab_id, tables, payload, goff, gw) -> np.ndarray:
    L = native.lib()
    ls = np.ascontiguousarray(lane_start, dtype=np.int64)
    nsym = int(ls[-1])
    syms = np.zeros(max(nsym, 1), np.uint8)
    freq = np.ascontiguousarray(np.stack(tables) if len(tables) else np.zeros((1, NSYM)), dtype=np.uint32)
    pay = np.frombuffer(payload, np.uint8).copy() if len(payload) else np.zeros(1, np.uint8)
    tid = np.ascontiguousarray(tab_id, dtype=np.uint8) if nsym else np.zeros(1, np.uint8)
    go = np.ascontiguousarray(goff, np.uint64)
    gwa = np.ascontiguousarray(gw if len(gw) else np.zeros(1), np.uint32)
    rc = L.or_rans_decode_static(len(ls) - 1, native.ptr(ls), native.ptr(tid), native.ptr(freq),
                                 len(tables), native.ptr(pay), len(payload), native.ptr(go),
                                 native.ptr(gwa), native.ptr(syms))
    if rc != 0:
        raise ValueError("corrupt rANS stream")
    return syms[:nsym]


def rans_decode_static16(lane_start, tab_id, tables, payload, goff, gw) -> np.ndarray:
    """As rans_decode_static with up to 65,535 tables (16-bit table ids)."""
    L = native.lib()
    ls = np.ascontiguousarray(lane_start, dtype=np.int64)
    nsym = int(ls[-1])
    syms = np.zeros(max(nsym, 1), np.uint8)
    freq = np.ascontiguousarray(np.stack(tables) if len(tables) else np.zeros((1, NSYM)), dtype=np.uint32)
    pay = np.frombuffer(payload, np.uint8).copy() if len(payload) else np.zeros(1, np.uint8)
    tid = np.ascontiguousarray(tab_id, dtype=np.uint16) if nsym else np.zeros(1, np.uint16)
    go = np.ascontiguousarray(goff, np.uint64)
    gwa = np.ascontiguousarray(gw if len(gw) else np.zeros(1), np.uint32)
    rc = L.or_rans_decode_static16(len(ls) - 1, native.ptr(ls), native.ptr(tid), native.ptr(freq),
                                   len(tables), native.ptr(pay), len(payload), native.ptr(go),
                                   native.ptr(gwa), native.ptr(syms))
    if rc != 0:
        raise ValueError("corrupt rANS stream")
    return syms[:nsym]


def static_fc(syms: np.ndarray, tab_id: np.ndarray, tables: list[np.ndarray]):
    F = np.stack(tables)
    C = np.stack([cum_of(t) for t in tables])
    return F[tab_id, syms], C[tab_id, syms]


# ----------------------------------------------------------------------------- learned model

def _model_arrays(m: dict) -> dict:
    return {
        "w1": np.asarray(m["w1"], np.int8).reshape(64, 4),
        "b1": np.asarray(m["b1"], np.int32).reshape(NCHAN, 64),
        "w2": np.asarray(m["w2"], np.int8).reshape(64, 64),
        "b2": np.asarray(m["b2"], np.int32).reshape(64),
        "w3": np.asarray(m["w3"], np.int8).reshape(256, 64),
        "b3": np.asarray(m["b3"], np.int32).reshape(256),
        "m1": int(m["m1"]), "sh1": int(m["sh1"]), "m2": int(m["m2"]), "sh2": int(m["sh2"]),
        "ms": int(m["ms"]), "ss": int(m["ss"]),
    }


def model_bytes(m: dict) -> bytes:
    a = _model_arrays(m)
    out = struct.pack("<4i4I", a["m1"], a["sh1"], a["m2"], a["sh2"], a["ms"], a["ss"], 0, 0)
    out += a["b1"].astype("<i4").tobytes() + a["b2"].astype("<i4").tobytes() + a["b3"].astype("<i4").tobytes()
    out += a["w1"].tobytes() + a["w2"].tobytes() + a["w3"].tobytes()
    assert len(out) == MODEL_BYTES
    return out


def parse_model(buf: bytes, off: int) -> dict:
    m1, sh1, m2, sh2, ms, ss, _, _ = struct.unpack_from("<4i4I", buf, off)
    p = off + 32
    b1 = np.frombuffer(buf, "<i4", NCHAN * 64, p).reshape(NCHAN, 64); p += NCHAN * 64 * 4
    b2 = np.frombuffer(buf, "<i4", 64, p); p += 256
    b3 = np.frombuffer(buf, "<i4", 256, p); p += 1024
    w1 = np.frombuffer(buf, np.int8, 256, p).reshape(64, 4); p += 256
    w2 = np.frombuffer(buf, np.int8, 4096, p).reshape(64, 64); p += 4096
    w3 = np.frombuffer(buf, np.int8, 16384, p).reshape(256, 64)
    m = dict(w1=w1, b1=b1, w2=w2, b2=b2, w3=w3, b3=b3, m1=m1, sh1=sh1, m2=m2, sh2=sh2, ms=ms, ss=ss)
    validate_model(m)
    return m


def validate_model(m: dict) -> None:
    ok = (1 <= m["sh1"] <= 47 and 1 <= m["sh2"] <= 47 and 0 <= m["m1"] < 2 ** 31 and 0 <= m["m2"] < 2 ** 31
          and 1 <= m["ms"] < 2 ** 24 and m["ss"] <= 24
          and all(np.abs(np.asarray(m[k], np.int64)).max() < 2 ** 24 for k in ("b1", "b2", "b3")))
    if not ok:
        raise ValueError("invalid model")


_EXP2Q = None


def _exp2q_arr() -> np.ndarray:
    """The table as a module-lifetime array (pointers to it stay valid across C calls)."""
    global _EXP2Q
    if _EXP2Q is None:
        _EXP2Q = np.array(exp2q_table(), dtype=np.uint32)
    return _EXP2Q


def learned_fc(model: dict, syms_rows: np.ndarray, lane_row: np.ndarray, lane_lo: int, lane_hi: int):
    L = native.lib()
    ms = native.model_struct(_model_arrays(model))
    nsym = int(lane_row[lane_hi] - lane_row[lane_lo]) * NCHAN
    f = np.zeros(max(nsym, 1), np.uint32)
    c = np.zeros(max(nsym, 1), np.uint32)
    sy = np.ascontiguousarray(syms_rows, np.uint8)
    lr = np.ascontiguousarray(lane_row, np.int64)
    ex = _exp2q_arr()
    if not sy.size:
        sy = np.zeros((1, NCHAN), np.uint8)
    L.or_learned_fc(native.ctypes.byref(ms), native.ptr(ex), native.ptr(sy),
                    native.ptr(lr), lane_lo, lane_hi, native.ptr(f), native.ptr(c))
    return f[:nsym], c[:nsym]


def learned_freq(model: dict, u: np.ndarray, c: int) -> np.ndarray:
    """Frequency table for context u[4] (u_j = s_{i-j} - 128) of channel c."""
    L = native.lib()
    ms = native.model_struct(_model_arrays(model))
    z = np.zeros(NSYM, np.int32)
    uu = np.ascontiguousarray(u, np.int32)
    L.or_model_logits(native.ctypes.byref(ms), native.ptr(uu), int(c), native.ptr(z))
    f = np.zeros(NSYM, np.uint32)
    ex = _exp2q_arr()
    L.or_logits_to_freq(native.ptr(z), ms.ms, ms.ss, native.ptr(ex), native.ptr(f))
    return f


def logits_to_freq(z: np.ndarray, ms: int, ss: int) -> np.ndarray:
    f = np.zeros(NSYM, np.uint32)
    zz = np.ascontiguousarray(z, np.int32)
    ex = _exp2q_arr()
    native.lib().or_logits_to_freq(native.ptr(zz), ms, ss, native.ptr(ex), native.ptr(f))
    return f


def rans_decode_learned(model, lane_row, lane_lo, lane_hi, payload, goff, gw, n_rows) -> np.ndarray:
    """Decodes lanes [lane_lo, lane_hi); returns row-major symbols [n_rows, 56] (rows of other
    lanes stay 0).  goff/gw are the full group tables."""
    L = native.lib()
    ms = native.model_struct(_model_arrays(model))
    syms = np.zeros((max(n_rows, 1), NCHAN), np.uint8)
    pay = np.frombuffer(payload, np.uint8).copy() if len(payload) else np.zeros(1, np.uint8)
    lr = np.ascontiguousarray(lane_row, np.int64)
    go = np.ascontiguousarray(goff, np.uint64)
    gwa = np.ascontiguousarray(gw if len(gw) else np.zeros(1), np.uint32)
    ex = _exp2q_arr()
    rc = L.or_rans_decode_learned(native.ctypes.byref(ms), native.ptr(ex), native.ptr(lr),
                                  lane_lo, lane_hi, native.ptr(pay), len(payload),
                                  native.ptr(go), native.ptr(gwa), native.ptr(syms))
    if rc != 0:
        raise ValueError("corrupt rANS stream")
    return syms[:n_rows]


def rans_decode_pe(model: dict, coord: np.ndarray, depth: int, lane_row: np.ndarray, payload, goff, gw,
                   lane_lo: int = 0, lane_hi: int | None = None) -> np.ndarray:
    """Position-aware learned decode of lanes [lane_lo, lane_hi) (all by default); row-major
    symbols [n_rows, 56] (rows of other lanes stay 0)."""
    L = native.lib()
    ms = native.pe_model_struct(model)
    n_rows = int(lane_row[-1])
    syms = np.zeros((max(n_rows, 1), NCHAN), np.uint8)
    pay = np.frombuffer(payload, np.uint8).copy() if len(payload) else np.zeros(1, np.uint8)
    crd = np.ascontiguousarray(coord if n_rows else np.zeros((3, 1)), np.uint32)
    lr = np.ascontiguousarray(lane_row, np.int64)
    go = np.ascontiguousarray(goff, np.uint64)
    gwa = np.ascontiguousarray(gw if len(gw) else np.zeros(1), np.uint32)
    ex = _exp2q_arr()
    s8 = _sin8_arr()
    lane_hi = len(lane_row) - 1 if lane_hi is None else lane_hi
    rc = L.or_rans_decode_pe(native.ctypes.byref(ms), native.ptr(ex), native.ptr(s8), native.ptr(crd), n_rows,
                             depth, native.ptr(lr), lane_lo, lane_hi, native.ptr(pay), len(payload),
                             native.ptr(go), native.ptr(gwa), native.ptr(syms))
    if rc != 0:
        raise ValueError("corrupt rANS stream")
    return syms[:n_rows]


_SIN8 = None


def _sin8_arr() -> np.ndarray:
    global _SIN8
    if _SIN8 is None:
        _SIN8 = model_pe.sin8_table().astype(np.int8)
    return _SIN8


# ----------------------------------------------------------------------------- the pipeline

@dataclass
class Prepared:
    """Everything steps 1-5 fix: the decoded scene is q, step, offset and the geometry."""
    depth: int
    n_in: int
    keep: np.ndarray          # original indices of the rows, in row order
    codes: np.ndarray         # Morton code of each row
    coord: np.ndarray         # uint32 [3, n_rows]
    leaf_codes: np.ndarray    # unique voxel codes U
    dups: np.ndarray          # [n_dup, 2] (leaf rank, extra copies)
    levels: list
    bits: np.ndarray          # uint32[56]
    q: np.ndarray             # uint32 [n_rows, 56] row-major tokens
    step: np.ndarray          # float32[56]
    offset: np.ndarray        # float32[56]
    attr: np.ndarray = field(default=None)  # dequantized float32 [56, n_rows]
    pos: np.ndarray = field(default=None)   # float32 [3, n_rows]

    @property
    def n_rows(self) -> int:
        return int(self.keep.shape[0])


def prepare(pos: np.ndarray, attr: np.ndarray, depth: int, bits) -> Prepared:
    if not (1 <= depth <= 21):
        raise ValueError("depth out of range")
    if not (np.all(np.isfinite(pos)) and np.all(np.isfinite(attr))):
        raise ValueError("non-finite input")
    if pos.size and (pos.min() < 0 or pos.max() >= 1):
        raise ValueError("positions outside [0, 1)")
    n = pos.shape[1]
    bits = np.broadcast_to(np.asarray(bits, np.uint32), (NCHAN,)).copy()
    keep = prune(attr)
    coord = voxelize(pos[:, keep], depth)
    codes = morton(coord, depth)
    order = np.lexsort((keep, codes))
    keep, coord, codes = keep[order], coord[:, order], codes[order]
    leaf, counts = np.unique(codes, return_counts=True)
    extra = counts - 1
    dup_rank = np.nonzero(extra)[0]
    dups = np.stack([dup_rank, extra[dup_rank]], axis=1).astype(np.uint32) if len(dup_rank) else np.zeros((0, 2), np.uint32)
    levels = octree_levels(leaf, depth) if len(leaf) else [np.zeros(0, np.uint8) for _ in range(depth)]
    nr = len(keep)
    q = np.zeros((nr, NCHAN), np.uint32)
    step = np.zeros(NCHAN, np.float32)
    offset = np.zeros(NCHAN, np.float32)
    out = np.zeros((NCHAN, nr), np.float32)
    for c in range(NCHAN):
        qc, s, o = quantize(attr[c, keep], int(bits[c]))
        q[:, c], step[c], offset[c] = qc, s, o
        out[c] = dequantize(qc, s, o)
    return Prepared(depth, n, keep, codes, coord, leaf, dups, levels, bits, q, step, offset,
                    out, position(coord, depth))


def geo_plan(levels: list[np.ndarray], geo_mode: int):
    coded = [geo_mode != GEO_RAW and len(b) >= GEO_RANS_MIN_LEVEL for b in levels]
    return coded


# ----------------------------------------------------------------------------- learned geometry

_POPCOUNT8 = np.array([bin(b).count("1") for b in range(256)], np.int64)


def geo_children_ctx(parent: np.ndarray) -> np.ndarray:
    """Context id 8 b + k of every node of a level, given the level above it: node order is
    the parents in order and, within a parent with byte b, its set bits k ascending (the
    breadth-first serialization of Sec. 3.4, "Geometry Occupancy Coding"); the parent level
    conditions the children, as Eq. 8's p(t_l | t_<l)."""
    b = np.asarray(parent, np.int64)
    bits = (b[:, None] >> np.arange(8)) & 1
    pi, k = np.nonzero(bits)
    return 8 * b[pi] + k


def geo_ctx_inputs(ctx: np.ndarray) -> np.ndarray:
    """Model inputs u [n, 4] of context ids: the parent byte, the child index, the parent's
    occupied-child count and the child's rank among them, each mapped into [-128, 127]."""
    ctx = np.asarray(ctx, np.int64)
    b, k = ctx >> 3, ctx & 7
    rank = _POPCOUNT8[b & ((1 << k) - 1)]
    return np.stack([b - 128, 32 * k - 112, 16 * _POPCOUNT8[b] - 64, 32 * rank - 112], axis=1)


def geo_samples(levels: list[np.ndarray], geo_mode: int = GEO_LEARNED):
    """Training samples (U [n, 4], C [n] = level, S [n] = token) of every coded level."""
    coded = geo_plan(levels, geo_mode)
    U, C, S = [], [], []
    for l in range(1, len(levels)):
        if not coded[l]:
            continue
        U.append(geo_ctx_inputs(geo_children_ctx(levels[l - 1])))
        C.append(np.full(len(levels[l]), l, np.int64))
        S.append(np.asarray(levels[l], np.int64))
    if not U:
        return np.zeros((0, 4), np.int64), np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(U), np.concatenate(C), np.concatenate(S)


def geo_level_tables(model: dict, level: int, ctx: np.ndarray):
    """(distinct context ids, their frequency tables [k][256], each token's table index)."""
    ids, tab = np.unique(ctx, return_inverse=True)
    U = geo_ctx_inputs(ids)
    tables = [learned_freq(model, U[i], level) for i in range(len(ids))]
    return ids, tables, tab.astype(np.uint16)


def geo_lanes_for_level(n: int) -> int:
    return default_geo_lanes(n)


def encode(pos: np.ndarray, attr: np.ndarray, *, mode: int, depth: int, bits=8, lanes: int = 32,
           geo_mode: int = GEO_RANS, geo_lanes: int = 0, model: dict | None = None,
           prep: Prepared | None = None, geo_model: dict | None = None) -> bytes:
    """Scene -> bitstream (layout documented in the design notes and in include/sgs.h)."""
    if mode in (MODE_STATIC, MODE_LEARNED, MODE_LEARNED_PE):
        bits = 8
    P = prep if prep is not None else prepare(pos, attr, depth, bits)
    if mode != MODE_FIXED and np.any(P.bits != 8):
        raise ValueError("entropy-coded modes use 8-bit tokens")
    nr = P.n_rows
    sections = {}
    # geometry
    coded = geo_plan(P.levels, geo_mode)
    n_level = np.array([len(b) for b in P.levels], np.uint32)
    raw_geo = b"".join(P.levels[l].tobytes() for l in range(depth) if not coded[l])
    coded_syms = [P.levels[l] for l in range(depth) if coded[l]]
    n_coded = int(sum(len(b) for b in coded_syms))
    geo_tab = b""
    geo_grp = b""
    geo_pay = b""
    Lg = 0
    if n_coded and geo_mode == GEO_LEARNED:
        # learned geometry: one model (geo_tab); each coded level's tokens in lanes of
        # contiguous chunks, coded with the context tables of the level above it
        if geo_model is None:
            raise ValueError("learned geometry needs a model")
        validate_model(_model_arrays(geo_model))
        geo_tab = model_bytes(geo_model)
        for l in range(depth):
            if not coded[l]:
                continue
            ctx = geo_children_ctx(P.levels[l - 1])
            _, tables, tab = geo_level_tables(geo_model, l, ctx)
            f, cc = static_fc(P.levels[l], tab, tables)
            Ll = geo_lanes_for_level(len(P.levels[l]))
            Lg += Ll
            pay, goff, gw = rans_encode(lane_bounds(len(P.levels[l]), Ll), f, cc)
            geo_grp += group_table_bytes(np.asarray(goff, np.uint64) + np.uint64(len(geo_pay)), gw)
            geo_pay += pay
    elif n_coded:
        Lg = geo_lanes if geo_lanes > 0 else default_geo_lanes(n_coded)
        tabs = [normalize_freq(np.bincount(b, minlength=NSYM)) for b in coded_syms]
        geo_tab = b"".join(table_bytes(t) for t in tabs)
        syms = np.concatenate(coded_syms)
        tab_id = np.concatenate([np.full(len(b), i, np.uint8) for i, b in enumerate(coded_syms)])
        gperm, gstart = static_row_order(n_coded, Lg)
        f, c = static_fc(syms[gperm], tab_id[gperm], tabs)
        geo_pay, goff, gw = rans_encode(gstart, f, c)
        geo_grp = group_table_bytes(goff, gw)
    # attributes
    L = 0
    if mode == MODE_FIXED:
        offs, pay = [], b""
        for c in range(NCHAN):
            offs.append(len(pay))
            pay += pack_fixed(P.q[:, c], int(P.bits[c]))
        attr_tab = np.array(offs + [len(pay)], "<u8").tobytes()
        attr_tab += b"\0" * (_align16(len(attr_tab)) - len(attr_tab))
        attr_grp, attr_pay = b"", pay
    else:
        L = lanes
        if L < 1:
            raise ValueError("lanes must be >= 1")
        lane_row = lane_bounds(nr, L)
        syms = P.q.astype(np.uint8)
        if mode == MODE_STATIC:
            tabs = [normalize_freq(np.bincount(syms[:, c], minlength=NSYM)) for c in range(NCHAN)]
            attr_tab = b"".join(table_bytes(t) for t in tabs)
            tab_id = np.tile(np.arange(NCHAN, dtype=np.uint8), nr)
            perm, rows_start = static_row_order(nr, L)
            f, cc = static_fc(syms[perm].ravel(), tab_id, tabs) if nr else (np.zeros(0), np.zeros(0))
        elif mode == MODE_LEARNED:
            if model is None:
                raise ValueError("learned mode needs a model")
            validate_model(_model_arrays(model))
            attr_tab = model_bytes(model)
            f, cc = learned_fc(model, syms, lane_row, 0, L)
        else:
            if model is None:
                raise ValueError("learned mode needs a model")
            model_pe.validate(model)
            attr_tab = model_pe.model_bytes(model)
            f, cc = model_pe.token_fc(model, syms, lane_row, P.coord, depth)
        starts = rows_start * NCHAN if mode == MODE_STATIC else lane_row * NCHAN
        attr_pay, goff, gw = rans_encode(starts, f, cc)
        attr_grp = group_table_bytes(goff, gw)
    dup = P.dups.astype("<u4").tobytes()
    chan = P.step.astype("<f4").tobytes() + P.offset.astype("<f4").tobytes() + P.bits.astype("<u4").tobytes()
    order = [("levels", n_level.astype("<u4").tobytes()), ("dup", dup), ("chan", chan),
             ("geo_raw", raw_geo), ("geo_tab", geo_tab), ("geo_grp", geo_grp), ("geo_pay", geo_pay),
             ("attr_tab", attr_tab), ("attr_grp", attr_grp), ("attr_pay", attr_pay)]
    body = b""
    offs = {}
    pos_ = HEADER_BYTES
    for name, blob in order:
        offs[name] = pos_
        padded = blob + b"\0" * (_align16(len(blob)) - len(blob))
        body += padded
        pos_ += len(padded)
    total = pos_
    hdr = struct.pack("<12I2Q", MAGIC, VERSION, mode, geo_mode, P.n_in, nr, depth, len(P.leaf_codes),
                      len(P.dups), NCHAN, L, Lg, sum(int(x) for x in n_level), n_coded)
    hdr += struct.pack("<11Q", *[offs[k] for k, _ in order], total)
    hdr += b"\0" * (HEADER_BYTES - len(hdr))
    return hdr + body


def default_geo_lanes(n_coded: int) -> int:
    """About 128 occupancy bytes per geometry lane, in whole groups of 32 lanes."""
    return max(32, (n_coded + 128 * 32 - 1) // (128 * 32) * 32)


def group_table_bytes(goff: np.ndarray, gw: np.ndarray) -> bytes:
    b = np.asarray(goff, "<u8").tobytes() + np.asarray(gw, "<u4").tobytes()
    return b + b"\0" * (_align16(len(b)) - len(b))


def pack_fixed(q: np.ndarray, b: int) -> bytes:
    """Channel-wise fixed-length code (Sec. 3.4.1): value i at bits [i b, (i+1) b) of a
    little-endian uint32 stream, LSB first; padded to 16 bytes."""
    if q.size == 0:
        return b""
    bitmat = ((q[:, None].astype(np.uint32) >> np.arange(b, dtype=np.uint32)) & 1).astype(np.uint8)
    by = np.packbits(bitmat.ravel(), bitorder="little").tobytes()
    nwords = (q.size * b + 31) // 32
    by = by + b"\0" * (4 * nwords - len(by))
    return by + b"\0" * (_align16(len(by)) - len(by))


def unpack_fixed(buf: bytes, off: int, n: int, b: int) -> np.ndarray:
    if n == 0:
        return np.zeros(0, np.uint32)
    nbytes = (n * b + 7) // 8
    bits = np.unpackbits(np.frombuffer(buf, np.uint8, nbytes, off), bitorder="little")[: n * b]
    return (bits.reshape(n, b).astype(np.uint32) << np.arange(b, dtype=np.uint32)).sum(axis=1).astype(np.uint32)


# ----------------------------------------------------------------------------- reader / decoder

HEADER_FMT = "<12I2Q11Q"
SECTIONS = ["levels", "dup", "chan", "geo_raw", "geo_tab", "geo_grp", "geo_pay", "attr_tab", "attr_grp", "attr_pay"]


def parse_header(buf: bytes) -> dict:
    if len(buf) < HEADER_BYTES:
        raise ValueError("short bitstream")
    v = struct.unpack_from(HEADER_FMT, buf, 0)
    keys = ["magic", "version", "mode", "geo_mode", "n_in", "n_rows", "depth", "n_leaves", "n_dup",
            "n_chan", "lanes", "geo_lanes", "n_geo", "n_geo_coded"] + ["off_" + s for s in SECTIONS] + ["total"]
    h = dict(zip(keys, v))
    if h["magic"] != MAGIC or h["version"] != VERSION or h["n_chan"] != NCHAN:
        raise ValueError("bad header")
    if h["total"] != len(buf):
        raise ValueError("length mismatch")
    return h


def decode(buf: bytes, attr_groups: int | None = None) -> dict:
    """Bitstream -> {attr [56][n], pos [3][n], coord [3][n], q [n][56]} (rows in Morton order).
    attr_groups = k limits a learned-model decode to the attribute lanes of the first k groups
    of 32 (rows of the other lanes stay 0): a bounded sample for timing."""
    h = parse_header(buf)
    D, nr, U = h["depth"], h["n_rows"], h["n_leaves"]
    n_level = np.frombuffer(buf, "<u4", D, h["off_levels"]).astype(np.int64)
    dups = np.frombuffer(buf, "<u4", 2 * h["n_dup"], h["off_dup"]).reshape(-1, 2)
    step = np.frombuffer(buf, "<f4", NCHAN, h["off_chan"])
    offset = np.frombuffer(buf, "<f4", NCHAN, h["off_chan"] + 4 * NCHAN)
    bits = np.frombuffer(buf, "<u4", NCHAN, h["off_chan"] + 8 * NCHAN)
    # geometry bytes
    coded = geo_plan([np.zeros(int(n)) for n in n_level], h["geo_mode"])
    levels = [None] * D
    p = h["off_geo_raw"]
    for l in range(D):
        if not coded[l]:
            levels[l] = np.frombuffer(buf, np.uint8, int(n_level[l]), p)
            p += int(n_level[l])
    n_coded = h["n_geo_coded"]
    if n_coded and h["geo_mode"] == GEO_LEARNED:
        geo_model = parse_model(buf, h["off_geo_tab"])
        pay = buf[h["off_geo_pay"]:h["off_attr_tab"]]
        gp = h["off_geo_grp"]
        for l in range(D):
            if not coded[l]:
                continue
            n_l = int(n_level[l])
            Ll = geo_lanes_for_level(n_l)
            G = (Ll + 31) // 32
            goff = np.frombuffer(buf, "<u8", G + 1, gp)
            gw = np.frombuffer(buf, "<u4", G, gp + 8 * (G + 1))
            gp += _align16(8 * (G + 1) + 4 * G)
            ctx = geo_children_ctx(levels[l - 1])
            if len(ctx) != n_l:
                raise ValueError("corrupt octree level")
            _, tables, tab = geo_level_tables(geo_model, l, ctx)
            levels[l] = rans_decode_static16(lane_bounds(n_l, Ll), tab, tables, pay, goff, gw)
    elif n_coded:
        cl = [l for l in range(D) if coded[l]]
        tabs, _ = parse_tables(buf, h["off_geo_tab"], len(cl))
        Lg = h["geo_lanes"]
        G = (Lg + 31) // 32
        goff = np.frombuffer(buf, "<u8", G + 1, h["off_geo_grp"])
        gw = np.frombuffer(buf, "<u4", G, h["off_geo_grp"] + 8 * (G + 1))
        tab_id = np.concatenate([np.full(int(n_level[l]), i, np.uint8) for i, l in enumerate(cl)])
        pay = buf[h["off_geo_pay"]:h["off_attr_tab"]]
        gperm, gstart = static_row_order(n_coded, Lg)
        dec = rans_decode_static(gstart, tab_id[gperm], tabs, pay, goff, gw)
        syms = np.zeros(n_coded, np.uint8)
        syms[gperm] = dec
        q0 = 0
        for l in cl:
            levels[l] = syms[q0:q0 + int(n_level[l])]
            q0 += int(n_level[l])
    leaf = octree_expand(levels, D)
    if len(leaf) != U:
        raise ValueError("corrupt octree leaf count")
    mult = np.ones(U, np.int64)
    if len(dups):
        mult[dups[:, 0].astype(np.int64)] += dups[:, 1]
    codes = np.repeat(leaf, mult)
    if len(codes) != nr:
        raise ValueError("corrupt duplicate list")
    coord = demorton(codes, D)
    # attributes
    mode = h["mode"]
    if mode == MODE_FIXED:
        offs = np.frombuffer(buf, "<u8", NCHAN + 1, h["off_attr_tab"])
        q = np.stack([unpack_fixed(buf, h["off_attr_pay"] + int(offs[c]), nr, int(bits[c])) for c in range(NCHAN)], axis=1) \
            if nr else np.zeros((0, NCHAN), np.uint32)
    else:
        L = h["lanes"]
        G = (L + 31) // 32
        goff = np.frombuffer(buf, "<u8", G + 1, h["off_attr_grp"])
        gw = np.frombuffer(buf, "<u4", G, h["off_attr_grp"] + 8 * (G + 1))
        pay = buf[h["off_attr_pay"]:h["total"]]
        lane_row = lane_bounds(nr, L)
        if mode == MODE_STATIC:
            tabs, _ = parse_tables(buf, h["off_attr_tab"], NCHAN)
            tab_id = np.tile(np.arange(NCHAN, dtype=np.uint8), nr)
            perm, rows_start = static_row_order(nr, L)
            syms = rans_decode_static(rows_start * NCHAN, tab_id, tabs, pay, goff, gw)
            q = np.zeros((nr, NCHAN), np.uint32)
            q[perm] = syms.reshape(nr, NCHAN)
        elif mode == MODE_LEARNED:
            model = parse_model(buf, h["off_attr_tab"])
            hi = L if attr_groups is None else min(L, 32 * attr_groups)
            q = rans_decode_learned(model, lane_row, 0, hi, pay, goff, gw, nr).astype(np.uint32)
        else:
            model = model_pe.parse_model(buf, h["off_attr_tab"])
            hi = L if attr_groups is None else min(L, 32 * attr_groups)
            q = rans_decode_pe(model, coord, D, lane_row, pay, goff, gw, 0, hi).astype(np.uint32)
    attr = np.stack([dequantize(q[:, c], step[c], offset[c]) for c in range(NCHAN)]) if nr else np.zeros((NCHAN, 0), np.float32)
    return {"attr": attr, "pos": position(coord, D), "coord": coord, "q": q, "header": h}
