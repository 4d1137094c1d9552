"""Oracle for the position-aware learned model: fp64 training, integer freeze, integer head
and CDF.  TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg).

The attribute model of Sec. 3.4.2 with the two parts of the paper's design that the plain
learned mode leaves out:
  * Fourier positional embedding (Sec. 3.4.2, "Fourier-based Positional Embedding"):
    phi(mu) = [mu; sin(2 pi F mu); cos(2 pi F mu)] with F = (2^0 .. 2^(L-1)), L = 12 bands,
    3 + 6L = 75 values, and a learned linear projection PE = Wp phi + bp to d = 32;
  * a conditional Laplace entropy model (Sec. 3.2, "Rate Proxy": p(y | c) is a Laplace
    distribution) instead of a 256-way softmax: the network predicts the mean and the
    log-rate of a Laplace over the 8-bit token, discretised at the half-integers.

Float model (training):
    x = [u / 128 (4), emb[c] (16), PE(phi) (32)],  u_j = s_{i-j,c} - 128 (0 past the lane
    start), h1 = ReLU(W1 x + b1), h2 = ReLU(W2 h1 + b2), (z0, z1) = W3 h2 + b3,
    mean m = clip(127.5 + 64 z0, 0, 255), log2-rate lam = clip(z1, -8, 6), r = 2^lam,
    F(x) = 2^(-r (m - x)) / 2 below the mean, 1 - 2^(-r (x - m)) / 2 above it,
    P(s) = F(s + 1/2) - F(s - 1/2) with F(-1/2) = 0 and F(255 + 1/2) = 1,
    p(s) = (1 + 65280 P(s)) / 65536 (the coder's floor of one count per symbol),
    loss = mean -log2 p(s) (attribute rate of Eq. 9 in bits per token).

Positions enter as the voxel coordinate v of the row (Sec. 3.4: attributes are coded upon
the decoded geometry): mu = (v + 1/2) / 2^D.  The embedding is computed on a 256-step phase
grid with an 8-bit sine table, so the float model and the integer model see the same
inputs: phi_q = [floor(128 mu) (3); SIN8[theta_k] (3L); SIN8[theta_k + 64] (3L)],
theta_k = floor(256 frac(2^k mu)), and the float model uses phi_q / 128.

Integer model (frozen): layer 1 over x_q = [u (4); phi_q (75); 0] with the projection folded
into it (W1_pe Wp, exact algebra of two linear maps) and the channel embedding and the
projection's bias folded into a per-channel bias; requantisation in fp32,
h = clamp(rint(float(acc) * s), 0, 127) (acc < 2^24 is exact in fp32, one rounding);
head: mu8 = 32640 + clamp(rint(z0 * smu), +-32640) (the mean in 1/256 symbol), lr8 =
clamp(rint(z1 * slr), -2048, 1536) (log2 of the rate in 1/256), n = 4096 + lr8; CDF from
the EXP2Q table (see pe_cdf).
"""
from __future__ import annotations

import math

import numpy as np

from . import model as M
from .exp2q import exp2q_table

NCHAN, HID, CTX, EMB, PED, BANDS = 56, 64, 4, 16, 32, 12
NPHI = 3 + 6 * BANDS          # 75
KIN = CTX + NPHI + 1          # 80: layer-1 inputs of the integer model (last one zero)
XF = CTX + EMB + PED          # 52: layer-1 inputs of the float model
MODEL_PE_BYTES = 23984
MU_HALF = 32640               # 127.5 * 256
MU_MAX = 65280                # 255 * 256
LR_MIN, LR_MAX = -2048, 1536  # log2-rate bounds (-8, 6) in 1/256
PARAMS = ("emb", "wp", "bp", "w1", "b1", "w2", "b2", "w3", "b3")
SHAPES = {"emb": (NCHAN, EMB), "wp": (PED, NPHI), "bp": (PED,), "w1": (HID, XF), "b1": (HID,),
          "w2": (HID, HID), "b2": (HID,), "w3": (2, HID), "b3": (2,)}
LN2 = math.log(2.0)


# ----------------------------------------------------------------------------- embedding

def sin8_table() -> np.ndarray:
    """SIN8[j] = round(127 sin(2 pi j / 256)), j = 0..255, from the fp64 sine; every value
    is checked to sit well away from a rounding tie."""
    out = np.zeros(256, np.int64)
    for j in range(256):
        y = 127.0 * math.sin(2.0 * math.pi * j / 256.0)
        r = math.floor(y + 0.5)
        assert abs(abs(y - r) - 0.5) > 1e-6
        out[j] = r
    return out


def phi_q(coord: np.ndarray, depth: int) -> np.ndarray:
    """Integer embedding inputs [n, 75] of voxel coordinates coord [3, n] at depth D."""
    v = np.asarray(coord, np.int64)
    n = v.shape[1]
    two = 2 * v + 1                                   # 2^(D+1) mu
    out = np.zeros((n, NPHI), np.int64)
    out[:, 0:3] = ((two << 6) >> depth).T             # floor(128 mu)
    sin8 = sin8_table()
    for k in range(BANDS):
        theta = ((two << (k + 8)) >> (depth + 1)) & 255   # floor(256 frac(2^k mu))
        out[:, 3 + 3 * k:6 + 3 * k] = sin8[theta].T
        out[:, 3 + 3 * BANDS + 3 * k:6 + 3 * BANDS + 3 * k] = sin8[(theta + 64) & 255].T
    return out


# ----------------------------------------------------------------------------- float model

def _head(z: np.ndarray, s: np.ndarray):
    """Code length and its derivatives with respect to (z0, z1), fp64."""
    mu_raw = 127.5 + 64.0 * z[:, 0]
    mu = np.clip(mu_raw, 0.0, 255.0)
    lam = np.clip(z[:, 1], -8.0, 6.0)
    r = np.exp2(lam)
    lo, hi = s - 0.5, s + 0.5
    first, last = s == 0, s == 255

    def edge(x, absent):
        d = np.abs(x - mu)
        e = np.where(absent, 0.0, np.exp2(-r * d))
        sg = np.sign(mu - x)                          # d|x - mu| / d mu
        de_dmu = np.where(absent, 0.0, -r * LN2 * sg * e)
        de_dr = np.where(absent, 0.0, -LN2 * d * e)
        return e, de_dmu, de_dr

    e_lo, dlo_mu, dlo_r = edge(lo, first)
    e_hi, dhi_mu, dhi_r = edge(hi, last)
    lo_below = first | (lo < mu)
    hi_above = last | (hi >= mu)
    straddle = lo_below & hi_above
    below = ~hi_above                                 # both boundaries below the mean
    # P and its partials with respect to e_hi, e_lo
    P = np.where(straddle, 1.0 - 0.5 * (e_hi + e_lo), np.where(below, 0.5 * (e_hi - e_lo), 0.5 * (e_lo - e_hi)))
    c_hi = np.where(straddle, -0.5, np.where(below, 0.5, -0.5))
    c_lo = np.where(straddle, -0.5, np.where(below, -0.5, 0.5))
    p = (1.0 + 65280.0 * P) / 65536.0
    bits = -np.log2(p)
    dL_dP = -(65280.0 / 65536.0) / (p * LN2)
    dP_dmu = c_hi * dhi_mu + c_lo * dlo_mu
    dP_dr = c_hi * dhi_r + c_lo * dlo_r
    dz0 = dL_dP * dP_dmu * 64.0 * ((mu_raw > 0.0) & (mu_raw < 255.0))
    dz1 = dL_dP * dP_dr * r * LN2 * ((z[:, 1] > -8.0) & (z[:, 1] < 6.0))
    return bits, np.stack([dz0, dz1], axis=1)


def forward_backward(p: dict, u: np.ndarray, c: np.ndarray, phi: np.ndarray, s: np.ndarray):
    """fp64 loss (bits per token) and gradients of every parameter; phi = phi_q rows."""
    B = len(s)
    ph = phi.astype(np.float64) / 128.0
    pe = ph @ p["wp"].T + p["bp"]
    x = np.concatenate([u.astype(np.float64) / 128.0, p["emb"][c], pe], axis=1)
    a1 = x @ p["w1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["w2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ p["w3"].T + p["b3"]
    bits, dz = _head(z, s.astype(np.float64))
    loss = float(bits.mean())
    dz = dz / B
    g = {}
    g["w3"] = dz.T @ h2
    g["b3"] = dz.sum(axis=0)
    da2 = (dz @ p["w3"]) * (a2 > 0)
    g["w2"] = da2.T @ h1
    g["b2"] = da2.sum(axis=0)
    da1 = (da2 @ p["w2"]) * (a1 > 0)
    g["w1"] = da1.T @ x
    g["b1"] = da1.sum(axis=0)
    dx = da1 @ p["w1"]
    g["emb"] = np.zeros_like(p["emb"])
    np.add.at(g["emb"], c, dx[:, CTX:CTX + EMB])
    dpe = dx[:, CTX + EMB:]
    g["wp"] = dpe.T @ ph
    g["bp"] = dpe.sum(axis=0)
    return loss, g


def loss_only(p: dict, u, c, phi, s) -> float:
    return forward_backward(p, u, c, phi, s)[0]


def batch(q: np.ndarray, lane_row: np.ndarray, phi_rows: np.ndarray, pos: np.ndarray):
    """(u, c, phi, s) of the tokens at positions pos = 56 row + channel."""
    u, c, s, row, _ = M.contexts(q, lane_row, pos)
    return u, c, phi_rows[row], s


def train(init: dict, q: np.ndarray, lane_row: np.ndarray, coord: np.ndarray, depth: int, steps: int,
          batch_size: int, seed: int, lr: float = 1e-3):
    """fp64 Adam training from float init (same sampler and optimizer as the plain model)."""
    p = {k: np.asarray(init[k], np.float64).copy() for k in PARAMS}
    m = {k: np.zeros_like(p[k]) for k in PARAMS}
    v = {k: np.zeros_like(p[k]) for k in PARAMS}
    phi_rows = phi_q(coord, depth)
    n_total = q.shape[0] * NCHAN
    losses = []
    for t in range(steps):
        pos = M.sample_positions(seed, t, batch_size, n_total)
        u, c, ph, s = batch(q, lane_row, phi_rows, pos)
        loss, g = forward_backward(p, u, c, ph, s)
        for k in PARAMS:
            m[k] = 0.9 * m[k] + 0.1 * g[k]
            v[k] = 0.999 * v[k] + 0.001 * g[k] * g[k]
            mh = m[k] / (1 - 0.9 ** (t + 1))
            vh = v[k] / (1 - 0.999 ** (t + 1))
            p[k] = p[k] - lr * mh / (np.sqrt(vh) + 1e-8)
        losses.append(loss)
    return p, losses


# ----------------------------------------------------------------------------- integer model

def _clamp23(x: np.ndarray) -> np.ndarray:
    lim = (1 << 23) - 1
    return np.clip(x, -lim, lim).astype(np.int32)


def _f32(x: float) -> np.float32:
    return np.float32(x)


def requant(acc: np.ndarray, s: np.float32) -> np.ndarray:
    """h = clamp(rint(float(acc) * s), 0, 127), one fp32 multiply (acc exact in fp32)."""
    return np.clip(np.rint(acc.astype(np.float32) * np.float32(s)), 0, 127).astype(np.int64)


def head_params(zm: np.ndarray, zl: np.ndarray, smu: np.float32, slr: np.float32):
    """(mu8, n) from the two head accumulators (fp32 multiply, round half to even)."""
    vm = np.clip(np.rint(zm.astype(np.float32) * np.float32(smu)), -MU_HALF, MU_HALF)
    vl = np.clip(np.rint(zl.astype(np.float32) * np.float32(slr)), LR_MIN, LR_MAX)
    return MU_HALF + vm.astype(np.int64), 4096 + vl.astype(np.int64)


def layer_inputs(u: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """x_q [B, 80] = [u (4); phi_q (75); 0]."""
    return np.concatenate([u.astype(np.int64), phi.astype(np.int64), np.zeros((len(u), 1), np.int64)], axis=1)


def _mm(a: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Integer a @ w.T, computed exactly (fp64 sums of integers below 2^53)."""
    return np.rint(a.astype(np.float64) @ w.astype(np.float64).T).astype(np.int64)


def forward_int(m: dict, u: np.ndarray, c: np.ndarray, phi: np.ndarray):
    """(mu8, n) of every token (vectorised; rows of u, c, phi are tokens)."""
    a1 = _mm(layer_inputs(u, phi), m["w1"]) + m["b1"][c]
    h1 = requant(a1, m["s1"])
    a2 = _mm(h1, m["w2"]) + m["b2"]
    h2 = requant(a2, m["s2"])
    z = _mm(h2, m["w3"]) + m["b3"]
    return head_params(z[:, 0], z[:, 1], m["smu"], m["slr"])


def pe_cdf(mu8, n, s):
    """Cumulative count of symbols below s (s in 0..256) of the integer Laplace:
    R = 2^(n/256) (the rate, 1/65536 per symbol) from EXP2Q; at the boundary x = s - 1/2,
    t = |x - mean| R (the base-2 exponent in 1/256), e = 2^(23 - t/256) from EXP2Q,
    F = e/2 below the mean and 2^23 - e/2 above it (F in 2^-23), cdf = s + floor(65280 F / 2^23).
    cdf(0) = 0 and cdf(256) = 65536, so every symbol keeps a count of at least 1."""
    ex = np.asarray(exp2q_table(), np.int64)
    mu8, n, s = np.broadcast_arrays(np.asarray(mu8, np.int64), np.asarray(n, np.int64), np.asarray(s, np.int64))
    q = (n + 255) >> 8
    R = ex[(-n) & 255] >> (23 - q)
    d = 256 * s - 128 - mu8
    t = np.minimum((np.abs(d) * R) >> 16, 6144)
    e = ex[t & 255] >> (t >> 8)
    F = np.where(d < 0, e >> 1, (1 << 23) - (e >> 1))
    cdf = s + ((F * 65280) >> 23)
    return np.where(s <= 0, 0, np.where(s >= 256, 65536, cdf))


def token_fc(m: dict, syms_rows: np.ndarray, lane_row: np.ndarray, coord: np.ndarray, depth: int,
             row_lo: int = 0, row_hi: int | None = None):
    """f and cum of the tokens of rows [row_lo, row_hi) (all by default) in lane-major order
    (lane by lane, row by row, channel by channel), the order of the attribute rANS streams."""
    n_rows = syms_rows.shape[0]
    row_hi = n_rows if row_hi is None else row_hi
    if row_hi <= row_lo:
        return np.zeros(0, np.uint32), np.zeros(0, np.uint32)
    pos = np.arange(row_lo * NCHAN, row_hi * NCHAN, dtype=np.int64)  # row-major = lane-major
    u, c, s, row, _ = M.contexts(syms_rows, lane_row, pos)
    phi = phi_q(coord, depth)[row]
    mu8, n = forward_int(m, u, c, phi)
    lo = pe_cdf(mu8, n, s)
    hi = pe_cdf(mu8, n, s + 1)
    return (hi - lo).astype(np.uint32), lo.astype(np.uint32)


# ----------------------------------------------------------------------------- freeze

def freeze(w: dict, q: np.ndarray, lane_row: np.ndarray, coord: np.ndarray, depth: int, seed: int,
           n_calib: int = 65536) -> dict:
    """Float weights (fp32 values) -> integer model.  Scales and biases in fp64 with a fixed
    operation order; activation ranges from an integer calibration pass over n_calib tokens
    drawn with the batch generator at step 2^20 - 1."""
    p = {k: np.asarray(w[k], np.float32).astype(np.float64).reshape(SHAPES[k]) for k in PARAMS}
    # fold the projection: W1_pe (Wp phi + bp) = (W1_pe Wp) phi + W1_pe bp
    wphi = np.zeros((HID, NPHI), np.float64)
    for e in range(PED):
        wphi = wphi + p["w1"][:, CTX + EMB + e][:, None] * p["wp"][e][None, :]
    w1cat = np.concatenate([p["w1"][:, :CTX], wphi, np.zeros((HID, 1))], axis=1)
    w1q, s_w1 = M._q8(w1cat)
    s_a1 = s_w1 / 128.0
    b1f = np.empty((NCHAN, HID), np.float64)
    for c in range(NCHAN):
        t = p["b1"].copy()
        for e in range(EMB):
            t = t + p["w1"][:, CTX + e] * p["emb"][c, e]
        for e in range(PED):
            t = t + p["w1"][:, CTX + EMB + e] * p["bp"][e]
        b1f[c] = t
    B1 = _clamp23(np.rint(b1f / s_a1))
    n_total = q.shape[0] * NCHAN
    pos = M.sample_positions(seed, M.CALIB_STEP, n_calib, n_total)
    u, c, s, row, _ = M.contexts(q, lane_row, pos)
    phi = phi_q(coord, depth)[row]
    a1 = _mm(layer_inputs(u, phi), w1q) + B1[c]
    A1 = max(int(a1.max()), 1)
    s1 = _f32(127.0 / A1)
    s_h1 = s_a1 * A1 / 127.0
    w2q, s_w2 = M._q8(p["w2"])
    s_a2 = s_h1 * s_w2
    b2q = _clamp23(np.rint(p["b2"] / s_a2))
    a2 = _mm(requant(a1, s1), w2q) + b2q
    A2 = max(int(a2.max()), 1)
    s2 = _f32(127.0 / A2)
    s_h2 = s_a2 * A2 / 127.0
    w3m, s_w3m = M._q8(p["w3"][0:1])
    w3l, s_w3l = M._q8(p["w3"][1:2])
    s_zm, s_zl = s_h2 * s_w3m, s_h2 * s_w3l
    b3q = np.array([_clamp23(np.rint(p["b3"][0] / s_zm)), _clamp23(np.rint(p["b3"][1] / s_zl))], np.int32)
    return dict(w1=w1q, b1=B1, s1=s1, w2=w2q, b2=b2q, s2=s2, w3=np.concatenate([w3m, w3l]), b3=b3q,
                smu=_f32(64.0 * 256.0 * s_zm), slr=_f32(256.0 * s_zl))


# ----------------------------------------------------------------------------- bytes

def model_bytes(m: dict) -> bytes:
    """Layout of the model section: f32 s1, s2, smu, slr; 16 zero bytes; i32 B1[56][64];
    i32 b2[64]; i32 b3[2] + 8 zero bytes; i8 W1[64][80]; i8 W2[64][64]; i8 W3[2][64]."""
    out = np.array([m["s1"], m["s2"], m["smu"], m["slr"]], "<f4").tobytes() + b"\0" * 16
    out += np.asarray(m["b1"], "<i4").reshape(NCHAN, HID).tobytes()
    out += np.asarray(m["b2"], "<i4").reshape(HID).tobytes()
    out += np.asarray(m["b3"], "<i4").reshape(2).tobytes() + b"\0" * 8
    out += np.asarray(m["w1"], np.int8).reshape(HID, KIN).tobytes()
    out += np.asarray(m["w2"], np.int8).reshape(HID, HID).tobytes()
    out += np.asarray(m["w3"], np.int8).reshape(2, HID).tobytes()
    assert len(out) == MODEL_PE_BYTES
    return out


def parse_model(buf: bytes, off: int) -> dict:
    s1, s2, smu, slr = np.frombuffer(buf, "<f4", 4, off)
    p = off + 32
    b1 = np.frombuffer(buf, "<i4", NCHAN * HID, p).reshape(NCHAN, HID).astype(np.int64); p += NCHAN * HID * 4
    b2 = np.frombuffer(buf, "<i4", HID, p).astype(np.int64); p += HID * 4
    b3 = np.frombuffer(buf, "<i4", 2, p).astype(np.int64); p += 16
    w1 = np.frombuffer(buf, np.int8, HID * KIN, p).reshape(HID, KIN).astype(np.int64); p += HID * KIN
    w2 = np.frombuffer(buf, np.int8, HID * HID, p).reshape(HID, HID).astype(np.int64); p += HID * HID
    w3 = np.frombuffer(buf, np.int8, 2 * HID, p).reshape(2, HID).astype(np.int64)
    m = dict(w1=w1, b1=b1, s1=np.float32(s1), w2=w2, b2=b2, s2=np.float32(s2), w3=w3, b3=b3,
             smu=np.float32(smu), slr=np.float32(slr))
    validate(m)
    return m


def validate(m: dict) -> None:
    """Bounds the decoder relies on: positive finite scales, requant scales at most 127,
    biases below 2^23 (every accumulator then stays below 2^24, exact in fp32)."""
    sc = [float(m[k]) for k in ("s1", "s2", "smu", "slr")]
    ok = all(math.isfinite(v) and v > 0.0 for v in sc) and sc[0] <= 127.0 and sc[1] <= 127.0
    ok = ok and all(np.abs(np.asarray(m[k], np.int64)).max() < (1 << 23) for k in ("b1", "b2", "b3"))
    if not ok:
        raise ValueError("invalid model")
