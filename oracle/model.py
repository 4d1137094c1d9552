"""Oracle for the learned part: fp64 training of the context MLP and its integer freeze.
TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg).

The model is the local autoregressive attribute model of Sec. 3.4.2 made small and
integer: for token (i, c) its context is the previous 4 tokens of channel c in the lane
(Morton order inside the group of W Gaussians; 0 past the group start) plus a learned
16-dim embedding of c.  Float mirror:
    x = [u / 128 (4 values), emb[c] (16 values)],  u_j = s_{i-j,c} - 128
    h1 = ReLU(W1 x + b1), h2 = ReLU(W2 h1 + b2), z = W3 h2 + b3,  p = softmax(z) over 256.
Training loss: mean code length in bits, -log2 p(s) (the attribute rate R_attr of Eq. 9,
summed over the tokens; the 1/G factor of Eq. 9 is only a scale).  Adam (Kingma & Ba:
beta = (0.9, 0.999), eps = 1e-8).  Batches of (i, c) pairs are drawn with a counter-based
generator (splitmix64, Steele et al. 2014), defined here and in the library independently.
"""
from __future__ import annotations

import math

import numpy as np

from . import native

NCHAN, HID, NSYM, CTX, EMB = 56, 64, 256, 4, 16
LOG2E = 1.4426950408889634
CALIB_STEP = (1 << 20) - 1
M64 = (1 << 64) - 1


def splitmix64(x: np.ndarray) -> np.ndarray:
    z = (x + np.uint64(0x9E3779B97F4A7C15)).astype(np.uint64)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def sample_positions(seed: int, step: int, batch: int, n_total: int) -> np.ndarray:
    """Token positions p = 56 i + c of one batch: p_k = hi32(splitmix64(key_k)) * n >> 32,
    key_k = (seed << 40) ^ (step << 20) ^ k."""
    with np.errstate(over="ignore"):
        k = np.arange(batch, dtype=np.uint64)
        key = (np.uint64((seed << 40) & M64) ^ np.uint64(step << 20)) ^ k
        z = splitmix64(key)
        return (((z >> np.uint64(32)) * np.uint64(n_total)) >> np.uint64(32)).astype(np.int64)


def contexts(q: np.ndarray, lane_row: np.ndarray, pos: np.ndarray):
    """(u [B,4] int, c [B], s [B], row [B], row0 [B]) for token positions pos."""
    row = pos // NCHAN
    c = pos % NCHAN
    lane = np.searchsorted(lane_row, row, side="right") - 1
    row0 = lane_row[lane]
    u = np.zeros((len(pos), CTX), np.int64)
    for j in range(1, CTX + 1):
        r = row - j
        ok = r >= row0
        u[ok, j - 1] = q[r[ok], c[ok]].astype(np.int64) - 128
    return u, c, q[row, c].astype(np.int64), row, row0


def forward_backward(p: dict, u: np.ndarray, c: np.ndarray, s: np.ndarray):
    """fp64 loss (bits per token) and gradients of every parameter."""
    B = len(s)
    x = np.concatenate([u.astype(np.float64) / 128.0, p["emb"][c]], axis=1)
    a1 = x @ p["w1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["w2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ p["w3"].T + p["b3"]
    zm = z - z.max(axis=1, keepdims=True)
    lse = np.log(np.exp(zm).sum(axis=1))
    logp = zm[np.arange(B), s] - lse
    loss = -logp.mean() / math.log(2.0)
    prob = np.exp(zm - lse[:, None])
    dz = prob
    dz[np.arange(B), s] -= 1.0
    dz /= B * math.log(2.0)
    g = {}
    g["w3"] = dz.T @ h2
    g["b3"] = dz.sum(axis=0)
    dh2 = dz @ p["w3"]
    da2 = dh2 * (a2 > 0)
    g["w2"] = da2.T @ h1
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ p["w2"]
    da1 = dh1 * (a1 > 0)
    g["w1"] = da1.T @ x
    g["b1"] = da1.sum(axis=0)
    dx = da1 @ p["w1"]
    g["emb"] = np.zeros_like(p["emb"])
    np.add.at(g["emb"], c, dx[:, CTX:])
    return loss, g


def loss_only(p: dict, u, c, s) -> float:
    x = np.concatenate([u.astype(np.float64) / 128.0, p["emb"][c]], axis=1)
    h1 = np.maximum(x @ p["w1"].T + p["b1"], 0.0)
    h2 = np.maximum(h1 @ p["w2"].T + p["b2"], 0.0)
    z = h2 @ p["w3"].T + p["b3"]
    zm = z - z.max(axis=1, keepdims=True)
    lse = np.log(np.exp(zm).sum(axis=1))
    return float(-(zm[np.arange(len(s)), s] - lse).mean() / math.log(2.0))


PARAMS = ("emb", "w1", "b1", "w2", "b2", "w3", "b3")


def adam_step(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    for k in PARAMS:
        m[k] = b1 * m[k] + (1 - b1) * g[k]
        v[k] = b2 * v[k] + (1 - b2) * g[k] * g[k]
        mh = m[k] / (1 - b1 ** t)
        vh = v[k] / (1 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def train(init: dict, q: np.ndarray, lane_row: np.ndarray, steps: int, batch: int, seed: int,
          lr: float = 1e-3):
    """fp64 training from float init; returns (params fp64, per-step losses)."""
    p = {k: np.asarray(init[k], np.float64).copy() for k in PARAMS}
    m = {k: np.zeros_like(p[k]) for k in PARAMS}
    v = {k: np.zeros_like(p[k]) for k in PARAMS}
    n_total = q.shape[0] * NCHAN
    losses = []
    for t in range(steps):
        pos = sample_positions(seed, t, batch, n_total)
        u, c, s, _, _ = contexts(q, lane_row, pos)
        loss, g = forward_backward(p, u, c, s)
        adam_step(p, g, m, v, t + 1, lr)
        losses.append(loss)
    return p, losses


# ----------------------------------------------------------------------------- freeze

def _q8(w: np.ndarray):
    s = float(np.abs(w).max()) / 127.0
    if s == 0.0:
        s = 1.0
    return np.clip(np.rint(w / s), -127, 127).astype(np.int8), s


def _requant_params(A: int):
    """Largest sh in [1, 31] with m = floor(127 * 2^sh / A) < 2^31."""
    A = max(int(A), 1)
    for sh in range(31, 0, -1):
        m = (127 << sh) // A
        if m < (1 << 31):
            return m, sh
    return (127 << 1) // A, 1


def _clamp24(x: np.ndarray) -> np.ndarray:
    lim = (1 << 24) - 1
    return np.clip(x, -lim, lim).astype(np.int32)


def freeze(w: dict, q: np.ndarray, lane_row: np.ndarray, seed: int, n_calib: int = 65536) -> dict:
    """Float weights (fp32 values) -> integer model.  Scales and biases in fp64 with a fixed
    operation order; activation ranges from an integer calibration pass over n_calib tokens
    drawn with the batch generator at step 2^20 - 1."""
    p = {k: np.asarray(w[k], np.float32).astype(np.float64) for k in PARAMS}
    s_u = 1.0 / 128.0
    w1q, s_w1 = _q8(p["w1"][:, :CTX])
    s_a1 = s_u * s_w1
    b1f = np.empty((NCHAN, HID), np.float64)
    for c in range(NCHAN):
        for o in range(HID):
            t = p["b1"][o]
            for e in range(EMB):
                t = t + p["w1"][o, CTX + e] * p["emb"][c, e]
            b1f[c, o] = t
    B1 = _clamp24(np.rint(b1f / s_a1))
    w2q, s_w2 = _q8(p["w2"])
    w3q, s_w3 = _q8(p["w3"])
    n_total = q.shape[0] * NCHAN
    pos = sample_positions(seed, CALIB_STEP, n_calib, n_total)
    rows = pos // NCHAN
    chans = (pos % NCHAN).astype(np.int32)
    row0 = lane_row[np.searchsorted(lane_row, rows, side="right") - 1].astype(np.int64)
    syms = np.ascontiguousarray(q, np.uint8)
    L = native.lib()
    a1 = np.zeros(1, np.int64)
    a2 = np.zeros(1, np.int64)
    b2_dummy = np.zeros(HID, np.int32)
    w1c, B1c, w2c = np.ascontiguousarray(w1q), np.ascontiguousarray(B1), np.ascontiguousarray(w2q)
    rows_c = np.ascontiguousarray(rows, np.int64)
    L.or_calib_max(native.ptr(w1c), native.ptr(B1c), 0, 1, native.ptr(w2c), native.ptr(b2_dummy),
                   native.ptr(syms), native.ptr(rows_c), native.ptr(row0), native.ptr(chans),
                   len(pos), native.ptr(a1), native.ptr(a2))
    A1 = max(int(a1[0]), 1)
    m1, sh1 = _requant_params(A1)
    s_h1 = s_a1 * A1 / 127.0
    s_a2 = s_h1 * s_w2
    b2q = _clamp24(np.rint(p["b2"] / s_a2))
    L.or_calib_max(native.ptr(w1c), native.ptr(B1c), m1, sh1, native.ptr(w2c), native.ptr(b2q),
                   native.ptr(syms), native.ptr(rows_c), native.ptr(row0), native.ptr(chans),
                   len(pos), native.ptr(a1), native.ptr(a2))
    A2 = max(int(a2[0]), 1)
    m2, sh2 = _requant_params(A2)
    s_h2 = s_a2 * A2 / 127.0
    s_z = s_h2 * s_w3
    b3q = _clamp24(np.rint(p["b3"] / s_z))
    ms = int(np.clip(np.rint(s_z * LOG2E * 256.0 * 65536.0), 1, (1 << 24) - 1))
    return dict(w1=w1q, b1=B1, m1=m1, sh1=sh1, w2=w2q, b2=b2q, m2=m2, sh2=sh2,
                w3=w3q, b3=b3q, ms=ms, ss=16)


# ----------------------------------------------------------------------------- explicit contexts

def train_ctx(init: dict, U: np.ndarray, C: np.ndarray, S: np.ndarray, steps: int, batch: int, seed: int,
              lr: float = 1e-3):
    """fp64 training on an explicit sample set: sample k of a step is entry
    sample_positions(seed, step, batch, n) of (U [n, 4], C [n], S [n])."""
    p = {k: np.asarray(init[k], np.float64).copy() for k in PARAMS}
    m = {k: np.zeros_like(p[k]) for k in PARAMS}
    v = {k: np.zeros_like(p[k]) for k in PARAMS}
    n = len(S)
    losses = []
    for t in range(steps):
        idx = sample_positions(seed, t, batch, n)
        loss, g = forward_backward(p, U[idx].astype(np.int64), C[idx].astype(np.int64), S[idx].astype(np.int64))
        adam_step(p, g, m, v, t + 1, lr)
        losses.append(loss)
    return p, losses


def freeze_ctx(w: dict, U: np.ndarray, C: np.ndarray, seed: int, n_calib: int = 65536) -> dict:
    """As freeze, with the calibration contexts drawn from an explicit sample set (entry
    sample_positions(seed, 2^20 - 1, n_calib, n) of (U, C)); the arithmetic is freeze's."""
    p = {k: np.asarray(w[k], np.float32).astype(np.float64) for k in PARAMS}
    s_u = 1.0 / 128.0
    w1q, s_w1 = _q8(p["w1"][:, :CTX])
    s_a1 = s_u * s_w1
    b1f = np.empty((NCHAN, HID), np.float64)
    for c in range(NCHAN):
        for o in range(HID):
            t = p["b1"][o]
            for e in range(EMB):
                t = t + p["w1"][o, CTX + e] * p["emb"][c, e]
            b1f[c, o] = t
    B1 = _clamp24(np.rint(b1f / s_a1))
    w2q, s_w2 = _q8(p["w2"])
    w3q, s_w3 = _q8(p["w3"])
    idx = sample_positions(seed, CALIB_STEP, n_calib, len(C))
    u = U[idx].astype(np.int64)
    c = C[idx].astype(np.int64)
    a1 = u @ w1q.astype(np.int64).T + B1[c].astype(np.int64)
    A1 = max(int(a1.max()), 1)
    m1, sh1 = _requant_params(A1)
    s_h1 = s_a1 * A1 / 127.0
    s_a2 = s_h1 * s_w2
    b2q = _clamp24(np.rint(p["b2"] / s_a2))
    h1 = np.clip((a1 * m1 + (1 << (sh1 - 1))) >> sh1, 0, 127)
    a2 = h1 @ w2q.astype(np.int64).T + b2q.astype(np.int64)
    A2 = max(int(a2.max()), 1)
    m2, sh2 = _requant_params(A2)
    s_h2 = s_a2 * A2 / 127.0
    s_z = s_h2 * s_w3
    b3q = _clamp24(np.rint(p["b3"] / s_z))
    ms = int(np.clip(np.rint(s_z * LOG2E * 256.0 * 65536.0), 1, (1 << 24) - 1))
    return dict(w1=w1q, b1=B1, m1=m1, sh1=sh1, w2=w2q, b2=b2q, m2=m2, sh2=sh2,
                w3=w3q, b3=b3q, ms=ms, ss=16)
