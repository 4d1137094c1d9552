"""Seeded synthetic 3DGS scenes shaped like the paper's workloads.

This module holds no arithmetic of the compression method: it only draws
positions and attribute values.  Both the CPU oracle (in tests) and the CUDA
library consume its arrays, so it imports neither.

Scene layout (structure of arrays, fp32):
  pos  [3][N]   positions in [0, 1)^3
  attr [56][N]  attribute channels in the token order a_i = [c_i, alpha_i, s_i, r_i]
                (Sec. 3.4, "Autoregressive Attribute Coding"):
                  0..2    SH DC colour (3)
                  3..47   SH rest, channel 3 + colour*15 + (k-1), k = 1..15, band floor(sqrt(k))
                  48      opacity logit
                  49..51  log-scales
                  52..55  rotation quaternion (unit norm)

Recipe (stated in full in the design notes):
  * positions: 16 isotropic Gaussian blobs (sigma 0.05) with centres ~ U[0.15, 0.85]^3,
    resampled until inside [0, 1)^3;
  * each channel is driven by a latent z = rho * g(p) + sqrt(1 - rho^2) * eps, where g is a
    unit-variance spatially correlated field (trilinear value noise on a 32^3 lattice,
    normalised by the interpolation weights so that g ~ N(0, 1) at every point) and eps is
    white N(0, 1).  rho = 0.8 by default; rho = 0 is the uncorrelated control;
  * marginals: log-scale -4 + 0.5 z, opacity 1.5 z, SH DC 0.5 z, SH rest Laplace with scale
    0.1 * 0.7^band via the Laplace quantile of Phi(z), quaternion normalize(z1..z4).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

N_CHAN = 56
GRID = 32


@dataclass
class Scene:
    pos: np.ndarray   # float32 [3, N]
    attr: np.ndarray  # float32 [56, N]
    seed: int
    rho: float

    @property
    def n(self) -> int:
        return int(self.pos.shape[1])


def _positions(rng: np.random.Generator, n: int, n_blobs: int = 16, sigma: float = 0.05) -> np.ndarray:
    centres = rng.uniform(0.15, 0.85, size=(n_blobs, 3))
    out = np.empty((n, 3), dtype=np.float64)
    filled = 0
    while filled < n:
        m = n - filled
        which = rng.integers(0, n_blobs, size=m)
        p = centres[which] + sigma * rng.standard_normal((m, 3))
        ok = np.all((p >= 0.0) & (p < 1.0), axis=1)
        p = p[ok]
        out[filled:filled + len(p)] = p
        filled += len(p)
    p32 = out.astype(np.float32)
    # float32 rounding can push a value to exactly 1.0; keep the half-open cube
    p32 = np.minimum(p32, np.float32(np.nextafter(np.float32(1.0), np.float32(0.0))))
    return np.ascontiguousarray(p32.T)


def _field(rng: np.random.Generator, pos: np.ndarray, n_fields: int) -> np.ndarray:
    """Unit-variance value-noise fields sampled at pos: [n_fields, N] float64."""
    n = pos.shape[1]
    g = pos.astype(np.float64) * (GRID - 1)
    i0 = np.clip(np.floor(g).astype(np.int64), 0, GRID - 2)
    t = g - i0
    lattice = rng.standard_normal((n_fields, GRID * GRID * GRID))
    corners = []
    wsq = np.zeros(n, dtype=np.float64)
    for dx in (0, 1):
        wx = t[0] if dx else 1.0 - t[0]
        for dy in (0, 1):
            wy = t[1] if dy else 1.0 - t[1]
            for dz in (0, 1):
                wz = t[2] if dz else 1.0 - t[2]
                w = wx * wy * wz
                wsq += w * w
                flat = ((i0[0] + dx) * GRID + (i0[1] + dy)) * GRID + (i0[2] + dz)
                corners.append((w, flat))
    norm = 1.0 / np.sqrt(wsq)
    out = np.empty((n_fields, n), dtype=np.float64)
    for f in range(n_fields):
        lat = lattice[f]
        acc = np.zeros(n, dtype=np.float64)
        for w, flat in corners:
            acc += w * np.take(lat, flat)
        out[f] = acc * norm
    return out


def _phi(z: np.ndarray) -> np.ndarray:
    from scipy.special import ndtr
    return ndtr(z)


def make_scene(n: int, seed: int, rho: float = 0.8) -> Scene:
    """Draw a scene of n Gaussians; identical arrays for identical (n, seed, rho)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if n == 0:
        return Scene(np.zeros((3, 0), np.float32), np.zeros((N_CHAN, 0), np.float32), seed, rho)
    pos = _positions(rng, n)
    g = _field(rng, pos, N_CHAN)
    eps = rng.standard_normal((N_CHAN, n))
    z = rho * g + math.sqrt(max(0.0, 1.0 - rho * rho)) * eps
    attr = np.empty((N_CHAN, n), dtype=np.float64)
    attr[0:3] = 0.5 * z[0:3]
    for colour in range(3):
        for k in range(1, 16):
            c = 3 + colour * 15 + (k - 1)
            b = 0.1 * 0.7 ** int(math.isqrt(k))
            u = _phi(z[c]) - 0.5
            u = np.clip(u, -0.5 + 1e-12, 0.5 - 1e-12)
            attr[c] = -b * np.sign(u) * np.log1p(-2.0 * np.abs(u))
    attr[48] = 1.5 * z[48]
    attr[49:52] = -4.0 + 0.5 * z[49:52]
    q = z[52:56]
    q = q / np.maximum(np.linalg.norm(q, axis=0, keepdims=True), 1e-12)
    attr[52:56] = q
    return Scene(pos, np.ascontiguousarray(attr.astype(np.float32)), seed, rho)


def fixed_bits(seed: int) -> np.ndarray:
    """Per-channel fixed-length bit widths drawn uniformly from 4..10 (uint32[56])."""
    rng = np.random.Generator(np.random.PCG64(seed + 17))
    return rng.integers(4, 11, size=N_CHAN).astype(np.uint32)


def loguniform_sizes(seed: int, count: int, lo: float, hi: float) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=count)).astype(np.int64)


def kaiming_init(seed: int, n_ctx: int = 4, n_emb: int = 16, hidden: int = 64, n_sym: int = 256,
                 n_chan: int = N_CHAN) -> dict:
    """Seeded initial float weights of the context MLP (Kaiming-uniform, biases zero,
    embedding N(0, 1)).  Passed as inputs to both trainers."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d_in = n_ctx + n_emb

    def ku(fan_out, fan_in):
        bound = math.sqrt(6.0 / fan_in)
        return rng.uniform(-bound, bound, size=(fan_out, fan_in)).astype(np.float32)

    return {
        "emb": rng.standard_normal((n_chan, n_emb)).astype(np.float32),
        "w1": ku(hidden, d_in), "b1": np.zeros(hidden, np.float32),
        "w2": ku(hidden, hidden), "b2": np.zeros(hidden, np.float32),
        "w3": ku(n_sym, hidden), "b3": np.zeros(n_sym, np.float32),
    }


def kaiming_init_pe(seed: int, n_chan: int = N_CHAN) -> dict:
    """Seeded initial float weights of the position-aware model: the projection of the 75
    embedding inputs to 32, layer 1 over [context (4), channel embedding (16), projection
    (32)], layer 2, and the 2-output head (Kaiming-uniform, head scaled by 0.1 so that the
    initial Laplace sits near the middle of the token range; biases zero, embedding N(0, 1)).
    Passed as inputs to both trainers."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def ku(fan_out, fan_in, scale=1.0):
        bound = math.sqrt(6.0 / fan_in)
        return (scale * rng.uniform(-bound, bound, size=(fan_out, fan_in))).astype(np.float32)

    return {
        "emb": rng.standard_normal((n_chan, 16)).astype(np.float32),
        "wp": ku(32, 75), "bp": np.zeros(32, np.float32),
        "w1": ku(64, 52), "b1": np.zeros(64, np.float32),
        "w2": ku(64, 64), "b2": np.zeros(64, np.float32),
        "w3": ku(2, 64, 0.1), "b3": np.zeros(2, np.float32),
    }


# Workload recipes (sizes of the paper-shaped configurations)
SMALL = dict(n=20_000, seed=0, depth=12, lanes=32)            # static channel-wise, 8-bit
FIXED_1M = dict(n=1_000_000, seed=1000, depth=16)             # fixed-length 4..10 bits
LEARNED_1M = dict(n=1_000_000, seed=2000, depth=16, lanes=4096)
