"""Oracle of the splatting consumer: renders decoded Gaussians into an image.  TEST
INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg).

The paper renders its decoded scenes with 3DGS rasterisation (Sec. 3, the decoded SoA is a
3DGS scene; the FPS column of its tables).  This is the forward pass of tile-based Gaussian
splatting (Kerbl et al., 2023), restated in plain numpy, in float32 because the kernel's
decisions (which tiles a Gaussian touches, which alphas count, where compositing stops) are
taken in float32 and the oracle must take them the same way:

  per Gaussian, with camera rotation Rw (world to camera), origin o, focal fx, fy, centre
  cx, cy:  t = Rw (p - o);  culled if t_z <= 0.2;  S = diag(exp(log scale)), R from the
  normalised quaternion (w, x, y, z), Sigma = R S S^T R^T;  J = [[fx / t_z, 0, -fx t_x / t_z^2],
  [0, fy / t_z, -fy t_y / t_z^2]], Sigma' = (J Rw) Sigma (J Rw)^T + 0.3 I;  culled if
  det Sigma' <= 0;  conic = Sigma'^-1;  radius = ceil(3 sqrt(lambda_max)) with lambda_max =
  m + sqrt(max(0.1, m^2 - det)), m = (a + c) / 2;  mean (u, v) = (fx t_x / t_z + cx,
  fy t_y / t_z + cy);  tiles of 16 x 16 pixels [floor((u - r) / 16), floor((u + r) / 16)]
  clipped to the image (culled if empty);  colour = max(0, 0.5 + sum_k sh_k Y_k(d)), real
  spherical harmonics of degree 3 along d = normalise(p - o);  opacity = sigmoid(logit);
  per pixel (x, y), the Gaussians of its tile in increasing depth t_z (ties by index):
  power = -0.5 (A dx^2 + C dy^2) - B dx dy with (dx, dy) = (u - x, v - y); skip if power > 0;
  alpha = min(0.99, opacity exp(power)); skip if alpha < 1/255; stop before a Gaussian that
  would bring the transmittance T below 1e-4; colour += c alpha T; T *= 1 - alpha.

Channels of the decoded attributes: 0-2 SH degree 0 (r, g, b), 3-47 SH degrees 1-3 (15 per
colour, colour-major), 48 opacity logit, 49-51 log scales, 52-55 quaternion (w, x, y, z).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

F32 = np.float32
TILE = 16
NEAR = F32(0.2)


@dataclass
class Camera:
    rot: np.ndarray     # [3, 3] world -> camera
    origin: np.ndarray  # [3]
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int


def look_at(origin, target, up, width: int, height: int, fov_y_deg: float) -> Camera:
    """A pinhole camera at `origin` looking at `target` (camera axes: x right, y down, z
    forward)."""
    o = np.asarray(origin, np.float64)
    z = np.asarray(target, np.float64) - o
    z /= np.linalg.norm(z)
    x = np.cross(z, np.asarray(up, np.float64))
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    f = 0.5 * height / math.tan(math.radians(fov_y_deg) / 2)
    return Camera(np.stack([x, y, z]).astype(np.float32), o.astype(np.float32), f, f, width / 2.0, height / 2.0,
                  width, height)


def sh_basis(d: np.ndarray) -> np.ndarray:
    """Real spherical harmonics Y_0 .. Y_15 (degrees 0-3, the 3DGS ordering) of unit vectors
    d [n, 3], from their closed forms, in float32."""
    x, y, z = d[:, 0], d[:, 1], d[:, 2]
    pi = math.pi
    c0 = 0.5 / math.sqrt(pi)
    c1 = math.sqrt(3.0 / (4.0 * pi))
    c2 = [0.5 * math.sqrt(15.0 / pi), -0.5 * math.sqrt(15.0 / pi), 0.25 * math.sqrt(5.0 / pi),
          -0.5 * math.sqrt(15.0 / pi), 0.25 * math.sqrt(15.0 / pi)]
    c3 = [-0.25 * math.sqrt(35.0 / (2.0 * pi)), 0.5 * math.sqrt(105.0 / pi), -0.25 * math.sqrt(21.0 / (2.0 * pi)),
          0.25 * math.sqrt(7.0 / pi), -0.25 * math.sqrt(21.0 / (2.0 * pi)), 0.25 * math.sqrt(105.0 / pi),
          -0.25 * math.sqrt(35.0 / (2.0 * pi))]
    xx, yy, zz = x * x, y * y, z * z
    Y = [np.full_like(x, c0),
         -c1 * y, c1 * z, -c1 * x,
         c2[0] * x * y, c2[1] * y * z, c2[2] * (2 * zz - xx - yy), c2[3] * x * z, c2[4] * (xx - yy),
         c3[0] * y * (3 * xx - yy), c3[1] * x * y * z, c3[2] * y * (4 * zz - xx - yy),
         c3[3] * z * (2 * zz - 3 * xx - 3 * yy), c3[4] * x * (4 * zz - xx - yy), c3[5] * z * (xx - yy),
         c3[6] * x * (xx - 3 * yy)]
    return np.stack(Y, axis=1).astype(F32)


def preprocess(pos: np.ndarray, attr: np.ndarray, cam: Camera):
    """Per Gaussian: screen mean, conic, radius, tile rectangle, depth, colour, opacity and
    a visibility flag (float32 throughout)."""
    p = np.asarray(pos, F32).T                                        # [n, 3]
    a = np.asarray(attr, F32)
    n = p.shape[0]
    Rw = cam.rot.astype(F32)
    t = (p - cam.origin.astype(F32)) @ Rw.T                           # [n, 3]
    tz = t[:, 2]
    vis = tz > NEAR
    s = np.exp(a[49:52].T)                                            # [n, 3]
    q = a[52:56].T
    q = q / np.sqrt((q * q).sum(axis=1, keepdims=True)).astype(F32)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], 1),
                  np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], 1),
                  np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], 1)], 1).astype(F32)
    M = R * s[:, None, :]
    Sig = M @ M.transpose(0, 2, 1)
    tzs = np.where(vis, tz, F32(1))
    J = np.zeros((n, 2, 3), F32)
    J[:, 0, 0] = F32(cam.fx) / tzs
    J[:, 0, 2] = -F32(cam.fx) * t[:, 0] / (tzs * tzs)
    J[:, 1, 1] = F32(cam.fy) / tzs
    J[:, 1, 2] = -F32(cam.fy) * t[:, 1] / (tzs * tzs)
    T = J @ Rw
    S2 = T @ Sig @ T.transpose(0, 2, 1)
    ca, cb, cc = S2[:, 0, 0] + F32(0.3), S2[:, 0, 1], S2[:, 1, 1] + F32(0.3)
    det = ca * cc - cb * cb
    vis &= det > 0
    dets = np.where(vis, det, F32(1))
    conic = np.stack([cc / dets, -cb / dets, ca / dets], 1)
    mid = F32(0.5) * (ca + cc)
    lam = mid + np.sqrt(np.maximum(F32(0.1), mid * mid - det))
    radius = np.ceil(F32(3) * np.sqrt(lam))
    u = F32(cam.fx) * t[:, 0] / tzs + F32(cam.cx)
    v = F32(cam.fy) * t[:, 1] / tzs + F32(cam.cy)
    tx_n = (cam.width + TILE - 1) // TILE
    ty_n = (cam.height + TILE - 1) // TILE
    x0 = np.clip(np.floor((u - radius) / F32(TILE)), 0, tx_n).astype(np.int64)
    x1 = np.clip(np.floor((u + radius) / F32(TILE)) + 1, 0, tx_n).astype(np.int64)
    y0 = np.clip(np.floor((v - radius) / F32(TILE)), 0, ty_n).astype(np.int64)
    y1 = np.clip(np.floor((v + radius) / F32(TILE)) + 1, 0, ty_n).astype(np.int64)
    vis &= (x1 > x0) & (y1 > y0)
    d = p - cam.origin.astype(F32)
    d = d / np.sqrt((d * d).sum(axis=1, keepdims=True)).astype(F32)
    Y = sh_basis(d)                                                   # [n, 16]
    colour = np.empty((n, 3), F32)
    for ch in range(3):
        coef = np.concatenate([a[ch:ch + 1].T, a[3 + 15 * ch:3 + 15 * (ch + 1)].T], axis=1)  # [n, 16]
        colour[:, ch] = np.maximum(F32(0.5) + (coef * Y).sum(axis=1, dtype=F32), F32(0))
    opacity = F32(1) / (F32(1) + np.exp(-a[48]))
    return dict(u=u, v=v, conic=conic, radius=radius, x0=x0, x1=x1, y0=y0, y1=y1, depth=tz, colour=colour,
                opacity=opacity, vis=vis)


def render(pos: np.ndarray, attr: np.ndarray, cam: Camera, pixels=None) -> np.ndarray:
    """The image [3, H, W] (float32), or the listed pixels [(x, y), ...] as [k, 3]."""
    g = preprocess(pos, attr, cam)
    H, W = cam.height, cam.width
    order = np.lexsort((np.arange(len(g["depth"])), g["depth"]))      # by depth, then index
    if pixels is None:
        pixels = [(x, y) for y in range(H) for x in range(W)]
    out = np.zeros((len(pixels), 3), F32)
    for k, (px, py) in enumerate(pixels):
        tx, ty = px // TILE, py // TILE
        sel = order[g["vis"][order] & (g["x0"][order] <= tx) & (tx < g["x1"][order]) &
                    (g["y0"][order] <= ty) & (ty < g["y1"][order])]
        T = F32(1)
        c = np.zeros(3, F32)
        for i in sel:
            dx = g["u"][i] - F32(px)
            dy = g["v"][i] - F32(py)
            A, B, C = g["conic"][i]
            power = F32(-0.5) * (A * dx * dx + C * dy * dy) - B * dx * dy
            if power > 0:
                continue
            alpha = min(F32(0.99), g["opacity"][i] * np.exp(power))
            if alpha < F32(1.0 / 255.0):
                continue
            test_t = T * (F32(1) - alpha)
            if test_t < F32(0.0001):
                break
            c = c + g["colour"][i] * (alpha * T)
            T = test_t
        out[k] = c
    if len(pixels) == H * W:
        return out.reshape(H, W, 3).transpose(2, 0, 1)
    return out
