"""Pins of the oracle renderer (3DGS tile splatting of the decoded scene): spherical harmonic
basis, projection, alpha compositing, thresholds and depth order, against closed forms."""
import math

import numpy as np

from oracle import render as R


def _cam(w=64, h=48):
    return R.look_at([0, 0, -2], [0, 0, 0], [0, -1, 0], w, h, 60.0)


def _scene(points):
    """Gaussians at `points` [(x, y, z, log_scale, opacity_logit, dc_r)], identity rotation,
    no higher SH."""
    n = len(points)
    pos = np.array([p[:3] for p in points], np.float32).T
    attr = np.zeros((56, n), np.float32)
    for i, p in enumerate(points):
        attr[49:52, i] = p[3]
        attr[48, i] = p[4]
        attr[0, i] = p[5]
        attr[52, i] = 1.0
    return pos, attr


def test_sh_basis_is_orthonormal():
    """The 16 real harmonics integrate to the identity over the sphere (Fibonacci quadrature),
    which fixes every normalisation constant and sign pattern up to the basis' own symmetry."""
    n = 200_000
    k = np.arange(n) + 0.5
    zc = 1 - 2 * k / n
    phi = math.pi * (1 + 5 ** 0.5) * k
    r = np.sqrt(1 - zc * zc)
    d = np.stack([r * np.cos(phi), r * np.sin(phi), zc], 1).astype(np.float32)
    Y = R.sh_basis(d).astype(np.float64)
    G = Y.T @ Y * (4 * math.pi / n)
    assert np.max(np.abs(G - np.eye(16))) < 2e-3


def test_projection_of_an_axis_aligned_gaussian():
    cam = _cam()
    s = math.exp(-3.0)
    pos, attr = _scene([(0.0, 0.0, 0.0, -3.0, 0.0, 0.0)])
    attr[49:52, 0] = [-3.0, -2.5, -4.0]
    g = R.preprocess(pos, attr, cam)
    f, z = cam.fx, 2.0
    sx, sy = math.exp(-3.0), math.exp(-2.5)
    a, c = (f * sx / z) ** 2 + 0.3, (f * sy / z) ** 2 + 0.3
    assert np.allclose(g["conic"][0], [1 / a, 0.0, 1 / c], rtol=1e-5)
    assert g["radius"][0] == math.ceil(3 * math.sqrt(max(a, c)))
    assert abs(g["u"][0] - cam.cx) < 1e-5 and abs(g["v"][0] - cam.cy) < 1e-5 and abs(g["depth"][0] - 2.0) < 1e-6


def test_single_gaussian_pixels_closed_form():
    """At the mean the pixel is colour x opacity; one pixel away the Gaussian falls off as
    exp(-dx^2 / (2 sigma'^2))."""
    cam = _cam()
    pos, attr = _scene([(0.0, 0.0, 0.0, -3.0, 0.0, 1.0)])  # opacity 0.5
    colour = 0.5 + 0.5 / math.sqrt(math.pi) * 1.0
    img = R.render(pos, attr, cam)
    x0, y0 = int(cam.cx), int(cam.cy)
    sig2 = (cam.fx * math.exp(-3.0) / 2.0) ** 2 + 0.3
    assert abs(img[0, y0, x0] - colour * 0.5) < 1e-6
    assert abs(img[0, y0, x0 + 1] - colour * 0.5 * math.exp(-0.5 / sig2)) < 1e-6
    # green and blue have no coefficient: colour 0.5 (the SH offset)
    assert abs(img[1, y0, x0] - 0.25) < 1e-6 and abs(img[2, y0, x0] - 0.25) < 1e-6
    assert img[0, 0, 0] == 0  # far corner: outside the Gaussian's tiles


def test_front_to_back_compositing_and_input_order():
    """Two Gaussians on the axis: C = c1 a1 + c2 a2 (1 - a1) with the nearer one first, in
    whatever order they are given."""
    cam = _cam()
    pts = [(0.0, 0.0, 0.5, -3.0, 1.0, 1.0), (0.0, 0.0, -0.5, -3.0, 0.0, -1.0)]
    pos, attr = _scene(pts)
    img = R.render(pos, attr, cam)
    pos2, attr2 = _scene(pts[::-1])
    assert np.array_equal(img, R.render(pos2, attr2, cam))
    x0, y0 = int(cam.cx), int(cam.cy)
    c0 = 0.5 / math.sqrt(math.pi)
    a_near, c_near = 0.5, 0.5 - c0           # z = -0.5 is nearer (camera at z = -2)
    a_far, c_far = 1 / (1 + math.exp(-1)), 0.5 + c0
    want = c_near * a_near + c_far * a_far * (1 - a_near)
    assert abs(img[0, y0, x0] - want) < 2e-6


def test_thresholds():
    """Alpha below 1/255 adds nothing; a stack of dense Gaussians (alpha 0.98) stops before
    the one that would bring the transmittance below 1e-4 (0.02^3 = 8e-6), after adding two."""
    cam = _cam()
    faint = _scene([(0.0, 0.0, 0.0, -3.0, -math.log(300 - 1), 1.0)])  # opacity 1/300
    assert R.render(*faint, cam).max() == 0
    logit = math.log(0.98 / 0.02)
    stack = [(0.0, 0.0, z, -3.0, logit, v) for z, v in ((-0.5, 1.0), (0.0, 2.0), (0.5, 3.0))]
    img = R.render(*_scene(stack), cam)
    x0, y0 = int(cam.cx), int(cam.cy)
    c0 = 0.5 / math.sqrt(math.pi)
    want = (0.5 + c0) * 0.98 + (0.5 + 2 * c0) * 0.98 * 0.02
    assert abs(img[0, y0, x0] - want) < 2e-6
