"""The seeded input recipe (synthetic stand-in for the paper's scenes): determinism, the
positions' support, each channel group's marginal, the unit quaternions, and the spatial
correlation that rho sets (a nearest neighbour's value correlates at about rho^2 with rho =
0.8 and not at all with rho = 0)."""
import math

import numpy as np
import pytest

from paper_2607_12656_b300.scenegen import fixed_bits, loguniform_sizes, make_scene


@pytest.fixture(scope="module", params=[0.8, 0.0])
def scene(request):
    return make_scene(200_000, 5, request.param)


def test_deterministic_and_seeded():
    a, b, c = make_scene(5000, 11), make_scene(5000, 11), make_scene(5000, 12)
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.attr, b.attr)
    assert not np.array_equal(a.attr, c.attr)
    e = make_scene(0, 1)
    assert e.pos.shape == (3, 0) and e.attr.shape == (56, 0)


def test_positions_in_the_half_open_cube(scene):
    assert scene.pos.dtype == np.float32 and scene.pos.shape == (3, 200_000)
    assert scene.pos.min() >= 0.0 and scene.pos.max() < 1.0


def test_marginals(scene):
    a = scene.attr.astype(np.float64)
    assert scene.attr.dtype == np.float32 and scene.attr.shape == (56, 200_000)
    assert np.allclose(a[0:3].std(axis=1), 0.5, rtol=0.05)          # SH DC 0.5 z
    assert np.allclose(a[49:52].mean(axis=1), -4.0, atol=0.05)      # log-scales -4 + 0.5 z
    assert np.allclose(a[49:52].std(axis=1), 0.5, rtol=0.05)
    assert a[48].std() == pytest.approx(1.5, rel=0.05)              # opacity logit 1.5 z
    for colour in range(3):
        for k in range(1, 16):                                      # SH rest Laplace(0.1 0.7^band)
            b = 0.1 * 0.7 ** math.isqrt(k)
            assert np.abs(a[3 + 15 * colour + k - 1]).mean() == pytest.approx(b, rel=0.05)
    assert np.abs(np.linalg.norm(a[52:56], axis=0) - 1.0).max() < 1e-6  # unit quaternions


def test_spatial_correlation_follows_rho(scene):
    from scipy.spatial import cKDTree
    _, j = cKDTree(scene.pos.T).query(scene.pos.T, k=2)
    nn = j[:, 1]
    a = scene.attr.astype(np.float64)
    for c in (0, 20, 48, 50):
        r = np.corrcoef(a[c], a[c][nn])[0, 1]
        if scene.rho > 0:
            assert 0.45 < r < 0.72, (c, r)  # rho^2 = 0.64 times the field's correlation at that distance
        else:
            assert abs(r) < 0.02, (c, r)


def test_bit_widths_and_sizes():
    for s in range(20):
        b = fixed_bits(s)
        assert b.dtype == np.uint32 and b.shape == (56,) and b.min() >= 4 and b.max() <= 10
    sz = loguniform_sizes(3000, 64, 5e4, 3e6)
    assert sz.min() >= 50_000 and sz.max() <= 3_000_000
    # log-uniform: the median of many draws sits near the geometric mean
    big = loguniform_sizes(1, 20_000, 5e4, 3e6)
    assert np.median(big) == pytest.approx(math.sqrt(5e4 * 3e6), rel=0.05)
