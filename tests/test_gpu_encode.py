"""The encoder's scene preparation on the device (prune, voxelize, Morton sort, unique voxels and
duplicates, octree tokens, per-channel quantization; Sec. 3.3-3.4): with a context,
`scene_encode` prepares on the GPU, without one on the host cores, and both write the oracle's
bytes, including every tie-break the bitstream depends on."""
import numpy as np
import pytest

from oracle import scene as S
from paper_2607_12656_b300 import sgs
from paper_2607_12656_b300.scenegen import fixed_bits, make_scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = sgs.Context(0, 1 << 20)
    yield c
    c.close()


def _same_three(ctx, pos, attr, **kw):
    want = S.encode(pos, attr, **kw)
    dev = sgs.scene_encode(pos, attr, ctx=ctx, **kw)
    host = sgs.scene_encode(pos, attr, **kw)
    assert dev == host, "device and host preparation differ"
    assert dev == want, "bitstream differs from the oracle's"


def _tricky_scene(n, seed):
    """Ties in opacity (with -0.0 and +0.0 among them), several Gaussians per voxel, a constant
    channel, a channel whose minimum is -0.0 and one whose minimum comes both signed."""
    sc = make_scene(n, seed)
    pos, attr = sc.pos.copy(), sc.attr.copy()
    rng = np.random.default_rng(seed)
    attr[48, : n // 3] = rng.choice(np.array([-1.0, -0.0, 0.0, 2.5], np.float32), n // 3)
    if n >= 40:
        k = n // 5
        pos[:, k: 2 * k] = pos[:, :1]  # a crowd in one voxel
        pos[:, 2 * k: 2 * k + 7] = pos[:, 5:6]
    attr[3, :] = 0.75
    attr[4, :] = np.abs(attr[4, :]) + 1.0
    attr[4, rng.integers(0, n, 9)] = -0.0
    attr[5, :] = np.abs(attr[5, :])
    attr[5, rng.integers(0, n, 5)] = -0.0
    attr[5, rng.integers(0, n, 5)] = 0.0
    return pos, attr


@pytest.mark.parametrize("n", [0, 1, 9, 10, 37, 20_000])
def test_prepare_static_edge_cases(ctx, n):
    if n == 0:
        pos, attr = np.zeros((3, 0), np.float32), np.zeros((56, 0), np.float32)
    else:
        pos, attr = _tricky_scene(n, 500 + n)
    _same_three(ctx, pos, attr, mode=S.MODE_STATIC, depth=12, lanes=33)


@pytest.mark.parametrize("depth", [1, 7, 11, 16, 21])
def test_prepare_depths_fixed_length(ctx, depth):
    """Morton codes that fit the low word, that span both words, and the 63-bit limit; fixed
    widths from 1 to 16 bits."""
    pos, attr = _tricky_scene(30_000, 600 + depth)
    bits = fixed_bits(depth)
    bits[0], bits[1] = 1, 16
    _same_three(ctx, pos, attr, mode=S.MODE_FIXED, depth=depth, bits=bits)


def test_prepare_large_scene_geometry_coded(ctx):
    """A 1M-Gaussian scene with rANS-coded octree levels: the prepared rows, octree and
    quantization behind the whole bitstream."""
    sc = make_scene(1_000_000, 1000)
    _same_three(ctx, sc.pos, sc.attr, mode=S.MODE_STATIC, depth=16, lanes=4096, geo_mode=S.GEO_RANS)


def test_prepare_refuses_what_the_host_refuses(ctx):
    pos, attr = _tricky_scene(100, 7)
    bad_pos = pos.copy()
    bad_pos[1, 3] = 1.0
    bad_attr = attr.copy()
    bad_attr[10, 50] = np.nan
    for p, a in ((bad_pos, attr), (pos, bad_attr)):
        with pytest.raises(sgs.SgsError) as e:
            sgs.scene_encode(p, a, ctx=ctx, mode=sgs.MODE_STATIC, depth=10, lanes=8)
        assert e.value.code == sgs.E_INVALID
