"""The element-wise training tolerance catches the mistakes it is meant to catch (planted in
the oracle's fp64 gradients, on the CPU) and passes fp32 rounding of the same values."""
import numpy as np
import pytest

from oracle import model as M
from oracle import scene as S
from paper_2607_12656_b300.scenegen import kaiming_init, make_scene
from tolerance import assert_close


@pytest.fixture(scope="module")
def grads():
    sc = make_scene(3000, 31)
    P = S.prepare(sc.pos, sc.attr, 11, 8)
    q = P.q.astype(np.uint8)
    lr = S.lane_bounds(P.n_rows, 24)
    pos = M.sample_positions(13, 0, 4096, P.n_rows * 56)
    u, c, s, _, _ = M.contexts(q, lr, pos)
    w = {k: np.asarray(v, np.float64) for k, v in kaiming_init(9).items()}
    return M.forward_backward(w, u, c, s)[1]


def test_fp32_rounding_passes(grads):
    for k, g in grads.items():
        assert_close(g.astype(np.float32), g, k)


def test_one_wrong_element_fails(grads):
    g = grads["w3"]
    bad = g.copy()
    i = np.unravel_index(int(np.argmax(np.abs(g))), g.shape)
    bad[i] *= 1.001  # one element 0.1% off
    with pytest.raises(AssertionError):
        assert_close(bad, g, "w3")


def test_one_wrong_row_fails(grads):
    g = grads["emb"]
    bad = g.copy()
    bad[7] = 0.0  # one channel's embedding gradient dropped
    with pytest.raises(AssertionError):
        assert_close(bad, g, "emb")


def test_sign_flip_of_a_small_element_fails(grads):
    g = grads["b1"]
    bad = g.copy()
    j = int(np.argsort(np.abs(g))[len(g) // 2])  # a median-size element
    bad[j] = -bad[j]
    with pytest.raises(AssertionError):
        assert_close(bad, g, "b1")
