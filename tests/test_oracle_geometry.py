"""Pins of the oracle's geometry steps (Sec. 3.4, "Geometry Occupancy Coding"; Morton order
of the attribute tokens): octree serialize/expand, Morton codes, pruning, positions."""
import itertools
import os

import numpy as np
import pytest

from oracle import scene as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _morton_by_strings(x, y, z, depth):
    """Independent Morton code: interleave binary digit strings, x first in each triple."""
    bx, by, bz = (format(int(v), "0%db" % depth) for v in (x, y, z))
    return int("".join(a + b + c for a, b, c in zip(bx, by, bz)) or "0", 2)


def test_golden_octree_d2():
    lines = [l for l in open(os.path.join(GOLD, "octree_d2.txt")) if l.strip() and not l.startswith("#")]
    kv = {l.split()[0]: l.split()[1:] for l in lines}
    depth = int(kv["depth"][0])
    vox = np.array([[int(t) for t in v.split(",")] for v in kv["voxels"]], np.uint32).T
    codes = np.unique(S.morton(vox, depth))
    levels = S.octree_levels(codes, depth)
    assert levels[0].tolist() == [int(t) for t in kv["level0"]]
    assert levels[1].tolist() == [int(t) for t in kv["level1"]]
    assert codes.tolist() == [int(t) for t in kv["leaves"]]
    assert S.octree_expand(levels, depth).tolist() == [int(t) for t in kv["leaves"]]
    pos = S.position(S.demorton(codes, depth), depth)
    want = np.array([[float(t) for t in p.split(",")] for p in kv["positions"]], np.float32).T
    assert np.array_equal(pos, want)


def test_morton_matches_string_interleave():
    rng = np.random.default_rng(1)
    for depth in (1, 3, 7, 16, 21):
        c = rng.integers(0, 1 << depth, size=(3, 200)).astype(np.uint32)
        m = S.morton(c, depth)
        for i in range(200):
            assert int(m[i]) == _morton_by_strings(c[0, i], c[1, i], c[2, i], depth)
        assert np.array_equal(S.demorton(m, depth), c)


def test_depth1_all_subsets():
    """Brute force: every non-empty subset of the 8 voxels at depth 1; the root token is the
    subset's bit mask with k = (x<<2)|(y<<1)|z."""
    for mask in range(1, 256):
        ks = [k for k in range(8) if mask >> k & 1]
        vox = np.array([[k >> 2 & 1, k >> 1 & 1, k & 1] for k in ks], np.uint32).T
        codes = np.unique(S.morton(vox, 1))
        levels = S.octree_levels(codes, 1)
        assert levels[0].tolist() == [mask]
        assert S.octree_expand(levels, 1).tolist() == sorted(ks)


@pytest.mark.parametrize("depth", [2, 3, 4, 8, 16])
def test_expand_equals_sorted_unique(depth):
    rng = np.random.default_rng(depth)
    n = 3000
    c = rng.integers(0, 1 << depth, size=(3, n)).astype(np.uint32)
    leaf = np.unique(S.morton(c, depth))
    levels = S.octree_levels(leaf, depth)
    assert levels[0].shape == (1,)
    for l in range(depth - 1):  # sum of popcounts of level l = node count of level l+1
        assert int(np.unpackbits(levels[l]).sum()) == len(levels[l + 1])
    assert int(np.unpackbits(levels[-1]).sum()) == len(leaf)
    assert np.array_equal(S.octree_expand(levels, depth), leaf)
    # textbook reference: sorted unique voxel set, compared in coordinates
    ref = sorted(set(map(tuple, c.T.tolist())), key=lambda v: _morton_by_strings(*v, depth))
    assert np.array_equal(S.demorton(S.octree_expand(levels, depth), depth).T, np.array(ref, np.uint32))


def test_small_scenes_exhaustive_positions():
    """All scenes of k <= 3 Gaussians on a 4x4x4 grid (depth 2): positions of the prepared
    rows are the voxel centres of the inputs in (Morton, index) order."""
    cells = list(itertools.product(range(4), repeat=3))
    rng = np.random.default_rng(3)
    for k in (1, 2, 3):
        combos = list(itertools.combinations(range(64), k)) if k < 3 else \
            [tuple(rng.choice(64, 3, replace=False)) for _ in range(400)]
        for combo in combos:
            vox = np.array([cells[i] for i in combo], np.float64).T
            pos = ((vox + 0.5) / 4.0).astype(np.float32)
            attr = np.zeros((56, k), np.float32)
            attr[48] = np.arange(k, dtype=np.float32)  # k < 10: nothing pruned
            P = S.prepare(pos, attr, 2, 8)
            want = sorted(range(k), key=lambda i: (_morton_by_strings(*vox[:, i].astype(int), 2), i))
            assert P.keep.tolist() == want
            assert np.array_equal(P.pos, pos[:, want])


def test_prune_lowest_opacity_ties_lower_index():
    attr = np.zeros((56, 20), np.float32)
    attr[48] = np.arange(20, dtype=np.float32) + 10
    attr[48, [4, 9, 2]] = -1.0  # three-way tie at the minimum; floor(20/10) = 2 pruned
    keep = S.prune(attr)
    assert sorted(set(range(20)) - set(keep.tolist())) == [2, 4]


def test_duplicates_rows_and_metadata():
    """Several Gaussians in one voxel: one position encoded, duplicates as metadata
    (Sec. 3.4), rows ordered by (Morton code, original index)."""
    rng = np.random.default_rng(5)
    n = 500
    pos = rng.uniform(0, 1, size=(3, n)).astype(np.float32)
    attr = rng.standard_normal((56, n)).astype(np.float32)
    P = S.prepare(pos, attr, 2, 8)
    assert len(P.leaf_codes) <= 64 and P.n_rows == n - n // 10
    assert int(P.dups[:, 1].sum()) + len(P.leaf_codes) == P.n_rows
    assert np.all(np.diff(P.codes.astype(np.int64)) >= 0)
    same = np.diff(P.codes.astype(np.int64)) == 0
    assert np.all(np.diff(P.keep)[same] > 0)


def test_position_exact_voxel_centres():
    for depth in (1, 12, 16, 21):
        c = np.array([[0, (1 << depth) - 1, 5 % (1 << depth)]] * 3, np.uint32)
        p = S.position(c, depth).astype(np.float64)
        assert np.array_equal(p, (c.astype(np.float64) * 2 + 1) / 2.0 ** (depth + 1))
