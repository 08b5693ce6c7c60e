"""Pins of the oracle's spatial tree of guide samples (Sec. 5.6): a hand-worked
one-dimensional case, invariants on random 6-D samples (every sample is its
own leaf's, inside that leaf's box, leaves at most T = floor(sqrt(|S|)) own
samples, the leaf boxes tile the root box, a query lands in the sample's
leaf), flat axes never cut, and coincident positions end at the depth limit."""
import math

import numpy as np

from oracle.stree import MAX_DEPTH, STree


def _line(n):
    p = np.zeros((n, 6), np.float32)
    p[:, 0] = np.arange(n, dtype=np.float64) / (n - 1)
    p[:, 2] = -1.5  # receiver plane
    p[:, 5] = 4.0   # light plane
    return p


def test_hand_worked_line():
    t = STree(_line(64))
    assert t.T == 8
    # midpoint splits of [0, 1] three levels deep: eight leaves of eight samples
    assert t.n_leaves == 8
    for j in range(8):
        assert list(t.leaf_own[j]) == list(range(8 * j, 8 * j + 8))
    # the last split of each leaf's parent (16 own samples) copies floor(0.1 16) = 1
    # sample of the sibling nearest to the plane into each side
    assert list(t.leaf_members[0]) == list(range(0, 9))
    assert list(t.leaf_members[1]) == list(range(7, 16))
    # the root split (64 samples) copies 6 across the plane into the children,
    # which do not pass them on
    assert all(32 not in m for m in t.leaf_members[:4])
    assert list(t.leaf_members[3]) == list(range(23, 32))
    ax = np.array(t.axis)
    assert np.all(ax[ax >= 0] == 0)  # the only axis with extent
    assert list(t.query(_line(64))) == [i // 8 for i in range(64)]


def test_invariants_on_random_samples():
    rng = np.random.default_rng(11)
    n = 1000
    p = np.zeros((n, 6), np.float32)
    p[:, 0:2] = rng.uniform(-2, 2, (n, 2))
    p[:, 2] = -1.5
    p[:, 3:5] = rng.uniform(-0.1, 0.1, (n, 2))
    p[:, 5] = 4.0
    t = STree(p)
    assert t.T == int(math.floor(math.sqrt(n)))
    own = np.concatenate(t.leaf_own)
    assert np.array_equal(np.sort(own), np.arange(n))  # each sample is own in exactly one leaf
    lo0, hi0 = p.astype(np.float64).min(axis=0), p.astype(np.float64).max(axis=0)
    vol = 0.0
    for j in range(t.n_leaves):
        lo, hi = t.leaf_box[j]
        q = p[t.leaf_own[j]].astype(np.float64)
        assert np.all(q >= lo) and np.all((q < hi) | (hi == hi0))
        assert t.leaf_own[j].size <= t.T
        extra = np.setdiff1d(t.leaf_members[j], t.leaf_own[j])
        assert extra.size <= math.floor(0.1 * 2 * t.T + 0.1 * n)  # copies from one split
        ext = np.where(hi0 > lo0, (hi - lo) / np.where(hi0 > lo0, hi0 - lo0, 1), 1.0)
        vol += float(np.prod(ext))
    assert abs(vol - 1.0) < 1e-9  # the leaf boxes tile the root box
    leaf_of = np.empty(n, np.int64)
    for j, o in enumerate(t.leaf_own):
        leaf_of[o] = j
    assert np.array_equal(t.query(p), leaf_of)
    # the receiver and light planes are never cut
    ax = np.array(t.axis)
    assert not np.any((ax == 2) | (ax == 5))


def test_coincident_samples_end_at_the_depth_limit():
    p = np.tile(np.array([[0.1, 0.2, -1.5, 0.0, 0.0, 4.0]], np.float32), (50, 1))
    p = np.concatenate([p, np.array([[0.9, 0.9, -1.5, 0.05, 0.05, 4.0]], np.float32)])
    t = STree(p)
    assert t.T == 7
    big = max(o.size for o in t.leaf_own)
    assert big == 50  # cannot be split: held by one leaf at the depth limit
    depth = 0
    i = 0
    while t.axis[i] >= 0:
        i = t.left[i] if p[0, t.axis[i]] < t.split[i] else t.right[i]
        depth += 1
    assert depth == MAX_DEPTH


def test_per_chain_cells_equal_point_cells_when_they_agree():
    """Seeds, sampled lengths and trials take a chain's own cell when given;
    with every chain on its point's cell the results are those of the
    per-point path."""
    from oracle import oracle as O
    from paper_2311_12818_gb300 import inputs as I
    wl = I.mixed(nx=32, ny=16, spq=8)
    recs = I.synthetic_guide_records(wl, per_cell=64)
    g = O.VmfGuide(wl.n_cells).build(*recs, wl.params.weight_shift)
    cc = np.repeat(wl.cell, wl.spq).astype(np.uint32)
    k1, p1 = O.sample_lengths(wl, g, I.GEOMETRIC_K_WEIGHTS, rng_offset=5)
    k2, p2 = O.sample_lengths(wl, g, I.GEOMETRIC_K_WEIGHTS, rng_offset=5, chain_cell=cc)
    assert np.array_equal(k1, k2) and np.array_equal(p1, p2)
    sc = O.Scene(wl)
    a = O.sample_seeds(wl, sc, g, rng_offset=5)
    b = O.sample_seeds(wl, sc, g, rng_offset=5, chain_cell=cc)
    assert all(np.array_equal(a[f], b[f]) for f in ("x", "surf", "tau", "pdf", "valid"))
    # and a different cell for some chains changes exactly their draws' guide
    cc2 = cc.copy()
    cc2[::7] = (cc2[::7] + 1) % wl.n_cells
    c = O.sample_seeds(wl, sc, g, rng_offset=5, chain_cell=cc2)
    same = np.ones(wl.B, bool)
    same[::7] = False
    assert np.array_equal(a["pdf"][same], c["pdf"][same])
    assert not np.array_equal(a["pdf"][~same], c["pdf"][~same])
