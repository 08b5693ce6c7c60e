"""The library's host builds of the spatial tree (Sec. 5.6) against the
oracle's tree, without a GPU (mpg_stree_build_host).

The recursive build partitions in place with linear-time selection and
builds the two subtrees of large nodes near the root on threads of their
own.  The level build runs the passes of the device build as host loops:
all split nodes of a level partitioned at once by prefix counts, all their
copies selected at once by digits of the distances' bit patterns.  The
oracle partitions with boolean masks and sorts.  Nodes, splits and leaf
members must be identical on seeded position sets shaped like the guide's
samples (x_D on a receiver plane, x_L on a small light), large enough that
the threaded subtrees run, with duplicated positions (ties in the copies'
distance to the plane), and on the degenerate sets (no sample, one sample,
all samples at one position, a flat axis)."""
import numpy as np
import pytest

from oracle.stree import STree


@pytest.fixture(scope="module")
def M():
    from paper_2311_12818_gb300 import build, mpg
    build.build()
    return mpg


def _planar(n, seed, dup=0.0):
    """x_D uniform on the receiver square [-2, 2]^2 at z = -1.5, x_L uniform on
    a 0.2 x 0.2 light at z = 4 (FP32); a fraction `dup` repeats earlier rows."""
    rng = np.random.default_rng(seed)
    p = np.zeros((n, 6), np.float32)
    p[:, 0:2] = rng.uniform(-2.0, 2.0, (n, 2))
    p[:, 2] = -1.5
    p[:, 3:5] = rng.uniform(-0.1, 0.1, (n, 2))
    p[:, 5] = 4.0
    if dup > 0 and n > 1:
        m = int(dup * n)
        p[n - m:] = p[rng.integers(0, n - m, m)]
    return p


METHODS = ["recursive", "levels"]


def _same(M, pos, eps=0.1, c=1.0, method="recursive"):
    ht = M.STree.from_host(pos, epsilon=eps, c=c,
                           method=M.STREE_LEVELS if method == "levels" else M.STREE_RECURSIVE)
    ot = STree(pos, eps=eps, c=c)
    ax, sp, lf, rt, ml, mr = ht.export()
    assert ht.n_samples == pos.shape[0]
    assert ht.n_leaves == ot.n_leaves and ht.n_nodes == len(ot.axis)
    assert np.array_equal(ax, ot.axis) and np.array_equal(sp, ot.split)
    assert np.array_equal(lf, ot.left) and np.array_equal(rt, ot.right)
    leaf = np.concatenate([np.full(m.size, j) for j, m in enumerate(ot.leaf_members)])
    assert np.array_equal(ml, leaf) and np.array_equal(mr, np.concatenate(ot.leaf_members))
    return ht, ot


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("n,seed,dup", [(700, 1, 0.0), (20000, 2, 0.0), (12000, 3, 0.25)])
def test_host_build_matches_oracle(M, n, seed, dup, method):
    ht, ot = _same(M, _planar(n, seed, dup), method=method)
    assert ht.n_leaves > 8
    # no leaf reaches the depth limit here: every leaf holds at most T own samples
    T = int(np.floor(np.sqrt(n)))
    assert max(len(o) for o in ot.leaf_own) <= T


@pytest.mark.parametrize("method", METHODS)
def test_quantised_positions_tie_at_the_copy_boundary(M, method):
    """Coordinates on a coarse grid: many samples share their distance to a
    split plane, so the copies are cut inside runs of equal distances and the
    record index decides."""
    p = _planar(30000, 9)
    p[:, 0:2] = np.round(p[:, 0:2] * 8) / 8
    p[:, 3:5] = np.round(p[:, 3:5] * 40) / 40
    ht, ot = _same(M, p, method=method)
    assert ht.n_leaves > 8


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("eps,c", [(0.0, 1.0), (0.25, 0.5), (0.1, 3.0)])
def test_host_build_matches_oracle_other_parameters(M, eps, c, method):
    _same(M, _planar(5000, 7), eps=eps, c=c, method=method)


@pytest.mark.parametrize("method", METHODS)
def test_degenerate_sets(M, method):
    ht, _ = _same(M, np.zeros((0, 6), np.float32), method=method)
    assert ht.n_leaves == 1 and ht.n_members == 0
    ht, _ = _same(M, _planar(1, 4), method=method)
    assert ht.n_leaves == 1 and ht.n_members == 1
    same = np.tile(_planar(1, 5), (50, 1))  # no extent on any axis: one leaf
    ht, _ = _same(M, same, method=method)
    assert ht.n_leaves == 1 and ht.n_members == 50
    flat = _planar(3000, 6)
    flat[:, 3:5] = 0.0  # a point light: the light-side axes never split
    ht, ot = _same(M, flat, method=method)
    ax = np.asarray(ot.axis)
    assert not np.isin(ax, [2, 3, 4, 5]).any()


def test_rejected_arguments(M):
    L = M.lib()
    import ctypes as C
    h = C.c_void_p()
    assert L.mpg_stree_build_host(None, 4, 0.1, 1.0, 0, C.byref(h)) == M.MPG_ERR_INVALID_ARG
    pos = np.zeros((6, 4), np.float32)
    assert L.mpg_stree_build_host(pos.ctypes.data, -1, 0.1, 1.0, 0, C.byref(h)) == M.MPG_ERR_INVALID_ARG
    assert L.mpg_stree_build_host(pos.ctypes.data, 4, 0.5, 1.0, 0, C.byref(h)) == M.MPG_ERR_INVALID_ARG
    assert L.mpg_stree_build_host(pos.ctypes.data, 4, 0.1, 0.0, 0, C.byref(h)) == M.MPG_ERR_INVALID_ARG
    assert L.mpg_stree_build_host(pos.ctypes.data, 4, 0.1, 1.0, 2, C.byref(h)) == M.MPG_ERR_INVALID_ARG
    assert b"method" in L.mpg_last_error()
    pos[3, 2] = np.nan
    assert L.mpg_stree_build_host(pos.ctypes.data, 4, 0.1, 1.0, 1, C.byref(h)) == M.MPG_ERR_INVALID_ARG
    assert b"not finite" in L.mpg_last_error()
    # a host-only tree has no device copy: queries and records are refused
    t = M.STree.from_host(_planar(64, 8))
    assert L.mpg_stree_query(None, t.h, None, None, None) == M.MPG_ERR_INVALID_ARG
    assert b"no device copy" in L.mpg_last_error()
    assert L.mpg_stree_records(None, t.h, None, None, None, None, 0, None, None, None, None, None, 0, None,
                               None) == M.MPG_ERR_INVALID_ARG
    assert b"no device copy" in L.mpg_last_error()
