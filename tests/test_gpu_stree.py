"""Spatial tree of the guide samples (Sec. 5.6) on the GPU path against the
oracle's tree.

Both sides build from the oracle's training records (the chain indices of its
admissible chains, positions from the same FP32 inputs): nodes, splits and
leaf members must be identical, queries of every chain of a new batch too
(FP64 comparisons on both sides).  The leaves' records build the vMF guide
(one cell per leaf) bit-exactly as the cell guides do, and seeds, walks and
trial counts drawn with per-chain leaves follow the usual parity bars."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from oracle.stree import STree, positions  # noqa: E402
from paper_2311_12818_gb300 import inputs as I  # noqa: E402
from test_gpu_parity import _compare_seeds, _compare_walk, _params  # noqa: E402
from test_gpu_vmf import _compare_guides  # noqa: E402


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_12818_gb300 import build, mpg
    build.build()
    return mpg


@pytest.fixture(scope="module")
def ctx(M):
    return M.Context(0)


def _training(wl):
    sc = O.Scene(wl)
    seeds = O.sample_seeds(wl, sc)
    ch = O.walk(wl, sc, seeds)
    con = O.contribution(wl, sc, ch)
    N, _ = O.bernoulli(wl, sc, ch, con["admissible"])
    idx = np.nonzero(con["admissible"])[0]
    return idx, O.records(wl, ch, con["T"], N, con["admissible"], with_types=True)


def _dev(recs):
    cell, om, w, k, tau = recs
    return (torch.as_tensor(cell.astype(np.int32), device="cuda"), torch.as_tensor(np.ascontiguousarray(om.T), device="cuda"),
            torch.as_tensor(w, device="cuda"), torch.as_tensor(k, device="cuda"), torch.as_tensor(tau, device="cuda"))


@pytest.mark.parametrize("method", ["recursive", "levels"])
@pytest.mark.parametrize("which", ["glass", "mixed"])
def test_tree_build_query_and_guide_match_oracle(M, ctx, which, method):
    wl = I.glass_sphere(n=32, spq=16) if which == "glass" else I.mixed(nx=64, ny=32, spq=8)
    idx, recs = _training(wl)
    assert idx.size > 300
    ot = STree(positions(wl, idx))
    ch = M.Chains(wl)
    gt = M.STree(ctx, ch, torch.as_tensor(idx.astype(np.int32), device="cuda"),
                 method=M.STREE_LEVELS if method == "levels" else M.STREE_RECURSIVE)
    ax, sp, lf, rt, ml, mr = gt.export()
    assert gt.n_samples == idx.size and gt.n_leaves == ot.n_leaves > 4
    assert np.array_equal(ax, ot.axis) and np.array_equal(sp, ot.split)
    assert np.array_equal(lf, ot.left) and np.array_equal(rt, ot.right)
    om_leaf = np.concatenate([np.full(m.size, j) for j, m in enumerate(ot.leaf_members)])
    assert np.array_equal(ml, om_leaf) and np.array_equal(mr, np.concatenate(ot.leaf_members))
    # queries of a fresh batch (other light-side points)
    wl2 = dataclasses.replace(wl, xL=I.glass_sphere(n=32, spq=16, seed=99).xL) if which == "glass" else wl
    ch2 = M.Chains(wl2)
    q = gt.query(ch2)
    ctx.sync()
    b = np.arange(wl2.B)
    assert np.array_equal(q.cpu().numpy(), ot.query(positions(wl2, b)))
    # the leaves' records and their vMF guide
    dev = _dev(recs)
    R = idx.size
    lr = gt.records(dev + (None,), R)
    ctx.sync()
    oexp = ot.expand(*recs)
    assert int(lr[5][0].item()) == oexp[0].size == gt.n_members
    og = O.VmfGuide(ot.n_leaves).build(*oexp, wl.params.weight_shift)
    gg = M.VmfGuide(gt.n_leaves, gt.n_members)
    M.mpg_vmf_build(ctx, gg, *lr[:5], R=lr[0].numel(), R_dev=lr[5], weight_shift=wl.params.weight_shift)
    ctx.sync()
    _compare_guides(og, gg)
    # guided seeds, walks and trials with per-chain leaves
    off = 1 << 28
    cells = q.cpu().numpy().astype(np.uint32)
    ch2.chain_cell = q
    P = _params(M, wl2)
    sc = M.Scene(ctx, wl2)
    M.mpg_sample_seeds(ctx, sc, gg, ch2, P, wl2.rng_seed, off)
    gs = ch2.aos()
    M.mpg_manifold_walk(ctx, sc, ch2, P)
    gw = ch2.aos()
    out = M.mpg_chain_contribution(ctx, sc, gg, ch2, P, wl2.rng_seed, off)
    ctx.sync()
    osc = O.Scene(wl2)
    os_ = O.sample_seeds(wl2, osc, og, rng_offset=off, chain_cell=cells)
    ow = O.walk(wl2, osc, os_)
    con = O.contribution(wl2, osc, ow)
    N, _ = O.bernoulli(wl2, osc, ow, con["admissible"], og, rng_offset=off, chain_cell=cells)
    _compare_seeds(wl2, gs, os_)
    both = _compare_walk(wl2, gw, ow)
    G = out.G.cpu().numpy()
    ab = (G > 0) & (con["admissible"] == 1) & both
    assert ab.sum() > 200
    gN = out.trials.cpu().numpy().astype(np.int64)
    assert (gN[ab] == N[ab]).mean() >= 0.999


@pytest.mark.parametrize("n_samples", [1000, 600_000])
def test_level_build_on_device_equals_recursive_build(M, ctx, n_samples):
    """The device's level-by-level build and the depth-first build give the
    same tree (nodes, splits, leaf members) on the benchmark workload's
    positions: a small sample set, then one of the size a training pass of
    the full glass-sphere batch gives.  The depth-first build is the one
    checked against the oracle's tree above."""
    wl = I.glass_sphere()
    ch = M.Chains(wl)
    rng = np.random.default_rng(0x4D50470015 + n_samples)
    idx = np.sort(rng.choice(wl.B, n_samples, replace=False)).astype(np.int32)
    rc = torch.as_tensor(idx, device="cuda")
    a = M.STree(ctx, ch, rc, method=M.STREE_RECURSIVE).export()
    b = M.STree(ctx, ch, rc, method=M.STREE_LEVELS).export()
    ctx.sync()
    assert a[0].size > 10
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
