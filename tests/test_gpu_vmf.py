"""vMF mixture guide of Sec. 5.5 (Eq. vMF) on the GPU against the oracle.

Both sides build the lobes from the same records (the oracle's own training
pass): cell starts, keys and weight prefix sums must be bit-exact, mu exact
(copies of the FP32 records) and kappa within FP32 rounding (1e-5 relative).
Sampled chain lengths are integer decisions (bit-exact, P(n) to 1e-6).
Guided seeds, walks, contributions and Bernoulli trial counts follow the
tolerances of the other pipeline tests."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2311_12818_gb300 import inputs as I  # noqa: E402
from test_gpu_parity import _assert_T_max, _compare_seeds, _compare_walk, _params, _polished  # noqa: E402


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


def _records(wl):
    """Training pass with p_0 in the oracle; its records with types."""
    sc = O.Scene(wl)
    seeds = O.sample_seeds(wl, sc)
    ch = O.walk(wl, sc, seeds)
    con = O.contribution(wl, sc, ch)
    N, _ = O.bernoulli(wl, sc, ch, con["admissible"])
    return O.records(wl, ch, con["T"], N, con["admissible"], with_types=True)


def _dev_records(recs):
    cell, om, w, k, tau = recs
    d = "cuda"
    return (torch.as_tensor(cell.astype(np.int32), device=d), torch.as_tensor(np.ascontiguousarray(om.T), device=d),
            torch.as_tensor(w, device=d), torch.as_tensor(k, device=d), torch.as_tensor(tau, device=d))


def _build_both(M, ctx, wl, recs, capacity=None):
    og = O.VmfGuide(wl.n_cells).build(*recs, wl.params.weight_shift)
    R = recs[0].size
    gg = M.VmfGuide(wl.n_cells, capacity or R)
    M.mpg_vmf_build(ctx, gg, *_dev_records(recs), weight_shift=wl.params.weight_shift)
    ctx.sync()
    return og, gg


def _compare_guides(og, gg):
    L = og.n_lobes
    assert gg.n_lobes == L
    assert np.array_equal(gg.cell_start.cpu().numpy().view(np.uint32), og.cell_start)
    assert np.array_equal(gg.lobe_key[:L].cpu().numpy().view(np.uint32), og.key[:L])
    assert np.array_equal(gg.lobe_prefix[:L].cpu().numpy().view(np.uint64), og.prefix[:L])
    lobe = gg.lobe[:L].cpu().numpy().astype(np.float64)
    assert np.array_equal(lobe[:, :3], og.lobe[:L, :3])
    assert np.allclose(lobe[:, 3], og.lobe[:L, 3], rtol=1e-5, atol=0)


@pytest.fixture(scope="module")
def mixed_small():
    wl = I.mixed(nx=64, ny=32, spq=8)
    return wl, _records(wl)


@pytest.fixture(scope="module")
def glass_small():
    wl = I.glass_sphere(n=32, spq=16)
    return wl, _records(wl)


def test_vmf_build_matches_oracle(M, ctx, mixed_small, glass_small):
    for wl, recs in (mixed_small, glass_small):
        assert recs[0].size > 300
        og, gg = _build_both(M, ctx, wl, recs)
        _compare_guides(og, gg)
    # the mixed records span several lengths and types per cell
    og, _ = _build_both(M, ctx, *mixed_small)
    assert len(np.unique(og.key[:og.n_lobes])) > 10


def test_vmf_build_keeps_record_order_and_flags_bad_records(M, ctx, glass_small):
    wl, recs = glass_small
    cell, om, w, k, tau = recs
    R = cell.size
    bad = R // 3
    # an out-of-range cell and a type beyond the length, inserted mid-stream
    ins = lambda a, v: np.insert(a, [bad, bad + 1], v, axis=0)  # noqa: E731
    recs_bad = (ins(cell, [wl.n_cells, 0]), ins(om, [[0, 0, 1], [0, 0, 1]]).astype(np.float32),
                ins(w, [1.0, 1.0]).astype(np.float32), ins(k, [2, 1]).astype(np.uint8),
                ins(tau, [3, 2]).astype(np.uint8))
    gg = M.VmfGuide(wl.n_cells, R + 2)
    M.mpg_vmf_build(ctx, gg, *_dev_records(recs_bad), weight_shift=wl.params.weight_shift)
    with pytest.raises(M.MpgError):
        ctx.sync()
    og = O.VmfGuide(wl.n_cells).build(*recs, wl.params.weight_shift)
    _compare_guides(og, gg)
    # the record count on the device bounds the records read
    gg2 = M.VmfGuide(wl.n_cells, R)
    Rd = torch.tensor([R // 2], dtype=torch.int32, device="cuda")
    M.mpg_vmf_build(ctx, gg2, *_dev_records(recs), R=R, R_dev=Rd, weight_shift=wl.params.weight_shift)
    ctx.sync()
    og2 = O.VmfGuide(wl.n_cells).build(*(a[:R // 2] for a in recs), wl.params.weight_shift)
    _compare_guides(og2, gg2)
    # an empty build leaves no lobes
    gg3 = M.VmfGuide(wl.n_cells, 16)
    M.mpg_vmf_build(ctx, gg3, *_dev_records(tuple(a[:0] for a in recs)), weight_shift=16)
    ctx.sync()
    assert gg3.n_lobes == 0


def test_sampled_lengths_match_oracle(M, ctx, mixed_small):
    wl, recs = mixed_small
    og, gg = _build_both(M, ctx, wl, recs)
    P = _params(M, wl)
    ch = M.Chains(wl)
    p0w = I.GEOMETRIC_K_WEIGHTS
    for guide_o, guide_g, off in ((og, gg, 0), (None, None, 12345)):
        k, pn = M.mpg_sample_lengths(ctx, guide_g, ch, p0w, P, wl.rng_seed, off)
        ctx.sync()
        ok, opn = O.sample_lengths(wl, guide_o, p0w, rng_offset=off)
        assert np.array_equal(k.cpu().numpy(), ok)
        assert np.allclose(pn.cpu().numpy(), opn, rtol=1e-6, atol=0)
        assert len(np.unique(ok)) == 8


def _guided_pipelines(M, ctx, wl, og, gg, sample_lengths):
    off = 1 << 24
    if sample_lengths:
        ok, opn = O.sample_lengths(wl, og, I.GEOMETRIC_K_WEIGHTS, rng_offset=off)
        wl = dataclasses.replace(wl, k=ok, pn=opn)
    ch = M.Chains(wl)
    P = _params(M, wl, k_uniform=0 if sample_lengths else int(wl.k[0]))
    sc = M.Scene(ctx, wl)
    if sample_lengths:
        k, pn = M.mpg_sample_lengths(ctx, gg, ch, I.GEOMETRIC_K_WEIGHTS, P, wl.rng_seed, off, out=(ch.k, ch.pn))
        ctx.sync()
        assert np.array_equal(k.cpu().numpy(), wl.k)
    M.mpg_sample_seeds(ctx, sc, gg, ch, P, wl.rng_seed, off)
    gs = ch.aos()
    M.mpg_manifold_walk(ctx, sc, ch, P)
    gw = ch.aos()
    out = M.mpg_chain_contribution(ctx, sc, gg, ch, P, wl.rng_seed, off)
    ctx.sync()
    osc = O.Scene(wl)
    seeds = O.sample_seeds(wl, osc, og, rng_offset=off)
    och = O.walk(wl, osc, seeds)
    con = O.contribution(wl, osc, och)
    N, _ = O.bernoulli(wl, osc, och, con["admissible"], og, rng_offset=off)
    return wl, gs, gw, out, seeds, och, _polished(wl, osc, och, con), N


@pytest.mark.parametrize("which", ["mixed", "glass"])
def test_vmf_guided_pipeline_parity(M, ctx, which, mixed_small, glass_small):
    wl, recs = mixed_small if which == "mixed" else glass_small
    og, gg = _build_both(M, ctx, wl, recs)
    wl, gs, gw, out, os_, ow, con, N = _guided_pipelines(M, ctx, wl, og, gg, sample_lengths=which == "mixed")
    _compare_seeds(wl, gs, os_)
    both = _compare_walk(wl, gw, ow)
    G = out.G.cpu().numpy()
    ab = (G > 0) & (con["admissible"] == 1) & both
    assert ab.sum() > 200
    _assert_T_max(wl, out.T.cpu().numpy(), con["T"], ab)
    gN = out.trials.cpu().numpy().astype(np.int64)
    assert (gN[ab] == N[ab]).mean() >= 0.999


def test_vmf_step_captured_in_a_graph(M, ctx, mixed_small):
    wl, recs = mixed_small
    sc = M.Scene(ctx, wl)
    ch = M.Chains(wl)
    P = _params(M, wl, k_uniform=0)
    res = M.Contribution.empty(wl.B, wl.Q)
    rec = M.mpg_guide_records(ctx, sc, ch, res.contrib, with_types=True)
    gA, gB = M.VmfGuide(wl.n_cells, wl.B), M.VmfGuide(wl.n_cells, wl.B)
    M.mpg_vmf_build(ctx, gA, *_dev_records(recs), weight_shift=wl.params.weight_shift)

    def step(off):
        M.mpg_sample_lengths(ctx, gA, ch, I.GEOMETRIC_K_WEIGHTS, P, wl.rng_seed, off, out=(ch.k, ch.pn))
        M.mpg_sample_seeds(ctx, sc, gA, ch, P, wl.rng_seed, off)
        M.mpg_manifold_walk(ctx, sc, ch, P)
        M.mpg_chain_contribution(ctx, sc, gA, ch, P, wl.rng_seed, off, out=res)
        M.mpg_guide_records(ctx, sc, ch, res.contrib, out=rec)
        M.mpg_vmf_build(ctx, gB, rec[0], rec[1], rec[2], rec[3], rec[4], R=wl.B, R_dev=rec[5],
                        weight_shift=wl.params.weight_shift)

    off = 5 * wl.B
    step(off)
    ctx.sync()
    ref = [t.clone() for t in (res.contrib, ch.k, gB.cell_start, gB.lobe_key, gB.lobe, gB.lobe_prefix)]
    assert int(rec[5][0].item()) == int((res.contrib > 0).sum().item()) > 100
    for t in (res.contrib, gB.lobe, gB.lobe_prefix):
        t.zero_()
    g = M.Graph(ctx, rng_advance=wl.B)
    with g:
        step(off)
    g.launch()
    ctx.sync()
    now = (res.contrib, ch.k, gB.cell_start, gB.lobe_key, gB.lobe, gB.lobe_prefix)
    for a, b in zip(ref, now):
        assert torch.equal(a, b)
