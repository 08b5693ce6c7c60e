"""Parity at the benchmark's full sizes, in the launch configuration it times.

The glass-sphere step (1,048,576 chains, guided, batched, replayed from a
captured graph) and the mixed-length batch (4,194,304 chains, batched graph)
run whole on the GPU; the oracle then recomputes blocks of chains aligned to
the receiver points -- at the start, in the middle and at the end of the batch.
A block [b0, b0 + n) is a workload of its own whose random-number counters are
those of the full run shifted by b0 (rng_offset + b0), so the oracle redraws
the same seeds and trials and the comparison is chain by chain.  Full-size
properties that need no oracle run are checked over the whole batch."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2311_12818_gb300 import inputs as I  # noqa: E402

BLOCK = 1024


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


def _block(wl, b0, n):
    q0, nq = b0 // wl.spq, n // wl.spq
    return dataclasses.replace(wl, xD=wl.xD[q0:q0 + nq], nD=wl.nD[q0:q0 + nq], cell=wl.cell[q0:q0 + nq],
                               xL=wl.xL[b0:b0 + n], k=wl.k[b0:b0 + n], tau=wl.tau[b0:b0 + n],
                               pn=wl.pn[b0:b0 + n], receiver_shape=(nq, 1))


def _starts(wl):
    B, s = wl.B, wl.spq
    mid = (B // 2) // s * s
    third = (B // 3) // s * s
    return [0, third, mid, B - BLOCK]


def _oracle_block(sub, guide, off):
    """Oracle pipeline on one block: seeds, walk, contribution (of chains
    polished to 1e-12, as in the reduced-size tests) and Bernoulli trials."""
    sc = O.Scene(sub)
    seeds = O.sample_seeds(sub, sc, guide, rng_offset=off)
    ch = O.walk(sub, sc, seeds)
    con = O.contribution(sub, sc, ch)
    N, _ = O.bernoulli(sub, sc, ch, con["admissible"], guide, rng_offset=off)
    tight = dataclasses.replace(sub, params=dataclasses.replace(sub.params, tol=1e-12))
    conv = dict(x=ch["x"], surf=ch["surf"], prim=ch["prim"], bary=ch["bary"], tau=ch["tau"],
                valid=(ch["status"] == 1).astype(np.uint8))
    pol = O.walk(tight, sc, conv)
    pol["status"] = np.where(pol["status"] == 1, ch["status"], 0).astype(np.uint8)
    cp = O.contribution(sub, sc, pol)
    adm = con["admissible"] & (cp["admissible"] | (ch["status"] != 1))
    return seeds, ch, cp["T"], adm.astype(bool), N


def _compare_blocks(M, wl, ch, res, guide_o, off, block=None):
    st = ch.status.cpu().numpy()
    x = ch.x.permute(2, 0, 1).double().cpu().numpy()
    surf = ch.surf.T.contiguous().cpu().numpy()
    T = res.T.cpu().numpy()
    N = res.trials.cpu().numpy().astype(np.int64)
    E = res.E.cpu().numpy()
    flags, same_T, same_N, rel_T, rel_E, dx, worst = [], [], [], [], [], [], []
    for b0 in _starts(wl):
        sl = slice(b0, b0 + BLOCK)
        sub = _block(wl, b0, BLOCK) if block is None else block(b0)
        seeds, och, oT, oadm, oN = _oracle_block(sub, guide_o, off + b0)
        g1, o1 = st[sl] == 1, och["status"] == 1
        flags.append(g1 == o1)
        both = g1 & o1
        for i in range(int(sub.k.max())):
            sel = both & (sub.k > i) & np.all(surf[sl][:, :i + 1] == och["surf"][:, :i + 1], axis=1)
            if sel.any():
                dx.append(np.linalg.norm(x[sl][sel, i] - och["x"][sel, i], axis=1).max())
        gadm = T[sl] > 0
        same_T.append(gadm == oadm)
        ab = gadm & oadm
        rel_T.append(np.abs(T[sl][ab] - oT[ab]) / oT[ab])
        worst.append((rel_T[-1].max(initial=0.0), b0, np.nonzero(ab)[0][np.argmax(rel_T[-1])] if ab.any() else -1))
        same_N.append(N[sl][ab] == oN[ab])
        # irradiance of the points whose every chain agrees in admissibility and N
        ok = ((gadm == oadm) & ((N[sl] == oN) | ~oadm)).reshape(-1, wl.spq).all(axis=1)
        oE = O.irradiance(sub, oT, oN, oadm)
        q0 = b0 // wl.spq
        nz = ok & (oE > 0)
        rel_E.append(np.abs(E[q0:q0 + BLOCK // wl.spq][nz] - oE[nz]) / oE[nz])
    flags, same_T, same_N = np.concatenate(flags), np.concatenate(same_T), np.concatenate(same_N)
    rel_T, rel_E = np.concatenate(rel_T), np.concatenate(rel_E)
    assert flags.mean() >= 0.999, flags.mean()
    assert max(dx) < 1e-4 * wl.scene_scale, max(dx)
    assert same_T.mean() >= 0.999, same_T.mean()
    # T of every chain both sides admit (the maximum, no quantile)
    assert rel_T.size > 200 and rel_T.max() < 1e-3, max(worst)
    assert same_N.mean() >= 0.999, same_N.mean()
    assert rel_E.size > 50 and rel_E.max() < 1e-3
    # whole batch: E is the per-point mean of the contributions
    c = res.contrib.cpu().numpy().astype(np.float64).reshape(wl.Q, wl.spq)
    assert np.allclose(E, c.sum(axis=1) / wl.spq, rtol=1e-5, atol=0)
    adm = T > 0
    assert np.all(N[adm] >= 1) and np.all(N[~adm] == 0)


def test_glass_sphere_full_size_captured_step(M, ctx):
    wl = I.glass_sphere()
    B = wl.B
    sc = M.Scene(ctx, wl)
    ch = M.Chains(wl)
    P = M.params_from(wl.params, walk_mode=M.WALK_BATCHED, k_uniform=2)
    res = M.Contribution.empty(B, wl.Q)
    rec = (torch.zeros(B, dtype=torch.int32, device="cuda"), torch.zeros((3, B), dtype=torch.float32, device="cuda"),
           torch.zeros(B, dtype=torch.float32, device="cuda"), torch.zeros(4, dtype=torch.int32, device="cuda"))
    guide = M.Guide(wl.n_cells, I.guide_edges())
    nxt = M.Guide(wl.n_cells, I.guide_edges())
    # training pass with p_0 in the oracle, over the whole batch; its records
    # fill both guides, and the update of all of them is bit-exact
    osc = O.Scene(wl)
    oseeds = O.sample_seeds(wl, osc, rng_offset=1 << 40)
    och = O.walk(wl, osc, oseeds)
    ocon = O.contribution(wl, osc, och)
    oN, _ = O.bernoulli(wl, osc, och, ocon["admissible"], rng_offset=1 << 40)
    cell0, om0, w0 = O.records(wl, och, ocon["T"], oN, ocon["admissible"])
    assert cell0.size > 500_000
    g_o = O.Guide(wl.n_cells, I.guide_edges())
    g_o.update(cell0, om0, w0, wl.params.weight_shift)
    M.mpg_guide_update(ctx, guide, torch.as_tensor(cell0.astype(np.int32), device="cuda"),
                       torch.as_tensor(np.ascontiguousarray(om0.T), device="cuda"),
                       torch.as_tensor(w0, device="cuda"), weight_shift=wl.params.weight_shift)
    ctx.sync()
    assert np.array_equal(guide.counts.cpu().numpy().view(np.uint64), g_o.counts)

    def step(off):
        M.mpg_sample_seeds(ctx, sc, guide, ch, P, wl.rng_seed, off)
        M.mpg_manifold_walk(ctx, sc, ch, P)
        M.mpg_chain_contribution(ctx, sc, guide, ch, P, wl.rng_seed, off, out=res)
        M.mpg_guide_records(ctx, sc, ch, res.contrib, out=rec)
        M.mpg_guide_clear(ctx, nxt)
        M.mpg_guide_update(ctx, nxt, rec[0], rec[1], rec[2], R=B, R_dev=rec[3], weight_shift=wl.params.weight_shift)

    off = 3 * B
    step(off)  # uncaptured first: sizes the buffers
    ctx.sync()
    g = M.Graph(ctx, rng_advance=B)
    with g:
        step(off)
    g.launch()  # replay 0 draws at `off`
    ctx.sync()
    _compare_blocks(M, wl, ch, res, g_o, off)
    # the step's own histogram update over every record (about 800,000): the
    # counts of each cell sum to the quantised weights q = floor(w 2^S) of its
    # records, exactly (the bin rule itself is pinned bit-exact above and in
    # the reduced-size tests)
    R = int(rec[3][0].item())
    assert R == int((res.contrib > 0).sum().item())
    rc = rec[0][:R].cpu().numpy().astype(np.int64)
    q = np.floor(rec[2][:R].cpu().numpy().astype(np.float64) * 2.0 ** wl.params.weight_shift).astype(np.uint64)
    per_cell = np.zeros(wl.n_cells, np.uint64)
    np.add.at(per_cell, rc, q)
    counts = nxt.counts.cpu().numpy().view(np.uint64)
    assert np.array_equal(counts.sum(axis=1, dtype=np.uint64), per_cell)
    assert np.count_nonzero(counts) > 1000 and np.count_nonzero(counts.sum(axis=1)) > 200


def test_mixed_batch_full_size_captured_step(M, ctx):
    wl = I.mixed()
    sc = M.Scene(ctx, wl)
    ch = M.Chains(wl)
    P = M.params_from(wl.params, walk_mode=M.WALK_BATCHED, tau_random=True)
    res = M.Contribution.empty(wl.B, wl.Q)

    def step(off):
        M.mpg_sample_seeds(ctx, sc, None, ch, P, wl.rng_seed, off)
        M.mpg_manifold_walk(ctx, sc, ch, P)
        M.mpg_chain_contribution(ctx, sc, None, ch, P, wl.rng_seed, off, out=res)

    off = 7 * wl.B
    step(off)
    ctx.sync()
    g = M.Graph(ctx, rng_advance=wl.B)
    with g:
        step(off)
    g.launch()
    ctx.sync()
    _compare_blocks(M, wl, ch, res, None, off)
    # every chain length is present and walked
    k = wl.k
    st = ch.status.cpu().numpy()
    for kk in range(1, 9):
        assert ((k == kk) & (st == 1)).sum() > 0


def test_mixed_vmf_full_size_captured_step(M, ctx):
    """The vMF-guided mixed batch (4,194,304 chains, sampled lengths, guided
    seeds and trials) replayed from its captured graph, as the benchmark's vMF
    measurement runs it.  The guide is built on both sides from the same seeded
    synthetic records (no training pass at this size); the oracle redraws the
    blocks' lengths itself, which must equal the GPU's bit for bit."""
    from test_gpu_vmf import _compare_guides, _dev_records
    wl = I.mixed()
    recs = I.synthetic_guide_records(wl)
    og = O.VmfGuide(wl.n_cells).build(*recs, wl.params.weight_shift)
    gg = M.VmfGuide(wl.n_cells, recs[0].size)
    M.mpg_vmf_build(ctx, gg, *_dev_records(recs), weight_shift=wl.params.weight_shift)
    ctx.sync()
    _compare_guides(og, gg)
    sc = M.Scene(ctx, wl)
    ch = M.Chains(wl)
    P = M.params_from(wl.params, walk_mode=M.WALK_BATCHED, tau_random=True)
    res = M.Contribution.empty(wl.B, wl.Q)
    p0w = I.GEOMETRIC_K_WEIGHTS

    def step(off):
        M.mpg_sample_lengths(ctx, gg, ch, p0w, P, wl.rng_seed, off, out=(ch.k, ch.pn))
        M.mpg_sample_seeds(ctx, sc, gg, ch, P, wl.rng_seed, off)
        M.mpg_manifold_walk(ctx, sc, ch, P)
        M.mpg_chain_contribution(ctx, sc, gg, ch, P, wl.rng_seed, off, out=res)

    off = 9 * wl.B
    step(off)
    ctx.sync()
    g = M.Graph(ctx, rng_advance=wl.B)
    with g:
        step(off)
    g.launch()
    ctx.sync()
    k_gpu = ch.k.cpu().numpy()

    def block(b0):
        sub = _block(wl, b0, BLOCK)
        ok, opn = O.sample_lengths(sub, og, p0w, rng_offset=off + b0)
        assert np.array_equal(ok, k_gpu[b0:b0 + BLOCK])
        return dataclasses.replace(sub, k=ok, pn=opn)

    _compare_blocks(M, wl, ch, res, og, off, block=block)
    for kk in range(1, 9):
        assert ((k_gpu == kk) & (ch.status.cpu().numpy() == 1)).sum() > 0


def _put_block(M, ch, b0, o, status):
    """Chains [b0, b0 + n) of the device batch set to the oracle's chains
    (rounded to FP32) with the given status."""
    n = status.size
    sl = slice(b0, b0 + n)
    ch.x[:, :, sl] = torch.as_tensor(np.ascontiguousarray(o["x"].transpose(1, 2, 0)).astype(np.float32), device="cuda")
    ch.surf[:, sl] = torch.as_tensor(np.ascontiguousarray(o["surf"].T).astype(np.int32), device="cuda")
    ch.prim[:, sl] = torch.as_tensor(np.ascontiguousarray(o["prim"].T).astype(np.int32), device="cuda")
    ch.bary[:, :, sl] = torch.as_tensor(np.ascontiguousarray(o["bary"].transpose(1, 2, 0)).astype(np.float32),
                                        device="cuda")
    ch.tau[sl] = torch.as_tensor(o["tau"].astype(np.uint8), device="cuda")
    ch.status[sl] = torch.as_tensor(status.astype(np.uint8), device="cuda")


def test_water_full_size_captured_step_and_adjoint(M, ctx):
    """The water heightfield at its full size (512 x 512 points x 4 seeds =
    1,048,576 chains, BVH traversal), batched and replayed from a captured
    graph, compared block by block with the oracle; then the adjoint of the
    irradiance with respect to the 128 x 128 heights over the whole batch
    (the launch the benchmark times): linear in the upstream gradient over
    the whole batch, and equal to the oracle's implicit-function gradient on
    receiver-aligned blocks of the oracle's chains placed in that batch."""
    wl = I.water()
    sc = M.Scene(ctx, wl)
    ch = M.Chains(wl)
    P = M.params_from(wl.params, walk_mode=M.WALK_BATCHED, k_uniform=0)
    res = M.Contribution.empty(wl.B, wl.Q)

    def step(off):
        M.mpg_sample_seeds(ctx, sc, None, ch, P, wl.rng_seed, off)
        M.mpg_manifold_walk(ctx, sc, ch, P)
        M.mpg_chain_contribution(ctx, sc, None, ch, P, wl.rng_seed, off, out=res)

    off = 5 * wl.B
    step(off)
    ctx.sync()
    g = M.Graph(ctx, rng_advance=wl.B)
    with g:
        step(off)
    g.launch()
    ctx.sync()
    _compare_blocks(M, wl, ch, res, None, off)
    st = ch.status.cpu().numpy()
    # one refraction converges for most points; the RT / TR chains need a
    # crest to bounce off and converge rarely
    assert ((wl.k == 1) & (st == 1)).sum() > 0.3 * (wl.k == 1).sum()
    # adjoint over the whole batch, and over the two halves of the receiver points
    dLdE = torch.as_tensor(I.upstream_grad(wl.Q), dtype=torch.float32, device="cuda")
    n_h = wl.hf_heights.size
    g_all = torch.zeros(n_h, dtype=torch.float32, device="cuda")
    M.mpg_walk_adjoint(ctx, sc, ch, res.T, res.contrib, dLdE, g_all)
    half = torch.zeros_like(dLdE)
    half[: wl.Q // 2] = dLdE[: wl.Q // 2]
    g_a, g_b = torch.zeros_like(g_all), torch.zeros_like(g_all)
    M.mpg_walk_adjoint(ctx, sc, ch, res.T, res.contrib, half, g_a)
    M.mpg_walk_adjoint(ctx, sc, ch, res.T, res.contrib, dLdE - half, g_b)
    ctx.sync()
    g_all = g_all.cpu().numpy().astype(np.float64)
    assert np.isfinite(g_all).all() and np.count_nonzero(g_all) > 0.5 * n_h
    assert np.linalg.norm(g_a.cpu().numpy() + g_b.cpu().numpy() - g_all) <= 1e-4 * np.linalg.norm(g_all)
    # receiver-aligned blocks of the oracle's chains inside the full batch
    osc = O.Scene(wl)
    q = np.arange(wl.B) // wl.spq
    T_in = np.zeros(wl.B, np.float32)
    c_in = np.zeros(wl.B, np.float32)
    up = np.zeros(wl.Q, np.float32)
    dl = I.upstream_grad(wl.Q).astype(np.float32)
    g_o = np.zeros(n_h)
    for b0 in _starts(wl):
        sub = _block(wl, b0, BLOCK)
        sseeds = O.sample_seeds(sub, osc, None, rng_offset=off + b0)
        och = O.walk(sub, osc, sseeds)
        con = O.contribution(sub, osc, och)
        oN, _ = O.bernoulli(sub, osc, och, con["admissible"], None, rng_offset=off + b0)
        tight = dataclasses.replace(sub, params=dataclasses.replace(sub.params, tol=1e-12))
        conv = dict(x=och["x"], surf=och["surf"], prim=och["prim"], bary=och["bary"], tau=och["tau"],
                    valid=(och["status"] == 1).astype(np.uint8))
        pol = O.walk(tight, osc, conv)
        pol["status"] = np.where(pol["status"] == 1, och["status"], 0).astype(np.uint8)
        cp = O.contribution(sub, osc, pol)
        adm = (con["admissible"] == 1) & (cp["admissible"] == 1)
        T = np.where(adm, cp["T"], 0.0)
        contrib = np.where(adm, sub.light_area * T * oN / sub.pn, 0.0)
        T32, c32 = T.astype(np.float32), contrib.astype(np.float32)
        sq = np.arange(BLOCK) // wl.spq
        w = np.where(T32 > 0, dl[b0 // wl.spq + sq] / wl.spq * c32.astype(np.float64) / np.maximum(T32, 1e-30), 0.0)
        gb, _ = O.adjoint(sub, osc, och, w)
        g_o += gb
        _put_block(M, ch, b0, och, np.where(adm, M.CHAIN_CONVERGED, M.CHAIN_FAILED))
        T_in[b0:b0 + BLOCK], c_in[b0:b0 + BLOCK] = T32, c32
        up[b0 // wl.spq: (b0 + BLOCK) // wl.spq] = dl[b0 // wl.spq: (b0 + BLOCK) // wl.spq]
    assert np.count_nonzero(T_in) > 1000
    g_gpu = torch.zeros(n_h, dtype=torch.float32, device="cuda")
    M.mpg_walk_adjoint(ctx, sc, ch, torch.as_tensor(T_in, device="cuda"), torch.as_tensor(c_in, device="cuda"),
                       torch.as_tensor(up, device="cuda"), g_gpu)
    ctx.sync()
    g_gpu = g_gpu.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g_o) > 0
    assert np.linalg.norm(g_gpu - g_o) <= 1e-2 * np.linalg.norm(g_o), np.linalg.norm(g_gpu - g_o) / np.linalg.norm(g_o)
