"""Schedules, captured graphs and the autotuner of the batched mode.

The schedule of the batched mode (threads per CTA, resident CTAs, refill
cadence of the persistent kernels, Bernoulli round sizes) decides only which
lane runs which chain when: every chain's walk and every trial use the same
arithmetic, so the results must be bit-identical across schedules.  A
captured graph replays the same kernels, so a replay must equal the
uncaptured calls at the same random-number offset, bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2311_12818_gb300 import inputs as I  # noqa: E402


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


def _step(M, ctx, sc, ch, res, wl, P, off, guide=None):
    M.mpg_sample_seeds(ctx, sc, guide, ch, P, wl.rng_seed, off)
    M.mpg_manifold_walk(ctx, sc, ch, P)
    M.mpg_chain_contribution(ctx, sc, guide, ch, P, wl.rng_seed, off, out=res)


def _snapshot(ch, res):
    return {"status": ch.status.cpu().numpy().copy(), "x": ch.x.cpu().numpy().copy(),
            "surf": ch.surf.cpu().numpy().copy(), "T": res.T.cpu().numpy().copy(),
            "G": res.G.cpu().numpy().copy(), "trials": res.trials.cpu().numpy().copy(),
            "capped": res.capped.cpu().numpy().copy(), "contrib": res.contrib.cpu().numpy().copy(),
            "E": res.E.cpu().numpy().copy()}


def _run(M, ctx, wl, P, off=0):
    sc = M.Scene(ctx, wl)
    ch = M.Chains(wl)
    res = M.Contribution.empty(wl.B, wl.Q)
    ctx.reset_stats()
    _step(M, ctx, sc, ch, res, wl, P, off)
    ctx.sync()
    snap = _snapshot(ch, res)
    st = ctx.stats()
    snap["converged_walks"] = np.array([st["converged"], st["uncounted"]])
    return snap


def _mixed():
    return I.mixed(nx=96, ny=48, spq=8)


def _bitwise_equal(a, b, keys=None):
    for k in keys or a:
        assert np.array_equal(a[k], b[k]), k


def test_schedules_give_identical_results(M, ctx):
    wl = _mixed()
    base = M.params_from(wl.params, walk_mode=M.WALK_BATCHED, tau_random=True)
    ref = _run(M, ctx, wl, base)
    assert (ref["status"] == 1).sum() > 1000
    assert ref["trials"].max() > 8  # the parallel Bernoulli rounds ran
    assert ref["converged_walks"][1] == 0
    # the count of converged walks is the sequential loop's, whatever the schedule:
    # the plain mode runs each chain's trials one after another
    plain = _run(M, ctx, wl, M.params_from(wl.params, walk_mode=M.WALK_PLAIN, tau_random=True))
    assert abs(int(plain["converged_walks"][0]) - int(ref["converged_walks"][0])) <= 1e-3 * ref["converged_walks"][0]
    for sched in ({"block_threads": 64, "ctas_per_sm": 2}, {"block_threads": 32, "refill_every": 4},
                  {"refill_every": 2, "trial_sync_rounds": 1, "trial_batch": 4},
                  {"trial_sync_rounds": 3, "trial_batch": 32, "ctas_per_sm": 1},
                  {"trial_sync_rounds": -1, "trial_batch": 1}, {"trial_sync_rounds": -1, "trial_batch": 4096}):
        P = M.params_from(wl.params, walk_mode=M.WALK_BATCHED, tau_random=True, **sched)
        _bitwise_equal(ref, _run(M, ctx, wl, P))


def test_fp64_split_moves_only_toward_fp64(M, ctx):
    wl = _mixed()
    ref = _run(M, ctx, wl, M.params_from(wl.params, walk_mode=M.WALK_BATCHED, tau_random=True))
    more = _run(M, ctx, wl, M.params_from(wl.params, walk_mode=M.WALK_BATCHED, tau_random=True, fp64_k=4))
    _bitwise_equal(ref, more, ["status", "surf"])
    ok = ref["T"] > 0
    assert np.array_equal(ok, more["T"] > 0)
    rel = np.abs(more["T"][ok] - ref["T"][ok]) / ref["T"][ok]
    assert np.quantile(rel, 0.999) < 1e-3
    with pytest.raises(M.MpgError):  # fewer FP64 chains than k >= 6 is refused
        _run(M, ctx, wl, M.params_from(wl.params, walk_mode=M.WALK_BATCHED, tau_random=True, fp64_k=7))
    with pytest.raises(M.MpgError):  # the kernels are compiled for at most 128 threads per CTA
        _run(M, ctx, wl, M.params_from(wl.params, walk_mode=M.WALK_BATCHED, tau_random=True, block_threads=256))


@pytest.mark.parametrize("name", ["glass", "mixed"])
def test_graph_replay_matches_uncaptured(M, ctx, name):
    wl = I.glass_sphere(n=48, spq=8) if name == "glass" else _mixed()
    kw = dict(k_uniform=2) if name == "glass" else dict(tau_random=True)
    P = M.params_from(wl.params, walk_mode=M.WALK_BATCHED, **kw)
    sc = M.Scene(ctx, wl)
    ch = M.Chains(wl)
    res = M.Contribution.empty(wl.B, wl.Q)
    off = 12345
    _step(M, ctx, sc, ch, res, wl, P, off)  # uncaptured first: sizes the buffers
    ctx.sync()
    n0 = ctx.launches()
    _step(M, ctx, sc, ch, res, wl, P, off)
    ctx.sync()
    uncaptured_launches = ctx.launches() - n0
    g = M.Graph(ctx, rng_advance=wl.B)
    with g:
        _step(M, ctx, sc, ch, res, wl, P, off)
    assert g.kernels() == uncaptured_launches + 1  # + the counter advance
    refs = []
    for r in range(3):
        _step(M, ctx, sc, ch, res, wl, P, off + r * wl.B)
        ctx.sync()
        refs.append(_snapshot(ch, res))
    for r in range(3):
        n0 = ctx.launches()
        g.launch()
        ctx.sync()
        assert ctx.launches() - n0 == g.kernels()
        _bitwise_equal(refs[r], _snapshot(ch, res))
    assert not np.array_equal(refs[0]["contrib"], refs[1]["contrib"])  # replays draw fresh numbers


def test_capture_without_sized_buffers_fails_cleanly(M, ctx):
    wl = I.glass_sphere(n=40, spq=8)
    c2 = M.Context(0)  # a fresh context has no Bernoulli buffers yet
    sc = M.Scene(c2, wl)
    ch = M.Chains(wl)
    res = M.Contribution.empty(wl.B, wl.Q)
    P = M.params_from(wl.params, walk_mode=M.WALK_BATCHED, k_uniform=2)
    with pytest.raises(M.MpgError):
        with M.Graph(c2, rng_advance=wl.B):
            _step(M, c2, sc, ch, res, wl, P, 0)
    torch.cuda.synchronize()
    _step(M, c2, sc, ch, res, wl, P, 0)  # the context still works uncaptured
    c2.sync()
    assert (ch.status.cpu().numpy() == 1).sum() > 0


def test_autotune_picks_a_valid_schedule(M, ctx):
    wl = _mixed()
    base = M.params_from(wl.params, walk_mode=M.WALK_BATCHED, tau_random=True)
    sc = M.Scene(ctx, wl)
    ch = M.Chains(wl)
    ctx.reset_stats()
    n0 = ctx.launches()
    tuned, ms = M.mpg_autotune(ctx, sc, None, ch, base, wl.rng_seed, 0, repeats=1)
    assert ms > 0
    assert ctx.stats()["walks"] == 0 and ctx.launches() == n0  # tuning left the caller's counters alone
    assert tuned.block_threads in (0, 32, 64, 128)
    assert tuned.refill_every in (0, 1, 2, 4, 8)
    assert tuned.trial_sync_rounds in (0, 1, 2, 3) and tuned.trial_batch in (0, 4, 16, 64, 256)
    assert tuned.fp64_k in (0, 4, 5)
    assert tuned.walk_group in (0, 1, 2, 3)
    for f in ("tol", "max_iter", "max_halvings", "max_trials", "dedup_eps", "walk_mode", "tau_random"):
        assert getattr(tuned, f) == getattr(base, f)
    ref = _run(M, ctx, wl, base)
    got = _run(M, ctx, wl, tuned)
    if tuned.walk_group:  # same per-vertex arithmetic, contracted differently: compared like the oracle
        assert (ref["status"] == got["status"]).mean() >= 0.999
        ok = (ref["T"] > 0) & (got["T"] > 0)
        assert np.quantile(np.abs(got["T"][ok] - ref["T"][ok]) / ref["T"][ok], 0.999) < 1e-3
    else:
        _bitwise_equal(ref, got, ["status", "surf", "trials", "converged_walks"] if tuned.fp64_k else None)


def test_two_context_graph_matches_uncaptured(M, ctx):
    """Two contexts recording into one capture (double buffering): replay r of
    batch j draws at offset + (2 r + j) B, bit-identical to the uncaptured calls."""
    wl = I.glass_sphere(n=48, spq=8)
    P = M.params_from(wl.params, walk_mode=M.WALK_BATCHED, k_uniform=2)
    ctxs = [ctx, M.Context(0)]
    parts = [(M.Scene(c, wl), M.Chains(wl), M.Contribution.empty(wl.B, wl.Q)) for c in ctxs]
    off = 777
    for j, c in enumerate(ctxs):  # size the buffers
        _step(M, c, *parts[j], wl, P, off + j * wl.B)
    torch.cuda.synchronize()
    refs = []
    for r in range(2):
        for j, c in enumerate(ctxs):
            _step(M, c, *parts[j], wl, P, off + (2 * r + j) * wl.B)
            c.sync()
            refs.append(_snapshot(parts[j][1], parts[j][2]))
    g = M.Graph(ctx, rng_advance=2 * wl.B, join=[ctxs[1]])
    side = [torch.cuda.Stream(), torch.cuda.Stream()]
    with g:
        for j, c in enumerate(ctxs):
            side[j].wait_stream(g.stream)
            sc, ch, res = parts[j]
            M.mpg_sample_seeds(c, sc, None, ch, P, wl.rng_seed, off + j * wl.B, stream=side[j])
            M.mpg_manifold_walk(c, sc, ch, P, stream=side[j])
            M.mpg_chain_contribution(c, sc, None, ch, P, wl.rng_seed, off + j * wl.B, out=res, stream=side[j])
        for s in side:
            g.stream.wait_stream(s)
    for r in range(2):
        g.launch()
        torch.cuda.synchronize()
        for j in range(2):
            _bitwise_equal(refs[2 * r + j], _snapshot(parts[j][1], parts[j][2]))
    with pytest.raises(M.MpgError):  # a context cannot join a capture twice
        with M.Graph(ctx, join=[ctxs[1], ctxs[1]]):
            pass


def test_group_walk_agrees_with_thread_walk(M, ctx):
    """One chain per lane group (walk and parallel Bernoulli rounds) against one
    thread per chain: the same per-vertex arithmetic, agreeing to FP32 rounding."""
    wl = _mixed()
    ref = _run(M, ctx, wl, M.params_from(wl.params, walk_mode=M.WALK_BATCHED, tau_random=True))
    got = _run(M, ctx, wl, M.params_from(wl.params, walk_mode=M.WALK_BATCHED, tau_random=True, walk_group=3))
    assert (ref["status"] == got["status"]).mean() >= 0.999
    both = (ref["status"] == 1) & (got["status"] == 1)
    assert np.abs(ref["x"][:, :, both] - got["x"][:, :, both]).max() < 1e-4 * wl.scene_scale
    ok = (ref["T"] > 0) & (got["T"] > 0)
    assert (ref["trials"][ok] == got["trials"][ok]).mean() >= 0.995
    assert abs(int(got["converged_walks"][0]) - int(ref["converged_walks"][0])) <= 0.01 * ref["converged_walks"][0]
    assert got["converged_walks"][1] == 0
