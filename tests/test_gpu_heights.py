"""Heights replaced on the device (mpg_scene_set_heights) against a scene built
on the host from the same heights, and the autograd function's repeated
forward calls (the heightfield's parameters are what the adjoint of the
continuity argument, Sec. 5.2, differentiates)."""
import dataclasses

import numpy as np
import pytest
import torch

from paper_2311_12818_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_2311_12818_gb300 import mpg
    return mpg


@pytest.fixture(scope="module")
def ctx(M):
    return M.Context(0)


def _heights(wl, scale):
    """Float32 heights: the workload's plus a smooth bump (as float64 copies of
    the float32 values, so the host build sees exactly what the device does)."""
    n = int(np.sqrt(wl.hf_heights.size))
    y, x = np.mgrid[0:n, 0:n] / (n - 1.0) * 2.0 - 1.0
    h = (wl.hf_heights.reshape(n, n) + scale * np.exp(-4.0 * (x * x + y * y))).astype(np.float32)
    return h.ravel()


def _rays(n, seed=11):
    rng = np.random.default_rng(seed)
    o = np.column_stack([rng.uniform(-1.1, 1.1, n), rng.uniform(-1.1, 1.1, n), rng.choice([-1.0, 2.0], n)])
    tgt = np.column_stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(-0.08, 0.08, n)])
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    f = lambda a: torch.as_tensor(a.T.astype(np.float32), device="cuda").contiguous()  # noqa: E731
    return f(o), f(d)


def test_set_heights_matches_host_build(M, ctx):
    wl = I.water(n=64, spq=4, grid=128)
    h1, h2 = _heights(wl, 0.0), _heights(wl, 0.03)
    host = M.Scene(ctx, dataclasses.replace(wl, hf_heights=h2.astype(np.float64)))
    dev = M.Scene(ctx, dataclasses.replace(wl, hf_heights=h1.astype(np.float64)))
    dev.set_heights(torch.as_tensor(h2, device="cuda"))
    assert host.info(0)[1] == dev.info(0)[1]
    o, d = _rays(50000)
    th, sh, ph, bh = (a.cpu().numpy() for a in M.mpg_trace_rays(ctx, host, o, d))
    td, sd, pd, bd = (a.cpu().numpy() for a in M.mpg_trace_rays(ctx, dev, o, d))
    ctx.sync()
    # the same triangles and normals; only the tree's shape differs (the refit
    # keeps the first build's), which can change which of two triangles sharing
    # an edge reports a hit on that edge
    assert np.array_equal(sh, sd)
    hit = sh >= 0
    assert hit.mean() > 0.9
    assert (ph[hit] == pd[hit]).mean() >= 0.9999
    same = hit & (ph == pd)
    assert np.array_equal(th[same], td[same])  # the same triangle: the same arithmetic
    assert np.abs(th[hit] - td[hit]).max() < 1e-5
    # the whole pipeline on both scenes
    outs = []
    for sc in (host, dev):
        ch = M.Chains(wl)
        out = M.run(ctx, sc, ch, wl)
        ctx.sync()
        outs.append((ch.status.cpu().numpy(), out.E.cpu().numpy()))
    (s0, E0), (s1, E1) = outs
    assert (s0 == s1).mean() >= 0.9999
    assert np.abs(E0 - E1).sum() <= 1e-4 * np.abs(E0).sum()


def test_set_heights_twice_returns_to_the_first_surface(M, ctx):
    wl = I.water(n=32, spq=2, grid=64)
    h1, h2 = _heights(wl, 0.0), _heights(wl, -0.05)
    sc = M.Scene(ctx, dataclasses.replace(wl, hf_heights=h1.astype(np.float64)))
    o, d = _rays(20000, seed=3)
    t0 = M.mpg_trace_rays(ctx, sc, o, d)[0].cpu().numpy()
    sc.set_heights(torch.as_tensor(h2, device="cuda"))
    t1 = M.mpg_trace_rays(ctx, sc, o, d)[0].cpu().numpy()
    sc.set_heights(torch.as_tensor(h1, device="cuda"))
    t2 = M.mpg_trace_rays(ctx, sc, o, d)[0].cpu().numpy()
    ctx.sync()
    assert not np.array_equal(t0, t1)
    assert np.array_equal(t0, t2)  # same heights, same tree: the same arrays


def test_set_heights_rejects_bad_arguments(M, ctx):
    wl = I.mirror_sphere(n=4, spq=1)
    sc = M.Scene(ctx, wl)  # no heightfield
    with pytest.raises(M.MpgError):
        sc.set_heights(torch.zeros(16, dtype=torch.float32, device="cuda"))


def test_autograd_forward_calls_follow_the_heights(M, ctx):
    from paper_2311_12818_gb300 import autograd as AG
    wl = I.water(n=24, spq=2, grid=64)
    h1, h2 = _heights(wl, 0.0), _heights(wl, 0.02)
    fn = AG.HeightfieldIrradiance(ctx, wl)
    E1 = fn(torch.as_tensor(h1, device="cuda").requires_grad_(True)).detach().clone()
    E2 = fn(torch.as_tensor(h2, device="cuda").requires_grad_(True)).detach().clone()
    # a fresh function whose first call builds the scene from h2 on the host
    ref = AG.HeightfieldIrradiance(ctx, wl)(torch.as_tensor(h2, device="cuda")).detach()
    ctx.sync()
    assert not torch.equal(E1, E2)
    assert (E2 - ref).abs().sum().item() <= 1e-4 * ref.abs().sum().item()
