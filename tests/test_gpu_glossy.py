"""Glossy chains on the GPU (Sec. 5.7) against the oracle's glossy chains.

Every vertex is a rough interface (isotropic Beckmann, roughness alpha); a
chain carries one offset normal per vertex, walks to C_i = o_i, and its
estimate is W = L_e prod f |n.l| prod(area factors) / (|det dC/du| prod p(o))
with the microfacet density cancelled; its reciprocal probability comes from
Bernoulli trials walked with the same offsets.  Bars as for specular chains:
offsets to FP32 rounding of the Beckmann transform, converged vertices within
1e-4 of the scene scale, flags on >= 99.9 % of chains, W within 1e-3 relative
on every chain both sides admit, trial counts equal where both sides walked
the same chains."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2311_12818_gb300 import inputs as I  # noqa: E402
from test_gpu_parity import _assert_T_max, _chains_from_oracle, _compare_seeds, _compare_walk, _params  # noqa: E402


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


def _rough(wl, alpha):
    return dataclasses.replace(wl, params=dataclasses.replace(wl.params, roughness=alpha))


@pytest.mark.parametrize("alpha", [0.05, 0.3])
def test_offsets_match_oracle(M, ctx, alpha):
    wl = I.mixed(nx=64, ny=32, spq=4)
    ch = M.Chains(wl)
    for off in (0, 12345):
        g = M.mpg_sample_offsets(ctx, ch, alpha, wl.rng_seed, off)
        ctx.sync()
        g = g.permute(2, 0, 1).double().cpu().numpy()  # [B, 8, 2]
        o = O.sample_offsets(wl, alpha, rng_offset=off)
        used = np.arange(8)[None, :] < wl.k[:, None]
        assert np.all(g[~used] == 0.0)
        assert np.abs(g - o).max() < 4e-6 * max(1.0, alpha / 0.3)


@pytest.mark.parametrize("which", ["glass", "mixed"])
def test_glossy_walk_from_identical_seeds_and_offsets(M, ctx, which):
    """The oracle's seeds and offsets (rounded to FP32) walked on the GPU to
    C = o, against the oracle's FP64 walk of the same seeds and offsets."""
    wl = _rough(I.glass_sphere(n=32, spq=16) if which == "glass" else I.mixed(nx=64, ny=32, spq=8), 0.1)
    osc = O.Scene(wl)
    seeds = O.sample_seeds(wl, osc)
    off = O.sample_offsets(wl, 0.1)
    ow = O.walk(wl, osc, seeds, offset=off)
    sc = M.Scene(ctx, wl)
    ch = _chains_from_oracle(M, wl, seeds, np.where(seeds["valid"] == 1, M.CHAIN_SEEDED, M.CHAIN_INVALID))
    ch.offset = torch.as_tensor(np.ascontiguousarray(off.transpose(1, 2, 0)).astype(np.float32), device="cuda")
    M.mpg_manifold_walk(ctx, sc, ch, _params(M, wl))  # batched asked: glossy chains take the plain kernels
    ctx.sync()
    gw = ch.aos()
    both = _compare_walk(wl, gw, ow)
    # the specular walk from the same seeds ends elsewhere: the offsets are used
    ch2 = _chains_from_oracle(M, wl, seeds, np.where(seeds["valid"] == 1, M.CHAIN_SEEDED, M.CHAIN_INVALID))
    M.mpg_manifold_walk(ctx, sc, ch2, _params(M, wl))
    ctx.sync()
    sw = ch2.aos()
    moved = both & (sw["status"] == 1)
    assert np.median(np.linalg.norm(gw["x"][moved, 0] - sw["x"][moved, 0], axis=-1)) > 1e-3


def _oracle_glossy(wl, alpha):
    sc = O.Scene(wl)
    seeds = O.sample_seeds(wl, sc)
    off = O.sample_offsets(wl, alpha)
    ch = O.walk(wl, sc, seeds, offset=off)
    g = O.glossy(wl, sc, ch, offset=off, alpha=alpha)
    N, capped = O.bernoulli(wl, sc, ch, g["admissible"], offset=off)
    # W of the chains polished to 1e-12 (C = o); admissibility of the walk at the tolerance
    tight = dataclasses.replace(wl, params=dataclasses.replace(wl.params, tol=1e-12))
    conv = dict(x=ch["x"], surf=ch["surf"], prim=ch["prim"], bary=ch["bary"], tau=ch["tau"],
                valid=(ch["status"] == 1).astype(np.uint8))
    pol = O.walk(tight, sc, conv, offset=off)
    pol["status"] = np.where(pol["status"] == 1, ch["status"], 0).astype(np.uint8)
    gp = O.glossy(wl, sc, pol, offset=off, alpha=alpha)
    # an admissible chain whose shadowing term vanishes (a direction behind its
    # microfacet) has W = 0 and contributes nothing: both sides leave it out
    adm = (g["admissible"] == 1) & ((gp["admissible"] == 1) | (ch["status"] != 1)) & (gp["W"] > 0)
    return seeds, off, ch, np.where(adm, gp["W"], 0.0), adm, N


@pytest.mark.parametrize("which,alpha", [("glass", 0.05), ("mixed", 0.1), ("water", 0.1)])
def test_glossy_pipeline_parity(M, ctx, which, alpha):
    wl = {"glass": lambda: I.glass_sphere(n=32, spq=16), "mixed": lambda: I.mixed(nx=64, ny=32, spq=8),
          "water": lambda: I.water(n=48, spq=4, grid=128)}[which]()
    wl = _rough(wl, alpha)
    P = _params(M, wl)
    sc = M.Scene(ctx, wl)
    ch = M.Chains(wl)
    M.mpg_sample_seeds(ctx, sc, None, ch, P, wl.rng_seed, 0)
    gs = ch.aos()
    ch.offset = M.mpg_sample_offsets(ctx, ch, alpha, wl.rng_seed, 0)
    M.mpg_manifold_walk(ctx, sc, ch, P)
    gw = ch.aos()
    out = M.mpg_chain_contribution(ctx, sc, None, ch, P, wl.rng_seed, 0)
    ctx.sync()
    os_, off, ow, W, adm, N = _oracle_glossy(wl, alpha)
    _compare_seeds(wl, gs, os_)
    both = _compare_walk(wl, gw, ow)
    T = out.T.cpu().numpy()
    assert ((T > 0) == adm)[both].mean() >= 0.999
    ab = (T > 0) & adm & both
    assert ab.sum() > 200
    _assert_T_max(wl, T, W, ab)
    assert np.all(out.G.cpu().numpy() == 0) and np.all(out.kappa.cpu().numpy() == 0)
    gN = out.trials.cpu().numpy().astype(np.int64)
    assert (gN[ab] == N[ab]).mean() >= 0.999
    # contributions and irradiance of the points whose every chain agrees
    c = out.contrib.cpu().numpy().astype(np.float64)
    assert np.allclose(c[T > 0], (wl.light_area * T.astype(np.float64) * gN / wl.pn)[T > 0], rtol=1e-5)
    E_o = O.irradiance(wl, W, N, adm)
    same = (((T > 0) == adm) & ((gN == N) | ~adm)).reshape(wl.Q, wl.spq).all(axis=1)
    nz = same & (E_o > 0)
    assert nz.sum() > 50
    E_g = out.E.cpu().numpy()
    assert np.max(np.abs(E_g[nz] - E_o[nz]) / E_o[nz]) < 1e-3


def test_zero_offsets_reproduce_the_specular_contribution(M, ctx):
    """With zero offsets and zero roughness the glossy estimate W (FP64, pivot
    determinant of the Jacobian, microfacet BSDF with D divided out) is the
    specular T = kappa G L_e (implicit-function G, Fresnel kappa) of the same
    chains: two independent routes on the GPU."""
    wl = I.mixed(nx=64, ny=32, spq=8)
    P = _params(M, wl, mode=M.WALK_PLAIN)
    sc = M.Scene(ctx, wl)
    ch = M.Chains(wl)
    M.mpg_sample_seeds(ctx, sc, None, ch, P, wl.rng_seed, 0)
    M.mpg_manifold_walk(ctx, sc, ch, P)
    ctx.sync()
    spec = M.mpg_chain_contribution(ctx, sc, None, ch, P, wl.rng_seed, 0)
    ctx.sync()
    ch.offset = torch.zeros((8, 2, wl.B), dtype=torch.float32, device="cuda")
    glos = M.mpg_chain_contribution(ctx, sc, None, ch, P, wl.rng_seed, 0)
    ctx.sync()
    Ts, Tg = spec.T.cpu().numpy(), glos.T.cpu().numpy()
    assert ((Ts > 0) == (Tg > 0)).mean() >= 0.999
    ab = (Ts > 0) & (Tg > 0)
    assert ab.sum() > 500
    rel = np.abs(Tg[ab] - Ts[ab]) / Ts[ab]
    assert rel.max() < 1e-3, rel.max()
    # zero offsets: the same trial walks
    assert (spec.trials.cpu().numpy()[ab] == glos.trials.cpu().numpy()[ab]).mean() >= 0.999
