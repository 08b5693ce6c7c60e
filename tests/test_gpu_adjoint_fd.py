"""The GPU adjoint (K7: implicit function theorem, transposed block Thomas
solve) against FP64 central finite differences of the oracle's forward map,
h = 1e-5 (continuity of the specular manifold, Sec. 5.2), on the water
heightfield: eight random unit directions over all 128 x 128 heights and 64
single heights under the chains.

L(theta) = sum_b w_b T_b(theta), w_b = dL/dE[q_b] / spq * <1/P>_b A_L with
<1/P> held fixed.  The forward map re-converges the oracle's chains (FP64,
|C| < 1e-13) on the perturbed heights; the GPU differentiates the same
chains (rounded to FP32) at the unperturbed heights.  The directional
derivatives over the probes are compared in 2-norm within 1e-2.  Chains
whose differences at h and 2h disagree by more than 1e-4 for some probe (a
chain that crosses a triangle edge, where the interpolated shading normals
are only piecewise smooth, or sits at a caustic fold) have no finite
difference reference: they are counted and left out on both sides."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2311_12818_gb300 import inputs as I  # noqa: E402
from test_gpu_parity import _chains_from_oracle  # noqa: E402


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_12818_gb300 import build, mpg
    build.build()
    return mpg


def _T_at(wl, heights, conv):
    w2 = dataclasses.replace(wl, hf_heights=heights, params=dataclasses.replace(wl.params, tol=1e-13, max_iter=40))
    sc = O.Scene(w2)
    ch = O.walk(w2, sc, conv)
    con = O.contribution(w2, sc, ch)
    return con["T"], con["admissible"] == 1


def test_gpu_gradient_matches_fp64_central_differences(M):
    ctx = M.Context(0)
    wl = I.water(n=48, spq=4, grid=128)
    wl = dataclasses.replace(wl, params=dataclasses.replace(wl.params, tol=1e-13))
    osc = O.Scene(wl)
    seeds = O.sample_seeds(wl, osc)
    ch = O.walk(wl, osc, seeds)
    con = O.contribution(wl, osc, ch)
    adm = con["admissible"] == 1
    N, _ = O.bernoulli(wl, osc, ch, con["admissible"])
    assert adm.sum() > 2000
    q = np.arange(wl.B) // wl.spq
    dLdE = I.upstream_grad(wl.Q).astype(np.float32)
    T32 = np.where(adm, con["T"], 0.0).astype(np.float32)
    c32 = np.where(adm, wl.light_area * con["T"] * N / wl.pn, 0.0).astype(np.float32)
    # the weight the kernel forms in FP32, in FP64 here
    w = np.where(T32 > 0, dLdE[q] / wl.spq * c32.astype(np.float64) / np.maximum(T32, 1e-30), 0.0)
    sc = M.Scene(ctx, wl)
    dch = _chains_from_oracle(M, wl, ch, np.where(adm, M.CHAIN_CONVERGED, M.CHAIN_FAILED))
    conv = dict(x=ch["x"], surf=ch["surf"], prim=ch["prim"], bary=ch["bary"], tau=ch["tau"],
                valid=adm.astype(np.uint8))
    rng = np.random.default_rng(0x4D50470005)
    h = 1e-5
    H0 = wl.hf_heights
    n_h = H0.size
    nx = int(wl.hf_desc[0, 0])
    probes = []
    for _ in range(8):
        v = rng.normal(size=n_h)
        probes.append(v / np.linalg.norm(v))
    quad = ch["prim"][adm, 0] // 2  # heights at the lower-left corners of the chains' quads
    under = np.unique((quad // (nx - 1)) * nx + quad % (nx - 1))
    for j in rng.choice(under, 64, replace=False):
        e = np.zeros(n_h)
        e[j] = 1.0
        probes.append(e)
    smooth = adm.copy()
    fds = []
    for v in probes:
        Tp, ap = _T_at(wl, H0 + h * v, conv)
        Tm, am = _T_at(wl, H0 - h * v, conv)
        T2p, a2p = _T_at(wl, H0 + 2 * h * v, conv)
        T2m, a2m = _T_at(wl, H0 - 2 * h * v, conv)
        fd1 = (Tp - Tm) / (2 * h)
        fd2 = (T2p - T2m) / (4 * h)
        smooth &= ap & am & a2p & a2m & (np.abs(fd1 - fd2) <= 1e-4 * np.maximum(np.abs(fd1), 1e-9 * np.abs(T2p).max()))
        fds.append(fd1)
    left_out = int(adm.sum() - smooth.sum())
    assert left_out <= 0.05 * adm.sum(), left_out
    g = torch.zeros(n_h, dtype=torch.float32, device="cuda")
    M.mpg_walk_adjoint(ctx, sc, dch, torch.as_tensor(np.where(smooth, T32, 0).astype(np.float32), device="cuda"),
                       torch.as_tensor(np.where(smooth, c32, 0).astype(np.float32), device="cuda"),
                       torch.as_tensor(dLdE, device="cuda"), g)
    ctx.sync()
    g = g.cpu().numpy().astype(np.float64)
    D_gpu = np.array([g @ v for v in probes])
    D_fd = np.array([np.sum(np.where(smooth, w * f, 0.0)) for f in fds])
    assert np.linalg.norm(D_fd[:8]) > 0 and np.linalg.norm(D_fd[8:]) > 0
    for part in (slice(0, 8), slice(8, None)):  # random directions, single heights
        err = np.linalg.norm(D_gpu[part] - D_fd[part]) / np.linalg.norm(D_fd[part])
        assert err <= 1e-2, (part, err)
