"""Pins of the oracle's glossy chains (Sec. 5.7, glossy chains): offset
normals drawn from the microfacet distribution, walks constrained to them,
and the estimate of each found chain.

* The offsets follow the Beckmann distribution they are drawn from (tan^2 of
  the normal's angle exponential with mean alpha^2, azimuth uniform), and that
  density on the unit disk of tangential components is D(m) itself.
* Zero offsets leave the specular walk unchanged bit for bit; a walk with
  offsets ends where the half-vector's tangential components are the offsets.
* Specular limit: with the microfacet density and shadowing divided out, the
  estimate L_e prod f |n.l| prod(area factors) / |det dC/du| (dense
  determinant of the full Jacobian) equals kappa G L_e of the specular path
  (generalized geometry term by the implicit function theorem) on every scene
  kind, point lights included -- an independent route to G and kappa.
* Unbiasedness: the Monte Carlo mean over offsets and seeds of W <1/P>
  (Bernoulli trials conditioned on the chain's offsets) equals the area
  integral of the rough-interface path integrand by quadrature, for rough
  reflection under a point light and rough refraction under an area light.
"""
import dataclasses
import math

import numpy as np
import pytest
from scipy import stats

import closed_forms as CF
import scenes
from oracle import oracle as O
from paper_2311_12818_gb300 import inputs as I


def _rough_dielectric_plane(xD, xL, spq):
    surf = I._surface(I.SURF_RECT, I.MAT_DIELECTRIC, 1.0, 1.5, (0, 0, 0), 0, (0, 0, 1), -1, (5, 0, 0), (0, 5, 0))
    light = I._light(I.LIGHT_POINT, xL, power=1.0)
    tg = I._target(I.TARGET_RECT, (0, 0, 0), 0, (1.5, 0, 0), (0, 1.5, 0), (0, 0, 1))
    return scenes.custom("rough_plane", surf, light, tg, xD, (0, 0, -1), xL, 1, 0, spq=spq)


def _polish(wl, sc, ch):
    tight = dataclasses.replace(wl, params=dataclasses.replace(wl.params, tol=1e-12))
    conv = dict(x=ch["x"], surf=ch["surf"], prim=ch["prim"], bary=ch["bary"], tau=ch["tau"],
                valid=(ch["status"] == 1).astype(np.uint8))
    return O.walk(tight, sc, conv)


def _point(wl, pos):
    return dataclasses.replace(wl, light=I._light(I.LIGHT_POINT, pos, power=1.0),
                               xL=np.tile(np.asarray(pos, np.float64), (wl.B, 1)))


@pytest.mark.parametrize("alpha", [0.05, 0.3])
def test_offsets_follow_the_beckmann_distribution(alpha):
    wl = I.mixed(nx=64, ny=32, spq=4)
    off = O.sample_offsets(wl, alpha)
    used = np.arange(8)[None, :] < wl.k[:, None]
    assert np.all(off[~used] == 0.0)
    o = off[used]
    r2 = (o ** 2).sum(-1)
    assert r2.max() < 1.0
    tan2 = r2 / (1.0 - r2)
    assert stats.kstest(tan2, stats.expon(scale=alpha ** 2).cdf).pvalue > 1e-3
    phi = np.arctan2(o[:, 1], o[:, 0])
    assert stats.kstest(phi, stats.uniform(-math.pi, 2 * math.pi).cdf).pvalue > 1e-3
    # consecutive vertices of a chain are independent draws
    two = used[:, 1]
    assert abs(np.corrcoef(off[two, 0, 0], off[two, 1, 0])[0, 1]) < 0.03
    # the density of the tangential components on the unit disk is D(m):
    # it integrates to one there (m.n = sqrt(1 - |o|^2))
    u, w = np.polynomial.legendre.leggauss(400)
    rho = 0.5 * (u + 1)
    mass = np.sum(0.5 * w * CF.beckmann_D(np.sqrt(1 - rho ** 2), alpha) * 2 * math.pi * rho)
    assert abs(mass - 1.0) < 1e-8
    # and the drawn |o| follow that density's radial CDF, 1 - exp(-rho^2 / ((1 - rho^2) alpha^2))
    cdf = lambda x: 1 - np.exp(-x ** 2 / ((1 - x ** 2) * alpha ** 2))  # noqa: E731
    assert stats.kstest(np.sqrt(r2), cdf).pvalue > 1e-3


def test_offsets_depend_on_the_counter_only():
    wl = I.glass_sphere(n=8, spq=4)
    a = O.sample_offsets(wl, 0.1)
    b = O.sample_offsets(wl, 0.1, rng_offset=5)
    assert np.array_equal(a[5:], b[:-5])
    assert not np.array_equal(a[:5], b[:5])


def test_zero_offsets_leave_the_walk_unchanged():
    wl = I.mixed(nx=24, ny=12, spq=4)
    sc = O.Scene(wl)
    s = O.sample_seeds(wl, sc)
    a = O.walk(wl, sc, s)
    b = O.walk(wl, sc, s, offset=np.zeros((wl.B, 8, 2)))
    for n in ("x", "surf", "status", "iters"):
        assert np.array_equal(a[n], b[n]), n


@pytest.mark.parametrize("which", ["glass", "water"])
def test_walk_solves_the_offset_constraint(which):
    wl = I.glass_sphere(n=16, spq=4) if which == "glass" else I.water(n=16, spq=4, grid=64)
    sc = O.Scene(wl)
    s = O.sample_seeds(wl, sc)
    off = O.sample_offsets(wl, 0.2)
    ch = O.walk(wl, sc, s, offset=off)
    ok = ch["status"] == 1
    assert ok.sum() > 0.2 * wl.B
    Cv, _ = O.constraint(wl, sc, ch)
    Cv = Cv.reshape(wl.B, 8, 2)
    for i in range(int(wl.k.max())):
        sel = ok & (wl.k > i)
        if i == 0:
            assert sel.sum() > 50
        if sel.any():
            assert np.abs(Cv[sel, i] - off[sel, i]).max() < wl.params.tol
    # the specular walk from the same seeds ends elsewhere
    plain = O.walk(wl, sc, s)
    both = ok & (plain["status"] == 1)
    assert np.median(np.linalg.norm(ch["x"][both, 0] - plain["x"][both, 0], axis=-1)) > 1e-3


@pytest.mark.parametrize("which", ["mirror_plane", "mirror_plane_area", "flat_water", "flat_water_point",
                                   "mirror_sphere", "glass_sphere", "glass_sphere_point", "water", "mixed",
                                   "mixed_point"])
def test_specular_limit_reproduces_kappa_G(which):
    rng = np.random.default_rng(11)
    up = np.c_[rng.uniform(-1, 1, (32, 2)), np.full(32, 1.0)]
    down = np.c_[rng.uniform(-1, 1, (32, 2)), np.full(32, -1.0)]
    wl = {"mirror_plane": lambda: scenes.mirror_plane(up, (0.3, 0.2, 2.0), point=True),
          "mirror_plane_area": lambda: scenes.mirror_plane(up, (0.3, 0.2, 2.0), point=False),
          "flat_water": lambda: scenes.flat_interface(down, (0.3, 0.2, 2.0)),
          "flat_water_point": lambda: _point(scenes.flat_interface(down, (0.3, 0.2, 2.0)), (0.3, 0.2, 2.0)),
          "mirror_sphere": lambda: I.mirror_sphere(n=16, spq=4),
          "glass_sphere": lambda: I.glass_sphere(n=16, spq=4),
          "glass_sphere_point": lambda: _point(I.glass_sphere(n=16, spq=4), (0.1, 0.2, 4.0)),
          "water": lambda: I.water(n=24, spq=4, grid=64),
          "mixed": lambda: I.mixed(nx=24, ny=12, spq=8),
          "mixed_point": lambda: _point(I.mixed(nx=24, ny=12, spq=8), (0.1, 0.2, 4.0))}[which]()
    sc = O.Scene(wl)
    ch = _polish(wl, sc, O.walk(wl, sc, O.sample_seeds(wl, sc)))
    con = O.contribution(wl, sc, ch)
    g = O.glossy(wl, sc, ch, alpha=0.0)
    adm = con["admissible"] == 1
    assert np.array_equal(adm, g["admissible"] == 1)
    assert adm.sum() > 50
    rel = np.abs(g["W"][adm] - con["T"][adm]) / con["T"][adm]
    assert rel.max() < 1e-7, rel.max()


def _mc(wl, alpha):
    sc = O.Scene(wl)
    s = O.sample_seeds(wl, sc)
    off = O.sample_offsets(wl, alpha)
    ch = O.walk(wl, sc, s, offset=off)
    g = O.glossy(wl, sc, ch, offset=off, alpha=alpha)
    N, capped = O.bernoulli(wl, sc, ch, g["admissible"], offset=off)
    assert capped.sum() == 0
    est = (g["W"] * N).reshape(wl.Q, wl.spq)
    return est.mean(1), est.std(1) / math.sqrt(wl.spq), N[g["admissible"] == 1]


@pytest.mark.parametrize("alpha", [0.02, 0.1, 0.3])
def test_rough_reflection_is_unbiased(alpha):
    """Rough dielectric plane (IOR 1.5) under a point light; one bounce."""
    xD = np.array([[0.2, -0.1, 1.0], [-0.4, 0.3, 1.2]])
    xL = (0.3, 0.2, 2.0)
    wl = _rough_dielectric_plane(xD, xL, spq=8000)
    mean, se, _ = _mc(wl, alpha)
    for q in range(wl.Q):
        ref = CF.rough_plane_irradiance(xD[q], (0, 0, -1), xL, None, alpha, 1.0, 1.5, False, 5.0)
        fine = CF.rough_plane_irradiance(xD[q], (0, 0, -1), xL, None, alpha, 1.0, 1.5, False, 5.0, n_r=800,
                                         n_phi=512)
        assert abs(ref - fine) < 1e-9 * ref
        assert abs(mean[q] - ref) < 4.5 * se[q] and abs(mean[q] - ref) < 1e-2 * ref, (q, mean[q], ref, se[q])


@pytest.mark.parametrize("alpha", [0.1, 0.3])
def test_rough_refraction_is_unbiased(alpha):
    """Rough water surface (IOR 1.33) under an area light, receivers in the
    water; the seeds often miss, so the Bernoulli trials carry weight."""
    xD = np.array([[0.2, -0.1, -1.0], [-0.6, 0.3, -0.8]])
    xL = (0.3, 0.2, 2.0)
    wl = scenes.flat_interface(xD, xL, etaB=1.33, spq=20000)
    mean, se, N = _mc(wl, alpha)
    assert N.mean() > 1.5  # trials beyond the first are exercised
    for q in range(wl.Q):
        ref = CF.rough_plane_irradiance(xD[q], (0, 0, 1), xL, (0, 0, -1), alpha, 1.33, 1.0, True, 5.0)
        fine = CF.rough_plane_irradiance(xD[q], (0, 0, 1), xL, (0, 0, -1), alpha, 1.33, 1.0, True, 5.0, n_r=800,
                                         n_phi=512)
        assert abs(ref - fine) < 1e-9 * ref
        assert abs(mean[q] - ref) < 4.5 * se[q] and abs(mean[q] - ref) < 5e-2 * ref, (q, mean[q], ref, se[q])
