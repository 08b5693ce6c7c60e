"""Pins of the glossy-separator extension (Sec. 5.7): the normalised Phong
separator BSDF integrates, against the cosine, to one for a normal camera ray
and to at most one otherwise (quadrature); product importance sampling only
reweights the guide, so the radiance estimate stays unbiased: on the mirror
sphere's single-solution point it converges to rho(w_i, w_D*) T either way."""
import dataclasses
import math

import numpy as np
import pytest
from scipy import integrate

import scenes
from oracle import oracle as O
from paper_2311_12818_gb300 import inputs as I


@pytest.mark.parametrize("e", [1.0, 10.0, 200.0])
def test_phong_lobe_normalisation(e):
    n = np.array([[0.0, 0.0, 1.0]])

    def flux(w_i):
        def f(th, ph):
            w = np.array([[math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)]])
            return O.phong(w_i, n, w, e)[0] * math.cos(th) * math.sin(th)
        return integrate.dblquad(lambda th, ph: f(th, ph), 0.0, 2 * math.pi, 0.0, math.pi / 2,
                                 epsabs=1e-10, epsrel=1e-8)[0]
    assert abs(flux(np.array([[0.0, 0.0, -1.0]])) - 1.0) < 1e-6  # camera ray along -n: lobe around +n
    oblique = np.array([[math.sin(1.0), 0.0, -math.cos(1.0)]])
    assert 0.0 < flux(oblique) <= 1.0 + 1e-9


def test_radiance_estimate_unbiased_with_product_weights():
    base = I.mirror_sphere(n=2, spq=1)
    M = 4096
    wl = scenes.custom("mirror_sphere_point", base.surfaces, base.light, base.targets,
                       np.array([[0.35, 0.9, -1.5]]), (0, 0, 1), base.light[1:4], 1, 0, spq=M)
    wl.rng_seed = 0xBEEF
    cam, e = (0.0, -4.0, 2.0), 20.0
    sc = O.Scene(wl)
    seeds = O.sample_seeds(wl, sc)
    ch = O.walk(wl, sc, seeds)
    con = O.contribution(wl, sc, ch)
    N, _ = O.bernoulli(wl, sc, ch, con["admissible"])
    adm = con["admissible"] == 1
    cell, om, w = O.records(wl, ch, con["T"], N, con["admissible"])
    chain = np.nonzero(adm)[0]
    wp = O.records_bsdf(wl, chain, om, w, cam, e)
    # the single solution's radiance toward the camera
    rho = O.phong(O.camera_rays(wl, cam), wl.nD, om[:1].astype(np.float64), e)[0]
    L_true = rho * con["T"][adm][0]
    for weights in (w, wp):
        g = O.Guide(wl.n_cells, I.guide_edges())
        g.update(cell, om, weights, wl.params.weight_shift)
        s2 = O.sample_seeds(wl, sc, g, rng_offset=1 << 30)
        c2 = O.walk(wl, sc, s2)
        k2 = O.contribution(wl, sc, c2)
        N2, _ = O.bernoulli(wl, sc, c2, k2["admissible"], g, rng_offset=1 << 30)
        contrib = np.where(k2["admissible"] == 1, wl.light_area * k2["T"] * N2 / wl.pn, 0.0)
        c, L = O.separator_radiance(wl, c2, contrib, cam, e)
        assert abs(L[0] - L_true) < 4 * c.std() / math.sqrt(M) + 1e-12


def test_product_weights_and_radiance_on_the_mirror_direction():
    """A direction along the mirror of the camera ray about the receiver normal
    gets the lobe's peak (e + 2) / (2 pi); one perpendicular to it gets zero --
    for the records' product weights and for the chains' radiance alike."""
    wl = I.glass_sphere(n=4, spq=2)
    cam, e = (0.3, -2.0, 1.0), 30.0
    xD, nD = wl.xD, wl.nD
    wi = (xD - np.array(cam)) / np.linalg.norm(xD - np.array(cam), axis=1, keepdims=True)
    r = wi - 2 * np.sum(wi * nD, axis=1, keepdims=True) * nD   # mirror of the camera ray
    perp = np.cross(r, [0.0, 0.0, 1.0])
    perp /= np.linalg.norm(perp, axis=1, keepdims=True)
    chain = np.arange(wl.B)
    q = chain // wl.spq
    om = np.where((chain % 2 == 0)[:, None], r[q], perp[q]).astype(np.float32)
    w = np.full(wl.B, 0.5, np.float32)
    got = O.records_bsdf(wl, chain, om, w, cam, e)
    peak = (e + 2) / (2 * math.pi)
    assert np.allclose(got[0::2], 0.5 * peak, rtol=1e-5) and np.all(got[1::2] < 1e-12)
    x = np.zeros((wl.B, I.MAXK, 3))
    x[:, 0, :] = xD[q] + 2.0 * om.astype(np.float64)
    c, L = O.separator_radiance(wl, dict(x=x), np.ones(wl.B), cam, e)
    assert np.allclose(c[0::2], peak, rtol=1e-5) and np.all(c[1::2] < 1e-12)
    assert np.allclose(L, peak / 2, rtol=1e-5)
