"""Flux balance (energy conservation) through a flat interface: a light in air
above a water surface (IOR 1.33) and a receiver disk of radius R below it.

Point light of intensity I: the power the disk receives, the integral of the
oracle's irradiance E = I kappa G over it, equals the power the light sends
through the interface into the directions that refract onto the disk,
2 pi I int_0^theta_max (1 - F(theta)) sin(theta) d theta with the textbook
Fresnel transmittance.

Area light (a Lambertian emitter of radiance L facing the water): the
oracle's T at one emitter point is the irradiance per unit emitter area, so
its integral over the disk equals the power one unit of emitter area sends
onto it, 2 pi L int_0^theta_max (1 - F) cos(theta) sin(theta) d theta.  This
holds only with the (eta_water / eta_air)^2 radiance scaling in kappa, which
the point-light balance must not have.

Both integrals are one-dimensional by symmetry (Gauss-Legendre on the
receiver side, adaptive quadrature on the light side)."""
import math

import numpy as np
from scipy import integrate, optimize

import closed_forms as CF
import scenes
from oracle import oracle as O
from paper_2311_12818_gb300 import inputs as I


def _balance(point):
    hL, hD, R, eta = 1.0, 1.0, 1.2, 1.33
    nodes, weights = np.polynomial.legendre.leggauss(24)
    r = 0.5 * R * (nodes + 1.0)
    wr = 0.5 * R * weights
    xD = np.stack([r, np.zeros_like(r), np.full_like(r, -hD)], axis=1)
    surf = I._surface(I.SURF_RECT, I.MAT_DIELECTRIC, 1.0, eta, (0, 0, 0), 0, (0, 0, 1), -1, (5, 0, 0), (0, 5, 0))
    if point:
        light = I._light(I.LIGHT_POINT, (0.0, 0.0, hL), power=1.0)
    else:
        light = I._light(I.LIGHT_RECT, (0.0, 0.0, hL), normal=(0, 0, -1), ex=(0.01, 0, 0), ey=(0, 0.01, 0),
                         power=1.0)
    tg = I._target(I.TARGET_RECT, (0, 0, 0), 0, (2.0, 0, 0), (0, 2.0, 0), (0, 0, 1))
    wl = scenes.custom("flux", surf, light, tg, xD, (0, 0, 1), (0.0, 0.0, hL), 1, 1, spq=64, tol=1e-12)
    sc = O.Scene(wl)
    s = O.sample_seeds(wl, sc)
    ch = O.walk(wl, sc, s)
    con = O.contribution(wl, sc, ch)
    E = np.zeros(r.size)
    for q in range(r.size):
        b = np.nonzero(con["admissible"][q * wl.spq:(q + 1) * wl.spq])[0]
        assert b.size > 0, q
        T = con["T"][q * wl.spq + b]
        assert np.all(np.abs(T - T[0]) < 1e-10 * T[0])  # one solution per point
        E[q] = T[0]
    received = 2 * math.pi * float(np.sum(wr * r * E))
    # light side: the polar angle in air whose refracted ray lands at radius R
    land = lambda th: hL * math.tan(th) + hD * math.tan(math.asin(math.sin(th) / eta)) - R  # noqa: E731
    th_max = optimize.brentq(land, 0.0, math.pi / 2 - 1e-9, xtol=1e-15)
    emit = (lambda th: 1.0) if point else math.cos  # intensity, or Lambertian radiance x cos
    sent = 2 * math.pi * integrate.quad(lambda th: (1 - CF.fresnel_unpolarised(math.cos(th), 1.0, eta))
                                        * emit(th) * math.sin(th), 0.0, th_max, epsabs=0, epsrel=1e-12)[0]
    return received, sent


def test_point_light_flux_balance_through_a_water_surface():
    received, sent = _balance(point=True)
    assert abs(received - sent) < 1e-4 * sent, (received, sent, received / sent)


def test_area_light_flux_balance_through_a_water_surface():
    received, sent = _balance(point=False)
    assert abs(received - sent) < 1e-4 * sent, (received, sent, received / sent)
