"""Closed-form and independent reference solutions used to pin the oracle.

Written from the mathematics (law of reflection, Snell's law, Fresnel
equations, solid-angle/area Jacobians) with numpy/scipy only -- nothing here
calls or mirrors the oracle's code paths.
"""
import math

import numpy as np
from scipy.optimize import brentq


def unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


def alhazen_sphere(xD, xL, c=(0.0, 0.0, 0.0), r=1.0, n_scan=20000, visible_only=True):
    """Reflection points on a sphere between two external points (Alhazen's
    problem).  The reflection point lies in the plane through the centre, x_D
    and x_L; on the circle p(t) = c + r (cos t e1 + sin t e2) the normal bisects
    the two unit directions, i.e. cross2(p - c, u_D + u_L) = 0.  Returns the
    roots seen from both points (in front of the tangent plane), or all roots
    of the equation with visible_only=False."""
    c = np.asarray(c, np.float64)
    D, L = np.asarray(xD, np.float64) - c, np.asarray(xL, np.float64) - c
    e1 = unit(D)
    l2 = L - e1 * (L @ e1)
    if np.linalg.norm(l2) < 1e-12:
        return []
    e2 = unit(l2)
    D2 = np.array([D @ e1, D @ e2])
    L2 = np.array([L @ e1, L @ e2])

    def f(t):
        p = r * np.array([math.cos(t), math.sin(t)])
        uD, uL = unit(D2 - p), unit(L2 - p)
        s = uD + uL
        return p[0] * s[1] - p[1] * s[0]

    ts = np.linspace(0, 2 * math.pi, n_scan + 1)
    fs = np.array([f(t) for t in ts])
    roots = []
    for i in range(n_scan):
        if fs[i] == 0 or fs[i] * fs[i + 1] < 0:
            t = brentq(f, ts[i], ts[i + 1], xtol=1e-15, rtol=1e-15, maxiter=200)
            p2 = r * np.array([math.cos(t), math.sin(t)])
            if not visible_only or ((D2 - p2) @ p2 > 0 and (L2 - p2) @ p2 > 0):
                roots.append(c + p2[0] * e1 + p2[1] * e2)
    # de-duplicate roots found on neighbouring intervals
    out = []
    for p in roots:
        if all(np.linalg.norm(p - q) > 1e-9 for q in out):
            out.append(p)
    return out


def mirror_plane_point(xD, xL, o, n):
    """Reflection point on the plane (o, n): intersection of the segment from x_D
    to the mirror image of x_L."""
    n = unit(n)
    xL_img = xL - 2.0 * ((xL - o) @ n) * n
    d = xL_img - xD
    t = ((o - xD) @ n) / (d @ n)
    return xD + t * d, np.linalg.norm(d)


def snell_flat(hD, hL, rho, etaD, etaL):
    """Refraction through a flat interface: the receiver point at depth hD below
    the interface (index etaD), the light point at height hL above (index etaL),
    horizontal distance rho.  Solves etaD sin(thD) = etaL sin(thL) with
    rho = hD tan(thD) + hL tan(thL) by bisection; returns thD, thL and the radial
    offset of the refraction point from x_D's vertical."""
    def g(thD):
        s = etaD * math.sin(thD) / etaL
        if s >= 1.0:
            return float("inf")
        thL = math.asin(s)
        return hD * math.tan(thD) + hL * math.tan(thL) - rho
    hi = math.pi / 2 - 1e-12
    if etaD > etaL:
        hi = min(hi, math.asin(etaL / etaD) - 1e-15)
    thD = brentq(g, 0.0, hi, xtol=1e-16, rtol=1e-15, maxiter=500)
    thL = math.asin(etaD * math.sin(thD) / etaL)
    return thD, thL, hD * math.tan(thD)


def fresnel_unpolarised(cos1, eta1, eta2):
    """Fresnel equations (s and p amplitude coefficients averaged in power)."""
    s2 = (eta1 / eta2) ** 2 * (1.0 - cos1 ** 2)
    if s2 >= 1.0:
        return 1.0
    cos2 = math.sqrt(1.0 - s2)
    rs = (eta1 * cos1 - eta2 * cos2) / (eta1 * cos1 + eta2 * cos2)
    rp = (eta2 * cos1 - eta1 * cos2) / (eta2 * cos1 + eta1 * cos2)
    return 0.5 * (rs * rs + rp * rp)


def flat_interface_G(hD, hL, thD, thL, etaD, etaL):
    """G = cos(thD) |d w_D / d A_L| for a horizontal light plane: by rotational
    symmetry dA_L = rho d rho d phi and d w_D = sin(thD) d thD d phi, with
    d rho/d thD = hD / cos^2 thD + hL / cos^2 thL * d thL/d thD and
    d thL/d thD = etaD cos thD / (etaL cos thL)."""
    rho = hD * math.tan(thD) + hL * math.tan(thL)
    dthL = etaD * math.cos(thD) / (etaL * math.cos(thL))
    drho = hD / math.cos(thD) ** 2 + hL / math.cos(thL) ** 2 * dthL
    return math.cos(thD) * math.sin(thD) / (rho * drho)
