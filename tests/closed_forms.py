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


# --- rough interfaces (microfacet BSDFs, Walter et al. 2007) -----------------

def beckmann_D(cos_m, alpha):
    """Isotropic Beckmann normal distribution (solid-angle density of m times
    m.n integrates to one over the hemisphere)."""
    cos_m = np.asarray(cos_m, np.float64)
    c2 = np.clip(cos_m, 1e-300, None) ** 2
    return np.where(cos_m > 0, np.exp(-(1 - c2) / c2 / alpha ** 2) / (math.pi * alpha ** 2 * c2 ** 2), 0.0)


def smith_G1(c, cm, alpha):
    """Smith masking for the Beckmann distribution, exact Lambda (erf form)."""
    c, cm = np.asarray(c, np.float64), np.asarray(cm, np.float64)
    ac = np.clip(np.abs(c), 1e-300, 1.0)
    tan_t = np.sqrt(np.clip(1 - ac ** 2, 0, None)) / ac
    a = np.minimum(1.0 / (alpha * np.clip(tan_t, 1e-300, None)), 1e8)  # Lambda is 0 to double precision beyond
    from scipy.special import erf
    lam = 0.5 * (erf(a) - 1) + np.exp(-a * a) / (2 * a * math.sqrt(math.pi))
    g = np.where(tan_t > 0, 1 / (1 + lam), 1.0)
    return np.where(c * cm > 0, g, 0.0)


def fresnel_vec(cos1, eta1, eta2):
    cos1 = np.abs(np.asarray(cos1, np.float64))
    s2 = (eta1 / eta2) ** 2 * (1 - cos1 ** 2)
    c2 = np.sqrt(np.clip(1 - s2, 0, None))
    rs = (eta1 * cos1 - eta2 * c2) / (eta1 * cos1 + eta2 * c2)
    rp = (eta2 * cos1 - eta1 * c2) / (eta2 * cos1 + eta1 * c2)
    return np.where(s2 >= 1, 1.0, 0.5 * (rs * rs + rp * rp))


def rough_plane_irradiance(xD, nD, xL, light_n, alpha, eta_v, eta_other, refract, half_extent, n_r=400, n_phi=256,
                           r_max=4.0, centre=None):
    """Irradiance at x_D from one bounce off (refract=False) or through
    (refract=True) the rough plane z = 0, |x|, |y| <= half_extent, normal +z:
    the area integral over x_1 of
        f(l, v) |n.l| * |n.v| / d_D^2 * |n_D.w_D| * L(x_L -> x_1)
    with L = |n_L.l| / d_L^2 per unit emitter area (light_n given) or 1 / d_L^2
    (point light, light_n None), by Gauss-Legendre in r (r = r_max u^2 around
    `centre`) and the periodic trapezoid rule in phi.  eta_v: index on the
    receiver's side, eta_other: index on the far side of the interface (the
    light's side when refract)."""
    eta_l = eta_other if refract else eta_v
    xD, xL, nD = (np.asarray(a, np.float64) for a in (xD, xL, nD))
    c = np.asarray(centre if centre is not None else xD[:2], np.float64)
    u, wu = np.polynomial.legendre.leggauss(n_r)
    u = 0.5 * (u + 1)
    wu = 0.5 * wu
    r = r_max * u * u
    wr = wu * 2 * r_max * u * r  # dr = 2 r_max u du, area element r dr dphi
    phi = np.arange(n_phi) * (2 * math.pi / n_phi)
    R, P = np.meshgrid(r, phi, indexing="ij")
    W = np.broadcast_to(wr[:, None] * (2 * math.pi / n_phi), R.shape)
    X = np.stack([c[0] + R * np.cos(P), c[1] + R * np.sin(P), np.zeros_like(R)], -1)
    inside = (np.abs(X[..., 0]) <= half_extent) & (np.abs(X[..., 1]) <= half_extent)
    n = np.array([0.0, 0.0, 1.0])
    dv, dl = xD - X, xL - X
    d0, dL = np.linalg.norm(dv, axis=-1), np.linalg.norm(dl, axis=-1)
    v, l = dv / d0[..., None], dl / dL[..., None]
    cv, cl = v @ n, l @ n
    m = eta_v * v + eta_l * l
    m = m / np.linalg.norm(m, axis=-1)[..., None]
    m = np.where((m @ n)[..., None] < 0, -m, m)
    vm, lm, mn = (v * m).sum(-1), (l * m).sum(-1), m @ n
    D = beckmann_D(mn, alpha)
    G2 = smith_G1(cv, vm, alpha) * smith_G1(cl, lm, alpha)
    F = fresnel_vec(vm, eta_v, eta_other)
    if refract:
        den = eta_l * lm + eta_v * vm
        f = np.abs(lm) * np.abs(vm) / (np.abs(cl) * np.abs(cv)) * eta_v ** 2 * (1 - F) * D * G2 / den ** 2
        ok = cv * cl < 0
    else:
        f = F * D * G2 / (4 * np.abs(cl) * np.abs(cv))
        ok = cv * cl > 0
    wD = -v
    Lin = (np.abs(l @ np.asarray(light_n, np.float64)) if light_n is not None else 1.0) / dL ** 2
    val = f * np.abs(cl) * np.abs(cv) / d0 ** 2 * np.abs(wD @ nD) * Lin
    return float(np.sum(np.where(inside & ok, val, 0.0) * W))
