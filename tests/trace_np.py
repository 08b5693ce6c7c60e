"""Independent FP64 ray tracer of analytic specular scenes, for the oracle's
pins: spheres, spherical caps and rectangles read from the surface table
format of the inputs module, nearest hits, mirror reflection and Snell
refraction in vector form, and the forward shooting map x_D, w_D -> chain
vertices -> light plane.  Written from the geometry with numpy only; it does
not call or mirror the oracle.

Surface rows: 0 type, 1 material, 2 eta_front, 3 eta_back, 4..6 centre,
7 radius, 8..10 cap axis / rectangle normal, 11 cap cosine, 12..14 and
15..17 rectangle half-axes.  The front side is the side the outward normal
points into."""
import math

import numpy as np

SPHERE, CAP, RECT = 0, 1, 2
MIRROR = 0


def unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


def surface_hits(row, o, d, tmin):
    """Parameters t > tmin where the ray o + t d meets the surface row."""
    typ = int(row[0])
    c = row[4:7]
    if typ in (SPHERE, CAP):
        r = row[7]
        dd = d @ d
        oc = o - c
        half_b = oc @ d
        disc = half_b * half_b - dd * (oc @ oc - r * r)
        if disc < 0:
            return []
        s = math.sqrt(disc)
        out = []
        for t in ((-half_b - s) / dd, (-half_b + s) / dd):
            if t <= tmin:
                continue
            if typ == CAP and (o + t * d - c) @ row[8:11] < r * row[11]:
                continue
            out.append(t)
        return out
    if typ == RECT:
        n = row[8:11]
        den = d @ n
        if den == 0:
            return []
        t = ((c - o) @ n) / den
        if t <= tmin:
            return []
        q = o + t * d - c
        ex, ey = row[12:15], row[15:18]
        if abs(q @ ex) > ex @ ex or abs(q @ ey) > ey @ ey:
            return []
        return [t]
    raise ValueError("surface type %d not traced here" % typ)


def nearest(surfaces, o, d, tmin=1e-9):
    """(t, surface index) of the nearest hit, or (None, -1)."""
    best, idx = None, -1
    for j, row in enumerate(surfaces):
        for t in surface_hits(row, o, d, tmin):
            if best is None or t < best:
                best, idx = t, j
    return best, idx


def normal(row, p):
    """Outward (front-side) unit normal of a surface at p."""
    if int(row[0]) in (SPHERE, CAP):
        return unit(p - row[4:7])
    return unit(row[8:11])


def etas(row, n, w_toward_prev):
    """IORs on the side of the previous vertex and on the other side."""
    if int(row[1]) == MIRROR:
        return 1.0, 1.0
    if w_toward_prev @ n > 0:
        return row[2], row[3]
    return row[3], row[2]


def reflect(d, n):
    return d - 2.0 * (d @ n) * n


def refract(d, n, eta1, eta2):
    """Snell's law in vector form for the propagation direction d; n may face
    either side.  None on total internal reflection."""
    if d @ n > 0:
        n = -n
    c = -(d @ n)
    e = eta1 / eta2
    k2 = 1.0 - e * e * (1.0 - c * c)
    if k2 < 0:
        return None
    return unit(e * d + (e * c - math.sqrt(k2)) * n)


def shoot(surfaces, xD, w, k, tau, tmin=1e-9, scatter_last=True):
    """Traces k specular vertices from x_D along w with types tau (bit i-1 set:
    vertex i refracts).  Returns (points [k,3], surface ids [k], outgoing
    direction of the last vertex) or None when a ray misses, a mirror is
    asked to refract, or refraction is totally reflected.  With
    scatter_last=False the last vertex is not scattered (a seed chain needs
    k - 1 scattered directions; the outgoing direction is then None)."""
    o, d = np.asarray(xD, np.float64), unit(w)
    pts, ids = [], []
    for i in range(k):
        t, j = nearest(surfaces, o, d, tmin)
        if t is None:
            return None
        p = o + t * d
        row = surfaces[j]
        if i == k - 1 and not scatter_last:
            pts.append(p)
            ids.append(j)
            return np.array(pts), np.array(ids), None
        n = normal(row, p)
        if (tau >> i) & 1:
            if int(row[1]) == MIRROR:
                return None
            e1, e2 = etas(row, n, -d)
            d2 = refract(d, n, e1, e2)
            if d2 is None:
                return None
        else:
            d2 = unit(reflect(d, n))
        pts.append(p)
        ids.append(j)
        o, d = p, d2
    return np.array(pts), np.array(ids), d


def plane_hit(o, d, c, n):
    den = d @ n
    if den == 0:
        return None
    t = ((c - o) @ n) / den
    return None if t <= 0 else o + t * d
