"""Pins of the FP64 oracle on the mixed-length scene (nested glass spheres,
four stacked biconvex lenses made of spherical caps, a mirror; chains of
k = 1..8 with random types), against what the geometry fixes independently:

* seed deduction (Eq. deduction, Sec. 5.3) against an independent numpy
  trace of the same direction through the caps, spheres and mirror;
* the generalized Snell law (the half-vector constraint of the manifold
  walk, Sec. 3) at every vertex of every converged chain, in vector form,
  in scalar form and as coplanarity, and the vertex types against the sides
  the chain crosses;
* the generalized geometry term of Eq. ThroughputEval against central
  differences of the independently traced forward shooting map
  w_D -> x_L for chains of k = 3..8.

None of these tests use the CUDA path."""
import numpy as np
import pytest

import trace_np as TN
from oracle import oracle as O
from paper_2311_12818_gb300 import inputs as I


@pytest.fixture(scope="module")
def mixed_run():
    wl = I.mixed(nx=128, ny=64, spq=32)
    wl.params.tol = 1e-12
    sc = O.Scene(wl)
    seeds = O.sample_seeds(wl, sc, threads=8)
    ch = O.walk(wl, sc, seeds, threads=8)
    con = O.contribution(wl, sc, ch, threads=8)
    return wl, seeds, ch, con


def test_mixed_seed_deduction_matches_independent_trace(mixed_run):
    wl, seeds, ch, con = mixed_run
    rng = np.random.default_rng(1)
    checked = np.zeros(9, int)
    for k in range(1, 9):
        ok = np.nonzero((seeds["valid"] == 1) & (wl.k == k))[0]
        for b in rng.permutation(ok)[:150]:
            q = b // wl.spq
            w = TN.unit(seeds["x"][b, 0] - wl.xD[q])
            r = TN.shoot(wl.surfaces, wl.xD[q], w, k, int(seeds["tau"][b]), tmin=1e-7, scatter_last=False)
            assert r is not None, b
            pts, ids, _ = r
            assert np.array_equal(ids, seeds["surf"][b, :k]), b
            assert np.abs(pts - seeds["x"][b, :k]).max() < 1e-10, b
            checked[k] += 1
    # caps of the lenses and both nested spheres are crossed by the long chains
    assert (checked[1:] > 0).all(), checked
    surfs = set(np.unique(seeds["surf"][(seeds["valid"] == 1)][:, :8]).tolist()) - {-1}
    assert set(range(wl.surfaces.shape[0])) <= surfs


def _normals(wl, pts, ids):
    """Outward normals of the surfaces ids at the points pts (vectorised)."""
    rows = wl.surfaces[ids]
    curved = rows[:, 0] != I.SURF_RECT
    n = np.where(curved[:, None], pts - rows[:, 4:7], rows[:, 8:11])
    return n / np.linalg.norm(n, axis=1, keepdims=True), rows


def test_mixed_vector_snell_at_every_converged_vertex(mixed_run):
    wl, seeds, ch, con = mixed_run
    seen = np.zeros(9, int)
    for k in range(1, 9):
        bs = np.nonzero((ch["status"] == I.ST_CONVERGED) & (wl.k == k))[0]
        if bs.size == 0:
            continue
        q = bs // wl.spq
        chain = np.concatenate([wl.xD[q][:, None], ch["x"][bs, :k], wl.xL[bs][:, None]], axis=1)
        tau = ch["tau"][bs].astype(np.int64)
        adm = con["admissible"][bs] == 1
        for i in range(1, k + 1):
            p = chain[:, i]
            wi = chain[:, i - 1] - p
            wo = chain[:, i + 1] - p
            wi /= np.linalg.norm(wi, axis=1, keepdims=True)
            wo /= np.linalg.norm(wo, axis=1, keepdims=True)
            n, rows = _normals(wl, p, ch["surf"][bs, i - 1])
            # the vertex lies on its surface
            curved = rows[:, 0] != I.SURF_RECT
            rad = np.linalg.norm(p - rows[:, 4:7], axis=1)
            off = np.where(curved, np.abs(rad - rows[:, 7]), np.abs(np.sum((p - rows[:, 4:7]) * rows[:, 8:11], 1)))
            assert off.max() < 1e-12
            refr = ((tau >> (i - 1)) & 1) == 1
            mirror = rows[:, 1] == I.MAT_MIRROR
            si, so = np.sum(wi * n, 1), np.sum(wo * n, 1)
            eta_i = np.where(mirror, 1.0, np.where(si > 0, rows[:, 2], rows[:, 3]))
            eta_o = np.where(refr & ~mirror, np.where(si > 0, rows[:, 3], rows[:, 2]), eta_i)
            h = eta_i[:, None] * wi + eta_o[:, None] * wo
            # vector Snell: eta_i w_i + eta_o w_o is parallel to n
            assert np.linalg.norm(np.cross(h, n), axis=1).max() < 1e-9
            # coplanarity of w_i, w_o and n
            assert np.abs(np.sum(np.cross(wi, wo) * n, 1)).max() < 1e-9
            # scalar Snell: eta_i sin(theta_i) = eta_o sin(theta_o)
            sin_i = np.linalg.norm(np.cross(wi, n), axis=1)
            sin_o = np.linalg.norm(np.cross(wo, n), axis=1)
            assert np.abs(eta_i * sin_i - eta_o * sin_o).max() < 1e-9
            # admissible chains cross the surface exactly where they refract
            assert np.array_equal((si[adm] > 0) != (so[adm] > 0), refr[adm])
        seen[k] = bs.size
    assert (seen[1:] > 0).all(), seen


def _light_hit(wl, q, w, k, tau):
    r = TN.shoot(wl.surfaces, wl.xD[q], w, k, tau, tmin=1e-7)
    if r is None:
        return None, None, None
    pts, ids, d = r
    return TN.plane_hit(pts[-1], d, wl.light[1:4], wl.light[4:7]), ids, pts


def test_mixed_G_against_fd_of_independent_shooting(mixed_run):
    """G = cos(theta_D) |det d(w_D)/d(u_L)| = cos(theta_D) / |det d(u_L)/d(w_D)|
    with u_L the light's orthonormal (x, y) coordinates: central differences
    of the traced map at h = 3e-8 (its h^2 term stays below 1e-7 relative
    on these chains, rounding below 1e-8)."""
    wl, seeds, ch, con = mixed_run
    assert abs(wl.light[7:10] @ [1, 0, 0]) > 0 and abs(wl.light[10:13] @ [0, 1, 0]) > 0  # axes x, y
    rng = np.random.default_rng(2)
    checked = np.zeros(9, int)
    h = 3e-8
    for k in range(3, 9):
        adm = np.nonzero((con["admissible"] == 1) & (wl.k == k))[0]
        for b in rng.permutation(adm)[:40]:
            q = b // wl.spq
            tau = int(ch["tau"][b])
            w = TN.unit(ch["x"][b, 0] - wl.xD[q])
            xl, ids, pts = _light_hit(wl, q, w, k, tau)
            # the traced chain is the converged one and reaches its x_L
            assert xl is not None and np.array_equal(ids, ch["surf"][b, :k])
            assert np.abs(pts - ch["x"][b, :k]).max() < 1e-8
            assert np.linalg.norm(xl - wl.xL[b]) < 1e-8
            a = TN.unit(np.cross(w, [0.1, 0.2, 0.97]))
            c = np.cross(w, a)
            cols = []
            for t in (a, c):
                up, iu, _ = _light_hit(wl, q, TN.unit(w + h * t), k, tau)
                um, im, _ = _light_hit(wl, q, TN.unit(w - h * t), k, tau)
                assert np.array_equal(iu, ids) and np.array_equal(im, ids)
                cols.append((up - um)[:2] / (2 * h))
            G_fd = abs(w @ wl.nD[q]) / abs(np.linalg.det(np.array(cols).T))
            assert abs(con["G"][b] - G_fd) < 1e-6 * G_fd, (b, k, con["G"][b], G_fd)
            checked[k] += 1
    # lens stacks and nested spheres give admissible chains of 3, 5, 6, 7 and 8 vertices
    assert checked[3] >= 40 and checked[5] >= 40 and checked[6] > 0 and checked[7] > 0 and checked[8] > 0, checked
