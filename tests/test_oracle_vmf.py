"""Pins of the oracle's vMF mixture guide (Sec. 5.5, Eq. vMF): lobe density and
sampler against closed forms, the lobe construction (kappa = sigma^-2 from the
nearest direction of the same group) on hand-built records, the discrete
distributions P_e(n) and P_e(tau | n) by their frequencies, the seed density
by the importance-sampling identity E[1{valid}/p] = solid angle of the valid
set, and the estimator's unbiasedness when the chain length is sampled."""
import dataclasses
import math

import numpy as np
import pytest
from scipy import integrate, stats

import scenes
from oracle import oracle as O
from paper_2311_12818_gb300 import inputs as I


def _dirs_on_circle(angles, axis=(0.0, 0.0, 1.0), tilt=0.3):
    """Unit vectors at the given angles along a great circle through `axis`."""
    a = np.asarray(axis, np.float64) / np.linalg.norm(axis)
    e = np.cross(a, [math.sin(tilt), math.cos(tilt), 0.0])
    e /= np.linalg.norm(e)
    ang = np.asarray(angles, np.float64)
    return np.cos(ang)[:, None] * a[None, :] + np.sin(ang)[:, None] * e[None, :]


# --------------------------------------------------------------------------
# Lobe density and sampler (Eq. vMF)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kappa", [0.1, 1.0, 10.0, 1e3, 1e6])
def test_vmf_density_integrates_to_one(kappa):
    mu = np.array([0.0, 0.0, 1.0])

    def ring(t):  # integral over the azimuth at 1 - mu.w = t (the density is symmetric about mu)
        ct = 1.0 - t
        st = math.sqrt(max(0.0, t * (2.0 - t)))
        return 2.0 * math.pi * O.vmf_pdf(mu, kappa, [st, 0.0, ct])

    # split [0, 2] at the lobe's scale so quad resolves the peak
    s = min(2.0, 50.0 / kappa)
    a, _ = integrate.quad(ring, 0.0, s, limit=200, epsabs=0, epsrel=1e-11)
    b, _ = integrate.quad(ring, s, 2.0, limit=200, epsabs=0, epsrel=1e-11) if s < 2.0 else (0.0, 0.0)
    assert abs(a + b - 1.0) < 1e-8
    # and it is rotation invariant: the same value at a rotated pair
    w = np.array([0.3, -0.2, 0.9])
    w /= np.linalg.norm(w)
    R = np.linalg.qr(np.random.default_rng(1).normal(size=(3, 3)))[0]
    assert math.isclose(O.vmf_pdf(mu, kappa, w), O.vmf_pdf(R @ mu, kappa, R @ w), rel_tol=1e-9)


@pytest.mark.parametrize("kappa", [0.5, 4.0, 60.0, 1e4])
def test_vmf_sampler_moments_match_closed_form(kappa):
    # mean resultant length of the 3-D vMF: E[mu.w] = coth(kappa) - 1/kappa,
    # and E[(mu.w)^2] = 1 - 2 (coth(kappa) - 1/kappa) / kappa
    mu = np.array([0.48, -0.6, 0.64])
    mu /= np.linalg.norm(mu)
    n = 400
    u = (np.arange(n) + 0.5) / n  # stratified in both coordinates
    W = np.array([O.vmf_sample(mu, kappa, u1, u2) for u1 in u for u2 in u[::8]])
    assert np.allclose(np.linalg.norm(W, axis=1), 1.0, atol=1e-12)
    c = W @ mu
    A = 1.0 / math.tanh(kappa) - 1.0 / kappa
    assert abs(c.mean() - A) < 2e-3 * max(1.0 - A, 1e-3) + 1e-9
    assert abs((c ** 2).mean() - (1.0 - 2.0 * A / kappa)) < 3e-3 * max(1.0 - A, 1e-3) + 1e-9
    # the mean direction is mu (the azimuth is uniform about it)
    m = W.mean(axis=0)
    assert np.linalg.norm(m - A * mu) < 1e-2 * max(1.0 - A, 1e-2) + 1e-9


def test_vmf_sampler_follows_its_density():
    kappa = 25.0
    mu = np.array([0.0, 0.6, 0.8])
    rng = np.random.default_rng(7)
    u1 = 1.0 - rng.random(20000)
    u2 = rng.random(20000)
    t = np.array([1.0 - O.vmf_sample(mu, kappa, a, b) @ mu for a, b in zip(u1, u2)])
    edges = np.array([0.0, 0.005, 0.01, 0.02, 0.04, 0.07, 0.12, 0.2, 2.0])

    def mass(lo, hi):  # probability of lo <= t < hi from the density by quadrature
        e = np.cross(mu, [1.0, 0.0, 0.0])
        e /= np.linalg.norm(e)
        f = lambda tt: 2 * math.pi * O.vmf_pdf(mu, kappa, (1 - tt) * mu + math.sqrt(max(0.0, tt * (2 - tt))) * e)
        return integrate.quad(f, lo, hi, epsrel=1e-10)[0]

    p = np.array([mass(a, b) for a, b in zip(edges[:-1], edges[1:])])
    assert abs(p.sum() - 1.0) < 1e-8
    obs = np.histogram(t, edges)[0]
    assert stats.chisquare(obs, p * t.size).pvalue > 1e-3


# --------------------------------------------------------------------------
# Lobe construction
# --------------------------------------------------------------------------
def test_lobes_kappa_from_nearest_direction_of_the_group():
    ang = np.array([0.0, 0.1, 0.3, 0.6, 1.0])
    d = _dirs_on_circle(ang)
    # nearest-neighbour angles along the circle: 0.1, 0.1, 0.2, 0.3, 0.4
    sig = np.array([0.1, 0.1, 0.2, 0.3, 0.4])
    # records: cell 1 holds the circle (n=2, tau=1), a lone (n=2, tau=2) record
    # equal to one of them, and two identical directions (n=1, tau=0); cell 0 a
    # lone record.  Record order is scrambled.
    om = np.concatenate([d, d[2:3], d[4:5], d[4:5], d[0:1]]).astype(np.float32)
    cell = np.array([1, 1, 1, 1, 1, 1, 1, 1, 0], np.uint32)
    k = np.array([2, 2, 2, 2, 2, 2, 1, 1, 3], np.uint8)
    tau = np.array([1, 1, 1, 1, 1, 2, 0, 0, 5], np.uint8)
    w = np.array([1.0, 2.0, 0.5, 0.25, 3.0, 1.5, 0.75, 1.25, 2.0], np.float32)
    perm = np.array([6, 3, 0, 8, 5, 1, 7, 4, 2])
    g = O.VmfGuide(3).build(cell[perm], om[perm], w[perm], k[perm], tau[perm], 16)
    assert list(g.cell_start) == [0, 1, 9, 9]
    key = list(g.key[:9])
    assert key == [(3 << 8) | 5, (1 << 8), (1 << 8), (2 << 8) | 1, (2 << 8) | 1, (2 << 8) | 1, (2 << 8) | 1,
                   (2 << 8) | 1, (2 << 8) | 2]
    # within a key the record order is kept: the circle records were given as
    # perm positions of 3, 0, 1, 4, 2
    circle_order = [r for r in perm if r < 5]
    mu = g.lobe[3:8, :3]
    assert np.allclose(mu, d[circle_order].astype(np.float32), atol=0)
    kap = g.lobe[3:8, 3]
    assert np.allclose(kap, 1.0 / sig[circle_order] ** 2, rtol=1e-6)  # FP32 directions
    # a lone sample: sigma = pi; identical directions: sigma at its 1e-6 floor
    assert math.isclose(g.lobe[0, 3], 1.0 / math.pi ** 2, rel_tol=1e-12)
    assert math.isclose(g.lobe[8, 3], 1.0 / math.pi ** 2, rel_tol=1e-12)
    assert np.allclose(g.lobe[1:3, 3], 1e12, rtol=1e-9)
    # prefix sums of q = floor(w 2^16) within each cell, in lobe order
    q = np.floor(w[perm].astype(np.float64) * 65536).astype(np.uint64)
    order = [3, 0, 6, 1, 2, 5, 7, 8, 4]  # perm positions in lobe order
    assert list(g.prefix[:1]) == [q[order[0]]]
    assert list(g.prefix[1:9]) == list(np.cumsum(q[order[1:]]))


def test_lobe_build_rejects_bad_records():
    g = O.VmfGuide(2)
    with pytest.raises(AssertionError):
        g.build(np.array([2], np.uint32), np.array([[0, 0, 1.0]], np.float32), np.ones(1, np.float32),
                np.ones(1, np.uint8), np.zeros(1, np.uint8), 16)
    with pytest.raises(AssertionError):  # tau has a bit beyond n
        g.build(np.array([0], np.uint32), np.array([[0, 0, 1.0]], np.float32), np.ones(1, np.float32),
                np.ones(1, np.uint8), np.full(1, 2, np.uint8), 16)


# --------------------------------------------------------------------------
# Discrete distributions P(n) and P(tau | n) (defensive one-sample MIS)
# --------------------------------------------------------------------------
def _point_workload(spq, k=1, tau=0, tau_random=False, xD=(0.35, 0.9, -1.5)):
    base = I.mirror_sphere(n=2, spq=1)
    wl = scenes.custom("vmf_point", base.surfaces, base.light, base.targets, np.array([xD]), (0, 0, 1),
                       base.light[1:4], k, tau, spq=spq, tau_random=tau_random)
    wl.rng_seed = 0xC0FFEE
    return wl


def test_lengths_follow_the_mixture_of_p0_and_guide_weights():
    # cell 0: weights 3 (n=1), 1 (n=3), 4 (n=3, another tau) -> W_1 = 3, W_3 = 5
    om = _dirs_on_circle([0.0, 0.2, 0.4]).astype(np.float32)
    g = O.VmfGuide(1).build(np.zeros(3, np.uint32), om, np.array([3.0, 1.0, 4.0], np.float32),
                            np.array([1, 3, 3], np.uint8), np.array([0, 2, 5], np.uint8), 16)
    p0w = np.array([5, 3, 0, 0, 0, 0, 0, 2], np.uint32)
    wl = _point_workload(200000)
    k, pn = O.sample_lengths(wl, g, p0w)
    P0 = p0w / p0w.sum()
    Pe = np.array([3, 0, 5, 0, 0, 0, 0, 0]) / 8.0
    P = 0.5 * P0 + 0.5 * Pe
    obs = np.bincount(k, minlength=9)[1:]
    m = P > 0
    assert obs[~m].sum() == 0
    assert stats.chisquare(obs[m], P[m] * k.size).pvalue > 1e-3
    assert np.allclose(pn, P[k - 1], rtol=1e-15)
    # no guide: P_0 alone
    k0, pn0 = O.sample_lengths(wl, None, p0w)
    obs0 = np.bincount(k0, minlength=9)[1:]
    m0 = P0 > 0
    assert stats.chisquare(obs0[m0], P0[m0] * k0.size).pvalue > 1e-3
    assert np.allclose(pn0, P0[k0 - 1], rtol=1e-15)


def test_types_follow_the_mixture_given_n():
    # n = 2: tau weights 1, 0, 2, 5 over two cells (only cell 0 is used)
    om = _dirs_on_circle([0.0, 0.1, 0.2, 0.3, 0.5], axis=(-0.2, -0.5, 0.84)).astype(np.float32)
    g = O.VmfGuide(2).build(np.array([0, 0, 0, 0, 1], np.uint32), om,
                            np.array([1.0, 2.0, 2.0, 3.0, 9.0], np.float32), np.full(5, 2, np.uint8),
                            np.array([0, 2, 3, 3, 1], np.uint8), 16)
    wl = _point_workload(100000, k=2, tau=0, tau_random=True)
    sc = O.Scene(wl)
    s = O.sample_seeds(wl, sc, g, threads=8)
    We = np.array([1.0, 0.0, 2.0, 5.0]) / 8.0
    P = 0.5 * 0.25 + 0.5 * We
    obs = np.bincount(s["tau"], minlength=4)
    assert stats.chisquare(obs, P * wl.B).pvalue > 1e-3


# --------------------------------------------------------------------------
# Seed density: E[1{valid} / p(w, tau | n)] = solid angle of the valid set
# --------------------------------------------------------------------------
@pytest.mark.parametrize("tau_random", [False, True])
def test_seed_density_integrates_over_the_visible_cone(tau_random):
    xD = np.array([0.35, 0.9, -1.5])
    d = np.linalg.norm(xD)
    axis = -xD / d
    # a spread of lobes around the sphere's direction, some beyond its rim
    rng = np.random.default_rng(3)
    v = axis + 0.35 * rng.normal(size=(40, 3))
    om = (v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32)
    g = O.VmfGuide(1).build(np.zeros(40, np.uint32), om, rng.uniform(0.1, 2.0, 40).astype(np.float32),
                            np.ones(40, np.uint8), np.zeros(40, np.uint8), 16)
    assert np.median(g.lobe[:40, 3]) > 20  # narrow lobes: the guided draws differ from p_0's
    wl = _point_workload(200000, k=1, tau=0, tau_random=tau_random)
    sc = O.Scene(wl)
    s = O.sample_seeds(wl, sc, g, threads=8)
    val = s["valid"] == 1
    # a k = 1 seed is valid exactly when its ray hits the unit sphere (the cone
    # lies above the receiver's horizon), whatever its type
    f = np.where(val, 1.0 / np.where(val, s["pdf"], 1.0), 0.0)
    omega = 2 * math.pi * (1 - math.sqrt(1 - 1 / d ** 2)) * (2 if tau_random else 1)
    assert abs(f.mean() - omega) < 4 * f.std() / math.sqrt(f.size)
    assert f.std() / math.sqrt(f.size) < 0.01 * omega


# --------------------------------------------------------------------------
# Estimator with sampled lengths and the vMF guide
# --------------------------------------------------------------------------
def test_estimator_unbiased_with_sampled_lengths_and_vmf_guide():
    wl = _point_workload(4096)
    sc, seeds, ch, con = None, None, None, None
    sc = O.Scene(wl)
    seeds = O.sample_seeds(wl, sc, threads=8)
    ch = O.walk(wl, sc, seeds, threads=8)
    con = O.contribution(wl, sc, ch, threads=8)
    adm = con["admissible"] == 1
    T = con["T"][adm][0]
    N, _ = O.bernoulli(wl, sc, ch, con["admissible"], threads=8)
    cell, om, w, kr, tr = O.records(wl, ch, con["T"], N, con["admissible"], with_types=True)
    g = O.VmfGuide(1).build(cell, om, w, kr, tr, 16)
    # guided pass: n in {1, 2} from the mixture (n = 2 has no solution on one
    # convex mirror), (w, tau) from the mixture given n
    p0w = np.array([1, 1, 0, 0, 0, 0, 0, 0], np.uint32)
    k, pn = O.sample_lengths(wl, g, p0w, rng_offset=1 << 30)
    assert math.isclose(pn[k == 1][0], 0.75) and math.isclose(pn[k == 2][0], 0.25)
    wg = dataclasses.replace(wl, k=k, pn=pn)
    s2 = O.sample_seeds(wg, sc, g, threads=8, rng_offset=1 << 30)
    c2 = O.walk(wg, sc, s2, threads=8)
    k2 = O.contribution(wg, sc, c2, threads=8)
    a2 = k2["admissible"] == 1
    assert np.all(k[a2] == 1)
    N2, capped = O.bernoulli(wg, sc, c2, k2["admissible"], g, threads=8, rng_offset=1 << 30)
    assert capped.sum() == 0
    # guided draws reach the solution far more often than p_0 alone
    assert a2[k == 1].mean() > adm.mean() + 0.1
    est = np.where(a2, k2["T"] * N2 / pn, 0.0)
    assert abs(est.mean() - T) < 4 * est.std() / math.sqrt(est.size)
