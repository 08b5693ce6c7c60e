"""Pin of the repeated reciprocal-probability estimate (the paper's R x 4 /
TR x 4 variants, Sec. 6.5): r independent Bernoulli estimates per chain are
averaged, so on a single-solution configuration N / r keeps the mean 1/P of
the geometric trial count and its variance falls to (1 - P) / (r P^2)."""
import dataclasses
import math

import numpy as np

import scenes
from oracle import oracle as O
from paper_2311_12818_gb300 import inputs as I


def _point(spq, repeats):
    base = I.mirror_sphere(n=2, spq=1)
    wl = scenes.custom("mirror_sphere_point", base.surfaces, base.light, base.targets,
                       np.array([[0.35, 0.9, -1.5]]), (0, 0, 1), base.light[1:4], 1, 0, spq=spq)
    wl.rng_seed = 0xBEEF
    return dataclasses.replace(wl, params=dataclasses.replace(wl.params, bern_repeats=repeats))


def test_repeated_estimates_keep_the_mean_and_divide_the_variance():
    M = 4096
    w1, w4 = _point(M, 1), _point(M, 4)
    sc = O.Scene(w1)
    seeds = O.sample_seeds(w1, sc, threads=8)
    ch = O.walk(w1, sc, seeds, threads=8)
    con = O.contribution(w1, sc, ch, threads=8)
    adm = con["admissible"] == 1
    P = adm.mean()  # probability that one draw reaches the single solution
    assert 0.2 < P < 0.95
    N1, c1 = O.bernoulli(w1, sc, ch, con["admissible"], threads=8)
    N4, c4 = O.bernoulli(w4, sc, ch, con["admissible"], threads=8)
    assert c1.sum() == 0 and c4.sum() == 0
    a1 = N1[adm].astype(np.float64)
    a4 = N4[adm].astype(np.float64) / 4.0
    # every repeat takes at least one trial; the first repeat is the single estimate
    assert np.all(N4[adm] >= N1[adm] + 3)
    n = a4.size
    var1 = (1 - P) / P ** 2
    assert abs(a4.mean() - 1 / P) < 4 * math.sqrt(var1 / 4 / n) + 4 * (1 / P ** 2) * math.sqrt(P * (1 - P) / M)
    ratio = a4.var() / a1.var()
    assert 0.17 < ratio < 0.36, ratio
    # the irradiance estimate stays unbiased: mean of 1{adm} T N / r = T
    T = con["T"][adm][0]
    E4 = O.irradiance(w4, con["T"], N4, con["admissible"])[0]
    est = np.where(adm, con["T"] * N4 / 4.0, 0.0)
    assert math.isclose(E4, est.mean(), rel_tol=1e-12)
    assert abs(est.mean() - T) < 4 * est.std() / math.sqrt(M)
