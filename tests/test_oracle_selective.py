"""Pin of selective activation (Sec. 5.8): with a guide, receiver points whose
cell holds no samples draw no seed; every other seed is the one drawn without
it (the switch only removes chains)."""
import dataclasses

import numpy as np

from oracle import oracle as O
from paper_2311_12818_gb300 import inputs as I


def _guides(wl):
    sc = O.Scene(wl)
    seeds = O.sample_seeds(wl, sc)
    ch = O.walk(wl, sc, seeds)
    con = O.contribution(wl, sc, ch)
    N, _ = O.bernoulli(wl, sc, ch, con["admissible"])
    cell, om, w, k, tau = O.records(wl, ch, con["T"], N, con["admissible"], with_types=True)
    # keep the records of half of the cells that have any, so that some cells
    # with caustic chains are empty too
    keep = (cell % 2) == 0
    hist = O.Guide(wl.n_cells, I.guide_edges())
    hist.update(cell[keep], om[keep], w[keep], wl.params.weight_shift)
    vmf = O.VmfGuide(wl.n_cells).build(cell[keep], om[keep], w[keep], k[keep], tau[keep], wl.params.weight_shift)
    return sc, hist, vmf, np.unique(cell[keep])


def test_selective_activation_drops_only_empty_cells():
    wl = I.glass_sphere(n=32, spq=4)
    sc, hist, vmf, full = _guides(wl)
    on = dataclasses.replace(wl, params=dataclasses.replace(wl.params, selective=1))
    cell_of_chain = np.repeat(wl.cell, wl.spq)
    # a cell is empty for the histogram guide when it holds no quantised
    # weight, for the vMF guide when it holds no lobe
    with_weight = np.nonzero(hist.counts.sum(axis=1) > 0)[0]
    with_lobes = np.nonzero(np.diff(vmf.cell_start) > 0)[0]
    assert set(with_weight) <= set(with_lobes) == set(full)
    for g, cells in ((hist, with_weight), (vmf, with_lobes)):
        active = np.isin(cell_of_chain, cells)
        assert 0.2 < active.mean() < 0.8
        a = O.sample_seeds(wl, sc, g, rng_offset=99)
        b = O.sample_seeds(on, sc, g, rng_offset=99)
        assert not b["valid"][~active].any()
        assert np.array_equal(a["valid"][active], b["valid"][active])
        va = active & (a["valid"] == 1)
        assert np.array_equal(a["x"][va], b["x"][va]) and np.array_equal(a["pdf"][va], b["pdf"][va])
