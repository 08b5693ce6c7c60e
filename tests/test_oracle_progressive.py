"""Pins of the oracle's online training schedule (Sec. 5.8): each stage
samples from the guide built from the previous iteration's records alone, the
first from p_0, and the image is the rendering stage's irradiance only
(training samples are not splatted)."""
import numpy as np

from oracle import oracle as O
from paper_2311_12818_gb300 import inputs as I


def test_guides_from_the_last_iteration_and_image_from_rendering_only():
    make = lambda spq, stage: I.glass_sphere(n=8, spq=spq, seed=0x4D50470002 + stage)  # noqa: E731
    plan, render, stages, image = O.progressive(make, 16, guide="histogram", threads=4)
    assert (plan, render) == ([1, 3], 12) and len(stages) == 3
    assert stages[0]["guide"] is None
    for i in (1, 2):
        prev = stages[i - 1]
        cell, om, w = O.records(prev["wl"], prev["chains"], prev["contrib"]["T"], prev["N"],
                                prev["contrib"]["admissible"])
        ref = O.Guide(prev["wl"].n_cells, I.guide_edges())
        ref.update(cell, om, w, prev["wl"].params.weight_shift)
        assert np.array_equal(stages[i]["guide"].counts, ref.counts)
    last = stages[-1]
    assert np.array_equal(image, O.irradiance(last["wl"], last["contrib"]["T"], last["N"],
                                              last["contrib"]["admissible"]))
    assert last["wl"].spq == render and image.size == last["wl"].Q
