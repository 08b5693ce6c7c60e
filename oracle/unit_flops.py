"""Writes paper_2311_12818_gb300/unit_flops.json: flops of one execution of
each primitive of the manifold walk, counted by running the oracle's own
primitives in a counted scalar type (orc_unit_flops).  The benchmark multiplies
these by the kernels' work counters to get algorithmic flop counts."""
import ctypes
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
from oracle import oracle as O  # noqa: E402

NAMES = ["frame_sphere", "frame_plane", "frame_triangle", "normal_sphere", "normal_triangle", "vertex_blocks",
         "vertex_constraint", "thomas_first_row", "thomas_row", "ggt_row", "ggt_tail", "ray_sphere",
         "ray_rect", "ray_triangle", "ray_box", "kappa_vertex"]


def unit_flops():
    L = O.lib()
    out = np.zeros(16)
    L.orc_unit_flops.argtypes = [np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")]
    L.orc_unit_flops.restype = ctypes.c_int32
    assert L.orc_unit_flops(out) == 0
    return dict(zip(NAMES, out.tolist()))


if __name__ == "__main__":
    d = unit_flops()
    path = os.path.join(os.path.dirname(HERE), "paper_2311_12818_gb300", "unit_flops.json")
    with open(path, "w") as f:
        json.dump({"source": "oracle/unit_flops.py (orc_unit_flops, counted scalar type)", "flops": d}, f, indent=1)
    print(json.dumps(d, indent=1))
