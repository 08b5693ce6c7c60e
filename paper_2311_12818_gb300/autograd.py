"""torch.autograd.Function over the hot path: receiver irradiance as a function
of the heights of a heightfield, with the hand-written adjoint kernel for the
backward pass (implicit function theorem; Bernoulli counts held fixed)."""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import mpg


class _Fn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, heights, runner):
        E = runner._forward(heights)
        fctx.runner = runner
        fctx.shape = heights.shape
        return E

    @staticmethod
    def backward(fctx, grad_E):
        r = fctx.runner
        g = torch.zeros(int(np.prod(fctx.shape)), dtype=torch.float32, device=grad_E.device)
        mpg.mpg_walk_adjoint(r.ctx, r.last_scene, r.last_chains, r.last_out.T, r.last_out.contrib,
                             grad_E.contiguous().float(), g)
        return g.view(fctx.shape), None


class HeightfieldIrradiance:
    """E = f(heights): seeds -> manifold walk -> contribution (with Bernoulli
    trials) on a workload whose scene has one heightfield; heights is a flat
    CUDA float32 tensor of the grid heights (row-major).

    The first call builds the scene (mesh and BVH on the host, from these
    heights); every later call replaces the heights on the device
    (mpg_scene_set_heights: positions, normals, triangles and a refit of the
    BVH boxes), so a gradient loop never copies the heights to the host.  The
    chain buffers are allocated once and reused; each call returns its own E."""

    def __init__(self, ctx, workload, params=None):
        self.ctx = ctx
        self.wl = workload
        uni = int(workload.k[0]) if (workload.k == workload.k[0]).all() else 0
        self.params = params or mpg.params_from(workload.params, walk_mode=mpg.WALK_BATCHED,
                                                tau_random=workload.tau_random, k_uniform=uni)
        self.last_scene = self.last_chains = self.last_out = None

    def _forward(self, heights):
        h = heights.detach().float().contiguous().view(-1)
        if self.last_scene is None:
            wl = dataclasses.replace(self.wl, hf_heights=h.cpu().numpy().astype(np.float64))
            self.last_scene = mpg.Scene(self.ctx, wl)
            self.last_chains = mpg.Chains(wl)
        else:
            self.last_scene.set_heights(h)
        self.last_out = mpg.run(self.ctx, self.last_scene, self.last_chains, self.wl, params=self.params)
        return self.last_out.E

    def __call__(self, heights):
        return _Fn.apply(heights, self)
