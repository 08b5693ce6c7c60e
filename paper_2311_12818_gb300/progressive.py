"""Progressive training and rendering (Sec. 5.8, online training and
rendering) on the CUDA path.

The sample schedule comes from mpg_training_plan: training iterations whose
seed counts per receiver point double, then the rendering stage.  Iteration i
samples from the guide built by iteration i - 1 (p_0 for the first), and its
own records build the next guide (histogram or vMF mixture over receiver
cells, or a vMF mixture over the leaves of a spatial tree of its samples);
only the rendering stage's contributions form the image.  Every stage is a
chain batch of its own (receiver points x its seeds per point, light-side
points from the workload generator), so with cell guides the whole schedule
is a fixed sequence of library calls that can be recorded once as a CUDA
graph and replayed."""
from __future__ import annotations

import dataclasses

import torch

from . import inputs as I
from . import mpg


class Progressive:
    """make_workload(spq, stage) -> inputs.Workload of the scene with `spq`
    seeds per receiver point (stage = 0, 1, ... numbers the batches; the last
    is the rendering stage)."""

    def __init__(self, ctx, make_workload, total_spp, first_spp=1, train_fraction=0.3, guide="histogram",
                 train_repeats=1, render_repeats=1, device="cuda", tree_method=None):
        """guide: 'histogram' or 'vmf' (one guide cell per receiver cell), or
        'vmf_tree' (the vMF mixture over the leaves of a spatial tree of each
        iteration's samples, Sec. 5.6; its build is synchronous -- the host
        decides the tree's nodes -- so that schedule is not recorded as a
        graph).  tree_method: mpg.STREE_LEVELS (level by level on the device,
        the default) or mpg.STREE_RECURSIVE (depth first on the host): the
        same tree."""
        self.tree_method = mpg.STREE_LEVELS if tree_method is None else tree_method
        if guide not in ("histogram", "vmf", "vmf_tree"):
            raise ValueError("guide must be 'histogram', 'vmf' or 'vmf_tree'")
        self.ctx, self.kind = ctx, guide
        self.plan, self.render_spp = mpg.mpg_training_plan(total_spp, first_spp, train_fraction)
        if self.render_spp < 1:
            raise ValueError("the plan leaves no rendering budget")
        spps = self.plan + [self.render_spp]
        self.workloads = [make_workload(s, i) for i, s in enumerate(spps)]
        wl0 = self.workloads[0]
        self.scene = mpg.Scene(ctx, wl0)
        self.chains = [mpg.Chains(wl, device=device) for wl in self.workloads]
        self.results = [mpg.Contribution.empty(wl.B, wl.Q, device=device) for wl in self.workloads]
        uniform = lambda wl: int(wl.k[0]) if (wl.k == wl.k[0]).all() else 0  # noqa: E731
        self.params = []
        for i, wl in enumerate(self.workloads):
            r = render_repeats if i == len(self.plan) else train_repeats
            p = dataclasses.replace(wl.params, bern_repeats=r)
            self.params.append(mpg.params_from(p, walk_mode=mpg.WALK_BATCHED, tau_random=wl.tau_random,
                                               k_uniform=uniform(wl)))
        cap = max(wl.B for wl in self.workloads[:-1]) if self.plan else 1
        if guide == "histogram":
            self.guides = [mpg.Guide(wl0.n_cells, I.guide_edges(), device=device) for _ in range(2)]
        elif guide == "vmf":
            self.guides = [mpg.VmfGuide(wl0.n_cells, cap, device=device) for _ in range(2)]
        else:
            self.guides = [None, None]  # sized per iteration by its tree
        self.trees = [None, None]
        self.records = [mpg.mpg_guide_records(ctx, self.scene, ch, res.contrib, with_chain=True)
                        for ch, res in zip(self.chains[:-1], self.results[:-1])]

    def guide_of(self, stage):
        """The guide stage `stage` samples from (None: p_0)."""
        return None if stage == 0 else self.guides[(stage - 1) % 2]

    def run(self, offset=0, stream=None):
        """All stages once; random numbers of stage i at offset + i * 2^36."""
        ctx, sc = self.ctx, self.scene
        n_train = len(self.plan)
        for i, (wl, ch, res, P) in enumerate(zip(self.workloads, self.chains, self.results, self.params)):
            g = self.guide_of(i)
            o = offset + (i << 36)
            if self.kind == "vmf_tree":  # each chain samples the leaf of its (x_D, x_L)
                ch.chain_cell = None if i == 0 else self.trees[(i - 1) % 2].query(ch, stream=stream)
            mpg.mpg_sample_seeds(ctx, sc, g, ch, P, wl.rng_seed, o, stream=stream)
            mpg.mpg_manifold_walk(ctx, sc, ch, P, stream=stream)
            mpg.mpg_chain_contribution(ctx, sc, g, ch, P, wl.rng_seed, o, out=res, stream=stream)
            if i == n_train:
                break
            # this iteration's records alone build the next guide
            rec = self.records[i]
            mpg.mpg_guide_records(ctx, sc, ch, res.contrib, out=rec, stream=stream)
            nxt = self.guides[i % 2]
            if self.kind == "histogram":
                mpg.mpg_guide_clear(ctx, nxt, stream=stream)
                mpg.mpg_guide_update(ctx, nxt, rec[0], rec[1], rec[2], R=wl.B, R_dev=rec[6],
                                     weight_shift=wl.params.weight_shift, stream=stream)
            elif self.kind == "vmf":
                mpg.mpg_vmf_build(ctx, nxt, rec[0], rec[1], rec[2], rec[3], rec[4], R=wl.B, R_dev=rec[6],
                                  weight_shift=wl.params.weight_shift, stream=stream)
            else:
                tree = mpg.STree(ctx, ch, rec[5], R=wl.B, R_dev=rec[6], method=self.tree_method, stream=stream)
                leaf_rec = tree.records(rec, wl.B, stream=stream)
                nxt = mpg.VmfGuide(tree.n_leaves, max(tree.n_members, 1))
                mpg.mpg_vmf_build(ctx, nxt, *leaf_rec[:5], R=leaf_rec[0].numel(), R_dev=leaf_rec[5],
                                  weight_shift=wl.params.weight_shift, stream=stream)
                self.trees[i % 2], self.guides[i % 2] = tree, nxt
        return self.results[-1]

    @property
    def image(self):
        """Irradiance per receiver point of the rendering stage."""
        return self.results[-1].E

    def capture(self, offset=0, advance=0):
        """The whole schedule as one graph (run() once first to size the buffers)."""
        if self.kind == "vmf_tree":
            raise ValueError("the tree build synchronises with the host: run the schedule uncaptured")
        g = mpg.Graph(self.ctx, rng_advance=advance)
        with g:
            self.run(offset, stream=g.stream)
        return g

    def total_chains(self):
        return sum(wl.B for wl in self.workloads)


def glass_sphere_stages(n=256, seed=0x4D50470002):
    """Stage workloads of the glass-sphere configuration: the same scene and
    receiver grid, light-side points drawn per stage from seed + stage."""
    return lambda spq, stage: I.glass_sphere(n=n, spq=spq, seed=seed + stage)
