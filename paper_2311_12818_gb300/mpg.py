"""Thin Python binding of libmpg.so (the C ABI declared in include/mpg.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  PyTorch provides device memory (tensors passed by pointer) and
streams.  The binding refuses to run without the compiled library -- there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import gc
import dataclasses
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmpg.so")

MAXK = 8
MPG_OK = 0
MPG_ERR_INVALID_ARG, MPG_ERR_CUDA, MPG_ERR_OOM, MPG_ERR_LIMIT, MPG_ERR_UNSUPPORTED = -1, -2, -3, -4, -5
CHAIN_INVALID, CHAIN_CONVERGED, CHAIN_FAILED, CHAIN_LIMIT, CHAIN_SEEDED = 0, 1, 2, 3, 255
WALK_PLAIN, WALK_BATCHED = 0, 1


class MpgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("mpg error %d: %s" % (code, msg))
        self.code = code


class mpg_params(C.Structure):
    _fields_ = [("tol", C.c_float), ("max_iter", C.c_int32), ("max_halvings", C.c_int32),
                ("ray_eps", C.c_float), ("sing_eps", C.c_float), ("dedup_eps", C.c_float),
                ("max_trials", C.c_int32), ("weight_shift", C.c_int32), ("alpha", C.c_float),
                ("walk_mode", C.c_int32), ("block_threads", C.c_int32), ("tau_random", C.c_int32),
                ("k_uniform", C.c_int32), ("stall_tol", C.c_float), ("fp64_tol", C.c_float),
                ("fp64_k", C.c_int32), ("ctas_per_sm", C.c_int32), ("refill_every", C.c_int32),
                ("trial_sync_rounds", C.c_int32), ("trial_batch", C.c_int32), ("walk_group", C.c_int32),
                ("bern_repeats", C.c_int32), ("selective", C.c_int32), ("roughness", C.c_float)]

SCHEDULE_FIELDS = ["block_threads", "ctas_per_sm", "refill_every", "trial_sync_rounds", "trial_batch", "fp64_k",
                   "walk_group"]


class mpg_chains(C.Structure):
    _fields_ = [("B", C.c_int32), ("Q", C.c_int32), ("spq", C.c_int32),
                ("xD", C.c_void_p), ("nD", C.c_void_p), ("cell", C.c_void_p), ("xL", C.c_void_p),
                ("k", C.c_void_p), ("pn", C.c_void_p), ("tau", C.c_void_p), ("x", C.c_void_p),
                ("surf", C.c_void_p), ("prim", C.c_void_p), ("bary", C.c_void_p), ("pdf", C.c_void_p),
                ("status", C.c_void_p), ("iters", C.c_void_p), ("chain_cell", C.c_void_p), ("offset", C.c_void_p)]


class mpg_guide(C.Structure):
    _fields_ = [("n_cells", C.c_int32), ("n_theta", C.c_int32), ("n_phi", C.c_int32),
                ("counts", C.c_void_p), ("cdf", C.c_void_p), ("cos_theta", C.c_void_p),
                ("phi_cos", C.c_void_p), ("phi_sin", C.c_void_p), ("kind", C.c_int32), ("capacity", C.c_int32),
                ("cell_start", C.c_void_p), ("lobe_key", C.c_void_p), ("lobe", C.c_void_p),
                ("lobe_prefix", C.c_void_p), ("lobe_coef", C.c_void_p), ("scratch", C.c_void_p)]


GUIDE_HISTOGRAM, GUIDE_VMF = 0, 1
STREE_RECURSIVE, STREE_LEVELS = 0, 1


STAT_FIELDS = ["newton_steps", "thomas_rows", "full_evals", "c_evals", "ray_casts", "sphere_tests",
               "plane_tests", "node_tests", "tri_tests", "walks", "converged", "ggt_rows", "trials", "seeds",
               "ggt_fp64", "uncounted"]
KERNEL_SEED, KERNEL_WALK, KERNEL_CONTRIB, KERNEL_BERNOULLI, KERNEL_TRACE, KERNEL_AUX = range(6)
KERNEL_NAMES = ["seed", "walk", "contrib", "bernoulli", "trace", "aux"]


class mpg_stats(C.Structure):
    _fields_ = [(f, C.c_uint64) for f in STAT_FIELDS]


EXPORTS = ["mpg_last_error", "mpg_version", "mpg_ctx_create", "mpg_ctx_destroy", "mpg_ctx_sync",
           "mpg_ctx_stats", "mpg_ctx_set_stats", "mpg_ctx_set_profile", "mpg_ctx_profile", "mpg_ctx_launches", "mpg_scene_create", "mpg_scene_destroy", "mpg_scene_info", "mpg_scene_set_heights",
           "mpg_sample_seeds", "mpg_manifold_walk", "mpg_chain_contribution", "mpg_guide_update",
           "mpg_guide_records", "mpg_walk_adjoint", "mpg_trace_rays", "mpg_fp32_peak",
           "mpg_manifold_walk_noalloc", "mpg_fp64_peak", "mpg_guide_clear", "mpg_graph_begin", "mpg_graph_join", "mpg_graph_end",
           "mpg_graph_launch", "mpg_graph_kernels", "mpg_graph_destroy", "mpg_autotune", "mpg_vmf_build",
           "mpg_sample_lengths", "mpg_training_plan", "mpg_stree_build", "mpg_stree_build_host", "mpg_stree_info", "mpg_stree_export",
           "mpg_stree_records", "mpg_stree_query", "mpg_stree_destroy", "mpg_separator_bsdf", "mpg_records_bsdf",
           "mpg_sample_offsets"]

_lib = None


def lib():
    """Load libmpg.so (raises if it was not built -- no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libmpg.so is missing: build it with paper_2311_12818_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, i32, u64, f32 = C.c_void_p, C.c_int32, C.c_uint64, C.c_float
        L.mpg_last_error.restype = C.c_char_p
        L.mpg_version.restype = i32
        L.mpg_ctx_create.argtypes = [i32, C.POINTER(vp)]
        L.mpg_ctx_destroy.argtypes = [vp]
        L.mpg_ctx_destroy.restype = None
        L.mpg_ctx_sync.argtypes = [vp, vp]
        L.mpg_ctx_stats.argtypes = [vp, i32, C.POINTER(mpg_stats), i32, vp]
        L.mpg_ctx_set_stats.argtypes = [vp, i32]
        L.mpg_ctx_set_profile.argtypes = [vp, i32]
        L.mpg_ctx_profile.argtypes = [vp, i32, C.POINTER(C.c_double), C.POINTER(C.c_int64), i32]
        L.mpg_ctx_launches.argtypes = [vp, C.POINTER(C.c_int64)]
        L.mpg_scene_create.argtypes = [vp, vp, i32, vp, vp, i32, vp, i32, vp, C.POINTER(vp)]
        L.mpg_scene_destroy.argtypes = [vp]
        L.mpg_scene_destroy.restype = None
        L.mpg_graph_destroy.restype = None
        L.mpg_scene_info.argtypes = [vp, i32, C.POINTER(i32), C.POINTER(i32)]
        L.mpg_scene_set_heights.argtypes = [vp, vp, i32, vp, vp]
        L.mpg_sample_seeds.argtypes = [vp, vp, C.POINTER(mpg_guide), C.POINTER(mpg_chains), u64, u64,
                                       C.POINTER(mpg_params), vp]
        L.mpg_manifold_walk.argtypes = [vp, vp, C.POINTER(mpg_chains), C.POINTER(mpg_params), vp]
        L.mpg_sample_offsets.argtypes = [vp, C.POINTER(mpg_chains), f32, u64, u64, vp, vp]
        L.mpg_manifold_walk_noalloc.argtypes = [vp, C.POINTER(mpg_chains), C.POINTER(mpg_params), vp]
        L.mpg_chain_contribution.argtypes = [vp, vp, C.POINTER(mpg_guide), C.POINTER(mpg_chains), u64, u64,
                                             C.POINTER(mpg_params), vp, vp, vp, vp, vp, vp, vp, vp]
        L.mpg_guide_update.argtypes = [vp, C.POINTER(mpg_guide), vp, vp, vp, i32, vp, i32, vp]
        L.mpg_guide_records.argtypes = [vp, vp, C.POINTER(mpg_chains), vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.mpg_vmf_build.argtypes = [vp, C.POINTER(mpg_guide), vp, vp, vp, vp, vp, i32, vp, i32, vp]
        L.mpg_training_plan.argtypes = [i32, i32, f32, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
        L.mpg_stree_build.argtypes = [vp, C.POINTER(mpg_chains), vp, i32, vp, f32, f32, i32, C.POINTER(vp), vp]
        L.mpg_stree_build_host.argtypes = [vp, i32, f32, f32, i32, C.POINTER(vp)]
        L.mpg_stree_info.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
        L.mpg_stree_export.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.mpg_stree_records.argtypes = [vp, vp, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp, i32, vp, vp]
        L.mpg_stree_query.argtypes = [vp, vp, C.POINTER(mpg_chains), vp, vp]
        L.mpg_stree_destroy.argtypes = [vp]
        L.mpg_separator_bsdf.argtypes = [vp, C.POINTER(mpg_chains), vp, C.POINTER(f32), f32, vp, vp, vp]
        L.mpg_records_bsdf.argtypes = [vp, C.POINTER(mpg_chains), vp, vp, vp, i32, vp, C.POINTER(f32), f32, vp]
        L.mpg_stree_destroy.restype = None
        L.mpg_sample_lengths.argtypes = [vp, C.POINTER(mpg_guide), C.POINTER(mpg_chains), vp, u64, u64,
                                         C.POINTER(mpg_params), vp, vp, vp]
        L.mpg_walk_adjoint.argtypes = [vp, vp, C.POINTER(mpg_chains), vp, vp, vp, vp, vp]
        L.mpg_trace_rays.argtypes = [vp, vp, vp, vp, i32, f32, f32, vp, vp, vp, vp, vp]
        L.mpg_fp32_peak.argtypes = [vp, C.POINTER(C.c_double), vp]
        L.mpg_fp64_peak.argtypes = [vp, C.POINTER(C.c_double), vp]
        L.mpg_guide_clear.argtypes = [vp, C.POINTER(mpg_guide), vp]
        L.mpg_graph_begin.argtypes = [vp, vp, u64]
        L.mpg_graph_end.argtypes = [vp, vp, C.POINTER(vp)]
        L.mpg_graph_join.argtypes = [vp, vp]
        L.mpg_graph_launch.argtypes = [vp, vp]
        L.mpg_graph_kernels.argtypes = [vp, C.POINTER(C.c_int64)]
        L.mpg_graph_destroy.argtypes = [vp]
        L.mpg_autotune.argtypes = [vp, vp, C.POINTER(mpg_guide), C.POINTER(mpg_chains), u64, u64,
                                   C.POINTER(mpg_params), i32, C.POINTER(mpg_params), C.POINTER(C.c_double), vp]
        for n in EXPORTS[2:]:
            if n not in ("mpg_ctx_destroy", "mpg_scene_destroy", "mpg_graph_destroy", "mpg_stree_destroy"):
                getattr(L, n).restype = i32
        _lib = L
    return _lib


def _check(code):
    if code != MPG_OK:
        raise MpgError(code, lib().mpg_last_error().decode())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def params_from(p, walk_mode=WALK_BATCHED, block_threads=0, tau_random=False, k_uniform=0, **schedule) -> mpg_params:
    """mpg_params from an inputs.Params (FP32 copy of the solver constants);
    `schedule` sets fields of SCHEDULE_FIELDS (0 = the library's default)."""
    P = mpg_params(p.tol, p.max_iter, p.max_halvings, p.ray_eps, p.sing_eps, p.dedup_eps, p.max_trials,
                   p.weight_shift, p.alpha, walk_mode, block_threads, int(bool(tau_random)), k_uniform,
                   p.stall_tol, p.fp64_tol)
    P.bern_repeats = int(getattr(p, "bern_repeats", 1))
    P.selective = int(getattr(p, "selective", 0))
    P.roughness = float(getattr(p, "roughness", 0.0))
    for f, v in schedule.items():
        if f not in SCHEDULE_FIELDS:
            raise TypeError("unknown schedule field %r" % f)
        setattr(P, f, int(v))
    return P


class Context:
    def __init__(self, device=0):
        self.device = device
        h = C.c_void_p()
        torch.cuda.set_device(device)
        _check(lib().mpg_ctx_create(device, C.byref(h)))
        self.h = h

    def sync(self, stream=None):
        _check(lib().mpg_ctx_sync(self.h, _stream(stream)))

    def stats(self, kind=-1, reset=False, stream=None):
        s = mpg_stats()
        _check(lib().mpg_ctx_stats(self.h, kind, C.byref(s), int(reset), _stream(stream)))
        return {f: int(getattr(s, f)) for f in STAT_FIELDS}

    def reset_stats(self, stream=None):
        _check(lib().mpg_ctx_stats(self.h, -1, None, 1, _stream(stream)))

    def set_profile(self, on):
        _check(lib().mpg_ctx_set_profile(self.h, int(bool(on))))

    def profile(self, kind=-1, reset=False):
        """(milliseconds, launches) of a kernel family since the last reset."""
        ms, n = C.c_double(), C.c_int64()
        _check(lib().mpg_ctx_profile(self.h, kind, C.byref(ms), C.byref(n), int(reset)))
        return ms.value, n.value

    def launches(self):
        n = C.c_int64()
        _check(lib().mpg_ctx_launches(self.h, C.byref(n)))
        return n.value

    def set_stats(self, on):
        _check(lib().mpg_ctx_set_stats(self.h, int(bool(on))))

    def fp32_peak(self, stream=None):
        v = C.c_double()
        _check(lib().mpg_fp32_peak(self.h, C.byref(v), _stream(stream)))
        return v.value

    def fp64_peak(self, stream=None):
        v = C.c_double()
        _check(lib().mpg_fp64_peak(self.h, C.byref(v), _stream(stream)))
        return v.value

    def __del__(self):
        if getattr(self, "h", None):
            lib().mpg_ctx_destroy(self.h)
            self.h = None


class Scene:
    def __init__(self, ctx: Context, wl):
        self.ctx = ctx
        keep = [np.ascontiguousarray(a, np.float64) for a in
                (wl.surfaces, wl.hf_desc.reshape(-1, 6), wl.hf_heights, wl.targets, wl.light)]
        s, hd, hh, tg, li = keep
        h = C.c_void_p()
        _check(lib().mpg_scene_create(ctx.h, s.ctypes.data, s.shape[0], hd.ctypes.data if hd.size else None,
                                      hh.ctypes.data if hh.size else None, hd.shape[0],
                                      tg.ctypes.data if tg.size else None, tg.shape[0], li.ctypes.data,
                                      C.byref(h)))
        self.h = h
        self.light_area = wl.light_area

    def info(self, h=0):
        n, t = C.c_int32(), C.c_int32()
        _check(lib().mpg_scene_info(self.h, h, C.byref(n), C.byref(t)))
        return n.value, t.value

    def set_heights(self, heights, h=0, stream=None):
        """mpg_scene_set_heights: heightfield h takes the heights of a CUDA
        float32 tensor (nx * ny, row-major), on the device."""
        if not (heights.is_cuda and heights.dtype == torch.float32 and heights.is_contiguous()):
            raise TypeError("heights must be a contiguous CUDA float32 tensor")
        _check(lib().mpg_scene_set_heights(self.ctx.h, self.h, h, _ptr(heights), _stream(stream)))

    def __del__(self):
        if getattr(self, "h", None):
            lib().mpg_scene_destroy(self.h)
            self.h = None


class Guide:
    """Guide histograms in device memory (counts and prefix sums uint64)."""

    def __init__(self, n_cells, edges, device="cuda"):
        ct, pc, ps = (torch.as_tensor(np.ascontiguousarray(e, np.float32), device=device) for e in edges)
        self.cos_theta, self.phi_cos, self.phi_sin = ct, pc, ps
        self.n_cells, self.n_theta, self.n_phi = n_cells, ct.numel() - 1, pc.numel() - 1
        bins = self.n_theta * self.n_phi
        self.counts = torch.zeros((n_cells, bins), dtype=torch.int64, device=device)
        self.cdf = torch.zeros((n_cells, bins), dtype=torch.int64, device=device)

    def struct(self):
        return mpg_guide(self.n_cells, self.n_theta, self.n_phi, self.counts.data_ptr(), self.cdf.data_ptr(),
                         self.cos_theta.data_ptr(), self.phi_cos.data_ptr(), self.phi_sin.data_ptr(),
                         GUIDE_HISTOGRAM, 0, None, None, None, None, None, None)

    def clear(self, ctx, stream=None):
        mpg_guide_clear(ctx, self, stream)


class VmfGuide:
    """vMF mixture guide (Sec. 5.5) in device memory: up to `capacity` lobes,
    cell_start [n_cells+1], lobe_key [capacity] ((n << 8) | tau), lobe
    [capacity, 4] (mu, kappa), lobe_prefix [capacity] (cell-local prefix sums
    of the quantised weights), lobe_coef [capacity] (density factors), and the
    build scratch; filled by mpg_vmf_build."""

    def __init__(self, n_cells, capacity, device="cuda"):
        self.n_cells, self.capacity = n_cells, capacity
        cap = max(capacity, 1)
        self.cell_start = torch.zeros(n_cells + 1, dtype=torch.int32, device=device)
        self.lobe_key = torch.zeros(cap, dtype=torch.int32, device=device)
        self.lobe = torch.zeros((cap, 4), dtype=torch.float32, device=device)
        self.lobe_prefix = torch.zeros(cap, dtype=torch.int64, device=device)
        self.lobe_coef = torch.zeros(cap, dtype=torch.float32, device=device)
        words = 4 * cap + 256 * ((cap + 1023) // 1024) + 64
        self.scratch = torch.zeros(words, dtype=torch.int32, device=device)

    def struct(self):
        return mpg_guide(self.n_cells, 0, 0, None, None, None, None, None, GUIDE_VMF, self.capacity,
                         self.cell_start.data_ptr(), self.lobe_key.data_ptr(), self.lobe.data_ptr(),
                         self.lobe_prefix.data_ptr(), self.lobe_coef.data_ptr(), self.scratch.data_ptr())

    @property
    def n_lobes(self):
        return int(self.cell_start[-1].item())


class Chains:
    """Device SoA state of a chain batch built from a workload (inputs module)."""

    def __init__(self, wl, device="cuda"):
        f32 = dict(dtype=torch.float32, device=device)
        self.B, self.Q, self.spq = wl.B, wl.Q, wl.spq
        self.xD = torch.as_tensor(np.ascontiguousarray(wl.xD.T, np.float32), device=device)
        self.nD = torch.as_tensor(np.ascontiguousarray(wl.nD.T, np.float32), device=device)
        self.cell = torch.as_tensor(wl.cell.astype(np.int32), device=device)
        self.xL = torch.as_tensor(np.ascontiguousarray(wl.xL.T, np.float32), device=device)
        self.k = torch.as_tensor(wl.k.astype(np.uint8), device=device)
        self.pn = torch.as_tensor(wl.pn.astype(np.float32), device=device)
        self.tau = torch.as_tensor(wl.tau.astype(np.uint8), device=device)
        B = self.B
        self.x = torch.zeros((MAXK, 3, B), **f32)
        self.surf = torch.full((MAXK, B), -1, dtype=torch.int32, device=device)
        self.prim = torch.full((MAXK, B), -1, dtype=torch.int32, device=device)
        self.bary = torch.zeros((MAXK, 2, B), **f32)
        self.pdf = torch.zeros(B, **f32)
        self.status = torch.zeros(B, dtype=torch.uint8, device=device)
        self.iters = torch.zeros(B, dtype=torch.uint8, device=device)
        self.chain_cell = None  # [B] int32 per-chain guide cells (a tree's leaves), or None
        self.offset = None  # [8, 2, B] float32 offset normals of glossy chains, or None (specular)

    def struct(self):
        return mpg_chains(self.B, self.Q, self.spq, self.xD.data_ptr(), self.nD.data_ptr(), self.cell.data_ptr(),
                          self.xL.data_ptr(), self.k.data_ptr(), self.pn.data_ptr(), self.tau.data_ptr(),
                          self.x.data_ptr(), self.surf.data_ptr(), self.prim.data_ptr(), self.bary.data_ptr(),
                          self.pdf.data_ptr(), self.status.data_ptr(), self.iters.data_ptr(),
                          None if self.chain_cell is None else self.chain_cell.data_ptr(),
                          None if self.offset is None else self.offset.data_ptr())

    def aos(self):
        """Host copy in the oracle's array-of-structures layout (tests)."""
        x = self.x.permute(2, 0, 1).double().cpu().numpy()
        return dict(x=np.ascontiguousarray(x), surf=self.surf.T.contiguous().cpu().numpy(),
                    prim=self.prim.T.contiguous().cpu().numpy(),
                    bary=np.ascontiguousarray(self.bary.permute(2, 0, 1).double().cpu().numpy()),
                    tau=self.tau.cpu().numpy(), status=self.status.cpu().numpy(),
                    iters=self.iters.cpu().numpy(), pdf=self.pdf.double().cpu().numpy())


@dataclasses.dataclass
class Contribution:
    G: torch.Tensor
    kappa: torch.Tensor
    T: torch.Tensor
    trials: torch.Tensor
    capped: torch.Tensor
    contrib: torch.Tensor
    E: torch.Tensor

    @classmethod
    def empty(cls, B, Q, device="cuda"):
        f = dict(dtype=torch.float32, device=device)
        return cls(torch.zeros(B, **f), torch.zeros(B, **f), torch.zeros(B, **f),
                   torch.zeros(B, dtype=torch.int32, device=device), torch.zeros(B, dtype=torch.uint8, device=device),
                   torch.zeros(B, **f), torch.zeros(Q, **f))


# ---------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# ---------------------------------------------------------------------------
def mpg_sample_seeds(ctx, scene, guide, chains, params, rng_seed, rng_offset=0, stream=None):
    cs = chains.struct()
    gs = guide.struct() if guide is not None else None
    _check(lib().mpg_sample_seeds(ctx.h, scene.h, C.byref(gs) if gs is not None else None, C.byref(cs),
                                  rng_seed, rng_offset, C.byref(params), _stream(stream)))


def mpg_guide_clear(ctx, guide, stream=None):
    gs = guide.struct()
    _check(lib().mpg_guide_clear(ctx.h, C.byref(gs), _stream(stream)))


def mpg_autotune(ctx, scene, guide, chains, params, rng_seed, rng_offset=0, repeats=2, stream=None):
    """Fastest batched schedule for this batch: (tuned mpg_params, ms per step)."""
    cs = chains.struct()
    gs = guide.struct() if guide is not None else None
    out, ms = mpg_params(), C.c_double()
    _check(lib().mpg_autotune(ctx.h, scene.h, C.byref(gs) if gs is not None else None, C.byref(cs), rng_seed,
                              rng_offset, C.byref(params), repeats, C.byref(out), C.byref(ms), _stream(stream)))
    return out, ms.value


class Graph:
    """Library calls recorded once on a side stream and replayed with one graph
    launch (mpg_graph_*).  Use as a context manager around the calls; they are
    recorded, not run.  Replay r draws its random numbers at rng_offset +
    r * rng_advance."""

    def __init__(self, ctx, rng_advance=0, join=()):
        self.ctx, self.rng_advance, self.h, self.join = ctx, int(rng_advance), None, list(join)
        self.stream = torch.cuda.Stream(device=ctx.device)

    def __enter__(self):
        # Objects whose destructors free device memory (contexts, scenes,
        # graphs) must not be collected while the capture is open: cudaFree
        # is not allowed then and would invalidate the capture.
        gc.collect()
        self._gc_was_enabled = gc.isenabled()
        gc.disable()
        self._outer = torch.cuda.current_stream()
        self.stream.wait_stream(self._outer)
        self._ctx_mgr = torch.cuda.stream(self.stream)
        self._ctx_mgr.__enter__()
        _check(lib().mpg_graph_begin(self.ctx.h, _stream(self.stream), self.rng_advance))
        for other in self.join:
            code = lib().mpg_graph_join(self.ctx.h, other.h)
            if code != MPG_OK:
                h = C.c_void_p()
                lib().mpg_graph_end(self.ctx.h, _stream(self.stream), C.byref(h))
                if h:
                    lib().mpg_graph_destroy(h)
                self._ctx_mgr.__exit__(None, None, None)
                if self._gc_was_enabled:
                    gc.enable()
                _check(code)
        return self

    def __exit__(self, et, ev, tb):
        h = C.c_void_p()
        code = lib().mpg_graph_end(self.ctx.h, _stream(self.stream), C.byref(h))
        if self._gc_was_enabled:
            gc.enable()
        self._ctx_mgr.__exit__(et, ev, tb)
        self._outer.wait_stream(self.stream)
        if et is None:
            _check(code)
            self.h = h
        elif code == MPG_OK and h:
            lib().mpg_graph_destroy(h)  # a recorded call failed: the graph is incomplete
        return False

    def launch(self, stream=None):
        _check(lib().mpg_graph_launch(self.h, _stream(stream)))

    def kernels(self):
        n = C.c_int64()
        _check(lib().mpg_graph_kernels(self.h, C.byref(n)))
        return n.value

    def __del__(self):
        if getattr(self, "h", None):
            lib().mpg_graph_destroy(self.h)
            self.h = None


def mpg_sample_offsets(ctx, chains, alpha, rng_seed, rng_offset=0, out=None, stream=None):
    """Offset normals of glossy chains (Sec. 5.7) into out ([8, 2, B] float32,
    allocated when None); returns it (set it as chains.offset to walk them)."""
    if out is None:
        out = torch.zeros((MAXK, 2, chains.B), dtype=torch.float32, device=chains.k.device)
    cs = chains.struct()
    _check(lib().mpg_sample_offsets(ctx.h, C.byref(cs), float(alpha), rng_seed, rng_offset, _ptr(out),
                                    _stream(stream)))
    return out


def mpg_manifold_walk(ctx, scene, chains, params, stream=None):
    cs = chains.struct()
    _check(lib().mpg_manifold_walk(ctx.h, scene.h, C.byref(cs), C.byref(params), _stream(stream)))


def mpg_manifold_walk_noalloc(scene, chains, params, stream=None):
    """Batched manifold walk that allocates no device memory (fixed library
    scratch, at most 1,048,576 chains per call; overlapping calls race)."""
    cs = chains.struct()
    _check(lib().mpg_manifold_walk_noalloc(scene.h, C.byref(cs), C.byref(params), _stream(stream)))


def mpg_chain_contribution(ctx, scene, guide, chains, params, rng_seed, rng_offset=0, out=None, stream=None):
    out = out if out is not None else Contribution.empty(chains.B, chains.Q)
    cs = chains.struct()
    gs = guide.struct() if guide is not None else None
    _check(lib().mpg_chain_contribution(ctx.h, scene.h, C.byref(gs) if gs is not None else None, C.byref(cs),
                                        rng_seed, rng_offset, C.byref(params), _ptr(out.G), _ptr(out.kappa),
                                        _ptr(out.T), _ptr(out.trials), _ptr(out.capped), _ptr(out.contrib),
                                        _ptr(out.E), _stream(stream)))
    return out


def mpg_guide_update(ctx, guide, cell, omega, w, R=None, R_dev=None, weight_shift=16, stream=None):
    """cell [R] int32, omega [3, R] float32, w [R] float32 (device tensors)."""
    R = int(cell.numel()) if R is None else R
    gs = guide.struct()
    _check(lib().mpg_guide_update(ctx.h, C.byref(gs), _ptr(cell), _ptr(omega), _ptr(w), R, _ptr(R_dev),
                                  weight_shift, _stream(stream)))


def mpg_guide_records(ctx, scene, chains, contrib, out=None, with_types=False, with_chain=False, stream=None):
    """Records of chains with contrib > 0, in chain order: (cell [B] int32,
    omega [3, B], w [B], count [4] int32 (entry 0)); with_types (or a
    six-tensor `out`): (cell, omega, w, k [B] uint8, tau [B] uint8, count);
    with_chain (or seven tensors): (cell, omega, w, k, tau, chain [B] int32, count)."""
    B = chains.B
    if out is None:
        out = [torch.zeros(B, dtype=torch.int32, device="cuda"), torch.zeros((3, B), dtype=torch.float32, device="cuda"),
               torch.zeros(B, dtype=torch.float32, device="cuda")]
        if with_types or with_chain:
            out += [torch.zeros(B, dtype=torch.uint8, device="cuda"), torch.zeros(B, dtype=torch.uint8, device="cuda")]
        if with_chain:
            out += [torch.zeros(B, dtype=torch.int32, device="cuda")]
        out = tuple(out + [torch.zeros(4, dtype=torch.int32, device="cuda")])
    chain = None
    if len(out) == 7:
        cell, om, w, k, tau, chain, R = out
    elif len(out) == 6:
        cell, om, w, k, tau, R = out
    else:
        (cell, om, w, R), k, tau = out, None, None
    cs = chains.struct()
    _check(lib().mpg_guide_records(ctx.h, scene.h, C.byref(cs), _ptr(contrib), _ptr(cell), _ptr(om), _ptr(w),
                                   _ptr(k), _ptr(tau), _ptr(chain), _ptr(R), _stream(stream)))
    return out


def mpg_separator_bsdf(ctx, chains, contrib, camera, exponent, out=None, stream=None):
    """Radiance toward the camera through the glossy separator (Sec. 5.7):
    (per-chain weighted contributions [B], per-point radiance [Q])."""
    rad, L = out if out is not None else (torch.zeros(chains.B, dtype=torch.float32, device="cuda"),
                                          torch.zeros(chains.Q, dtype=torch.float32, device="cuda"))
    cam = (C.c_float * 3)(*[float(v) for v in camera])
    cs = chains.struct()
    _check(lib().mpg_separator_bsdf(ctx.h, C.byref(cs), _ptr(contrib), cam, float(exponent), _ptr(rad), _ptr(L),
                                    _stream(stream)))
    return rad, L


def mpg_records_bsdf(ctx, chains, rec_chain, omega, w, camera, exponent, R=None, R_dev=None, stream=None):
    """Product importance sampling weights (Eq. eq_weight_pis), in place on w."""
    R = int(w.numel()) if R is None else R
    cam = (C.c_float * 3)(*[float(v) for v in camera])
    cs = chains.struct()
    _check(lib().mpg_records_bsdf(ctx.h, C.byref(cs), _ptr(rec_chain), _ptr(omega), _ptr(w), R, _ptr(R_dev), cam,
                                  float(exponent), _stream(stream)))


class STree:
    """Spatial tree of the guide samples (Sec. 5.6; mpg_stree_*): built from
    the records of a pass (their chain indices) over those chains' (x_D, x_L)."""

    def __init__(self, ctx, chains, rec_chain, R=None, R_dev=None, epsilon=0.1, c=1.0, method=None, stream=None):
        """method: STREE_LEVELS (level by level on the device, the default: the
        same tree as the depth-first build, faster in the progressive schedule)
        or STREE_RECURSIVE (depth first on the host)."""
        self.ctx = ctx
        R = int(rec_chain.numel()) if R is None else R
        h = C.c_void_p()
        cs = chains.struct()
        method = STREE_LEVELS if method is None else method
        _check(lib().mpg_stree_build(ctx.h, C.byref(cs), _ptr(rec_chain), R, _ptr(R_dev), epsilon, c, method,
                                     C.byref(h), _stream(stream)))
        self._adopt(h)

    @classmethod
    def from_host(cls, pos, epsilon=0.1, c=1.0, method=None):
        """The tree of host positions pos [n, 6] (x_D, x_L) with no device copy
        (mpg_stree_build_host; needs no GPU): info and export only.  method:
        STREE_RECURSIVE (default) or STREE_LEVELS (the device build's passes
        as host loops)."""
        pos = np.ascontiguousarray(np.asarray(pos, np.float32).reshape(-1, 6).T)
        h = C.c_void_p()
        method = STREE_RECURSIVE if method is None else method
        _check(lib().mpg_stree_build_host(pos.ctypes.data if pos.size else None, pos.shape[1], epsilon, c, method,
                                          C.byref(h)))
        t = cls.__new__(cls)
        t.ctx = None
        t._adopt(h)
        return t

    def _adopt(self, h):
        self.h = h
        v = [C.c_int32() for _ in range(4)]
        _check(lib().mpg_stree_info(self.h, *[C.byref(x) for x in v]))
        self.n_samples, self.n_nodes, self.n_leaves, self.n_members = (x.value for x in v)

    def export(self):
        """Host arrays: axis, split, left, right [n_nodes]; member_leaf, member_rec [n_members]."""
        n, m = self.n_nodes, self.n_members
        ax, lf, rt = (np.zeros(n, np.int32) for _ in range(3))
        sp = np.zeros(n, np.float64)
        ml, mr = np.zeros(max(m, 1), np.int32), np.zeros(max(m, 1), np.int32)
        _check(lib().mpg_stree_export(self.h, ax.ctypes.data, sp.ctypes.data, lf.ctypes.data, rt.ctypes.data,
                                      ml.ctypes.data, mr.ctypes.data))
        return ax, sp, lf, rt, ml[:m], mr[:m]

    def records(self, rec, R_in, out=None, stream=None):
        """Guide records of the leaves from records (cell, omega, w, k, tau, ...)
        of capacity R_in: (cell, omega, w, k, tau, count), n_members of them."""
        M = max(self.n_members, 1)
        if out is None:
            out = (torch.zeros(M, dtype=torch.int32, device="cuda"), torch.zeros((3, M), dtype=torch.float32, device="cuda"),
                   torch.zeros(M, dtype=torch.float32, device="cuda"), torch.zeros(M, dtype=torch.uint8, device="cuda"),
                   torch.zeros(M, dtype=torch.uint8, device="cuda"), torch.zeros(4, dtype=torch.int32, device="cuda"))
        cell, om, w, k, tau, R = out
        _check(lib().mpg_stree_records(self.ctx.h, self.h, _ptr(rec[1]), _ptr(rec[2]), _ptr(rec[3]), _ptr(rec[4]),
                                       R_in, _ptr(cell), _ptr(om), _ptr(w), _ptr(k), _ptr(tau), om.shape[1], _ptr(R),
                                       _stream(stream)))
        return out

    def query(self, chains, out=None, stream=None):
        """Leaf of each chain (int32 [B]), for chains.chain_cell."""
        out = out if out is not None else torch.zeros(chains.B, dtype=torch.int32, device="cuda")
        cs = chains.struct()
        _check(lib().mpg_stree_query(self.ctx.h, self.h, C.byref(cs), _ptr(out), _stream(stream)))
        return out

    def __del__(self):
        if getattr(self, "h", None):
            lib().mpg_stree_destroy(self.h)
            self.h = None


def mpg_vmf_build(ctx, guide, cell, omega, w, k, tau, R=None, R_dev=None, weight_shift=16, stream=None):
    """Lobes of the vMF guide from records: cell [R] int32, omega [3, R], w [R],
    k [R] uint8, tau [R] uint8 (device tensors; R_dev a device count <= R)."""
    R = int(cell.numel()) if R is None else R
    gs = guide.struct()
    _check(lib().mpg_vmf_build(ctx.h, C.byref(gs), _ptr(cell), _ptr(omega), _ptr(w), _ptr(k), _ptr(tau), R,
                               _ptr(R_dev), weight_shift, _stream(stream)))


def mpg_training_plan(total_spp, first_spp=1, train_fraction=0.3, max_iters=32):
    """Seeds per point of each training iteration and of the rendering stage
    (Sec. 5.8, online training): returns (list of iteration counts, render count)."""
    it = (C.c_int32 * max_iters)()
    n, r = C.c_int32(), C.c_int32()
    _check(lib().mpg_training_plan(total_spp, first_spp, train_fraction, max_iters, it, C.byref(n), C.byref(r)))
    return [int(it[i]) for i in range(n.value)], int(r.value)


def mpg_sample_lengths(ctx, guide, chains, p0_weights, params, rng_seed, rng_offset=0, out=None, stream=None):
    """Chain lengths and P(n) from the mixture of P_0 (integer weights
    p0_weights[n-1]) and the vMF guide (or None): returns (k [B] uint8, pn [B] f32)."""
    B = chains.B
    k, pn = out if out is not None else (torch.zeros(B, dtype=torch.uint8, device="cuda"),
                                         torch.zeros(B, dtype=torch.float32, device="cuda"))
    w = (C.c_uint32 * 8)(*[int(x) for x in p0_weights])
    cs = chains.struct()
    gs = guide.struct() if guide is not None else None
    _check(lib().mpg_sample_lengths(ctx.h, C.byref(gs) if gs is not None else None, C.byref(cs), w, rng_seed,
                                    rng_offset, C.byref(params), _ptr(k), _ptr(pn), _stream(stream)))
    return k, pn


def mpg_walk_adjoint(ctx, scene, chains, T, contrib, dL_dE, dL_dtheta, stream=None):
    """dL_dtheta (heights of heightfield 0, accumulated) += sum_b dL_dE[q] d(contrib_b/spq)/dtheta."""
    cs = chains.struct()
    _check(lib().mpg_walk_adjoint(ctx.h, scene.h, C.byref(cs), _ptr(T), _ptr(contrib), _ptr(dL_dE),
                                  _ptr(dL_dtheta), _stream(stream)))


def mpg_trace_rays(ctx, scene, o, d, tmin=1e-4, tmax=3.0e38, out=None, stream=None):
    """o, d: [3, n] float32 device tensors; out: optional (t, surf, prim, bary)."""
    n = o.shape[1]
    if out is None:
        out = (torch.empty(n, dtype=torch.float32, device=o.device), torch.empty(n, dtype=torch.int32, device=o.device),
               torch.empty(n, dtype=torch.int32, device=o.device), torch.empty((2, n), dtype=torch.float32, device=o.device))
    t, surf, prim, bary = out
    _check(lib().mpg_trace_rays(ctx.h, scene.h, _ptr(o), _ptr(d), n, tmin, tmax, _ptr(t), _ptr(surf), _ptr(prim),
                                _ptr(bary), _stream(stream)))
    return t, surf, prim, bary


def run(ctx, scene, chains, wl, guide=None, params=None, out=None, stream=None):
    """Whole hot path on the GPU: seeds -> walk -> contribution + Bernoulli -> E."""
    P = params if params is not None else params_from(wl.params, tau_random=wl.tau_random,
                                                      k_uniform=int(wl.k[0]) if (wl.k == wl.k[0]).all() else 0)
    mpg_sample_seeds(ctx, scene, guide, chains, P, wl.rng_seed, 0, stream)
    mpg_manifold_walk(ctx, scene, chains, P, stream)
    return mpg_chain_contribution(ctx, scene, guide, chains, P, wl.rng_seed, 0, out, stream)
