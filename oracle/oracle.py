"""ctypes front end of the FP64 oracle (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg import
this module; the CUDA library never does.  Arrays are numpy, float64 unless
stated, array-of-structures: x[B, 8, 3], surf/prim[B, 8], bary[B, 8, 2].
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import build as _build

MAXK = 8

_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")


class orc_params(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("max_halvings", C.c_int32),
                ("ray_eps", C.c_double), ("sing_eps", C.c_double), ("dedup_eps", C.c_double),
                ("max_trials", C.c_int32), ("weight_shift", C.c_int32), ("alpha", C.c_double),
                ("bern_repeats", C.c_int32), ("selective", C.c_int32)]


class orc_vmf(C.Structure):
    _fields_ = [("n_cells", C.c_int32), ("n_lobes", C.c_int32), ("cell_start", C.c_void_p),
                ("key", C.c_void_p), ("lobe", C.c_void_p), ("prefix", C.c_void_p)]


class orc_guide(C.Structure):
    _fields_ = [("counts", C.c_void_p), ("n_cells", C.c_int32), ("n_theta", C.c_int32),
                ("n_phi", C.c_int32), ("cos_theta", C.c_void_p), ("phi_cos", C.c_void_p),
                ("phi_sin", C.c_void_p), ("vmf", C.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_scene_create.restype = C.c_void_p
        L.orc_scene_create.argtypes = [_f64p, C.c_int32, _f64p, _f64p, C.c_int32, _f64p, C.c_int32, _f64p]
        L.orc_scene_destroy.argtypes = [C.c_void_p]
        L.orc_intersect.argtypes = [C.c_void_p, C.c_int32, _f64p, _f64p, C.c_double, C.c_double,
                                    C.c_int32, _f64p, _i32p, _i32p, _f64p]
        L.orc_sample_seeds.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, _f64p, _f64p, _u32p,
                                       C.c_int32, _f64p, _u8p, _u8p, C.c_int32, C.c_uint64,
                                       C.c_uint64, C.c_uint32, C.POINTER(orc_params), _f64p, _i32p,
                                       _i32p, _f64p, _u8p, _f64p, _u8p, C.c_int32, C.c_void_p]
        L.orc_walk.argtypes = [C.c_void_p, C.c_int32, C.c_int32, _f64p, _f64p, _f64p, _u8p, _u8p,
                               C.POINTER(orc_params), _u8p, _f64p, _i32p, _i32p, _f64p, _u8p, _u8p,
                               C.c_int32, C.c_void_p]
        L.orc_contribution.argtypes = [C.c_void_p, C.c_int32, C.c_int32, _f64p, _f64p, _f64p, _u8p,
                                       _u8p, _f64p, _i32p, _i32p, _f64p, _u8p,
                                       C.POINTER(orc_params), _f64p, _f64p, _f64p, _u8p, C.c_int32]
        L.orc_bernoulli.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, _f64p, _f64p, _u32p,
                                    C.c_int32, _f64p, _u8p, _u8p, C.c_int32, C.c_uint64, C.c_uint64,
                                    C.POINTER(orc_params), _f64p, _i32p, _u8p, _u32p, _u8p, C.c_void_p,
                                    C.c_int32, C.c_void_p, C.c_void_p]
        L.orc_sample_offsets.argtypes = [C.c_int32, _u8p, C.c_double, C.c_uint64, C.c_uint64, _f64p]
        L.orc_glossy.argtypes = [C.c_void_p, C.c_int32, C.c_int32, _f64p, _f64p, _f64p, _u8p, _u8p, _f64p, _i32p,
                                 _i32p, _f64p, _u8p, C.POINTER(orc_params), C.c_void_p, C.c_double, _f64p, _u8p,
                                 C.c_int32]
        L.orc_guide_bin.argtypes = [C.POINTER(orc_guide), C.c_int32, _f32p, _i32p]
        L.orc_guide_update.argtypes = [C.POINTER(orc_guide), _u64p, C.c_int32, _u32p, _f32p, _f32p,
                                       C.c_int32]
        L.orc_constraint.argtypes = [C.c_void_p, C.c_int32, C.c_int32, _f64p, _f64p, _f64p, _u8p, _u8p,
                                     _f64p, _i32p, _i32p, _f64p, _f64p, _f64p]
        L.orc_shoot.argtypes = [C.c_void_p, _f64p, _f64p, C.c_int32, C.c_uint8, C.c_double, _f64p, _f64p]
        L.orc_adjoint.argtypes = [C.c_void_p, C.c_int32, C.c_int32, _f64p, _f64p, _f64p, _u8p, _u8p, _f64p, _i32p,
                                  _i32p, _f64p, _f64p, _f64p, _f64p, C.c_int32]
        L.orc_adjoint.restype = C.c_int32
        L.orc_vmf_build.argtypes = [C.c_int32, C.c_int32, _u32p, _f32p, _f32p, _u8p, _u8p, C.c_int32, _u32p,
                                    _u32p, _f64p, _u64p]
        L.orc_sample_lengths.argtypes = [C.c_void_p, C.c_int32, _u32p, C.c_int32, _u32p, C.c_uint64, C.c_uint64,
                                         C.POINTER(orc_params), _u8p, _f64p, C.c_void_p]
        L.orc_vmf_pdf.argtypes = [_f64p, C.c_double, _f64p]
        L.orc_vmf_pdf.restype = C.c_double
        L.orc_vmf_sample.argtypes = [_f64p, C.c_double, C.c_double, C.c_double, _f64p]
        L.orc_vmf_sample.restype = None
        L.orc_philox.argtypes = [_u32p, _u32p, _u32p]
        L.orc_philox.restype = None
        for name in ("orc_intersect", "orc_sample_seeds", "orc_walk", "orc_contribution",
                     "orc_bernoulli", "orc_guide_bin", "orc_guide_update", "orc_constraint",
                     "orc_shoot", "orc_vmf_build", "orc_sample_lengths", "orc_sample_offsets", "orc_glossy"):
            getattr(L, name).restype = C.c_int32
        _lib = L
    return _lib


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def params(p) -> orc_params:
    return orc_params(p.tol, p.max_iter, p.max_halvings, p.ray_eps, p.sing_eps, p.dedup_eps,
                      p.max_trials, p.weight_shift, p.alpha, int(getattr(p, "bern_repeats", 1)),
                      int(getattr(p, "selective", 0)))


def default_threads():
    return max(1, os.cpu_count() or 1)


class Scene:
    """Oracle scene built from a workload's surface/heightfield/target/light tables."""

    def __init__(self, wl):
        L = lib()
        self._keep = [_c(wl.surfaces, np.float64), _c(wl.hf_desc.reshape(-1, 6), np.float64),
                      _c(wl.hf_heights, np.float64), _c(wl.targets, np.float64), _c(wl.light, np.float64)]
        s, hd, hh, tg, li = self._keep
        hd_arg = hd if hd.size else np.zeros(6, np.float64)
        hh_arg = hh if hh.size else np.zeros(1, np.float64)
        self.h = L.orc_scene_create(s, s.shape[0], hd_arg, hh_arg, hd.shape[0], tg, tg.shape[0], li)
        if not self.h:
            raise ValueError("oracle rejected the scene description")

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_scene_destroy(self.h)
            self.h = None


class Guide:
    """Histogram state for the oracle: counts[n_cells, n_theta*n_phi] uint64 plus edge tables."""

    def __init__(self, n_cells, edges, counts=None):
        ct, pc, ps = (np.ascontiguousarray(e, np.float32) for e in edges)
        self.ct, self.pc, self.ps = ct, pc, ps
        self.n_theta, self.n_phi = ct.size - 1, pc.size - 1
        self.n_cells = n_cells
        self.counts = (np.zeros((n_cells, self.n_theta * self.n_phi), np.uint64) if counts is None
                       else np.ascontiguousarray(counts, np.uint64))

    def struct(self, with_counts=True):
        return orc_guide(self.counts.ctypes.data if with_counts else None, self.n_cells,
                         self.n_theta, self.n_phi, self.ct.ctypes.data, self.pc.ctypes.data,
                         self.ps.ctypes.data, None)

    def bins(self, omega):
        om = _c(omega, np.float32).reshape(-1, 3)
        out = np.zeros(om.shape[0], np.int32)
        g = self.struct()
        assert lib().orc_guide_bin(C.byref(g), om.shape[0], om, out) == 0
        return out

    def update(self, cell, omega, w, shift):
        om = _c(omega, np.float32).reshape(-1, 3)
        g = self.struct()
        rc = lib().orc_guide_update(C.byref(g), self.counts, om.shape[0], _c(cell, np.uint32), om,
                                    _c(w, np.float32), shift)
        assert rc == 0, rc


class VmfGuide:
    """vMF mixture guide (Sec. 5.5) of the oracle: one lobe per record, lobes of
    a cell contiguous and ordered by (n, tau) and record order.  Arrays:
    cell_start[n_cells+1], key[L] = (n << 8) | tau, lobe[L, 4] = (mu, kappa),
    prefix[L] = inclusive prefix sums of the quantised weights within the cell."""

    def __init__(self, n_cells):
        self.n_cells = n_cells
        self.build(np.zeros(0, np.uint32), np.zeros((0, 3), np.float32), np.zeros(0, np.float32),
                   np.zeros(0, np.uint8), np.zeros(0, np.uint8), 16)

    def build(self, cell, omega, w, k, tau, shift):
        om = _c(omega, np.float32).reshape(-1, 3)
        R = om.shape[0]
        self.cell_start = np.zeros(self.n_cells + 1, np.uint32)
        self.key = np.zeros(max(R, 1), np.uint32)
        self.lobe = np.zeros((max(R, 1), 4), np.float64)
        self.prefix = np.zeros(max(R, 1), np.uint64)
        rc = lib().orc_vmf_build(self.n_cells, R, _c(cell, np.uint32), om, _c(w, np.float32), _c(k, np.uint8),
                                 _c(tau, np.uint8), shift, self.cell_start, self.key, self.lobe, self.prefix)
        assert rc == 0, rc
        self.n_lobes = R
        self._v = orc_vmf(self.n_cells, R, self.cell_start.ctypes.data, self.key.ctypes.data,
                          self.lobe.ctypes.data, self.prefix.ctypes.data)
        return self

    def struct(self):
        return orc_guide(None, self.n_cells, 0, 0, None, None, None, C.addressof(self._v))


def training_plan(total_spp, first_spp=1, train_fraction=0.3):
    """Seeds per point of the training iterations and of rendering, following
    the online training of Sec. 5.8 step by step: the sample count doubles
    each iteration; training stops as soon as train_fraction of the budget is
    used; when an iteration ends, a new one starts if less than half of the
    training budget is used, else the current one continues until training
    ends.  Returns (iteration counts, rendering count)."""
    budget = math.floor(train_fraction * total_spp)
    iters = []
    used, size = 0, first_spp
    while used < budget:
        take = min(size, budget - used)          # stop immediately at the training budget
        iters.append(take)
        used += take
        if used >= budget:
            break
        if used < budget / 2:                    # start a new, doubled iteration
            size *= 2
        else:                                    # continue the current iteration
            iters[-1] += budget - used
            used = budget
    return iters, total_spp - used


def sample_lengths(wl, guide, p0w, rng_offset=0, chain_cell=None):
    """Chain lengths and P(n) from the defensive mixture of P_0 (integer weights
    p0w[n-1]) and the vMF guide's P_e(n | cell) (Sec. 5.5)."""
    cc = _cells(chain_cell)
    k = np.zeros(wl.B, np.uint8)
    pn = np.zeros(wl.B)
    g = guide.struct() if guide is not None else None
    P = params(wl.params)
    rc = lib().orc_sample_lengths(C.byref(g) if g is not None else None, wl.Q, _c(wl.cell, np.uint32), wl.spq,
                                  _c(p0w, np.uint32), wl.rng_seed, rng_offset, C.byref(P), k, pn,
                                  None if cc is None else cc.ctypes.data)
    assert rc == 0, rc
    return k, pn


def vmf_pdf(mu, kappa, w):
    return lib().orc_vmf_pdf(_c(mu, np.float64), float(kappa), _c(w, np.float64))


def vmf_sample(mu, kappa, u1, u2):
    out = np.zeros(3)
    lib().orc_vmf_sample(_c(mu, np.float64), float(kappa), float(u1), float(u2), out)
    return out


def intersect(scene, o, d, tmin=1e-4, tmax=np.inf, brute=False):
    o = _c(o, np.float64).reshape(-1, 3)
    d = _c(d, np.float64).reshape(-1, 3)
    n = o.shape[0]
    t = np.zeros(n); surf = np.zeros(n, np.int32); prim = np.zeros(n, np.int32); bary = np.zeros((n, 2))
    assert lib().orc_intersect(scene.h, n, o, d, tmin, tmax, int(brute), t, surf, prim, bary) == 0
    return t, surf, prim, bary


def _cells(chain_cell):
    """Per-chain guide cells (uint32, kept alive by the caller) or None."""
    return None if chain_cell is None else _c(chain_cell, np.uint32)


def sample_seeds(wl, scene, guide=None, trial=0, threads=None, rng_offset=0, chain_cell=None):
    B = wl.B
    cc = _cells(chain_cell)
    out = dict(x=np.zeros((B, MAXK, 3)), surf=np.zeros((B, MAXK), np.int32),
               prim=np.zeros((B, MAXK), np.int32), bary=np.zeros((B, MAXK, 2)),
               tau=np.zeros(B, np.uint8), pdf=np.zeros(B), valid=np.zeros(B, np.uint8))
    g = guide.struct() if guide is not None else None
    P = params(wl.params)
    rc = lib().orc_sample_seeds(scene.h, C.byref(g) if g is not None else None, wl.Q,
                                _c(wl.xD, np.float64), _c(wl.nD, np.float64), _c(wl.cell, np.uint32),
                                wl.spq, _c(wl.xL, np.float64), _c(wl.k, np.uint8), _c(wl.tau, np.uint8),
                                int(wl.tau_random), wl.rng_seed, rng_offset, trial, C.byref(P),
                                out["x"], out["surf"], out["prim"], out["bary"], out["tau"], out["pdf"],
                                out["valid"], threads or default_threads(), None if cc is None else cc.ctypes.data)
    assert rc == 0, rc
    return out


def _offsets(offset, B):
    if offset is None:
        return None
    o = np.ascontiguousarray(offset, np.float64)
    assert o.shape == (B, MAXK, 2), o.shape
    return o


def walk(wl, scene, seeds, threads=None, offset=None):
    """Walk the seeds in place (copies); returns dict with x/surf/prim/bary/status/iters.
    offset [B, 8, 2]: offset normals of glossy chains (Sec. 5.7), or None."""
    B = wl.B
    ch = {n: seeds[n].copy() for n in ("x", "surf", "prim", "bary")}
    status = np.zeros(B, np.uint8)
    iters = np.zeros(B, np.uint8)
    P = params(wl.params)
    rc = lib().orc_walk(scene.h, B, wl.spq, _c(wl.xD, np.float64), _c(wl.nD, np.float64),
                        _c(wl.xL, np.float64), _c(wl.k, np.uint8), _c(seeds["tau"], np.uint8),
                        C.byref(P), _c(seeds["valid"], np.uint8), ch["x"], ch["surf"], ch["prim"],
                        ch["bary"], status, iters, threads or default_threads(),
                        None if (o := _offsets(offset, B)) is None else o.ctypes.data)
    assert rc == 0, rc
    ch.update(status=status, iters=iters, tau=seeds["tau"].copy())
    return ch


def contribution(wl, scene, chains, threads=None):
    B = wl.B
    G = np.zeros(B); kap = np.zeros(B); T = np.zeros(B); adm = np.zeros(B, np.uint8)
    P = params(wl.params)
    rc = lib().orc_contribution(scene.h, B, wl.spq, _c(wl.xD, np.float64), _c(wl.nD, np.float64),
                                _c(wl.xL, np.float64), _c(wl.k, np.uint8), _c(chains["tau"], np.uint8),
                                chains["x"], chains["surf"], chains["prim"], chains["bary"],
                                _c(chains["status"], np.uint8), C.byref(P), G, kap, T, adm,
                                threads or default_threads())
    assert rc == 0, rc
    return dict(G=G, kappa=kap, T=T, admissible=adm)


def bernoulli(wl, scene, chains, admissible, guide=None, threads=None, rng_offset=0, max_trials=None,
              trial_walks=None, chain_cell=None, offset=None):
    B = wl.B
    cc = _cells(chain_cell)
    N = np.zeros(B, np.uint32)
    capped = np.zeros(B, np.uint8)
    tw = None if trial_walks is None else trial_walks.ctypes.data
    p = wl.params
    if max_trials is not None:
        import dataclasses
        p = dataclasses.replace(p, max_trials=max_trials)
    P = params(p)
    g = guide.struct() if guide is not None else None
    rc = lib().orc_bernoulli(scene.h, C.byref(g) if g is not None else None, wl.Q,
                             _c(wl.xD, np.float64), _c(wl.nD, np.float64), _c(wl.cell, np.uint32),
                             wl.spq, _c(wl.xL, np.float64), _c(wl.k, np.uint8),
                             _c(chains["tau"], np.uint8), int(wl.tau_random), wl.rng_seed, rng_offset,
                             C.byref(P), chains["x"], chains["surf"], _c(admissible, np.uint8), N,
                             capped, tw, threads or default_threads(), None if cc is None else cc.ctypes.data,
                             None if (o := _offsets(offset, B)) is None else o.ctypes.data)
    assert rc == 0, rc
    return N, capped


def sample_offsets(wl, alpha, rng_offset=0):
    """Offset normals of glossy chains (Sec. 5.7): [B, 8, 2] tangential
    components drawn from a Beckmann distribution of roughness alpha."""
    out = np.zeros((wl.B, MAXK, 2))
    rc = lib().orc_sample_offsets(wl.B, _c(wl.k, np.uint8), float(alpha), wl.rng_seed, rng_offset, out)
    assert rc == 0, rc
    return out


def glossy(wl, scene, chains, offset=None, alpha=0.0, threads=None):
    """Terms of converged glossy chains (Sec. 5.7): |det dC/du|, the BSDF
    product with D divided out, the geometric factors, the offsets' density,
    the estimate W (alpha = 0: the specular limit) and admissibility."""
    B = wl.B
    out = np.zeros((B, 5))
    adm = np.zeros(B, np.uint8)
    P = params(wl.params)
    o = _offsets(offset, B)
    rc = lib().orc_glossy(scene.h, B, wl.spq, _c(wl.xD, np.float64), _c(wl.nD, np.float64), _c(wl.xL, np.float64),
                          _c(wl.k, np.uint8), _c(chains["tau"], np.uint8), _c(chains["x"], np.float64),
                          _c(chains["surf"], np.int32), _c(chains["prim"], np.int32), _c(chains["bary"], np.float64),
                          _c(chains["status"], np.uint8), C.byref(P), None if o is None else o.ctypes.data,
                          float(alpha), out, adm, threads or default_threads())
    assert rc == 0, rc
    return dict(detJ=out[:, 0], bsdf=out[:, 1], geom=out[:, 2], dens=out[:, 3], W=out[:, 4], admissible=adm)


def constraint(wl, scene, chains):
    B = wl.B
    Cv = np.zeros((B, 2 * MAXK))
    cmax = np.zeros(B)
    rc = lib().orc_constraint(scene.h, B, wl.spq, _c(wl.xD, np.float64), _c(wl.nD, np.float64),
                              _c(wl.xL, np.float64), _c(wl.k, np.uint8), _c(chains["tau"], np.uint8),
                              _c(chains["x"], np.float64), _c(chains["surf"], np.int32),
                              _c(chains["prim"], np.int32), _c(chains["bary"], np.float64), Cv, cmax)
    assert rc == 0, rc
    return Cv, cmax


def philox(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().orc_philox(_c(ctr, np.uint32), _c(key, np.uint32), out)
    return out


def shoot(scene, xD, omega, k, tau, ray_eps=1e-4):
    """Trace x_D along omega through k vertices with types tau (the forward map)."""
    x = np.zeros((k, 3))
    d = np.zeros(3)
    rc = lib().orc_shoot(scene.h, _c(xD, np.float64), _c(omega, np.float64), k, tau, ray_eps, x, d)
    return (x, d) if rc == 0 else (None, None)


def adjoint(wl, scene, chains, weight, threads=None):
    """dL/dtheta (heights of heightfield 0) for L = sum_b weight[b] T_b; also
    the per-chain flag of a formed gradient."""
    n_h = int(wl.hf_heights.size)
    g = np.zeros(n_h)
    okf = np.zeros(wl.B)
    rc = lib().orc_adjoint(scene.h, wl.B, wl.spq, _c(wl.xD, np.float64), _c(wl.nD, np.float64),
                           _c(wl.xL, np.float64), _c(wl.k, np.uint8), _c(chains["tau"], np.uint8),
                           _c(chains["x"], np.float64), _c(chains["surf"], np.int32), _c(chains["prim"], np.int32),
                           _c(chains["bary"], np.float64), _c(weight, np.float64), g, okf,
                           threads or default_threads())
    assert rc == 0, rc
    return g, okf


def _repeats(wl):
    return max(1, int(getattr(wl.params, "bern_repeats", 1)))


def irradiance(wl, T, N, admissible):
    """E(x_D) = (1/M) sum_seeds A_L T <1/P>, <1/P> = N / (repeats P(n))   (Eq. ThroughputMC; Sec. 5.8)."""
    c = np.where(admissible.astype(bool), wl.light_area * T * N.astype(np.float64) / (_repeats(wl) * wl.pn), 0.0)
    return c.reshape(wl.Q, wl.spq).sum(axis=1) / wl.spq


def records(wl, chains, T, N, admissible, with_types=False):
    """Guide-update records of the admissible chains in chain order: (cell, w_D
    as FP32, w = T <1/P> as FP32), and with_types: also (n, tau)."""
    idx = np.nonzero(admissible)[0]
    q = idx // wl.spq
    x1 = chains["x"][idx, 0, :]
    d = x1 - wl.xD[q]
    om = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    w = (T[idx] * N[idx].astype(np.float64) / (_repeats(wl) * wl.pn[idx])).astype(np.float32)
    if with_types:
        return (wl.cell[q].astype(np.uint32), om, w, wl.k[idx].astype(np.uint8),
                chains["tau"][idx].astype(np.uint8))
    return wl.cell[q].astype(np.uint32), om, w


def run(wl, guide=None, threads=None, max_trials=None):
    """Whole hot path in the oracle: seeds -> walk -> contribution -> Bernoulli -> E."""
    sc = Scene(wl)
    seeds = sample_seeds(wl, sc, guide, threads=threads)
    ch = walk(wl, sc, seeds, threads=threads)
    con = contribution(wl, sc, ch, threads=threads)
    N, capped = bernoulli(wl, sc, ch, con["admissible"], guide, threads=threads, max_trials=max_trials)
    E = irradiance(wl, con["T"], N, con["admissible"])
    return dict(scene=sc, seeds=seeds, chains=ch, contrib=con, N=N, capped=capped, E=E)


def progressive(make_workload, total_spp, first_spp=1, train_fraction=0.3, guide="histogram", threads=None):
    """Online training and rendering (Sec. 5.8) in the oracle: each training
    iteration samples from the guide of the previous one (p_0 first) and its
    records alone build the next guide; the rendering stage's irradiance is
    the image.  Stage i draws its random numbers at offset i * 2^36.
    Returns (plan, render spp, per-stage dicts, image)."""
    from paper_2311_12818_gb300 import inputs as I
    plan, render = training_plan(total_spp, first_spp, train_fraction)
    wls = [make_workload(s, i) for i, s in enumerate(plan + [render])]
    sc = Scene(wls[0])
    g = None
    stages = []
    for i, wl in enumerate(wls):
        o = i << 36
        seeds = sample_seeds(wl, sc, g, threads=threads, rng_offset=o)
        ch = walk(wl, sc, seeds, threads=threads)
        con = contribution(wl, sc, ch, threads=threads)
        N, capped = bernoulli(wl, sc, ch, con["admissible"], g, threads=threads, rng_offset=o)
        stages.append(dict(wl=wl, seeds=seeds, chains=ch, contrib=con, N=N, guide=g))
        if i == len(plan):
            break
        cell, om, w, k, tau = records(wl, ch, con["T"], N, con["admissible"], with_types=True)
        if guide == "histogram":
            g = Guide(wl.n_cells, I.guide_edges())
            g.update(cell, om, w, wl.params.weight_shift)
        else:
            g = VmfGuide(wl.n_cells).build(cell, om, w, k, tau, wl.params.weight_shift)
    last = stages[-1]
    image = irradiance(last["wl"], last["contrib"]["T"], last["N"], last["contrib"]["admissible"])
    return plan, render, stages, image


def phong(w_i, n, w, exponent):
    """Separator BSDF of the glossy-separator extension (Sec. 5.7): a
    normalised Phong lobe (e + 2) / (2 pi) max(0, r.w)^e around the mirror
    direction r = w_i - 2 (w_i.n) n of the incoming camera ray w_i (unit,
    toward x_D), for unit directions w leaving x_D.  Arrays [m, 3]."""
    w_i, n, w = (np.atleast_2d(np.asarray(a, np.float64)) for a in (w_i, n, w))
    r = w_i - 2.0 * np.sum(w_i * n, axis=1, keepdims=True) * n
    c = np.maximum(np.sum(r * w, axis=1), 0.0)
    return (exponent + 2.0) / (2.0 * math.pi) * c ** exponent


def camera_rays(wl, camera):
    """Unit directions from the camera position to each receiver point [Q, 3]."""
    d = wl.xD - np.asarray(camera, np.float64)[None, :]
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def separator_radiance(wl, chains, contrib, camera, exponent):
    """Radiance toward the camera at each receiver point: (1/M) sum over its
    seeds of rho(w_i, w_D) times the chain's contribution, w_D = unit(x_1 - x_D).
    Returns (per-chain weighted contributions [B], per-point radiance [Q])."""
    q = np.arange(wl.B) // wl.spq
    d = chains["x"][:, 0, :] - wl.xD[q]
    nrm = np.linalg.norm(d, axis=1, keepdims=True)
    w_D = d / np.where(nrm > 0, nrm, 1.0)
    rho = phong(camera_rays(wl, camera)[q], wl.nD[q], w_D, exponent)
    c = np.where(contrib > 0, rho * contrib, 0.0)
    return c, c.reshape(wl.Q, wl.spq).sum(axis=1) / wl.spq


def records_bsdf(wl, chain, omega, w, camera, exponent):
    """Product importance sampling weights (Eq. eq_weight_pis): each record's
    weight times the separator BSDF at its receiver point toward its direction."""
    q = np.asarray(chain, np.int64) // wl.spq
    rho = phong(camera_rays(wl, camera)[q], wl.nD[q], np.asarray(omega, np.float64), exponent)
    return (np.asarray(w, np.float64) * rho).astype(np.float32)
