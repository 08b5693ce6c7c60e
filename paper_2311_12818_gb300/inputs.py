"""Seeded synthetic workloads for the batched manifold walk.

This module is the one place both the CUDA path and the FP64 oracle take their
inputs from.  It builds plain data only -- scene tables, receiver grids, light
samples, chain lengths and scattering types -- and holds none of the method's
arithmetic (no constraint, no ray casting, no Newton step, no geometry term).

Every workload stands in for one of the paper's scene classes (Sec. 6 renders
sphere-like casters, stacked slabs/lenses and a water surface); the paper's own
scenes are not public, so all inputs here are procedural and seeded.

Data formats (shared by both sides as *formats*, each side parses them itself):

surface table, float64 [S, 24], one row per specular surface
    0 type (SURF_*), 1 material (MAT_*), 2 eta_front, 3 eta_back
    4..6 centre (sphere/cap) or rectangle centre, 7 radius
    8..10 cap axis (unit) or rectangle normal, 11 cap cosine: a cap keeps the
          sphere points p with dot(p - c, axis) >= radius * cap_cos
    12..14 rectangle half-axis e_x, 15..17 rectangle half-axis e_y
    18 heightfield index (type SURF_HEIGHTFIELD)
    The front side is the side the surface normal points into: outward for
    spheres and caps, +normal for rectangles, +z (up) for heightfields.

heightfield descriptor, float64 [H, 6]: nx, ny, x0, y0, x1, y1 -- an nx*ny
    vertex grid over [x0,x1]x[y0,y1]; heights concatenated row-major (y outer).

light, float64 [16]: 0 type (LIGHT_*), 1..3 position / rectangle centre,
    4..6 emitting normal, 7..9 half-axis e_x, 10..12 half-axis e_y,
    13 intensity (point, W/sr) or radiance (rectangle).

seed targets, float64 [T, 16]: 0 type (TARGET_*), 1..3 centre, 4 radius,
    5..7 half-axis e_x, 8..10 half-axis e_y, 11..13 normal.  The initial
    seed distribution p_0 (Sec. 5.4) picks a target uniformly and samples a
    point on it (visible cap of a sphere target, uniform area on a rectangle).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SURF_SPHERE, SURF_CAP, SURF_RECT, SURF_HEIGHTFIELD = 0, 1, 2, 3
MAT_MIRROR, MAT_DIELECTRIC = 0, 1
LIGHT_POINT, LIGHT_RECT = 0, 1
TARGET_SPHERE, TARGET_RECT = 0, 1

MAXK = 8
N_THETA = 64
N_PHI = 64

# Status codes written per chain (same values on both sides).
ST_INVALID, ST_CONVERGED, ST_FAILED, ST_LIMIT = 0, 1, 2, 3


def _surface(type_, material, eta_front=1.0, eta_back=1.0, centre=(0, 0, 0), radius=0.0,
             axis=(0, 0, 1), cap_cos=-1.0, ex=(0, 0, 0), ey=(0, 0, 0), hf=0):
    row = np.zeros(24, np.float64)
    row[0], row[1], row[2], row[3] = type_, material, eta_front, eta_back
    row[4:7], row[7] = centre, radius
    row[8:11], row[11] = axis, cap_cos
    row[12:15], row[15:18] = ex, ey
    row[18] = hf
    return row


def _light(type_, pos, normal=(0, 0, -1), ex=(0, 0, 0), ey=(0, 0, 0), power=1.0):
    row = np.zeros(16, np.float64)
    row[0], row[1:4], row[4:7], row[7:10], row[10:13], row[13] = type_, pos, normal, ex, ey, power
    return row


def _target(type_, centre, radius=0.0, ex=(0, 0, 0), ey=(0, 0, 0), normal=(0, 0, 1)):
    row = np.zeros(16, np.float64)
    row[0], row[1:4], row[4], row[5:8], row[8:11], row[11:14] = type_, centre, radius, ex, ey, normal
    return row


@dataclasses.dataclass
class Params:
    """Solver constants (the paper fixes none of them; the values are a reading of it)."""
    tol: float = 1e-6            # converged when max_i |C_i|_inf < tol
    max_iter: int = 20           # Newton steps
    max_halvings: int = 8        # step halvings per Newton step
    ray_eps: float = 1e-4        # ray origin offset / segment shrink (scene units)
    sing_eps: float = 1e-10      # |det B'| <= sing_eps * max|B'|^2 => singular
    dedup_eps: float = 3.4641e-4  # two chains are one solution below this distance
    max_trials: int = 10000      # Bernoulli trial cap
    alpha: float = 0.5           # defensive mixture weight of p_0 (Sec. 5.5)
    weight_shift: int = 16       # histogram weight quantisation q = floor(w * 2^S)
    stall_tol: float = 2e-5      # FP32 walks only: stalled line search within this |C| counts as converged
    fp64_tol: float = 1e-4       # FP32 G recomputed in FP64 when its two reciprocal forms differ by more
    bern_repeats: int = 1        # independent Bernoulli estimates averaged per chain
    selective: int = 0           # selective activation: no seeds where the guide's cell is empty
    roughness: float = 0.0       # Beckmann roughness of glossy chains (their offsets' distribution)


@dataclasses.dataclass
class Workload:
    name: str
    surfaces: np.ndarray          # [S,24] f64
    hf_desc: np.ndarray           # [H,6] f64
    hf_heights: np.ndarray        # [sum nx*ny] f64
    targets: np.ndarray           # [T,16] f64
    light: np.ndarray             # [16] f64
    xD: np.ndarray                # [Q,3] f64 receiver points (separators x_D)
    nD: np.ndarray                # [Q,3] f64 receiver normals
    cell: np.ndarray              # [Q] u32 guide cell of each receiver point
    spq: int                      # seeds per receiver point
    xL: np.ndarray                # [B,3] f64 light-side separator x_L per seed
    k: np.ndarray                 # [B] u8 chain length n (called k here)
    tau: np.ndarray               # [B] u8 scattering types, bit i-1 set => vertex i is T
    tau_random: bool              # draw tau per trial (Bernoulli 0.5 per vertex)
    pn: np.ndarray                # [B] f64 P(n) of each chain's length
    n_cells: int
    rng_seed: int
    scene_scale: float
    params: Params
    receiver_shape: tuple = (0, 0)

    @property
    def Q(self):
        return self.xD.shape[0]

    @property
    def B(self):
        return self.xL.shape[0]

    @property
    def light_area(self):
        if int(self.light[0]) == LIGHT_POINT:
            return 1.0
        return 4.0 * float(np.linalg.norm(self.light[7:10]) * np.linalg.norm(self.light[10:13]))

    @property
    def max_k(self):
        return int(self.k.max()) if self.k.size else 1


def guide_edges(n_theta: int = N_THETA, n_phi: int = N_PHI):
    """Bin edges of the (theta, phi) guide histogram, as FP32 data.

    theta is measured from +z and split uniformly over [0, pi]; phi uniformly
    over [0, 2 pi).  Edges are evaluated once in FP64 and rounded to FP32 so
    both sides classify directions against the very same numbers.
    Returns cos_theta[n_theta+1] (cos_theta[0]=1, [-1]=-1), phi_cos[n_phi+1],
    phi_sin[n_phi+1].
    """
    j = np.arange(n_theta + 1, dtype=np.float64)
    ct = np.cos(j * math.pi / n_theta).astype(np.float32)
    ct[0], ct[-1] = 1.0, -1.0
    i = np.arange(n_phi + 1, dtype=np.float64)
    pc = np.cos(i * 2.0 * math.pi / n_phi).astype(np.float32)
    ps = np.sin(i * 2.0 * math.pi / n_phi).astype(np.float32)
    return ct, pc, ps


def _receiver_grid(n_x, n_y, x0, x1, y0, y1, z, normal, cells_x=16, cells_y=16):
    ix, iy = np.meshgrid(np.arange(n_x), np.arange(n_y), indexing="xy")
    x = x0 + (ix + 0.5) * (x1 - x0) / n_x
    y = y0 + (iy + 0.5) * (y1 - y0) / n_y
    xD = np.stack([x.ravel(), y.ravel(), np.full(x.size, z)], axis=1).astype(np.float64)
    nD = np.tile(np.asarray(normal, np.float64), (xD.shape[0], 1))
    cx = (ix.ravel() * cells_x) // n_x
    cy = (iy.ravel() * cells_y) // n_y
    cell = (cy * cells_x + cx).astype(np.uint32)
    return xD, nD, cell


def _light_samples(light, B, rng):
    if int(light[0]) == LIGHT_POINT:
        return np.tile(light[1:4], (B, 1)).astype(np.float64)
    u = rng.random((B, 2))
    return (light[1:4][None, :] + (2 * u[:, :1] - 1) * light[7:10][None, :]
            + (2 * u[:, 1:2] - 1) * light[10:13][None, :])


def mirror_sphere(n: int = 64, spq: int = 16, seed: int = 0x4D50470001) -> Workload:
    """Single reflection off an analytic mirror sphere (radius 1 at the origin),
    point light at (0,3,2), receiver z=-1.5 over [-3,3]^2 with n x n points,
    spq seeds per point drawn uniformly on the visible cap, k=1, tau=R."""
    surfaces = np.stack([_surface(SURF_SPHERE, MAT_MIRROR, 1.0, 1.0, (0, 0, 0), 1.0)])
    light = _light(LIGHT_POINT, (0.0, 3.0, 2.0), power=1.0)
    targets = np.stack([_target(TARGET_SPHERE, (0, 0, 0), 1.0)])
    xD, nD, cell = _receiver_grid(n, n, -3, 3, -3, 3, -1.5, (0, 0, 1))
    B = xD.shape[0] * spq
    xL = _light_samples(light, B, np.random.default_rng(seed))
    scale = 2.0 * math.sqrt(3.0)
    return Workload("mirror_sphere_k1", surfaces, np.zeros((0, 6)), np.zeros(0), targets, light,
                    xD, nD, cell, spq, xL, np.ones(B, np.uint8), np.zeros(B, np.uint8), False,
                    np.ones(B), 256, seed, scale, Params(dedup_eps=1e-4 * scale), (n, n))


def glass_sphere(n: int = 256, spq: int = 16, seed: int = 0x4D50470002) -> Workload:
    """Refractive caustic through a glass sphere (radius 1, IOR 1.5), k=2 (T,T),
    0.2x0.2 area light at z=4 facing down, receiver z=-1.5 over [-2,2]^2 with
    n x n points grouped into 16x16 guide cells."""
    surfaces = np.stack([_surface(SURF_SPHERE, MAT_DIELECTRIC, 1.0, 1.5, (0, 0, 0), 1.0)])
    light = _light(LIGHT_RECT, (0.0, 0.0, 4.0), (0, 0, -1), (0.1, 0, 0), (0, 0.1, 0), 1.0)
    targets = np.stack([_target(TARGET_SPHERE, (0, 0, 0), 1.0)])
    xD, nD, cell = _receiver_grid(n, n, -2, 2, -2, 2, -1.5, (0, 0, 1))
    B = xD.shape[0] * spq
    xL = _light_samples(light, B, np.random.default_rng(seed))
    scale = 2.0 * math.sqrt(3.0)
    return Workload("glass_sphere_k2", surfaces, np.zeros((0, 6)), np.zeros(0), targets, light,
                    xD, nD, cell, spq, xL, np.full(B, 2, np.uint8), np.full(B, 0b11, np.uint8),
                    False, np.ones(B), 256, seed, scale, Params(dedup_eps=1e-4 * scale), (n, n))


def water_heights(grid: int = 128, seed: int = 0x4D50470003, n_waves: int = 8):
    """h(x,y) = sum_i a_i sin(k_i . (x,y) + phi_i) on a grid x grid lattice over
    [-1,1]^2, a_i ~ U(0,0.02), |k_i| ~ U(2,12), direction ~ U(0,2pi), phi_i ~ U(0,2pi)."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.0, 0.02, n_waves)
    kmag = rng.uniform(2.0, 12.0, n_waves)
    kdir = rng.uniform(0.0, 2 * math.pi, n_waves)
    ph = rng.uniform(0.0, 2 * math.pi, n_waves)
    xs = np.linspace(-1.0, 1.0, grid)
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    h = np.zeros_like(X)
    for i in range(n_waves):
        h += a[i] * np.sin(kmag[i] * (math.cos(kdir[i]) * X + math.sin(kdir[i]) * Y) + ph[i])
    return h.ravel().astype(np.float64)


def water(n: int = 512, spq: int = 4, grid: int = 128, seed: int = 0x4D50470003) -> Workload:
    """Water surface as a grid x grid triangulated heightfield over [-1,1]^2
    (IOR 1.33 below, air above, interpolated vertex normals), pool floor
    receiver z=-1 with n x n points, 0.2x0.2 area light at z=4.  Per point,
    spq seeds: k=1 (T) with probability 3/4, else k=2 with tau RT or TR."""
    surfaces = np.stack([_surface(SURF_HEIGHTFIELD, MAT_DIELECTRIC, 1.0, 1.33, hf=0)])
    hf_desc = np.array([[grid, grid, -1.0, -1.0, 1.0, 1.0]], np.float64)
    heights = water_heights(grid, seed)
    light = _light(LIGHT_RECT, (0.0, 0.0, 4.0), (0, 0, -1), (0.1, 0, 0), (0, 0.1, 0), 1.0)
    targets = np.stack([_target(TARGET_RECT, (0, 0, 0), 0.0, (1, 0, 0), (0, 1, 0), (0, 0, 1))])
    xD, nD, cell = _receiver_grid(n, n, -1, 1, -1, 1, -1.0, (0, 0, 1))
    B = xD.shape[0] * spq
    rng = np.random.default_rng(seed ^ 0x5A5A)
    xL = _light_samples(light, B, rng)
    u = rng.random(B)
    k = np.where(u < 0.75, 1, 2).astype(np.uint8)
    tau = np.where(k == 1, 0b01, np.where(rng.random(B) < 0.5, 0b10, 0b01)).astype(np.uint8)
    scale = float(math.sqrt(8.0 + (heights.max() - heights.min()) ** 2))
    pn = np.where(k == 1, 0.75, 0.25)
    return Workload("water_heightfield", surfaces, hf_desc, heights, targets, light, xD, nD, cell,
                    spq, xL, k, tau, False, pn, 256, seed, scale, Params(dedup_eps=1e-4 * scale),
                    (n, n))


GEOMETRIC_K_PMF = np.array([0.35 * 0.65 ** (i - 1) for i in range(1, MAXK + 1)])
GEOMETRIC_K_PMF = GEOMETRIC_K_PMF / GEOMETRIC_K_PMF.sum()
# The same law as integer weights (sampled lengths draw n by exact integer
# inverse CDF): round(pmf * 2^20).
GEOMETRIC_K_WEIGHTS = np.round(GEOMETRIC_K_PMF * (1 << 20)).astype(np.uint32)


def mixed(nx: int = 1024, ny: int = 512, spq: int = 8, seed: int = 0x4D50470004) -> Workload:
    """Mixed-length batch: nested glass spheres (r=1 IOR 1.5 around r=0.5 IOR 1.7)
    at (-2,0,0), four stacked biconvex lenses (two caps of radius 1.5, centre
    thickness 0.2, IORs 1.5/1.7/1.5/1.7) along z at x=2, a mirror plane z=-0.5
    under them; receiver points on a downward-facing plane z=3 over
    [-4,4]x[-2,2]; 0.2x0.2 area light at (0,0,4) facing down.  k ~ Geometric(0.35)
    truncated to 1..8, tau_i ~ Bernoulli(0.5) drawn per trial."""
    rows = [
        _surface(SURF_SPHERE, MAT_DIELECTRIC, 1.0, 1.5, (-2, 0, 0), 1.0),
        _surface(SURF_SPHERE, MAT_DIELECTRIC, 1.5, 1.7, (-2, 0, 0), 0.5),
    ]
    targets = [_target(TARGET_SPHERE, (-2, 0, 0), 1.0)]
    R, half_t = 1.5, 0.1
    cap_cos = (R - half_t) / R
    for j, eta in enumerate((1.5, 1.7, 1.5, 1.7)):
        zc = 0.3 + 0.5 * j
        rows.append(_surface(SURF_CAP, MAT_DIELECTRIC, 1.0, eta, (2, 0, zc + half_t - R), R,
                             (0, 0, 1), cap_cos))
        rows.append(_surface(SURF_CAP, MAT_DIELECTRIC, 1.0, eta, (2, 0, zc - half_t + R), R,
                             (0, 0, -1), cap_cos))
        targets.append(_target(TARGET_SPHERE, (2, 0, zc), 0.55))
    rows.append(_surface(SURF_RECT, MAT_MIRROR, 1.0, 1.0, (0, 0, -0.5), 0.0, (0, 0, 1), -1.0,
                         (4, 0, 0), (0, 2, 0)))
    targets.append(_target(TARGET_RECT, (0, 0, -0.5), 0.0, (4, 0, 0), (0, 2, 0), (0, 0, 1)))
    surfaces = np.stack(rows)
    light = _light(LIGHT_RECT, (0.0, 0.0, 4.0), (0, 0, -1), (0.1, 0, 0), (0, 0.1, 0), 1.0)
    xD, nD, cell = _receiver_grid(nx, ny, -4, 4, -2, 2, 3.0, (0, 0, -1))
    B = xD.shape[0] * spq
    rng = np.random.default_rng(seed)
    xL = _light_samples(light, B, rng)
    k = (rng.choice(MAXK, size=B, p=GEOMETRIC_K_PMF) + 1).astype(np.uint8)
    scale = float(math.sqrt(8.0 ** 2 + 4.0 ** 2 + 2.9 ** 2))
    return Workload("mixed_k1to8", surfaces, np.zeros((0, 6)), np.zeros(0), np.stack(targets), light,
                    xD, nD, cell, spq, xL, k, np.zeros(B, np.uint8), True, GEOMETRIC_K_PMF[k - 1],
                    256, seed, scale, Params(dedup_eps=1e-4 * scale), (ny, nx))


def water_rays(n: int, seed: int = 0x4D50470013):
    """Ray batch for the standalone BVH pass on the water heightfield: origins
    above (z = 2) or below (z = -1) the surface over [-1.1, 1.1]^2, aimed at
    uniform points of the surface's bounding slab (|z| < 0.05).  Returns
    (o, d) as [n, 3] float64."""
    rng = np.random.default_rng(seed)
    o = np.column_stack([rng.uniform(-1.1, 1.1, n), rng.uniform(-1.1, 1.1, n), rng.choice([-1.0, 2.0], n)])
    tgt = np.column_stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(-0.05, 0.05, n)])
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o, d


def upstream_grad(Q: int, seed: int = 0x4D50470005):
    """dL/dE per receiver point, U(0,1), for the adjoint workload."""
    return np.random.default_rng(seed).random(Q)


WORKLOADS = {
    "mirror_sphere": mirror_sphere,
    "glass_sphere": glass_sphere,
    "water": water,
    "mixed": mixed,
}


def synthetic_guide_records(wl: Workload, per_cell: int = 512, seed: int = 0x4D50470014):
    """Seeded synthetic guide records for a workload (for tests at sizes where
    no training pass is run): per receiver cell, `per_cell` records with a
    receiver point of the cell, a direction from it toward a random point
    within 1.2 radii of a random sphere seed target (or on a rectangle
    target), a log-uniform weight in [1e-6, 1e-1], a length drawn like the
    workload's (the geometric law for the mixed batch) and random types.
    Returns (cell [R] u32, omega [R, 3] f32, w [R] f32, k [R] u8, tau [R] u8)."""
    rng = np.random.default_rng(seed)
    cells = np.unique(wl.cell)
    R = cells.size * per_cell
    cell = np.repeat(cells, per_cell).astype(np.uint32)
    pts = np.empty((R, 3))
    for j, c in enumerate(cells):
        q = np.nonzero(wl.cell == c)[0]
        pts[j * per_cell:(j + 1) * per_cell] = wl.xD[rng.choice(q, per_cell)]
    tg = wl.targets[rng.integers(0, wl.targets.shape[0], R)]
    off = rng.normal(size=(R, 3))
    off /= np.linalg.norm(off, axis=1, keepdims=True)
    aim = np.where((tg[:, 0] == TARGET_SPHERE)[:, None],
                   tg[:, 1:4] + off * (1.2 * tg[:, 4:5]) * rng.random((R, 1)),
                   tg[:, 1:4] + (2 * rng.random((R, 1)) - 1) * tg[:, 5:8] + (2 * rng.random((R, 1)) - 1) * tg[:, 8:11])
    d = aim - pts
    om = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    w = np.exp(rng.uniform(math.log(1e-6), math.log(1e-1), R)).astype(np.float32)
    if (wl.k == wl.k[0]).all():
        k = np.full(R, wl.k[0], np.uint8)
    else:
        k = (rng.choice(MAXK, size=R, p=GEOMETRIC_K_PMF) + 1).astype(np.uint8)
    tau = (rng.integers(0, 256, R) & ((1 << k.astype(np.int64)) - 1)).astype(np.uint8)
    if not wl.tau_random:
        tau = np.full(R, wl.tau[0], np.uint8)
    return cell, om, w, k, tau
