"""Pin of the per-unit operation counts (oracle/unit_flops.py, orc_unit_flops)
that turn the kernels' work counters into algorithmic FLOP/s.

The oracle counts by running its own primitives in a counted scalar type.
Here every count is derived again by hand from the formula each primitive
evaluates: the constraint and Jacobian of the manifold walk (the generalized
half-vector of Sec. 3), the 2x2-block Thomas sweep, the generalized geometry
term of Eq. ThroughputEval by the implicit function theorem, the Fresnel
factor, the ray tests, and the tangent frames.  Convention: +, -, *, / and
sqrt are one operation each; negation, absolute value and comparisons are
free; there is no fused multiply-add.  A mistake in the counting harness (an
operation counted twice, a helper call leaking into a unit, a stale json)
fails here."""
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# building blocks on 3-vectors and 2x2 matrices
VADD = 3                      # a + b, a - b
VSCALE = 3                    # a * s, a / s
DOT = 3 + 2                   # 3 products, 2 sums
NORM = DOT + 1                # sqrt(a.a)
NORMALIZE = NORM + 3          # a / |a|
CROSS = 6 + 3                 # 6 products, 3 differences
ONB = 13                      # Duff et al. 2017, counted below
M2MUL = 8 + 4                 # 2x2 times 2x2
DET2 = 2 + 1                  # ad - bc
INV2 = 4                      # (d, -b, -c, a) / det: four divisions
M2VEC = 4 + 2                 # 2x2 times a 2-vector


def hand_counts():
    c = {}
    # Duff's basis of a unit n: a = -1/(s + n_z) [1 add, 1 div], b = n_x n_y a
    # [2 mul], b1 = (1 + s n_x n_x a, s b, -s n_x) [3 mul + 1 add, 1 mul,
    # 1 mul], b2 = (b, s + n_y n_y a, -n_y) [2 mul + 1 add]
    onb = (1 + 1) + 2 + (3 + 1) + 1 + 1 + (2 + 1)
    assert onb == ONB
    # sphere frame: n = normalize(p - c), the basis, dn/du = dp/du / r (twice)
    c["frame_sphere"] = VADD + NORMALIZE + ONB + 2 * VSCALE
    # plane frame: the basis of the fixed normal only
    c["frame_plane"] = ONB
    # triangle with corner normals at barycentrics (b1, b2):
    #   edges e1, e2; p = P0 + e1 b1 + e2 b2; geometric normal and its basis;
    #   N = N0 (1 - b1 - b2) + N1 b1 + N2 b2, |N|, n = N / |N|;
    #   Gram entries g11, g12, g22 and their determinant;
    #   per tangent direction: r1, r2; db1, db2 (2 mul + 1 add + 1 div each);
    #   dN = (N1 - N0) db1 + (N2 - N0) db2; dn = (dN - n (n.dN)) / |N|
    shading = 2 + 3 * VSCALE + 2 * VADD
    per_dir = 2 * DOT + 2 * (2 + 1 + 1) + (2 * VADD + 2 * VSCALE + VADD) + (DOT + VSCALE + VADD + VSCALE)
    c["frame_triangle"] = (2 * VADD + (2 * VSCALE + 2 * VADD) + (CROSS + NORMALIZE) + ONB + shading + NORM + VSCALE
                           + 3 * DOT + DET2 + 2 * per_dir)
    c["normal_sphere"] = VADD + NORMALIZE
    c["normal_triangle"] = shading + NORMALIZE
    # vertex constraint C = (h.s, h.t): w_i, w_o from the neighbours (difference,
    # length, division), the side test w_i.n, h~ = eta_i w_i + eta_o w_o,
    # h = h~ / |h~|, the shading basis (s, t), two dot products
    constraint = 2 * (VADD + NORM + VSCALE) + DOT + (2 * VSCALE + VADD) + NORM + VSCALE + ONB + 2 * DOT
    c["vertex_constraint"] = constraint
    # Jacobian blocks: h.n once; per tangent direction j of each vertex the
    # projections P_w a = (a - w (w.a)) / d (DOT + 3 mul + 3 sub + 3 div);
    #   A: P_h(eta_i P_wi(dp_prev)) then two dots;
    #   Cc: P_h(eta_o P_wo(dp_next)) then two dots;
    #   B: -P_h(eta_i P_wi(dp) + eta_o P_wo(dp)), each component
    #      dot(dhB, s) - (h.n) (s.dn): two dots, 1 mul, 1 sub
    proj = DOT + VSCALE + VADD + VSCALE
    a_blk = proj + VSCALE + proj + 2 * DOT
    b_blk = 2 * (proj + VSCALE) + VADD + proj + 2 * (2 * DOT + 1 + 1)
    c["vertex_blocks"] = constraint + DOT + 2 * (2 * a_blk + b_blk)
    # block Thomas, one right-hand column: first row = det, inverse and the
    # back substitution x = B'^-1 r; every further row also forms
    # L = A B'^-1_prev and L Cc_prev, B' = B - L Cc_prev (4 sub), r' = r - L r'_prev
    # (2 x (2 mul + 2 add)) and, in the backward sweep, r - Cc x_next (same)
    c["thomas_first_row"] = DET2 + INV2 + M2VEC
    rhs_upd = 2 * (2 + 2)
    c["thomas_row"] = 2 * M2MUL + 4 + rhs_upd + DET2 + INV2 + rhs_upd + M2VEC
    # two right-hand columns (the geometry term's J Y = -B_e)
    c["ggt_row"] = 2 * M2MUL + 4 + 2 * rhs_upd + DET2 + INV2 + 2 * (rhs_upd + M2VEC)
    # geometry-term tail after the solve: w = x_1 - x_D, |w|, w / |w|; basis of
    # w; per column dx = dp/du y0 + dp/dv y1, dw = (dx - w (w.dx)) / |w|, two
    # projections onto the basis; |det M|; cos(theta_D) = n_D.w and G = cos |det|
    per_col = (2 * VSCALE + VADD) + (DOT + VSCALE + VADD + VSCALE) + 2 * DOT
    c["ggt_tail"] = VADD + NORM + VSCALE + ONB + 2 * per_col + DET2 + DOT + 1
    # ray/sphere with a unit direction: oc = o - c, b = oc.d, cc = oc.oc - r r,
    # disc = b b - cc, sqrt, roots -b -+ sqrt (negation free)
    c["ray_sphere"] = VADD + DOT + (DOT + 1 + 1) + (1 + 1) + 1 + 2
    # ray/rectangle: t = ((c - o).n) / (d.n); q = o + d t - c; the two in-plane
    # projections q.ex, q.ey and the extents ex.ex, ey.ey
    c["ray_rect"] = VADD + DOT + DOT + 1 + (VSCALE + 2 * VADD) + 4 * DOT
    # Moeller-Trumbore: e1, e2; pv = d x e2; det = e1.pv; 1/det; tv = o - p0;
    # b1 = (tv.pv) inv; qv = tv x e1; b2 = (d.qv) inv; t = (e2.qv) inv
    c["ray_triangle"] = 2 * VADD + CROSS + DOT + 1 + VADD + (DOT + 1) + CROSS + (DOT + 1) + (DOT + 1)
    # slab test: per axis (lo - o) / d and (hi - o) / d
    c["ray_box"] = 3 * (2 + 2)
    # kappa of one refracting dielectric vertex: w_i = normalize(x_prev - x),
    # cos = |w_i.n|; Fresnel: s2 = (e1/e2)(e1/e2)(1 - c c) [2 div, 3 mul, 1 sub],
    # cos2 = sqrt(1 - s2), r_s and r_p (4 mul + 2 add + 1 div each), F =
    # 0.5 (rs rs + rp rp) [3 mul + 1 add]; r = eta_i / eta_o; (1 - F) r r
    fresnel = (2 + 3 + 1) + (1 + 1) + 2 * (4 + 2 + 1) + (3 + 1)
    c["kappa_vertex"] = VADD + NORMALIZE + DOT + fresnel + 1 + (1 + 2)
    return c


def test_hand_counted_building_blocks():
    assert (DOT, NORM, NORMALIZE, CROSS, M2MUL, DET2, M2VEC) == (5, 6, 9, 9, 12, 3, 6)


def test_counted_oracle_equals_hand_counts():
    pytest.importorskip("numpy")
    from oracle import unit_flops as U
    got = U.unit_flops()
    want = hand_counts()
    assert set(got) == set(want)
    bad = {k: (got[k], want[k]) for k in want if got[k] != want[k]}
    assert not bad, bad


def test_committed_unit_flops_json_is_the_oracle_count():
    from oracle import unit_flops as U
    with open(os.path.join(ROOT, "paper_2311_12818_gb300", "unit_flops.json")) as f:
        stored = json.load(f)["flops"]
    assert stored == U.unit_flops() == {k: float(v) for k, v in hand_counts().items()}
