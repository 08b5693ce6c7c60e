// Device-side math of the manifold walk (sm_103a, FP32 unless noted).
//
// One CUDA thread owns one chain; vertex state lives in registers, templated
// on the chain length K so the 2x2-block arrays are fully unrolled.  The
// formulas follow the paper's problem statement (Sec. 3-5) and the standard
// manifold-walk definitions it cites:
//   constraint  C_i = (h.s_i, h.t_i),  h = (eta_i w_i + eta_o w_o)/|...|
//   Jacobian    block-tridiagonal, 2x2 blocks A_i, B_i, Cc_i (analytic)
//   solve       2x2-block Thomas sweep
//   step        tangent-plane move, step halving, reprojection of each vertex
//               onto its own surface (radial / normal / vertical ray cast)
//   G           implicit function theorem, 2-column Thomas solve
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mpg.h"

namespace mpg {

constexpr int MAXK = 8;
constexpr int MAX_SURF = 16;
constexpr int MAX_HF = 2;
constexpr int MAX_TG = 16;
constexpr int BVH_STACK = 64;

enum { SURF_SPHERE = 0, SURF_CAP = 1, SURF_RECT = 2, SURF_HEIGHTFIELD = 3 };
enum { MAT_MIRROR = 0, MAT_DIELECTRIC = 1 };
enum { LIGHT_POINT = 0, LIGHT_RECT = 1 };
enum { TARGET_SPHERE = 0, TARGET_RECT = 1 };
enum { ST_INVALID = 0, ST_CONVERGED = 1, ST_FAILED = 2, ST_LIMIT = 3, ST_SEEDED = 255 };
enum { ERR_BVH_STACK = 1, ERR_GUIDE_CELL = 2, ERR_VMF_RECORD = 4 };

// ---------------------------------------------------------------------------
// Scene description passed by value (kernel parameter space).
// ---------------------------------------------------------------------------
struct DSurf {
  int type, mat, hf;
  float etaF, etaB, r, cap_cos;
  float3 c, axis, ex, ey;
  float ex2, ey2;  // squared half-axis lengths of a rectangle
};

struct DHF {
  int nx, ny, surf, n_nodes;
  float x0, y0, dx, dy;
  const float4* P;      // [ny*nx] vertex positions (w unused)
  const float4* N;      // [ny*nx] vertex interpolation normals
  const float4* nodes;  // [n_nodes*4] two-child BVH nodes
  const float4* tris;   // [n_tris*3] leaf-ordered (v0|prim, e1, e2)
};

struct DLight {
  int type;
  float3 p, n, exu, eyu;  // centre, emitting normal, unit half-axes
  float power, area;
};

struct DTarget {
  int type;
  float3 c, ex, ey, n;
  float r, area;
};

struct DScene {
  int n_surf, n_hf, n_tg;
  DSurf s[MAX_SURF];
  DHF hf[MAX_HF];
  DTarget tg[MAX_TG];
  DLight L;
};

// The scene copied to shared memory at the start of a walk kernel.  The walk
// indexes the surface table by each lane's own surface id; read from the
// kernel's parameter (constant) space, such loads are served one distinct
// address of the warp at a time, from shared memory in one pass (bank
// conflicts apart).  The persistent kernels of the batched mode (a few
// blocks per SM) use it; the kernels launched with one block per 128 chains
// (seeds, contributions, the adjoint and the plain mode's walk and trial
// loops) read the parameter space directly: there the copy per block cost
// more than it saved.  Every thread of the block must call it, before any
// thread returns.
__device__ __forceinline__ const DScene& scene_in_smem(const DScene& S, DScene& sm) {
  static_assert(sizeof(DScene) % 4 == 0, "copied as 32-bit words");
  for (int i = threadIdx.x; i < (int)(sizeof(DScene) / 4); i += blockDim.x)
    reinterpret_cast<int*>(&sm)[i] = reinterpret_cast<const int*>(&S)[i];
  __syncthreads();
  return sm;
}

struct DGuide {
  int n_cells, n_theta, n_phi, bins;
  const uint64_t* counts;
  const uint64_t* cdf;
  const float* cos_theta;
  const float* phi_cos;
  const float* phi_sin;
  int kind;                     // MPG_GUIDE_HISTOGRAM or MPG_GUIDE_VMF
  const uint32_t* cell_start;   // vMF: [n_cells+1]
  const uint32_t* lobe_key;     // vMF: (n << 8) | tau
  const float4* lobe;           // vMF: (mu, kappa)
  const uint64_t* lobe_prefix;  // vMF: cell-local inclusive prefix sums of the quantised weights
  const float* lobe_coef;       // vMF: q_i kappa_i / (2 pi (1 - e^{-2 kappa_i}))
};

// Per-thread work counters (flushed once per warp).
struct Counters {
  uint32_t newton, rows, full_evals, c_evals, casts, sphere, plane, node, tri, ggt, seeds, ggt64;
};

// ---------------------------------------------------------------------------
// Vector helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator-(float3 a) { return make_float3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return make_float3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float len(float3 a) { return sqrtf(dot(a, a)); }
__device__ __forceinline__ float3 unit(float3 a) { return a * (1.0f / sqrtf(dot(a, a))); }
__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }

// Branchless orthonormal basis completing the unit vector n (Duff et al. 2017,
// JCGT 6(1)); the constraint components are expressed in this frame.
__device__ __forceinline__ void onb(float3 n, float3& b1, float3& b2) {
  float s = n.z >= 0.0f ? 1.0f : -1.0f;
  float a = -1.0f / (s + n.z);
  float b = n.x * n.y * a;
  b1 = make_float3(1.0f + s * n.x * n.x * a, s * b, -s * n.x);
  b2 = make_float3(b, s + n.y * n.y * a, -n.y);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC 2011): counter (idx_lo, idx_hi, trial, block).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
    uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}
__device__ __forceinline__ float u01(uint32_t r) { return (float)(r >> 8) * (1.0f / 16777216.0f); }

// ---------------------------------------------------------------------------
// Ray casting: r(x, w) of Eq. (deduction), nearest hit with all surfaces.
// ---------------------------------------------------------------------------
struct Hit {
  float t;
  int surf, prim;
  float b1, b2;
};

// Roots of |o + t d - c|^2 = r^2 for unit d.  The discriminant is taken from
// the distance of the line to the centre and the near root from the product of
// the roots, which keeps FP32 accurate when o is far from or on the sphere.
__device__ __forceinline__ bool sphere_roots(float3 o, float3 d, float3 c, float r, float& t0, float& t1) {
  float3 oc = o - c;
  float b = dot(oc, d);
  float3 q = oc - d * b;
  float disc = fmaf(r, r, -dot(q, q));
  if (disc < 0.0f) return false;
  float sq = sqrtf(disc);
  float cc = fmaf(-r, r, dot(oc, oc));
  float qq = -b - copysignf(sq, b);  // |qq| = |b| + sq
  float ta = qq, tb = (qq != 0.0f) ? cc / qq : 0.0f;
  t0 = fminf(ta, tb);
  t1 = fmaxf(ta, tb);
  return true;
}

__device__ __forceinline__ bool box_hit(float3 o, float3 inv, float lox, float hix, float loy, float hiy,
                                        float loz, float hiz, float tmin, float tmax) {
  float tx0 = (lox - o.x) * inv.x, tx1 = (hix - o.x) * inv.x;
  float ty0 = (loy - o.y) * inv.y, ty1 = (hiy - o.y) * inv.y;
  float tz0 = (loz - o.z) * inv.z, tz1 = (hiz - o.z) * inv.z;
  float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), tmin));
  float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tmax));
  return tn <= tf;
}

// Moeller-Trumbore test against a leaf triangle (v0, e1, e2).
__device__ __forceinline__ bool tri_hit(float3 o, float3 d, float3 v0, float3 e1, float3 e2, float tmin,
                                        float tmax, float& t, float& b1, float& b2) {
  float3 pv = cross(d, e2);
  float det = dot(e1, pv);
  if (fabsf(det) < 1e-30f) return false;
  float inv = 1.0f / det;
  float3 tv = o - v0;
  b1 = dot(tv, pv) * inv;
  if (b1 < 0.0f || b1 > 1.0f) return false;
  float3 qv = cross(tv, e1);
  b2 = dot(d, qv) * inv;
  if (b2 < 0.0f || b1 + b2 > 1.0f) return false;
  t = dot(e2, qv) * inv;
  return t > tmin && t < tmax;
}

// BVH traversal of a heightfield's triangles (closest hit below tbest).
template <bool kStats>
__device__ __forceinline__ void hf_traverse(const DHF& H, float3 o, float3 d, float tmin, float& tbest, Hit& best,
                                            int* err, Counters& cnt) {
  float3 inv = make_float3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
  int stack[BVH_STACK];
  int sp = 0;
  int node = 0;
  while (true) {
    const float4* nd = H.nodes + 4 * node;
    float4 a = __ldg(nd + 0), b = __ldg(nd + 1), c = __ldg(nd + 2);
    int4 ch = __ldg(reinterpret_cast<const int4*>(nd + 3));
    if (kStats) cnt.node += 2;
    bool hl = box_hit(o, inv, a.x, a.y, a.z, a.w, c.x, c.y, tmin, tbest);
    bool hr = box_hit(o, inv, b.x, b.y, b.z, b.w, c.z, c.w, tmin, tbest);
    int next = -1;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      bool h = side == 0 ? hl : hr;
      if (!h) continue;
      int idx = side == 0 ? ch.x : ch.y;
      int count = side == 0 ? ch.z : ch.w;
      if (count > 0) {
        for (int q = idx; q < idx + count; ++q) {
          const float4* tr = H.tris + 3 * q;
          float4 v0 = __ldg(tr), e1 = __ldg(tr + 1), e2 = __ldg(tr + 2);
          float t, b1, b2;
          if (kStats) cnt.tri++;
          if (tri_hit(o, d, f3(v0), f3(e1), f3(e2), tmin, tbest, t, b1, b2)) {
            tbest = t;
            best.t = t; best.surf = H.surf; best.prim = __float_as_int(v0.w);
            best.b1 = b1; best.b2 = b2;
          }
        }
      } else if (next < 0) {
        next = idx;
      } else {
        if (sp >= BVH_STACK) { atomicOr(err, ERR_BVH_STACK); return; }
        stack[sp++] = idx;
      }
    }
    if (next >= 0) { node = next; continue; }
    if (sp == 0) return;
    node = stack[--sp];
  }
}

// The traversal kept out of line: inlined into every ray cast it made the
// kernels that cast rays over analytic scenes too large for the instruction
// cache (the mixed batch's one-launch seed kernel took 4.1 ms per step
// inlined, 1.4 ms out of line; the water scene's BVH-heavy kernels pay the
// calls, about 8 %).
template <bool kStats>
__device__ __noinline__ void hf_intersect(const DHF& H, float3 o, float3 d, float tmin, float& tbest, Hit& best,
                                          int* err, Counters& cnt) {
  hf_traverse<kStats>(H, o, d, tmin, tbest, best, err, cnt);
}

// How a ray cast reaches the heightfields' BVHs: BVH_NONE, the scene holds
// none (the branch compiled out; a call alone costs a kernel registers: the
// plain mode's trial loop has 168 registers without it, 128 and spills with
// it); BVH_CALL, the out-of-line traversal; BVH_INLINE, the traversal inlined
// (the ray-batch kernel, whose loop is the traversal).  The batched seed
// kernel keeps the call whatever the scene: without it the compiler gives it
// 80 registers against 64, and at the lower occupancy its dependent loads
// take longer than the spills it saves.
enum { BVH_NONE = 0, BVH_CALL = 1, BVH_INLINE = 2 };

template <bool kStats, int kBVH = BVH_CALL>
__device__ Hit intersect(const DScene& S, float3 o, float3 d, float tmin, float tmax, int* err, Counters& cnt) {
  Hit best;
  best.t = -1.0f; best.surf = -1; best.prim = -1; best.b1 = best.b2 = 0.0f;
  float tbest = tmax;
  if (kStats) cnt.casts++;
  for (int s = 0; s < S.n_surf; ++s) {
    const DSurf& sf = S.s[s];
    if (sf.type == SURF_SPHERE || sf.type == SURF_CAP) {
      if (kStats) cnt.sphere++;
      float t0, t1;
      if (!sphere_roots(o, d, sf.c, sf.r, t0, t1)) continue;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        float t = q == 0 ? t0 : t1;
        if (!(t > tmin && t < tbest)) continue;
        if (sf.type == SURF_CAP) {
          float3 p = o + d * t;
          if (dot(p - sf.c, sf.axis) < sf.r * sf.cap_cos) continue;
        }
        tbest = t; best.t = t; best.surf = s; best.prim = -1;
        break;
      }
    } else if (sf.type == SURF_RECT) {
      if (kStats) cnt.plane++;
      float den = dot(d, sf.axis);
      if (fabsf(den) < 1e-30f) continue;
      float t = dot(sf.c - o, sf.axis) / den;
      if (!(t > tmin && t < tbest)) continue;
      float3 q = o + d * t - sf.c;
      if (fabsf(dot(q, sf.ex)) > sf.ex2 || fabsf(dot(q, sf.ey)) > sf.ey2) continue;
      tbest = t; best.t = t; best.surf = s; best.prim = -1;
    } else if (kBVH == BVH_CALL) {
      hf_intersect<kStats>(S.hf[sf.hf], o, d, tmin, tbest, best, err, cnt);
    } else if (kBVH == BVH_INLINE) {
      hf_traverse<kStats>(S.hf[sf.hf], o, d, tmin, tbest, best, err, cnt);
    }
  }
  return best;
}

// Heightfield triangle corners (grid vertex indices) of triangle `tri`.
__device__ __forceinline__ void hf_tri(const DHF& H, int tri, int& v0, int& v1, int& v2) {
  int quad = tri >> 1, t = tri & 1;
  int i = quad % (H.nx - 1), j = quad / (H.nx - 1);
  int v00 = j * H.nx + i;
  v0 = v00;
  v1 = t == 0 ? v00 + 1 : v00 + H.nx + 1;
  v2 = t == 0 ? v00 + H.nx + 1 : v00 + H.nx;
}

// Vertex of a hit: analytic surfaces snap the ray point onto the surface;
// triangles take the barycentric combination of their corners.
__device__ __forceinline__ float3 hit_point(const DScene& S, float3 o, float3 d, const Hit& h) {
  const DSurf& sf = S.s[h.surf];
  float3 p = o + d * h.t;
  if (sf.type == SURF_SPHERE || sf.type == SURF_CAP) {
    p = sf.c + unit(p - sf.c) * sf.r;
  } else if (sf.type == SURF_RECT) {
    p = p - sf.axis * dot(p - sf.c, sf.axis);
  } else {
    const DHF& H = S.hf[sf.hf];
    int v0, v1, v2;
    hf_tri(H, h.prim, v0, v1, v2);
    float3 P0 = f3(__ldg(H.P + v0)), P1 = f3(__ldg(H.P + v1)), P2 = f3(__ldg(H.P + v2));
    p = P0 + (P1 - P0) * h.b1 + (P2 - P0) * h.b2;
  }
  return p;
}

// ---------------------------------------------------------------------------
// Local frames
// ---------------------------------------------------------------------------
// Unit shading normal n, tangent basis (dpdu, dpdv) of the surface, and the
// shape operator in the constraint's frame (s, t) = onb(n): W = (s.dn/du,
// s.dn/dv, t.dn/du, t.dn/dv), row-major.
struct Frame {
  float3 n, dpdu, dpdv;
  float4 W;
};

// Unit shading normal only (constraint-only evaluations).
__device__ __forceinline__ float3 vertex_normal(const DScene& S, int surf, int prim, float3 p, float b1, float b2) {
  const DSurf& sf = S.s[surf];
  if (sf.type == SURF_SPHERE || sf.type == SURF_CAP) return unit(p - sf.c);
  if (sf.type == SURF_RECT) return sf.axis;
  const DHF& H = S.hf[sf.hf];
  int v0, v1, v2;
  hf_tri(H, prim, v0, v1, v2);
  float3 N0 = f3(__ldg(H.N + v0)), N1 = f3(__ldg(H.N + v1)), N2 = f3(__ldg(H.N + v2));
  return unit(N0 * (1.0f - b1 - b2) + N1 * b1 + N2 * b2);
}

__device__ __forceinline__ Frame vertex_frame(const DScene& S, int surf, int prim, float3 p, float b1, float b2) {
  Frame f;
  const DSurf& sf = S.s[surf];
  if (sf.type == SURF_SPHERE || sf.type == SURF_CAP) {
    // (dpdu, dpdv) = (s, t) and dn = da / r: W = I / r
    f.n = unit(p - sf.c);
    onb(f.n, f.dpdu, f.dpdv);
    float ir = 1.0f / sf.r;
    f.W = make_float4(ir, 0.f, 0.f, ir);
  } else if (sf.type == SURF_RECT) {
    f.n = sf.axis;
    onb(f.n, f.dpdu, f.dpdv);
    f.W = make_float4(0.f, 0.f, 0.f, 0.f);
  } else {
    // n = normalize(sum b_j N_j); a tangent move a changes the barycentrics by
    // the solution of a = db1 e1 + db2 e2.
    const DHF& H = S.hf[sf.hf];
    int v0, v1, v2;
    hf_tri(H, prim, v0, v1, v2);
    float3 P0 = f3(__ldg(H.P + v0)), P1 = f3(__ldg(H.P + v1)), P2 = f3(__ldg(H.P + v2));
    float3 N0 = f3(__ldg(H.N + v0)), N1 = f3(__ldg(H.N + v1)), N2 = f3(__ldg(H.N + v2));
    float3 e1 = P1 - P0, e2 = P2 - P0;
    onb(unit(cross(e1, e2)), f.dpdu, f.dpdv);
    float3 Ns = N0 * (1.0f - b1 - b2) + N1 * b1 + N2 * b2;
    float il = 1.0f / len(Ns);
    f.n = Ns * il;
    float g11 = dot(e1, e1), g12 = dot(e1, e2), g22 = dot(e2, e2);
    float igd = 1.0f / (g11 * g22 - g12 * g12);
    float3 dN1 = N1 - N0, dN2 = N2 - N0;
    float3 s, t;
    onb(f.n, s, t);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      float3 a = q == 0 ? f.dpdu : f.dpdv;
      float r1 = dot(e1, a), r2 = dot(e2, a);
      float db1 = (g22 * r1 - g12 * r2) * igd, db2 = (g11 * r2 - g12 * r1) * igd;
      float3 dN = dN1 * db1 + dN2 * db2;
      float3 dn = (dN - f.n * dot(f.n, dN)) * il;
      if (q == 0) { f.W.x = dot(s, dn); f.W.z = dot(t, dn); }
      else { f.W.y = dot(s, dn); f.W.w = dot(t, dn); }
    }
  }
  return f;
}

// Indices of refraction on the previous / next vertex's side (R: equal).
__device__ __forceinline__ bool etas(const DSurf& sf, bool front, bool refract, float& ei, float& eo) {
  if (sf.mat == MAT_MIRROR) { ei = eo = 1.0f; return !refract; }
  ei = front ? sf.etaF : sf.etaB;
  eo = refract ? (front ? sf.etaB : sf.etaF) : ei;
  return true;
}

// ---------------------------------------------------------------------------
// Constraint and Jacobian blocks at one vertex
// ---------------------------------------------------------------------------
struct VB {
  float2 C;
  float4 A, B, Cc;  // row-major 2x2: (m00, m01, m10, m11)
  float ei, eo;
  bool front;
};

// Constraint only (line-search evaluations).
__device__ __forceinline__ bool vertex_c(float3 xp, float3 x, float3 xn, float3 n, const DSurf& sf,
                                         bool refract, float2& C) {
  float3 wi = unit(xp - x), wo = unit(xn - x);
  float ei, eo;
  if (!etas(sf, dot(wi, n) > 0.0f, refract, ei, eo)) return false;
  float3 ht = wi * ei + wo * eo;
  float L2 = dot(ht, ht);
  if (!(L2 > 0.0f)) return false;
  float3 h = ht * (1.0f / sqrtf(L2));
  float3 s, t;
  onb(n, s, t);
  C = make_float2(dot(h, s), dot(h, t));
  return true;
}

// Full evaluation.  want_a / want_c: also the off-diagonal blocks (for the
// first / last vertex they are derivatives with respect to the separators).
__device__ __forceinline__ bool vertex_blocks(float3 xp, float3 tpu, float3 tpv, float3 x, const Frame& f,
                                              float3 xn, float3 tnu, float3 tnv, const DSurf& sf,
                                              bool refract, bool want_a, bool want_c, VB& o) {
  float3 wi = xp - x, wo = xn - x;
  float di = len(wi), dO = len(wo);
  if (!(di > 0.0f) || !(dO > 0.0f)) return false;
  float idi = 1.0f / di, ido = 1.0f / dO;
  wi = wi * idi;
  wo = wo * ido;
  o.front = dot(wi, f.n) > 0.0f;
  if (!etas(sf, o.front, refract, o.ei, o.eo)) return false;
  float3 ht = wi * o.ei + wo * o.eo;
  float L = len(ht);
  if (!(L > 0.0f)) return false;
  float iL = 1.0f / L;
  float3 h = ht * iL;
  float3 s, t;
  onb(f.n, s, t);
  o.C = make_float2(dot(h, s), dot(h, t));
  float hn = dot(h, f.n);
  // The derivative of C along dh is (s.dh, t.dh) with dh = (I - h h^T) dht / L;
  // fold the projection into the row vectors: s' = (s - h (h.s)) / L.
  float3 sp = (s - h * o.C.x) * iL, tp = (t - h * o.C.y) * iL;
  // d(w)/d(y) a = (a - w (w.a)) / d for w = (y - x)/|y - x|, so moving x_{i-1}
  // by a changes ht by ei (a - wi (wi.a)) / di, and a row r of the derivative
  // gives r.dht = ai (r.a) - ai (r.wi) (wi.a) with ai = ei / di (likewise
  // ao = eo / dO for x_{i+1}); moving x itself changes ht by minus both.  The
  // blocks are formed from these dot products, the scale factors kept scalar.
  const float ai = o.ei * idi, ao = o.eo * ido, aa = ai + ao;
  const float spi = ai * dot(sp, wi), tpi = ai * dot(tp, wi);
  const float spo = ao * dot(sp, wo), tpo = ao * dot(tp, wo);
  {
    const float wiu = dot(wi, f.dpdu), wiv = dot(wi, f.dpdv), wou = dot(wo, f.dpdu), wov = dot(wo, f.dpdv);
    o.B = make_float4(fmaf(spi, wiu, fmaf(spo, wou, -aa * dot(sp, f.dpdu))) - hn * f.W.x,
                      fmaf(spi, wiv, fmaf(spo, wov, -aa * dot(sp, f.dpdv))) - hn * f.W.y,
                      fmaf(tpi, wiu, fmaf(tpo, wou, -aa * dot(tp, f.dpdu))) - hn * f.W.z,
                      fmaf(tpi, wiv, fmaf(tpo, wov, -aa * dot(tp, f.dpdv))) - hn * f.W.w);
  }
  if (want_a) {
    const float wiu = dot(wi, tpu), wiv = dot(wi, tpv);
    o.A = make_float4(fmaf(ai, dot(sp, tpu), -spi * wiu), fmaf(ai, dot(sp, tpv), -spi * wiv),
                      fmaf(ai, dot(tp, tpu), -tpi * wiu), fmaf(ai, dot(tp, tpv), -tpi * wiv));
  }
  if (want_c) {
    const float wou = dot(wo, tnu), wov = dot(wo, tnv);
    o.Cc = make_float4(fmaf(ao, dot(sp, tnu), -spo * wou), fmaf(ao, dot(sp, tnv), -spo * wov),
                       fmaf(ao, dot(tp, tnu), -tpo * wou), fmaf(ao, dot(tp, tnv), -tpo * wov));
  }
  return true;
}

__device__ __forceinline__ float4 mm(float4 a, float4 b) {
  return make_float4(a.x * b.x + a.y * b.z, a.x * b.y + a.y * b.w, a.z * b.x + a.w * b.z, a.z * b.y + a.w * b.w);
}
__device__ __forceinline__ float2 mv(float4 a, float2 v) {
  return make_float2(a.x * v.x + a.y * v.y, a.z * v.x + a.w * v.y);
}
__device__ __forceinline__ bool inv2(float4 m, float sing_eps, float4& r) {
  float det = m.x * m.w - m.y * m.z;
  float mx = fmaxf(fmaxf(fabsf(m.x), fabsf(m.y)), fmaxf(fabsf(m.z), fabsf(m.w)));
  if (!(fabsf(det) > sing_eps * mx * mx)) return false;
  float id = 1.0f / det;
  r = make_float4(m.w * id, -m.y * id, -m.z * id, m.x * id);
  return true;
}

// Block Thomas sweep J X = R for M right-hand-side columns.  R[i][c] holds
// the 2-vector of block row i, column c; overwritten by X.
template <int K, int M>
__device__ __forceinline__ bool thomas(const VB* vb, float2 (&R)[K][M], float sing_eps) {
  float4 Binv[K];
  float4 Bp = vb[0].B;
  if (!inv2(Bp, sing_eps, Binv[0])) return false;
#pragma unroll
  for (int i = 1; i < K; ++i) {
    float4 Lm = mm(vb[i].A, Binv[i - 1]);
    float4 LC = mm(Lm, vb[i - 1].Cc);
    Bp = make_float4(vb[i].B.x - LC.x, vb[i].B.y - LC.y, vb[i].B.z - LC.z, vb[i].B.w - LC.w);
#pragma unroll
    for (int c = 0; c < M; ++c) {
      float2 l = mv(Lm, R[i - 1][c]);
      R[i][c] = make_float2(R[i][c].x - l.x, R[i][c].y - l.y);
    }
    if (!inv2(Bp, sing_eps, Binv[i])) return false;
  }
#pragma unroll
  for (int i = K - 1; i >= 0; --i) {
#pragma unroll
    for (int c = 0; c < M; ++c) {
      float2 r = R[i][c];
      if (i < K - 1) {
        float2 cx = mv(vb[i].Cc, R[i + 1][c]);
        r = make_float2(r.x - cx.x, r.y - cx.y);
      }
      R[i][c] = mv(Binv[i], r);
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// Chain state of one thread
// ---------------------------------------------------------------------------
template <int K>
struct Chain {
  float3 x[K];
  int surf[K], prim[K];
  float b1[K], b2[K];
};

struct Ends {
  float3 xD, nD, xL;
  uint32_t tau;
};

// Full evaluation of all K vertices; fills vb and the tangent bases.
// off (NULL for specular chains): the offset normals of a glossy chain, one
// 2-vector of tangential components per vertex; the constraint becomes
// C_i = (h.s_i, h.t_i) - off_i (Sec. 5.7) and the Jacobian blocks stay.
template <int K, bool kStats>
__device__ __forceinline__ bool eval_full(const DScene& S, const Chain<K>& ch, const Ends& e, VB (&vb)[K],
                                          float3 (&tu)[K], float3 (&tv)[K], float& cnorm2, float& cmax,
                                          bool want_ends, Counters& cnt, const float2* off = nullptr) {
  Frame fr[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    fr[i] = vertex_frame(S, ch.surf[i], ch.prim[i], ch.x[i], ch.b1[i], ch.b2[i]);
    tu[i] = fr[i].dpdu;
    tv[i] = fr[i].dpdv;
  }
  float3 ru, rv, lu, lv;
  onb(e.nD, ru, rv);
  lu = S.L.exu;
  lv = S.L.eyu;
  cnorm2 = 0.0f;
  cmax = 0.0f;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    float3 xp = i == 0 ? e.xD : ch.x[i - 1];
    float3 xn = i == K - 1 ? e.xL : ch.x[i + 1];
    float3 pu = i == 0 ? ru : tu[i > 0 ? i - 1 : 0], pv = i == 0 ? rv : tv[i > 0 ? i - 1 : 0];
    float3 nu = i == K - 1 ? lu : tu[i < K - 1 ? i + 1 : 0], nv = i == K - 1 ? lv : tv[i < K - 1 ? i + 1 : 0];
    bool wa = i > 0 || want_ends, wc = i < K - 1 || want_ends;
    if (!vertex_blocks(xp, pu, pv, ch.x[i], fr[i], xn, nu, nv, S.s[ch.surf[i]], (e.tau >> i) & 1u, wa, wc, vb[i]))
      return false;
    if (off) vb[i].C = make_float2(vb[i].C.x - off[i].x, vb[i].C.y - off[i].y);
    cnorm2 = fmaf(vb[i].C.x, vb[i].C.x, fmaf(vb[i].C.y, vb[i].C.y, cnorm2));
    cmax = fmaxf(cmax, fmaxf(fabsf(vb[i].C.x), fabsf(vb[i].C.y)));
  }
  if (kStats) cnt.full_evals += K;
  return true;
}

template <int K, bool kStats>
__device__ __forceinline__ bool eval_c(const DScene& S, const Chain<K>& ch, const Ends& e, float& cnorm2,
                                       Counters& cnt, const float2* off = nullptr) {
  cnorm2 = 0.0f;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    float3 xp = i == 0 ? e.xD : ch.x[i - 1];
    float3 xn = i == K - 1 ? e.xL : ch.x[i + 1];
    float3 n = vertex_normal(S, ch.surf[i], ch.prim[i], ch.x[i], ch.b1[i], ch.b2[i]);
    float2 C;
    if (!vertex_c(xp, ch.x[i], xn, n, S.s[ch.surf[i]], (e.tau >> i) & 1u, C)) return false;
    if (off) C = make_float2(C.x - off[i].x, C.y - off[i].y);
    cnorm2 = fmaf(C.x, C.x, fmaf(C.y, C.y, cnorm2));
  }
  if (kStats) cnt.c_evals += K;
  return true;
}

// Vertical ray cast into a heightfield at (x, y): the triangle of the grid
// cell holding (x, y) and the barycentrics of the point in it (O(1): the
// height grid is its own acceleration structure for vertical rays).
__device__ __forceinline__ bool hf_vertical_hit(const DHF& H, float x, float y, float3& p, int& prim, float& b1,
                                                float& b2) {
  float fx = (x - H.x0) / H.dx, fy = (y - H.y0) / H.dy;
  if (!(fx >= 0.0f && fy >= 0.0f && fx <= (float)(H.nx - 1) && fy <= (float)(H.ny - 1))) return false;
  int i = min((int)fx, H.nx - 2), j = min((int)fy, H.ny - 2);
  float u = fx - (float)i, w = fy - (float)j;
  int quad = j * (H.nx - 1) + i;
  if (u >= w) { prim = 2 * quad; b1 = u - w; b2 = w; }
  else { prim = 2 * quad + 1; b1 = u; b2 = w - u; }
  int v0, v1, v2;
  hf_tri(H, prim, v0, v1, v2);
  float3 P0 = f3(__ldg(H.P + v0)), P1 = f3(__ldg(H.P + v1)), P2 = f3(__ldg(H.P + v2));
  p = P0 + (P1 - P0) * b1 + (P2 - P0) * b2;
  return true;
}

// Reprojection of a moved vertex onto its own surface by a ray cast along the
// surface's projection direction: from the centre (spheres and caps), along
// the normal (rectangles), vertically (heightfields).
__device__ __forceinline__ bool reproject(const DScene& S, int surf, float3 target, float3& p, int& prim, float& b1,
                                          float& b2) {
  const DSurf& sf = S.s[surf];
  if (sf.type == SURF_SPHERE || sf.type == SURF_CAP) {
    float3 d = target - sf.c;
    float l2 = dot(d, d);
    if (!(l2 > 0.0f)) return false;
    p = sf.c + d * (sf.r / sqrtf(l2));
    return sf.type == SURF_SPHERE || dot(p - sf.c, sf.axis) >= sf.r * sf.cap_cos;
  }
  if (sf.type == SURF_RECT) {
    p = target - sf.axis * dot(target - sf.c, sf.axis);
    float3 q = p - sf.c;
    return fabsf(dot(q, sf.ex)) <= sf.ex2 && fabsf(dot(q, sf.ey)) <= sf.ey2;
  }
  return hf_vertical_hit(S.hf[sf.hf], target.x, target.y, p, prim, b1, b2);
}

// Newton step of every vertex as a 3-D tangent vector dpdu du_0 + dpdv du_1.
template <int K>
__device__ __forceinline__ void step_vectors(const float3 (&tu)[K], const float3 (&tv)[K], const float2 (&du)[K][1],
                                             float3 (&d)[K]) {
#pragma unroll
  for (int i = 0; i < K; ++i) d[i] = tu[i] * du[i][0].x + tv[i] * du[i][0].y;
}

// Move every vertex by beta d_i in its tangent plane and reproject it onto its
// surface; chain visibility is checked once converged.
template <int K>
__device__ __forceinline__ bool propose(const DScene& S, const Chain<K>& ch, const float3 (&d)[K], float beta,
                                        Chain<K>& out) {
#pragma unroll
  for (int i = 0; i < K; ++i) {
    float3 target = ch.x[i] + d[i] * beta;
    out.surf[i] = ch.surf[i];
    out.prim[i] = ch.prim[i];
    out.b1[i] = ch.b1[i];
    out.b2[i] = ch.b2[i];
    if (!reproject(S, ch.surf[i], target, out.x[i], out.prim[i], out.b1[i], out.b2[i])) return false;
  }
  return true;
}

// Newton manifold walk of one chain.  Returns the chain status; `iters` gets
// the number of Newton steps taken.
template <int K, bool kStats>
__device__ int walk(const DScene& S, Chain<K>& ch, const Ends& e, const mpg_params& P, int& iters, int* err,
                    Counters& cnt, const float2* off = nullptr) {
  VB vb[K];
  float3 tu[K], tv[K];
  float cn2, cmax;
  for (int it = 0;; ++it) {
    iters = it;
    if (!eval_full<K, kStats>(S, ch, e, vb, tu, tv, cn2, cmax, false, cnt, off)) return ST_FAILED;
    if (cmax < P.tol) return ST_CONVERGED;
    if (it >= P.max_iter) return cmax < P.stall_tol ? ST_CONVERGED : ST_LIMIT;
    float2 du[K][1];
#pragma unroll
    for (int i = 0; i < K; ++i) du[i][0] = make_float2(-vb[i].C.x, -vb[i].C.y);
    if (kStats) { cnt.newton++; cnt.rows += K; }
    if (!thomas<K, 1>(vb, du, P.sing_eps)) return ST_FAILED;
    float3 dstep[K];
    step_vectors<K>(tu, tv, du, dstep);
    float beta = 1.0f;
    bool accepted = false;
    for (int hv = 0; hv <= P.max_halvings; ++hv, beta *= 0.5f) {
      Chain<K> cand;
      if (!propose<K>(S, ch, dstep, beta, cand)) continue;
      float cc2;
      if (eval_c<K, kStats>(S, cand, e, cc2, cnt, off) && cc2 < cn2) {
        ch = cand;
        accepted = true;
        break;
      }
    }
    // FP32 resolution: C cannot be evaluated much below ~1e-6 at unit scene
    // scale, so a step that no longer lowers |C| ends a walk already within
    // stall_tol as converged.
    if (!accepted) return cmax < P.stall_tol ? ST_CONVERGED : ST_FAILED;
  }
}

// ---------------------------------------------------------------------------
// Seeds (Eq. deduction; p_0 of Sec. 5.4; guided mixture of Sec. 5.5)
// ---------------------------------------------------------------------------
// Scattered propagation direction (mirror reflection or Snell refraction).
__device__ __forceinline__ bool scatter(const DSurf& sf, float3 n, float3 d, bool refract, float3& out) {
  if (!refract) {
    out = d - n * (2.0f * dot(d, n));
    return true;
  }
  if (sf.mat == MAT_MIRROR) return false;
  float ci = -dot(d, n);
  float e1 = sf.etaF, e2 = sf.etaB;
  float3 nn = n;
  if (ci < 0.0f) { ci = -ci; e1 = sf.etaB; e2 = sf.etaF; nn = -n; }
  float eta = e1 / e2;
  float k2 = 1.0f - eta * eta * (1.0f - ci * ci);
  if (k2 < 0.0f) return false;
  out = unit(d * eta + nn * (eta * ci - sqrtf(k2)));
  return true;
}

// Bin of a direction: the theta bin counts the FP32 edges cos(theta_j) above
// w.z; the phi bin counts, within the half plane of w, the edge vectors
// (c_j, s_j) that w is counter-clockwise of, by the exact FP64 sign of
// c_j y - s_j x (a product of two FP32 values is exact in FP64).  Both
// predicates are monotone in j, so each count is a binary search.
// Exact sign test c y - s x >= 0 for FP32 inputs.  The FP32 products p1, p2
// are within max(|p1|,|p2|) 2^-24 + 2^-150 of the exact ones and the rounded
// difference d within |d| 2^-24 of p1 - p2, so when |d| exceeds
// max(|p1|,|p2|) 2^-21 + 2^-126 its sign is the sign of the exact value.
// Otherwise (near ties, rare) the products are formed in FP64, where a product
// of two FP32 values is exact and the one rounding of the difference keeps its
// sign.  Either way the result is the exact predicate, the same on every
// machine.
// The FP64 form is a separate, non-inlined call so that the compiler cannot
// turn the rare branch into straight-line code executed for every test.
static __device__ __noinline__ bool ccw_or_on_fp64(float c, float s, float x, float y) {
  return __dsub_rn(__dmul_rn((double)c, (double)y), __dmul_rn((double)s, (double)x)) >= 0.0;
}
__device__ __forceinline__ bool ccw_or_on(float c, float s, float x, float y) {
  float p1 = __fmul_rn(c, y), p2 = __fmul_rn(s, x);
  float d = __fsub_rn(p1, p2);
  float m = fmaxf(fabsf(p1), fabsf(p2));
  if (fabsf(d) > __fmaf_rn(m, 0x1p-21f, 0x1p-126f)) return d >= 0.0f;
  return ccw_or_on_fp64(c, s, x, y);
}

__device__ __forceinline__ int guide_bin(const DGuide& g, float3 w) {
  int lo = 1, hi = g.n_theta;  // count of j in [1, n_theta) with w.z < cos_theta[j]
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (w.z < __ldg(g.cos_theta + mid)) lo = mid + 1; else hi = mid;
  }
  int it = lo - 1;
  bool upper = (w.y > 0.0f) || (w.y == 0.0f && w.x >= 0.0f);
  int half = g.n_phi >> 1;
  int j0 = upper ? 1 : half + 1, j1 = upper ? half : g.n_phi;
  int a = j0, b = j1;  // first j in [j0, j1) where w is no longer counter-clockwise of edge j
  while (a < b) {
    int mid = (a + b) >> 1;
    if (ccw_or_on(__ldg(g.phi_cos + mid), __ldg(g.phi_sin + mid), w.x, w.y)) a = mid + 1; else b = mid;
  }
  int ip = (upper ? 0 : half) + (a - j0);
  return it * g.n_phi + ip;
}

// Solid-angle density of p_0 at direction w from x_D.
__device__ __forceinline__ float p0_pdf(const DScene& S, float3 xD, float3 w) {
  float sum = 0.0f;
  for (int i = 0; i < S.n_tg; ++i) {
    const DTarget& tg = S.tg[i];
    if (tg.type == TARGET_SPHERE) {
      float d = len(xD - tg.c);
      if (d <= tg.r) continue;
      float t0, t1;
      if (!sphere_roots(xD, w, tg.c, tg.r, t0, t1) || t0 <= 0.0f) continue;
      // at the near hit (p - c).w = b + t0 = -sqrt(disc): the cosine is sqrt(disc)/r,
      // well conditioned at grazing incidence where 1/cos makes the density steep
      float3 oc = xD - tg.c;
      float3 qd = oc - w * dot(oc, w);
      float cp = sqrtf(fmaxf(fmaf(tg.r, tg.r, -dot(qd, qd)), 0.0f)) / tg.r;
      float pA = 1.0f / (6.28318530717958647f * tg.r * tg.r * (1.0f - tg.r / d));
      sum += pA * t0 * t0 / cp;
    } else {
      float den = dot(w, tg.n);
      if (fabsf(den) < 1e-30f) continue;
      float t = dot(tg.c - xD, tg.n) / den;
      if (t <= 0.0f) continue;
      float3 q = xD + w * t - tg.c;
      if (fabsf(dot(q, tg.ex)) > dot(tg.ex, tg.ex) || fabsf(dot(q, tg.ey)) > dot(tg.ey, tg.ey)) continue;
      sum += t * t / (tg.area * fabsf(den));
    }
  }
  return S.n_tg > 0 ? sum / (float)S.n_tg : 0.0f;
}

// floor(r * total / 2^32) in exact integer arithmetic.
__device__ __forceinline__ uint64_t scaled_target(uint32_t r, uint64_t total) {
  uint64_t lo = (uint64_t)r * total, hi = __umul64hi((uint64_t)r, total);
  return (hi << 32) | (lo >> 32);
}

__device__ __forceinline__ uint64_t ldg64(const uint64_t* p) {
  return __ldg(reinterpret_cast<const unsigned long long*>(p));
}

// ---------------------------------------------------------------------------
// vMF mixture guide (Sec. 5.5, Eq. vMF).  The lobes of a cell are contiguous
// and ordered by key (n << 8) | tau, so the lobes of one length, or of one
// length and type, are a sub-range found by binary search; the cell-local
// prefix sums of the integer weights make every discrete choice exact.
// ---------------------------------------------------------------------------
// Uniform in (0, 1]: the 24-bit draw of u01 shifted up by one step.
__device__ __forceinline__ float u01c(uint32_t r) { return (float)((r >> 8) + 1u) * (1.0f / 16777216.0f); }

// First lobe in [a, b) whose key is >= key.
__device__ __forceinline__ uint32_t lobe_bound(const DGuide& g, uint32_t a, uint32_t b, uint32_t key) {
  while (a < b) {
    uint32_t m = (a + b) >> 1;
    if (__ldg(g.lobe_key + m) < key) a = m + 1; else b = m;
  }
  return a;
}

// Weight of the lobes of the cell before lobe i.
__device__ __forceinline__ uint64_t lobe_cum(const DGuide& g, uint32_t cs, uint32_t i) {
  return i > cs ? ldg64(g.lobe_prefix + i - 1) : 0ull;
}

// Lobes of a cell with klo <= key < khi: [a, b), the weight before a, and the range's weight.
struct VmfRange {
  uint32_t cs, a, b;
  uint64_t base, total;
};
static __device__ __noinline__ VmfRange vmf_range(const DGuide& g, uint32_t cell, uint32_t klo, uint32_t khi) {
  VmfRange r;
  r.cs = __ldg(g.cell_start + cell);
  uint32_t ce = __ldg(g.cell_start + cell + 1);
  r.a = lobe_bound(g, r.cs, ce, klo);
  r.b = lobe_bound(g, r.a, ce, khi);
  r.base = lobe_cum(g, r.cs, r.a);
  r.total = lobe_cum(g, r.cs, r.b) - r.base;
  return r;
}

// The bin of an inverse-CDF draw: the smallest i in [0, n) with
// cdf[i] - base > target (cdf non-decreasing, target < cdf[n - 1] - base).  Eight-way search: each round loads
// seven pivots at once, so a draw over 4,096 bins waits on four rounds of
// loads instead of the twelve dependent loads of a binary search (inside the
// walk kernels a drawing lane stalls its whole warp for that wait).  The
// result is the binary search's.
__device__ __forceinline__ int cdf_search(const uint64_t* cdf, int n, uint64_t target, uint64_t base = 0) {
  int lo = 0;
  while (n > 1) {
    const int step = (n + 7) >> 3;
    int j = 0;
#pragma unroll
    for (int q = 1; q < 8; ++q) {
      const int m = lo + q * step;  // first index of part q
      if (m < lo + n && __ldg(reinterpret_cast<const unsigned long long*>(cdf + m - 1)) - base <= target) j = q;
    }
    lo += j * step;
    n = min(step, n - j * step);
  }
  return lo;
}

// The vMF guide's pieces of a seed draw (vmf_range, vmf_search, vmf_sample,
// vmf_mix_pdf) are kept out of line, like the BVH traversal: they run only
// with a vMF guide, and inlined they enlarge every kernel that draws seeds.
// The lobe whose weight interval holds target: first i in [a, b) whose
// prefix sum exceeds base + target (total > 0, target < total).
static __device__ __noinline__ uint32_t vmf_search(const DGuide& g, const VmfRange& r, uint64_t target) {
  return r.a + (uint32_t)cdf_search(g.lobe_prefix + r.a, (int)(r.b - r.a), target, r.base);
}

// Draw from the lobe (mu, kappa): t = 1 - mu.w has density
// kappa e^{-kappa t} / (1 - e^{-2 kappa}) on [0, 2], inverted with u1 in
// (0, 1]; the azimuth 2 pi u2 is taken in the Duff et al. frame of mu.
static __device__ __noinline__ float3 vmf_sample(float4 L, float u1, float u2) {
  float3 mu = make_float3(L.x, L.y, L.z);
  float t = -logf(fmaf(1.0f - u1, expf(-2.0f * L.w), u1)) / L.w;
  t = fminf(fmaxf(t, 0.0f), 2.0f);
  float ct = 1.0f - t, st = sqrtf(fmaxf(0.0f, t * (2.0f - t)));
  float3 e1, e2;
  onb(mu, e1, e2);
  float sp, cp;
  sincospif(2.0f * u2, &sp, &cp);
  return mu * ct + (e1 * cp + e2 * sp) * st;
}

// Mixture density of the lobes of key kt within the range r, weights q_i / total.
// The lobe density (Eq. vMF) kappa / (4 pi sinh kappa) e^{kappa mu.w} is written
// kappa / (2 pi (1 - e^{-2 kappa})) e^{-kappa |w - mu|^2 / 2} (|w - mu|^2 / 2 =
// 1 - mu.w for unit vectors, without its cancellation), so the sum is
// sum_i coef_i e^{-kappa_i |w - mu_i|^2 / 2} / total with the lobe factors
// coef_i = q_i kappa_i / (2 pi (1 - e^{-2 kappa_i})) formed once by the build.
static __device__ __noinline__ float vmf_mix_pdf(const DGuide& g, VmfRange r, uint32_t kt, float3 w) {
  uint32_t a = lobe_bound(g, r.a, r.b, kt), b = lobe_bound(g, a, r.b, kt + 1);
  float sum = 0.0f;
  for (uint32_t i = a; i < b; ++i) {
    float4 L = __ldg(g.lobe + i);
    float3 d = w - make_float3(L.x, L.y, L.z);
    sum = fmaf(__ldg(g.lobe_coef + i), expf(-0.5f * L.w * dot(d, d)), sum);
  }
  return sum / (float)r.total;
}

// The vMF part of a seed's density left to the caller: the lobes of group kt
// in range vr, evaluated at w (summed by a whole warp, vmf_sum_warp).
struct VmfDeferred {
  bool need;
  VmfRange vr;
  uint32_t kt;
  float3 w;
};

// Sum over the lobes of each lane's group at its direction, for the lanes
// with `need`, taken by the whole warp one lane at a time: consecutive lanes
// read consecutive lobes (coalesced 16-byte loads) and a butterfly reduction
// adds the partial sums.  Every lane of the warp must call it; returns the
// lane's sum divided by the cell's total weight (0 without `need`).
__device__ __forceinline__ float vmf_sum_warp(const DGuide& g, bool need, const VmfDeferred& d) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  uint32_t a = 0, b = 0;
  if (need) {
    a = lobe_bound(g, d.vr.a, d.vr.b, d.kt);
    b = lobe_bound(g, a, d.vr.b, d.kt + 1);
  }
  float mine = 0.0f;
  unsigned m = __ballot_sync(FULL, need);
  while (m) {
    const int src = __ffs(m) - 1;
    m &= m - 1;
    const uint32_t sa = __shfl_sync(FULL, a, src), sb = __shfl_sync(FULL, b, src);
    const float3 w = make_float3(__shfl_sync(FULL, d.w.x, src), __shfl_sync(FULL, d.w.y, src),
                                 __shfl_sync(FULL, d.w.z, src));
    float part = 0.0f;
    for (uint32_t i = sa + (uint32_t)lane; i < sb; i += 32u) {
      const float4 L = __ldg(g.lobe + i);
      const float3 dv = w - make_float3(L.x, L.y, L.z);
      part = fmaf(__ldg(g.lobe_coef + i), expf(-0.5f * L.w * dot(dv, dv)), part);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
    if (lane == src) mine = part;
  }
  return need ? mine / (float)d.vr.total : 0.0f;
}

// First part of a seed draw for a chain of K vertices (K at run time): the
// mixture component, the types tau and the direction w from x_D with its
// density pdf; false when the draw fails before any ray is cast.  tau_out is
// set on every path (the guided vMF component may replace the drawn types).
template <bool kStats>
__device__ __forceinline__ bool draw_dir(const DScene& S, const DGuide* g, const Ends& e, uint32_t cell,
                                         uint32_t tau_in, bool tau_random, uint2 key, uint64_t idx, uint32_t trial,
                                         const mpg_params& P, int K, float3& w, uint32_t& tau_out, float& pdf,
                                         int* err, Counters& cnt, bool want_pdf, bool need_tau_in,
                                         VmfDeferred* defer) {
  if (kStats) cnt.seeds++;
  uint4 r1 = philox(make_uint4((uint32_t)idx, (uint32_t)(idx >> 32), trial, 1u), key);
  uint32_t tau = tau_random ? (r1.y & ((1u << K) - 1u)) : tau_in;
  tau_out = tau;  // the guided vMF component may replace it below
  const bool vmf = g != nullptr && g->kind == MPG_GUIDE_VMF;
  if (!vmf) {
    // a Bernoulli trial must sample the chain's own types: when it drew others it
    // has failed already, before any ray is cast
    if (need_tau_in && tau != tau_in) return false;
  }
  uint4 r0 = philox(make_uint4((uint32_t)idx, (uint32_t)(idx >> 32), trial, 0u), key);
  uint64_t total = 0;
  bool use_guide = g != nullptr;
  const uint64_t* cdf = nullptr;
  VmfRange vr = {};
  if (use_guide && cell >= (uint32_t)g->n_cells) {  // bad cell index: flag it, sample p_0 only
    atomicOr(err, 2);
    use_guide = false;
  }
  if (use_guide && vmf) {
    // selective activation: a cell without any lobe is not sampled at all
    if (P.selective && __ldg(g->cell_start + cell) == __ldg(g->cell_start + cell + 1)) return false;
    // the guided component draws (w, tau) given n, or w given n and tau when
    // the types are fixed
    uint32_t klo = ((uint32_t)K << 8) | (tau_random ? 0u : tau_in);
    uint32_t khi = tau_random ? ((uint32_t)(K + 1) << 8) : klo + 1;
    vr = vmf_range(*g, cell, klo, khi);
    total = vr.total;
    use_guide = total > 0;
  } else if (use_guide) {
    cdf = g->cdf + (size_t)cell * g->bins;
    total = __ldg(reinterpret_cast<const unsigned long long*>(cdf + g->bins - 1));
    use_guide = total > 0;
    if (P.selective && !use_guide) return false;  // selective activation: an empty cell is not sampled
  }
  bool pick_p0 = !use_guide || u01(r0.x) < P.alpha;
  uint32_t li = 0;
  if (vmf) {
    if (!pick_p0) {
      li = vmf_search(*g, vr, scaled_target(r0.y, total));
      tau = __ldg(g->lobe_key + li) & 255u;
    }
    tau_out = tau;
    if (need_tau_in && tau != tau_in) return false;
  }
  if (!pick_p0 && vmf) {
    w = vmf_sample(__ldg(g->lobe + li), u01c(r0.z), u01(r0.w));
  } else if (pick_p0) {
    if (S.n_tg == 0) return false;
    int ti = min((int)(u01(r1.x) * (float)S.n_tg), S.n_tg - 1);
    const DTarget& tg = S.tg[ti];
    float u1 = u01(r0.z), u2 = u01(r0.w);
    float3 p;
    if (tg.type == TARGET_SPHERE) {
      float3 ax = e.xD - tg.c;
      float d = len(ax);
      if (d <= tg.r) return false;
      ax = ax * (1.0f / d);
      float3 e1, e2;
      onb(ax, e1, e2);
      float ca = tg.r / d + u1 * (1.0f - tg.r / d);
      float sa = sqrtf(fmaxf(0.0f, 1.0f - ca * ca));
      float sp, cp;
      sincospif(2.0f * u2, &sp, &cp);
      p = tg.c + (ax * ca + (e1 * cp + e2 * sp) * sa) * tg.r;
    } else {
      p = tg.c + tg.ex * (2.0f * u1 - 1.0f) + tg.ey * (2.0f * u2 - 1.0f);
    }
    w = unit(p - e.xD);
  } else {
    // inverse CDF on exact integers: target = floor(r * total / 2^32)
    uint64_t r = r0.y;
    uint64_t lo = r * total, hi = __umul64hi(r, total);
    uint64_t target = (hi << 32) | (lo >> 32);
    const int a = cdf_search(cdf, g->bins, target);
    int it = a / g->n_phi, ip = a % g->n_phi;
    float clo = __ldg(g->cos_theta + it), chi = __ldg(g->cos_theta + it + 1);
    float ct = clo + u01(r0.z) * (chi - clo);
    float st = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
    float sp, cp;
    sincospif(2.0f * ((float)ip + u01(r0.w)) / (float)g->n_phi, &sp, &cp);
    w = make_float3(st * cp, st * sp, ct);
  }
  if (dot(w, e.nD) <= 0.0f) return false;
  pdf = 0.0f;
  if (!want_pdf) {
  } else if (vmf) {
    // joint density of (w, tau) given n: p_0 draws the types uniformly
    float p0 = p0_pdf(S, e.xD, w);
    if (tau_random) p0 = ldexpf(p0, -K);
    if (defer && use_guide) {
      defer->need = true;
      defer->vr = vr;
      defer->kt = ((uint32_t)K << 8) | tau;
      defer->w = w;
      pdf = P.alpha * p0;
    } else {
      pdf = use_guide ? P.alpha * p0 + (1.0f - P.alpha) * vmf_mix_pdf(*g, vr, ((uint32_t)K << 8) | tau, w) : p0;
    }
  } else if (use_guide) {
    float p0 = p0_pdf(S, e.xD, w);
    int bin = guide_bin(*g, w);
    uint64_t cnt_b = __ldg(reinterpret_cast<const unsigned long long*>(g->counts + (size_t)cell * g->bins + bin));
    int it = bin / g->n_phi;
    float dcos = __ldg(g->cos_theta + it) - __ldg(g->cos_theta + it + 1);
    float ph = ((float)cnt_b / (float)total) / ((6.28318530717958647f / (float)g->n_phi) * dcos);
    pdf = P.alpha * p0 + (1.0f - P.alpha) * ph;
  } else {
    pdf = p0_pdf(S, e.xD, w);
  }
  return true;
}

// Draw seed `trial` of chain idx and deduce its vertices (Eq. deduction).
// Returns validity; fills ch (first K vertices), tau and pdf.  With `defer`
// (vMF guide), the sum over the lobes is not formed here: pdf gets the p_0
// part alone and defer what the caller needs to add (1 - alpha)
// vmf_sum_warp(...) to it.
template <int K, bool kStats, int kBVH = BVH_CALL>
__device__ bool draw_seed(const DScene& S, const DGuide* g, const Ends& e, uint32_t cell, uint32_t tau_in,
                          bool tau_random, uint2 key, uint64_t idx, uint32_t trial, const mpg_params& P,
                          Chain<K>& ch, uint32_t& tau_out, float& pdf, int* err, Counters& cnt,
                          bool want_pdf = true, bool need_tau_in = false, VmfDeferred* defer = nullptr) {
  float3 w;
  if (!draw_dir<kStats>(S, g, e, cell, tau_in, tau_random, key, idx, trial, P, K, w, tau_out, pdf, err, cnt, want_pdf,
                        need_tau_in, defer))
    return false;
  const uint32_t tau = tau_out;
  float3 o = e.xD, d = w;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    Hit h = intersect<kStats, kBVH>(S, o, d, P.ray_eps, 3.0e38f, err, cnt);
    if (h.surf < 0) return false;
    ch.x[i] = hit_point(S, o, d, h);
    ch.surf[i] = h.surf;
    ch.prim[i] = h.prim;
    ch.b1[i] = h.b1;
    ch.b2[i] = h.b2;
    if (i < K - 1) {
      float3 n = vertex_normal(S, h.surf, h.prim, ch.x[i], h.b1, h.b2);
      float3 dn;
      if (!scatter(S.s[h.surf], n, d, (tau >> i) & 1u, dn)) return false;
      o = ch.x[i];
      d = dn;
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// Contribution (Eq. ThroughputEval)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float fresnel(float c1, float e1, float e2) {
  float r = e1 / e2;
  float s2 = r * r * (1.0f - c1 * c1);
  if (s2 >= 1.0f) return 1.0f;
  float c2 = sqrtf(1.0f - s2);
  float rs = (e1 * c1 - e2 * c2) / (e1 * c1 + e2 * c2);
  float rp = (e2 * c1 - e1 * c2) / (e2 * c1 + e1 * c2);
  return 0.5f * (rs * rs + rp * rp);
}

template <bool kStats>
__device__ __forceinline__ bool segment_clear(const DScene& S, float3 a, float3 b, float eps, int* err, Counters& cnt) {
  float3 d = b - a;
  float l = len(d);
  if (!(l > 2.0f * eps)) return true;
  Hit h = intersect<kStats>(S, a, d * (1.0f / l), eps, l - eps, err, cnt);
  return h.surf < 0;
}

// Admissibility of a converged chain: every vertex type matches the sides of
// its neighbours (refraction crosses the surface, reflection stays on one
// side), the receiver and an area light face the chain, and every segment is
// unoccluded.
template <int K, bool kStats>
__device__ __forceinline__ bool admissible(const DScene& S, const Chain<K>& ch, const Ends& e, const mpg_params& P,
                                           int* err, Counters& cnt) {
#pragma unroll
  for (int i = 0; i < K; ++i) {
    float3 xp = i == 0 ? e.xD : ch.x[i - 1];
    float3 xn = i == K - 1 ? e.xL : ch.x[i + 1];
    float3 n = vertex_normal(S, ch.surf[i], ch.prim[i], ch.x[i], ch.b1[i], ch.b2[i]);
    float si = dot(xp - ch.x[i], n), so = dot(xn - ch.x[i], n);
    bool refract = (e.tau >> i) & 1u;
    if (refract ? !(si * so < 0.0f) : !(si * so > 0.0f)) return false;
  }
  float3 wD = unit(ch.x[0] - e.xD);
  if (!(dot(e.nD, wD) > 0.0f)) return false;
  float3 wL = unit(ch.x[K - 1] - e.xL);
  if (S.L.type != LIGHT_POINT && !(dot(S.L.n, wL) > 0.0f)) return false;
  if (!segment_clear<kStats>(S, e.xD, ch.x[0], P.ray_eps, err, cnt)) return false;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    float3 b = i == K - 1 ? e.xL : ch.x[i + 1];
    if (!segment_clear<kStats>(S, ch.x[i], b, P.ray_eps, err, cnt)) return false;
  }
  return true;
}

// Admissibility, G (implicit function theorem) and kappa in FP32.  G is
// formed twice from one Thomas sweep (with the remaining Newton step as a
// fifth column): X_L = cos_D |det d(w_D)/d(u_L)| (light end moved) and
// X_D = |det d(w_L)/d(u_D)| (receiver moved).  By reciprocity
// eta_D^2 X_L = eta_L^2 |n_L.w_L| X_D, so their relative mismatch estimates
// the FP32 error of G (out: mismatch; on heightfield chains the determinant's
// conditioning instead, see below); cmax (out) is the chain's FP32 residual.
// Returns false for an inadmissible chain.
template <int K, bool kStats>
__device__ bool contribution(const DScene& S, const Chain<K>& ch, const Ends& e, const mpg_params& P, float& G,
                             float& kappa, float& mismatch, float& cmax, float& kappa_err, float& step_err, int* err,
                             Counters& cnt) {
  VB vb[K];
  float3 tu[K], tv[K];
  float cn2;
  if (!eval_full<K, kStats>(S, ch, e, vb, tu, tv, cn2, cmax, true, cnt)) return false;
  if (!admissible<K, kStats>(S, ch, e, P, err, cnt)) return false;
  float3 wD = unit(ch.x[0] - e.xD);
  float cosD = dot(e.nD, wD);
  bool point = S.L.type == LIGHT_POINT;
  float3 wL = unit(ch.x[K - 1] - e.xL);
  // J Y = -dC/du_end: columns 0,1 light end (block row K-1), 2,3 receiver end
  // (row 0); column 4 the Newton step -J^-1 C the chain is still away from the
  // solution (its size bounds the error of the converged vertices).
  float2 Y[K][5];
#pragma unroll
  for (int i = 0; i < K; ++i) {
#pragma unroll
    for (int c = 0; c < 4; ++c) Y[i][c] = make_float2(0.f, 0.f);
    Y[i][4] = make_float2(-vb[i].C.x, -vb[i].C.y);
  }
  Y[K - 1][0] = make_float2(-vb[K - 1].Cc.x, -vb[K - 1].Cc.z);
  Y[K - 1][1] = make_float2(-vb[K - 1].Cc.y, -vb[K - 1].Cc.w);
  Y[0][2] = make_float2(-vb[0].A.x, -vb[0].A.z);
  Y[0][3] = make_float2(-vb[0].A.y, -vb[0].A.w);
  if (kStats) cnt.ggt += 2 * K;
  if (!thomas<K, 5>(vb, Y, P.sing_eps)) return false;
  // direction error of the converged chain: the largest remaining vertex
  // displacement over the shortest segment
  float dx2 = 0.0f, dmin = len(ch.x[0] - e.xD);
#pragma unroll
  for (int i = 0; i < K; ++i) {
    float3 d = tu[i] * Y[i][4].x + tv[i] * Y[i][4].y;
    dx2 = fmaxf(dx2, dot(d, d));
    dmin = fminf(dmin, len((i == K - 1 ? e.xL : ch.x[i + 1]) - ch.x[i]));
  }
  const float dir_err = 2.0f * sqrtf(dx2) / fmaxf(dmin, 1e-30f);
  float X[2], cond[2];
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    int vi = side == 0 ? 0 : K - 1;
    float3 w = side == 0 ? ch.x[0] - e.xD : ch.x[K - 1] - e.xL;
    float dist = len(w);
    w = w * (1.0f / dist);
    float3 a, b;
    onb(w, a, b);
    float M[2][2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      float2 y = Y[vi][2 * side + c];
      float3 dx = tu[vi] * y.x + tv[vi] * y.y;
      float3 dw = (dx - w * dot(w, dx)) * (1.0f / dist);
      M[0][c] = dot(a, dw);
      M[1][c] = dot(b, dw);
    }
    X[side] = fabsf(M[0][0] * M[1][1] - M[0][1] * M[1][0]);
    cond[side] = (fabsf(M[0][0] * M[1][1]) + fabsf(M[0][1] * M[1][0])) / fmaxf(X[side], 1e-30f);
  }
  float XL = cosD * X[0], XD = X[1];
  float3 nl = point ? cross(S.L.exu, S.L.eyu) : S.L.n;
  float etaD = vb[0].ei, etaL = vb[K - 1].eo;
  float rc = (etaL * etaL) / (etaD * etaD) * fabsf(dot(nl, wL));
  float XDs = rc * XD;
  mismatch = fabsf(XL - XDs) / fmaxf(fmaxf(XL, XDs), 1e-30f);
  G = point ? XD : XL;
  // With interpolated shading normals (heightfield vertices) the normal field
  // is not the surface's, the two ends' terms are not reciprocal, and their
  // mismatch (1e-4 to 1e-3 on the water scene) measures the interpolation
  // rather than rounding.  There the estimate is the cancellation in the
  // determinant instead: entries good to about 1e-6 relative after the
  // solve, times (|m00 m11| + |m01 m10|) / |det m|.
  bool shading = false;
#pragma unroll
  for (int i = 0; i < K; ++i) shading = shading || S.s[ch.surf[i]].type == SURF_HEIGHTFIELD;
  if (shading) mismatch = 1e-6f * cond[point ? 1 : 0];
  // kappa: mirror 1; dielectric R -> F, T -> (1 - F)(eta_i/eta_o)^2 under an
  // area light, T -> (1 - F) under a point light (G maps the intensity's solid
  // angle onto receiver area, so flux carries no radiance scaling).  The
  // transmittance is formed directly, (1 - F) = (T_s + T_p)/2 with
  // T_s = 4 n1 n2 c1 c2/(n1 c1 + n2 c2)^2 and T_p = 4 n1 n2 c1 c2/(n2 c1 + n1 c2)^2,
  // c2 the refracted cosine of the converged chain: 1 - F would cancel in FP32
  // near total internal reflection.
  // kappa_err, step_err (out): relative error estimates of the
  // transmittances, which scale like the smaller cosine at grazing incidence
  // or exit.  The cosines come from the chain's own unit directions: their
  // FP32 rounding (~1e-7) gives kappa_err; the remaining Newton step over the
  // shortest segment (dir_err: near grazing a residual C below the tolerance
  // can still leave the vertices off the solution) gives step_err, a bound
  // rather than an estimate (the largest vertex step, over the shortest
  // segment, doubled).
  float kap = 1.0f;
  kappa_err = 0.0f;
  step_err = 0.0f;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const DSurf& sf = S.s[ch.surf[i]];
    if (sf.mat == MAT_MIRROR) continue;
    float3 xp = i == 0 ? e.xD : ch.x[i - 1];
    float3 xn = i == K - 1 ? e.xL : ch.x[i + 1];
    float3 n = vertex_normal(S, ch.surf[i], ch.prim[i], ch.x[i], ch.b1[i], ch.b2[i]);
    float ci = fabsf(dot(unit(xp - ch.x[i]), n));
    if ((e.tau >> i) & 1u) {
      float n1 = vb[i].ei, n2 = vb[i].eo;
      float co = fabsf(dot(unit(xn - ch.x[i]), n));
      float num = 4.0f * n1 * n2 * ci * co;
      float ds = n1 * ci + n2 * co, dp = n2 * ci + n1 * co;
      float Tr = 0.5f * (num / (ds * ds) + num / (dp * dp));
      float r = point ? 1.0f : n1 / n2;
      kap *= Tr * r * r;
      const float ic = 1.0f / fmaxf(fminf(ci, co), 1e-30f);
      kappa_err = fmaxf(kappa_err, 1.2e-7f * ic);
      step_err = fmaxf(step_err, dir_err * ic);
    } else {
      float e2 = vb[i].front ? sf.etaB : sf.etaF;
      kap *= fresnel(ci, vb[i].ei, e2);
    }
  }
  kappa = kap;
  return true;
}

// FP64 distance test of two converged chains (same types and surfaces).
template <int K>
__device__ __forceinline__ bool same_solution(const Chain<K>& a, const Chain<K>& b, double eps2) {
#pragma unroll
  for (int i = 0; i < K; ++i) {
    if (a.surf[i] != b.surf[i]) return false;
    double dx = (double)a.x[i].x - (double)b.x[i].x;
    double dy = (double)a.x[i].y - (double)b.x[i].y;
    double dz = (double)a.x[i].z - (double)b.x[i].z;
    if (!(dx * dx + dy * dy + dz * dz < eps2)) return false;
  }
  return true;
}

}  // namespace mpg
