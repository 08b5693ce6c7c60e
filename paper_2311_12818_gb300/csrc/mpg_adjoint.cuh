// Adjoint of the receiver irradiance with respect to heightfield heights (K7).
//
// For a converged chain with local coordinates u (two per vertex) and the
// heights theta of the grid vertices that move it, C(u*, theta) = 0 defines
// u*(theta) (implicit function theorem), so
//   dT/dtheta = dT/dtheta|_u - lambda^T dC/dtheta,   J^T lambda = (dT/du)^T,
// a transposed solve instead of differentiating through the Newton steps.
// The partial derivatives are taken in forward mode: the chain's constraint,
// geometry term and kappa are evaluated once more in dual numbers whose lanes
// carry the directions u_1..u_2K, theta_1..theta_m.
#pragma once

#include "mpg_device.cuh"

namespace mpg {
namespace adj {

// Directions carried per dual evaluation.  Two keep a chain's dual state in
// registers (at four the frames spilled: 346 MB of local-memory writes per
// launch on the water scene against 35 MB at two), at the price of more
// evaluations per chain.
constexpr int LANES = 2;

struct DF {
  float v;
  float d[LANES];
};
__device__ __forceinline__ DF cst(float x) {
  DF r;
  r.v = x;
#pragma unroll
  for (int i = 0; i < LANES; ++i) r.d[i] = 0.f;
  return r;
}
__device__ __forceinline__ DF operator+(const DF& a, const DF& b) {
  DF r; r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < LANES; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
__device__ __forceinline__ DF operator-(const DF& a, const DF& b) {
  DF r; r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < LANES; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
__device__ __forceinline__ DF operator-(const DF& a) {
  DF r; r.v = -a.v;
#pragma unroll
  for (int i = 0; i < LANES; ++i) r.d[i] = -a.d[i];
  return r;
}
__device__ __forceinline__ DF operator*(const DF& a, const DF& b) {
  DF r; r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < LANES; ++i) r.d[i] = fmaf(a.d[i], b.v, a.v * b.d[i]);
  return r;
}
__device__ __forceinline__ DF operator*(const DF& a, float s) {
  DF r; r.v = a.v * s;
#pragma unroll
  for (int i = 0; i < LANES; ++i) r.d[i] = a.d[i] * s;
  return r;
}
__device__ __forceinline__ DF operator/(const DF& a, const DF& b) {
  DF r; float ib = 1.0f / b.v; r.v = a.v * ib;
#pragma unroll
  for (int i = 0; i < LANES; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
__device__ __forceinline__ DF dsqrt(const DF& a) {
  DF r; r.v = sqrtf(a.v); float h = 0.5f / r.v;
#pragma unroll
  for (int i = 0; i < LANES; ++i) r.d[i] = a.d[i] * h;
  return r;
}
__device__ __forceinline__ DF dabs(const DF& a) { return a.v < 0.f ? -a : a; }

struct V {
  DF x, y, z;
};
__device__ __forceinline__ V vcst(float3 a) { return V{cst(a.x), cst(a.y), cst(a.z)}; }
__device__ __forceinline__ V operator+(const V& a, const V& b) { return V{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V operator-(const V& a, const V& b) { return V{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V operator-(const V& a) { return V{-a.x, -a.y, -a.z}; }
__device__ __forceinline__ V operator*(const V& a, const DF& s) { return V{a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ V operator*(const V& a, float s) { return V{a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ DF dot(const V& a, const V& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V cross(const V& a, const V& b) {
  return V{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ DF norm(const V& a) { return dsqrt(dot(a, a)); }
__device__ __forceinline__ V unitv(const V& a) {
  DF il = cst(1.0f) / norm(a);
  return a * il;
}

// Orthonormal basis completing n (same branchless rule as the walk).
__device__ __forceinline__ void onbv(const V& n, V& b1, V& b2) {
  float sg = n.z.v >= 0.0f ? 1.0f : -1.0f;
  DF s = cst(sg);
  DF a = cst(-1.0f) / (s + n.z);
  DF b = n.x * n.y * a;
  b1 = V{cst(1.0f) + s * n.x * n.x * a, s * b, -(s * n.x)};
  b2 = V{b, s + n.y * n.y * a, -n.y};
}

struct FrameD {
  V p, n, dpdu, dpdv, dndu, dndv;
};

// Same local geometry as vertex_frame for a heightfield triangle, in duals.
__device__ __forceinline__ FrameD frame_tri(const V& P0, const V& P1, const V& P2, const V& N0, const V& N1,
                                            const V& N2, const DF& b1, const DF& b2) {
  FrameD f;
  V e1 = P1 - P0, e2 = P2 - P0;
  f.p = P0 + e1 * b1 + e2 * b2;
  onbv(unitv(cross(e1, e2)), f.dpdu, f.dpdv);
  V Ns = N0 * (cst(1.0f) - b1 - b2) + N1 * b1 + N2 * b2;
  DF il = cst(1.0f) / norm(Ns);
  f.n = Ns * il;
  DF g11 = dot(e1, e1), g12 = dot(e1, e2), g22 = dot(e2, e2);
  DF igd = cst(1.0f) / (g11 * g22 - g12 * g12);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    V a = q == 0 ? f.dpdu : f.dpdv;
    DF r1 = dot(e1, a), r2 = dot(e2, a);
    DF db1 = (g22 * r1 - g12 * r2) * igd, db2 = (g11 * r2 - g12 * r1) * igd;
    V dN = (N1 - N0) * db1 + (N2 - N0) * db2;
    V dn = (dN - f.n * dot(f.n, dN)) * il;
    if (q == 0) f.dndu = dn; else f.dndv = dn;
  }
  return f;
}

struct VBD {
  DF C[2], A[4], B[4], Cc[4];
  float ei, eo;
  bool front;
};

__device__ __forceinline__ bool blocks(const FrameD& fp, const FrameD& f, const FrameD& fn, const DSurf& sf,
                                       bool refract, VBD& o) {
  V wi = fp.p - f.p, wo = fn.p - f.p;
  DF di = norm(wi), dO = norm(wo);
  DF idi = cst(1.0f) / di, ido = cst(1.0f) / dO;
  wi = wi * idi;
  wo = wo * ido;
  o.front = dot(wi, f.n).v > 0.0f;
  if (!etas(sf, o.front, refract, o.ei, o.eo)) return false;
  V ht = wi * o.ei + wo * o.eo;
  DF L = norm(ht);
  DF iL = cst(1.0f) / L;
  V h = ht * iL, s, t;
  onbv(f.n, s, t);
  o.C[0] = dot(h, s);
  o.C[1] = dot(h, t);
  DF hn = dot(h, f.n);
  V sp = (s - h * o.C[0]) * iL, tp = (t - h * o.C[1]) * iL;
  auto Pi = [&](const V& a) { return (a - wi * dot(wi, a)) * idi; };
  auto Po = [&](const V& a) { return (a - wo * dot(wo, a)) * ido; };
  V bu = -(Pi(f.dpdu) * o.ei + Po(f.dpdu) * o.eo), bv = -(Pi(f.dpdv) * o.ei + Po(f.dpdv) * o.eo);
  o.B[0] = dot(sp, bu) - hn * dot(s, f.dndu);
  o.B[1] = dot(sp, bv) - hn * dot(s, f.dndv);
  o.B[2] = dot(tp, bu) - hn * dot(t, f.dndu);
  o.B[3] = dot(tp, bv) - hn * dot(t, f.dndv);
  V au = Pi(fp.dpdu) * o.ei, av = Pi(fp.dpdv) * o.ei;
  o.A[0] = dot(sp, au); o.A[1] = dot(sp, av); o.A[2] = dot(tp, au); o.A[3] = dot(tp, av);
  V cu = Po(fn.dpdu) * o.eo, cv = Po(fn.dpdv) * o.eo;
  o.Cc[0] = dot(sp, cu); o.Cc[1] = dot(sp, cv); o.Cc[2] = dot(tp, cu); o.Cc[3] = dot(tp, cv);
  return true;
}

// Grid-vertex normal from heights (central differences, one-sided on the
// border), in duals; hgt(i, j) returns the seeded height.
template <class H>
__device__ __forceinline__ V grid_normal(const DHF& hf, int i, int j, H hgt) {
  DF dhdx, dhdy;
  if (i == 0) dhdx = (hgt(1, j) - hgt(0, j)) * (1.0f / hf.dx);
  else if (i == hf.nx - 1) dhdx = (hgt(hf.nx - 1, j) - hgt(hf.nx - 2, j)) * (1.0f / hf.dx);
  else dhdx = (hgt(i + 1, j) - hgt(i - 1, j)) * (0.5f / hf.dx);
  if (j == 0) dhdy = (hgt(i, 1) - hgt(i, 0)) * (1.0f / hf.dy);
  else if (j == hf.ny - 1) dhdy = (hgt(i, hf.ny - 1) - hgt(i, hf.ny - 2)) * (1.0f / hf.dy);
  else dhdy = (hgt(i, j + 1) - hgt(i, j - 1)) * (0.5f / hf.dy);
  return unitv(V{-dhdx, -dhdy, cst(1.0f)});
}

// T (value and lanes) and C of the chain for the direction chunk starting
// at dir0.  Directions: u of vertex i are 2i, 2i+1; height params[p] is 2K+p.
template <int K>
__device__ bool chain_eval(const DScene& S, const Chain<K>& ch, const Ends& e, const int* params, int m,
                           const float (&D)[K][4], int dir0, DF (&C)[2 * K], DF& T) {
  const DHF& hf = S.hf[S.s[ch.surf[0]].hf];
  auto lane_of = [&](int dir) { int l = dir - dir0; return (l >= 0 && l < LANES) ? l : -1; };
  auto hgt = [&](int i, int j) {
    int id = j * hf.nx + i;
    DF h = cst(__ldg(hf.P + id).z);
    for (int p = 0; p < m; ++p)
      if (params[p] == id) {
        const int l = lane_of(2 * K + p);
#pragma unroll
        for (int q = 0; q < LANES; ++q)  // a constant index keeps the dual in registers
          if (q == l) h.d[q] = 1.0f;
      }
    return h;
  };
  FrameD f[K + 2];
  float3 ru, rv;
  onb(e.nD, ru, rv);
  f[0].p = vcst(e.xD); f[0].n = vcst(e.nD); f[0].dpdu = vcst(ru); f[0].dpdv = vcst(rv);
  f[K + 1].p = vcst(e.xL); f[K + 1].n = vcst(S.L.n); f[K + 1].dpdu = vcst(S.L.exu); f[K + 1].dpdv = vcst(S.L.eyu);
#pragma unroll
  for (int i = 0; i < K; ++i) {
    int v[3];
    hf_tri(hf, ch.prim[i], v[0], v[1], v[2]);
    V P[3], N[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      int gi = v[c] % hf.nx, gj = v[c] / hf.nx;
      P[c] = V{cst(hf.x0 + gi * hf.dx), cst(hf.y0 + gj * hf.dy), hgt(gi, gj)};
      N[c] = grid_normal(hf, gi, gj, hgt);
    }
    DF u0 = cst(0.f), u1 = cst(0.f);
    int l0 = lane_of(2 * i), l1 = lane_of(2 * i + 1);
#pragma unroll
    for (int q = 0; q < LANES; ++q) {
      if (q == l0) u0.d[q] = 1.0f;
      if (q == l1) u1.d[q] = 1.0f;
    }
    DF b1 = cst(ch.b1[i]) + u0 * D[i][0] + u1 * D[i][1];
    DF b2 = cst(ch.b2[i]) + u0 * D[i][2] + u1 * D[i][3];
    f[i + 1] = frame_tri(P[0], P[1], P[2], N[0], N[1], N[2], b1, b2);
  }
  VBD vb[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    if (!blocks(f[i], f[i + 1], f[i + 2], S.s[ch.surf[i]], (e.tau >> i) & 1u, vb[i])) return false;
    C[2 * i] = vb[i].C[0];
    C[2 * i + 1] = vb[i].C[1];
  }
  // G (area light: light end moved; point light: receiver moved), 2-column Thomas in duals
  bool point = S.L.type == LIGHT_POINT;
  DF R[K][2][2];
#pragma unroll
  for (int i = 0; i < K; ++i) R[i][0][0] = R[i][0][1] = R[i][1][0] = R[i][1][1] = cst(0.f);
  if (point) {
    R[0][0][0] = -vb[0].A[0]; R[0][0][1] = -vb[0].A[1]; R[0][1][0] = -vb[0].A[2]; R[0][1][1] = -vb[0].A[3];
  } else {
    R[K - 1][0][0] = -vb[K - 1].Cc[0]; R[K - 1][0][1] = -vb[K - 1].Cc[1];
    R[K - 1][1][0] = -vb[K - 1].Cc[2]; R[K - 1][1][1] = -vb[K - 1].Cc[3];
  }
  DF Bi[K][4];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    DF Bp[4] = {vb[i].B[0], vb[i].B[1], vb[i].B[2], vb[i].B[3]};
    if (i > 0) {
      const DF* A = vb[i].A;
      DF Lm[4] = {A[0] * Bi[i - 1][0] + A[1] * Bi[i - 1][2], A[0] * Bi[i - 1][1] + A[1] * Bi[i - 1][3],
                  A[2] * Bi[i - 1][0] + A[3] * Bi[i - 1][2], A[2] * Bi[i - 1][1] + A[3] * Bi[i - 1][3]};
      const DF* Cp = vb[i - 1].Cc;
      Bp[0] = Bp[0] - (Lm[0] * Cp[0] + Lm[1] * Cp[2]);
      Bp[1] = Bp[1] - (Lm[0] * Cp[1] + Lm[1] * Cp[3]);
      Bp[2] = Bp[2] - (Lm[2] * Cp[0] + Lm[3] * Cp[2]);
      Bp[3] = Bp[3] - (Lm[2] * Cp[1] + Lm[3] * Cp[3]);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        DF r0 = R[i - 1][0][c], r1 = R[i - 1][1][c];
        R[i][0][c] = R[i][0][c] - (Lm[0] * r0 + Lm[1] * r1);
        R[i][1][c] = R[i][1][c] - (Lm[2] * r0 + Lm[3] * r1);
      }
    }
    DF det = Bp[0] * Bp[3] - Bp[1] * Bp[2];
    if (!(fabsf(det.v) > 0.0f)) return false;
    DF id = cst(1.0f) / det;
    Bi[i][0] = Bp[3] * id; Bi[i][1] = -(Bp[1] * id); Bi[i][2] = -(Bp[2] * id); Bi[i][3] = Bp[0] * id;
  }
#pragma unroll
  for (int i = K - 1; i >= 0; --i) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      DF r0 = R[i][0][c], r1 = R[i][1][c];
      if (i < K - 1) {
        const DF* Cc = vb[i].Cc;
        r0 = r0 - (Cc[0] * R[i + 1][0][c] + Cc[1] * R[i + 1][1][c]);
        r1 = r1 - (Cc[2] * R[i + 1][0][c] + Cc[3] * R[i + 1][1][c]);
      }
      R[i][0][c] = Bi[i][0] * r0 + Bi[i][1] * r1;
      R[i][1][c] = Bi[i][2] * r0 + Bi[i][3] * r1;
    }
  }
  // the vertex whose motion moves the measured direction: x_K (point light)
  // or x_1 (area light); selected by value so that every array index stays a
  // compile-time constant (a runtime index would move the arrays to memory)
  const V vp = point ? f[K].p : f[1].p, vdu = point ? f[K].dpdu : f[1].dpdu, vdv = point ? f[K].dpdv : f[1].dpdv;
  DF Ry[2][2];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) Ry[r][c] = point ? R[K - 1][r][c] : R[0][r][c];
  V w = vp - (point ? f[K + 1].p : f[0].p);
  DF dist = norm(w);
  w = w * (cst(1.0f) / dist);
  V a, b;
  onbv(w, a, b);
  DF M[2][2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    V dx = vdu * Ry[0][c] + vdv * Ry[1][c];
    V dw = (dx - w * dot(w, dx)) * (cst(1.0f) / dist);
    M[0][c] = dot(a, dw);
    M[1][c] = dot(b, dw);
  }
  DF G = dabs(M[0][0] * M[1][1] - M[0][1] * M[1][0]);
  if (!point) G = dot(f[0].n, w) * G;
  // kappa with the chain's cosines (transmittance formed directly; the
  // radiance scaling (eta_i/eta_o)^2 under an area light only)
  DF kap = cst(1.0f);
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const DSurf& sf = S.s[ch.surf[i]];
    if (sf.mat == MAT_MIRROR) continue;
    V wi = unitv(f[i].p - f[i + 1].p), wo = unitv(f[i + 2].p - f[i + 1].p);
    DF ci = dabs(dot(wi, f[i + 1].n));
    float n1 = vb[i].ei;
    if ((e.tau >> i) & 1u) {
      float n2 = vb[i].eo;
      DF co = dabs(dot(wo, f[i + 1].n));
      DF num = ci * co * (4.0f * n1 * n2);
      DF ds = ci * n1 + co * n2, dp = ci * n2 + co * n1;
      DF Tr = (num / (ds * ds) + num / (dp * dp)) * 0.5f;
      kap = point ? kap * Tr : kap * Tr * ((n1 / n2) * (n1 / n2));
    } else {
      float n2 = vb[i].front ? sf.etaB : sf.etaF;
      DF s2 = (cst(1.0f) - ci * ci) * ((n1 / n2) * (n1 / n2));
      DF F = cst(1.0f);
      if (s2.v < 1.0f) {
        DF c2 = dsqrt(cst(1.0f) - s2);
        DF rs = (ci * n1 - c2 * n2) / (ci * n1 + c2 * n2), rp = (ci * n2 - c2 * n1) / (ci * n2 + c2 * n1);
        F = (rs * rs + rp * rp) * 0.5f;
      }
      kap = kap * F;
    }
  }
  T = kap * G * S.L.power;
  return true;
}

}  // namespace adj
}  // namespace mpg
