// FP64 evaluation of the generalized geometry term for ill-conditioned chains.
//
// G = cos(theta_D) |det d(w_D)/d(u_L)| (area light) or |det d(w_L)/d(u_D)|
// (point light) with the implicit function theorem: J Y = -dC/du_end, J the
// block-tridiagonal constraint Jacobian.  Near caustic folds d(w)/d(u) has one
// small singular value, and FP32 rounding of J's entries and of the 2x2
// determinant leaves too few digits; the contribution kernel then repeats the
// evaluation here in FP64 from the same (FP32) vertices.
#pragma once

#include "mpg_device.cuh"

namespace mpg {

struct D3 {
  double x, y, z;
};
__device__ __forceinline__ D3 d3(float3 a) { return D3{(double)a.x, (double)a.y, (double)a.z}; }
__device__ __forceinline__ D3 d3(float4 a) { return D3{(double)a.x, (double)a.y, (double)a.z}; }
__device__ __forceinline__ D3 operator+(D3 a, D3 b) { return D3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ D3 operator-(D3 a, D3 b) { return D3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ D3 operator-(D3 a) { return D3{-a.x, -a.y, -a.z}; }
__device__ __forceinline__ D3 operator*(D3 a, double s) { return D3{a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ double dot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 cross(D3 a, D3 b) {
  return D3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double len(D3 a) { return sqrt(dot(a, a)); }
__device__ __forceinline__ D3 unit(D3 a) { return a * (1.0 / sqrt(dot(a, a))); }

__device__ __forceinline__ void onb(D3 n, D3& b1, D3& b2) {
  double s = n.z >= 0.0 ? 1.0 : -1.0;
  double a = -1.0 / (s + n.z);
  double b = n.x * n.y * a;
  b1 = D3{1.0 + s * n.x * n.x * a, s * b, -s * n.x};
  b2 = D3{b, s + n.y * n.y * a, -n.y};
}

struct Frame64 {
  D3 p, n, dpdu, dpdv, dndu, dndv;
};

// Same local geometry as vertex_frame, in FP64.
__device__ __forceinline__ Frame64 frame64(const DScene& S, int surf, int prim, float3 pf, float b1f, float b2f) {
  Frame64 f;
  const DSurf& sf = S.s[surf];
  if (sf.type == SURF_SPHERE || sf.type == SURF_CAP) {
    D3 c = d3(sf.c);
    double r = sf.r;
    // the FP32 vertex is on the sphere to FP32 rounding: project it exactly
    D3 m = unit(d3(pf) - c);
    f.p = c + m * r;
    f.n = m;
    onb(f.n, f.dpdu, f.dpdv);
    f.dndu = f.dpdu * (1.0 / r);
    f.dndv = f.dpdv * (1.0 / r);
  } else if (sf.type == SURF_RECT) {
    f.p = d3(pf);
    f.n = d3(sf.axis);
    onb(f.n, f.dpdu, f.dpdv);
    f.dndu = D3{0.0, 0.0, 0.0};
    f.dndv = f.dndu;
  } else {
    const DHF& H = S.hf[sf.hf];
    int v0, v1, v2;
    hf_tri(H, prim, v0, v1, v2);
    D3 P0 = d3(__ldg(H.P + v0)), P1 = d3(__ldg(H.P + v1)), P2 = d3(__ldg(H.P + v2));
    D3 N0 = d3(__ldg(H.N + v0)), N1 = d3(__ldg(H.N + v1)), N2 = d3(__ldg(H.N + v2));
    double b1 = b1f, b2 = b2f;
    D3 e1 = P1 - P0, e2 = P2 - P0;
    f.p = P0 + e1 * b1 + e2 * b2;
    onb(unit(cross(e1, e2)), f.dpdu, f.dpdv);
    D3 Ns = N0 * (1.0 - b1 - b2) + N1 * b1 + N2 * b2;
    double il = 1.0 / len(Ns);
    f.n = Ns * il;
    double g11 = dot(e1, e1), g12 = dot(e1, e2), g22 = dot(e2, e2);
    double igd = 1.0 / (g11 * g22 - g12 * g12);
    for (int q = 0; q < 2; ++q) {
      D3 a = q == 0 ? f.dpdu : f.dpdv;
      double r1 = dot(e1, a), r2 = dot(e2, a);
      double db1 = (g22 * r1 - g12 * r2) * igd, db2 = (g11 * r2 - g12 * r1) * igd;
      D3 dN = (N1 - N0) * db1 + (N2 - N0) * db2;
      D3 dn = (dN - f.n * dot(f.n, dN)) * il;
      if (q == 0) f.dndu = dn; else f.dndv = dn;
    }
  }
  return f;
}

struct VB64 {
  double A[4], B[4], Cc[4];
};

__device__ __forceinline__ bool blocks64(D3 xp, D3 tpu, D3 tpv, const Frame64& f, D3 xn, D3 tnu, D3 tnv,
                                         const DSurf& sf, bool refract, VB64& o) {
  D3 wi = xp - f.p, wo = xn - f.p;
  double di = len(wi), dO = len(wo);
  if (!(di > 0.0) || !(dO > 0.0)) return false;
  double idi = 1.0 / di, ido = 1.0 / dO;
  wi = wi * idi;
  wo = wo * ido;
  float eif, eof;
  if (!etas(sf, dot(wi, f.n) > 0.0, refract, eif, eof)) return false;
  double ei = eif, eo = eof;
  D3 ht = wi * ei + wo * eo;
  double L = len(ht);
  if (!(L > 0.0)) return false;
  double iL = 1.0 / L;
  D3 h = ht * iL;
  D3 s, t;
  onb(f.n, s, t);
  double cs = dot(h, s), ct = dot(h, t), hn = dot(h, f.n);
  D3 sp = (s - h * cs) * iL, tp = (t - h * ct) * iL;
  auto Pi = [&](D3 a) { return (a - wi * dot(wi, a)) * idi; };
  auto Po = [&](D3 a) { return (a - wo * dot(wo, a)) * ido; };
  D3 bu = -(Pi(f.dpdu) * ei + Po(f.dpdu) * eo), bv = -(Pi(f.dpdv) * ei + Po(f.dpdv) * eo);
  o.B[0] = dot(sp, bu) - hn * dot(s, f.dndu);
  o.B[1] = dot(sp, bv) - hn * dot(s, f.dndv);
  o.B[2] = dot(tp, bu) - hn * dot(t, f.dndu);
  o.B[3] = dot(tp, bv) - hn * dot(t, f.dndv);
  D3 au = Pi(tpu) * ei, av = Pi(tpv) * ei;
  o.A[0] = dot(sp, au); o.A[1] = dot(sp, av); o.A[2] = dot(tp, au); o.A[3] = dot(tp, av);
  D3 cu = Po(tnu) * eo, cv = Po(tnv) * eo;
  o.Cc[0] = dot(sp, cu); o.Cc[1] = dot(sp, cv); o.Cc[2] = dot(tp, cu); o.Cc[3] = dot(tp, cv);
  return true;
}

// Chain vertices in FP64 (positions on the surfaces, triangle ids, barycentrics).
template <int K>
struct Chain64 {
  D3 x[K];
  int surf[K], prim[K];
  double b1[K], b2[K];
};

// FP64 local frame at a chain vertex (positions already on the surface).
__device__ __forceinline__ Frame64 frame64_at(const DScene& S, int surf, int prim, D3 p, double b1, double b2) {
  const DSurf& sf = S.s[surf];
  if (sf.type == SURF_SPHERE || sf.type == SURF_CAP || sf.type == SURF_RECT) {
    Frame64 f = frame64(S, surf, prim, make_float3((float)p.x, (float)p.y, (float)p.z), 0.f, 0.f);
    if (sf.type != SURF_RECT) {
      D3 c = d3(sf.c);
      f.n = unit(p - c);
      f.p = p;
      onb(f.n, f.dpdu, f.dpdv);
      f.dndu = f.dpdu * (1.0 / (double)sf.r);
      f.dndv = f.dpdv * (1.0 / (double)sf.r);
    } else {
      f.p = p;
    }
    return f;
  }
  Frame64 f = frame64(S, surf, prim, make_float3(0.f, 0.f, 0.f), (float)b1, (float)b2);
  // recompute with the FP64 barycentrics
  const DHF& H = S.hf[sf.hf];
  int v0, v1, v2;
  hf_tri(H, prim, v0, v1, v2);
  D3 P0 = d3(__ldg(H.P + v0)), P1 = d3(__ldg(H.P + v1)), P2 = d3(__ldg(H.P + v2));
  D3 N0 = d3(__ldg(H.N + v0)), N1 = d3(__ldg(H.N + v1)), N2 = d3(__ldg(H.N + v2));
  D3 e1 = P1 - P0, e2 = P2 - P0;
  f.p = P0 + e1 * b1 + e2 * b2;
  D3 Ns = N0 * (1.0 - b1 - b2) + N1 * b1 + N2 * b2;
  double il = 1.0 / len(Ns);
  f.n = Ns * il;
  double g11 = dot(e1, e1), g12 = dot(e1, e2), g22 = dot(e2, e2);
  double igd = 1.0 / (g11 * g22 - g12 * g12);
  for (int q = 0; q < 2; ++q) {
    D3 a = q == 0 ? f.dpdu : f.dpdv;
    double r1 = dot(e1, a), r2 = dot(e2, a);
    double db1 = (g22 * r1 - g12 * r2) * igd, db2 = (g11 * r2 - g12 * r1) * igd;
    D3 dN = (N1 - N0) * db1 + (N2 - N0) * db2;
    D3 dn = (dN - f.n * dot(f.n, dN)) * il;
    if (q == 0) f.dndu = dn; else f.dndv = dn;
  }
  return f;
}

// Constraint value at a vertex in FP64.
__device__ __forceinline__ bool constraint64(D3 xp, const Frame64& f, D3 xn, const DSurf& sf, bool refract,
                                             double& c0, double& c1) {
  D3 wi = unit(xp - f.p), wo = unit(xn - f.p);
  float eif, eof;
  if (!etas(sf, dot(wi, f.n) > 0.0, refract, eif, eof)) return false;
  D3 ht = wi * (double)eif + wo * (double)eof;
  double L = len(ht);
  if (!(L > 0.0)) return false;
  D3 h = ht * (1.0 / L), s, t;
  onb(f.n, s, t);
  c0 = dot(h, s);
  c1 = dot(h, t);
  return true;
}

// Vertical ray cast into a heightfield in FP64.
__device__ __forceinline__ bool hf_vertical64(const DHF& H, double x, double y, D3& p, int& prim, double& b1,
                                              double& b2) {
  double fx = (x - (double)H.x0) / (double)H.dx, fy = (y - (double)H.y0) / (double)H.dy;
  if (!(fx >= 0.0 && fy >= 0.0 && fx <= (double)(H.nx - 1) && fy <= (double)(H.ny - 1))) return false;
  int i = min((int)fx, H.nx - 2), j = min((int)fy, H.ny - 2);
  double u = fx - i, w = fy - j;
  int quad = j * (H.nx - 1) + i;
  if (u >= w) { prim = 2 * quad; b1 = u - w; b2 = w; }
  else { prim = 2 * quad + 1; b1 = u; b2 = w - u; }
  int v0, v1, v2;
  hf_tri(H, prim, v0, v1, v2);
  D3 P0 = d3(__ldg(H.P + v0)), P1 = d3(__ldg(H.P + v1)), P2 = d3(__ldg(H.P + v2));
  p = P0 + (P1 - P0) * b1 + (P2 - P0) * b2;
  return true;
}

__device__ __forceinline__ bool reproject64(const DScene& S, int surf, D3 target, D3& p, int& prim, double& b1,
                                            double& b2) {
  const DSurf& sf = S.s[surf];
  if (sf.type == SURF_SPHERE || sf.type == SURF_CAP) {
    D3 c = d3(sf.c), d = target - c;
    double l = len(d);
    if (!(l > 0.0)) return false;
    p = c + d * ((double)sf.r / l);
    return sf.type == SURF_SPHERE || dot(p - c, d3(sf.axis)) >= (double)sf.r * (double)sf.cap_cos;
  }
  if (sf.type == SURF_RECT) {
    D3 ax = d3(sf.axis);
    p = target - ax * dot(target - d3(sf.c), ax);
    D3 q = p - d3(sf.c);
    return fabs(dot(q, d3(sf.ex))) <= (double)sf.ex2 && fabs(dot(q, d3(sf.ey))) <= (double)sf.ey2;
  }
  return hf_vertical64(S.hf[sf.hf], target.x, target.y, p, prim, b1, b2);
}

template <int K>
__device__ __forceinline__ void to64(const DScene& S, const Chain<K>& ch, Chain64<K>& c) {
#pragma unroll
  for (int i = 0; i < K; ++i) {
    c.surf[i] = ch.surf[i];
    c.prim[i] = ch.prim[i];
    c.b1[i] = ch.b1[i];
    c.b2[i] = ch.b2[i];
    const DSurf& sf = S.s[ch.surf[i]];
    D3 p = d3(ch.x[i]);
    if (sf.type == SURF_SPHERE || sf.type == SURF_CAP) p = d3(sf.c) + unit(p - d3(sf.c)) * (double)sf.r;
    c.x[i] = p;
  }
}

// Frames and Jacobian blocks of the whole chain; C (2K) and max |C| optional.
template <int K>
__device__ bool chain64(const DScene& S, const Chain64<K>& ch, const Ends& e, Frame64 (&f)[K], VB64 (&vb)[K],
                        double* C, double& cmax) {
#pragma unroll
  for (int i = 0; i < K; ++i) f[i] = frame64_at(S, ch.surf[i], ch.prim[i], ch.x[i], ch.b1[i], ch.b2[i]);
  D3 xD = d3(e.xD), xL = d3(e.xL), ru, rv;
  onb(d3(e.nD), ru, rv);
  D3 lu = d3(S.L.exu), lv = d3(S.L.eyu);
  cmax = 0.0;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    D3 xp = i == 0 ? xD : f[i > 0 ? i - 1 : 0].p;
    D3 xn = i == K - 1 ? xL : f[i < K - 1 ? i + 1 : 0].p;
    D3 pu = i == 0 ? ru : f[i > 0 ? i - 1 : 0].dpdu, pv = i == 0 ? rv : f[i > 0 ? i - 1 : 0].dpdv;
    D3 nu = i == K - 1 ? lu : f[i < K - 1 ? i + 1 : 0].dpdu, nv = i == K - 1 ? lv : f[i < K - 1 ? i + 1 : 0].dpdv;
    const DSurf& sf = S.s[ch.surf[i]];
    bool refract = (e.tau >> i) & 1u;
    if (!blocks64(xp, pu, pv, f[i], xn, nu, nv, sf, refract, vb[i])) return false;
    double c0, c1;
    if (!constraint64(xp, f[i], xn, sf, refract, c0, c1)) return false;
    if (C) { C[2 * i] = c0; C[2 * i + 1] = c1; }
    cmax = fmax(cmax, fmax(fabs(c0), fabs(c1)));
  }
  return true;
}

// Block Thomas sweep in FP64 for M columns; R[i][r][c].
template <int K, int M>
__device__ bool thomas64(const VB64 (&vb)[K], double (&R)[K][2][M], double sing_eps) {
  double Binv[K][4];
  double Bp[4] = {vb[0].B[0], vb[0].B[1], vb[0].B[2], vb[0].B[3]};
#pragma unroll
  for (int i = 0; i < K; ++i) {
    if (i > 0) {
      const double* Ai = vb[i].A;
      double Lm[4] = {Ai[0] * Binv[i - 1][0] + Ai[1] * Binv[i - 1][2], Ai[0] * Binv[i - 1][1] + Ai[1] * Binv[i - 1][3],
                      Ai[2] * Binv[i - 1][0] + Ai[3] * Binv[i - 1][2], Ai[2] * Binv[i - 1][1] + Ai[3] * Binv[i - 1][3]};
      const double* Cp = vb[i - 1].Cc;
      Bp[0] = vb[i].B[0] - (Lm[0] * Cp[0] + Lm[1] * Cp[2]);
      Bp[1] = vb[i].B[1] - (Lm[0] * Cp[1] + Lm[1] * Cp[3]);
      Bp[2] = vb[i].B[2] - (Lm[2] * Cp[0] + Lm[3] * Cp[2]);
      Bp[3] = vb[i].B[3] - (Lm[2] * Cp[1] + Lm[3] * Cp[3]);
      for (int c = 0; c < M; ++c) {
        double r0 = R[i - 1][0][c], r1 = R[i - 1][1][c];
        R[i][0][c] -= Lm[0] * r0 + Lm[1] * r1;
        R[i][1][c] -= Lm[2] * r0 + Lm[3] * r1;
      }
    }
    double det = Bp[0] * Bp[3] - Bp[1] * Bp[2];
    double mx = fmax(fmax(fabs(Bp[0]), fabs(Bp[1])), fmax(fabs(Bp[2]), fabs(Bp[3])));
    if (!(fabs(det) > sing_eps * mx * mx)) return false;
    double id = 1.0 / det;
    Binv[i][0] = Bp[3] * id; Binv[i][1] = -Bp[1] * id; Binv[i][2] = -Bp[2] * id; Binv[i][3] = Bp[0] * id;
  }
#pragma unroll
  for (int i = K - 1; i >= 0; --i) {
    for (int c = 0; c < M; ++c) {
      double r0 = R[i][0][c], r1 = R[i][1][c];
      if (i < K - 1) {
        const double* Cc = vb[i].Cc;
        r0 -= Cc[0] * R[i + 1][0][c] + Cc[1] * R[i + 1][1][c];
        r1 -= Cc[2] * R[i + 1][0][c] + Cc[3] * R[i + 1][1][c];
      }
      R[i][0][c] = Binv[i][0] * r0 + Binv[i][1] * r1;
      R[i][1][c] = Binv[i][2] * r0 + Binv[i][3] * r1;
    }
  }
  return true;
}

// Newton polish in FP64 of a converged FP32 chain (a few steps, each accepted
// only if it lowers |C|), then G in FP64.  Returns false if the chain is not a
// solution in FP64 (no step brings max|C| under tol) or G cannot be formed.
template <int K>
__device__ bool polish_ggt64(const DScene& S, Chain64<K>& ch, const Ends& e, double tol, double sing_eps, int steps,
                             double& G, double& kappa) {
  Frame64 f[K];
  VB64 vb[K];
  double C[2 * K], cmax;
  if (!chain64<K>(S, ch, e, f, vb, C, cmax)) return false;
  for (int it = 0; it < steps && cmax >= 1e-3 * tol; ++it) {
    double R[K][2][1];
#pragma unroll
    for (int i = 0; i < K; ++i) { R[i][0][0] = -C[2 * i]; R[i][1][0] = -C[2 * i + 1]; }
    if (!thomas64<K, 1>(vb, R, sing_eps)) break;
    Chain64<K> cand = ch;
    bool ok = true;
#pragma unroll
    for (int i = 0; i < K && ok; ++i) {
      D3 target = ch.x[i] + f[i].dpdu * R[i][0][0] + f[i].dpdv * R[i][1][0];
      ok = reproject64(S, ch.surf[i], target, cand.x[i], cand.prim[i], cand.b1[i], cand.b2[i]);
    }
    if (!ok) break;
    Frame64 fc[K];
    VB64 vc[K];
    double Cn[2 * K], cn;
    if (!chain64<K>(S, cand, e, fc, vc, Cn, cn) || !(cn < cmax)) break;
    ch = cand;
#pragma unroll
    for (int i = 0; i < K; ++i) { f[i] = fc[i]; vb[i] = vc[i]; }
#pragma unroll
    for (int i = 0; i < 2 * K; ++i) C[i] = Cn[i];
    cmax = cn;
  }
  if (!(cmax < tol)) return false;
  bool point = S.L.type == LIGHT_POINT;
  double R[K][2][2];
#pragma unroll
  for (int i = 0; i < K; ++i) R[i][0][0] = R[i][0][1] = R[i][1][0] = R[i][1][1] = 0.0;
  const double* E = point ? vb[0].A : vb[K - 1].Cc;
  int row = point ? 0 : K - 1;
  R[row][0][0] = -E[0]; R[row][0][1] = -E[1]; R[row][1][0] = -E[2]; R[row][1][1] = -E[3];
  if (!thomas64<K, 2>(vb, R, sing_eps)) return false;
  int vi = point ? K - 1 : 0;
  D3 anchor = point ? d3(e.xL) : d3(e.xD);
  D3 w = f[vi].p - anchor;
  double dist = len(w);
  w = w * (1.0 / dist);
  D3 a, b;
  onb(w, a, b);
  double M[2][2];
  for (int c = 0; c < 2; ++c) {
    D3 dx = f[vi].dpdu * R[vi][0][c] + f[vi].dpdv * R[vi][1][c];
    D3 dw = (dx - w * dot(w, dx)) * (1.0 / dist);
    M[0][c] = dot(a, dw);
    M[1][c] = dot(b, dw);
  }
  double det = fabs(M[0][0] * M[1][1] - M[0][1] * M[1][0]);
  G = point ? det : dot(d3(e.nD), w) * det;
  // kappa in FP64: mirror 1, dielectric R -> F, T -> (T_s + T_p)/2 (eta_i/eta_o)^2
  // (area light) or (T_s + T_p)/2 (point light)
  kappa = 1.0;
  D3 xD = d3(e.xD), xL = d3(e.xL);
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const DSurf& sf = S.s[ch.surf[i]];
    if (sf.mat == MAT_MIRROR) continue;
    D3 xp = i == 0 ? xD : f[i > 0 ? i - 1 : 0].p;
    D3 xn = i == K - 1 ? xL : f[i < K - 1 ? i + 1 : 0].p;
    D3 wi = unit(xp - f[i].p), wo = unit(xn - f[i].p);
    double ci = fabs(dot(wi, f[i].n));
    bool front = dot(wi, f[i].n) > 0.0;
    double n1 = front ? sf.etaF : sf.etaB;
    if ((e.tau >> i) & 1u) {
      double n2 = front ? sf.etaB : sf.etaF;
      double co = fabs(dot(wo, f[i].n));
      double num = 4.0 * n1 * n2 * ci * co, ds = n1 * ci + n2 * co, dp = n2 * ci + n1 * co;
      double r = point ? 1.0 : n1 / n2;
      kappa *= 0.5 * (num / (ds * ds) + num / (dp * dp)) * r * r;
    } else {
      double n2 = front ? sf.etaB : sf.etaF;
      double s2 = (n1 / n2) * (n1 / n2) * (1.0 - ci * ci);
      double F = 1.0;
      if (s2 < 1.0) {
        double c2 = sqrt(1.0 - s2);
        double rs = (n1 * ci - n2 * c2) / (n1 * ci + n2 * c2), rp = (n2 * ci - n1 * c2) / (n2 * ci + n1 * c2);
        F = 0.5 * (rs * rs + rp * rp);
      }
      kappa *= F;
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// The same FP64 polish and geometry term with one chain per group of G >= K
// lanes: lane j owns vertex j (frame, blocks and constraint of that vertex;
// the neighbours' positions and tangents come by shuffles within the group),
// the blocks are staged in shared memory, and every lane of the group runs the
// same block Thomas sweep over them.  The serial per-chain work of
// polish_ggt64 is K frames and block rows per evaluation; here each lane
// evaluates one, so a chain costs about 1/K of the instructions in sequence
// and its arrays stay in registers.  Decisions and arithmetic per vertex are
// those of polish_ggt64 (the product of the kappa factors is taken in
// another order).
// ---------------------------------------------------------------------------
__device__ __forceinline__ D3 shfl_d3(unsigned mask, D3 v, int src, int width) {
  return D3{__shfl_sync(mask, v.x, src, width), __shfl_sync(mask, v.y, src, width), __shfl_sync(mask, v.z, src, width)};
}
__device__ __forceinline__ D3 shfl_up_d3(unsigned mask, D3 v, int width) {
  return D3{__shfl_up_sync(mask, v.x, 1, width), __shfl_up_sync(mask, v.y, 1, width), __shfl_up_sync(mask, v.z, 1, width)};
}
__device__ __forceinline__ D3 shfl_down_d3(unsigned mask, D3 v, int width) {
  return D3{__shfl_down_sync(mask, v.x, 1, width), __shfl_down_sync(mask, v.y, 1, width),
            __shfl_down_sync(mask, v.z, 1, width)};
}

// Staged blocks of one vertex: A, B, Cc (row-major 2x2) and the constraint.
struct VS64 {
  double A[4], B[4], Cc[4], C[2];
};

// Own vertex j of a group: frame, blocks and constraint at the group's chain;
// false in every lane of the group when any vertex fails.  cmax is the
// group's maximum |C|.  The blocks are staged in sv[j].
template <int K, int G>
__device__ __forceinline__ bool chain64_g(const DScene& S, int j, unsigned gmask, int surf, int prim, D3 x, double b1,
                                         double b2, const Ends& e, Frame64& f, VS64* sv, double& cmax) {
  const bool own = j < K;
  if (own) f = frame64_at(S, surf, prim, x, b1, b2);
  D3 xp = shfl_up_d3(gmask, f.p, G), xn = shfl_down_d3(gmask, f.p, G);
  D3 pu = shfl_up_d3(gmask, f.dpdu, G), pv = shfl_up_d3(gmask, f.dpdv, G);
  D3 nu = shfl_down_d3(gmask, f.dpdu, G), nv = shfl_down_d3(gmask, f.dpdv, G);
  if (j == 0) {
    xp = d3(e.xD);
    onb(d3(e.nD), pu, pv);
  }
  if (j == K - 1) {
    xn = d3(e.xL);
    nu = d3(S.L.exu);
    nv = d3(S.L.eyu);
  }
  bool ok = true;
  double c0 = 0.0, c1 = 0.0;
  if (own) {
    const DSurf& sf = S.s[surf];
    const bool refract = (e.tau >> j) & 1u;
    VB64 vb;
    ok = blocks64(xp, pu, pv, f, xn, nu, nv, sf, refract, vb) && constraint64(xp, f, xn, sf, refract, c0, c1);
    if (ok) {
#pragma unroll
      for (int q = 0; q < 4; ++q) { sv[j].A[q] = vb.A[q]; sv[j].B[q] = vb.B[q]; sv[j].Cc[q] = vb.Cc[q]; }
      sv[j].C[0] = c0;
      sv[j].C[1] = c1;
    }
  }
  if (!__all_sync(gmask, ok)) return false;
  double m = fmax(fabs(c0), fabs(c1));
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(gmask, m, o, G));
  cmax = m;
  __syncwarp(gmask);  // the staged blocks are read by every lane of the group
  return true;
}

// thomas64 over staged blocks (every lane of a group runs it alike).
template <int K, int M>
__device__ __forceinline__ bool thomas64_s(const VS64* vb, double (&R)[K][2][M], double sing_eps) {
  double Binv[K][4];
  double Bp[4] = {vb[0].B[0], vb[0].B[1], vb[0].B[2], vb[0].B[3]};
#pragma unroll
  for (int i = 0; i < K; ++i) {
    if (i > 0) {
      const double* Ai = vb[i].A;
      double Lm[4] = {Ai[0] * Binv[i - 1][0] + Ai[1] * Binv[i - 1][2], Ai[0] * Binv[i - 1][1] + Ai[1] * Binv[i - 1][3],
                      Ai[2] * Binv[i - 1][0] + Ai[3] * Binv[i - 1][2], Ai[2] * Binv[i - 1][1] + Ai[3] * Binv[i - 1][3]};
      const double* Cp = vb[i - 1].Cc;
      Bp[0] = vb[i].B[0] - (Lm[0] * Cp[0] + Lm[1] * Cp[2]);
      Bp[1] = vb[i].B[1] - (Lm[0] * Cp[1] + Lm[1] * Cp[3]);
      Bp[2] = vb[i].B[2] - (Lm[2] * Cp[0] + Lm[3] * Cp[2]);
      Bp[3] = vb[i].B[3] - (Lm[2] * Cp[1] + Lm[3] * Cp[3]);
#pragma unroll
      for (int c = 0; c < M; ++c) {
        double r0 = R[i - 1][0][c], r1 = R[i - 1][1][c];
        R[i][0][c] -= Lm[0] * r0 + Lm[1] * r1;
        R[i][1][c] -= Lm[2] * r0 + Lm[3] * r1;
      }
    }
    double det = Bp[0] * Bp[3] - Bp[1] * Bp[2];
    double mx = fmax(fmax(fabs(Bp[0]), fabs(Bp[1])), fmax(fabs(Bp[2]), fabs(Bp[3])));
    if (!(fabs(det) > sing_eps * mx * mx)) return false;
    double id = 1.0 / det;
    Binv[i][0] = Bp[3] * id; Binv[i][1] = -Bp[1] * id; Binv[i][2] = -Bp[2] * id; Binv[i][3] = Bp[0] * id;
  }
#pragma unroll
  for (int i = K - 1; i >= 0; --i) {
#pragma unroll
    for (int c = 0; c < M; ++c) {
      double r0 = R[i][0][c], r1 = R[i][1][c];
      if (i < K - 1) {
        const double* Cc = vb[i].Cc;
        r0 -= Cc[0] * R[i + 1][0][c] + Cc[1] * R[i + 1][1][c];
        r1 -= Cc[2] * R[i + 1][0][c] + Cc[3] * R[i + 1][1][c];
      }
      R[i][0][c] = Binv[i][0] * r0 + Binv[i][1] * r1;
      R[i][1][c] = Binv[i][2] * r0 + Binv[i][3] * r1;
    }
  }
  return true;
}


// polish_ggt64 in group form.  Lane j < K holds vertex j in (x, prim, b1, b2)
// and gets the polished vertex back; G and kappa come back in every lane of
// the group.  The staging area sv holds K vertices and is private to the group.
template <int K, int G>
__device__ bool polish_ggt64_g(const DScene& S, int j, unsigned gmask, int surf, int& prim, D3& x, double& b1,
                               double& b2, const Ends& e, double tol, double sing_eps, int steps, VS64* sv, double& G64,
                               double& kappa) {
  const bool own = j < K;
  Frame64 f;
  f.p = f.n = f.dpdu = f.dpdv = f.dndu = f.dndv = D3{0.0, 0.0, 0.0};
  double cmax;
  if (!chain64_g<K, G>(S, j, gmask, surf, prim, x, b1, b2, e, f, sv, cmax)) return false;
  for (int it = 0; it < steps && cmax >= 1e-3 * tol; ++it) {
    double R[K][2][1];
#pragma unroll
    for (int i = 0; i < K; ++i) { R[i][0][0] = -sv[i].C[0]; R[i][1][0] = -sv[i].C[1]; }
    if (!thomas64_s<K, 1>(sv, R, sing_eps)) break;
    double r0 = 0.0, r1 = 0.0;
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (i == j) { r0 = R[i][0][0]; r1 = R[i][1][0]; }
    D3 cx = x;
    int cprim = prim;
    double cb1 = b1, cb2 = b2;
    bool ok = !own || reproject64(S, surf, x + f.dpdu * r0 + f.dpdv * r1, cx, cprim, cb1, cb2);
    if (!__all_sync(gmask, ok)) break;
    __syncwarp(gmask);  // every lane has read the staged blocks of the current chain
    Frame64 fc = f;
    double cn;
    // a failed or worse candidate leaves the staging area overwritten: the
    // loop ends then, and only the current vertices and frame are used below
    const bool ev = chain64_g<K, G>(S, j, gmask, surf, cprim, cx, cb1, cb2, e, fc, sv, cn);
    if (!ev || !(cn < cmax)) {
      // restore the staged blocks of the current chain for the geometry term
      // (the same evaluation as before this attempt, so the same values)
      chain64_g<K, G>(S, j, gmask, surf, prim, x, b1, b2, e, f, sv, cmax);
      break;
    }
    x = cx; prim = cprim; b1 = cb1; b2 = cb2;
    f = fc;
    cmax = cn;
  }
  if (!(cmax < tol)) return false;
  const bool point = S.L.type == LIGHT_POINT;
  double R[K][2][2];
#pragma unroll
  for (int i = 0; i < K; ++i) R[i][0][0] = R[i][0][1] = R[i][1][0] = R[i][1][1] = 0.0;
  const double* E = point ? sv[0].A : sv[K - 1].Cc;
  const int row = point ? 0 : K - 1;
  R[row][0][0] = -E[0]; R[row][0][1] = -E[1]; R[row][1][0] = -E[2]; R[row][1][1] = -E[3];
  if (!thomas64_s<K, 2>(sv, R, sing_eps)) return false;
  const int vi = point ? K - 1 : 0;
  // the frame of vertex vi, from its lane
  D3 pv = shfl_d3(gmask, f.p, vi, G), du = shfl_d3(gmask, f.dpdu, vi, G), dv = shfl_d3(gmask, f.dpdv, vi, G);
  D3 anchor = point ? d3(e.xL) : d3(e.xD);
  D3 w = pv - anchor;
  double dist = len(w);
  w = w * (1.0 / dist);
  D3 a, b;
  onb(w, a, b);
  double M[2][2];
  for (int c = 0; c < 2; ++c) {
    D3 dx = du * R[vi][0][c] + dv * R[vi][1][c];
    D3 dw = (dx - w * dot(w, dx)) * (1.0 / dist);
    M[0][c] = dot(a, dw);
    M[1][c] = dot(b, dw);
  }
  double det = fabs(M[0][0] * M[1][1] - M[0][1] * M[1][0]);
  G64 = point ? det : dot(d3(e.nD), w) * det;
  // kappa: each lane its vertex's factor (as polish_ggt64), multiplied over the group
  double kf = 1.0;
  D3 xp = shfl_up_d3(gmask, f.p, G), xn = shfl_down_d3(gmask, f.p, G);
  if (j == 0) xp = d3(e.xD);
  if (j == K - 1) xn = d3(e.xL);
  if (own) {
    const DSurf& sf = S.s[surf];
    if (sf.mat != MAT_MIRROR) {
      D3 wi = unit(xp - f.p), wo = unit(xn - f.p);
      double ci = fabs(dot(wi, f.n));
      bool front = dot(wi, f.n) > 0.0;
      double n1 = front ? sf.etaF : sf.etaB;
      double n2 = front ? sf.etaB : sf.etaF;
      if ((e.tau >> j) & 1u) {
        double co = fabs(dot(wo, f.n));
        double num = 4.0 * n1 * n2 * ci * co, ds = n1 * ci + n2 * co, dp = n2 * ci + n1 * co;
        double r = point ? 1.0 : n1 / n2;
        kf = 0.5 * (num / (ds * ds) + num / (dp * dp)) * r * r;
      } else {
        double s2 = (n1 / n2) * (n1 / n2) * (1.0 - ci * ci);
        double F = 1.0;
        if (s2 < 1.0) {
          double c2 = sqrt(1.0 - s2);
          double rs = (n1 * ci - n2 * c2) / (n1 * ci + n2 * c2), rp = (n2 * ci - n1 * c2) / (n2 * ci + n1 * c2);
          F = 0.5 * (rs * rs + rp * rp);
        }
        kf = F;
      }
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) kf *= __shfl_xor_sync(gmask, kf, o, G);
  kappa = kf;
  return true;
}

}  // namespace mpg
