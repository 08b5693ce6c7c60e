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

// G in FP64 for the chain ch (vertices as stored by the walk).
template <int K>
__device__ bool ggt64(const DScene& S, const Chain<K>& ch, const Ends& e, double sing_eps, double& G) {
  Frame64 f[K];
#pragma unroll
  for (int i = 0; i < K; ++i) f[i] = frame64(S, ch.surf[i], ch.prim[i], ch.x[i], ch.b1[i], ch.b2[i]);
  D3 xD = d3(e.xD), xL = d3(e.xL), nD = d3(e.nD);
  D3 ru, rv;
  onb(nD, ru, rv);
  D3 lu = d3(S.L.exu), lv = d3(S.L.eyu);
  VB64 vb[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    D3 xp = i == 0 ? xD : f[i > 0 ? i - 1 : 0].p;
    D3 xn = i == K - 1 ? xL : f[i < K - 1 ? i + 1 : 0].p;
    D3 pu = i == 0 ? ru : f[i > 0 ? i - 1 : 0].dpdu, pv = i == 0 ? rv : f[i > 0 ? i - 1 : 0].dpdv;
    D3 nu = i == K - 1 ? lu : f[i < K - 1 ? i + 1 : 0].dpdu, nv = i == K - 1 ? lv : f[i < K - 1 ? i + 1 : 0].dpdv;
    if (!blocks64(xp, pu, pv, f[i], xn, nu, nv, S.s[ch.surf[i]], (e.tau >> i) & 1u, vb[i])) return false;
  }
  bool point = S.L.type == LIGHT_POINT;
  // right-hand side: -dC/du_end in block row 0 (point light) or K-1 (area light)
  double R[K][2][2];
#pragma unroll
  for (int i = 0; i < K; ++i) R[i][0][0] = R[i][0][1] = R[i][1][0] = R[i][1][1] = 0.0;
  const double* E = point ? vb[0].A : vb[K - 1].Cc;
  int row = point ? 0 : K - 1;
  R[row][0][0] = -E[0]; R[row][0][1] = -E[1]; R[row][1][0] = -E[2]; R[row][1][1] = -E[3];
  // block Thomas sweep, two columns
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
      for (int c = 0; c < 2; ++c) {
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
    for (int c = 0; c < 2; ++c) {
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
  int vi = point ? K - 1 : 0;
  D3 anchor = point ? xL : xD;
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
  G = point ? det : dot(nD, w) * det;
  return true;
}

}  // namespace mpg
