// Glossy chains (Sec. 5.7): every vertex is a rough interface with an
// isotropic Beckmann distribution of one roughness alpha.  A chain carries one
// offset normal per vertex, drawn from the distribution, and the walk solves
// C_i = (h.s_i, h.t_i) - o_i with o_i the offset's tangential components in
// the vertex's shading frame (the Jacobian blocks are those of the specular
// constraint).  A found chain's estimate is the path integrand in area
// measure over the offsets' density,
//   W = L_e prod_i f_i |n_i.l_i| prod(area factors) / (|det dC/du| prod_i p(o_i)),
// with f the microfacet BSDF of Walter et al. 2007 and p(o) = D(m) on the
// unit disk (drawing m with density D(m) (m.n) in solid angle gives that), so
// D cancels and only the Fresnel, shadowing and Jacobian factors remain.
// Here W is formed in FP64 after an FP64 polish of the FP32 converged vertices
// to C = o, and |det dC/du| as the product of the pivot determinants of the
// block Thomas elimination.
#pragma once

#include "mpg_ggt64.cuh"

namespace mpg {

// Smith masking of one direction with cosine c to the macro normal and cosine
// cm to the microfacet normal, Beckmann distribution, exact Lambda (erf form).
__device__ __forceinline__ double smith_g1(double c, double cm, double alpha) {
  if (!(c * cm > 0.0)) return 0.0;
  const double ac = fabs(c);
  if (ac >= 1.0) return 1.0;
  const double tan_t = sqrt(1.0 - ac * ac) / ac;
  const double a = 1.0 / (alpha * tan_t);
  const double lambda = 0.5 * (erf(a) - 1.0) + exp(-a * a) / (2.0 * a * 1.7724538509055160273);
  return 1.0 / (1.0 + lambda);
}

// Unpolarised Fresnel reflectance for incidence cosine c1 from eta1 into eta2.
__device__ __forceinline__ double fresnel64(double c1, double eta1, double eta2) {
  const double s2 = (eta1 / eta2) * (eta1 / eta2) * (1.0 - c1 * c1);
  if (s2 >= 1.0) return 1.0;
  const double c2 = sqrt(1.0 - s2);
  const double rs = (eta1 * c1 - eta2 * c2) / (eta1 * c1 + eta2 * c2);
  const double rp = (eta2 * c1 - eta1 * c2) / (eta2 * c1 + eta1 * c2);
  return 0.5 * (rs * rs + rp * rp);
}

// |det J| of the block-tridiagonal Jacobian as the product of the pivot
// determinants det(B'_i) of the block LU elimination (B'_0 = B_0,
// B'_i = B_i - A_i B'_{i-1}^{-1} Cc_{i-1}).  0 when a pivot is singular.
template <int K>
__device__ __forceinline__ double block_det64(const VB64 (&vb)[K]) {
  double Bp[4] = {vb[0].B[0], vb[0].B[1], vb[0].B[2], vb[0].B[3]};
  double det = 1.0;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    if (i > 0) {
      const double d0 = Bp[0] * Bp[3] - Bp[1] * Bp[2];
      if (d0 == 0.0) return 0.0;
      const double id = 1.0 / d0;
      const double Bi[4] = {Bp[3] * id, -Bp[1] * id, -Bp[2] * id, Bp[0] * id};
      const double* A = vb[i].A;
      const double L[4] = {A[0] * Bi[0] + A[1] * Bi[2], A[0] * Bi[1] + A[1] * Bi[3], A[2] * Bi[0] + A[3] * Bi[2],
                           A[2] * Bi[1] + A[3] * Bi[3]};
      const double* Cp = vb[i - 1].Cc;
      Bp[0] = vb[i].B[0] - (L[0] * Cp[0] + L[1] * Cp[2]);
      Bp[1] = vb[i].B[1] - (L[0] * Cp[1] + L[1] * Cp[3]);
      Bp[2] = vb[i].B[2] - (L[2] * Cp[0] + L[3] * Cp[2]);
      Bp[3] = vb[i].B[3] - (L[2] * Cp[1] + L[3] * Cp[3]);
    }
    det *= Bp[0] * Bp[3] - Bp[1] * Bp[2];
  }
  return fabs(det);
}

// Frames, blocks and the residual max |C_i - o_i| of a glossy chain in FP64.
template <int K>
__device__ __forceinline__ bool glossy_chain64(const DScene& S, const Chain64<K>& ch, const Ends& e,
                                               const float2 (&off)[K], Frame64 (&f)[K], VB64 (&vb)[K],
                                               double (&C)[2 * K], double& cmax) {
  if (!chain64<K>(S, ch, e, f, vb, C, cmax)) return false;
  cmax = 0.0;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    C[2 * i] -= (double)off[i].x;
    C[2 * i + 1] -= (double)off[i].y;
    cmax = fmax(cmax, fmax(fabs(C[2 * i]), fabs(C[2 * i + 1])));
  }
  return true;
}

// Newton polish in FP64 of a glossy chain converged in FP32 (C = o): at most
// `steps` steps, each accepted only if it lowers max |C - o|, until it is
// below 1e-3 tol.  Returns false if the chain is not a solution in FP64
// (max |C - o| stays at or above tol); f and vb are those of the final chain.
template <int K>
__device__ bool glossy_polish64(const DScene& S, Chain64<K>& ch, const Ends& e, const float2 (&off)[K], double tol,
                                double sing_eps, int steps, Frame64 (&f)[K], VB64 (&vb)[K]) {
  double C[2 * K], cmax;
  if (!glossy_chain64<K>(S, ch, e, off, f, vb, C, cmax)) return false;
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
    if (!glossy_chain64<K>(S, cand, e, off, fc, vc, Cn, cn) || !(cn < cmax)) break;
    ch = cand;
#pragma unroll
    for (int i = 0; i < K; ++i) { f[i] = fc[i]; vb[i] = vc[i]; }
#pragma unroll
    for (int i = 0; i < 2 * K; ++i) C[i] = Cn[i];
    cmax = cn;
  }
  return cmax < tol;
}

// Estimate W of one converged, admissible glossy chain (alpha > 0), or with
// alpha = 0 its specular limit (shadowing dropped), after polishing the chain
// in FP64 to C = o (ch is updated with the polished vertices).  Near a
// vanishing shadowing term or a grazing cosine W moves fast with the
// vertices, so it is formed at the FP64 solution rather than at the FP32 one.
// Returns false when the polish fails, the Jacobian is singular or a term
// cannot be formed.
template <int K>
__device__ bool glossy_w64(const DScene& S, Chain64<K>& ch, const Ends& e, const float2 (&off)[K], double alpha,
                           double tol, double sing_eps, double& W) {
  Frame64 f[K];
  VB64 vb[K];
  if (!glossy_polish64<K>(S, ch, e, off, tol, sing_eps, 4, f, vb)) return false;
  const double detJ = block_det64<K>(vb);
  if (!(detJ > 0.0)) return false;
  const D3 xD = d3(e.xD), xL = d3(e.xL);
  double bsdf = 1.0, geom = 1.0;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const DSurf& sf = S.s[ch.surf[i]];
    const D3 xp = i == 0 ? xD : f[i > 0 ? i - 1 : 0].p;
    const D3 xn = i == K - 1 ? xL : f[i < K - 1 ? i + 1 : 0].p;
    const D3 tv = xp - f[i].p;
    const double dv = len(tv);
    const D3 v = tv * (1.0 / dv), l = unit(xn - f[i].p);
    const double cv = dot(v, f[i].n), cl = dot(l, f[i].n);
    const bool refract = (e.tau >> i) & 1u;
    float eif, eof;
    if (!etas(sf, cv > 0.0, refract, eif, eof)) return false;
    const double ev = eif, el = eof;  // indices on the receiver and on the light side
    D3 m = unit(v * ev + l * el);
    if (dot(m, f[i].n) < 0.0) m = -m;
    const double vm = dot(v, m), lm = dot(l, m);
    double F = 1.0;
    if (sf.mat != MAT_MIRROR) F = fresnel64(fabs(vm), ev, cv > 0.0 ? (double)sf.etaB : (double)sf.etaF);
    const double G2 = alpha > 0.0 ? smith_g1(cv, vm, alpha) * smith_g1(cl, lm, alpha) : 1.0;
    double fhat;  // the BSDF over D(m)
    if (refract) {
      const double den = ev * vm + el * lm;
      fhat = fabs(lm) * fabs(vm) / (fabs(cl) * fabs(cv)) * ev * ev * (1.0 - F) * G2 / (den * den);
    } else {
      fhat = F * G2 / (4.0 * fabs(cl) * fabs(cv));
    }
    bsdf *= fhat * fabs(cl);
    // area measure at x_i: cosine to the geometric normal over the squared distance
    const D3 ng = unit(cross(f[i].dpdu, f[i].dpdv));
    geom *= fabs(dot(ng, v)) / (dv * dv);
  }
  geom *= fabs(dot(d3(e.nD), unit(f[0].p - xD)));
  const D3 tl = f[K - 1].p - xL;
  const double dL = len(tl);
  geom *= (S.L.type == LIGHT_POINT ? 1.0 : fabs(dot(d3(S.L.n), tl * (1.0 / dL)))) / (dL * dL);
  W = (double)S.L.power * bsdf * geom / detJ;
  return W > 0.0;
}

}  // namespace mpg
