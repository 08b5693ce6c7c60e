// K7 -- adjoint kernel: per converged chain on heightfield 0, the transposed
// implicit-function solve for dT/dtheta (see mpg_adjoint.cuh), scattered into
// dL/dtheta with the upstream weight of the chain's receiver point.
#include "mpg_adjoint.cuh"
#include "mpg_kernels.cuh"

namespace mpg {
namespace {

constexpr int MAXP = 15;  // grid heights that can move one triangle vertex (corners and normal stencils)

template <int K>
__global__ void __launch_bounds__(64) k_adjoint(const __grid_constant__ DScene S, DChains c, const float* T,
                                                const float* contrib, const float* dL_dE, float* dL_dtheta,
                                                int* skipped) {
  constexpr int NU = 2 * K;
  constexpr int ND = NU + MAXP * K;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < c.B; b += gridDim.x * blockDim.x) {
    if (c.k[b] != K) continue;
    float cb = contrib[b], Tb = T[b];
    if (!(cb > 0.0f) || !(Tb > 0.0f)) continue;
    int q = b / c.spq;
    float scale = dL_dE[q] / (float)c.spq * (cb / Tb);  // d(contrib_b / spq)/dT_b, <1/P> fixed
    if (scale == 0.0f) continue;
    Chain<K> ch;
    Ends e;
    {
      const size_t B = (size_t)c.B;
#pragma unroll
      for (int i = 0; i < K; ++i) {
        ch.x[i] = make_float3(c.x[(3 * i + 0) * B + b], c.x[(3 * i + 1) * B + b], c.x[(3 * i + 2) * B + b]);
        ch.surf[i] = c.surf[i * B + b];
        ch.prim[i] = c.prim[i * B + b];
        ch.b1[i] = c.bary[(2 * i + 0) * B + b];
        ch.b2[i] = c.bary[(2 * i + 1) * B + b];
      }
      e.xD = make_float3(c.xD[q], c.xD[c.Q + q], c.xD[2 * c.Q + q]);
      e.nD = make_float3(c.nD[q], c.nD[c.Q + q], c.nD[2 * c.Q + q]);
      e.xL = make_float3(c.xL[b], c.xL[B + b], c.xL[2 * B + b]);
      e.tau = c.tau[b];
    }
    bool hf_only = true;
#pragma unroll
    for (int i = 0; i < K; ++i) hf_only = hf_only && S.s[ch.surf[i]].type == SURF_HEIGHTFIELD && S.s[ch.surf[i]].hf == 0;
    if (!hf_only) { atomicAdd(skipped, 1); continue; }
    const DHF& hf = S.hf[0];
    // grid heights moving the chain, and the map from local coordinates to barycentrics
    int params[MAXP * K];
    int m = 0;
    float D[K][4];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      int v[3];
      hf_tri(hf, ch.prim[i], v[0], v[1], v[2]);
      for (int cc = 0; cc < 3; ++cc) {
        int gi = v[cc] % hf.nx, gj = v[cc] / hf.nx;
        int cand[5][2] = {{gi, gj}, {gi - 1, gj}, {gi + 1, gj}, {gi, gj - 1}, {gi, gj + 1}};
        for (int r = 0; r < 5; ++r) {
          if (cand[r][0] < 0 || cand[r][0] >= hf.nx || cand[r][1] < 0 || cand[r][1] >= hf.ny) continue;
          int id = cand[r][1] * hf.nx + cand[r][0];
          bool seen = false;
          for (int p = 0; p < m; ++p) seen = seen || params[p] == id;
          if (!seen && m < MAXP * K) params[m++] = id;
        }
      }
      float3 P0 = f3(__ldg(hf.P + v[0])), P1 = f3(__ldg(hf.P + v[1])), P2 = f3(__ldg(hf.P + v[2]));
      float3 e1 = P1 - P0, e2 = P2 - P0, du, dv;
      onb(unit(cross(e1, e2)), du, dv);
      float g11 = dot(e1, e1), g12 = dot(e1, e2), g22 = dot(e2, e2), igd = 1.0f / (g11 * g22 - g12 * g12);
#pragma unroll
      for (int qq = 0; qq < 2; ++qq) {
        float3 a = qq == 0 ? du : dv;
        float r1 = dot(e1, a), r2 = dot(e2, a);
        D[i][qq] = (g22 * r1 - g12 * r2) * igd;
        D[i][2 + qq] = (g11 * r2 - g12 * r1) * igd;
      }
    }
    const int nd = NU + m;
    float dC[NU][ND], dT[ND];
    bool ok = true;
    for (int d0 = 0; d0 < nd && ok; d0 += adj::LANES) {
      adj::DF C[NU], Tv;
      ok = adj::chain_eval<K>(S, ch, e, params, m, D, d0, C, Tv);
      for (int l = 0; l < adj::LANES && ok; ++l) {
        int d = d0 + l;
        if (d >= nd) break;
#pragma unroll
        for (int r = 0; r < NU; ++r) dC[r][d] = C[r].d[l];
        dT[d] = Tv.d[l];
      }
    }
    if (!ok) { atomicAdd(skipped, 1); continue; }
    // J^T lambda = dT/du by the 2x2-block Thomas sweep on the transposed
    // block-tridiagonal system: its diagonal blocks are B_i^T, its sub- and
    // super-diagonal blocks Cc_{i-1}^T and A_{i+1}^T (J = dC/du, dC[r][d] for d < 2k).
    VB vt[K];
    float2 lam2[K][1];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const int r = 2 * i;
      vt[i].B = make_float4(dC[r][r], dC[r + 1][r], dC[r][r + 1], dC[r + 1][r + 1]);
      if (i > 0) vt[i].A = make_float4(dC[r - 2][r], dC[r - 1][r], dC[r - 2][r + 1], dC[r - 1][r + 1]);
      if (i < K - 1) vt[i].Cc = make_float4(dC[r + 2][r], dC[r + 3][r], dC[r + 2][r + 1], dC[r + 3][r + 1]);
      lam2[i][0] = make_float2(dT[r], dT[r + 1]);
    }
    if (!thomas<K, 1>(vt, lam2, 0.0f)) { atomicAdd(skipped, 1); continue; }
    float lam[NU];
#pragma unroll
    for (int i = 0; i < K; ++i) { lam[2 * i] = lam2[i][0].x; lam[2 * i + 1] = lam2[i][0].y; }
    for (int p = 0; p < m; ++p) {
      float g = dT[NU + p];
#pragma unroll
      for (int r = 0; r < NU; ++r) g -= lam[r] * dC[r][NU + p];
      atomicAdd(dL_dtheta + params[p], scale * g);
    }
  }
}

}  // namespace

void launch_adjoint(int K, const DScene& S, const DChains& c, const float* T, const float* contrib,
                    const float* dL_dE, float* dL_dtheta, int* skipped, int sms, cudaStream_t st) {
  int grid = sms * 8;
  switch (K) {
    case 1: k_adjoint<1><<<grid, 64, 0, st>>>(S, c, T, contrib, dL_dE, dL_dtheta, skipped); break;
    case 2: k_adjoint<2><<<grid, 64, 0, st>>>(S, c, T, contrib, dL_dE, dL_dtheta, skipped); break;
    case 3: k_adjoint<3><<<grid, 64, 0, st>>>(S, c, T, contrib, dL_dE, dL_dtheta, skipped); break;
    case 4: k_adjoint<4><<<grid, 64, 0, st>>>(S, c, T, contrib, dL_dE, dL_dtheta, skipped); break;
    default: break;
  }
}

}  // namespace mpg
