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
    // J = dC/du (NU x NU) and dT/du from the u directions, in chunks of
    // LANES directions whose indices are compile-time constants (so J stays
    // in registers); no height lanes are seeded in these chunks.
    constexpr int NCU = (NU + adj::LANES - 1) / adj::LANES;
    float J[NU][NU], dTu[NU];
    bool ok = true;
#pragma unroll
    for (int cu = 0; cu < NCU; ++cu) {
      adj::DF C[NU], Tv;
      ok = ok && adj::chain_eval<K>(S, ch, e, params, 0, D, cu * adj::LANES, C, Tv);
#pragma unroll
      for (int l = 0; l < adj::LANES; ++l) {
        const int d = cu * adj::LANES + l;
        if (d < NU) {
#pragma unroll
          for (int r = 0; r < NU; ++r) J[r][d] = C[r].d[l];
          dTu[d] = Tv.d[l];
        }
      }
    }
    if (!ok) { atomicAdd(skipped, 1); continue; }
    // J^T lambda = dT/du by the 2x2-block Thomas sweep on the transposed
    // block-tridiagonal system: its diagonal blocks are B_i^T, its sub- and
    // super-diagonal blocks Cc_{i-1}^T and A_{i+1}^T.
    VB vt[K];
    float2 lam2[K][1];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const int r = 2 * i;
      vt[i].B = make_float4(J[r][r], J[r + 1][r], J[r][r + 1], J[r + 1][r + 1]);
      if (i > 0) vt[i].A = make_float4(J[r - 2][r], J[r - 1][r], J[r - 2][r + 1], J[r - 1][r + 1]);
      if (i < K - 1) vt[i].Cc = make_float4(J[r + 2][r], J[r + 3][r], J[r + 2][r + 1], J[r + 3][r + 1]);
      lam2[i][0] = make_float2(dTu[r], dTu[r + 1]);
    }
    if (!thomas<K, 1>(vt, lam2, 0.0f)) { atomicAdd(skipped, 1); continue; }
    float lam[NU];
#pragma unroll
    for (int i = 0; i < K; ++i) { lam[2 * i] = lam2[i][0].x; lam[2 * i + 1] = lam2[i][0].y; }
    // dT/dtheta_p - lambda^T dC/dtheta_p for the heights, LANES at a time,
    // scattered as soon as they are formed (the values of every chunk are
    // those of the u chunks, so a chain that passed them passes these too)
    for (int p0 = 0; p0 < m; p0 += adj::LANES) {
      adj::DF C[NU], Tv;
      if (!adj::chain_eval<K>(S, ch, e, params, m, D, NU + p0, C, Tv)) break;
#pragma unroll
      for (int l = 0; l < adj::LANES; ++l) {
        const int p = p0 + l;
        if (p >= m) break;
        float g = Tv.d[l];
#pragma unroll
        for (int r = 0; r < NU; ++r) g -= lam[r] * C[r].d[l];
        atomicAdd(dL_dtheta + params[p], scale * g);
      }
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
