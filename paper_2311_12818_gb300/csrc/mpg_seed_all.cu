// Seeds of a mixed-length batch in one launch (batched mode).
//
// The per-length seed kernels of the plain mode each take the chains of one
// length k, whose indices are spread over the whole batch: their stores of k
// vertex rows (SoA, chain index fastest) fill 4 of every 32 bytes of a sector,
// and at 4M chains (rows of 16 MB) every such store costs a sector read and
// write in DRAM -- about 850 bytes each way per chain at k = 4 against 130
// useful.  Here a warp takes 32 consecutive chains whatever their lengths, so
// the rows of a sector are written together.  The draw (p_0 of Sec. 5.4 and
// the guided mixture of Sec. 5.5, as k_seed) takes the length at run time and
// the deduction (Eq. deduction) loops over it, so one copy of the code serves
// every length (eight copies, one per length, overflow the instruction cache:
// a version that switched between the per-length draws took 194 ms for the
// 4M-chain mixed batch).  With a vMF guide the lobe sum of the density is
// taken after the draws, by the whole warp.
#include "mpg_kernels_impl.cuh"

namespace mpg {
namespace kern {

template <bool kS>
__global__ void __launch_bounds__(128) k_seed_all(const __grid_constant__ DScene S, DGuide g, int has_guide,
                                                  DChains c, uint2 key, uint64_t offset, mpg_params P, DCtx ctx) {
  Tally t = {};
  const int n = c.B;
  const size_t B = (size_t)c.B;
  offset = rng_offset(offset, ctx);
  const bool vmf = has_guide && g.kind == MPG_GUIDE_VMF;
  const DGuide* gp = has_guide ? &g : nullptr;
  const int lane = threadIdx.x & 31;
  for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += gridDim.x * blockDim.x) {
    const int b = base + lane;
    const int k = b < n ? (int)c.k[b] : 0;
    const bool mine = k >= 1 && k <= MAXK;  // a length outside 1..8 is not seeded
    VmfDeferred df;
    df.need = false;
    float pdf = 0.0f;
    bool ok = false;
    if (mine) {
      const Ends e = load_ends(c, b);
      uint32_t tau = 0;
      float3 w;
      ok = draw_dir<kS>(S, gp, e, cell_of(c, b), e.tau, P.tau_random != 0, key, (uint64_t)b + offset, 0u, P, k, w,
                        tau, pdf, ctx.err, t.c, true, false, vmf ? &df : nullptr);
      // Eq. deduction with k at run time, each vertex stored as it is found
      float3 o = e.xD, d = w;
      for (int i = 0; ok && i < k; ++i) {
        Hit h = intersect<kS>(S, o, d, P.ray_eps, 3.0e38f, ctx.err, t.c);
        if (h.surf < 0) { ok = false; break; }
        const float3 x = hit_point(S, o, d, h);
        c.x[(3 * i + 0) * B + b] = x.x;
        c.x[(3 * i + 1) * B + b] = x.y;
        c.x[(3 * i + 2) * B + b] = x.z;
        c.surf[i * B + b] = h.surf;
        c.prim[i * B + b] = h.prim;
        c.bary[(2 * i + 0) * B + b] = h.b1;
        c.bary[(2 * i + 1) * B + b] = h.b2;
        if (i < k - 1) {
          float3 nrm = vertex_normal(S, h.surf, h.prim, x, h.b1, h.b2);
          float3 dn;
          if (!scatter(S.s[h.surf], nrm, d, (tau >> i) & 1u, dn)) { ok = false; break; }
          o = x;
          d = dn;
        }
      }
      if (!ok) {
        for (int i = 0; i < k; ++i) {
          c.x[(3 * i + 0) * B + b] = 0.f;
          c.x[(3 * i + 1) * B + b] = 0.f;
          c.x[(3 * i + 2) * B + b] = 0.f;
          c.surf[i * B + b] = -1;
          c.prim[i * B + b] = -1;
          c.bary[(2 * i + 0) * B + b] = 0.f;
          c.bary[(2 * i + 1) * B + b] = 0.f;
        }
      }
      c.tau[b] = (uint8_t)tau;
      c.status[b] = ok ? ST_SEEDED : ST_INVALID;
      c.iters[b] = 0;
    }
    if (vmf) {
      const float sum = vmf_sum_warp(g, ok && df.need, df);
      if (ok && df.need) pdf += (1.0f - P.alpha) * sum;
    }
    if (mine) c.pdf[b] = ok ? pdf : 0.0f;
  }
  if (kS) flush(t, ctx.stats);
}

}  // namespace kern

void launch_seed_all(const DScene& S, const DGuide* g, const DChains& c, uint2 key, uint64_t offset,
                     const mpg_params& P, DCtx ctx, int grid, cudaStream_t st) {
  DGuide gg = g ? *g : DGuide{};
  kern::k_seed_all<true><<<grid, 128, 0, st>>>(S, gg, g != nullptr, c, key, offset, P, ctx);
}

}  // namespace mpg
