// Kernel templates of the hot path, instantiated once per chain length K in
// mpg_k<K>.cu: seed sampling (K1), manifold walk (K2), contribution (K4) and
// Bernoulli trials (K5).  Each kernel is templated on K (registers sized for K
// vertices) and on whether it tallies work counters.
#pragma once

#include "mpg_ggt64.cuh"
#include "mpg_glossy.cuh"
#include "mpg_kernels.cuh"

namespace mpg {
namespace kern {


struct Tally {
  Counters c;
  uint32_t walks, conv, trials;
};

// Warp-reduced flush of the tallies into the family's counters (mpg_stats order).
__device__ __forceinline__ void flush(const Tally& t, unsigned long long* stats) {
  if (!stats) return;
  __syncwarp();
  uint32_t v[15] = {t.c.newton, t.c.rows, t.c.full_evals, t.c.c_evals, t.c.casts, t.c.sphere, t.c.plane,
                    t.c.node, t.c.tri, t.walks, t.conv, t.c.ggt, t.trials, t.c.seeds, t.c.ggt64};
#pragma unroll
  for (int i = 0; i < 15; ++i) {
    uint32_t s = __reduce_add_sync(0xffffffffu, v[i]);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(stats + i, (unsigned long long)s);
  }
}

template <int K>
__device__ __forceinline__ void load_chain(const DChains& c, int b, Chain<K>& ch) {
  const size_t B = (size_t)c.B;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    ch.x[i] = make_float3(c.x[(3 * i + 0) * B + b], c.x[(3 * i + 1) * B + b], c.x[(3 * i + 2) * B + b]);
    ch.surf[i] = c.surf[i * B + b];
    ch.prim[i] = c.prim[i * B + b];
    ch.b1[i] = c.bary[(2 * i + 0) * B + b];
    ch.b2[i] = c.bary[(2 * i + 1) * B + b];
  }
}

template <int K>
__device__ __forceinline__ void store_chain(const DChains& c, int b, const Chain<K>& ch) {
  const size_t B = (size_t)c.B;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    c.x[(3 * i + 0) * B + b] = ch.x[i].x;
    c.x[(3 * i + 1) * B + b] = ch.x[i].y;
    c.x[(3 * i + 2) * B + b] = ch.x[i].z;
    c.surf[i * B + b] = ch.surf[i];
    c.prim[i * B + b] = ch.prim[i];
    c.bary[(2 * i + 0) * B + b] = ch.b1[i];
    c.bary[(2 * i + 1) * B + b] = ch.b2[i];
  }
}

// Offset normals of glossy chain b (its K vertices' tangential components).
template <int K>
__device__ __forceinline__ void load_offsets(const DChains& c, int b, float2 (&off)[K]) {
  const size_t B = (size_t)c.B;
#pragma unroll
  for (int i = 0; i < K; ++i) off[i] = make_float2(c.offset[(2 * i + 0) * B + b], c.offset[(2 * i + 1) * B + b]);
}

__device__ __forceinline__ Ends load_ends(const DChains& c, int b) {
  Ends e;
  int q = b / c.spq;
  e.xD = make_float3(c.xD[q], c.xD[c.Q + q], c.xD[2 * c.Q + q]);
  e.nD = make_float3(c.nD[q], c.nD[c.Q + q], c.nD[2 * c.Q + q]);
  e.xL = make_float3(c.xL[b], c.xL[c.B + b], c.xL[2 * (size_t)c.B + b]);
  e.tau = c.tau[b];
  return e;
}

// Work item i of bucket K -> chain index, or -1 to skip.
template <int K>
__device__ __forceinline__ int item(const DWork& w, const DChains& c, int i) {
  if (w.order) return w.order[w.base[K] + i];
  return c.k[i] == K ? i : -1;
}
template <int K>
__device__ __forceinline__ int n_items(const DWork& w, const DChains& c) {
  return w.order ? w.count[K] : c.B;
}

// kHF: the scene may hold heightfields (intersect's BVH branch compiled in).
template <int K, bool kS, bool kHF>
__global__ void __launch_bounds__(128) k_seed(const __grid_constant__ DScene S, DGuide g, int has_guide, DChains c,
                                              DWork w, uint2 key, uint64_t offset, mpg_params P, DCtx ctx) {
  Tally t = {};
  const int n = n_items<K>(w, c);
  offset = rng_offset(offset, ctx);
  // with a vMF guide the lobe sum of each seed's density is taken by the whole
  // warp (vmf_sum_warp), so the loop runs warp-uniformly
  const bool vmf = has_guide && g.kind == MPG_GUIDE_VMF;
  const int lane = threadIdx.x & 31;
  for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += gridDim.x * blockDim.x) {
    const int i = base + lane;
    const int b = i < n ? item<K>(w, c, i) : -1;
    VmfDeferred df;
    df.need = false;
    Chain<K> ch;
    uint32_t tau = 0;
    float pdf = 0.0f;
    bool ok = false;
    if (b >= 0) {
      Ends e = load_ends(c, b);
      ok = draw_seed<K, kS, kHF ? BVH_CALL : BVH_NONE>(S, has_guide ? &g : nullptr, e, cell_of(c, b), e.tau, P.tau_random != 0, key,
                            (uint64_t)b + offset, 0u, P, ch, tau, pdf, ctx.err, t.c, true, false,
                            vmf ? &df : nullptr);
    }
    if (vmf) {
      const float s = vmf_sum_warp(g, ok && df.need, df);
      if (ok && df.need) pdf += (1.0f - P.alpha) * s;
    }
    if (b < 0) continue;
    if (!ok) {
#pragma unroll
      for (int v = 0; v < K; ++v) {
        ch.x[v] = make_float3(0.f, 0.f, 0.f);
        ch.surf[v] = -1; ch.prim[v] = -1; ch.b1[v] = 0.f; ch.b2[v] = 0.f;
      }
    }
    store_chain<K>(c, b, ch);
    c.tau[b] = (uint8_t)tau;
    c.pdf[b] = ok ? pdf : 0.0f;
    c.status[b] = ok ? ST_SEEDED : ST_INVALID;
    c.iters[b] = 0;
  }
  if (kS) flush(t, ctx.stats);
}

// kOff: glossy chains, walked to C_i = o_i with the chain's offset normals.
template <int K, bool kS, bool kOff>
__global__ void __launch_bounds__(128) k_walk(const __grid_constant__ DScene S, DChains c, DWork w, mpg_params P,
                                              DCtx ctx) {
  Tally t = {};
  const int n = n_items<K>(w, c);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int b = item<K>(w, c, i);
    if (b < 0 || c.status[b] != ST_SEEDED) continue;
    Chain<K> ch;
    load_chain<K>(c, b, ch);
    Ends e = load_ends(c, b);
    float2 off[K];
    if (kOff) load_offsets<K>(c, b, off);
    int it = 0;
    int st = walk<K, kS>(S, ch, e, P, it, ctx.err, t.c, kOff ? off : nullptr);
    t.walks++;
    t.conv += st == ST_CONVERGED;
    store_chain<K>(c, b, ch);
    c.status[b] = (uint8_t)st;
    c.iters[b] = (uint8_t)it;
  }
  if (kS) flush(t, ctx.stats);
}

template <int K, bool kS>
__global__ void __launch_bounds__(128) k_contrib(const __grid_constant__ DScene S, DChains c, DWork w, mpg_params P,
                                                 DOut o, DCtx ctx) {
  Tally t = {};
  const int n = n_items<K>(w, c);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int b = item<K>(w, c, i);
    if (b < 0) continue;
    float G = 0.f, kap = 0.f;
    bool adm = false;
    if (c.status[b] == ST_CONVERGED) {
      Chain<K> ch;
      load_chain<K>(c, b, ch);
      Ends e = load_ends(c, b);
      float mismatch = 0.0f, cmax = 0.0f, kerr = 0.0f, serr = 0.0f;
      adm = contribution<K, kS>(S, ch, e, P, G, kap, mismatch, cmax, kerr, serr, ctx.err, t.c);
      // Escalate to FP64 where FP32 is not enough: long chains, a geometry term
      // whose two reciprocal FP32 evaluations disagree, a transmittance at a
      // grazing cosine (FP32 rounding, or the walk's remaining step: that bound
      // is allowed five times fp64_tol), or a walk that stopped at the FP32
      // resolution of C.  The chain is queued for k_contrib64, which polishes
      // it and recomputes G and kappa in FP64.
      if (adm && (K >= fp64_k_of(P) || mismatch > P.fp64_tol || kerr > P.fp64_tol || serr > 5.0f * P.fp64_tol ||
                  !(cmax < P.tol)) && o.fp64_list) {
        o.fp64_list[*o.fp64_base + atomicAdd(o.fp64_count, 1)] = b;
        t.c.ggt64++;
      }
    }
    if (!adm) { G = 0.f; kap = 0.f; }
    if (o.G) o.G[b] = G;
    if (o.kappa) o.kappa[b] = kap;
    o.T[b] = kap * G * S.L.power;
  }
  if (kS) flush(t, ctx.stats);
}

// FP64 polish, G and kappa of the chains k_contrib queued (rare: near caustic
// folds, grazing transmission, stalled walks, k >= 6).  Writes back the
// polished vertices and the final G, kappa and T.  The queue is short (a few
// thousand chains) and each chain is a long serial FP64 computation with its
// arrays in local memory, so warps of 32 consecutive chains are dealt to the
// blocks in turn (the first warp of every block before any second warp): the
// work spreads over all SMs instead of filling the first few blocks.
template <int K>
__global__ void __launch_bounds__(64) k_contrib64(const __grid_constant__ DScene S, DChains c, mpg_params P, DOut o) {
  const int n = *o.fp64_count;
  const int* list = o.fp64_list + *o.fp64_base;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long first = ((long long)(threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32 + (threadIdx.x & 31);
  for (long long j = first; j < n; j += stride) {
    int b = list[j];
    Chain<K> ch;
    load_chain<K>(c, b, ch);
    Ends e = load_ends(c, b);
    Chain64<K> c64;
    to64<K>(S, ch, c64);
    double g, k64;
    float G = 0.f, kap = 0.f;
    if (polish_ggt64<K>(S, c64, e, (double)P.tol, (double)P.sing_eps, 3, g, k64)) {
      G = (float)g;
      kap = (float)k64;
#pragma unroll
      for (int v = 0; v < K; ++v) {
        ch.x[v] = make_float3((float)c64.x[v].x, (float)c64.x[v].y, (float)c64.x[v].z);
        ch.prim[v] = c64.prim[v];
        ch.b1[v] = (float)c64.b1[v];
        ch.b2[v] = (float)c64.b2[v];
      }
      store_chain<K>(c, b, ch);
    }
    if (o.G) o.G[b] = G;
    if (o.kappa) o.kappa[b] = kap;
    o.T[b] = kap * G * S.L.power;
  }
}

// k_contrib64 with one chain per group of G >= K lanes (polish_ggt64_g): the
// FP64 queue of long chains is short, and each chain's serial FP64 work shrinks
// by about K; groups are dealt to the blocks in turn as in k_contrib64.
template <int K, int G>
__global__ void __launch_bounds__(64) k_contrib64_g(const __grid_constant__ DScene S, DChains c, mpg_params P, DOut o) {
  static_assert(G >= K && G <= 32 && (G & (G - 1)) == 0, "group of a power of two >= K lanes");
  constexpr int NG = 64 / G;
  __shared__ VS64 sv[NG][K];
  const int n = *o.fp64_count;
  const int* list = o.fp64_list + *o.fp64_base;
  const int lane = threadIdx.x & 31, j = threadIdx.x % G, grp = threadIdx.x / G;
  const int leader = lane & ~(G - 1);
  const unsigned gmask = (G == 32 ? 0xffffffffu : ((1u << G) - 1u)) << leader;
  const size_t Bz = (size_t)c.B;
  for (long long q = (long long)grp * gridDim.x + blockIdx.x; q < n; q += (long long)gridDim.x * NG) {
    const int b = list[q];
    const Ends e = load_ends(c, b);
    int surf = 0, prim = 0;
    D3 x = D3{0.0, 0.0, 0.0};
    double b1 = 0.0, b2 = 0.0;
    if (j < K) {
      surf = c.surf[j * Bz + b];
      prim = c.prim[j * Bz + b];
      b1 = c.bary[(2 * j + 0) * Bz + b];
      b2 = c.bary[(2 * j + 1) * Bz + b];
      x = D3{(double)c.x[(3 * j + 0) * Bz + b], (double)c.x[(3 * j + 1) * Bz + b], (double)c.x[(3 * j + 2) * Bz + b]};
      const DSurf& sf = S.s[surf];
      if (sf.type == SURF_SPHERE || sf.type == SURF_CAP) x = d3(sf.c) + unit(x - d3(sf.c)) * (double)sf.r;
    }
    double g, k64;
    float G32 = 0.f, kap = 0.f;
    if (polish_ggt64_g<K, G>(S, j, gmask, surf, prim, x, b1, b2, e, (double)P.tol, (double)P.sing_eps, 3, sv[grp], g,
                             k64)) {
      G32 = (float)g;
      kap = (float)k64;
      if (j < K) {
        c.x[(3 * j + 0) * Bz + b] = (float)x.x;
        c.x[(3 * j + 1) * Bz + b] = (float)x.y;
        c.x[(3 * j + 2) * Bz + b] = (float)x.z;
        c.prim[j * Bz + b] = prim;
        c.bary[(2 * j + 0) * Bz + b] = (float)b1;
        c.bary[(2 * j + 1) * Bz + b] = (float)b2;
      }
    }
    if (j == 0) {
      if (o.G) o.G[b] = G32;
      if (o.kappa) o.kappa[b] = kap;
      o.T[b] = kap * G32 * S.L.power;
    }
  }
}

// Glossy contribution: admissibility (as for specular chains) and the
// estimate W of each converged glossy chain in FP64 after an FP64 polish to
// C = o (mpg_glossy.cuh), written as T; the polished vertices are written
// back; G and kappa are not formed for glossy chains (0).
template <int K, bool kS>
__global__ void __launch_bounds__(64) k_glossy(const __grid_constant__ DScene S, DChains c, DWork w, mpg_params P,
                                               DOut o, DCtx ctx) {
  Tally t = {};
  const int n = n_items<K>(w, c);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int b = item<K>(w, c, i);
    if (b < 0) continue;
    float T = 0.f;
    if (c.status[b] == ST_CONVERGED) {
      Chain<K> ch;
      load_chain<K>(c, b, ch);
      Ends e = load_ends(c, b);
      float2 off[K];
      load_offsets<K>(c, b, off);
      Chain64<K> c64;
      to64<K>(S, ch, c64);
      double W;
      if (admissible<K, kS>(S, ch, e, P, ctx.err, t.c) &&
          glossy_w64<K>(S, c64, e, off, (double)P.roughness, (double)P.tol, (double)P.sing_eps, W)) {
        T = (float)W;
        // the polished vertices replace the FP32 ones (the Bernoulli trials
        // compare against them)
#pragma unroll
        for (int v = 0; v < K; ++v) {
          ch.x[v] = make_float3((float)c64.x[v].x, (float)c64.x[v].y, (float)c64.x[v].z);
          ch.prim[v] = c64.prim[v];
          ch.b1[v] = (float)c64.b1[v];
          ch.b2[v] = (float)c64.b2[v];
        }
        store_chain<K>(c, b, ch);
      }
    }
    if (o.G) o.G[b] = 0.f;
    if (o.kappa) o.kappa[b] = 0.f;
    o.T[b] = T;
  }
  if (kS) flush(t, ctx.stats);
}

// kOff: glossy chains; every trial is walked with the chain's own offset
// normals, so N estimates the reciprocal probability given the offsets.
// kHF: the scene may hold heightfields (as for k_seed).
template <int K, bool kS, bool kOff, bool kHF>
__global__ void __launch_bounds__(128) k_bernoulli(const __grid_constant__ DScene S, DGuide g, int has_guide,
                                                   DChains c, DWork w, uint2 key, uint64_t offset, mpg_params P,
                                                   DOut o, DCtx ctx) {
  Tally t = {};
  const int n = n_items<K>(w, c);
  const double eps2 = (double)P.dedup_eps * (double)P.dedup_eps;
  offset = rng_offset(offset, ctx);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int b = item<K>(w, c, i);
    if (b < 0) continue;
    float T = o.T[b];
    uint32_t N = 0;  // summed over the repeats
    bool cap = false;
    if (T > 0.0f) {
      Chain<K> target;
      load_chain<K>(c, b, target);
      Ends e = load_ends(c, b);
      float2 off[K];
      if (kOff) load_offsets<K>(c, b, off);
      uint32_t cell = cell_of(c, b);
      for (int rep = 0; rep < o.repeats; ++rep) {
        bool cap_r = true;
        for (int tr = 1; tr <= P.max_trials; ++tr) {
          t.trials++;
          Chain<K> ch;
          uint32_t tau;
          float pdf;
          Ends et = e;
          if (!draw_seed<K, kS, kHF ? BVH_CALL : BVH_NONE>(S, has_guide ? &g : nullptr, e, cell, e.tau, P.tau_random != 0, key,
                                (uint64_t)b + offset, (uint32_t)tr | ((uint32_t)rep << 24), P, ch, tau, pdf, ctx.err,
                                t.c, false, true))
            continue;
          if (tau != e.tau) continue;  // a different type sequence cannot be the same solution
          et.tau = tau;
          int it;
          int st = walk<K, kS>(S, ch, et, P, it, ctx.err, t.c, kOff ? off : nullptr);
          t.walks++;
          t.conv += st == ST_CONVERGED;
          if (st == ST_CONVERGED && same_solution<K>(ch, target, eps2)) {
            N += (uint32_t)tr;
            cap_r = false;
            break;
          }
        }
        if (cap_r) N += (uint32_t)P.max_trials;
        cap = cap || cap_r;
      }
    }
    DOut one = o;  // the sum over all repeats is written at once
    one.rep = 0;
    bern_write(S.L.area, c, one, b, T, N, cap);
  }
  if (kS) flush(t, ctx.stats);
}


}  // namespace kern
}  // namespace mpg

#include "mpg_persistent.cuh"

namespace mpg {

template <int K>
void KLaunch<K>::walk_p(bool stats, const DScene& S, const DChains& c, DWork w, const mpg_params& P, DCtx ctx,
                        int* queue, int grid, int block, cudaStream_t st) {
  kern::k_walk_p<K, true><<<grid, block, 0, st>>>(S, c, w, P, ctx, queue);
}

template <int K>
void KLaunch<K>::walk_g(bool stats, const DScene& S, const DChains& c, DWork w, const mpg_params& P, DCtx ctx,
                        int* queue, int grid, cudaStream_t st) {
  if constexpr (K == 1) {
    kern::k_walk_p<K, true><<<grid, 128, 0, st>>>(S, c, w, P, ctx, queue);
  } else {
    constexpr int G = K <= 2 ? 2 : K <= 4 ? 4 : 8;
    kern::k_walk_g<K, G, true><<<grid, 128, 0, st>>>(S, c, w, P, ctx, queue);
  }
}

template <int K>
void KLaunch<K>::contrib64(const DScene& S, const DChains& c, const mpg_params& P, DOut o, int grid, cudaStream_t st) {
  // one chain per lane group from three vertices on (K <= 2: a thread per chain)
  constexpr int G = K <= 2 ? 1 : K <= 4 ? 4 : 8;
  if constexpr (G == 1) kern::k_contrib64<K><<<grid, 64, 0, st>>>(S, c, P, o);
  else kern::k_contrib64_g<K, G><<<grid, 64, 0, st>>>(S, c, P, o);
}

template <int K>
void KLaunch<K>::trial_init(const DScene& S, const DChains& c, DWork w, DOut o, int* list, const int* base,
                            int* n_list, unsigned* nbest, int grid, cudaStream_t st) {
  kern::k_trial_init<K><<<grid, 256, 0, st>>>(S, c, w, o, list, base, n_list, nbest);
}

template <int K>
void KLaunch<K>::trial_seed(const DScene& S, const DGuide* g, const DChains& c, const DChains& tc, const int* list,
                            const int* base, const int* n_list, uint2 key, uint64_t offset, const mpg_params& P,
                            DCtx ctx, int t, int grid, int block, cudaStream_t st) {
  DGuide gg = g ? *g : DGuide{};
  kern::k_trial_seed<K, true><<<grid, block, 0, st>>>(S, gg, g != nullptr, c, tc, list, base, n_list, key, offset, P,
                                                       ctx, t);
}

template <int K>
void KLaunch<K>::trial_check(const DScene& S, const DChains& c, const DChains& tc, DOut o, const int* list,
                             const int* base, const int* n_list, int t, int last, const mpg_params& P, int* next,
                             int* n_next, unsigned* nbest, int grid, cudaStream_t st) {
  kern::k_trial_check<K><<<grid, 256, 0, st>>>(S, c, tc, o, list, base, n_list, t, last, P, next, n_next, nbest);
}

template <int K>
void KLaunch<K>::bern_round(bool stats, const DScene& S, const DGuide* g, const DChains& c, uint2 key, uint64_t offset,
                            const mpg_params& P, DCtx ctx, int* queue, const int* list, const int* n_list,
                            const int* base, unsigned* nbest, int t0, int TB, DPairs pr, int grid, int block,
                            cudaStream_t st) {
  DGuide gg = g ? *g : DGuide{};
  if constexpr (K > 1) {
    if (P.walk_group & 2) {
      constexpr int G = K <= 2 ? 2 : K <= 4 ? 4 : 8;
      kern::k_bern_round_g<K, G, true><<<grid, 128, 0, st>>>(S, gg, g != nullptr, c, key, offset, P, ctx, queue, list,
                                                             n_list, base, nbest, t0, TB, pr);
      return;
    }
  }
  kern::k_bern_round<K, true><<<grid, block, 0, st>>>(S, gg, g != nullptr, c, key, offset, P, ctx, queue, list,
                                                         n_list, base, nbest, t0, TB, pr);
}

template <int K>
void KLaunch<K>::seed(bool stats, const DScene& S, const DGuide* g, const DChains& c, DWork w, uint2 key,
                      uint64_t offset, const mpg_params& P, DCtx ctx, int grid, int block, cudaStream_t st) {
  DGuide gg = g ? *g : DGuide{};
  if (S.n_hf > 0) kern::k_seed<K, true, true><<<grid, block, 0, st>>>(S, gg, g != nullptr, c, w, key, offset, P, ctx);
  else kern::k_seed<K, true, false><<<grid, block, 0, st>>>(S, gg, g != nullptr, c, w, key, offset, P, ctx);
}

template <int K>
void KLaunch<K>::walk(bool stats, const DScene& S, const DChains& c, DWork w, const mpg_params& P, DCtx ctx, int grid,
                      int block, cudaStream_t st) {
  if (c.offset) kern::k_walk<K, true, true><<<grid, block, 0, st>>>(S, c, w, P, ctx);
  else kern::k_walk<K, true, false><<<grid, block, 0, st>>>(S, c, w, P, ctx);
}

template <int K>
void KLaunch<K>::glossy(const DScene& S, const DChains& c, DWork w, const mpg_params& P, DOut o, DCtx ctx, int grid,
                        cudaStream_t st) {
  kern::k_glossy<K, true><<<grid, 64, 0, st>>>(S, c, w, P, o, ctx);
}

template <int K>
void KLaunch<K>::contrib(bool stats, const DScene& S, const DChains& c, DWork w, const mpg_params& P, DOut o, DCtx ctx,
                         int grid, int block, cudaStream_t st) {
  kern::k_contrib<K, true><<<grid, block, 0, st>>>(S, c, w, P, o, ctx);
}

template <int K>
void KLaunch<K>::bernoulli(bool stats, const DScene& S, const DGuide* g, const DChains& c, DWork w, uint2 key,
                           uint64_t offset, const mpg_params& P, DOut o, DCtx ctx, int grid, int block,
                           cudaStream_t st) {
  DGuide gg = g ? *g : DGuide{};
  const bool hf = S.n_hf > 0;
  if (c.offset && hf)
    kern::k_bernoulli<K, true, true, true><<<grid, block, 0, st>>>(S, gg, g != nullptr, c, w, key, offset, P, o, ctx);
  else if (c.offset)
    kern::k_bernoulli<K, true, true, false><<<grid, block, 0, st>>>(S, gg, g != nullptr, c, w, key, offset, P, o, ctx);
  else if (hf)
    kern::k_bernoulli<K, true, false, true><<<grid, block, 0, st>>>(S, gg, g != nullptr, c, w, key, offset, P, o, ctx);
  else
    kern::k_bernoulli<K, true, false, false><<<grid, block, 0, st>>>(S, gg, g != nullptr, c, w, key, offset, P, o, ctx);
}

template <int K>
int KLaunch<K>::blocks_per_sm(int which, bool stats, int block) {
  const void* fn;
  if (which == 0) fn = (const void*)kern::k_seed<K, true, true>;
  else if (which == 1) fn = (const void*)kern::k_walk<K, true, false>;
  else if (which == 2) fn = (const void*)kern::k_contrib<K, true>;
  else if (which == 3) fn = (const void*)kern::k_bernoulli<K, true, false, true>;
  else if (which == 4) fn = (const void*)kern::k_walk_p<K, true>;
  else if (which == 5) fn = (const void*)kern::k_trial_seed<K, true>;
  else if (which == 7) {
    if constexpr (K == 1) fn = (const void*)kern::k_walk_p<K, true>;
    else fn = (const void*)kern::k_walk_g<K, (K <= 2 ? 2 : K <= 4 ? 4 : 8), true>;
  } else if (which == 8) {
    if constexpr (K == 1) fn = (const void*)kern::k_bern_round<K, true>;
    else fn = (const void*)kern::k_bern_round_g<K, (K <= 2 ? 2 : K <= 4 ? 4 : 8), true>;
  }
  else fn = (const void*)kern::k_bern_round<K, true>;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, 0) != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

}  // namespace mpg
