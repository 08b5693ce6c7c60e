// Persistent work-queue kernels of the batched mode.
//
// A thread keeps one chain (or one Bernoulli trial) in registers and advances
// it by one line-search attempt per pass; each attempt evaluates constraint
// and Jacobian blocks at its candidate, so every lane of a warp runs the same
// instructions in a pass whatever state its walk is in.  A lane whose walk ends takes
// the next item of the launch's queue in the same pass (warp-aggregated
// atomic), so a warp stays full until the queue is empty instead of waiting
// for its slowest chain.  All loops are bounded: each pass either consumes a
// queue item or advances a walk, and walks end after max_iter steps.
#pragma once

#include "mpg_ggt64.cuh"
#include "mpg_kernels.cuh"

namespace mpg {
namespace kern {

constexpr int RUNNING = -1;

// Resident CTAs of 128 threads per SM the one-thread-per-chain kernels are
// compiled for: the register need grows with K (about 128 registers at
// K <= 2, 168 at K <= 4, the 255 maximum beyond), and a tighter bound spills.
template <int K>
constexpr int walk_min_ctas() { return K <= 2 ? 4 : K <= 4 ? 3 : 2; }

// float3 from the previous / next lane of a segment of `width` lanes (the lane
// itself at the segment's start / end); `mask` holds the segment's lanes.
__device__ __forceinline__ float3 shfl_up3(unsigned mask, float3 v, int width) {
  return make_float3(__shfl_up_sync(mask, v.x, 1, width), __shfl_up_sync(mask, v.y, 1, width),
                     __shfl_up_sync(mask, v.z, 1, width));
}
__device__ __forceinline__ float3 shfl_down3(unsigned mask, float3 v, int width) {
  return make_float3(__shfl_down_sync(mask, v.x, 1, width), __shfl_down_sync(mask, v.y, 1, width),
                     __shfl_down_sync(mask, v.z, 1, width));
}

template <int K>
struct WalkLane {
  Chain<K> ch;
  Ends e;
  float3 d[K];  // Newton step of each vertex (tangent vector), kept through the halvings
  float cn2, cmax, beta;
  int it, hv;
  bool need_eval;  // the walk has not evaluated its seed yet
};

template <int K>
__device__ __forceinline__ void walk_begin(WalkLane<K>& w) {
  w.it = 0;
  w.hv = 0;
  w.beta = 1.0f;
  w.need_eval = true;
}

// One pass of the walk in fused form: every attempt evaluates the constraint
// together with its Jacobian blocks at the candidate, so that each pass runs
// the same instructions in every lane (a two-phase pass, Jacobian after an
// accepted step and constraint-only line-search attempts otherwise, leaves the
// lanes in the other phase waiting).  The first pass of a walk evaluates the seed itself; a candidate is
// accepted when its |C|^2 is below the current one, and the blocks already
// evaluated there give the next Newton direction.  The constraint values are
// those of the two-phase form (vertex_c and vertex_blocks form C with the same
// operations), so the decisions are the same as walk<K>()'s.  A rejected
// candidate costs a full evaluation instead of a constraint-only one; the
// counters record only the constraint evaluation it needed.
template <int K, bool kS>
__device__ __forceinline__ int walk_pass_fused(const DScene& S, WalkLane<K>& w, const mpg_params& P, Counters& cnt,
                                               int attempts = 1) {
  for (int a = 0; a < attempts; ++a) {
    const bool first = w.need_eval;
    Chain<K> cand;
    bool ok = true;
    if (first) cand = w.ch;
    else ok = propose<K>(S, w.ch, w.d, w.beta, cand);
    VB vb[K];
    float3 tu[K], tv[K];
    float c2 = 0.0f, cm = 0.0f;
    ok = ok && eval_full<K, false>(S, cand, w.e, vb, tu, tv, c2, cm, false, cnt);
    if (ok && (first || c2 < w.cn2)) {
      if (kS) cnt.full_evals += K;
      w.ch = cand;
      w.it += first ? 0 : 1;
      w.need_eval = false;
      w.cn2 = c2;
      w.cmax = cm;
      if (cm < P.tol) return ST_CONVERGED;
      if (w.it >= P.max_iter) return cm < P.stall_tol ? ST_CONVERGED : ST_LIMIT;
      float2 du[K][1];
#pragma unroll
      for (int i = 0; i < K; ++i) du[i][0] = make_float2(-vb[i].C.x, -vb[i].C.y);
      if (kS) { cnt.newton++; cnt.rows += K; }
      if (!thomas<K, 1>(vb, du, P.sing_eps)) return ST_FAILED;
      step_vectors<K>(tu, tv, du, w.d);
      w.beta = 1.0f;
      w.hv = 0;
      return RUNNING;
    }
    if (first) return ST_FAILED;  // the seed chain itself cannot be evaluated
    if (kS && ok) cnt.c_evals += K;
    w.hv++;
    w.beta *= 0.5f;
    if (w.hv > P.max_halvings) return w.cmax < P.stall_tol ? ST_CONVERGED : ST_FAILED;
  }
  return RUNNING;
}

// Line-search attempts per pass once a launch's work queue is empty.
constexpr int TAIL_ATTEMPTS = 4;

// Warp-aggregated take of one queue item per lane that asks for one.  Returns
// the lane's item index (or -1) and sets `done` (warp-uniform) once the queue
// holds no more items.
__device__ __forceinline__ int take_item(bool want, int* queue, int n, bool& done) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  unsigned need = __ballot_sync(FULL, want);
  if (!need || done) return -1;
  int base = 0;
  if (lane == 0) base = atomicAdd(queue, __popc(need));
  base = __shfl_sync(FULL, base, 0);
  if (base + __popc(need) >= n) done = true;
  if (!want) return -1;
  int i = base + __popc(need & ((1u << lane) - 1u));
  return i < n ? i : -1;
}

// The same over a 64-bit item space (parallel Bernoulli rounds: chains x trials).
__device__ __forceinline__ long long take_item64(bool want, unsigned long long* queue, long long n, bool& done) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  unsigned need = __ballot_sync(FULL, want);
  if (!need || done) return -1;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(queue, (unsigned long long)__popc(need));
  base = __shfl_sync(FULL, base, 0);
  if ((long long)base + __popc(need) >= n) done = true;
  if (!want) return -1;
  long long i = (long long)base + __popc(need & ((1u << lane) - 1u));
  return i < n ? i : -1;
}

// ---------------------------------------------------------------------------
// Walk (K2): one lane per chain, refilled from the bucket's queue.
// ---------------------------------------------------------------------------
template <int K, bool kS>
__global__ void __launch_bounds__(128, walk_min_ctas<K>()) k_walk_p(const __grid_constant__ DScene S_, DChains c, DWork w, mpg_params P,
                                                DCtx ctx, int* queue) {
  __shared__ DScene s_scene;
  const DScene& S = scene_in_smem(S_, s_scene);
  Tally t = {};
  const int n = n_items<K>(w, c);
  WalkLane<K> L;
  L.need_eval = false;
  int b = -1;
  bool done = false;
  const unsigned FULL = 0xffffffffu;
  const int refill = P.refill_every > 1 ? P.refill_every : 1;
  int pass = 0;
  while (true) {
    // idle lanes refill every `refill` passes, or at once when the whole warp is idle
    bool idle_warp = __all_sync(FULL, b < 0);
    int i = take_item(b < 0 && (idle_warp || pass % refill == 0), queue, n, done);
    ++pass;
    if (i >= 0) {
      int bb = item<K>(w, c, i);
      if (bb >= 0 && c.status[bb] == ST_SEEDED) {
        b = bb;
        load_chain<K>(c, b, L.ch);
        L.e = load_ends(c, b);
        walk_begin(L);
      }
    }
    bool any = __any_sync(FULL, b >= 0);
    if (!any && done) break;
    if (b >= 0) {
      int st = walk_pass_fused<K, kS>(S, L, P, t.c, done ? TAIL_ATTEMPTS : 1);
      if (st != RUNNING) {
        t.walks++;
        t.conv += st == ST_CONVERGED;
        store_chain<K>(c, b, L.ch);
        c.status[b] = (uint8_t)st;
        c.iters[b] = (uint8_t)L.it;
        b = -1;
      }
    }
  }
  if (kS) flush(t, ctx.stats);
}

// ---------------------------------------------------------------------------
// Walk (K2), one chain per thread group: lane j of a group of G >= K lanes
// owns vertex j (its position, surface coordinates and step vector); the
// neighbours' positions and tangent bases come by shuffles within the group,
// and each lane stages its vertex's 2x2 blocks and constraint in shared
// memory, where every lane of the group reads all of them and runs the same
// block Thomas sweep.  Per vertex the arithmetic is that of walk_pass_fused() and
// the sums over vertices are taken in the same order (the compiler may still
// contract some products differently, so the two forms agree to FP32
// rounding); the group form cuts the latency of a pass by up to K, at the
// price of idle lanes for K < G and of the staging.
// ---------------------------------------------------------------------------
template <int K>
struct GroupLane {
  float3 x, d;  // own vertex and its Newton step
  int surf, prim;
  float b1, b2;
  Ends e;
  float cn2, cmax, beta;
  int it, hv;
  bool need_eval;
};

// One pass of the group walk (the group form of walk_pass_fused): every attempt
// reprojects the group's vertices, evaluates frames, blocks and constraint at
// the candidate and stages them, so that all groups of a warp run the same
// instructions in each pass; an accepted candidate's blocks give the next
// Newton direction.  Per vertex the arithmetic and the decisions are those
// of walk_pass_fused.
template <int K, int G, bool kS>
__device__ __forceinline__ int walk_pass_g_fused(const DScene& S, GroupLane<K>& w, const mpg_params& P, Counters& cnt,
                                                 unsigned gmask, int j, float2* sC, float4* sA, float4* sB,
                                                 float4* sCc, int attempts = 1) {
  const bool own = j < K;
  for (int a = 0; a < attempts; ++a) {
    const bool first = w.need_eval;  // the same in every lane of the group
    float3 cx = w.x;
    int cprim = w.prim;
    float cb1 = w.b1, cb2 = w.b2;
    bool ok = true;
    if (!first && own) ok = reproject(S, w.surf, w.x + w.d * w.beta, cx, cprim, cb1, cb2);
    ok = __all_sync(gmask, ok);
    bool evaluated = false, accept = false;
    VB blk[K];
    float2 du[K][1];
    float cn2 = 0.0f, cmax = 0.0f;
    float3 tu = make_float3(0.f, 0.f, 0.f), tv = tu;
    if (ok) {
      Frame fr = {};
      if (own) fr = vertex_frame(S, w.surf, cprim, cx, cb1, cb2);
      tu = fr.dpdu;
      tv = fr.dpdv;
      float3 xp = shfl_up3(gmask, cx, G), xn = shfl_down3(gmask, cx, G);
      float3 pu = shfl_up3(gmask, tu, G), pv = shfl_up3(gmask, tv, G);
      float3 nu = shfl_down3(gmask, tu, G), nv = shfl_down3(gmask, tv, G);
      if (j == 0) xp = w.e.xD;
      if (j == K - 1) xn = w.e.xL;
      VB vb;
      bool okb = !own || vertex_blocks(xp, pu, pv, cx, fr, xn, nu, nv, S.s[w.surf], (w.e.tau >> j) & 1u, j > 0,
                                       j < K - 1, vb);
      if (__all_sync(gmask, okb)) {
        if (own) { sC[j] = vb.C; sA[j] = vb.A; sB[j] = vb.B; sCc[j] = vb.Cc; }
        __syncwarp(gmask);
#pragma unroll
        for (int i = 0; i < K; ++i) {
          blk[i].C = sC[i]; blk[i].A = sA[i]; blk[i].B = sB[i]; blk[i].Cc = sCc[i];
          cn2 = fmaf(blk[i].C.x, blk[i].C.x, fmaf(blk[i].C.y, blk[i].C.y, cn2));
          cmax = fmaxf(cmax, fmaxf(fabsf(blk[i].C.x), fabsf(blk[i].C.y)));
          du[i][0] = make_float2(-blk[i].C.x, -blk[i].C.y);
        }
        __syncwarp(gmask);  // the staging area is rewritten by the next evaluation
        evaluated = true;
        accept = first || cn2 < w.cn2;
      }
    }
    if (accept) {
      if (kS && j == 0) cnt.full_evals += K;
      w.x = cx; w.prim = cprim; w.b1 = cb1; w.b2 = cb2;
      w.it += first ? 0 : 1;
      w.need_eval = false;
      w.cn2 = cn2;
      w.cmax = cmax;
      if (cmax < P.tol) return ST_CONVERGED;
      if (w.it >= P.max_iter) return cmax < P.stall_tol ? ST_CONVERGED : ST_LIMIT;
      if (kS && j == 0) { cnt.newton++; cnt.rows += K; }
      if (!thomas<K, 1>(blk, du, P.sing_eps)) return ST_FAILED;
#pragma unroll
      for (int i = 0; i < K; ++i)
        if (i == j) w.d = tu * du[i][0].x + tv * du[i][0].y;
      w.beta = 1.0f;
      w.hv = 0;
      return RUNNING;
    }
    if (first) return ST_FAILED;  // the seed chain itself cannot be evaluated
    if (kS && j == 0 && evaluated) cnt.c_evals += K;
    w.hv++;
    w.beta *= 0.5f;
    if (w.hv > P.max_halvings) return w.cmax < P.stall_tol ? ST_CONVERGED : ST_FAILED;
  }
  return RUNNING;
}

template <int K, int G, bool kS>
__global__ void __launch_bounds__(128) k_walk_g(const __grid_constant__ DScene S_, DChains c, DWork w, mpg_params P,
                                                DCtx ctx, int* queue) {
  __shared__ DScene s_scene;
  const DScene& S = scene_in_smem(S_, s_scene);
  static_assert(G >= K && G <= 32 && (G & (G - 1)) == 0, "group of a power of two >= K lanes");
  constexpr int NG = 128 / G;
  __shared__ float2 sC[NG][K];
  __shared__ float4 sA[NG][K], sB[NG][K], sCc[NG][K];
  Tally t = {};
  const int n = n_items<K>(w, c);
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, j = threadIdx.x % G, grp = threadIdx.x / G;
  const int leader = lane & ~(G - 1);
  const unsigned gmask = (G == 32 ? FULL : ((1u << G) - 1u)) << leader;
  const size_t Bz = (size_t)c.B;
  GroupLane<K> L;
  L.need_eval = false;
  int b = -1;  // the group's chain (the same in every lane of the group)
  bool done = false;
  const int refill = P.refill_every > 1 ? P.refill_every : 1;
  int pass = 0;
  while (true) {
    bool idle_warp = __all_sync(FULL, b < 0);
    int i = take_item(j == 0 && b < 0 && (idle_warp || pass % refill == 0), queue, n, done);
    i = __shfl_sync(FULL, i, leader);
    ++pass;
    if (i >= 0) {
      int bb = item<K>(w, c, i);
      if (bb >= 0 && c.status[bb] == ST_SEEDED) {
        b = bb;
        if (j < K) {
          L.x = make_float3(c.x[(3 * j + 0) * Bz + b], c.x[(3 * j + 1) * Bz + b], c.x[(3 * j + 2) * Bz + b]);
          L.surf = c.surf[j * Bz + b];
          L.prim = c.prim[j * Bz + b];
          L.b1 = c.bary[(2 * j + 0) * Bz + b];
          L.b2 = c.bary[(2 * j + 1) * Bz + b];
        }
        L.e = load_ends(c, b);
        L.it = 0;
        L.hv = 0;
        L.beta = 1.0f;
        L.need_eval = true;
      }
    }
    bool any = __any_sync(FULL, b >= 0);
    if (!any && done) break;
    if (b >= 0) {
      int st = walk_pass_g_fused<K, G, kS>(S, L, P, t.c, gmask, j, sC[grp], sA[grp], sB[grp], sCc[grp],
                                           done ? TAIL_ATTEMPTS : 1);
      if (st != RUNNING) {
        if (j < K) {
          c.x[(3 * j + 0) * Bz + b] = L.x.x;
          c.x[(3 * j + 1) * Bz + b] = L.x.y;
          c.x[(3 * j + 2) * Bz + b] = L.x.z;
          c.surf[j * Bz + b] = L.surf;
          c.prim[j * Bz + b] = L.prim;
          c.bary[(2 * j + 0) * Bz + b] = L.b1;
          c.bary[(2 * j + 1) * Bz + b] = L.b2;
        }
        if (j == 0) {
          t.walks++;
          t.conv += st == ST_CONVERGED;
          c.status[b] = (uint8_t)st;
          c.iters[b] = (uint8_t)L.it;
        }
        b = -1;
      }
    }
  }
  if (kS) flush(t, ctx.stats);
}

// ---------------------------------------------------------------------------
// Bernoulli trials (K5) in synchronous rounds: round t draws trial t for every
// chain still without a hit (k_trial_seed), the persistent walk kernel walks
// them all, and k_trial_check retires the hits and compacts the rest.  Each
// kernel is uniform across lanes; the trial index of a chain's first hit is
// the same as in a sequential loop over t.
// ---------------------------------------------------------------------------

// Chains of this length with a contribution enter the rounds; the others get
// their final (zero) outputs.
template <int K>
__global__ void __launch_bounds__(256) k_trial_init(const __grid_constant__ DScene S, DChains c, DWork w, DOut o,
                                                    int* list, const int* base, int* n_list, unsigned* nbest) {
  const int n = n_items<K>(w, c);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int b = item<K>(w, c, i);
    if (b < 0) continue;
    if (o.T[b] > 0.0f) {
      list[base[K] + atomicAdd(n_list + K, 1)] = b;
      nbest[b] = 0xffffffffu;  // no success yet
    } else {
      bern_write(S.L.area, c, o, b, 0.0f, 0, false);
    }
  }
}

// Trial t of every listed chain: a fresh seed from the same distribution and
// length (Sec. 5.8, n reused), written to the trial state; a seed with another type
// sequence cannot reach the same solution and is marked invalid.
template <int K, bool kS>
__global__ void __launch_bounds__(128) k_trial_seed(const __grid_constant__ DScene S, DGuide g, int has_guide,
                                                    DChains c, DChains tc, const int* list, const int* base,
                                                    const int* n_list, uint2 key, uint64_t offset, mpg_params P,
                                                    DCtx ctx, int t) {
  Tally tl = {};
  const int n = n_list[K];
  offset = rng_offset(offset, ctx);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    int b = list[base[K] + j];
    Ends e = load_ends(c, b);
    Chain<K> ch;
    uint32_t tau;
    float pdf;
    tl.trials++;
    bool ok = draw_seed<K, kS>(S, has_guide ? &g : nullptr, e, cell_of(c, b), e.tau,
                               P.tau_random != 0, key, (uint64_t)b + offset, (uint32_t)t | ctx.trial_base, P, ch, tau,
                               pdf, ctx.err, tl.c, false, true) &&
              tau == e.tau;
    if (ok) store_chain<K>(tc, b, ch);
    tc.status[b] = ok ? ST_SEEDED : ST_INVALID;
  }
  if (kS) flush(tl, ctx.stats);
}

// Retire the chains whose trial t walked to their own solution (FP64 distance
// test); the others move to the next list.  After the last sequential round
// the next list feeds the speculative rounds (nbest reset).
template <int K>
__global__ void __launch_bounds__(256) k_trial_check(const __grid_constant__ DScene S, DChains c, DChains tc, DOut o,
                                                     const int* list, const int* base, const int* n_list, int t,
                                                     int last, mpg_params P, int* next, int* n_next, unsigned* nbest) {
  const int n = n_list[K];
  const double eps2 = (double)P.dedup_eps * (double)P.dedup_eps;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    int b = list[base[K] + j];
    bool hit = false;
    if (tc.status[b] == ST_CONVERGED) {
      Chain<K> a, ref;
      load_chain<K>(tc, b, a);
      load_chain<K>(c, b, ref);
      hit = same_solution<K>(a, ref, eps2);
    }
    if (hit) {
      bern_write(S.L.area, c, o, b, o.T[b], (uint32_t)t, false);
    } else if (t >= P.max_trials) {
      bern_write(S.L.area, c, o, b, o.T[b], (uint32_t)P.max_trials, true);
    } else {
      next[base[K] + atomicAdd(n_next + K, 1)] = b;
      if (last) nbest[b] = 0xffffffffu;
    }
  }
}

// ---------------------------------------------------------------------------
// Parallel Bernoulli rounds: trials t0 .. t0+TB-1 of every listed chain run as
// independent items; the first success is the smallest successful index
// (atomicMin), exactly as a sequential loop would find.  Items are issued
// trial-major (trial t0 of every chain, then trial t0+1, ...), so by the time a
// chain's later trials are taken its earlier ones have mostly finished, and
// items above a chain's best success so far are skipped: the speculative work
// is bounded by the items in flight, not by TB.
// ---------------------------------------------------------------------------
// Item filter of the parallel rounds.  Item i is trial tt of chain bb (the
// trial-major order above).  It is dropped when tt is past the trial cap or
// not below the chain's best success so far, and -- for seeds whose types are
// drawn at random from the first counter block (p_0 and histogram guides) --
// when that draw gives a type sequence other than the chain's: draw_seed
// fails such a trial before any ray is cast, so it never needs a walking lane.
struct BernFilter {
  const int* over;
  int nl, t0;
  unsigned* nbest;
  uint64_t offset;
  uint32_t trial_base;
  bool types;  // the type test applies (random types, no vMF guide)
};

template <int K, bool kS>
__device__ __forceinline__ bool bern_keep(const DChains& c, const BernFilter& f, uint2 key, const mpg_params& P,
                                          long long i, Tally& t) {
  const int bb = f.over[i % f.nl];
  const int tt = f.t0 + (int)(i / f.nl);
  if (tt > P.max_trials || (unsigned)tt >= *((volatile unsigned*)(f.nbest + bb))) return false;
  t.trials++;
  if (!f.types) return true;
  const uint64_t idx = (uint64_t)bb + f.offset;
  const uint4 r1 = philox(make_uint4((uint32_t)idx, (uint32_t)(idx >> 32), (uint32_t)tt | f.trial_base, 1u), key);
  if ((r1.y & ((1u << K) - 1u)) == (uint32_t)c.tau[bb]) return true;
  if (kS) t.c.seeds++;  // the seed was drawn (its types) and failed
  return false;
}

// Filter sweeps per pass at most (each takes one item per free pool slot).
constexpr int POOL_SWEEPS = 8;

// Warp-collective take from a per-warp pool of filtered items (pool[0..np)
// in shared memory, np warp-uniform).  While the pool holds fewer items than
// lanes asking (`want`), every lane with a free slot takes one raw item from
// the queue and filters it, and the survivors are appended; the asking lanes
// then take items from the top of the pool.  Returns the lane's item or -1.
// The pool only changes which lane walks which trial and when: the outputs
// (the smallest successful trial of each chain, and the walks below it) are
// the same.
template <int K, bool kS>
__device__ __forceinline__ long long bern_pool_take(bool want, long long* pool, int& np,
                                                    unsigned long long* queue64, long long n, bool& done,
                                                    const DChains& c, const BernFilter& f, uint2 key,
                                                    const mpg_params& P, Tally& t) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const unsigned need = __ballot_sync(FULL, want);
  const int nneed = __popc(need);
  for (int s = 0; s < POOL_SWEEPS && np < nneed && !done; ++s) {
    long long i = take_item64(lane >= np, queue64, n, done);
    const bool keep = i >= 0 && bern_keep<K, kS>(c, f, key, P, i, t);
    const unsigned km = __ballot_sync(FULL, keep);
    if (keep) pool[np + __popc(km & lt)] = i;  // slots np.. (at most 32 - np survivors)
    np += __popc(km);
  }
  __syncwarp();
  const int give = min(nneed, np);
  const int rank = __popc(need & lt);
  long long mine = -1;
  if (want && rank < give) mine = pool[np - 1 - rank];
  np -= give;
  __syncwarp();  // the slots handed out are rewritten by the next sweep
  return mine;
}

template <int K, bool kS>
__global__ void __launch_bounds__(128, walk_min_ctas<K>()) k_bern_round(const __grid_constant__ DScene S_, DGuide g, int has_guide,
                                                    DChains c, uint2 key, uint64_t offset, mpg_params P, DCtx ctx,
                                                    int* queue, const int* list, const int* n_list, const int* base,
                                                    unsigned* nbest, int t0, int TB, DPairs pr) {
  __shared__ DScene s_scene;
  const DScene& S = scene_in_smem(S_, s_scene);
  __shared__ long long pools[4][32];
  Tally t = {};
  const double eps2 = (double)P.dedup_eps * (double)P.dedup_eps;
  const int* over = list + *base;
  const int nl = *n_list;
  const long long n = (long long)nl * TB;
  unsigned long long* queue64 = reinterpret_cast<unsigned long long*>(queue);
  offset = rng_offset(offset, ctx);
  const BernFilter f{over, nl, t0, nbest, offset, ctx.trial_base,
                     P.tau_random != 0 && !(has_guide && g.kind == MPG_GUIDE_VMF)};
  long long* pool = pools[threadIdx.x >> 5];
  int np = 0;
  const int refill = P.refill_every > 1 ? P.refill_every : 1;
  int pass = 0;
  WalkLane<K> L;
  L.need_eval = false;
  Chain<K> target;
  int b = -1, tr = 0;
  bool done = false;
  const unsigned FULL = 0xffffffffu;
  while (true) {
    // idle lanes refill every `refill` passes, or at once when the whole warp is idle
    bool idle_warp = __all_sync(FULL, b < 0);
    long long i = bern_pool_take<K, kS>(b < 0 && (idle_warp || pass % refill == 0), pool, np, queue64, n, done, c,
                                        f, key, P, t);
    ++pass;
    if (i >= 0) {
      int bb = over[i % nl];
      int tt = t0 + (int)(i / nl);
      if ((unsigned)tt < *((volatile unsigned*)(nbest + bb))) {  // no success below it meanwhile
        Ends e = load_ends(c, bb);
        uint32_t tau;
        float pdf;
        uint32_t cell = cell_of(c, bb);
        if (draw_seed<K, kS>(S, has_guide ? &g : nullptr, e, cell, e.tau, P.tau_random != 0, key,
                             (uint64_t)bb + offset, (uint32_t)tt | ctx.trial_base, P, L.ch, tau, pdf, ctx.err, t.c, false, true) &&
            tau == e.tau) {
          b = bb;
          tr = tt;
          L.e = e;
          load_chain<K>(c, b, target);
          walk_begin(L);
        }
      }
    }
    const bool tail = done && np == 0;
    bool any = __any_sync(FULL, b >= 0);
    if (!any && tail) break;
    if (b < 0) continue;
    int st = walk_pass_fused<K, kS>(S, L, P, t.c, tail ? TAIL_ATTEMPTS : 1);
    if (st != RUNNING) {
      t.walks++;
      // converged walks of the trial sequence (t <= N) are counted by the
      // round's finish kernel: the success itself once per chain, and the
      // walks to other solutions that lie below the first success (parallel
      // trials past it are not part of the estimator)
      if (st == ST_CONVERGED) {
        if (same_solution<K>(L.ch, target, eps2)) {
          atomicMin(nbest + b, (unsigned)tr);
        } else if ((unsigned)tr < *((volatile unsigned*)(nbest + b))) {  // not past a known success
          int j = atomicAdd(pr.n, 1);
          if (j < pairs_cap(pr)) pr.buf[PAIRS_PER_CHAIN * *base + j] = make_uint2((unsigned)b, (unsigned)tr);
        }
      }
      b = -1;
    }
  }
  if (kS) flush(t, ctx.stats);
}

// Parallel Bernoulli round, one chain per lane group (see k_walk_g): the
// group's leader takes the (chain, trial) item, every lane draws the same trial
// seed from the same counters and keeps its own vertex, the group walks it,
// and the same-solution test is taken per vertex in FP64 and combined over the
// group -- the decisions of k_bern_round.
template <int K, int G, bool kS>
__global__ void __launch_bounds__(128) k_bern_round_g(const __grid_constant__ DScene S_, DGuide g, int has_guide,
                                                      DChains c, uint2 key, uint64_t offset, mpg_params P, DCtx ctx,
                                                      int* queue, const int* list, const int* n_list, const int* base,
                                                      unsigned* nbest, int t0, int TB, DPairs pr) {
  __shared__ DScene s_scene;
  const DScene& S = scene_in_smem(S_, s_scene);
  static_assert(G >= K && G <= 32 && (G & (G - 1)) == 0, "group of a power of two >= K lanes");
  constexpr int NG = 128 / G;
  __shared__ float2 sC[NG][K];
  __shared__ float4 sA[NG][K], sB[NG][K], sCc[NG][K];
  __shared__ long long pools[4][32];
  Tally t = {};
  Counters dummy = {};
  const double eps2 = (double)P.dedup_eps * (double)P.dedup_eps;
  const int* over = list + *base;
  const int nl = *n_list;
  const long long n = (long long)nl * TB;
  unsigned long long* queue64 = reinterpret_cast<unsigned long long*>(queue);
  offset = rng_offset(offset, ctx);
  const BernFilter f{over, nl, t0, nbest, offset, ctx.trial_base,
                     P.tau_random != 0 && !(has_guide && g.kind == MPG_GUIDE_VMF)};
  long long* pool = pools[threadIdx.x >> 5];
  int np = 0;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, j = threadIdx.x % G, grp = threadIdx.x / G;
  const int leader = lane & ~(G - 1);
  const unsigned gmask = (G == 32 ? FULL : ((1u << G) - 1u)) << leader;
  const size_t Bz = (size_t)c.B;
  GroupLane<K> L;
  L.need_eval = false;
  float3 tx = make_float3(0.f, 0.f, 0.f);  // own vertex of the chain's solution
  int tsurf = -1;
  int b = -1, tr = 0;
  bool done = false;
  const int refill = P.refill_every > 1 ? P.refill_every : 1;
  int pass = 0;
  while (true) {
    bool idle_warp = __all_sync(FULL, b < 0);
    long long i = bern_pool_take<K, kS>(j == 0 && b < 0 && (idle_warp || pass % refill == 0), pool, np, queue64, n,
                                        done, c, f, key, P, t);
    i = __shfl_sync(FULL, i, leader);
    ++pass;
    // The leader alone reads the chain's best success (it changes under other
    // groups' atomics) and decides for its group; every warp-wide shuffle below
    // is executed by all 32 lanes.
    int bb = -1, tt = 0;
    bool take = false;
    if (i >= 0) {
      bb = over[i % nl];
      tt = t0 + (int)(i / nl);
      if (j == 0) take = (unsigned)tt < *((volatile unsigned*)(nbest + bb));  // no success below it meanwhile
    }
    take = __shfl_sync(FULL, take ? 1 : 0, leader) != 0;
    bool drawn = false;
    Chain<K> ch;
    Ends e;
    if (take) {
      e = load_ends(c, bb);
      uint32_t cell = cell_of(c, bb);
      uint32_t tau;
      float pdf;
      drawn = draw_seed<K, kS>(S, has_guide ? &g : nullptr, e, cell, e.tau, P.tau_random != 0, key,
                               (uint64_t)bb + offset, (uint32_t)tt | ctx.trial_base, P, ch, tau, pdf, ctx.err, j == 0 ? t.c : dummy,
                               false, true) &&
              tau == e.tau;
    }
    drawn = __shfl_sync(FULL, drawn ? 1 : 0, leader) != 0;
    if (take && drawn) {
#pragma unroll
      for (int v = 0; v < K; ++v)
        if (v == j) { L.x = ch.x[v]; L.surf = ch.surf[v]; L.prim = ch.prim[v]; L.b1 = ch.b1[v]; L.b2 = ch.b2[v]; }
      if (j < K) {
        tx = make_float3(c.x[(3 * j + 0) * Bz + bb], c.x[(3 * j + 1) * Bz + bb], c.x[(3 * j + 2) * Bz + bb]);
        tsurf = c.surf[j * Bz + bb];
      }
      b = bb;
      tr = tt;
      L.e = e;
      L.it = 0;
      L.hv = 0;
      L.beta = 1.0f;
      L.need_eval = true;
    }
    const bool tail = done && np == 0;
    bool any = __any_sync(FULL, b >= 0);
    if (!any && tail) break;
    if (b < 0) continue;
    int st = walk_pass_g_fused<K, G, kS>(S, L, P, j == 0 ? t.c : dummy, gmask, j, sC[grp], sA[grp], sB[grp],
                                         sCc[grp], tail ? TAIL_ATTEMPTS : 1);
    if (st != RUNNING) {
      if (j == 0) t.walks++;
      if (st == ST_CONVERGED) {
        bool same_v = true;
        if (j < K) {
          double dx = (double)L.x.x - (double)tx.x, dy = (double)L.x.y - (double)tx.y,
                 dz = (double)L.x.z - (double)tx.z;
          same_v = L.surf == tsurf && dx * dx + dy * dy + dz * dz < eps2;
        }
        bool same = __all_sync(gmask, same_v);
        if (j == 0) {
          if (same) {
            atomicMin(nbest + b, (unsigned)tr);
          } else if ((unsigned)tr < *((volatile unsigned*)(nbest + b))) {  // not past a known success
            int q = atomicAdd(pr.n, 1);
            if (q < pairs_cap(pr)) pr.buf[PAIRS_PER_CHAIN * *base + q] = make_uint2((unsigned)b, (unsigned)tr);
          }
        }
      }
      b = -1;
    }
  }
  if (kS) flush(t, ctx.stats);
}

}  // namespace kern
}  // namespace mpg
