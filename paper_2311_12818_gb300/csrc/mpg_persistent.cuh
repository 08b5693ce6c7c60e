// Persistent work-queue kernels of the batched mode.
//
// A thread keeps one chain (or one Bernoulli trial) in registers and advances
// it by one line-search attempt per pass; every pass re-evaluates only the
// lanes whose previous attempt was accepted.  A lane whose walk ends takes
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

template <int K>
struct WalkLane {
  Chain<K> ch;
  Ends e;
  float3 tu[K], tv[K];
  float2 du[K][1];
  float cn2, cmax, beta;
  int it, hv;
  bool need_eval;
};

template <int K>
__device__ __forceinline__ void walk_begin(WalkLane<K>& w) {
  w.it = 0;
  w.hv = 0;
  w.beta = 1.0f;
  w.need_eval = true;
}

// One pass of the walk: Jacobian and Newton direction when the previous
// attempt was accepted (or at the start), then one reprojection attempt.
// Same decisions, in the same order, as walk<K>().
template <int K, bool kS>
__device__ __forceinline__ int walk_pass(const DScene& S, WalkLane<K>& w, const mpg_params& P, Counters& cnt) {
  if (w.need_eval) {
    VB vb[K];
    if (!eval_full<K, kS>(S, w.ch, w.e, vb, w.tu, w.tv, w.cn2, w.cmax, false, cnt)) return ST_FAILED;
    if (w.cmax < P.tol) return ST_CONVERGED;
    if (w.it >= P.max_iter) return ST_LIMIT;
#pragma unroll
    for (int i = 0; i < K; ++i) w.du[i][0] = make_float2(-vb[i].C.x, -vb[i].C.y);
    if (kS) { cnt.newton++; cnt.rows += K; }
    if (!thomas<K, 1>(vb, w.du, P.sing_eps)) return ST_FAILED;
    w.beta = 1.0f;
    w.hv = 0;
    w.need_eval = false;
  }
  Chain<K> cand;
  float cc2;
  if (propose<K>(S, w.ch, w.tu, w.tv, w.du, w.beta, cand) && eval_c<K, kS>(S, cand, w.e, cc2, cnt) &&
      cc2 < w.cn2) {
    w.ch = cand;
    w.it++;
    w.need_eval = true;
    return RUNNING;
  }
  w.hv++;
  w.beta *= 0.5f;
  if (w.hv > P.max_halvings) return w.cmax < P.stall_tol ? ST_CONVERGED : ST_FAILED;
  return RUNNING;
}

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

// ---------------------------------------------------------------------------
// Walk (K2): one lane per chain, refilled from the bucket's queue.
// ---------------------------------------------------------------------------
template <int K, bool kS>
__global__ void __launch_bounds__(128) k_walk_p(const __grid_constant__ DScene S, DChains c, DWork w, mpg_params P,
                                                DCtx ctx, int* queue) {
  Tally t = {};
  const int n = n_items<K>(w, c);
  WalkLane<K> L;
  int b = -1;
  bool done = false;
  const unsigned FULL = 0xffffffffu;
  while (true) {
    int i = take_item(b < 0, queue, n, done);
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
      int st = walk_pass<K, kS>(S, L, P, t.c);
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
// Bernoulli trials (K5), first pass: one lane per admissible chain runs trials
// 1..T1 in order; chains without a hit are appended to the overflow list.
// ---------------------------------------------------------------------------
template <int K>
struct TrialLane {
  WalkLane<K> w;
  Chain<K> target;
  uint32_t cell;
  int t;           // current trial index
  bool walking;    // a trial walk is in progress
};

// Final outputs of one chain.
__device__ __forceinline__ void bern_write(const DScene& S, const DChains& c, const DOut& o, int b, float T, uint32_t N,
                                           bool cap) {
  if (o.trials) o.trials[b] = N;
  if (o.capped) o.capped[b] = cap ? 1 : 0;
  float pn = c.pn ? c.pn[b] : 1.0f;
  o.contrib[b] = (T > 0.0f && N > 0) ? S.L.area * T * (float)N / pn : 0.0f;
}

template <int K, bool kS>
__global__ void __launch_bounds__(128) k_bern_p(const __grid_constant__ DScene S, DGuide g, int has_guide, DChains c,
                                                DWork w, uint2 key, uint64_t offset, mpg_params P, DOut o, DCtx ctx,
                                                int* queue, DBernScratch bern) {
  Tally t = {};
  const int n = n_items<K>(w, c);
  const double eps2 = (double)P.dedup_eps * (double)P.dedup_eps;
  const int T1 = min(bern.T1, P.max_trials);
  TrialLane<K> L;
  int b = -1;
  bool done = false;
  const unsigned FULL = 0xffffffffu;
  while (true) {
    int i = take_item(b < 0, queue, n, done);
    if (i >= 0) {
      int bb = item<K>(w, c, i);
      if (bb >= 0) {
        float T = o.T[bb];
        if (T > 0.0f) {
          b = bb;
          load_chain<K>(c, b, L.target);
          L.w.e = load_ends(c, b);
          L.cell = c.cell ? c.cell[b / c.spq] : 0u;
          L.t = 0;
          L.walking = false;
        } else {
          bern_write(S, c, o, bb, 0.0f, 0, false);
        }
      }
    }
    bool any = __any_sync(FULL, b >= 0);
    if (!any && done) break;
    if (b < 0) continue;
    if (!L.walking) {
      // next trial: fresh seed from the same distribution, same n
      L.t++;
      t.trials++;
      uint32_t tau;
      float pdf;
      Ends e = L.w.e;
      if (draw_seed<K, kS>(S, has_guide ? &g : nullptr, e, L.cell, e.tau, P.tau_random != 0, key,
                           (uint64_t)b + offset, (uint32_t)L.t, P, L.w.ch, tau, pdf, ctx.err, t.c, false) &&
          tau == e.tau) {
        walk_begin(L.w);
        L.walking = true;
      }
    } else {
      int st = walk_pass<K, kS>(S, L.w, P, t.c);
      if (st != RUNNING) {
        L.walking = false;
        t.walks++;
        t.conv += st == ST_CONVERGED;
        if (st == ST_CONVERGED && same_solution<K>(L.w.ch, L.target, eps2)) {
          bern_write(S, c, o, b, o.T[b], (uint32_t)L.t, false);
          b = -1;
          continue;
        }
      }
    }
    if (!L.walking && b >= 0 && L.t >= T1) {
      if (T1 >= P.max_trials) {
        bern_write(S, c, o, b, o.T[b], (uint32_t)P.max_trials, true);
      } else {
        int slot = atomicAdd(bern.n_list[0], 1);
        bern.list[0][*bern.base + slot] = b;
        bern.nbest[b] = 0xffffffffu;
      }
      b = -1;
    }
  }
  if (kS) flush(t, ctx.stats);
}

// ---------------------------------------------------------------------------
// Bernoulli trial rounds for the overflow chains: trials t0 .. t0+TB-1 of every
// listed chain run in parallel as independent items; the first success is the
// smallest successful index (atomicMin), exactly as a sequential loop would
// find.  Items above a chain's best success so far are skipped.
// ---------------------------------------------------------------------------
template <int K, bool kS>
__global__ void __launch_bounds__(128) k_bern_round(const __grid_constant__ DScene S, DGuide g, int has_guide,
                                                    DChains c, uint2 key, uint64_t offset, mpg_params P, DCtx ctx,
                                                    int* queue, const int* list, const int* n_list, const int* base,
                                                    unsigned* nbest, int t0, int TB) {
  Tally t = {};
  const double eps2 = (double)P.dedup_eps * (double)P.dedup_eps;
  const int* over = list + *base;
  const long long n = (long long)(*n_list) * TB;
  const int n_items_i = n > 0x7fffffff ? 0x7fffffff : (int)n;
  WalkLane<K> L;
  Chain<K> target;
  int b = -1, tr = 0;
  bool done = false;
  const unsigned FULL = 0xffffffffu;
  while (true) {
    int i = take_item(b < 0, queue, n_items_i, done);
    if (i >= 0) {
      int bb = over[i / TB];
      int tt = t0 + i % TB;
      if (tt <= P.max_trials && (unsigned)tt < *((volatile unsigned*)(nbest + bb))) {
        t.trials++;
        Ends e = load_ends(c, bb);
        uint32_t tau;
        float pdf;
        uint32_t cell = c.cell ? c.cell[bb / c.spq] : 0u;
        if (draw_seed<K, kS>(S, has_guide ? &g : nullptr, e, cell, e.tau, P.tau_random != 0, key,
                             (uint64_t)bb + offset, (uint32_t)tt, P, L.ch, tau, pdf, ctx.err, t.c, false) &&
            tau == e.tau) {
          b = bb;
          tr = tt;
          L.e = e;
          load_chain<K>(c, b, target);
          walk_begin(L);
        }
      }
    }
    bool any = __any_sync(FULL, b >= 0);
    if (!any && done) break;
    if (b < 0) continue;
    int st = walk_pass<K, kS>(S, L, P, t.c);
    if (st != RUNNING) {
      t.walks++;
      if (st == ST_CONVERGED && same_solution<K>(L.ch, target, eps2)) {
        atomicMin(nbest + b, (unsigned)tr);
        t.conv++;  // only the successful trial of a round counts as a converged walk
      }
      b = -1;
    }
  }
  if (kS) flush(t, ctx.stats);
}

}  // namespace kern
}  // namespace mpg
