// Kernel declarations shared by the kernel and host translation units.
#pragma once

#include "mpg_device.cuh"

namespace mpg {

// Raw device view of a chain batch (see mpg_chains in mpg.h).
struct DChains {
  int B, Q, spq;
  const float* xD;
  const float* nD;
  const uint32_t* cell;
  const float* xL;
  const uint8_t* k;
  const float* pn;
  uint8_t* tau;
  float* x;
  int32_t* surf;
  int32_t* prim;
  float* bary;
  float* pdf;
  uint8_t* status;
  uint8_t* iters;
  const uint32_t* chain_cell;  // per-chain guide cell, or NULL
  const float* offset;         // [8][2][B] offset normals of glossy chains, or NULL (specular)
};

// Guide cell of chain b: its own (a spatial tree's leaf) or its receiver point's.
__device__ __forceinline__ uint32_t cell_of(const DChains& c, int b) {
  return c.chain_cell ? c.chain_cell[b] : (c.cell ? c.cell[b / c.spq] : 0u);
}

// Optional k-bucketed work list: chains order[base[K] .. base[K]+count[K]).
struct DWork {
  const int* order;   // NULL => identity over [0, B)
  const int* base;    // [MAXK+1] bucket starts (device)
  const int* count;   // [MAXK+1] bucket sizes (device)
};

struct DOut {
  float* G;
  float* kappa;
  float* T;
  uint32_t* trials;
  uint8_t* capped;
  float* contrib;
  int* fp64_list;        // chains queued for the FP64 geometry term
  int* fp64_count;       // length of this chain length's queue
  const int* fp64_base;  // start of this chain length's region of fp64_list
  int rep = 0;           // Bernoulli estimate being formed (0 .. repeats-1)
  int repeats = 1;       // independent estimates averaged per chain
};

struct DCtx {
  int* err;                          // device error word
  unsigned long long* stats;         // [16] counters of the kernel family (mpg_stats layout)
  const unsigned long long* rng_add; // NULL, or a device counter added to rng offsets (captured graphs)
  uint32_t trial_base;               // Bernoulli repeat j draws trial t as t | trial_base (= j << 24)
};

// Final outputs of a chain's Bernoulli estimate: N trials (capped when the
// cap ran out).  Repeat j > 0 adds its N to the previous repeats' sum in
// trials[b] (which then must not be NULL) and ORs its cap flag; contrib is
// the running mean, A_L T (sum N) / (repeats P(n)), final after the last.
__device__ __forceinline__ void bern_write(float area, const DChains& c, const DOut& o, int b, float T, uint32_t N,
                                           bool cap) {
  if (o.rep > 0) {
    N += o.trials[b];
    cap = cap || (o.capped && o.capped[b]);
  }
  if (o.trials) o.trials[b] = N;
  if (o.capped) o.capped[b] = cap ? 1 : 0;
  float pn = c.pn ? c.pn[b] : 1.0f;
  o.contrib[b] = (T > 0.0f && N > 0) ? area * T * (float)N / ((float)o.repeats * pn) : 0.0f;
}

// Trial walks of a parallel Bernoulli round that converged to another
// solution, as (chain, trial) pairs; the round's finish counts those below the
// chain's first recurrence, which a sequential loop over the trials would have
// walked.  Region of chain length K: PAIRS_PER_CHAIN entries per chain of the
// bucket, buf[PAIRS_PER_CHAIN * *base ..), PAIRS_PER_CHAIN * bucket size long.
constexpr int PAIRS_PER_CHAIN = 8;
struct DPairs {
  uint2* buf;
  int* n;              // pairs recorded in this round (device counter of length K)
  const int* cap_dev;  // bucket size, or NULL => cap_host
  int cap_host;
};
__device__ __forceinline__ int pairs_cap(const DPairs& p) {
  return PAIRS_PER_CHAIN * (p.cap_dev ? *p.cap_dev : p.cap_host);
}

// Random-number offset of a launch: the host value plus, inside a replayed
// graph, the graph's device counter.
__device__ __forceinline__ uint64_t rng_offset(uint64_t offset, const DCtx& ctx) {
  return ctx.rng_add ? offset + *ctx.rng_add : offset;
}

// Length from which the geometry term is always formed in FP64.
__host__ __device__ __forceinline__ int fp64_k_of(const mpg_params& P) { return P.fp64_k > 0 ? P.fp64_k : 6; }



void launch_seed(int K, bool stats, const DScene& S, const DGuide* g, const DChains& c, DWork w, uint2 key,
                 uint64_t offset, const mpg_params& P, DCtx ctx, int grid, int block, cudaStream_t st);
// Seeds of every chain of a batch in one launch, whatever its length
// (mpg_seed_all.cu; batched mode).
void launch_seed_all(const DScene& S, const DGuide* g, const DChains& c, uint2 key, uint64_t offset,
                     const mpg_params& P, DCtx ctx, int grid, cudaStream_t st);
void launch_walk(int K, bool stats, const DScene& S, const DChains& c, DWork w, const mpg_params& P, DCtx ctx,
                 int grid, int block, cudaStream_t st);
void launch_contrib(int K, bool stats, const DScene& S, const DChains& c, DWork w, const mpg_params& P, DOut o,
                    DCtx ctx, int grid, int block, cudaStream_t st);
void launch_bernoulli(int K, bool stats, const DScene& S, const DGuide* g, const DChains& c, DWork w, uint2 key,
                      uint64_t offset, const mpg_params& P, DOut o, DCtx ctx, int grid, int block, cudaStream_t st);

// K7 adjoint for chains of length K (1..4) on heightfield 0.
void launch_adjoint(int K, const DScene& S, const DChains& c, const float* T, const float* contrib,
                    const float* dL_dE, float* dL_dtheta, int* skipped, int sms, cudaStream_t st);

// Occupancy-derived grid for the per-K kernels (blocks per SM x SMs).
int blocks_per_sm(int which, int K, bool stats, int block);

// Host launchers of the kernels for one chain length K (see mpg_kernels_impl.cuh).
template <int K>
struct KLaunch {
  static void seed(bool stats, const DScene& S, const DGuide* g, const DChains& c, DWork w, uint2 key,
                   uint64_t offset, const mpg_params& P, DCtx ctx, int grid, int block, cudaStream_t st);
  static void walk(bool stats, const DScene& S, const DChains& c, DWork w, const mpg_params& P, DCtx ctx, int grid,
                   int block, cudaStream_t st);
  static void contrib(bool stats, const DScene& S, const DChains& c, DWork w, const mpg_params& P, DOut o, DCtx ctx,
                      int grid, int block, cudaStream_t st);
  static void bernoulli(bool stats, const DScene& S, const DGuide* g, const DChains& c, DWork w, uint2 key,
                        uint64_t offset, const mpg_params& P, DOut o, DCtx ctx, int grid, int block,
                        cudaStream_t st);
  static void walk_p(bool stats, const DScene& S, const DChains& c, DWork w, const mpg_params& P, DCtx ctx,
                     int* queue, int grid, int block, cudaStream_t st);
  // one chain per group of G >= K lanes (128 threads per CTA)
  static void walk_g(bool stats, const DScene& S, const DChains& c, DWork w, const mpg_params& P, DCtx ctx,
                     int* queue, int grid, cudaStream_t st);
  static void trial_init(const DScene& S, const DChains& c, DWork w, DOut o, int* list, const int* base, int* n_list,
                         unsigned* nbest, int grid, cudaStream_t st);
  static void contrib64(const DScene& S, const DChains& c, const mpg_params& P, DOut o, int grid, cudaStream_t st);
  static void trial_seed(const DScene& S, const DGuide* g, const DChains& c, const DChains& tc, const int* list,
                         const int* base, const int* n_list, uint2 key, uint64_t offset, const mpg_params& P,
                         DCtx ctx, int t, int grid, int block, cudaStream_t st);
  static void trial_check(const DScene& S, const DChains& c, const DChains& tc, DOut o, const int* list,
                          const int* base, const int* n_list, int t, int last, const mpg_params& P, int* next,
                          int* n_next, unsigned* nbest, int grid, cudaStream_t st);
  static void bern_round(bool stats, const DScene& S, const DGuide* g, const DChains& c, uint2 key, uint64_t offset,
                         const mpg_params& P, DCtx ctx, int* queue, const int* list, const int* n_list,
                         const int* base, unsigned* nbest, int t0, int TB, DPairs pr, int grid, int block,
                         cudaStream_t st);
  // glossy chains: admissibility and the estimate W (FP64) as T
  static void glossy(const DScene& S, const DChains& c, DWork w, const mpg_params& P, DOut o, DCtx ctx, int grid,
                     cudaStream_t st);
  static int blocks_per_sm(int which, bool stats, int block);
};

void launch_glossy(int K, const DScene& S, const DChains& c, DWork w, const mpg_params& P, DOut o, DCtx ctx, int grid,
                   cudaStream_t st);
// Offset normals of glossy chains (Beckmann, roughness alpha), [8][2][B].
void launch_offsets(const DChains& c, float alpha, uint2 key, uint64_t offset, DCtx ctx, float* out, int sms,
                    cudaStream_t st);

// Persistent-mode launchers by chain length (dispatch to KLaunch<K>).
void launch_walk_p(int K, bool stats, const DScene& S, const DChains& c, DWork w, const mpg_params& P, DCtx ctx,
                   int* queue, int grid, int block, cudaStream_t st);
void launch_contrib64(int K, const DScene& S, const DChains& c, const mpg_params& P, DOut o, int grid,
                      cudaStream_t st);
void launch_trial_init(int K, const DScene& S, const DChains& c, DWork w, DOut o, int* list, const int* base,
                       int* n_list, unsigned* nbest, int grid, cudaStream_t st);
void launch_trial_seed(int K, const DScene& S, const DGuide* g, const DChains& c, const DChains& tc,
                       const int* list, const int* base, const int* n_list, uint2 key, uint64_t offset,
                       const mpg_params& P, DCtx ctx, int t, int grid, int block, cudaStream_t st);
void launch_trial_check(int K, const DScene& S, const DChains& c, const DChains& tc, DOut o, const int* list,
                        const int* base, const int* n_list, int t, int last, const mpg_params& P, int* next,
                        int* n_next, unsigned* nbest, int grid, cudaStream_t st);
void launch_bern_round(int K, bool stats, const DScene& S, const DGuide* g, const DChains& c, uint2 key,
                       uint64_t offset, const mpg_params& P, DCtx ctx, int* queue, const int* list, const int* n_list,
                       const int* base, unsigned* nbest, int t0, int TB, DPairs pr, int grid, int block,
                       cudaStream_t st);
// Ends a trial round: chains with a success get N, chains past the cap are
// capped, the rest move to the next list.
void launch_bern_finish(const DScene& S, const DChains& c, DOut o, const int* list, const int* n_list,
                        const int* base, unsigned* nbest, int t_end, int max_trials, int* next, int* n_next,
                        DPairs pr, unsigned long long* stats, int sms, cudaStream_t st);

}  // namespace mpg
