// Dispatch of the per-chain-length kernels to their instantiations
// (mpg_k1.cu .. mpg_k8.cu, compiled as separate translation units).
#include "mpg_kernels.cuh"

namespace mpg {

extern template struct KLaunch<1>;
extern template struct KLaunch<2>;
extern template struct KLaunch<3>;
extern template struct KLaunch<4>;
extern template struct KLaunch<5>;
extern template struct KLaunch<6>;
extern template struct KLaunch<7>;
extern template struct KLaunch<8>;

#define MPG_SWITCH(K_, CALL) \
  switch (K_) {              \
    case 1: CALL(1); break;  \
    case 2: CALL(2); break;  \
    case 3: CALL(3); break;  \
    case 4: CALL(4); break;  \
    case 5: CALL(5); break;  \
    case 6: CALL(6); break;  \
    case 7: CALL(7); break;  \
    case 8: CALL(8); break;  \
    default: break;          \
  }

void launch_seed(int K, bool stats, const DScene& S, const DGuide* g, const DChains& c, DWork w, uint2 key,
                 uint64_t offset, const mpg_params& P, DCtx ctx, int grid, int block, cudaStream_t st) {
#define C_(KK) KLaunch<KK>::seed(stats, S, g, c, w, key, offset, P, ctx, grid, block, st)
  MPG_SWITCH(K, C_)
#undef C_
}

void launch_walk(int K, bool stats, const DScene& S, const DChains& c, DWork w, const mpg_params& P, DCtx ctx,
                 int grid, int block, cudaStream_t st) {
#define C_(KK) KLaunch<KK>::walk(stats, S, c, w, P, ctx, grid, block, st)
  MPG_SWITCH(K, C_)
#undef C_
}

void launch_contrib(int K, bool stats, const DScene& S, const DChains& c, DWork w, const mpg_params& P, DOut o,
                    DCtx ctx, int grid, int block, cudaStream_t st) {
#define C_(KK) KLaunch<KK>::contrib(stats, S, c, w, P, o, ctx, grid, block, st)
  MPG_SWITCH(K, C_)
#undef C_
}

void launch_bernoulli(int K, bool stats, const DScene& S, const DGuide* g, const DChains& c, DWork w, uint2 key,
                      uint64_t offset, const mpg_params& P, DOut o, DCtx ctx, int grid, int block, cudaStream_t st) {
#define C_(KK) KLaunch<KK>::bernoulli(stats, S, g, c, w, key, offset, P, o, ctx, grid, block, st)
  MPG_SWITCH(K, C_)
#undef C_
}

void launch_walk_p(int K, bool stats, const DScene& S, const DChains& c, DWork w, const mpg_params& P, DCtx ctx,
                   int* queue, int grid, int block, cudaStream_t st) {
  if ((P.walk_group & 1) && K > 1) {
#define C_(KK) KLaunch<KK>::walk_g(stats, S, c, w, P, ctx, queue, grid, st)
    MPG_SWITCH(K, C_)
#undef C_
    return;
  }
#define C_(KK) KLaunch<KK>::walk_p(stats, S, c, w, P, ctx, queue, grid, block, st)
  MPG_SWITCH(K, C_)
#undef C_
}

void launch_glossy(int K, const DScene& S, const DChains& c, DWork w, const mpg_params& P, DOut o, DCtx ctx, int grid,
                   cudaStream_t st) {
#define C_(KK) KLaunch<KK>::glossy(S, c, w, P, o, ctx, grid, st)
  MPG_SWITCH(K, C_)
#undef C_
}

void launch_contrib64(int K, const DScene& S, const DChains& c, const mpg_params& P, DOut o, int grid,
                      cudaStream_t st) {
#define C_(KK) KLaunch<KK>::contrib64(S, c, P, o, grid, st)
  MPG_SWITCH(K, C_)
#undef C_
}

void launch_trial_init(int K, const DScene& S, const DChains& c, DWork w, DOut o, int* list, const int* base,
                       int* n_list, unsigned* nbest, int grid, cudaStream_t st) {
#define C_(KK) KLaunch<KK>::trial_init(S, c, w, o, list, base, n_list, nbest, grid, st)
  MPG_SWITCH(K, C_)
#undef C_
}

void launch_trial_seed(int K, const DScene& S, const DGuide* g, const DChains& c, const DChains& tc,
                       const int* list, const int* base, const int* n_list, uint2 key, uint64_t offset,
                       const mpg_params& P, DCtx ctx, int t, int grid, int block, cudaStream_t st) {
#define C_(KK) KLaunch<KK>::trial_seed(S, g, c, tc, list, base, n_list, key, offset, P, ctx, t, grid, block, st)
  MPG_SWITCH(K, C_)
#undef C_
}

void launch_trial_check(int K, const DScene& S, const DChains& c, const DChains& tc, DOut o, const int* list,
                        const int* base, const int* n_list, int t, int last, const mpg_params& P, int* next,
                        int* n_next, unsigned* nbest, int grid, cudaStream_t st) {
#define C_(KK) KLaunch<KK>::trial_check(S, c, tc, o, list, base, n_list, t, last, P, next, n_next, nbest, grid, st)
  MPG_SWITCH(K, C_)
#undef C_
}

void launch_bern_round(int K, bool stats, const DScene& S, const DGuide* g, const DChains& c, uint2 key,
                       uint64_t offset, const mpg_params& P, DCtx ctx, int* queue, const int* list, const int* n_list,
                       const int* base, unsigned* nbest, int t0, int TB, DPairs pr, int grid, int block,
                       cudaStream_t st) {
#define C_(KK) KLaunch<KK>::bern_round(stats, S, g, c, key, offset, P, ctx, queue, list, n_list, base, nbest, t0, TB, pr, grid, block, st)
  MPG_SWITCH(K, C_)
#undef C_
}

int blocks_per_sm(int which, int K, bool stats, int block) {
  int n = 1;
#define C_(KK) n = KLaunch<KK>::blocks_per_sm(which, stats, block)
  MPG_SWITCH(K, C_)
#undef C_
  return n;
}

}  // namespace mpg
