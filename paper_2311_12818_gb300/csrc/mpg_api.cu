// C ABI of libmpg.so: context, scene construction (meshes, normals and a
// binned-SAH BVH built on the host), argument checks and launch planning.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <string>
#include <array>
#include <vector>

#include "mpg_aux.cuh"

using namespace mpg;

namespace {

thread_local std::string g_last_error;

mpg_status fail(mpg_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define CUDA_TRY(expr)                                                                    \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(e_ == cudaErrorMemoryAllocation ? MPG_ERR_OOM : MPG_ERR_CUDA, "%s: %s", \
                  #expr, cudaGetErrorString(e_));                                         \
  } while (0)

#define LAUNCH_CHECK(what)                                                                \
  do {                                                                                    \
    cudaError_t e_ = cudaGetLastError();                                                  \
    if (e_ != cudaSuccess) return fail(MPG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e_)); \
  } while (0)

bool aligned16(const void* p) { return p && ((uintptr_t)p & 15u) == 0; }

}  // namespace

struct mpg_ctx {
  struct ProfRec {
    int kind;
    cudaEvent_t a, b;
  };
  int device = 0, sms = 1;
  bool profile = false;
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> pool;
  double prof_ms[MPG_KERNEL_KINDS] = {};
  int64_t prof_n[MPG_KERNEL_KINDS] = {};
  int64_t launches = 0;
  int* d_err = nullptr;
  unsigned long long* d_stats = nullptr;
  int* d_order = nullptr;
  int order_cap = 0;
  int* d_count = nullptr;
  int* d_base = nullptr;
  int* d_cursor = nullptr;
  float* d_scratch = nullptr;
  int* d_queue = nullptr;        // [MAXK+1][32] work-queue counters of the persistent launches
  int* d_nlist = nullptr;        // [2][MAXK+1] overflow list lengths
  int* d_zero = nullptr;         // [MAXK+1] zeros (list regions when chains are not bucketed)
  int* d_fp64 = nullptr;         // [B] chains queued for the FP64 geometry term
  int* d_fp64_count = nullptr;   // [MAXK+1] queue lengths per chain length
  int fp64_cap = 0;
  int* d_list[2] = {nullptr, nullptr};
  unsigned* d_nbest = nullptr;
  uint32_t* d_nsum = nullptr;    // [B] sum of N over Bernoulli repeats when the caller keeps no trials
  int nsum_cap = 0;
  uint32_t* d_rec = nullptr;     // per-tile counts of the ordered record compaction
  int rec_cap = 0;
  uint2* d_pairs = nullptr;      // [8B] converged trial walks of the parallel rounds (chain, trial)
  int* d_npairs = nullptr;       // [MAXK+1] pair counts per chain length
  int bern_cap = 0;
  // trial chain state of the Bernoulli rounds (same layout as mpg_chains)
  float* t_x = nullptr;
  int32_t* t_surf = nullptr;
  int32_t* t_prim = nullptr;
  float* t_bary = nullptr;
  uint8_t* t_status = nullptr;
  uint8_t* t_iters = nullptr;
  bool stats_on = true;
  // stream capture in progress (mpg_graph_begin .. mpg_graph_end)
  bool capturing = false;
  bool profile_saved = false;
  unsigned long long* cap_rng = nullptr;  // the recorded graph's random-number counter
  uint64_t cap_advance = 0;
  std::vector<mpg_ctx*> cap_joined;       // other contexts recording into this capture
  int64_t cap_launch0 = 0;
  cudaStream_t aux[MAXK] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[MAXK] = {};
};

struct mpg_scene {
  DScene S;
  std::vector<void*> allocs;
  std::vector<int> n_nodes, n_tris;
  // per heightfield, for height updates on the device (mpg_scene_set_heights):
  // the grid's extent in FP64, each node's parent and number of inner
  // children, and a counter per node for the bottom-up refit
  std::vector<std::array<double, 4>> hf_extent;
  std::vector<const int*> hf_parent, hf_ninner;
  std::vector<int*> hf_count;
  int device = 0;
};

// ---------------------------------------------------------------------------
// BVH over the heightfield triangles (two children per node, binned SAH)
// ---------------------------------------------------------------------------
namespace {

struct Box {
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  void grow(const float* p) {
    for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], p[a]); hi[a] = std::max(hi[a], p[a]); }
  }
  void grow(const Box& b) {
    for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], b.lo[a]); hi[a] = std::max(hi[a], b.hi[a]); }
  }
  float area() const {
    if (lo[0] > hi[0]) return 0.0f;
    float d0 = hi[0] - lo[0], d1 = hi[1] - lo[1], d2 = hi[2] - lo[2];
    return 2.0f * (d0 * d1 + d1 * d2 + d2 * d0);
  }
};

struct BuildTri {
  Box box;
  float c[3];
  int id;
};

struct ChildRef {
  Box box;
  int idx = 0, count = 0;  // count > 0: leaf over tri slots [idx, idx+count)
};

struct BVHBuilder {
  std::vector<BuildTri> tris;
  std::vector<float4> nodes;     // 4 float4 per node
  std::vector<int> leaf_order;   // triangle ids in leaf order
  int max_depth = 0;
  static const int LEAF = 4;

  ChildRef make_leaf(int first, int count, const Box& box) {
    ChildRef r;
    r.box = box;
    r.idx = (int)leaf_order.size();
    r.count = count;
    for (int i = first; i < first + count; ++i) leaf_order.push_back(tris[i].id);
    return r;
  }

  void write_node(int ni, const ChildRef& L, const ChildRef& R) {
    float4* n = &nodes[4 * (size_t)ni];
    n[0] = make_float4(L.box.lo[0], L.box.hi[0], L.box.lo[1], L.box.hi[1]);
    n[1] = make_float4(R.box.lo[0], R.box.hi[0], R.box.lo[1], R.box.hi[1]);
    n[2] = make_float4(L.box.lo[2], L.box.hi[2], R.box.lo[2], R.box.hi[2]);
    int4 ch = make_int4(L.idx, R.idx, L.count, R.count);
    memcpy(&n[3], &ch, sizeof(int4));
  }

  ChildRef build(int first, int count, int depth) {
    max_depth = std::max(max_depth, depth);
    Box box, cbox;
    for (int i = first; i < first + count; ++i) { box.grow(tris[i].box); cbox.grow(tris[i].c); }
    if (count <= LEAF) return make_leaf(first, count, box);
    int axis = 0;
    for (int a = 1; a < 3; ++a)
      if (cbox.hi[a] - cbox.lo[a] > cbox.hi[axis] - cbox.lo[axis]) axis = a;
    float extent = cbox.hi[axis] - cbox.lo[axis];
    int mid = first + count / 2;
    if (extent > 0.0f && depth < 48) {
      const int NB = 16;
      Box bb[NB];
      int bc[NB] = {0};
      auto bin_of = [&](const BuildTri& t) {
        int b = (int)((t.c[axis] - cbox.lo[axis]) / extent * NB);
        return std::min(std::max(b, 0), NB - 1);
      };
      for (int i = first; i < first + count; ++i) { int b = bin_of(tris[i]); bb[b].grow(tris[i].box); bc[b]++; }
      float best = INFINITY;
      int best_split = -1;
      for (int s = 1; s < NB; ++s) {
        Box l, r;
        int nl = 0, nr = 0;
        for (int b = 0; b < s; ++b) { if (bc[b]) { l.grow(bb[b]); nl += bc[b]; } }
        for (int b = s; b < NB; ++b) { if (bc[b]) { r.grow(bb[b]); nr += bc[b]; } }
        if (!nl || !nr) continue;
        float cost = l.area() * nl + r.area() * nr;
        if (cost < best) { best = cost; best_split = s; }
      }
      if (best_split > 0) {
        auto it = std::partition(tris.begin() + first, tris.begin() + first + count,
                                 [&](const BuildTri& t) { return bin_of(t) < best_split; });
        mid = (int)(it - tris.begin());
      }
      if (mid == first || mid == first + count) mid = first + count / 2;
    }
    std::nth_element(tris.begin() + first, tris.begin() + mid, tris.begin() + first + count,
                     [&](const BuildTri& a, const BuildTri& b) {
                       return a.c[axis] < b.c[axis] || (a.c[axis] == b.c[axis] && a.id < b.id);
                     });
    int ni = (int)(nodes.size() / 4);
    nodes.resize(nodes.size() + 4);
    ChildRef L = build(first, mid - first, depth + 1);
    ChildRef R = build(mid, first + count - mid, depth + 1);
    write_node(ni, L, R);
    ChildRef r;
    r.box = box;
    r.idx = ni;
    r.count = 0;
    return r;
  }
};

// Heightfield vertex positions and interpolation normals.  The normal of
// grid vertex (i, j) is normalize(-dh/dx, -dh/dy, 1) with central
// differences inside the grid and one-sided differences on its border.
void heightfield_mesh(int nx, int ny, double x0, double y0, double x1, double y1, const double* h,
                      std::vector<float4>& P, std::vector<float4>& N) {
  double dx = (x1 - x0) / (nx - 1), dy = (y1 - y0) / (ny - 1);
  P.resize((size_t)nx * ny);
  N.resize((size_t)nx * ny);
  auto H = [&](int i, int j) { return h[(size_t)j * nx + i]; };
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double gx = i == 0 ? (H(1, j) - H(0, j)) / dx
                : i == nx - 1 ? (H(nx - 1, j) - H(nx - 2, j)) / dx
                              : (H(i + 1, j) - H(i - 1, j)) / (2.0 * dx);
      double gy = j == 0 ? (H(i, 1) - H(i, 0)) / dy
                : j == ny - 1 ? (H(i, ny - 1) - H(i, ny - 2)) / dy
                              : (H(i, j + 1) - H(i, j - 1)) / (2.0 * dy);
      double l = std::sqrt(gx * gx + gy * gy + 1.0);
      P[(size_t)j * nx + i] = make_float4((float)(x0 + i * dx), (float)(y0 + j * dy), (float)H(i, j), 0.0f);
      N[(size_t)j * nx + i] = make_float4((float)(-gx / l), (float)(-gy / l), (float)(1.0 / l), 0.0f);
    }
}

template <class T>
mpg_status upload(mpg_scene* sc, const std::vector<T>& v, const T** out) {
  void* p = nullptr;
  size_t bytes = std::max<size_t>(v.size() * sizeof(T), 16);
  CUDA_TRY(cudaMalloc(&p, bytes));
  sc->allocs.push_back(p);
  if (!v.empty()) CUDA_TRY(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  *out = (const T*)p;
  return MPG_OK;
}

float3 ld3(const double* p) { return make_float3((float)p[0], (float)p[1], (float)p[2]); }
double dlen(const double* p) { return std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]); }

mpg_status check_chains(const mpg_chains* c, bool need_walk_state) {
  if (!c) return fail(MPG_ERR_INVALID_ARG, "chains is NULL");
  if (c->B <= 0 || c->Q <= 0 || c->spq <= 0 || (long long)c->Q * c->spq != c->B)
    return fail(MPG_ERR_INVALID_ARG, "B (%d) must equal Q (%d) * spq (%d) > 0", c->B, c->Q, c->spq);
  const void* req[] = {c->xD, c->nD, c->xL, c->k, c->tau, c->x, c->surf, c->prim, c->bary, c->status, c->iters};
  const char* names[] = {"xD", "nD", "xL", "k", "tau", "x", "surf", "prim", "bary", "status", "iters"};
  for (int i = 0; i < 11; ++i)
    if (!aligned16(req[i])) return fail(MPG_ERR_INVALID_ARG, "chains.%s is NULL or not 16-byte aligned", names[i]);
  if (need_walk_state && !aligned16(c->pdf)) return fail(MPG_ERR_INVALID_ARG, "chains.pdf is NULL or unaligned");
  if (c->chain_cell && !aligned16(c->chain_cell)) return fail(MPG_ERR_INVALID_ARG, "chains.chain_cell is not 16-byte aligned");
  if (c->offset && !aligned16(c->offset)) return fail(MPG_ERR_INVALID_ARG, "chains.offset is not 16-byte aligned");
  return MPG_OK;
}

mpg_status check_params(const mpg_params* p) {
  if (!p) return fail(MPG_ERR_INVALID_ARG, "params is NULL");
  if (!(p->tol > 0.0f) || p->max_iter < 0 || p->max_iter > 255 || p->max_halvings < 0 || p->max_halvings > 60 ||
      !(p->ray_eps > 0.0f) || !(p->sing_eps >= 0.0f) || !(p->dedup_eps > 0.0f) || p->max_trials < 1 || p->max_trials > (1 << 24) ||
      !(p->alpha >= 0.0f && p->alpha <= 1.0f) || p->weight_shift < 0 || p->weight_shift > 60 ||
      (p->walk_mode != MPG_WALK_PLAIN && p->walk_mode != MPG_WALK_BATCHED) || p->k_uniform < 0 || p->k_uniform > MAXK ||
      p->block_threads < 0 || p->block_threads > 128 || (p->block_threads % 32) != 0 || !(p->stall_tol >= 0.0f) ||
      !(p->fp64_tol >= 0.0f) || p->fp64_k < 0 || p->fp64_k > 6 || p->ctas_per_sm < 0 || p->ctas_per_sm > 64 ||
      p->refill_every < 0 || p->refill_every > 64 || p->trial_sync_rounds < -1 || p->trial_sync_rounds > 8 ||
      p->trial_batch < 0 || p->trial_batch > 4096 || p->walk_group < 0 || p->walk_group > 3 ||
      p->bern_repeats < 0 || p->bern_repeats > 64 || (p->bern_repeats > 1 && p->max_trials >= (1 << 24)) ||
      p->selective < 0 || p->selective > 1 || !(p->roughness >= 0.0f && p->roughness <= 1.0f))
    return fail(MPG_ERR_INVALID_ARG, "invalid solver parameters");
  return MPG_OK;
}

DChains to_dev(const mpg_chains* c) {
  DChains d;
  d.B = c->B; d.Q = c->Q; d.spq = c->spq;
  d.xD = c->xD; d.nD = c->nD; d.cell = c->cell; d.xL = c->xL; d.k = c->k; d.pn = c->pn; d.tau = c->tau;
  d.x = c->x; d.surf = c->surf; d.prim = c->prim; d.bary = c->bary; d.pdf = c->pdf;
  d.status = c->status; d.iters = c->iters; d.chain_cell = c->chain_cell; d.offset = c->offset;
  return d;
}

mpg_status check_guide(const mpg_guide* g, DGuide& out) {
  if (!g) return fail(MPG_ERR_INVALID_ARG, "guide is NULL");
  out = DGuide{};
  if (g->kind == MPG_GUIDE_VMF) {
    if (g->n_cells <= 0 || g->n_cells > (1 << 20) || g->capacity < 0 || !aligned16(g->cell_start) ||
        !aligned16(g->lobe_key) || !aligned16(g->lobe) || !aligned16(g->lobe_prefix) || !aligned16(g->lobe_coef) ||
        !aligned16(g->scratch))
      return fail(MPG_ERR_INVALID_ARG, "invalid vMF guide (cells %d, capacity %d)", g->n_cells, g->capacity);
    out.kind = MPG_GUIDE_VMF;
    out.n_cells = g->n_cells;
    out.cell_start = g->cell_start;
    out.lobe_key = g->lobe_key;
    out.lobe = reinterpret_cast<const float4*>(g->lobe);
    out.lobe_prefix = g->lobe_prefix;
    out.lobe_coef = g->lobe_coef;
    return MPG_OK;
  }
  if (g->kind != MPG_GUIDE_HISTOGRAM) return fail(MPG_ERR_INVALID_ARG, "unknown guide kind %d", g->kind);
  if (g->n_cells <= 0 || g->n_theta <= 0 || g->n_phi < 2 || (g->n_phi & 1) || !aligned16(g->counts) ||
      !aligned16(g->cdf) || !g->cos_theta || !g->phi_cos || !g->phi_sin)
    return fail(MPG_ERR_INVALID_ARG, "invalid guide (cells %d, theta %d, phi %d)", g->n_cells, g->n_theta, g->n_phi);
  out.n_cells = g->n_cells; out.n_theta = g->n_theta; out.n_phi = g->n_phi; out.bins = g->n_theta * g->n_phi;
  out.counts = g->counts; out.cdf = g->cdf; out.cos_theta = g->cos_theta; out.phi_cos = g->phi_cos;
  out.phi_sin = g->phi_sin;
  out.kind = MPG_GUIDE_HISTOGRAM;
  return MPG_OK;
}

cudaEvent_t pooled_event(mpg_ctx* ctx);
template <class F>
void timed(mpg_ctx* ctx, int kind, cudaStream_t st, int n, F fn);

// A call recorded into a graph cannot grow the context's buffers.
mpg_status capture_grow_error() {
  return fail(MPG_ERR_INVALID_ARG,
              "the context's buffers are too small for this batch and cannot grow during a capture: "
              "run the same calls once uncaptured first");
}

// Which per-K launches to make, and over which work list.
struct Plan {
  int K[MAXK];
  int nK = 0;
  DWork w{nullptr, nullptr, nullptr};
  bool concurrent = false;
};

mpg_status make_plan(mpg_ctx* ctx, const mpg_chains* c, const mpg_params* p, int status_filter, cudaStream_t st,
                     Plan& plan) {
  if (p->k_uniform >= 1) {
    plan.K[0] = p->k_uniform;
    plan.nK = 1;
    return MPG_OK;
  }
  for (int k = 1; k <= MAXK; ++k) plan.K[plan.nK++] = k;
  if (p->walk_mode == MPG_WALK_PLAIN) return MPG_OK;
  if (ctx->order_cap < c->B) {
    if (ctx->capturing) return capture_grow_error();
    if (ctx->d_order) cudaFree(ctx->d_order);
    ctx->d_order = nullptr;
    CUDA_TRY(cudaMalloc(&ctx->d_order, sizeof(int) * (size_t)c->B));
    ctx->order_cap = c->B;
  }
  cudaError_t be = cudaSuccess;
  timed(ctx, MPG_KERNEL_AUX, st, 3, [&] {
    be = launch_bucket(c->k, c->status, status_filter, c->B, ctx->d_count, ctx->d_base, ctx->d_cursor, ctx->d_order,
                       ctx->sms, st);
  });
  if (be != cudaSuccess) return fail(MPG_ERR_CUDA, "bucket: %s", cudaGetErrorString(be));
  plan.w = DWork{ctx->d_order, ctx->d_base, ctx->d_count};
  plan.concurrent = true;
  return MPG_OK;
}

cudaEvent_t pooled_event(mpg_ctx* ctx) {
  if (!ctx->pool.empty()) {
    cudaEvent_t e = ctx->pool.back();
    ctx->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launches `n` kernels through fn() on stream st, bracketed by events when
// launch profiling is on.
template <class F>
void timed(mpg_ctx* ctx, int kind, cudaStream_t st, int n, F fn) {
  mpg_ctx::ProfRec r{kind, nullptr, nullptr};
  if (ctx->profile) {
    r.a = pooled_event(ctx);
    cudaEventRecord(r.a, st);
  }
  fn();
  ctx->launches += n;
  if (ctx->profile) {
    r.b = pooled_event(ctx);
    cudaEventRecord(r.b, st);
    ctx->prof.push_back(r);
  }
}

DCtx dctx(mpg_ctx* ctx, int kind) {
  return DCtx{ctx->d_err, ctx->stats_on ? ctx->d_stats + 16 * kind : nullptr, ctx->capturing ? ctx->cap_rng : nullptr,
              0u};
}

// Runs fn(K, stream) for each planned K, on forked streams when concurrent.
// With launch timing on (mpg_ctx_set_profile), the lengths run one after
// another on the call's stream, so that each bracketed launch has the GPU to
// itself and its events time that kernel alone.
template <class F>
mpg_status run_plan(mpg_ctx* ctx, const Plan& plan, cudaStream_t st, F fn) {
  if (!plan.concurrent || ctx->profile) {
    for (int i = 0; i < plan.nK; ++i) fn(plan.K[i], st);
    LAUNCH_CHECK("kernel launch");
    return MPG_OK;
  }
  CUDA_TRY(cudaEventRecord(ctx->ev_fork, st));
  for (int i = 0; i < plan.nK; ++i) {
    CUDA_TRY(cudaStreamWaitEvent(ctx->aux[i], ctx->ev_fork, 0));
    fn(plan.K[i], ctx->aux[i]);
    CUDA_TRY(cudaEventRecord(ctx->ev_join[i], ctx->aux[i]));
  }
  for (int i = 0; i < plan.nK; ++i) CUDA_TRY(cudaStreamWaitEvent(st, ctx->ev_join[i], 0));
  LAUNCH_CHECK("kernel launch");
  return MPG_OK;
}

int block_of(const mpg_params* p) { return p->block_threads > 0 ? p->block_threads : 128; }

// Persistent walk kernel of the batched mode: occupancy entry and block size
// (the group form runs 128 threads per CTA).
int walk_which(const mpg_params* p) { return (p->walk_group & 1) ? 7 : 4; }
int walk_block(const mpg_params* p) { return (p->walk_group & 1) ? 128 : block_of(p); }
int round_which(const mpg_params* p) { return (p->walk_group & 2) ? 8 : 6; }
int round_block(const mpg_params* p) { return (p->walk_group & 2) ? 128 : block_of(p); }

// Synchronous Bernoulli rounds before the parallel ones (-1: none, 0: default).
int sync_rounds_of(const mpg_params* p) { return p->trial_sync_rounds < 0 ? 0 : p->trial_sync_rounds > 0 ? p->trial_sync_rounds : 2; }

int grid_of(mpg_ctx* ctx, const mpg_params* P, int which, int K, int block, int B, bool persistent) {
  int per_sm = blocks_per_sm(which, K, ctx->stats_on, block);
  if (P->ctas_per_sm > 0) per_sm = std::min(per_sm, P->ctas_per_sm);
  int full = ctx->sms * per_sm;
  int need = (B + block - 1) / block;
  return persistent ? std::max(1, std::min(full, need)) : std::max(1, need);
}

}  // namespace

extern "C" {

const char* mpg_last_error(void) { return g_last_error.c_str(); }
int32_t mpg_version(void) { return 1; }

mpg_status mpg_ctx_create(int32_t device, mpg_ctx** out) {
  if (!out) return fail(MPG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int n = 0;
  CUDA_TRY(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return fail(MPG_ERR_INVALID_ARG, "device %d out of range (%d devices)", device, n);
  CUDA_TRY(cudaSetDevice(device));
  mpg_ctx* c = new mpg_ctx();
  c->device = device;
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  bool ok = cudaMalloc(&c->d_err, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&c->d_stats, sizeof(unsigned long long) * 16 * MPG_KERNEL_KINDS) == cudaSuccess &&
            cudaMalloc(&c->d_count, sizeof(int) * 16) == cudaSuccess &&
            cudaMalloc(&c->d_base, sizeof(int) * 16) == cudaSuccess &&
            cudaMalloc(&c->d_cursor, sizeof(int) * 16) == cudaSuccess &&
            cudaMalloc(&c->d_scratch, sizeof(float) * 16) == cudaSuccess &&
            cudaMalloc(&c->d_queue, sizeof(int) * 32 * (MAXK + 1)) == cudaSuccess &&
            cudaMalloc(&c->d_nlist, sizeof(int) * 2 * (MAXK + 1)) == cudaSuccess &&
            cudaMalloc(&c->d_zero, sizeof(int) * (MAXK + 1)) == cudaSuccess &&
            cudaMalloc(&c->d_fp64_count, sizeof(int) * (MAXK + 1)) == cudaSuccess &&
            cudaMalloc(&c->d_npairs, sizeof(int) * (MAXK + 1)) == cudaSuccess &&
            cudaMemset(c->d_zero, 0, sizeof(int) * (MAXK + 1)) == cudaSuccess &&
            cudaMemset(c->d_err, 0, sizeof(int)) == cudaSuccess &&
            cudaMemset(c->d_stats, 0, sizeof(unsigned long long) * 16 * MPG_KERNEL_KINDS) == cudaSuccess &&
            cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; ok && i < MAXK; ++i)
    ok = cudaStreamCreateWithFlags(&c->aux[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->ev_join[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    mpg_ctx_destroy(c);
    return fail(MPG_ERR_OOM, "context allocation failed: %s", cudaGetErrorString(cudaGetLastError()));
  }
  *out = c;
  return MPG_OK;
}

void mpg_ctx_destroy(mpg_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaFree(c->d_err); cudaFree(c->d_stats); cudaFree(c->d_order); cudaFree(c->d_count);
  cudaFree(c->d_base); cudaFree(c->d_cursor); cudaFree(c->d_scratch);
  cudaFree(c->d_queue); cudaFree(c->d_nlist); cudaFree(c->d_zero); cudaFree(c->d_fp64); cudaFree(c->d_fp64_count);
  cudaFree(c->d_list[0]); cudaFree(c->d_list[1]); cudaFree(c->d_nbest); cudaFree(c->d_pairs); cudaFree(c->d_npairs);
  cudaFree(c->d_rec); cudaFree(c->d_nsum);
  cudaFree(c->t_x); cudaFree(c->t_surf); cudaFree(c->t_prim); cudaFree(c->t_bary); cudaFree(c->t_status);
  cudaFree(c->t_iters);
  for (int i = 0; i < MAXK; ++i) {
    if (c->aux[i]) cudaStreamDestroy(c->aux[i]);
    if (c->ev_join[i]) cudaEventDestroy(c->ev_join[i]);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  for (auto& r : c->prof) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
  delete c;
  (void)cudaGetLastError();  // a failure here must not surface in a later call's launch check
}

mpg_status mpg_ctx_sync(mpg_ctx* c, cudaStream_t st) {
  if (!c) return fail(MPG_ERR_INVALID_ARG, "ctx is NULL");
  CUDA_TRY(cudaSetDevice(c->device));
  CUDA_TRY(cudaStreamSynchronize(st));
  int err = 0;
  CUDA_TRY(cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    CUDA_TRY(cudaMemset(c->d_err, 0, sizeof(int)));
    if (err & ERR_BVH_STACK) return fail(MPG_ERR_LIMIT, "BVH traversal stack overflow (device flag %d)", err);
    if (err & ERR_VMF_RECORD)
      return fail(MPG_ERR_INVALID_ARG, "device-side argument error (flag %d): vMF record with a cell, length or "
                  "types out of range (left out)", err);
    return fail(MPG_ERR_INVALID_ARG, "device-side argument error (flag %d): guide cell out of range", err);
  }
  return MPG_OK;
}

mpg_status mpg_ctx_stats(mpg_ctx* c, int32_t kind, mpg_stats* out, int32_t reset, cudaStream_t st) {
  if (!c) return fail(MPG_ERR_INVALID_ARG, "ctx is NULL");
  if (kind < -1 || kind >= MPG_KERNEL_KINDS) return fail(MPG_ERR_INVALID_ARG, "kernel kind %d out of range", kind);
  CUDA_TRY(cudaSetDevice(c->device));
  static_assert(sizeof(mpg_stats) == 16 * sizeof(uint64_t), "stats layout");
  if (out) {
    unsigned long long v[16 * MPG_KERNEL_KINDS];
    CUDA_TRY(cudaMemcpyAsync(v, c->d_stats, sizeof(v), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    uint64_t acc[16] = {0};
    for (int k = 0; k < MPG_KERNEL_KINDS; ++k)
      if (kind < 0 || kind == k)
        for (int i = 0; i < 16; ++i) acc[i] += v[16 * k + i];
    memcpy(out, acc, sizeof(mpg_stats));
  }
  if (reset) {
    if (kind < 0) CUDA_TRY(cudaMemsetAsync(c->d_stats, 0, sizeof(unsigned long long) * 16 * MPG_KERNEL_KINDS, st));
    else CUDA_TRY(cudaMemsetAsync(c->d_stats + 16 * kind, 0, sizeof(unsigned long long) * 16, st));
  }
  return MPG_OK;
}

mpg_status mpg_ctx_set_profile(mpg_ctx* c, int32_t on) {
  if (!c) return fail(MPG_ERR_INVALID_ARG, "ctx is NULL");
  c->profile = on != 0;
  return MPG_OK;
}

mpg_status mpg_ctx_profile(mpg_ctx* c, int32_t kind, double* ms, int64_t* launches, int32_t reset) {
  if (!c) return fail(MPG_ERR_INVALID_ARG, "ctx is NULL");
  if (kind < -1 || kind >= MPG_KERNEL_KINDS) return fail(MPG_ERR_INVALID_ARG, "kernel kind %d out of range", kind);
  CUDA_TRY(cudaSetDevice(c->device));
  for (auto& r : c->prof) {
    CUDA_TRY(cudaEventSynchronize(r.b));
    float t = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&t, r.a, r.b));
    c->prof_ms[r.kind] += t;
    c->prof_n[r.kind] += 1;
    c->pool.push_back(r.a);
    c->pool.push_back(r.b);
  }
  c->prof.clear();
  double m = 0.0;
  int64_t n = 0;
  for (int k = 0; k < MPG_KERNEL_KINDS; ++k)
    if (kind < 0 || kind == k) { m += c->prof_ms[k]; n += c->prof_n[k]; }
  if (ms) *ms = m;
  if (launches) *launches = n;
  if (reset)
    for (int k = 0; k < MPG_KERNEL_KINDS; ++k) { c->prof_ms[k] = 0.0; c->prof_n[k] = 0; }
  return MPG_OK;
}

mpg_status mpg_ctx_launches(mpg_ctx* c, int64_t* count) {
  if (!c || !count) return fail(MPG_ERR_INVALID_ARG, "ctx or count is NULL");
  *count = c->launches;
  return MPG_OK;
}

mpg_status mpg_ctx_set_stats(mpg_ctx* c, int32_t on) {
  if (!c) return fail(MPG_ERR_INVALID_ARG, "ctx is NULL");
  c->stats_on = on != 0;
  return MPG_OK;
}

mpg_status mpg_scene_create(mpg_ctx* ctx, const double* surfaces, int32_t n_surf, const double* hf_desc,
                            const double* hf_heights, int32_t n_hf, const double* targets, int32_t n_targets,
                            const double* light, mpg_scene** out) {
  if (!ctx || !out || !light || (n_surf > 0 && !surfaces) || (n_hf > 0 && (!hf_desc || !hf_heights)) ||
      (n_targets > 0 && !targets))
    return fail(MPG_ERR_INVALID_ARG, "NULL scene table");
  if (n_surf < 1 || n_surf > MAX_SURF || n_hf < 0 || n_hf > MAX_HF || n_targets < 0 || n_targets > MAX_TG)
    return fail(MPG_ERR_INVALID_ARG, "scene sizes out of range (surfaces %d <= %d, heightfields %d <= %d, targets %d <= %d)",
                n_surf, MAX_SURF, n_hf, MAX_HF, n_targets, MAX_TG);
  *out = nullptr;
  CUDA_TRY(cudaSetDevice(ctx->device));
  mpg_scene* sc = new mpg_scene();
  sc->device = ctx->device;
  DScene& S = sc->S;
  memset(&S, 0, sizeof(S));
  S.n_surf = n_surf;
  S.n_hf = n_hf;
  S.n_tg = n_targets;
  size_t hoff = 0;
  for (int h = 0; h < n_hf; ++h) {
    const double* d = hf_desc + 6 * h;
    int nx = (int)d[0], ny = (int)d[1];
    if (nx < 2 || ny < 2 || (long long)nx * ny > (1 << 26)) {
      mpg_scene_destroy(sc);
      return fail(MPG_ERR_INVALID_ARG, "heightfield %d: bad grid %d x %d", h, nx, ny);
    }
    std::vector<float4> P, N;
    heightfield_mesh(nx, ny, d[2], d[3], d[4], d[5], hf_heights + hoff, P, N);
    hoff += (size_t)nx * ny;
    BVHBuilder bb;
    int nt = 2 * (nx - 1) * (ny - 1);
    bb.tris.resize(nt);
    for (int t = 0; t < nt; ++t) {
      int quad = t / 2, tt = t % 2, i = quad % (nx - 1), j = quad / (nx - 1);
      int v00 = j * nx + i, v[3] = {v00, tt == 0 ? v00 + 1 : v00 + nx + 1, tt == 0 ? v00 + nx + 1 : v00 + nx};
      BuildTri& bt = bb.tris[t];
      bt.id = t;
      for (int a = 0; a < 3; ++a) {
        float p[3] = {P[v[a]].x, P[v[a]].y, P[v[a]].z};
        bt.box.grow(p);
      }
      for (int a = 0; a < 3; ++a) bt.c[a] = 0.5f * (bt.box.lo[a] + bt.box.hi[a]);
    }
    // build() allocates the first internal node first, so the root lands in slot 0
    ChildRef root = bb.build(0, nt, 0);
    if (root.count > 0) {  // whole mesh in one leaf: a root node whose two children are that leaf
      bb.nodes.resize(4);
      bb.write_node(0, root, root);
    }
    std::vector<float4> tris((size_t)nt * 3);
    for (int s = 0; s < nt; ++s) {
      int t = bb.leaf_order[s];
      int quad = t / 2, tt = t % 2, i = quad % (nx - 1), j = quad / (nx - 1);
      int v00 = j * nx + i, v1 = tt == 0 ? v00 + 1 : v00 + nx + 1, v2 = tt == 0 ? v00 + nx + 1 : v00 + nx;
      float4 a = P[v00], b = P[v1], c = P[v2];
      float4 v0 = a;
      memcpy(&v0.w, &t, sizeof(float));  // primitive id stored as int bits
      tris[3 * (size_t)s + 0] = v0;
      tris[3 * (size_t)s + 1] = make_float4(b.x - a.x, b.y - a.y, b.z - a.z, 0.f);
      tris[3 * (size_t)s + 2] = make_float4(c.x - a.x, c.y - a.y, c.z - a.z, 0.f);
    }
    DHF& H = S.hf[h];
    H.nx = nx; H.ny = ny; H.surf = -1;
    H.x0 = (float)d[2]; H.y0 = (float)d[3];
    H.dx = (float)((d[4] - d[2]) / (nx - 1)); H.dy = (float)((d[5] - d[3]) / (ny - 1));
    H.n_nodes = (int)(bb.nodes.size() / 4);
    mpg_status st;
    if ((st = upload(sc, P, &H.P)) || (st = upload(sc, N, &H.N)) || (st = upload(sc, bb.nodes, &H.nodes)) ||
        (st = upload(sc, tris, &H.tris))) {
      mpg_scene_destroy(sc);
      return st;
    }
    sc->n_nodes.push_back(H.n_nodes);
    sc->n_tris.push_back(nt);
    // the tree's shape for the refit: nodes are numbered parents first
    std::vector<int> parent(H.n_nodes, -1), ninner(H.n_nodes, 0);
    for (int v = 0; v < H.n_nodes; ++v) {
      int4 ch;
      memcpy(&ch, &bb.nodes[4 * (size_t)v + 3], sizeof(int4));
      if (ch.z == 0) { parent[ch.x] = v; ninner[v]++; }
      if (ch.w == 0) { parent[ch.y] = v; ninner[v]++; }
    }
    const int* dp = nullptr;
    const int* dn = nullptr;
    const int* dc = nullptr;
    if ((st = upload(sc, parent, &dp)) || (st = upload(sc, ninner, &dn)) || (st = upload(sc, ninner, &dc))) {
      mpg_scene_destroy(sc);
      return st;
    }
    sc->hf_extent.push_back({d[2], d[3], d[4], d[5]});
    sc->hf_parent.push_back(dp);
    sc->hf_ninner.push_back(dn);
    sc->hf_count.push_back(const_cast<int*>(dc));
  }
  for (int s = 0; s < n_surf; ++s) {
    const double* r = surfaces + 24 * s;
    DSurf& f = S.s[s];
    f.type = (int)r[0]; f.mat = (int)r[1]; f.etaF = (float)r[2]; f.etaB = (float)r[3];
    f.c = ld3(r + 4); f.r = (float)r[7]; f.cap_cos = (float)r[11]; f.hf = (int)r[18];
    double ax = dlen(r + 8);
    f.axis = ax > 0 ? make_float3((float)(r[8] / ax), (float)(r[9] / ax), (float)(r[10] / ax)) : make_float3(0, 0, 1);
    if (f.type == SURF_CAP) f.axis = ld3(r + 8);
    f.ex = ld3(r + 12); f.ey = ld3(r + 15);
    f.ex2 = (float)(r[12] * r[12] + r[13] * r[13] + r[14] * r[14]);
    f.ey2 = (float)(r[15] * r[15] + r[16] * r[16] + r[17] * r[17]);
    bool bad = f.type < SURF_SPHERE || f.type > SURF_HEIGHTFIELD || (f.mat != MAT_MIRROR && f.mat != MAT_DIELECTRIC) ||
               ((f.type == SURF_SPHERE || f.type == SURF_CAP) && !(f.r > 0.0f)) ||
               (f.type == SURF_HEIGHTFIELD && (f.hf < 0 || f.hf >= n_hf)) ||
               (f.mat == MAT_DIELECTRIC && !(f.etaF > 0.0f && f.etaB > 0.0f));
    if (bad) {
      mpg_scene_destroy(sc);
      return fail(MPG_ERR_INVALID_ARG, "surface %d is invalid", s);
    }
    if (f.type == SURF_HEIGHTFIELD) S.hf[f.hf].surf = s;
  }
  for (int t = 0; t < n_targets; ++t) {
    const double* r = targets + 16 * t;
    DTarget& g = S.tg[t];
    g.type = (int)r[0]; g.c = ld3(r + 1); g.r = (float)r[4]; g.ex = ld3(r + 5); g.ey = ld3(r + 8);
    double nl = dlen(r + 11);
    g.n = nl > 0 ? make_float3((float)(r[11] / nl), (float)(r[12] / nl), (float)(r[13] / nl)) : make_float3(0, 0, 1);
    g.area = (float)(4.0 * dlen(r + 5) * dlen(r + 8));
  }
  DLight& L = S.L;
  L.type = (int)light[0];
  L.p = ld3(light + 1);
  double nl = dlen(light + 4);
  L.n = nl > 0 ? make_float3((float)(light[4] / nl), (float)(light[5] / nl), (float)(light[6] / nl)) : make_float3(0, 0, -1);
  double ex = dlen(light + 7), ey = dlen(light + 10);
  L.exu = ex > 0 ? make_float3((float)(light[7] / ex), (float)(light[8] / ex), (float)(light[9] / ex)) : make_float3(1, 0, 0);
  L.eyu = ey > 0 ? make_float3((float)(light[10] / ey), (float)(light[11] / ey), (float)(light[12] / ey)) : make_float3(0, 1, 0);
  L.power = (float)light[13];
  L.area = L.type == LIGHT_RECT ? (float)(4.0 * ex * ey) : 1.0f;
  if (L.type != LIGHT_POINT && L.type != LIGHT_RECT) {
    mpg_scene_destroy(sc);
    return fail(MPG_ERR_INVALID_ARG, "light type %d is invalid", L.type);
  }
  *out = sc;
  return MPG_OK;
}

void mpg_scene_destroy(mpg_scene* sc) {
  if (!sc) return;
  cudaSetDevice(sc->device);
  for (void* p : sc->allocs) cudaFree(p);
  delete sc;
  (void)cudaGetLastError();  // a failure here must not surface in a later call's launch check
}

mpg_status mpg_scene_set_heights(mpg_ctx* ctx, mpg_scene* sc, int32_t h, const float* heights, cudaStream_t st) {
  if (!ctx || !sc || !aligned16(heights)) return fail(MPG_ERR_INVALID_ARG, "ctx, scene or heights NULL or unaligned");
  if (h < 0 || h >= (int)sc->n_nodes.size()) return fail(MPG_ERR_INVALID_ARG, "no heightfield %d", h);
  CUDA_TRY(cudaSetDevice(ctx->device));
  cudaError_t e = cudaSuccess;
  timed(ctx, MPG_KERNEL_AUX, st, 3, [&] {
    e = launch_hf_update(sc->S.hf[h], sc->hf_extent[h].data(), heights, sc->n_tris[h], sc->hf_parent[h],
                         sc->hf_ninner[h], sc->hf_count[h], st);
  });
  if (e != cudaSuccess) return fail(MPG_ERR_CUDA, "heightfield update: %s", cudaGetErrorString(e));
  return MPG_OK;
}

mpg_status mpg_scene_info(const mpg_scene* sc, int32_t h, int32_t* n_nodes, int32_t* n_tris) {
  if (!sc || h < 0 || h >= (int)sc->n_nodes.size()) return fail(MPG_ERR_INVALID_ARG, "no heightfield %d", h);
  if (n_nodes) *n_nodes = sc->n_nodes[h];
  if (n_tris) *n_tris = sc->n_tris[h];
  return MPG_OK;
}

mpg_status mpg_sample_seeds(mpg_ctx* ctx, const mpg_scene* sc, const mpg_guide* guide, mpg_chains* chains,
                            uint64_t rng_seed, uint64_t rng_offset, const mpg_params* P, cudaStream_t st) {
  if (!ctx || !sc) return fail(MPG_ERR_INVALID_ARG, "ctx or scene is NULL");
  if (chains && chains->B == 0 && chains->Q == 0) return MPG_OK;  // empty batch
  mpg_status s;
  if ((s = check_chains(chains, true)) || (s = check_params(P))) return s;
  DGuide g;
  if (guide && (s = check_guide(guide, g))) return s;
  CUDA_TRY(cudaSetDevice(ctx->device));
  DChains c = to_dev(chains);
  uint2 key = make_uint2((uint32_t)rng_seed, (uint32_t)(rng_seed >> 32));
  DCtx dc = dctx(ctx, MPG_KERNEL_SEED);
  if (P->walk_mode == MPG_WALK_BATCHED) {
    // one launch over the batch in chain order, every length at once
    const int grid = std::max(1, std::min((chains->B + 127) / 128, ctx->sms * 16));
    timed(ctx, MPG_KERNEL_SEED, st, 1,
          [&] { launch_seed_all(sc->S, guide ? &g : nullptr, c, key, rng_offset, *P, dc, grid, st); });
    LAUNCH_CHECK("seed");
    return MPG_OK;
  }
  Plan plan;
  mpg_params Pn = *P;
  if ((s = make_plan(ctx, chains, &Pn, -1, st, plan))) return s;
  int block = block_of(P);
  return run_plan(ctx, plan, st, [&](int K, cudaStream_t s2) {
    timed(ctx, MPG_KERNEL_SEED, s2, 1, [&] {
      launch_seed(K, ctx->stats_on, sc->S, guide ? &g : nullptr, c, plan.w, key, rng_offset, *P, dc,
                  grid_of(ctx, P, 0, K, block, c.B, true), block, s2);
    });
  });
}

mpg_status mpg_sample_offsets(mpg_ctx* ctx, const mpg_chains* chains, float alpha, uint64_t rng_seed,
                              uint64_t rng_offset, float* offset, cudaStream_t st) {
  if (!ctx) return fail(MPG_ERR_INVALID_ARG, "ctx is NULL");
  if (chains && chains->B == 0 && chains->Q == 0) return MPG_OK;  // empty batch
  if (!chains || chains->B <= 0 || !aligned16(chains->k) || !aligned16(offset))
    return fail(MPG_ERR_INVALID_ARG, "chains (B > 0, k) and offset must be 16-byte aligned device arrays");
  if (!(alpha > 0.0f && alpha <= 1.0f)) return fail(MPG_ERR_INVALID_ARG, "roughness alpha %g outside (0, 1]", alpha);
  CUDA_TRY(cudaSetDevice(ctx->device));
  DChains c = to_dev(chains);
  uint2 key = make_uint2((uint32_t)rng_seed, (uint32_t)(rng_seed >> 32));
  timed(ctx, MPG_KERNEL_SEED, st, 1,
        [&] { launch_offsets(c, alpha, key, rng_offset, dctx(ctx, MPG_KERNEL_SEED), offset, ctx->sms, st); });
  LAUNCH_CHECK("offsets");
  return MPG_OK;
}

mpg_status mpg_manifold_walk(mpg_ctx* ctx, const mpg_scene* sc, mpg_chains* chains, const mpg_params* Pin,
                             cudaStream_t st) {
  if (!ctx || !sc) return fail(MPG_ERR_INVALID_ARG, "ctx or scene is NULL");
  if (chains && chains->B == 0 && chains->Q == 0) return MPG_OK;  // empty batch
  mpg_status s;
  if ((s = check_chains(chains, false)) || (s = check_params(Pin))) return s;
  mpg_params Pg = *Pin;
  if (chains->offset) Pg.walk_mode = MPG_WALK_PLAIN;  // glossy chains: one launch per length, one thread per chain
  const mpg_params* P = &Pg;
  CUDA_TRY(cudaSetDevice(ctx->device));
  Plan plan;
  if ((s = make_plan(ctx, chains, P, ST_SEEDED, st, plan))) return s;
  DChains c = to_dev(chains);
  DCtx dc = dctx(ctx, MPG_KERNEL_WALK);
  int block = block_of(P);
  if (P->walk_mode == MPG_WALK_BATCHED) {
    CUDA_TRY(cudaMemsetAsync(ctx->d_queue, 0, sizeof(int) * 32 * (MAXK + 1), st));
    return run_plan(ctx, plan, st, [&](int K, cudaStream_t s2) {
      timed(ctx, MPG_KERNEL_WALK, s2, 1, [&] {
        launch_walk_p(K, ctx->stats_on, sc->S, c, plan.w, *P, dc, ctx->d_queue + 32 * K,
                      grid_of(ctx, P, walk_which(P), K, walk_block(P), c.B, true), walk_block(P), s2);
      });
    });
  }
  return run_plan(ctx, plan, st, [&](int K, cudaStream_t s2) {
    timed(ctx, MPG_KERNEL_WALK, s2, 1, [&] {
      launch_walk(K, ctx->stats_on, sc->S, c, plan.w, *P, dc, grid_of(ctx, P, 1, K, block, c.B, true), block, s2);
    });
  });
}

mpg_status mpg_chain_contribution(mpg_ctx* ctx, const mpg_scene* sc, const mpg_guide* guide, const mpg_chains* chains,
                                  uint64_t rng_seed, uint64_t rng_offset, const mpg_params* Pin, float* G,
                                  float* kappa, float* T, uint32_t* trials, uint8_t* capped, float* contrib, float* E,
                                  cudaStream_t st) {
  if (!ctx || !sc) return fail(MPG_ERR_INVALID_ARG, "ctx or scene is NULL");
  if (chains && chains->B == 0 && chains->Q == 0) return MPG_OK;  // empty batch
  mpg_status s;
  if ((s = check_chains(chains, false)) || (s = check_params(Pin))) return s;
  mpg_params Pg = *Pin;
  if (chains->offset) Pg.walk_mode = MPG_WALK_PLAIN;  // glossy chains: the plain kernels
  const mpg_params* P = &Pg;
  if (!aligned16(T) || !aligned16(contrib) || !aligned16(E))
    return fail(MPG_ERR_INVALID_ARG, "T, contrib and E must be non-NULL 16-byte aligned device arrays");
  DGuide g;
  if (guide && (s = check_guide(guide, g))) return s;
  CUDA_TRY(cudaSetDevice(ctx->device));
  Plan plan;
  if ((s = make_plan(ctx, chains, P, ST_CONVERGED, st, plan))) return s;
  DChains c = to_dev(chains);
  DCtx dcc = dctx(ctx, MPG_KERNEL_CONTRIB), dcb = dctx(ctx, MPG_KERNEL_BERNOULLI), dcw = dctx(ctx, MPG_KERNEL_WALK);
  if (ctx->fp64_cap < c.B) {
    if (ctx->capturing) return capture_grow_error();
    cudaFree(ctx->d_fp64);
    ctx->d_fp64 = nullptr;
    ctx->fp64_cap = 0;
    CUDA_TRY(cudaMalloc(&ctx->d_fp64, sizeof(int) * (size_t)c.B));
    ctx->fp64_cap = c.B;
  }
  CUDA_TRY(cudaMemsetAsync(ctx->d_fp64_count, 0, sizeof(int) * (MAXK + 1), st));
  const int repeats = std::max(1, P->bern_repeats);
  if (repeats > 1 && !trials && ctx->nsum_cap < c.B) {  // the repeats' sum of N needs a home
    if (ctx->capturing) return capture_grow_error();
    cudaFree(ctx->d_nsum);
    ctx->d_nsum = nullptr;
    ctx->nsum_cap = 0;
    CUDA_TRY(cudaMalloc(&ctx->d_nsum, sizeof(uint32_t) * (size_t)c.B));
    ctx->nsum_cap = c.B;
  }
  DOut o{G, kappa, T, (repeats > 1 && !trials) ? ctx->d_nsum : trials, capped, contrib, ctx->d_fp64, nullptr, nullptr,
         0, repeats};
  uint2 key = make_uint2((uint32_t)rng_seed, (uint32_t)(rng_seed >> 32));
  int block = block_of(P);
  if (plan.w.order) {
    // zero the outputs of chains outside the converged buckets
    CUDA_TRY(cudaMemsetAsync(T, 0, sizeof(float) * (size_t)c.B, st));
    CUDA_TRY(cudaMemsetAsync(contrib, 0, sizeof(float) * (size_t)c.B, st));
    if (G) CUDA_TRY(cudaMemsetAsync(G, 0, sizeof(float) * (size_t)c.B, st));
    if (kappa) CUDA_TRY(cudaMemsetAsync(kappa, 0, sizeof(float) * (size_t)c.B, st));
    if (trials) CUDA_TRY(cudaMemsetAsync(trials, 0, sizeof(uint32_t) * (size_t)c.B, st));
    if (capped) CUDA_TRY(cudaMemsetAsync(capped, 0, (size_t)c.B, st));
  }
  const bool batched = P->walk_mode == MPG_WALK_BATCHED;
  if (batched) {
    if (ctx->bern_cap < c.B) {
      if (ctx->capturing) return capture_grow_error();
      void** bufs[] = {(void**)&ctx->d_list[0], (void**)&ctx->d_list[1], (void**)&ctx->d_nbest, (void**)&ctx->t_x,
                       (void**)&ctx->t_surf, (void**)&ctx->t_prim, (void**)&ctx->t_bary, (void**)&ctx->t_status,
                       (void**)&ctx->t_iters, (void**)&ctx->d_pairs};
      for (void** b : bufs) { cudaFree(*b); *b = nullptr; }
      ctx->bern_cap = 0;
      size_t n = (size_t)c.B;
      CUDA_TRY(cudaMalloc(&ctx->d_list[0], sizeof(int) * n));
      CUDA_TRY(cudaMalloc(&ctx->d_list[1], sizeof(int) * n));
      CUDA_TRY(cudaMalloc(&ctx->d_nbest, sizeof(unsigned) * n));
      CUDA_TRY(cudaMalloc(&ctx->t_x, sizeof(float) * 3 * MAXK * n));
      CUDA_TRY(cudaMalloc(&ctx->t_surf, sizeof(int32_t) * MAXK * n));
      CUDA_TRY(cudaMalloc(&ctx->t_prim, sizeof(int32_t) * MAXK * n));
      CUDA_TRY(cudaMalloc(&ctx->t_bary, sizeof(float) * 2 * MAXK * n));
      CUDA_TRY(cudaMalloc(&ctx->t_status, n));
      CUDA_TRY(cudaMalloc(&ctx->t_iters, n));
      CUDA_TRY(cudaMalloc(&ctx->d_pairs, sizeof(uint2) * PAIRS_PER_CHAIN * n));
      ctx->bern_cap = c.B;
    }
    CUDA_TRY(cudaMemsetAsync(ctx->d_queue, 0, sizeof(int) * 32 * (MAXK + 1), st));
    CUDA_TRY(cudaMemsetAsync(ctx->d_nlist, 0, sizeof(int) * 2 * (MAXK + 1), st));
  }
  DChains tc = c;  // trial chains: same separators and types, own vertex state
  tc.x = ctx->t_x; tc.surf = ctx->t_surf; tc.prim = ctx->t_prim; tc.bary = ctx->t_bary;
  tc.status = ctx->t_status; tc.iters = ctx->t_iters; tc.pdf = nullptr;
  s = run_plan(ctx, plan, st, [&](int K, cudaStream_t s2) {
    // each length queues its FP64 chains in its own bucket region of the list
    DOut oK = o;
    oK.fp64_count = ctx->d_fp64_count + K;
    oK.fp64_base = (plan.w.base ? plan.w.base : ctx->d_zero) + K;
    timed(ctx, MPG_KERNEL_CONTRIB, s2, c.offset ? 1 : 2, [&] {
      if (c.offset) {  // glossy chains: admissibility and the estimate W in FP64
        launch_glossy(K, sc->S, c, plan.w, *P, oK, dcc, grid_of(ctx, P, 2, K, 64, c.B, true), s2);
        return;
      }
      launch_contrib(K, ctx->stats_on, sc->S, c, plan.w, *P, oK, dcc, grid_of(ctx, P, 2, K, block, c.B, true), block,
                     s2);
      launch_contrib64(K, sc->S, c, *P, oK, ctx->sms * 4, s2);
    });
    if (!batched) {
      timed(ctx, MPG_KERNEL_BERNOULLI, s2, 1, [&] {
        launch_bernoulli(K, ctx->stats_on, sc->S, guide ? &g : nullptr, c, plan.w, key, rng_offset, *P, o, dcb,
                         grid_of(ctx, P, 3, K, block, c.B, true), block, s2);
      });
      return;
    }
    // Synchronous rounds t = 1..T1: every chain without a hit draws and walks
    // trial t; then parallel rounds of TB = TB0, 4 TB0, 16 TB0, ... trials per
    // remaining chain, issued trial-major.  Each round lasts at least as long
    // as its slowest walk, so few rounds keep the pass short.
    const int T1 = std::min(sync_rounds_of(P), P->max_trials);
    int* lists[2] = {ctx->d_list[0], ctx->d_list[1]};
    int* counts[2] = {ctx->d_nlist, ctx->d_nlist + (MAXK + 1)};
    const int* base = plan.w.base ? plan.w.base : ctx->d_zero;
    int* q = ctx->d_queue + 32 * K;
    int small_grid = ctx->sms * 4;
    for (int rep = 0; rep < repeats; ++rep) {  // independent estimates, trial counters t | rep << 24
      DOut oR = o;
      oR.rep = rep;
      DCtx dcr = dcb;
      dcr.trial_base = (uint32_t)rep << 24;
      if (rep > 0) {  // this length's list lengths and queue counters start from zero again
        cudaMemsetAsync(q, 0, sizeof(int) * 32, s2);
        cudaMemsetAsync(counts[0] + K, 0, sizeof(int), s2);
        cudaMemsetAsync(counts[1] + K, 0, sizeof(int), s2);
      }
      timed(ctx, MPG_KERNEL_BERNOULLI, s2, 1, [&] {
        launch_trial_init(K, sc->S, c, plan.w, oR, lists[0], base, counts[0], ctx->d_nbest, small_grid, s2);
      });
      int cur = 0;
      for (int t = 1; t <= T1; ++t) {
        int nxt = 1 - cur;
        cudaMemsetAsync(counts[nxt] + K, 0, sizeof(int), s2);
        DWork tw{lists[cur], base, counts[cur]};
        timed(ctx, MPG_KERNEL_BERNOULLI, s2, 1, [&] {
          launch_trial_seed(K, sc->S, guide ? &g : nullptr, c, tc, lists[cur], base, counts[cur], key, rng_offset, *P,
                            dcr, t, grid_of(ctx, P, 5, K, block, c.B, true), block, s2);
        });
        // trial walks run the walk kernel and are tallied with the walk family
        timed(ctx, MPG_KERNEL_WALK, s2, 1, [&] {
          launch_walk_p(K, ctx->stats_on, sc->S, tc, tw, *P, dcw, q + t,
                        grid_of(ctx, P, walk_which(P), K, walk_block(P), c.B, true), walk_block(P), s2);
        });
        timed(ctx, MPG_KERNEL_BERNOULLI, s2, 1, [&] {
          launch_trial_check(K, sc->S, c, tc, oR, lists[cur], base, counts[cur], t, t == T1, *P, lists[nxt], counts[nxt],
                             ctx->d_nbest, small_grid, s2);
        });
        cur = nxt;
      }
      long long TB = P->trial_batch > 0 ? P->trial_batch : 64;
      int t0 = T1 + 1;
      // 64-bit queue counter of the parallel rounds (two int slots, 8-byte aligned)
      int* q64 = q + 10;
      for (int r = 0; t0 <= P->max_trials; ++r) {
        TB = std::min<long long>(TB, (long long)P->max_trials - t0 + 1);  // the last round reaches the cap
        int t_end = t0 + (int)TB - 1;
        int nxt = 1 - cur;
        cudaMemsetAsync(counts[nxt] + K, 0, sizeof(int), s2);
        cudaMemsetAsync(ctx->d_npairs + K, 0, sizeof(int), s2);
        cudaMemsetAsync(q64, 0, sizeof(unsigned long long), s2);
        DPairs pr{ctx->d_pairs, ctx->d_npairs + K, plan.w.count ? plan.w.count + K : nullptr, c.B};
        timed(ctx, MPG_KERNEL_BERNOULLI, s2, 2, [&] {
          launch_bern_round(K, ctx->stats_on, sc->S, guide ? &g : nullptr, c, key, rng_offset, *P, dcr, q64,
                            lists[cur], counts[cur] + K, base + K, ctx->d_nbest, t0, (int)TB, pr,
                            grid_of(ctx, P, round_which(P), K, round_block(P), c.B, true), round_block(P), s2);
          launch_bern_finish(sc->S, c, oR, lists[cur], counts[cur] + K, base + K, ctx->d_nbest, t_end, P->max_trials,
                             lists[nxt], counts[nxt] + K, pr, dcb.stats, ctx->sms, s2);
        });
        t0 = t_end + 1;
        TB *= 4;
        cur = nxt;
      }
    }
  });
  if (s) return s;
  timed(ctx, MPG_KERNEL_AUX, st, 1, [&] { launch_irradiance(contrib, c.Q, c.spq, E, ctx->sms, st); });
  LAUNCH_CHECK("irradiance");
  return MPG_OK;
}

mpg_status mpg_guide_update(mpg_ctx* ctx, const mpg_guide* guide, const uint32_t* cell, const float* omega,
                            const float* w, int32_t R, const int32_t* R_dev, int32_t shift, cudaStream_t st) {
  if (!ctx) return fail(MPG_ERR_INVALID_ARG, "ctx is NULL");
  DGuide g;
  mpg_status s;
  if ((s = check_guide(guide, g))) return s;
  if (g.kind != MPG_GUIDE_HISTOGRAM)
    return fail(MPG_ERR_INVALID_ARG, "mpg_guide_update fills histogram guides; vMF guides are built by mpg_vmf_build");
  if (R < 0 || shift < 0 || shift > 60 || (R > 0 && (!aligned16(cell) || !aligned16(omega) || !aligned16(w))))
    return fail(MPG_ERR_INVALID_ARG, "invalid records (R %d, shift %d)", R, shift);
  CUDA_TRY(cudaSetDevice(ctx->device));
  timed(ctx, MPG_KERNEL_AUX, st, R > 0 ? 2 : 1,
        [&] { launch_guide_update(g, cell, omega, w, R, R_dev, shift, ctx->d_err, ctx->sms, st); });
  LAUNCH_CHECK("guide update");
  return MPG_OK;
}

mpg_status mpg_guide_clear(mpg_ctx* ctx, const mpg_guide* guide, cudaStream_t st) {
  if (!ctx) return fail(MPG_ERR_INVALID_ARG, "ctx is NULL");
  DGuide g;
  mpg_status s;
  if ((s = check_guide(guide, g))) return s;
  CUDA_TRY(cudaSetDevice(ctx->device));
  if (g.kind == MPG_GUIDE_VMF) {  // no lobes in any cell
    CUDA_TRY(cudaMemsetAsync(guide->cell_start, 0, sizeof(uint32_t) * ((size_t)guide->n_cells + 1), st));
    return MPG_OK;
  }
  const size_t bytes = sizeof(uint64_t) * (size_t)guide->n_cells * (size_t)guide->n_theta * (size_t)guide->n_phi;
  CUDA_TRY(cudaMemsetAsync(guide->counts, 0, bytes, st));
  CUDA_TRY(cudaMemsetAsync(guide->cdf, 0, bytes, st));
  return MPG_OK;
}

mpg_status mpg_guide_records(mpg_ctx* ctx, const mpg_scene* sc, const mpg_chains* chains, const float* contrib,
                             uint32_t* cell_out, float* omega_out, float* w_out, uint8_t* k_out, uint8_t* tau_out,
                             int32_t* chain_out, int32_t* R_dev, cudaStream_t st) {
  if (!ctx || !sc) return fail(MPG_ERR_INVALID_ARG, "ctx or scene is NULL");
  mpg_status s;
  if ((s = check_chains(chains, false))) return s;
  if (!aligned16(contrib) || !aligned16(cell_out) || !aligned16(omega_out) || !aligned16(w_out) || !R_dev ||
      (k_out && !aligned16(k_out)) || (tau_out && !aligned16(tau_out)) || (chain_out && !aligned16(chain_out)))
    return fail(MPG_ERR_INVALID_ARG, "record arrays must be non-NULL 16-byte aligned device arrays");
  CUDA_TRY(cudaSetDevice(ctx->device));
  DChains c = to_dev(chains);
  const int tiles = rec_tiles(c.B);
  if (ctx->rec_cap < tiles) {
    if (ctx->capturing) return capture_grow_error();
    if (ctx->d_rec) cudaFree(ctx->d_rec);
    ctx->d_rec = nullptr;
    CUDA_TRY(cudaMalloc(&ctx->d_rec, sizeof(uint32_t) * (size_t)tiles));
    ctx->rec_cap = tiles;
  }
  timed(ctx, MPG_KERNEL_AUX, st, tiles ? 3 : 0, [&] {
    launch_guide_records_ordered(c, contrib, 1.0f / sc->S.L.area, ctx->d_rec, cell_out, omega_out, w_out, k_out,
                                 tau_out, chain_out, R_dev, st);
  });
  LAUNCH_CHECK("guide records");
  return MPG_OK;
}

mpg_status mpg_vmf_build(mpg_ctx* ctx, const mpg_guide* guide, const uint32_t* cell, const float* omega,
                         const float* w, const uint8_t* k, const uint8_t* tau, int32_t R, const int32_t* R_dev,
                         int32_t weight_shift, cudaStream_t st) {
  if (!ctx) return fail(MPG_ERR_INVALID_ARG, "ctx is NULL");
  mpg_status s;
  DGuide g;
  if ((s = check_guide(guide, g))) return s;
  if (g.kind != MPG_GUIDE_VMF) return fail(MPG_ERR_INVALID_ARG, "mpg_vmf_build needs a guide of kind MPG_GUIDE_VMF");
  if (R < 0 || R > guide->capacity)
    return fail(MPG_ERR_INVALID_ARG, "record count %d outside [0, capacity %d]", R, guide->capacity);
  if (R > 0 && (!aligned16(cell) || !aligned16(omega) || !aligned16(w) || !aligned16(k) || !aligned16(tau)))
    return fail(MPG_ERR_INVALID_ARG, "record arrays must be non-NULL 16-byte aligned device arrays");
  if (weight_shift < 0 || weight_shift > 32) return fail(MPG_ERR_INVALID_ARG, "weight_shift %d outside [0, 32]", weight_shift);
  CUDA_TRY(cudaSetDevice(ctx->device));
  timed(ctx, MPG_KERNEL_AUX, st, vmf_build_launches(R, g.n_cells), [&] {
    launch_vmf_build(g, guide->scratch, cell, omega, w, k, tau, R, R_dev, weight_shift, ctx->d_err, ctx->sms, st);
  });
  LAUNCH_CHECK("vMF build");
  return MPG_OK;
}

mpg_status mpg_sample_lengths(mpg_ctx* ctx, const mpg_guide* guide, const mpg_chains* chains,
                              const uint32_t* p0_weights, uint64_t rng_seed, uint64_t rng_offset,
                              const mpg_params* P, uint8_t* k_out, float* pn_out, cudaStream_t st) {
  if (!ctx) return fail(MPG_ERR_INVALID_ARG, "ctx is NULL");
  if (!chains || chains->B < 0 || chains->Q < 0 || chains->spq <= 0 || (int64_t)chains->Q * chains->spq != chains->B)
    return fail(MPG_ERR_INVALID_ARG, "invalid chain batch sizes");
  if (chains->B == 0) return MPG_OK;
  mpg_status s;
  if ((s = check_params(P))) return s;
  if (!p0_weights) return fail(MPG_ERR_INVALID_ARG, "p0_weights is NULL");
  uint64_t W0 = 0;
  for (int n = 0; n < MAXK; ++n) W0 += p0_weights[n];
  if (W0 == 0) return fail(MPG_ERR_INVALID_ARG, "the P_0 weights sum to zero");
  if (!aligned16(k_out) || !aligned16(pn_out))
    return fail(MPG_ERR_INVALID_ARG, "k_out and pn_out must be non-NULL 16-byte aligned device arrays");
  DGuide g;
  if (guide) {
    if ((s = check_guide(guide, g))) return s;
    if (g.kind != MPG_GUIDE_VMF) return fail(MPG_ERR_INVALID_ARG, "sampled lengths need a vMF guide (or NULL)");
  }
  CUDA_TRY(cudaSetDevice(ctx->device));
  uint2 key = make_uint2((uint32_t)rng_seed, (uint32_t)(rng_seed >> 32));
  timed(ctx, MPG_KERNEL_SEED, st, 1, [&] {
    launch_sample_lengths(guide ? &g : nullptr, to_dev(chains), p0_weights, key, rng_offset, P->alpha,
                          dctx(ctx, MPG_KERNEL_SEED), k_out, pn_out, ctx->sms, st);
  });
  LAUNCH_CHECK("sample lengths");
  return MPG_OK;
}

mpg_status mpg_walk_adjoint(mpg_ctx* ctx, const mpg_scene* sc, const mpg_chains* chains, const float* T,
                            const float* contrib, const float* dL_dE, float* dL_dtheta, cudaStream_t st) {
  if (!ctx || !sc) return fail(MPG_ERR_INVALID_ARG, "ctx or scene is NULL");
  if (chains && chains->B == 0 && chains->Q == 0) return MPG_OK;
  mpg_status s;
  if ((s = check_chains(chains, false))) return s;
  if (!aligned16(T) || !aligned16(contrib) || !aligned16(dL_dE) || !aligned16(dL_dtheta))
    return fail(MPG_ERR_INVALID_ARG, "T, contrib, dL_dE and dL_dtheta must be non-NULL 16-byte aligned device arrays");
  if (sc->S.n_hf < 1) return fail(MPG_ERR_UNSUPPORTED, "the adjoint differentiates heightfield heights: no heightfield");
  CUDA_TRY(cudaSetDevice(ctx->device));
  DChains c = to_dev(chains);
  timed(ctx, MPG_KERNEL_AUX, st, 4, [&] {
    for (int K = 1; K <= 4; ++K)
      launch_adjoint(K, sc->S, c, T, contrib, dL_dE, dL_dtheta, ctx->d_err + 0, ctx->sms, st);
  });
  LAUNCH_CHECK("adjoint");
  return MPG_OK;
}

mpg_status mpg_trace_rays(mpg_ctx* ctx, const mpg_scene* sc, const float* o, const float* d, int32_t n, float tmin,
                          float tmax, float* t, int32_t* surf, int32_t* prim, float* bary, cudaStream_t st) {
  if (!ctx || !sc) return fail(MPG_ERR_INVALID_ARG, "ctx or scene is NULL");
  if (n < 0 || (n > 0 && (!aligned16(o) || !aligned16(d) || !aligned16(t) || !aligned16(surf) || !aligned16(prim) ||
                          !aligned16(bary))))
    return fail(MPG_ERR_INVALID_ARG, "invalid ray arrays");
  if (n == 0) return MPG_OK;
  CUDA_TRY(cudaSetDevice(ctx->device));
  timed(ctx, MPG_KERNEL_TRACE, st, 1, [&] {
    launch_trace(sc->S, o, d, n, tmin, tmax, t, surf, prim, bary, ctx->d_err, ctx->d_stats + 16 * MPG_KERNEL_TRACE,
                 ctx->stats_on, ctx->sms, st);
  });
  LAUNCH_CHECK("trace");
  return MPG_OK;
}

mpg_status mpg_fp32_peak(mpg_ctx* ctx, double* flops, cudaStream_t st) {
  if (!ctx || !flops) return fail(MPG_ERR_INVALID_ARG, "ctx or flops is NULL");
  CUDA_TRY(cudaSetDevice(ctx->device));
  *flops = run_fp32_peak(ctx->d_scratch, ctx->sms, st);
  LAUNCH_CHECK("fp32 peak");
  return MPG_OK;
}

mpg_status mpg_fp64_peak(mpg_ctx* ctx, double* flops, cudaStream_t st) {
  if (!ctx || !flops) return fail(MPG_ERR_INVALID_ARG, "ctx or flops is NULL");
  CUDA_TRY(cudaSetDevice(ctx->device));
  *flops = run_fp64_peak(ctx->d_scratch, ctx->sms, st);
  LAUNCH_CHECK("fp64 peak");
  return MPG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Captured steps (CUDA graphs).
// ---------------------------------------------------------------------------
struct mpg_graph {
  mpg_ctx* ctx = nullptr;
  int device = 0;  // kept apart from ctx: the context may be destroyed first
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned long long* counter = nullptr;
  int64_t kernels = 0;
};

extern "C" {

mpg_status mpg_graph_begin(mpg_ctx* ctx, cudaStream_t st, uint64_t rng_advance) {
  if (!ctx) return fail(MPG_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->capturing) return fail(MPG_ERR_INVALID_ARG, "a capture is already in progress on this context");
  if (st == 0 || st == cudaStreamLegacy || st == cudaStreamPerThread)
    return fail(MPG_ERR_INVALID_ARG, "capture needs a created (non-default) stream");
  CUDA_TRY(cudaSetDevice(ctx->device));
  unsigned long long* counter = nullptr;
  CUDA_TRY(cudaMalloc(&counter, sizeof(unsigned long long)));
  cudaError_t e = cudaMemset(counter, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaFree(counter);
    return fail(MPG_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
  }
  ctx->capturing = true;
  ctx->cap_rng = counter;
  ctx->profile_saved = ctx->profile;
  ctx->profile = false;
  ctx->cap_launch0 = ctx->launches;
  // the advance is recorded now and runs last: it is the final node on the
  // capture stream, after every recorded call has joined back onto it
  ctx->cap_advance = rng_advance;
  return MPG_OK;
}

mpg_status mpg_graph_join(mpg_ctx* ctx, mpg_ctx* other) {
  if (!ctx || !other) return fail(MPG_ERR_INVALID_ARG, "ctx or other is NULL");
  if (!ctx->capturing || !ctx->cap_rng) return fail(MPG_ERR_INVALID_ARG, "no capture begun on this context");
  if (other == ctx || other->capturing) return fail(MPG_ERR_INVALID_ARG, "the other context is already recording");
  if (other->device != ctx->device) return fail(MPG_ERR_INVALID_ARG, "contexts on different devices");
  other->capturing = true;
  other->cap_rng = ctx->cap_rng;
  other->profile_saved = other->profile;
  other->profile = false;
  other->cap_launch0 = other->launches;
  ctx->cap_joined.push_back(other);
  return MPG_OK;
}

mpg_status mpg_graph_end(mpg_ctx* ctx, cudaStream_t st, mpg_graph** out) {
  if (!ctx || !out) return fail(MPG_ERR_INVALID_ARG, "ctx or out is NULL");
  *out = nullptr;
  if (!ctx->capturing || !ctx->cap_rng) return fail(MPG_ERR_INVALID_ARG, "no capture begun on this context");
  CUDA_TRY(cudaSetDevice(ctx->device));
  launch_rng_advance(ctx->cap_rng, ctx->cap_advance, st);
  cudaError_t le = cudaGetLastError();
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &graph);
  mpg_graph* g = new mpg_graph();
  g->ctx = ctx;
  g->device = ctx->device;
  g->counter = ctx->cap_rng;
  g->kernels = ctx->launches - ctx->cap_launch0 + 1;
  ctx->launches = ctx->cap_launch0;
  for (mpg_ctx* o : ctx->cap_joined) {  // their recorded launches replay with this graph
    g->kernels += o->launches - o->cap_launch0;
    o->launches = o->cap_launch0;
    o->capturing = false;
    o->cap_rng = nullptr;
    o->profile = o->profile_saved;
  }
  ctx->cap_joined.clear();
  ctx->capturing = false;
  ctx->cap_rng = nullptr;
  ctx->profile = ctx->profile_saved;
  if (le == cudaSuccess && e == cudaSuccess && graph) {
    g->graph = graph;
    e = cudaGraphInstantiate(&g->exec, graph, 0);
  } else if (e == cudaSuccess) {
    e = le != cudaSuccess ? le : cudaErrorStreamCaptureInvalidated;
  }
  if (e != cudaSuccess || !g->exec) {
    if (graph) cudaGraphDestroy(graph);
    g->graph = nullptr;
    cudaFree(g->counter);
    delete g;
    return fail(MPG_ERR_CUDA, "capture failed: %s", cudaGetErrorString(e));
  }
  *out = g;
  return MPG_OK;
}

mpg_status mpg_graph_launch(mpg_graph* g, cudaStream_t st) {
  if (!g || !g->exec) return fail(MPG_ERR_INVALID_ARG, "graph is NULL");
  CUDA_TRY(cudaSetDevice(g->device));
  CUDA_TRY(cudaGraphLaunch(g->exec, st));
  g->ctx->launches += g->kernels;
  return MPG_OK;
}

mpg_status mpg_graph_kernels(const mpg_graph* g, int64_t* count) {
  if (!g || !count) return fail(MPG_ERR_INVALID_ARG, "graph or count is NULL");
  *count = g->kernels;
  return MPG_OK;
}

void mpg_graph_destroy(mpg_graph* g) {
  if (!g) return;
  cudaSetDevice(g->device);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  cudaFree(g->counter);
  delete g;
  (void)cudaGetLastError();  // a failure here must not surface in a later call's launch check
}

// ---------------------------------------------------------------------------
// Autotuner of the batched schedule.
// ---------------------------------------------------------------------------
struct mpg_stree {
  int device = 0;
  StreeHost h;
  int* d_axis = nullptr;
  int* d_left = nullptr;
  int* d_right = nullptr;
  int* d_member_leaf = nullptr;
  int* d_member_rec = nullptr;
  double* d_split = nullptr;
};

void mpg_stree_destroy(mpg_stree* t) {
  if (!t) return;
  if (t->device < 0) {  // host-only tree
    delete t;
    return;
  }
  cudaSetDevice(t->device);
  cudaFree(t->d_axis); cudaFree(t->d_left); cudaFree(t->d_right); cudaFree(t->d_split);
  cudaFree(t->d_member_leaf); cudaFree(t->d_member_rec);
  delete t;
  (void)cudaGetLastError();  // a failure here must not surface in a later call's launch check
}

mpg_status mpg_stree_build(mpg_ctx* ctx, const mpg_chains* chains, const int32_t* rec_chain, int32_t R,
                           const int32_t* R_dev, float epsilon, float c, int32_t method, mpg_stree** out,
                           cudaStream_t st) {
  if (!ctx || !out) return fail(MPG_ERR_INVALID_ARG, "ctx or out is NULL");
  *out = nullptr;
  mpg_status s;
  if ((s = check_chains(chains, false))) return s;
  if (R < 0 || (R > 0 && !aligned16(rec_chain)) || !(epsilon >= 0.0f && epsilon < 0.5f) || !(c > 0.0f) ||
      (method != MPG_STREE_RECURSIVE && method != MPG_STREE_LEVELS))
    return fail(MPG_ERR_INVALID_ARG, "invalid tree arguments (R %d, epsilon %g, c %g, method %d)", R, epsilon, c,
                method);
  if (ctx->capturing) return fail(MPG_ERR_INVALID_ARG, "mpg_stree_build is synchronous and cannot be captured");
  CUDA_TRY(cudaSetDevice(ctx->device));
  int n = R;
  if (R_dev) {
    CUDA_TRY(cudaMemcpyAsync(&n, R_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    n = std::min(std::max(n, 0), R);
  }
  std::vector<int> idx(n);
  if (n > 0) {
    CUDA_TRY(cudaMemcpyAsync(idx.data(), rec_chain, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
  }
  for (int i = 0; i < n; ++i)
    if (idx[i] < 0 || idx[i] >= chains->B)
      return fail(MPG_ERR_INVALID_ARG, "record %d names chain %d outside the batch", i, idx[i]);
  mpg_stree* t = new mpg_stree;
  t->device = ctx->device;
  float* d_pos = nullptr;
  if (n > 0) {
    cudaError_t e = cudaMalloc(&d_pos, sizeof(float) * (size_t)6 * n);
    if (e != cudaSuccess) {
      delete t;
      return fail(MPG_ERR_CUDA, "tree positions: %s", cudaGetErrorString(e));
    }
    launch_stree_gather(to_dev(chains), rec_chain, n, d_pos, st);
    ctx->launches += 1;
  }
  if (method == MPG_STREE_LEVELS) {
    // level by level on the device, from the gathered positions
    const char* why = nullptr;
    const bool ok = stree_build_levels_device(d_pos, n, (double)epsilon, (double)c, t->h, st, &why);
    if (d_pos) cudaFree(d_pos);
    if (!ok) {
      delete t;
      return fail(MPG_ERR_CUDA, "device tree build: %s", why);
    }
  } else {
    std::vector<float> pos((size_t)6 * n);
    if (n > 0) {
      cudaError_t e = cudaMemcpyAsync(pos.data(), d_pos, sizeof(float) * pos.size(), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      cudaFree(d_pos);
      if (e != cudaSuccess) {
        delete t;
        return fail(MPG_ERR_CUDA, "tree positions: %s", cudaGetErrorString(e));
      }
    }
    stree_build(pos.data(), n, (double)epsilon, (double)c, t->h);
  }
  auto upload = [](auto** d, const auto& h) {
    const size_t bytes = sizeof(h[0]) * h.size();
    cudaError_t e = cudaMalloc((void**)d, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess && bytes) e = cudaMemcpy(*d, h.data(), bytes, cudaMemcpyHostToDevice);
    return e;
  };
  cudaError_t e = upload(&t->d_axis, t->h.axis);
  if (e == cudaSuccess) e = upload(&t->d_left, t->h.left);
  if (e == cudaSuccess) e = upload(&t->d_right, t->h.right);
  if (e == cudaSuccess) e = upload(&t->d_split, t->h.split);
  if (e == cudaSuccess) e = upload(&t->d_member_leaf, t->h.member_leaf);
  if (e == cudaSuccess) e = upload(&t->d_member_rec, t->h.member_rec);
  if (e != cudaSuccess) {
    mpg_stree_destroy(t);
    return fail(MPG_ERR_CUDA, "tree upload: %s", cudaGetErrorString(e));
  }
  *out = t;
  return MPG_OK;
}

mpg_status mpg_stree_build_host(const float* pos, int32_t n, float epsilon, float c, int32_t method,
                                mpg_stree** out) {
  if (!out) return fail(MPG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n < 0 || (n > 0 && !pos) || !(epsilon >= 0.0f && epsilon < 0.5f) || !(c > 0.0f) ||
      (method != MPG_STREE_RECURSIVE && method != MPG_STREE_LEVELS))
    return fail(MPG_ERR_INVALID_ARG, "invalid tree arguments (n %d, epsilon %g, c %g, method %d)", n, epsilon, c,
                method);
  for (size_t i = 0; i < (size_t)6 * n; ++i)
    if (!std::isfinite(pos[i])) return fail(MPG_ERR_INVALID_ARG, "position %zu is not finite", i);
  mpg_stree* t = new mpg_stree;
  t->device = -1;
  if (method == MPG_STREE_LEVELS) stree_build_levels_host(pos, n, (double)epsilon, (double)c, t->h);
  else stree_build(pos, n, (double)epsilon, (double)c, t->h);
  *out = t;
  return MPG_OK;
}

mpg_status mpg_stree_info(const mpg_stree* t, int32_t* n_samples, int32_t* n_nodes, int32_t* n_leaves,
                          int32_t* n_members) {
  if (!t) return fail(MPG_ERR_INVALID_ARG, "tree is NULL");
  if (n_samples) *n_samples = t->h.n_samples;
  if (n_nodes) *n_nodes = (int32_t)t->h.axis.size();
  if (n_leaves) *n_leaves = t->h.n_leaves;
  if (n_members) *n_members = (int32_t)t->h.member_rec.size();
  return MPG_OK;
}

mpg_status mpg_stree_export(const mpg_stree* t, int32_t* axis, double* split, int32_t* left, int32_t* right,
                            int32_t* member_leaf, int32_t* member_rec) {
  if (!t) return fail(MPG_ERR_INVALID_ARG, "tree is NULL");
  if (axis) std::copy(t->h.axis.begin(), t->h.axis.end(), axis);
  if (split) std::copy(t->h.split.begin(), t->h.split.end(), split);
  if (left) std::copy(t->h.left.begin(), t->h.left.end(), left);
  if (right) std::copy(t->h.right.begin(), t->h.right.end(), right);
  if (member_leaf) std::copy(t->h.member_leaf.begin(), t->h.member_leaf.end(), member_leaf);
  if (member_rec) std::copy(t->h.member_rec.begin(), t->h.member_rec.end(), member_rec);
  return MPG_OK;
}

mpg_status mpg_stree_records(mpg_ctx* ctx, const mpg_stree* t, const float* omega, const float* w, const uint8_t* k,
                             const uint8_t* tau, int32_t R_in, uint32_t* cell_out, float* omega_out, float* w_out,
                             uint8_t* k_out, uint8_t* tau_out, int32_t R_out, int32_t* R_out_dev, cudaStream_t st) {
  if (t && t->device < 0) return fail(MPG_ERR_INVALID_ARG, "the tree has no device copy (built from host positions)");
  if (!ctx || !t) return fail(MPG_ERR_INVALID_ARG, "ctx or tree is NULL");
  const int M = (int)t->h.member_rec.size();
  if (R_out < M || R_in < t->h.n_samples)
    return fail(MPG_ERR_INVALID_ARG, "record arrays too small (R_in %d < %d samples or R_out %d < %d members)", R_in,
                t->h.n_samples, R_out, M);
  if (!R_out_dev || (M > 0 && (!aligned16(omega) || !aligned16(w) || !aligned16(k) || !aligned16(tau) ||
                               !aligned16(cell_out) || !aligned16(omega_out) || !aligned16(w_out) ||
                               !aligned16(k_out) || !aligned16(tau_out))))
    return fail(MPG_ERR_INVALID_ARG, "record arrays must be non-NULL 16-byte aligned device arrays");
  CUDA_TRY(cudaSetDevice(ctx->device));
  timed(ctx, MPG_KERNEL_AUX, st, 1, [&] {
    launch_stree_records(t->d_member_leaf, t->d_member_rec, M, omega, w, k, tau, R_in, cell_out, omega_out, w_out,
                         k_out, tau_out, R_out, R_out_dev, ctx->sms, st);
  });
  LAUNCH_CHECK("tree records");
  return MPG_OK;
}

mpg_status mpg_stree_query(mpg_ctx* ctx, const mpg_stree* t, const mpg_chains* chains, uint32_t* chain_cell,
                           cudaStream_t st) {
  if (t && t->device < 0) return fail(MPG_ERR_INVALID_ARG, "the tree has no device copy (built from host positions)");
  if (!ctx || !t) return fail(MPG_ERR_INVALID_ARG, "ctx or tree is NULL");
  mpg_status s;
  if ((s = check_chains(chains, false))) return s;
  if (!aligned16(chain_cell)) return fail(MPG_ERR_INVALID_ARG, "chain_cell must be a 16-byte aligned device array");
  if (chains->B == 0) return MPG_OK;
  CUDA_TRY(cudaSetDevice(ctx->device));
  timed(ctx, MPG_KERNEL_AUX, st, 1, [&] {
    launch_stree_query(t->d_axis, t->d_split, t->d_left, t->d_right, to_dev(chains), chain_cell, ctx->sms, st);
  });
  LAUNCH_CHECK("tree query");
  return MPG_OK;
}

mpg_status mpg_separator_bsdf(mpg_ctx* ctx, const mpg_chains* chains, const float* contrib, const float* camera,
                              float exponent, float* radiance, float* L, cudaStream_t st) {
  if (!ctx || !camera) return fail(MPG_ERR_INVALID_ARG, "ctx or camera is NULL");
  mpg_status s;
  if ((s = check_chains(chains, false))) return s;
  if (!(exponent > 0.0f) || !aligned16(contrib) || !aligned16(radiance) || !aligned16(L))
    return fail(MPG_ERR_INVALID_ARG, "invalid separator BSDF arguments (exponent %g, arrays)", exponent);
  CUDA_TRY(cudaSetDevice(ctx->device));
  DChains c = to_dev(chains);
  timed(ctx, MPG_KERNEL_AUX, st, 2, [&] {
    launch_separator_bsdf(c, contrib, make_float3(camera[0], camera[1], camera[2]), exponent, radiance, ctx->sms, st);
    launch_irradiance(radiance, c.Q, c.spq, L, ctx->sms, st);
  });
  LAUNCH_CHECK("separator BSDF");
  return MPG_OK;
}

mpg_status mpg_records_bsdf(mpg_ctx* ctx, const mpg_chains* chains, const int32_t* rec_chain, const float* omega,
                            float* w, int32_t R, const int32_t* R_dev, const float* camera, float exponent,
                            cudaStream_t st) {
  if (!ctx || !camera) return fail(MPG_ERR_INVALID_ARG, "ctx or camera is NULL");
  mpg_status s;
  if ((s = check_chains(chains, false))) return s;
  if (R < 0 || !(exponent > 0.0f) || (R > 0 && (!aligned16(rec_chain) || !aligned16(omega) || !aligned16(w))))
    return fail(MPG_ERR_INVALID_ARG, "invalid record arguments (R %d, exponent %g)", R, exponent);
  if (R == 0) return MPG_OK;
  CUDA_TRY(cudaSetDevice(ctx->device));
  timed(ctx, MPG_KERNEL_AUX, st, 1, [&] {
    launch_records_bsdf(to_dev(chains), rec_chain, omega, w, R, R_dev, make_float3(camera[0], camera[1], camera[2]),
                        exponent, ctx->sms, st);
  });
  LAUNCH_CHECK("record BSDF weights");
  return MPG_OK;
}

mpg_status mpg_training_plan(int32_t total_spp, int32_t first_spp, float train_fraction, int32_t max_iters,
                             int32_t* iter_spp, int32_t* n_iters, int32_t* render_spp) {
  if (total_spp < 0 || first_spp < 1 || !(train_fraction >= 0.0f && train_fraction <= 1.0f) || max_iters < 0 ||
      !n_iters || !render_spp || (max_iters > 0 && !iter_spp))
    return fail(MPG_ERR_INVALID_ARG, "invalid training plan arguments");
  const int64_t budget = (int64_t)std::floor((double)train_fraction * (double)total_spp);
  int64_t used = 0, next = first_spp;
  int n = 0;
  while (used < budget) {
    if (n == max_iters) return fail(MPG_ERR_LIMIT, "training plan needs more than %d iterations", max_iters);
    const int64_t cur = std::min(next, budget - used);  // cut at the training budget
    iter_spp[n++] = (int32_t)cur;
    used += cur;
    if (used >= budget) break;
    if (2 * used < budget) {  // less than half of the training budget used: a new iteration
      next *= 2;
    } else {  // otherwise the current iteration continues until the budget is spent
      iter_spp[n - 1] += (int32_t)(budget - used);
      used = budget;
    }
  }
  *n_iters = n;
  *render_spp = (int32_t)(total_spp - used);
  return MPG_OK;
}

mpg_status mpg_autotune(mpg_ctx* ctx, const mpg_scene* sc, const mpg_guide* guide, mpg_chains* chains,
                        uint64_t rng_seed, uint64_t rng_offset, const mpg_params* in, int32_t repeats,
                        mpg_params* out, double* best_ms, cudaStream_t st) {
  if (!ctx || !sc || !in || !out || !chains) return fail(MPG_ERR_INVALID_ARG, "NULL argument");
  mpg_status s;
  if ((s = check_chains(chains, true)) || (s = check_params(in))) return s;
  if (in->walk_mode != MPG_WALK_BATCHED) return fail(MPG_ERR_INVALID_ARG, "the autotuner tunes the batched mode");
  if (ctx->capturing) return fail(MPG_ERR_INVALID_ARG, "cannot tune during a capture");
  if (repeats < 1 || repeats > 16) return fail(MPG_ERR_INVALID_ARG, "repeats %d out of 1..16", repeats);
  CUDA_TRY(cudaSetDevice(ctx->device));
  const size_t B = (size_t)chains->B, Q = (size_t)chains->Q;
  auto up = [](size_t n) { return (n + 255) & ~(size_t)255; };
  const size_t oG = 0, oK = oG + up(4 * B), oT = oK + up(4 * B), oN = oT + up(4 * B), oC = oN + up(4 * B),
               oW = oC + up(B), oE = oW + up(4 * B), total = oE + up(4 * Q);
  char* scratch = nullptr;
  CUDA_TRY(cudaMalloc(&scratch, total));
  // the tuner's own work is kept out of the caller's counters and timings
  unsigned long long saved[16 * MPG_KERNEL_KINDS];
  cudaError_t e = cudaMemcpy(saved, ctx->d_stats, sizeof(saved), cudaMemcpyDeviceToHost);
  const bool prof = ctx->profile;
  const int64_t launches = ctx->launches;
  ctx->profile = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  auto time_one = [&](const mpg_params& P, double& ms) -> mpg_status {
    ms = 1e300;
    for (int r = 0; r <= repeats; ++r) {  // the first run is a warm-up
      mpg_status rs;
      CUDA_TRY(cudaEventRecord(e0, st));
      if ((rs = mpg_sample_seeds(ctx, sc, guide, chains, rng_seed, rng_offset, &P, st)) ||
          (rs = mpg_manifold_walk(ctx, sc, chains, &P, st)) ||
          (rs = mpg_chain_contribution(ctx, sc, guide, chains, rng_seed, rng_offset, &P, (float*)(scratch + oG),
                                       (float*)(scratch + oK), (float*)(scratch + oT), (uint32_t*)(scratch + oN),
                                       (uint8_t*)(scratch + oC), (float*)(scratch + oW), (float*)(scratch + oE), st)))
        return rs;
      CUDA_TRY(cudaEventRecord(e1, st));
      CUDA_TRY(cudaEventSynchronize(e1));
      float t = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
      if (r > 0) ms = std::min(ms, (double)t);
    }
    return MPG_OK;
  };
  mpg_params best = *in;
  double bms = 0.0;
  if (e == cudaSuccess) s = time_one(best, bms);
  // Coordinate descent, one group of schedule fields at a time; a candidate
  // replaces the best one only when it is faster by more than the timing
  // noise of one step (3 %).
  auto group = [&](const std::vector<mpg_params>& cands) -> mpg_status {
    for (const mpg_params& P : cands) {
      double ms;
      mpg_status rs = time_one(P, ms);
      if (rs) return rs;
      if (ms < 0.97 * bms) { bms = ms; best = P; }
    }
    return MPG_OK;
  };
  if (e == cudaSuccess && !s) {  // tile shape: threads per CTA x resident CTAs per SM
    std::vector<mpg_params> c;
    const int cur_block = best.block_threads ? best.block_threads : 128;
    for (int block : {32, 64, 128}) {
      // resident CTAs: the occupancy maximum (0) or half of it, from the k = 2 walk kernel
      int occ = blocks_per_sm(4, 2, ctx->stats_on, block);
      for (int ctas : {0, occ / 2}) {
        if (ctas != 0 && (ctas < 1 || ctas >= occ)) continue;
        if (block == cur_block && ctas == best.ctas_per_sm) continue;  // the starting point
        mpg_params P = best;
        P.block_threads = block;
        P.ctas_per_sm = ctas;
        c.push_back(P);
      }
    }
    s = group(c);
  }
  if (e == cudaSuccess && !s) {  // walk form: one thread or one lane group per chain, in walks / rounds
    std::vector<mpg_params> c;
    for (int wg = 0; wg < 4; ++wg) {
      if (wg == best.walk_group) continue;
      mpg_params P = best;
      P.walk_group = wg;
      c.push_back(P);
    }
    s = group(c);
  }
  if (e == cudaSuccess && !s) {  // refill cadence of the persistent kernels
    std::vector<mpg_params> c;
    for (int r : {1, 2, 4, 8}) {
      if (r == std::max(1, best.refill_every)) continue;
      mpg_params P = best;
      P.refill_every = r;
      c.push_back(P);
    }
    s = group(c);
  }
  if (e == cudaSuccess && !s) {  // Bernoulli rounds: synchronous rounds x first parallel batch
    std::vector<mpg_params> c;
    for (int t1 : {1, 2, 3})
      for (int tb : {4, 16, 64, 256}) {
        if (t1 == sync_rounds_of(&best) && tb == (best.trial_batch ? best.trial_batch : 64)) continue;
        mpg_params P = best;
        P.trial_sync_rounds = t1;
        P.trial_batch = tb;
        c.push_back(P);
      }
    s = group(c);
  }
  if (e == cudaSuccess && !s) {  // FP32/FP64 split: only toward more FP64
    std::vector<mpg_params> c;
    for (int k : {5, 4}) {
      if (k >= fp64_k_of(best)) continue;
      mpg_params P = best;
      P.fp64_k = k;
      c.push_back(P);
    }
    s = group(c);
  }
  if (e == cudaSuccess && !s) {
    // confirm against the starting schedule with three more timings of each,
    // taken alternately: the descent's single timings can pick a schedule on
    // noise, and the tuned schedule must not be slower than the one given
    double tb = 1e300, ti = 1e300;
    for (int r = 0; r < 3 && !s; ++r) {
      double m;
      if (!(s = time_one(best, m))) tb = std::min(tb, m);
      if (!s && !(s = time_one(*in, m))) ti = std::min(ti, m);
    }
    if (!s && ti < tb) { best = *in; bms = ti; }
    else if (!s) bms = tb;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaError_t e2 = cudaStreamSynchronize(st);
  if (e2 == cudaSuccess) e2 = cudaMemcpy(ctx->d_stats, saved, sizeof(saved), cudaMemcpyHostToDevice);
  cudaFree(scratch);
  ctx->profile = prof;
  ctx->launches = launches;
  if (e != cudaSuccess) return fail(MPG_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
  if (s) return s;
  if (e2 != cudaSuccess) return fail(MPG_ERR_CUDA, "autotune: %s", cudaGetErrorString(e2));
  *out = best;
  if (best_ms) *best_ms = bms;
  return MPG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free manifold walk.  Its scratch (work-queue counters, length
// buckets and the bucketed chain order) is a file-scope device array instead
// of context memory, so a call needs no device allocation at all.
// ---------------------------------------------------------------------------
namespace {

constexpr int NOALLOC_MAX_CHAINS = 1 << 20;

struct NoAllocScratch {
  int queue[16 * (MAXK + 1)];
  int count[MAXK + 1];
  int base[MAXK + 1];
  int cursor[MAXK + 1];
  int err;
  int order[NOALLOC_MAX_CHAINS];
};

// Held by every GPU that loads the library, for the life of the process.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
NoAllocScratch* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch on the current device.  In host code the
// array's name only stands for it, so it is looked up once per device with
// cudaGetSymbolAddress (with that device current) and cached.
mpg_status noalloc_scratch(int device, NoAllocScratch** out) {
  if (device < 0 || device >= NOALLOC_MAX_DEVICES) return fail(MPG_ERR_UNSUPPORTED, "device %d out of range", device);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(MPG_ERR_CUDA, "cudaGetSymbolAddress of the walk scratch: %s", cudaGetErrorString(e));
    g_noalloc_addr[device] = (NoAllocScratch*)p;
  }
  *out = g_noalloc_addr[device];
  return MPG_OK;
}

}  // namespace

extern "C" mpg_status mpg_manifold_walk_noalloc(const mpg_scene* sc, mpg_chains* chains, const mpg_params* P,
                                                cudaStream_t st) {
  if (!sc) return fail(MPG_ERR_INVALID_ARG, "scene is NULL");
  if (chains && chains->B == 0 && chains->Q == 0) return MPG_OK;
  mpg_status s;
  if ((s = check_chains(chains, false)) || (s = check_params(P))) return s;
  if (chains->offset)
    return fail(MPG_ERR_UNSUPPORTED, "mpg_manifold_walk_noalloc walks specular chains only (chains.offset is set)");
  if (chains->B > NOALLOC_MAX_CHAINS)
    return fail(MPG_ERR_INVALID_ARG, "mpg_manifold_walk_noalloc takes at most %d chains per call (got %d)",
                NOALLOC_MAX_CHAINS, chains->B);
  int device = -1;
  CUDA_TRY(cudaGetDevice(&device));
  if (device != sc->device) return fail(MPG_ERR_INVALID_ARG, "the scene lives on device %d, current is %d", sc->device, device);
  NoAllocScratch* scr = nullptr;
  if ((s = noalloc_scratch(device, &scr))) return s;
  int sms = 1;
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  // what must start at zero: the queue counters, the bucket sizes and the
  // device error word (a previous call's flag must not leak into this one)
  CUDA_TRY(cudaMemsetAsync(scr->queue, 0, sizeof(scr->queue), st));
  CUDA_TRY(cudaMemsetAsync(&scr->err, 0, sizeof(int), st));
  DChains c = to_dev(chains);
  DWork w{nullptr, nullptr, nullptr};
  int k_lo = 1, k_hi = MAXK;
  if (P->k_uniform >= 1) {
    k_lo = k_hi = P->k_uniform;
  } else {
    CUDA_TRY(launch_bucket(c.k, c.status, ST_SEEDED, c.B, scr->count, scr->base, scr->cursor, scr->order, sms, st));
    w = DWork{scr->order, scr->base, scr->count};
  }
  DCtx dc{&scr->err, nullptr};
  // the schedule of mpg_manifold_walk's batched mode: the walk form the
  // caller picked (one thread or one lane group per chain), its block size
  // and resident CTAs per SM, clamped by ctas_per_sm
  const int which = walk_which(P), block = walk_block(P);
  for (int K = k_lo; K <= k_hi; ++K) {
    int per_sm = blocks_per_sm(which, K, false, block);
    if (P->ctas_per_sm > 0) per_sm = std::min(per_sm, P->ctas_per_sm);
    int grid = std::max(1, std::min(sms * per_sm, (c.B + block - 1) / block));
    launch_walk_p(K, false, sc->S, c, w, *P, dc, scr->queue + 16 * K, grid, block, st);
  }
  LAUNCH_CHECK("walk (no-alloc)");
  // Device-side failures (a BVH traversal stack overflow) are read back here:
  // the call waits for `stream` and reports them like mpg_ctx_sync.
  int err = 0;
  CUDA_TRY(cudaMemcpyAsync(&err, &scr->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (err & ERR_BVH_STACK) return fail(MPG_ERR_LIMIT, "BVH traversal stack overflow (device flag %d)", err);
  if (err) return fail(MPG_ERR_INVALID_ARG, "device-side argument error (flag %d)", err);
  return MPG_OK;
}
