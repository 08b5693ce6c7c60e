// Spatial tree of the guide samples (Sec. 5.6): the host build of the binary
// tree over the samples' (x_D, x_L), and the device kernels around it --
// gathering the samples' positions, turning the leaves' members into guide
// records, and the per-chain leaf query.  The tree is built on the host once
// per training pass (the paper's tree is a host structure too); the queries
// run on the GPU for every chain.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <future>

#include "mpg_aux.cuh"
#include "mpg_stree_level.cuh"

namespace mpg {

namespace {
constexpr int STREE_MAX_DEPTH = 48;
constexpr int STREE_PAR_DEPTH = 4;  // subtrees below this depth are built on threads of their own

// What every part of one build shares: the samples and the index array whose
// disjoint ranges the parts partition in place.
struct Shared {
  const float* pos;  // [6][n]
  int n;
  double eps;
  int T;
  double root_ext[6];
  std::vector<int> idx;     // sample indices; a node owns a contiguous range
  std::vector<float> X[6];  // the samples' coordinates, permuted with idx
};

// Appends part `p` (nodes, leaves and members numbered from 0) to `t`;
// returns the index its root node gets.
int splice(StreeHost& t, const StreeHost& p) {
  const int off = (int)t.axis.size(), leaf0 = t.n_leaves;
  for (size_t j = 0; j < p.axis.size(); ++j) {
    const bool leaf = p.axis[j] < 0;
    t.axis.push_back(p.axis[j]);
    t.split.push_back(p.split[j]);
    t.left.push_back(leaf ? p.left[j] + leaf0 : p.left[j] + off);
    t.right.push_back(leaf ? -1 : p.right[j] + off);
  }
  for (size_t m = 0; m < p.member_rec.size(); ++m) {
    t.member_leaf.push_back(p.member_leaf[m] + leaf0);
    t.member_rec.push_back(p.member_rec[m]);
  }
  t.n_leaves += p.n_leaves;
  return off;
}

struct Builder {
  Shared& sh;
  StreeHost& t;
  std::vector<double> dist;  // selection scratch
  const std::vector<float>* X;
  std::vector<int>& idx;
  const double eps;
  const int T;
  const double* root_ext;

  Builder(Shared& s, StreeHost& out) : sh(s), t(out), X(s.X), idx(s.idx), eps(s.eps), T(s.T), root_ext(s.root_ext) {}

  int node() {
    t.axis.push_back(-1);
    t.split.push_back(0.0);
    t.left.push_back(-1);
    t.right.push_back(-1);
    return (int)t.axis.size() - 1;
  }

  // The m samples of idx[b, e) nearest to the plane x = mid (ties: lower
  // index), as a set: the m-th smallest distance by linear-time selection,
  // then every sample below it and, at it, the lowest indices.
  std::vector<int> nearest(size_t b, size_t e, int a, double mid, size_t m) {
    m = std::min(m, e - b);
    if (m == 0) return {};
    const float* x = X[a].data();
    dist.resize(e - b);
    for (size_t j = b; j < e; ++j) dist[j - b] = std::fabs((double)x[j] - mid);
    std::nth_element(dist.begin(), dist.begin() + (m - 1), dist.end());
    const double thr = dist[m - 1];
    std::vector<int> out, tie;
    out.reserve(m);
    for (size_t j = b; j < e; ++j) {
      const double d = std::fabs((double)x[j] - mid);
      if (d < thr) out.push_back(idx[j]);
      else if (d == thr) tie.push_back(idx[j]);
    }
    std::sort(tie.begin(), tie.end());
    for (size_t j = 0; out.size() < m; ++j) out.push_back(tie[j]);
    return out;
  }

  // Node over the own samples idx[b, e) and the copies it received.
  int build(size_t b, size_t e, const std::vector<int>& copies, const double* lo, const double* hi, int depth) {
    const int i = node();
    int a = 0;
    double best = -1.0;
    for (int ax = 0; ax < 6; ++ax) {  // largest extent relative to the root box, first on ties
      double rel = root_ext[ax] > 0.0 ? (hi[ax] - lo[ax]) / root_ext[ax] : 0.0;
      if (rel > best) { best = rel; a = ax; }
    }
    const size_t k = e - b;
    if ((int)k <= T || depth >= STREE_MAX_DEPTH || !(best > 0.0)) {
      const int leaf = t.n_leaves++;
      t.left[i] = leaf;
      std::vector<int> mem(idx.begin() + b, idx.begin() + e);
      mem.insert(mem.end(), copies.begin(), copies.end());
      std::sort(mem.begin(), mem.end());
      mem.erase(std::unique(mem.begin(), mem.end()), mem.end());
      for (int r : mem) {
        t.member_leaf.push_back(leaf);
        t.member_rec.push_back(r);
      }
      return i;
    }
    const double mid = 0.5 * (lo[a] + hi[a]);
    // in-place partition without branches, coordinates moved along: [b, j)
    // below the plane, [j, e) not
    size_t j = b;
    std::vector<float>* Xs = sh.X;
    const float* xa = Xs[a].data();
    for (size_t p = b; p < e; ++p) {
      const bool left = (double)xa[p] < mid;
      std::swap(idx[p], idx[j]);
      for (int c = 0; c < 6; ++c) std::swap(Xs[c][p], Xs[c][j]);
      j += left;
    }
    const size_t m = (size_t)std::floor(eps * (double)k);
    std::vector<int> to_right = nearest(b, j, a, mid, m), to_left = nearest(j, e, a, mid, m);
    t.axis[i] = a;
    t.split[i] = mid;
    double hl[6], lr[6];
    std::copy(hi, hi + 6, hl);
    std::copy(lo, lo + 6, lr);
    hl[a] = mid;
    lr[a] = mid;
    if (depth < STREE_PAR_DEPTH && k > 4096) {
      // the two subtrees on two threads, each into a part of its own, then
      // appended in the order the sequential build numbers them
      StreeHost pl, pr;
      auto left = std::async(std::launch::async, [&] { Builder(sh, pl).build(b, j, to_left, lo, hl, depth + 1); });
      Builder(sh, pr).build(j, e, to_right, lr, hi, depth + 1);
      left.get();
      const int l = splice(t, pl);
      t.left[i] = l;
      const int r = splice(t, pr);
      t.right[i] = r;
      return i;
    }
    const int l = build(b, j, to_left, lo, hl, depth + 1);
    t.left[i] = l;
    const int r = build(j, e, to_right, lr, hi, depth + 1);
    t.right[i] = r;
    return i;
  }
};

__global__ void k_stree_gather(DChains c, const int* rec_chain, int n, float* pos) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int b = rec_chain[i];
    const int q = b / c.spq;
    pos[i] = c.xD[q];
    pos[(size_t)n + i] = c.xD[c.Q + q];
    pos[2 * (size_t)n + i] = c.xD[2 * c.Q + q];
    pos[3 * (size_t)n + i] = c.xL[b];
    pos[4 * (size_t)n + i] = c.xL[(size_t)c.B + b];
    pos[5 * (size_t)n + i] = c.xL[2 * (size_t)c.B + b];
  }
}

__global__ void k_stree_records(const int* member_leaf, const int* member_rec, int M, const float* omega,
                                const float* w, const uint8_t* k, const uint8_t* tau, int R_in, uint32_t* cell_out,
                                float* omega_out, float* w_out, uint8_t* k_out, uint8_t* tau_out, int R_out,
                                int* R_out_dev) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *R_out_dev = M;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
    const int r = member_rec[m];
    cell_out[m] = (uint32_t)member_leaf[m];
    omega_out[m] = omega[r];
    omega_out[R_out + m] = omega[R_in + r];
    omega_out[2 * (size_t)R_out + m] = omega[2 * (size_t)R_in + r];
    w_out[m] = w[r];
    k_out[m] = k[r];
    tau_out[m] = tau[r];
  }
}

// Descend from the root by (x_D, x_L); the comparisons are the build's, in FP64.
__global__ void k_stree_query(const int* axis, const double* split, const int* left, const int* right, DChains c,
                              uint32_t* chain_cell) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < c.B; b += gridDim.x * blockDim.x) {
    const int q = b / c.spq;
    double p[6] = {(double)c.xD[q], (double)c.xD[c.Q + q], (double)c.xD[2 * c.Q + q],
                   (double)c.xL[b], (double)c.xL[(size_t)c.B + b], (double)c.xL[2 * (size_t)c.B + b]};
    int i = 0;
    for (int d = 0; d <= STREE_MAX_DEPTH && axis[i] >= 0; ++d) {
      const int a = axis[i];
      double x = a == 0 ? p[0] : a == 1 ? p[1] : a == 2 ? p[2] : a == 3 ? p[3] : a == 4 ? p[4] : p[5];
      i = x < split[i] ? left[i] : right[i];
    }
    chain_cell[b] = (uint32_t)left[i];
  }
}
}  // namespace

void stree_build(const float* pos, int n, double eps, double c, StreeHost& t) {
  t = StreeHost{};
  t.n_samples = n;
  Shared sh;
  sh.pos = pos;
  sh.n = n;
  sh.eps = eps;
  sh.T = std::max(1, (int)std::floor(c * std::sqrt((double)n)));
  double lo[6], hi[6];
  for (int a = 0; a < 6; ++a) {
    lo[a] = hi[a] = 0.0;
    for (int i = 0; i < n; ++i) {
      double x = (double)pos[(size_t)a * n + i];
      if (i == 0 || x < lo[a]) lo[a] = x;
      if (i == 0 || x > hi[a]) hi[a] = x;
    }
    sh.root_ext[a] = hi[a] - lo[a];
  }
  sh.idx.resize(n);
  for (int i = 0; i < n; ++i) sh.idx[i] = i;
  for (int a = 0; a < 6; ++a) sh.X[a].assign(pos + (size_t)a * n, pos + (size_t)(a + 1) * n);
  Builder(sh, t).build(0, (size_t)n, {}, lo, hi, 0);
}

// ---------------------------------------------------------------------------
// Level-by-level build (mpg_stree_level.cuh): the passes on the host ...
// ---------------------------------------------------------------------------
namespace {
using stree::LeafOut;
using stree::Segment;
using stree::SplitNode;

void exclusive_scan(std::vector<uint32_t>& a) {
  uint32_t run = 0;
  for (auto& v : a) {
    const uint32_t x = v;
    v = run;
    run += x;
  }
}

// Plain loops taking the device passes' decisions in the same order: owner
// tables, flags, exclusive scans, scatters, digit histograms.
struct HostLevels {
  int n;
  std::vector<int> idx, idx2;
  std::vector<float> X, X2;  // [6][n]
  std::vector<int> pool;
  StreeHost* t;

  HostLevels(const float* pos, int n_, StreeHost* out) : n(n_), idx(n_), idx2(n_), X(pos, pos + (size_t)6 * n_),
                                                         X2((size_t)6 * n_), t(out) {
    for (int i = 0; i < n; ++i) idx[i] = i;
  }
  float x(int a, int64_t p) const { return X[(size_t)a * n + p]; }

  void root_box(double lo[6], double hi[6]) {
    for (int a = 0; a < 6; ++a) {
      float mn = x(a, 0), mx = mn;
      for (int p = 1; p < n; ++p) {
        mn = std::min(mn, x(a, p));
        mx = std::max(mx, x(a, p));
      }
      lo[a] = mn;
      hi[a] = mx;
    }
  }

  void partition(const std::vector<SplitNode>& sn, std::vector<uint32_t>& nleft) {
    std::vector<int> owner(n, -1);
    for (size_t q = 0; q < sn.size(); ++q)
      for (int64_t p = sn[q].b; p < sn[q].e; ++p) owner[p] = (int)q;
    std::vector<uint32_t> f(n + 1, 0);
    for (int p = 0; p < n; ++p)
      if (owner[p] >= 0) f[p] = stree::goes_left(x(sn[owner[p]].axis, p), sn[owner[p]].mid);
    exclusive_scan(f);
    for (int p = 0; p < n; ++p) {
      int64_t d = p;
      if (owner[p] >= 0) {
        const SplitNode& s = sn[owner[p]];
        d = stree::partition_dest(p, s.b, f[p], f[s.b], f[s.e] - f[s.b], stree::goes_left(x(s.axis, p), s.mid));
      }
      idx2[d] = idx[p];
      for (int a = 0; a < 6; ++a) X2[(size_t)a * n + d] = X[(size_t)a * n + p];
    }
    idx.swap(idx2);
    X.swap(X2);
    nleft.resize(sn.size());
    for (size_t q = 0; q < sn.size(); ++q) nleft[q] = f[sn[q].e] - f[sn[q].b];
  }

  void select(const std::vector<Segment>& sg, std::vector<int64_t>& off) {
    const size_t S = sg.size();
    std::vector<int> owner(n, -1);
    for (size_t s = 0; s < S; ++s)
      for (int64_t p = sg[s].b; p < sg[s].e; ++p) owner[p] = (int)s;
    std::vector<uint64_t> prefix(S, 0);
    std::vector<uint32_t> rank(S), hist(S * 256);
    for (size_t s = 0; s < S; ++s) rank[s] = sg[s].m;
    for (int shift = 56; shift >= 0; shift -= 8) {
      std::fill(hist.begin(), hist.end(), 0u);
      for (int p = 0; p < n; ++p) {
        const int s = owner[p];
        if (s < 0) continue;
        const uint64_t u = stree::dist_bits(x(sg[s].axis, p), sg[s].mid);
        if (stree::candidate(u, prefix[s], shift)) hist[(size_t)s * 256 + ((u >> shift) & 255u)]++;
      }
      for (size_t s = 0; s < S; ++s) prefix[s] |= (uint64_t)stree::pick_digit(&hist[s * 256], rank[s]) << shift;
    }
    std::vector<uint32_t> tie(n + 1, 0), sel(n + 1, 0);
    for (int p = 0; p < n; ++p) {
      const int s = owner[p];
      if (s >= 0) tie[p] = stree::dist_bits(x(sg[s].axis, p), sg[s].mid) == prefix[s];
    }
    exclusive_scan(tie);
    for (int p = 0; p < n; ++p) {
      const int s = owner[p];
      if (s < 0) continue;
      const uint64_t u = stree::dist_bits(x(sg[s].axis, p), sg[s].mid);
      sel[p] = u < prefix[s] || (u == prefix[s] && tie[p] - tie[sg[s].b] < rank[s]);
    }
    exclusive_scan(sel);
    const int64_t base = (int64_t)pool.size();
    int64_t total = 0;
    off.resize(S);
    for (size_t s = 0; s < S; ++s) {
      off[s] = base + total;
      total += sg[s].m;
    }
    pool.resize(base + total);
    for (int p = 0; p < n; ++p)
      if (sel[p + 1] != sel[p]) pool[base + sel[p]] = idx[p];
  }

  void emit(const std::vector<LeafOut>& lv, int64_t members) {
    t->member_leaf.assign(members, 0);
    t->member_rec.assign(members, 0);
    for (const LeafOut& L : lv) {
      const int* own = idx.data() + L.b;
      const int* cp = pool.data() + L.copy_off;
      const int64_t no = L.e - L.b, nc = L.copy_cnt;
      for (int64_t i = 0; i < no; ++i) {
        const int64_t pos = i + (std::lower_bound(cp, cp + nc, own[i]) - cp);
        t->member_rec[L.out_off + pos] = own[i];
        t->member_leaf[L.out_off + pos] = L.leaf;
      }
      for (int64_t j = 0; j < nc; ++j) {
        const int64_t pos = j + (std::lower_bound(own, own + no, cp[j]) - own);
        t->member_rec[L.out_off + pos] = cp[j];
        t->member_leaf[L.out_off + pos] = L.leaf;
      }
    }
  }
};

// ... and on the device: the same passes as kernels over all samples of a
// level (owner tables, flags, one-CTA scans, scatters, per-segment digit
// histograms), the node decisions on the host between them.
constexpr int LV_THREADS = 256;

int lv_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(4096, (n + LV_THREADS - 1) / LV_THREADS)); }

__global__ void k_lv_owner(const int64_t* b, const int64_t* e, int stride, int count, int* owner) {
  for (int q = blockIdx.x; q < count; q += gridDim.x) {
    const int64_t lo = b[(size_t)q * stride], hi = e[(size_t)q * stride];
    for (int64_t p = lo + threadIdx.x; p < hi; p += blockDim.x) owner[p] = q;
  }
}

__global__ void k_lv_minmax(const float* X, int n, float* part) {
  __shared__ float smn[LV_THREADS], smx[LV_THREADS];
  for (int a = 0; a < 6; ++a) {
    float mn = INFINITY, mx = -INFINITY;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
      const float v = X[(size_t)a * n + p];
      mn = fminf(mn, v);
      mx = fmaxf(mx, v);
    }
    smn[threadIdx.x] = mn;
    smx[threadIdx.x] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        smn[threadIdx.x] = fminf(smn[threadIdx.x], smn[threadIdx.x + o]);
        smx[threadIdx.x] = fmaxf(smx[threadIdx.x], smx[threadIdx.x + o]);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      part[(size_t)blockIdx.x * 12 + a] = smn[0];
      part[(size_t)blockIdx.x * 12 + 6 + a] = smx[0];
    }
    __syncthreads();
  }
}

__global__ void k_lv_flags(const int* owner, const SplitNode* sn, const float* X, int n, uint32_t* f) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int q = owner[p];
    f[p] = q >= 0 && stree::goes_left(X[(size_t)sn[q].axis * n + p], sn[q].mid);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) f[n] = 0;
}

__global__ void k_lv_scatter(const int* owner, const SplitNode* sn, const float* X, const int* idx, const uint32_t* f,
                             int n, float* X2, int* idx2) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int q = owner[p];
    int64_t d = p;
    if (q >= 0) {
      const SplitNode s = sn[q];
      d = stree::partition_dest(p, s.b, f[p], f[s.b], f[s.e] - f[s.b],
                                stree::goes_left(X[(size_t)s.axis * n + p], s.mid));
    }
    idx2[d] = idx[p];
    for (int a = 0; a < 6; ++a) X2[(size_t)a * n + d] = X[(size_t)a * n + p];
  }
}

__global__ void k_lv_nleft(const SplitNode* sn, int count, const uint32_t* f, uint32_t* nleft) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x)
    nleft[q] = f[sn[q].e] - f[sn[q].b];
}

__global__ void k_lv_hist(const int* owner, const Segment* sg, const uint64_t* prefix, int shift, const float* X,
                          int n, uint32_t* hist) {
  // Every lane of a warp runs the same iterations (the loop test uses the
  // warp's first index), so the whole warp takes part in the match: lanes
  // counting into the same bin add once (the top digits of a segment's
  // distances mostly share one bin).
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p - lane < n; p += stride) {
    unsigned bin = 0xffffffffu;
    if (p < n) {
      const int s = owner[p];
      if (s >= 0) {
        const uint64_t u = stree::dist_bits(X[(size_t)sg[s].axis * n + p], sg[s].mid);
        if (stree::candidate(u, prefix[s], shift)) bin = (unsigned)s * 256u + (unsigned)((u >> shift) & 255u);
      }
    }
    const unsigned peers = __match_any_sync(0xffffffffu, bin);
    if (bin != 0xffffffffu && lane == __ffs(peers) - 1) atomicAdd(hist + bin, (uint32_t)__popc(peers));
  }
}

__global__ void k_lv_pick(int S, const uint32_t* hist, uint64_t* prefix, uint32_t* rank, int shift) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
    uint32_t r = rank[s];
    const uint32_t d = stree::pick_digit(hist + (size_t)s * 256, r);
    rank[s] = r;
    prefix[s] |= (uint64_t)d << shift;
  }
}

__global__ void k_lv_ties(const int* owner, const Segment* sg, const uint64_t* prefix, const float* X, int n,
                          uint32_t* tie) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int s = owner[p];
    tie[p] = s >= 0 && stree::dist_bits(X[(size_t)sg[s].axis * n + p], sg[s].mid) == prefix[s];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) tie[n] = 0;
}

__device__ __forceinline__ bool lv_selected(const int* owner, const Segment* sg, const uint64_t* prefix,
                                            const uint32_t* rank, const uint32_t* tie, const float* X, int n, int p) {
  const int s = owner[p];
  if (s < 0) return false;
  const uint64_t u = stree::dist_bits(X[(size_t)sg[s].axis * n + p], sg[s].mid);
  return u < prefix[s] || (u == prefix[s] && tie[p] - tie[sg[s].b] < rank[s]);
}

__global__ void k_lv_sel(const int* owner, const Segment* sg, const uint64_t* prefix, const uint32_t* rank,
                         const uint32_t* tie, const float* X, int n, uint32_t* sel) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
    sel[p] = lv_selected(owner, sg, prefix, rank, tie, X, n, p);
  if (blockIdx.x == 0 && threadIdx.x == 0) sel[n] = 0;
}

__global__ void k_lv_write(const int* owner, const Segment* sg, const uint64_t* prefix, const uint32_t* rank,
                           const uint32_t* tie, const float* X, const int* idx, const uint32_t* sel, int n,
                           int64_t base, int* pool) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
    if (lv_selected(owner, sg, prefix, rank, tie, X, n, p)) pool[base + sel[p]] = idx[p];
}

__device__ __forceinline__ int64_t count_below(const int* a, int64_t n, int v) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t m = (lo + hi) >> 1;
    if (a[m] < v) lo = m + 1;
    else hi = m;
  }
  return lo;
}

__global__ void k_lv_emit(const LeafOut* lv, int count, const int* idx, const int* pool, int* member_leaf,
                          int* member_rec) {
  for (int q = blockIdx.x; q < count; q += gridDim.x) {
    const LeafOut L = lv[q];
    const int* own = idx + L.b;
    const int* cp = pool + L.copy_off;
    const int64_t no = L.e - L.b, nc = L.copy_cnt;
    for (int64_t i = threadIdx.x; i < no; i += blockDim.x) {
      const int64_t pos = L.out_off + i + count_below(cp, nc, own[i]);
      member_rec[pos] = own[i];
      member_leaf[pos] = L.leaf;
    }
    for (int64_t j = threadIdx.x; j < nc; j += blockDim.x) {
      const int64_t pos = L.out_off + j + count_below(own, no, cp[j]);
      member_rec[pos] = cp[j];
      member_leaf[pos] = L.leaf;
    }
  }
}

struct DevLevels {
  int n;
  cudaStream_t st;
  cudaError_t e = cudaSuccess;
  float *X = nullptr, *X2 = nullptr;
  int *idx = nullptr, *idx2 = nullptr, *owner = nullptr, *pool = nullptr;
  uint32_t *f = nullptr, *tie = nullptr, *sel = nullptr, *scan_sums = nullptr;
  int64_t pool_cap = 0, pool_size = 0;
  std::vector<void*> owned;
  StreeHost* t;

  template <class T>
  T* alloc(size_t count) {
    void* p = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&p, std::max<size_t>(count * sizeof(T), 16));
    if (e == cudaSuccess) owned.push_back(p);
    return (T*)p;
  }
  // a table of host structs on the device, freed with the build
  template <class T>
  T* upload(const std::vector<T>& h) {
    T* d = alloc<T>(h.size());
    if (e == cudaSuccess && !h.empty()) e = cudaMemcpyAsync(d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, st);
    return d;
  }
  // the int64 field at byte offset `at` of the first entry of a device table
  // (entries of the tables are multiples of 8 bytes)
  template <class T>
  static const int64_t* field(const T* d, size_t at) {
    static_assert(sizeof(T) % sizeof(int64_t) == 0, "table entries are read as int64 strides");
    return (const int64_t*)((const char*)d + at);
  }
  bool sync() {
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess;
  }

  DevLevels(float* d_pos, int n_, cudaStream_t s, StreeHost* out) : n(n_), st(s), X(d_pos), t(out) {
    X2 = alloc<float>((size_t)6 * n);
    idx = alloc<int>(n);
    idx2 = alloc<int>(n);
    owner = alloc<int>(n);
    f = alloc<uint32_t>(n + 1);
    tie = alloc<uint32_t>(n + 1);
    sel = alloc<uint32_t>(n + 1);
    scan_sums = alloc<uint32_t>(scan_tiles(n + 1) + 1);
    if (e == cudaSuccess) {
      std::vector<int> iota(n);
      for (int i = 0; i < n; ++i) iota[i] = i;
      e = cudaMemcpy(idx, iota.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice);
    }
  }
  ~DevLevels() {
    cudaStreamSynchronize(st);
    for (void* p : owned) cudaFree(p);
    if (pool) cudaFree(pool);
  }

  void root_box(double lo[6], double hi[6]) {
    const int g = std::min(256, lv_grid(n));
    float* part = alloc<float>((size_t)g * 12);
    if (e == cudaSuccess) k_lv_minmax<<<g, LV_THREADS, 0, st>>>(X, n, part);
    std::vector<float> h((size_t)g * 12, 0.0f);
    if (sync()) e = cudaMemcpy(h.data(), part, sizeof(float) * h.size(), cudaMemcpyDeviceToHost);
    for (int a = 0; a < 6; ++a) {
      float mn = h[a], mx = h[6 + a];
      for (int b = 1; b < g; ++b) {
        mn = std::min(mn, h[(size_t)b * 12 + a]);
        mx = std::max(mx, h[(size_t)b * 12 + 6 + a]);
      }
      lo[a] = mn;
      hi[a] = mx;
    }
  }

  void owners(const int64_t* b, const int64_t* e_, int stride, int count) {
    if (e != cudaSuccess) return;
    e = cudaMemsetAsync(owner, 0xff, sizeof(int) * (size_t)n, st);  // -1 everywhere
    if (e == cudaSuccess && count > 0) k_lv_owner<<<std::min(count, 4096), LV_THREADS, 0, st>>>(b, e_, stride, count, owner);
  }

  void partition(const std::vector<SplitNode>& sn, std::vector<uint32_t>& nleft) {
    nleft.assign(sn.size(), 0);
    SplitNode* d_sn = upload(sn);
    uint32_t* d_nl = alloc<uint32_t>(sn.size());
    owners(field(d_sn, offsetof(SplitNode, b)), field(d_sn, offsetof(SplitNode, e)),
           sizeof(SplitNode) / sizeof(int64_t), (int)sn.size());
    const int g = lv_grid(n);
    if (e == cudaSuccess) {
      k_lv_flags<<<g, LV_THREADS, 0, st>>>(owner, d_sn, X, n, f);
      launch_scan_exclusive_tiled(f, n + 1, scan_sums, st);
      k_lv_scatter<<<g, LV_THREADS, 0, st>>>(owner, d_sn, X, idx, f, n, X2, idx2);
      k_lv_nleft<<<lv_grid((int64_t)sn.size()), LV_THREADS, 0, st>>>(d_sn, (int)sn.size(), f, d_nl);
      std::swap(X, X2);
      std::swap(idx, idx2);
    }
    if (sync()) e = cudaMemcpy(nleft.data(), d_nl, sizeof(uint32_t) * sn.size(), cudaMemcpyDeviceToHost);
  }

  void grow_pool(int64_t need) {
    if (e != cudaSuccess || need <= pool_cap) return;
    const int64_t cap = std::max<int64_t>(need, 2 * pool_cap);
    int* np = nullptr;
    e = cudaMalloc((void**)&np, sizeof(int) * (size_t)cap);
    if (e == cudaSuccess && pool_size > 0)
      e = cudaMemcpyAsync(np, pool, sizeof(int) * (size_t)pool_size, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      if (np) cudaFree(np);
      return;
    }
    if (pool) cudaFree(pool);
    pool = np;
    pool_cap = cap;
  }

  void select(const std::vector<Segment>& sg, std::vector<int64_t>& off) {
    const int S = (int)sg.size();
    off.resize(S);
    // k_lv_hist keys a bin as segment * 256 + digit in 32 bits with 2^32 - 1
    // meaning "no bin": fewer than 2^24 segments per level keep the two apart
    // (a level has at most 2 sqrt(n) segments, each split node holding more
    // than sqrt(n) samples)
    if (S >= (1 << 24)) e = cudaErrorInvalidValue;
    int64_t total = 0;
    for (int s = 0; s < S; ++s) {
      off[s] = pool_size + total;
      total += sg[s].m;
    }
    grow_pool(pool_size + total);
    Segment* d_sg = upload(sg);
    std::vector<uint32_t> r0(S);
    for (int s = 0; s < S; ++s) r0[s] = sg[s].m;
    uint32_t* d_rank = upload(r0);
    uint64_t* d_prefix = alloc<uint64_t>(S);
    uint32_t* d_hist = alloc<uint32_t>((size_t)S * 256);
    owners(field(d_sg, offsetof(Segment, b)), field(d_sg, offsetof(Segment, e)), sizeof(Segment) / sizeof(int64_t),
           S);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_prefix, 0, sizeof(uint64_t) * S, st);
    const int g = lv_grid(n);
    for (int shift = 56; shift >= 0 && e == cudaSuccess; shift -= 8) {
      e = cudaMemsetAsync(d_hist, 0, sizeof(uint32_t) * (size_t)S * 256, st);
      if (e != cudaSuccess) break;
      k_lv_hist<<<g, LV_THREADS, 0, st>>>(owner, d_sg, d_prefix, shift, X, n, d_hist);
      k_lv_pick<<<lv_grid(S), LV_THREADS, 0, st>>>(S, d_hist, d_prefix, d_rank, shift);
    }
    if (e == cudaSuccess) {
      k_lv_ties<<<g, LV_THREADS, 0, st>>>(owner, d_sg, d_prefix, X, n, tie);
      launch_scan_exclusive_tiled(tie, n + 1, scan_sums, st);
      k_lv_sel<<<g, LV_THREADS, 0, st>>>(owner, d_sg, d_prefix, d_rank, tie, X, n, sel);
      launch_scan_exclusive_tiled(sel, n + 1, scan_sums, st);
      k_lv_write<<<g, LV_THREADS, 0, st>>>(owner, d_sg, d_prefix, d_rank, tie, X, idx, sel, n, pool_size, pool);
    }
    sync();
    pool_size += total;
  }

  void emit(const std::vector<LeafOut>& lv, int64_t members) {
    int* d_leaf = alloc<int>(members);
    int* d_rec = alloc<int>(members);
    LeafOut* d_lv = upload(lv);
    if (e == cudaSuccess && !lv.empty())
      k_lv_emit<<<(int)std::min<size_t>(lv.size(), 4096), LV_THREADS, 0, st>>>(d_lv, (int)lv.size(), idx, pool,
                                                                               d_leaf, d_rec);
    t->member_leaf.assign(members, 0);
    t->member_rec.assign(members, 0);
    if (sync() && members > 0) {
      e = cudaMemcpy(t->member_leaf.data(), d_leaf, sizeof(int) * (size_t)members, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess)
        e = cudaMemcpy(t->member_rec.data(), d_rec, sizeof(int) * (size_t)members, cudaMemcpyDeviceToHost);
    }
  }
};

void take_result(const stree::Result& r, int n, StreeHost& t) {
  t.axis = r.axis;
  t.left = r.left;
  t.right = r.right;
  t.split = r.split;
  t.n_leaves = r.n_leaves;
  t.n_samples = n;
}
}  // namespace

void stree_build_levels_host(const float* pos, int n, double eps, double c, StreeHost& t) {
  t = StreeHost{};
  HostLevels ex(pos, n, &t);
  stree::Result r;
  stree::build_levels(ex, n, eps, c, r);
  take_result(r, n, t);
}

bool stree_build_levels_device(float* d_pos, int n, double eps, double c, StreeHost& t, cudaStream_t st,
                               const char** err) {
  t = StreeHost{};
  DevLevels ex(d_pos, n, st, &t);
  stree::Result r;
  if (ex.e == cudaSuccess) stree::build_levels(ex, n, eps, c, r);
  if (ex.e != cudaSuccess) {
    *err = cudaGetErrorString(ex.e);
    return false;
  }
  take_result(r, n, t);
  return true;
}

void launch_stree_gather(const DChains& c, const int* rec_chain, int n, float* pos, cudaStream_t st) {
  if (n > 0) k_stree_gather<<<std::min(1024, (n + 255) / 256), 256, 0, st>>>(c, rec_chain, n, pos);
}

void launch_stree_records(const int* member_leaf, const int* member_rec, int M, const float* omega, const float* w,
                          const uint8_t* k, const uint8_t* tau, int R_in, uint32_t* cell_out, float* omega_out,
                          float* w_out, uint8_t* k_out, uint8_t* tau_out, int R_out, int* R_out_dev, int sms,
                          cudaStream_t st) {
  const int grid = std::max(1, std::min(sms * 8, (M + 255) / 256));
  k_stree_records<<<grid, 256, 0, st>>>(member_leaf, member_rec, M, omega, w, k, tau, R_in, cell_out, omega_out,
                                        w_out, k_out, tau_out, R_out, R_out_dev);
}

void launch_stree_query(const int* axis, const double* split, const int* left, const int* right, const DChains& c,
                        uint32_t* chain_cell, int sms, cudaStream_t st) {
  const int grid = std::max(1, std::min(sms * 8, (c.B + 255) / 256));
  k_stree_query<<<grid, 256, 0, st>>>(axis, split, left, right, c, chain_cell);
}

}  // namespace mpg
