// Spatial tree of the guide samples (Sec. 5.6): the host build of the binary
// tree over the samples' (x_D, x_L), and the device kernels around it --
// gathering the samples' positions, turning the leaves' members into guide
// records, and the per-chain leaf query.  The tree is built on the host once
// per training pass (the paper's tree is a host structure too); the queries
// run on the GPU for every chain.
#include <algorithm>
#include <cmath>
#include <future>

#include "mpg_aux.cuh"

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
