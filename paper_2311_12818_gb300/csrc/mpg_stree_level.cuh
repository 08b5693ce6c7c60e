// Level-by-level build of the spatial tree of Sec. 5.6 (the same tree as the
// recursive host build of mpg_stree.cu): every level partitions the samples
// of all its split nodes at once and selects the copies of spatial filtering
// for all of them at once, so each step is a pass over the level's samples
// that a GPU runs as a few kernels.  The driver below decides nodes, boxes
// and numbering on the host (a few thousand nodes); an executor supplies the
// passes over the samples -- kernels on the device (mpg_stree.cu), or plain
// loops on the host that take the same decisions in the same order, which
// lets the algorithm be checked against the oracle's tree without a GPU.
//
// Invariants the passes keep:
//   * a node owns the contiguous range [b, e) of the sample permutation, and
//     its sample indices are ascending there (the root holds 0..n-1 and every
//     partition is stable), so the ties of the copy selection, broken by
//     sample index, are broken by position;
//   * the distance of a sample to the split plane is |x - mid| in FP64 from
//     the FP32 coordinate, as in the recursive build and the oracle; for
//     non-negative doubles the order of their bit patterns is the order of
//     their values, so the m-th smallest distance of a side is found digit
//     by digit on the bit patterns.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace mpg {
namespace stree {

constexpr int MAX_DEPTH = 48;

__host__ __device__ __forceinline__ bool goes_left(float x, double mid) { return (double)x < mid; }

__host__ __device__ __forceinline__ uint64_t dist_bits(float x, double mid) {
  const double d = fabs((double)x - mid);
  uint64_t u;
#ifdef __CUDA_ARCH__
  u = (uint64_t)__double_as_longlong(d);
#else
  std::memcpy(&u, &d, sizeof u);
#endif
  return u;
}

// Destination of the sample at position p of a split node [b, e) in the
// stable partition, from the exclusive prefix counts of left samples:
// Lp = count before p, Lb = count before b, nl = left samples of the node.
__host__ __device__ __forceinline__ int64_t partition_dest(int64_t p, int64_t b, uint32_t Lp, uint32_t Lb,
                                                          uint32_t nl, bool left) {
  const int64_t before_left = (int64_t)Lp - (int64_t)Lb;
  return left ? b + before_left : b + (int64_t)nl + ((p - b) - before_left);
}

// Does a sample with distance bits u still compete for the digit at `shift`
// of its segment whose higher digits are fixed to `prefix`?
__host__ __device__ __forceinline__ bool candidate(uint64_t u, uint64_t prefix, int shift) {
  return shift >= 56 || ((u ^ prefix) >> (shift + 8)) == 0;
}

// After the digit histogram h[256] of a segment: the digit holding its
// rank-th candidate (1-based); rank becomes the rank within that digit.
__host__ __device__ __forceinline__ uint32_t pick_digit(const uint32_t* h, uint32_t& rank) {
  uint32_t cum = 0;
  for (uint32_t d = 0; d < 256; ++d) {
    if (cum + h[d] >= rank) {
      rank -= cum;
      return d;
    }
    cum += h[d];
  }
  return 255;  // not reached while rank <= the segment's candidates
}

// One split node of a level, as the passes see it.
struct SplitNode {
  int64_t b, e;
  int axis;
  double mid;
};

// One side of a split node whose nearest samples are copied into the other
// child (only when that child is a leaf).
struct Segment {
  int64_t b, e;
  int axis;
  double mid;
  uint32_t m;  // samples to select, <= e - b, > 0
};

// A leaf to emit: own samples [b, e) of the final permutation merged with
// its copies pool[copy_off, copy_off + copy_cnt), written from out_off.
struct LeafOut {
  int64_t b, e, copy_off, copy_cnt, out_off;
  int leaf;
};

struct Node {
  int64_t b, e;
  double lo[6], hi[6];
  int depth;
  int axis = -1;
  double mid = 0.0;
  int left = -1, right = -1;   // children (node indices) of a split node
  int64_t copy_off = 0, copy_cnt = 0;
  bool leaf = false;
};

struct Result {
  std::vector<int> axis, left, right;
  std::vector<double> split;
  int n_leaves = 0;
  int64_t n_members = 0;
};

// Executor interface (Exec):
//   void root_box(double lo[6], double hi[6]);                          n > 0
//   void partition(const std::vector<SplitNode>&, std::vector<uint32_t>& nleft);
//   void select(const std::vector<Segment>&, std::vector<int64_t>& copy_off);  copies of segment s at
//        copy_off[s] .. + m in the pool, ascending by sample index
//   void emit(const std::vector<LeafOut>&, int64_t n_members);
template <class Exec>
void build_levels(Exec& ex, int n, double eps, double c, Result& out) {
  const int T = n > 0 ? (int)std::max(1.0, std::floor(c * std::sqrt((double)n))) : 1;
  std::vector<Node> nodes(1);
  Node& root = nodes[0];
  root.b = 0;
  root.e = n;
  root.depth = 0;
  for (int a = 0; a < 6; ++a) root.lo[a] = root.hi[a] = 0.0;
  if (n > 0) ex.root_box(root.lo, root.hi);
  double root_ext[6];
  for (int a = 0; a < 6; ++a) root_ext[a] = root.hi[a] - root.lo[a];
  // axis of largest extent relative to the root box (first on ties), or -1
  // when the node becomes a leaf
  auto decide = [&](const Node& nd) {
    int a = 0;
    double best = -1.0;
    for (int ax = 0; ax < 6; ++ax) {
      double rel = root_ext[ax] > 0.0 ? (nd.hi[ax] - nd.lo[ax]) / root_ext[ax] : 0.0;
      if (rel > best) {
        best = rel;
        a = ax;
      }
    }
    const int64_t k = nd.e - nd.b;
    return (k <= T || nd.depth >= MAX_DEPTH || !(best > 0.0)) ? -1 : a;
  };
  std::vector<int> active{0};
  root.axis = decide(root);
  root.leaf = root.axis < 0;
  while (!active.empty()) {
    std::vector<int> split;
    for (int j : active)
      if (!nodes[j].leaf) split.push_back(j);
    if (split.empty()) break;
    std::vector<SplitNode> sn;
    for (int j : split) {
      Node& nd = nodes[j];
      nd.mid = 0.5 * (nd.lo[nd.axis] + nd.hi[nd.axis]);
      sn.push_back({nd.b, nd.e, nd.axis, nd.mid});
    }
    std::vector<uint32_t> nleft;
    ex.partition(sn, nleft);
    std::vector<int> next;
    std::vector<Segment> segs;
    std::vector<int> seg_child;
    for (size_t q = 0; q < split.size(); ++q) {
      const int j = split[q];
      const int64_t b = nodes[j].b, e = nodes[j].e, mcut = nodes[j].b + nleft[q];
      const int a = nodes[j].axis;
      const double mid = nodes[j].mid;
      const int64_t m = (int64_t)std::floor(eps * (double)(e - b));
      Node L, R;
      L.b = b; L.e = mcut; R.b = mcut; R.e = e;
      for (int x = 0; x < 6; ++x) {
        L.lo[x] = R.lo[x] = nodes[j].lo[x];
        L.hi[x] = R.hi[x] = nodes[j].hi[x];
      }
      L.hi[a] = mid;
      R.lo[a] = mid;
      L.depth = R.depth = nodes[j].depth + 1;
      L.axis = decide(L);
      L.leaf = L.axis < 0;
      R.axis = decide(R);
      R.leaf = R.axis < 0;
      const int li = (int)nodes.size();
      nodes.push_back(L);
      nodes.push_back(R);
      nodes[j].left = li;
      nodes[j].right = li + 1;
      next.push_back(li);
      next.push_back(li + 1);
      // the left side's nearest samples go to the right child and back
      if (nodes[li + 1].leaf && m > 0 && mcut > b) {
        segs.push_back({b, mcut, a, mid, (uint32_t)std::min<int64_t>(m, mcut - b)});
        seg_child.push_back(li + 1);
      }
      if (nodes[li].leaf && m > 0 && e > mcut) {
        segs.push_back({mcut, e, a, mid, (uint32_t)std::min<int64_t>(m, e - mcut)});
        seg_child.push_back(li);
      }
    }
    if (!segs.empty()) {
      std::vector<int64_t> off;
      ex.select(segs, off);
      for (size_t s = 0; s < segs.size(); ++s) {
        nodes[seg_child[s]].copy_off = off[s];
        nodes[seg_child[s]].copy_cnt = segs[s].m;
      }
    }
    active.swap(next);
  }
  // depth-first numbering, left first (nodes and leaves)
  out = Result{};
  std::vector<int> id(nodes.size(), -1), leaf_id(nodes.size(), -1);
  std::vector<int> order, stack{0};
  while (!stack.empty()) {
    const int j = stack.back();
    stack.pop_back();
    id[j] = (int)order.size();
    order.push_back(j);
    if (nodes[j].leaf) {
      leaf_id[j] = out.n_leaves++;
    } else {
      stack.push_back(nodes[j].right);
      stack.push_back(nodes[j].left);
    }
  }
  std::vector<LeafOut> leaves;
  int64_t members = 0;
  for (int j : order) {
    const Node& nd = nodes[j];
    out.axis.push_back(nd.leaf ? -1 : nd.axis);
    out.split.push_back(nd.leaf ? 0.0 : nd.mid);
    out.left.push_back(nd.leaf ? leaf_id[j] : id[nd.left]);
    out.right.push_back(nd.leaf ? -1 : id[nd.right]);
    if (nd.leaf) {
      leaves.push_back({nd.b, nd.e, nd.copy_off, nd.copy_cnt, members, leaf_id[j]});
      members += (nd.e - nd.b) + nd.copy_cnt;
    }
  }
  out.n_members = members;
  ex.emit(leaves, members);
}

}  // namespace stree
}  // namespace mpg
