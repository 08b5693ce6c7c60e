// FP64 CPU oracle of the batched manifold walk (Manifold Path Guiding, Fan et
// al., TOG 42(6) 2023).  TEST INFRASTRUCTURE ONLY -- the CUDA library shares no
// code with this file; only tests, the smoke check and the benchmark's CPU
// baseline load it.
//
// Plain, slow and written to be read against the paper: one chain at a time,
// FP64, no blocking or fusion.  Where the paper defers the numerics to the
// manifold-walk literature (Sec. 3 "Manifold walks": Newton + reprojection; the
// generalized geometry term after Eq. ThroughputEval), the definitions used are
// the textbook ones restated below:
//   * constraint at specular vertex i: generalized half-vector
//       h~ = eta_i w_i + eta_o w_o,  h = h~/|h~|,  C_i = (h.s_i, h.t_i)
//     with w_i, w_o the unit directions to the previous / next vertex, eta_i
//     the index on the previous vertex's side, eta_o the index on the next
//     vertex's side (eta_o = eta_i for reflection) and (s_i, t_i) an
//     orthonormal tangent frame of the shading normal.  C_i = 0 is the law of
//     reflection / Snell's law in vector form.
//   * Newton on the block-tridiagonal Jacobian dC/du (u_i: tangent-plane
//     offsets of vertex i), a 2x2 block Thomas sweep, step halving and
//     reprojection of each moved vertex onto its own surface by a ray cast along
//     the surface's projection direction (radial / normal / vertical); chain
//     visibility is checked once the walk has converged (admissibility).
//   * G by the implicit function theorem: du/du_L = -J^{-1} dC/du_L.
#include "mpg_oracle.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

namespace orc {

static const int MAXK = 8;
static const double PI = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// Scalar types.  double for the oracle proper; Counted tallies the floating
// point operations of one evaluation (algorithmic flop counts); Dual<N> is
// forward-mode differentiation (adjoint reference).
// ---------------------------------------------------------------------------
struct Tally {
  uint64_t add = 0, mul = 0, div = 0, sqrt = 0;
};
static thread_local Tally g_tally;

struct Counted {
  double v;
  Counted(double x = 0.0) : v(x) {}
};
inline Counted operator+(Counted a, Counted b) { g_tally.add++; return Counted(a.v + b.v); }
inline Counted operator-(Counted a, Counted b) { g_tally.add++; return Counted(a.v - b.v); }
inline Counted operator-(Counted a) { return Counted(-a.v); }
inline Counted operator*(Counted a, Counted b) { g_tally.mul++; return Counted(a.v * b.v); }
inline Counted operator/(Counted a, Counted b) { g_tally.div++; return Counted(a.v / b.v); }
inline Counted& operator+=(Counted& a, Counted b) { a = a + b; return a; }
inline Counted& operator-=(Counted& a, Counted b) { a = a - b; return a; }
inline Counted& operator*=(Counted& a, Counted b) { a = a * b; return a; }
inline Counted sqrt(Counted a) { g_tally.sqrt++; return Counted(std::sqrt(a.v)); }
inline double sqrt(double a) { return std::sqrt(a); }
inline double fabs(double a) { return std::fabs(a); }
inline Counted fabs(Counted a) { return Counted(std::fabs(a.v)); }

template <int N>
struct Dual {
  double v;
  double d[N];
  Dual(double x = 0.0) : v(x) { for (int i = 0; i < N; ++i) d[i] = 0.0; }
};
template <int N> inline Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v + b.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v - b.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
template <int N> inline Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r(-a.v); for (int i = 0; i < N; ++i) r.d[i] = -a.d[i]; return r; }
template <int N> inline Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v * b.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
template <int N> inline Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v / b.v);
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r; }
template <int N> inline Dual<N>& operator+=(Dual<N>& a, const Dual<N>& b) { a = a + b; return a; }
template <int N> inline Dual<N>& operator-=(Dual<N>& a, const Dual<N>& b) { a = a - b; return a; }
template <int N> inline Dual<N>& operator*=(Dual<N>& a, const Dual<N>& b) { a = a * b; return a; }
template <int N> inline Dual<N> sqrt(const Dual<N>& a) {
  double s = std::sqrt(a.v); Dual<N> r(s);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / (2.0 * s);
  return r; }
template <int N> inline Dual<N> fabs(const Dual<N>& a) { return a.v < 0 ? -a : a; }

inline double val(double x) { return x; }
inline double val(const Counted& x) { return x.v; }
template <int N> inline double val(const Dual<N>& x) { return x.v; }

// ---------------------------------------------------------------------------
// 3-vectors
// ---------------------------------------------------------------------------
template <class T>
struct V3 {
  T x, y, z;
  V3() : x(0.0), y(0.0), z(0.0) {}
  V3(T a, T b, T c) : x(a), y(b), z(c) {}
};
typedef V3<double> V3d;
template <class T> inline V3<T> operator+(const V3<T>& a, const V3<T>& b) { return V3<T>(a.x + b.x, a.y + b.y, a.z + b.z); }
template <class T> inline V3<T> operator-(const V3<T>& a, const V3<T>& b) { return V3<T>(a.x - b.x, a.y - b.y, a.z - b.z); }
template <class T> inline V3<T> operator-(const V3<T>& a) { return V3<T>(-a.x, -a.y, -a.z); }
template <class T> inline V3<T> operator*(const V3<T>& a, const T& s) { return V3<T>(a.x * s, a.y * s, a.z * s); }
template <class T> inline V3<T> operator*(const T& s, const V3<T>& a) { return V3<T>(a.x * s, a.y * s, a.z * s); }
template <class T> inline V3<T> operator/(const V3<T>& a, const T& s) { return V3<T>(a.x / s, a.y / s, a.z / s); }
template <class T> inline T dot(const V3<T>& a, const V3<T>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> inline V3<T> cross(const V3<T>& a, const V3<T>& b) {
  return V3<T>(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
template <class T> inline T norm(const V3<T>& a) { using std::sqrt; return sqrt(dot(a, a)); }
template <class T> inline V3<T> normalize(const V3<T>& a) { return a / norm(a); }
template <class T> inline V3<T> lift(const V3d& a) { return V3<T>(T(a.x), T(a.y), T(a.z)); }
inline V3d vval(const V3d& a) { return a; }
template <class T> inline V3d vval(const V3<T>& a) { return V3d(val(a.x), val(a.y), val(a.z)); }
inline V3d load3(const double* p) { return V3d(p[0], p[1], p[2]); }
inline void store3(double* p, const V3d& a) { p[0] = a.x; p[1] = a.y; p[2] = a.z; }

// Orthonormal basis (b1, b2) completing a unit vector n, following the
// branchless construction of Duff et al. 2017 ("Building an orthonormal basis,
// revisited", JCGT 6(1)).  Both sides of the test use this rule because the
// constraint's two components are expressed in this frame.
template <class T>
inline void onb(const V3<T>& n, V3<T>& b1, V3<T>& b2) {
  double sgn = val(n.z) >= 0.0 ? 1.0 : -1.0;
  T s(sgn);
  T a = T(-1.0) / (s + n.z);
  T b = n.x * n.y * a;
  b1 = V3<T>(T(1.0) + s * n.x * n.x * a, s * b, -s * n.x);
  b2 = V3<T>(b, s + n.y * n.y * a, -n.y);
}

// ---------------------------------------------------------------------------
// Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC 2011).
// ---------------------------------------------------------------------------
static void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += W0; k1 += W1; }
    uint64_t p0 = (uint64_t)M0 * c0;
    uint64_t p1 = (uint64_t)M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}
// Uniform in [0,1) from the top 24 bits of a 32-bit draw.
static inline double u01(uint32_t r) { return (double)(r >> 8) * (1.0 / 16777216.0); }

// ---------------------------------------------------------------------------
// Scene
// ---------------------------------------------------------------------------
enum { SURF_SPHERE = 0, SURF_CAP = 1, SURF_RECT = 2, SURF_HEIGHTFIELD = 3 };
enum { MAT_MIRROR = 0, MAT_DIELECTRIC = 1 };
enum { LIGHT_POINT = 0, LIGHT_RECT = 1 };
enum { TARGET_SPHERE = 0, TARGET_RECT = 1 };
enum { ST_INVALID = 0, ST_CONVERGED = 1, ST_FAILED = 2, ST_LIMIT = 3 };

struct Surface {
  int type, mat, hf;
  double etaF, etaB;
  V3d c, axis, ex, ey;
  double r, cap_cos;
};

struct BVHNode {
  double lo[3], hi[3];
  int left, right, first, count;  // count > 0 => leaf over tri_index[first..first+count)
};

struct HField {
  int nx, ny, surf;
  double x0, y0, x1, y1, dx, dy;
  std::vector<double> h;
  std::vector<V3d> P, N;  // vertex positions and interpolation normals
  std::vector<BVHNode> nodes;
  std::vector<int> tri_index;
  int n_tris() const { return 2 * (nx - 1) * (ny - 1); }
  void tri_vertices(int tri, int v[3]) const {
    int quad = tri / 2, t = tri % 2;
    int i = quad % (nx - 1), j = quad / (nx - 1);
    int v00 = j * nx + i, v10 = v00 + 1, v01 = v00 + nx, v11 = v01 + 1;
    if (t == 0) { v[0] = v00; v[1] = v10; v[2] = v11; }
    else { v[0] = v00; v[1] = v11; v[2] = v01; }
  }
};

struct Light {
  int type;
  V3d p, n, ex, ey;
  double power, area;
};

struct Target {
  int type;
  V3d c, ex, ey, n;
  double r;
};

struct Scene {
  std::vector<Surface> surf;
  std::vector<HField> hf;
  std::vector<Target> tg;
  Light light;
};

// Height-grid vertex position and normal.  The normal is the normalised
// (-dh/dx, -dh/dy, 1) with central differences inside the grid and one-sided
// differences on its border.
template <class T, class HeightFn>
V3<T> hf_normal(const HField& H, int i, int j, HeightFn hgt) {
  T dhdx, dhdy;
  if (i == 0) dhdx = (hgt(1, j) - hgt(0, j)) / T(H.dx);
  else if (i == H.nx - 1) dhdx = (hgt(H.nx - 1, j) - hgt(H.nx - 2, j)) / T(H.dx);
  else dhdx = (hgt(i + 1, j) - hgt(i - 1, j)) / T(2.0 * H.dx);
  if (j == 0) dhdy = (hgt(i, 1) - hgt(i, 0)) / T(H.dy);
  else if (j == H.ny - 1) dhdy = (hgt(i, H.ny - 1) - hgt(i, H.ny - 2)) / T(H.dy);
  else dhdy = (hgt(i, j + 1) - hgt(i, j - 1)) / T(2.0 * H.dy);
  return normalize(V3<T>(-dhdx, -dhdy, T(1.0)));
}

static void bvh_build_rec(HField& H, std::vector<V3d>& cen, std::vector<V3d>& blo,
                          std::vector<V3d>& bhi, int first, int count) {
  int node_id = (int)H.nodes.size();
  H.nodes.push_back(BVHNode());
  BVHNode nd;
  for (int a = 0; a < 3; ++a) { nd.lo[a] = 1e300; nd.hi[a] = -1e300; }
  double clo[3] = {1e300, 1e300, 1e300}, chi[3] = {-1e300, -1e300, -1e300};
  for (int q = first; q < first + count; ++q) {
    int t = H.tri_index[q];
    double l[3] = {blo[t].x, blo[t].y, blo[t].z}, h[3] = {bhi[t].x, bhi[t].y, bhi[t].z};
    double c[3] = {cen[t].x, cen[t].y, cen[t].z};
    for (int a = 0; a < 3; ++a) {
      nd.lo[a] = std::min(nd.lo[a], l[a]); nd.hi[a] = std::max(nd.hi[a], h[a]);
      clo[a] = std::min(clo[a], c[a]); chi[a] = std::max(chi[a], c[a]);
    }
  }
  if (count <= 4) {
    nd.left = nd.right = -1; nd.first = first; nd.count = count;
    H.nodes[node_id] = nd;
    return;
  }
  int axis = 0;
  for (int a = 1; a < 3; ++a) if (chi[a] - clo[a] > chi[axis] - clo[axis]) axis = a;
  int mid = first + count / 2;
  auto key = [&](int t) { return axis == 0 ? cen[t].x : axis == 1 ? cen[t].y : cen[t].z; };
  std::nth_element(H.tri_index.begin() + first, H.tri_index.begin() + mid,
                   H.tri_index.begin() + first + count,
                   [&](int a, int b) { return key(a) < key(b) || (key(a) == key(b) && a < b); });
  nd.count = 0; nd.first = -1;
  nd.left = (int)H.nodes.size();
  bvh_build_rec(H, cen, blo, bhi, first, mid - first);
  nd.right = (int)H.nodes.size();
  bvh_build_rec(H, cen, blo, bhi, mid, first + count - mid);
  H.nodes[node_id] = nd;
}

static void hf_build(HField& H) {
  H.dx = (H.x1 - H.x0) / (H.nx - 1);
  H.dy = (H.y1 - H.y0) / (H.ny - 1);
  H.P.resize((size_t)H.nx * H.ny);
  H.N.resize((size_t)H.nx * H.ny);
  auto hgt = [&](int i, int j) { return H.h[(size_t)j * H.nx + i]; };
  for (int j = 0; j < H.ny; ++j)
    for (int i = 0; i < H.nx; ++i) {
      H.P[(size_t)j * H.nx + i] = V3d(H.x0 + i * H.dx, H.y0 + j * H.dy, hgt(i, j));
      H.N[(size_t)j * H.nx + i] = hf_normal<double>(H, i, j, hgt);
    }
  int nt = H.n_tris();
  std::vector<V3d> cen(nt), blo(nt), bhi(nt);
  for (int t = 0; t < nt; ++t) {
    int v[3]; H.tri_vertices(t, v);
    V3d a = H.P[v[0]], b = H.P[v[1]], c = H.P[v[2]];
    cen[t] = (a + b + c) / 3.0;
    blo[t] = V3d(std::min({a.x, b.x, c.x}), std::min({a.y, b.y, c.y}), std::min({a.z, b.z, c.z}));
    bhi[t] = V3d(std::max({a.x, b.x, c.x}), std::max({a.y, b.y, c.y}), std::max({a.z, b.z, c.z}));
  }
  H.tri_index.resize(nt);
  for (int t = 0; t < nt; ++t) H.tri_index[t] = t;
  H.nodes.clear();
  bvh_build_rec(H, cen, blo, bhi, 0, nt);
}

// ---------------------------------------------------------------------------
// Ray casting: the operator r(x, w) of Eq. (deduction) -- nearest intersection
// of a ray with all specular surfaces.
// ---------------------------------------------------------------------------
struct Hit {
  bool hit = false;
  double t = 0.0;
  int surf = -1, prim = -1;
  double b1 = 0.0, b2 = 0.0;
};

// Ray/sphere roots t of |o + t d - c|^2 = r^2 (d unit), ascending.
template <class T>
int sphere_roots(const V3<T>& o, const V3<T>& d, const V3<T>& c, T r, T roots[2]) {
  using std::sqrt;
  V3<T> oc = o - c;
  T b = dot(oc, d);
  T cc = dot(oc, oc) - r * r;
  T disc = b * b - cc;
  if (val(disc) < 0.0) return 0;
  T sq = sqrt(disc);
  roots[0] = -b - sq;
  roots[1] = -b + sq;
  return 2;
}

// Moeller-Trumbore ray/triangle test (Moeller & Trumbore 1997).
template <class T>
bool tri_hit(const V3<T>& o, const V3<T>& d, const V3<T>& p0, const V3<T>& p1, const V3<T>& p2,
             T& t, T& b1, T& b2) {
  V3<T> e1 = p1 - p0, e2 = p2 - p0;
  V3<T> pv = cross(d, e2);
  T det = dot(e1, pv);
  if (std::fabs(val(det)) < 1e-300) return false;
  T inv = T(1.0) / det;
  V3<T> tv = o - p0;
  b1 = dot(tv, pv) * inv;
  if (val(b1) < 0.0 || val(b1) > 1.0) return false;
  V3<T> qv = cross(tv, e1);
  b2 = dot(d, qv) * inv;
  if (val(b2) < 0.0 || val(b1) + val(b2) > 1.0) return false;
  t = dot(e2, qv) * inv;
  return true;
}

// Slab test of a ray against an axis-aligned box, clipped to (tmin, tmax).
static bool box_hit(const V3d& o, const V3d& d, const double lo[3], const double hi[3],
                    double tmin, double tmax) {
  double oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
  for (int a = 0; a < 3; ++a) {
    if (dd[a] == 0.0) {
      if (oo[a] < lo[a] || oo[a] > hi[a]) return false;
      continue;
    }
    double t0 = (lo[a] - oo[a]) / dd[a], t1 = (hi[a] - oo[a]) / dd[a];
    if (t0 > t1) std::swap(t0, t1);
    tmin = std::max(tmin, t0);
    tmax = std::min(tmax, t1);
    if (tmin > tmax) return false;
  }
  return true;
}

static void hf_intersect(const HField& H, const V3d& o, const V3d& d, double tmin, double& tbest,
                         Hit& best, bool brute) {
  auto test_tri = [&](int tri) {
    int v[3]; H.tri_vertices(tri, v);
    double t, b1, b2;
    if (tri_hit<double>(o, d, H.P[v[0]], H.P[v[1]], H.P[v[2]], t, b1, b2) && t > tmin && t < tbest) {
      tbest = t; best.hit = true; best.t = t; best.surf = H.surf; best.prim = tri;
      best.b1 = b1; best.b2 = b2;
    }
  };
  if (brute) {
    for (int tri = 0; tri < H.n_tris(); ++tri) test_tri(tri);
    return;
  }
  std::vector<int> stack;
  stack.push_back(0);
  while (!stack.empty()) {
    int ni = stack.back(); stack.pop_back();
    const BVHNode& nd = H.nodes[ni];
    if (!box_hit(o, d, nd.lo, nd.hi, tmin, tbest)) continue;
    if (nd.count > 0) {
      for (int q = nd.first; q < nd.first + nd.count; ++q) test_tri(H.tri_index[q]);
    } else {
      stack.push_back(nd.left);
      stack.push_back(nd.right);
    }
  }
}

// Nearest hit of the ray (o, d) with any specular surface, t in (tmin, tmax).
static Hit intersect(const Scene& S, const V3d& o, const V3d& d, double tmin, double tmax,
                     bool brute = false) {
  Hit best;
  double tbest = tmax;
  for (int s = 0; s < (int)S.surf.size(); ++s) {
    const Surface& sf = S.surf[s];
    if (sf.type == SURF_SPHERE || sf.type == SURF_CAP) {
      double roots[2];
      if (!sphere_roots<double>(o, d, sf.c, sf.r, roots)) continue;
      for (int q = 0; q < 2; ++q) {
        double t = roots[q];
        if (!(t > tmin && t < tbest)) continue;
        if (sf.type == SURF_CAP) {
          V3d p = o + d * t;
          if (dot(p - sf.c, sf.axis) < sf.r * sf.cap_cos) continue;
        }
        tbest = t; best.hit = true; best.t = t; best.surf = s; best.prim = -1;
        break;
      }
    } else if (sf.type == SURF_RECT) {
      double den = dot(d, sf.axis);
      if (std::fabs(den) < 1e-300) continue;
      double t = dot(sf.c - o, sf.axis) / den;
      if (!(t > tmin && t < tbest)) continue;
      V3d q = o + d * t - sf.c;
      if (std::fabs(dot(q, sf.ex)) > dot(sf.ex, sf.ex) || std::fabs(dot(q, sf.ey)) > dot(sf.ey, sf.ey))
        continue;
      tbest = t; best.hit = true; best.t = t; best.surf = s; best.prim = -1;
    } else if (sf.type == SURF_HEIGHTFIELD) {
      hf_intersect(S.hf[sf.hf], o, d, tmin, tbest, best, brute);
    }
  }
  return best;
}

// ---------------------------------------------------------------------------
// Chain vertices and their local differential geometry
// ---------------------------------------------------------------------------
struct Vtx {
  int surf = -1, prim = -1;
  double b1 = 0.0, b2 = 0.0;
  V3d p;
};

// Point of a hit: on analytic surfaces the ray point snapped onto the surface,
// on triangles the barycentric combination of the corners.
static Vtx hit_vertex(const Scene& S, const V3d& o, const V3d& d, const Hit& h) {
  Vtx v;
  v.surf = h.surf; v.prim = h.prim; v.b1 = h.b1; v.b2 = h.b2;
  const Surface& sf = S.surf[h.surf];
  V3d p = o + d * h.t;
  if (sf.type == SURF_SPHERE || sf.type == SURF_CAP) {
    p = sf.c + normalize(p - sf.c) * sf.r;
  } else if (sf.type == SURF_RECT) {
    p = p - sf.axis * dot(p - sf.c, sf.axis);
  } else {
    const HField& H = S.hf[sf.hf];
    int vv[3]; H.tri_vertices(h.prim, vv);
    p = H.P[vv[0]] + (H.P[vv[1]] - H.P[vv[0]]) * h.b1 + (H.P[vv[2]] - H.P[vv[0]]) * h.b2;
  }
  v.p = p;
  return v;
}

// Local frame of a vertex: position, unit shading normal n (front-facing per
// the surface definition), an orthonormal basis (dpdu, dpdv) of the geometric
// tangent plane, and the derivatives dndu, dndv of n along dpdu and dpdv.
template <class T>
struct Frame {
  V3<T> p, n, dpdu, dpdv, dndu, dndv;
};

template <class T>
Frame<T> frame_sphere(const V3<T>& p, const V3<T>& c, T r) {
  Frame<T> f;
  f.p = p;
  f.n = normalize(p - c);
  onb(f.n, f.dpdu, f.dpdv);
  f.dndu = f.dpdu / r;
  f.dndv = f.dpdv / r;
  return f;
}

template <class T>
Frame<T> frame_plane(const V3<T>& p, const V3<T>& n) {
  Frame<T> f;
  f.p = p;
  f.n = n;
  onb(f.n, f.dpdu, f.dpdv);
  f.dndu = V3<T>();
  f.dndv = V3<T>();
  return f;
}

// Triangle with per-corner normals: n = normalize(sum b_j N_j).  Moving the
// point by a tangent vector a changes the barycentrics by the solution of
// a = db1 e1 + db2 e2, hence the interpolated normal by db1 (N1-N0) + db2 (N2-N0).
template <class T>
Frame<T> frame_triangle(const V3<T>& P0, const V3<T>& P1, const V3<T>& P2, const V3<T>& N0,
                        const V3<T>& N1, const V3<T>& N2, T b1, T b2) {
  Frame<T> f;
  V3<T> e1 = P1 - P0, e2 = P2 - P0;
  f.p = P0 + e1 * b1 + e2 * b2;
  V3<T> ng = normalize(cross(e1, e2));
  onb(ng, f.dpdu, f.dpdv);
  V3<T> Ns = N0 * (T(1.0) - b1 - b2) + N1 * b1 + N2 * b2;
  T len = norm(Ns);
  f.n = Ns / len;
  T g11 = dot(e1, e1), g12 = dot(e1, e2), g22 = dot(e2, e2);
  T gdet = g11 * g22 - g12 * g12;
  V3<T> dirs[2] = {f.dpdu, f.dpdv};
  V3<T> out[2];
  for (int q = 0; q < 2; ++q) {
    T r1 = dot(e1, dirs[q]), r2 = dot(e2, dirs[q]);
    T db1 = (g22 * r1 - g12 * r2) / gdet;
    T db2 = (g11 * r2 - g12 * r1) / gdet;
    V3<T> dN = (N1 - N0) * db1 + (N2 - N0) * db2;
    out[q] = (dN - f.n * dot(f.n, dN)) / len;
  }
  f.dndu = out[0];
  f.dndv = out[1];
  return f;
}

static Frame<double> vertex_frame(const Scene& S, const Vtx& v) {
  const Surface& sf = S.surf[v.surf];
  if (sf.type == SURF_SPHERE || sf.type == SURF_CAP) return frame_sphere<double>(v.p, sf.c, sf.r);
  if (sf.type == SURF_RECT) return frame_plane<double>(v.p, sf.axis);
  const HField& H = S.hf[sf.hf];
  int vv[3]; H.tri_vertices(v.prim, vv);
  return frame_triangle<double>(H.P[vv[0]], H.P[vv[1]], H.P[vv[2]], H.N[vv[0]], H.N[vv[1]],
                                H.N[vv[2]], v.b1, v.b2);
}

// Frames of the two separators: the receiver's tangent plane at x_D (used by
// the point-light geometry term) and the emitter's axes at x_L (area light).
static Frame<double> receiver_frame(const V3d& xD, const V3d& nD) {
  return frame_plane<double>(xD, nD);
}
static Frame<double> light_frame(const Light& L, const V3d& xL) {
  Frame<double> f;
  f.p = xL;
  f.n = L.n;
  if (L.type == LIGHT_RECT) {
    f.dpdu = normalize(L.ex);
    f.dpdv = normalize(L.ey);
  } else {
    onb(L.n, f.dpdu, f.dpdv);
  }
  return f;
}

// ---------------------------------------------------------------------------
// Constraint and Jacobian blocks at one specular vertex
// ---------------------------------------------------------------------------
template <class T>
struct VBlocks {
  T C[2];
  T A[2][2];   // dC_i / du_{i-1}
  T B[2][2];   // dC_i / du_i
  T Cc[2][2];  // dC_i / du_{i+1}
  T eta_i, eta_o;
  bool front;
};

// Indices of refraction on the previous / next vertex's side.  Returns false
// for a refraction requested on a mirror.
static bool vertex_etas(const Surface& sf, bool front, bool refract, double& eta_i, double& eta_o) {
  if (sf.mat == MAT_MIRROR) {
    eta_i = eta_o = 1.0;
    return !refract;
  }
  eta_i = front ? sf.etaF : sf.etaB;
  eta_o = refract ? (front ? sf.etaB : sf.etaF) : eta_i;
  return true;
}

template <class T>
bool vertex_blocks(const Frame<T>& fp, const Frame<T>& f, const Frame<T>& fn, const Surface& sf,
                   bool refract, VBlocks<T>& out, bool c_only = false) {
  using std::sqrt;
  V3<T> wi = fp.p - f.p, wo = fn.p - f.p;
  T di = norm(wi), dO = norm(wo);
  if (val(di) <= 0.0 || val(dO) <= 0.0) return false;
  wi = wi / di;
  wo = wo / dO;
  out.front = val(dot(wi, f.n)) > 0.0;
  double ei, eo;
  if (!vertex_etas(sf, out.front, refract, ei, eo)) return false;
  out.eta_i = T(ei);
  out.eta_o = T(eo);
  V3<T> ht = wi * out.eta_i + wo * out.eta_o;
  T L = norm(ht);
  if (val(L) <= 0.0) return false;
  V3<T> h = ht / L;
  V3<T> s, t;
  onb(f.n, s, t);
  out.C[0] = dot(h, s);
  out.C[1] = dot(h, t);
  if (c_only) return true;
  // Projections: P_w a = (a - w (w.a)) / d is the derivative of a unit
  // direction w = (y - x)/|y - x| with respect to y along a.
  auto Pwi = [&](const V3<T>& a) { return (a - wi * dot(wi, a)) / di; };
  auto Pwo = [&](const V3<T>& a) { return (a - wo * dot(wo, a)) / dO; };
  auto Ph = [&](const V3<T>& a) { return (a - h * dot(h, a)) / L; };
  const V3<T>* tp[2] = {&fp.dpdu, &fp.dpdv};
  const V3<T>* tn[2] = {&fn.dpdu, &fn.dpdv};
  const V3<T>* tc[2] = {&f.dpdu, &f.dpdv};
  const V3<T>* dn[2] = {&f.dndu, &f.dndv};
  T hn = dot(h, f.n);
  for (int j = 0; j < 2; ++j) {
    V3<T> dhA = Ph(Pwi(*tp[j]) * out.eta_i);
    out.A[0][j] = dot(dhA, s);
    out.A[1][j] = dot(dhA, t);
    V3<T> dhC = Ph(Pwo(*tn[j]) * out.eta_o);
    out.Cc[0][j] = dot(dhC, s);
    out.Cc[1][j] = dot(dhC, t);
    V3<T> dhB = -Ph(Pwi(*tc[j]) * out.eta_i + Pwo(*tc[j]) * out.eta_o);
    // The frame (s, t) turns with the normal: ds = -(s.dn) n, dt = -(t.dn) n.
    out.B[0][j] = dot(dhB, s) - hn * dot(s, *dn[j]);
    out.B[1][j] = dot(dhB, t) - hn * dot(t, *dn[j]);
  }
  return true;
}

// Whole-chain evaluation: frames f[0..k+1] (f[0] receiver, f[k+1] light).
template <class T>
bool chain_blocks(const Scene& S, int k, uint8_t tau, const Frame<T>* f, const int* surf,
                  VBlocks<T>* vb) {
  for (int i = 1; i <= k; ++i) {
    bool refract = (tau >> (i - 1)) & 1;
    if (!vertex_blocks(f[i - 1], f[i], f[i + 1], S.surf[surf[i]], refract, vb[i - 1])) return false;
  }
  return true;
}

// ---------------------------------------------------------------------------
// 2x2 block Thomas sweep for J X = R, J block-tridiagonal with rows
// (A_i, B_i, Cc_i); R has m columns (1 for the Newton step, 2 for G).
// ---------------------------------------------------------------------------
template <class T>
struct M2 {
  T a[2][2];
};
template <class T> inline M2<T> mmul(const M2<T>& x, const M2<T>& y) {
  M2<T> r;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) r.a[i][j] = x.a[i][0] * y.a[0][j] + x.a[i][1] * y.a[1][j];
  return r;
}

template <class T>
bool block_thomas(int k, const VBlocks<T>* vb, int m, const T* rhs /*[k][2][m]*/, T* x /*[k][2][m]*/,
                  double sing_eps) {
  std::vector<M2<T>> Bp(k), Binv(k);
  std::vector<T> rp((size_t)k * 2 * m);
  auto R = [&](int i, int r, int c) -> T& { return rp[((size_t)i * 2 + r) * m + c]; };
  for (int i = 0; i < k; ++i) {
    M2<T> B;
    for (int r = 0; r < 2; ++r) for (int c = 0; c < 2; ++c) B.a[r][c] = vb[i].B[r][c];
    for (int r = 0; r < 2; ++r) for (int c = 0; c < m; ++c) R(i, r, c) = rhs[((size_t)i * 2 + r) * m + c];
    if (i > 0) {
      M2<T> A, Cp;
      for (int r = 0; r < 2; ++r) for (int c = 0; c < 2; ++c) {
        A.a[r][c] = vb[i].A[r][c];
        Cp.a[r][c] = vb[i - 1].Cc[r][c];
      }
      M2<T> Lm = mmul(A, Binv[i - 1]);
      M2<T> LC = mmul(Lm, Cp);
      for (int r = 0; r < 2; ++r) for (int c = 0; c < 2; ++c) B.a[r][c] = B.a[r][c] - LC.a[r][c];
      for (int c = 0; c < m; ++c) {
        T r0 = R(i - 1, 0, c), r1 = R(i - 1, 1, c);
        R(i, 0, c) = R(i, 0, c) - (Lm.a[0][0] * r0 + Lm.a[0][1] * r1);
        R(i, 1, c) = R(i, 1, c) - (Lm.a[1][0] * r0 + Lm.a[1][1] * r1);
      }
    }
    T det = B.a[0][0] * B.a[1][1] - B.a[0][1] * B.a[1][0];
    double mx = 0.0;
    for (int r = 0; r < 2; ++r) for (int c = 0; c < 2; ++c) mx = std::max(mx, std::fabs(val(B.a[r][c])));
    if (!(std::fabs(val(det)) > sing_eps * mx * mx)) return false;
    Bp[i] = B;
    Binv[i].a[0][0] = B.a[1][1] / det;
    Binv[i].a[0][1] = -B.a[0][1] / det;
    Binv[i].a[1][0] = -B.a[1][0] / det;
    Binv[i].a[1][1] = B.a[0][0] / det;
  }
  for (int i = k - 1; i >= 0; --i) {
    for (int c = 0; c < m; ++c) {
      T r0 = R(i, 0, c), r1 = R(i, 1, c);
      if (i < k - 1) {
        T x0 = x[((size_t)(i + 1) * 2 + 0) * m + c], x1 = x[((size_t)(i + 1) * 2 + 1) * m + c];
        r0 = r0 - (vb[i].Cc[0][0] * x0 + vb[i].Cc[0][1] * x1);
        r1 = r1 - (vb[i].Cc[1][0] * x0 + vb[i].Cc[1][1] * x1);
      }
      x[((size_t)i * 2 + 0) * m + c] = Binv[i].a[0][0] * r0 + Binv[i].a[0][1] * r1;
      x[((size_t)i * 2 + 1) * m + c] = Binv[i].a[1][0] * r0 + Binv[i].a[1][1] * r1;
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// Seed chains: Eq. (deduction) -- x_1 = r(x_D, w_D), then each next vertex is
// the hit of the ray scattered at the previous one by its type tau_i.
// ---------------------------------------------------------------------------
// Scattered direction of the propagation direction d at a vertex with shading
// normal n.  Reflection: mirror about n.  Refraction: Snell's law with the
// indices of the surface's two sides; returns false on total internal reflection.
static bool scatter(const Surface& sf, const V3d& n, const V3d& d, bool refract, V3d& out) {
  if (!refract) {
    out = d - n * (2.0 * dot(d, n));
    return true;
  }
  if (sf.mat == MAT_MIRROR) return false;
  double cos_i = -dot(d, n);
  double eta1 = sf.etaF, eta2 = sf.etaB;
  V3d nn = n;
  if (cos_i < 0.0) {  // arriving from the back side
    cos_i = -cos_i; eta1 = sf.etaB; eta2 = sf.etaF; nn = -n;
  }
  double eta = eta1 / eta2;
  double k2 = 1.0 - eta * eta * (1.0 - cos_i * cos_i);
  if (k2 < 0.0) return false;
  out = normalize(d * eta + nn * (eta * cos_i - std::sqrt(k2)));
  return true;
}

struct ChainIO {
  int k;
  uint8_t tau;
  Vtx v[MAXK + 2];  // v[0] = x_D, v[k+1] = x_L
};

static bool deduce(const Scene& S, const V3d& xD, const V3d& wD, int k, uint8_t tau, double ray_eps,
                   ChainIO& ch) {
  V3d o = xD, d = wD;
  for (int i = 1; i <= k; ++i) {
    Hit h = intersect(S, o, d, ray_eps, std::numeric_limits<double>::infinity());
    if (!h.hit) return false;
    ch.v[i] = hit_vertex(S, o, d, h);
    if (i < k) {
      Frame<double> f = vertex_frame(S, ch.v[i]);
      V3d dn;
      if (!scatter(S.surf[h.surf], f.n, d, (tau >> (i - 1)) & 1, dn)) return false;
      o = ch.v[i].p;
      d = dn;
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// Guide histogram over world directions: theta from +z uniform over [0,pi],
// phi uniform over [0,2pi).  The bin rule uses only comparisons of the FP32
// direction with FP32 edge data (theta) and exact FP64 signs of 2x2 cross
// products of FP32 values (phi), so it is reproducible bit for bit.
// ---------------------------------------------------------------------------
static int guide_bin(const orc_guide& g, const float w[3]) {
  int it = 0;
  for (int j = 1; j < g.n_theta; ++j)
    if (w[2] < g.cos_theta[j]) ++it;
  float x = w[0], y = w[1];
  bool upper = (y > 0.0f) || (y == 0.0f && x >= 0.0f);
  int half = g.n_phi / 2;
  int ip = upper ? 0 : half;
  int j0 = upper ? 1 : half + 1, j1 = upper ? half : g.n_phi;
  for (int j = j0; j < j1; ++j) {
    double cr = (double)g.phi_cos[j] * (double)y - (double)g.phi_sin[j] * (double)x;
    if (cr >= 0.0) ++ip;
  }
  return it * g.n_phi + ip;
}

static uint64_t quantise_weight(float w, int shift) {
  if (!(w > 0.0f)) return 0;
  double q = std::floor((double)w * std::ldexp(1.0, shift));
  if (q >= 4294967295.0) return 4294967295ull;
  return (uint64_t)q;
}

struct GuideCDF {
  std::vector<uint64_t> cdf;  // [n_cells][bins] inclusive prefix sums
  int bins = 0;
};

static void guide_cdf(const orc_guide& g, GuideCDF& out) {
  out.bins = g.n_theta * g.n_phi;
  out.cdf.assign((size_t)g.n_cells * out.bins, 0);
  for (int c = 0; c < g.n_cells; ++c) {
    uint64_t s = 0;
    for (int b = 0; b < out.bins; ++b) {
      s += g.counts[(size_t)c * out.bins + b];
      out.cdf[(size_t)c * out.bins + b] = s;
    }
  }
}

// Solid-angle density at x_D of the direction sampler p_0 for direction w:
// targets are picked uniformly; a sphere target is sampled uniformly by area on
// the cap visible from x_D, a rectangle uniformly by area.
static double p0_pdf(const Scene& S, const V3d& xD, const V3d& w) {
  double sum = 0.0;
  for (const Target& tg : S.tg) {
    if (tg.type == TARGET_SPHERE) {
      double d = norm(xD - tg.c);
      if (d <= tg.r) continue;
      double roots[2];
      if (!sphere_roots<double>(xD, w, tg.c, tg.r, roots) || roots[0] <= 0.0) continue;
      V3d p = xD + w * roots[0];
      double cosp = std::fabs(dot(normalize(p - tg.c), w));
      double pA = 1.0 / (2.0 * PI * tg.r * tg.r * (1.0 - tg.r / d));
      sum += pA * roots[0] * roots[0] / cosp;
    } else {
      double den = dot(w, tg.n);
      if (std::fabs(den) < 1e-300) continue;
      double t = dot(tg.c - xD, tg.n) / den;
      if (t <= 0.0) continue;
      V3d q = xD + w * t - tg.c;
      if (std::fabs(dot(q, tg.ex)) > dot(tg.ex, tg.ex) || std::fabs(dot(q, tg.ey)) > dot(tg.ey, tg.ey))
        continue;
      double area = 4.0 * norm(tg.ex) * norm(tg.ey);
      sum += t * t / (area * std::fabs(den));
    }
  }
  return S.tg.empty() ? 0.0 : sum / (double)S.tg.size();
}

static double hist_pdf(const orc_guide& g, const GuideCDF& cdf, int cell, const V3d& w) {
  float wf[3] = {(float)w.x, (float)w.y, (float)w.z};
  int bin = guide_bin(g, wf);
  uint64_t total = cdf.cdf[(size_t)cell * cdf.bins + cdf.bins - 1];
  if (total == 0) return 0.0;
  uint64_t cnt = g.counts[(size_t)cell * cdf.bins + bin];
  int it = bin / g.n_phi;
  double dphi = 2.0 * PI / g.n_phi;
  double dcos = (double)g.cos_theta[it] - (double)g.cos_theta[it + 1];
  return ((double)cnt / (double)total) / (dphi * dcos);
}

// ---------------------------------------------------------------------------
// vMF mixture guide (Sec. 5.5).  The samples of the last pass that share the
// receiver cell stand for the neighbourhood S(x_D, x_L); grouped by chain
// length n and types tau they give
//   P_e(n)        = W(n) / W              (weights summed over the cell),
//   P_e(tau | n)  = W(n, tau) / W(n),
//   p_e(w | tau)  = sum_i (w_i / W(n, tau)) v(w; mu_i, kappa_i)   (Eq. vMF)
// with mu_i the sample's direction w_D and kappa_i = sigma_i^-2, sigma_i the
// angle between w_D and the nearest other direction of its group.  Weights
// are the Eq. eq_weight weights quantised as for the histograms, so the
// discrete choices are exact integer decisions.
// ---------------------------------------------------------------------------
static const double VMF_SIGMA_MIN = 1e-6;  // identical directions

// Uniform in (0,1]: the draw of u01 shifted up by one step.
static inline double u01c(uint32_t r) { return (double)((r >> 8) + 1u) * (1.0 / 16777216.0); }

// v(w; mu, kappa) = kappa / (4 pi sinh kappa) e^{kappa mu.w}, written as
// kappa / (2 pi (1 - e^{-2 kappa})) e^{-kappa (1 - mu.w)} with
// 1 - mu.w = |w - mu|^2 / 2 for unit vectors.
static double vmf_pdf(const V3d& mu, double kappa, const V3d& w) {
  V3d d = w - mu;
  double h = 0.5 * dot(d, d);
  return kappa / (2.0 * PI * -std::expm1(-2.0 * kappa)) * std::exp(-kappa * h);
}

// t = 1 - mu.w has density kappa e^{-kappa t} / (1 - e^{-2 kappa}) on [0, 2]
// and the azimuth is uniform; t by inverting its distribution function with
// u1 in (0, 1], the azimuth 2 pi u2 in the Duff et al. frame of mu.
static V3d vmf_sample(const V3d& mu, double kappa, double u1, double u2) {
  double t = -std::log(u1 + (1.0 - u1) * std::exp(-2.0 * kappa)) / kappa;
  t = std::min(std::max(t, 0.0), 2.0);
  double ct = 1.0 - t, st = std::sqrt(std::max(0.0, t * (2.0 - t)));
  V3d e1, e2;
  onb(mu, e1, e2);
  double ph = 2.0 * PI * u2;
  return mu * ct + (e1 * std::cos(ph) + e2 * std::sin(ph)) * st;
}

// Lobes of `cell` whose key lies in [klo, khi): index range [a, b), the
// cell-local prefix sum before a, and the range's total weight.
struct LobeRange {
  uint32_t a = 0, b = 0;
  uint64_t base = 0, total = 0;
};
static LobeRange lobe_range(const orc_vmf& v, uint32_t cell, uint32_t klo, uint32_t khi) {
  LobeRange r;
  uint32_t c0 = v.cell_start[cell], c1 = v.cell_start[cell + 1];
  r.a = c1;
  r.b = c1;
  for (uint32_t i = c0; i < c1; ++i)
    if (v.key[i] >= klo) { r.a = i; break; }
  for (uint32_t i = r.a; i < c1; ++i)
    if (v.key[i] >= khi) { r.b = i; break; }
  r.base = r.a > c0 ? v.prefix[r.a - 1] : 0;
  r.total = r.b > r.a ? v.prefix[r.b - 1] - r.base : 0;
  return r;
}

// Quantised weight of lobe i (difference of the cell-local prefix sums).
static uint64_t lobe_weight(const orc_vmf& v, uint32_t cell, uint32_t i) {
  return v.prefix[i] - (i > v.cell_start[cell] ? v.prefix[i - 1] : 0);
}

// First lobe of [a, b) whose cell-local prefix sum exceeds base + target.
static uint32_t lobe_search(const orc_vmf& v, const LobeRange& r, uint64_t target) {
  for (uint32_t i = r.a; i < r.b; ++i)
    if (v.prefix[i] - r.base > target) return i;
  return r.b - 1;
}

// floor(r * total / 2^32) in exact integer arithmetic.
static uint64_t scaled_target(uint32_t r, uint64_t total) {
  unsigned __int128 prod = (unsigned __int128)r * (unsigned __int128)total;
  return (uint64_t)(prod >> 32);
}

struct SeedDraw {
  bool valid = false;
  uint8_t tau = 0;
  double pdf = 0.0;
  ChainIO ch;
};

static SeedDraw sample_seed(const Scene& S, const orc_guide* g, const GuideCDF* cdf, const V3d& xD,
                            const V3d& nD, uint32_t cell, const V3d& xL, int k, uint8_t tau_in,
                            bool tau_random, uint64_t rng_seed, uint64_t idx, uint32_t trial,
                            const orc_params& prm) {
  SeedDraw sd;
  uint32_t key[2] = {(uint32_t)rng_seed, (uint32_t)(rng_seed >> 32)};
  uint32_t c0[4] = {(uint32_t)idx, (uint32_t)(idx >> 32), trial, 0u};
  uint32_t c1[4] = {(uint32_t)idx, (uint32_t)(idx >> 32), trial, 1u};
  uint32_t r0[4], r1[4];
  philox4x32_10(c0, key, r0);
  philox4x32_10(c1, key, r1);
  uint8_t tau = tau_random ? (uint8_t)(r1[1] & ((1u << k) - 1u)) : tau_in;
  sd.tau = tau;  // the guided vMF component may replace it below
  uint64_t total = 0;
  const orc_vmf* vm = g ? g->vmf : nullptr;
  LobeRange lr;
  bool use_guide = false;
  if (vm) {
    // the guided component draws (w, tau) given n, or w given n and tau when
    // the types are fixed
    uint32_t klo = ((uint32_t)k << 8) | (tau_random ? 0u : tau_in);
    uint32_t khi = tau_random ? ((uint32_t)(k + 1) << 8) : klo + 1;
    lr = lobe_range(*vm, cell, klo, khi);
    total = lr.total;
    use_guide = total > 0;
    // selective activation (Sec. 5.8): no sample in the cell, no seed
    if (prm.selective && vm->cell_start[cell] == vm->cell_start[cell + 1]) return sd;
  } else {
    use_guide = g && g->counts && cdf;
    if (use_guide) total = cdf->cdf[(size_t)cell * cdf->bins + cdf->bins - 1];
    if (prm.selective && use_guide && total == 0) return sd;  // selective activation
    use_guide = use_guide && total > 0;
  }
  bool pick_p0 = !use_guide || u01(r0[0]) < prm.alpha;
  V3d w;
  if (!pick_p0 && vm) {
    uint32_t i = lobe_search(*vm, lr, scaled_target(r0[1], total));
    tau = (uint8_t)(vm->key[i] & 255u);
    const double* L = vm->lobe + 4 * (size_t)i;
    w = vmf_sample(V3d(L[0], L[1], L[2]), L[3], u01c(r0[2]), u01(r0[3]));
  }
  sd.tau = tau;
  if (!pick_p0 && vm) {
  } else if (pick_p0) {
    if (S.tg.empty()) return sd;
    int nt = (int)S.tg.size();
    int ti = std::min((int)(u01(r1[0]) * nt), nt - 1);
    const Target& tg = S.tg[ti];
    double u1 = u01(r0[2]), u2 = u01(r0[3]);
    V3d p;
    if (tg.type == TARGET_SPHERE) {
      double d = norm(xD - tg.c);
      if (d <= tg.r) return sd;
      V3d a = (xD - tg.c) / d, e1, e2;
      onb(a, e1, e2);
      double ca = tg.r / d + u1 * (1.0 - tg.r / d);
      double sa = std::sqrt(std::max(0.0, 1.0 - ca * ca));
      double ph = 2.0 * PI * u2;
      p = tg.c + (a * ca + (e1 * std::cos(ph) + e2 * std::sin(ph)) * sa) * tg.r;
    } else {
      p = tg.c + tg.ex * (2.0 * u1 - 1.0) + tg.ey * (2.0 * u2 - 1.0);
    }
    w = normalize(p - xD);
  } else {
    // bin by inverse CDF on exact integers: target = floor(r * total / 2^32)
    uint64_t r = r0[1];
    unsigned __int128 prod = (unsigned __int128)r * (unsigned __int128)total;
    uint64_t target = (uint64_t)(prod >> 32);
    const uint64_t* c = &cdf->cdf[(size_t)cell * cdf->bins];
    int lo = 0, hi = cdf->bins - 1;
    while (lo < hi) {
      int mid = (lo + hi) / 2;
      if (c[mid] > target) hi = mid; else lo = mid + 1;
    }
    int it = lo / g->n_phi, ip = lo % g->n_phi;
    double clo = g->cos_theta[it], chi = g->cos_theta[it + 1];
    double ct = clo + u01(r0[2]) * (chi - clo);
    double st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
    double ph = 2.0 * PI * ((double)ip + u01(r0[3])) / g->n_phi;
    w = V3d(st * std::cos(ph), st * std::sin(ph), ct);
  }
  if (dot(w, nD) <= 0.0) return sd;
  double p0 = p0_pdf(S, xD, w);
  if (vm) {
    // joint density of (w, tau) given n: p_0 draws the types uniformly
    if (tau_random) p0 *= std::ldexp(1.0, -k);
    double pe = 0.0;
    if (use_guide) {
      uint32_t kt = ((uint32_t)k << 8) | tau;
      for (uint32_t i = lr.a; i < lr.b; ++i) {
        if (vm->key[i] != kt) continue;
        const double* L = vm->lobe + 4 * (size_t)i;
        pe += (double)lobe_weight(*vm, cell, i) / (double)total * vmf_pdf(V3d(L[0], L[1], L[2]), L[3], w);
      }
    }
    sd.pdf = use_guide ? prm.alpha * p0 + (1.0 - prm.alpha) * pe : p0;
  } else {
    sd.pdf = use_guide ? prm.alpha * p0 + (1.0 - prm.alpha) * hist_pdf(*g, *cdf, cell, w) : p0;
  }
  sd.ch.k = k;
  sd.ch.tau = tau;
  sd.ch.v[0].p = xD;
  sd.ch.v[k + 1].p = xL;
  if (!deduce(S, xD, w, k, tau, prm.ray_eps, sd.ch)) return sd;
  sd.valid = true;
  return sd;
}

// ---------------------------------------------------------------------------
// Manifold walk (Sec. 3): Newton's method on C(u) = 0 with reprojection.
// ---------------------------------------------------------------------------
struct EvalOut {
  bool ok = false;
  double cmax = 0.0, cnorm2 = 0.0;
  VBlocks<double> vb[MAXK];
  Frame<double> f[MAXK + 2];
};

static void chain_frames(const Scene& S, const ChainIO& ch, const V3d& nD, Frame<double>* f) {
  f[0] = receiver_frame(ch.v[0].p, nD);
  for (int i = 1; i <= ch.k; ++i) f[i] = vertex_frame(S, ch.v[i]);
  f[ch.k + 1] = light_frame(S.light, ch.v[ch.k + 1].p);
}

// off (may be NULL): offset normals of a glossy chain, [k][2] tangential
// components in each vertex's (s, t) frame; the constraint becomes
// C_i = (h.s, h.t) - off_i (Sec. 5.7, glossy chains).  The Jacobian blocks do
// not change.
static void eval_chain(const Scene& S, const ChainIO& ch, const V3d& nD, EvalOut& ev,
                       const double* off = nullptr) {
  chain_frames(S, ch, nD, ev.f);
  int surf[MAXK + 2];
  for (int i = 0; i <= ch.k + 1; ++i) surf[i] = ch.v[i].surf;
  ev.ok = chain_blocks<double>(S, ch.k, ch.tau, ev.f, surf, ev.vb);
  if (!ev.ok) return;
  if (off)
    for (int i = 0; i < ch.k; ++i)
      for (int c = 0; c < 2; ++c) ev.vb[i].C[c] -= off[2 * i + c];
  ev.cmax = 0.0;
  ev.cnorm2 = 0.0;
  for (int i = 0; i < ch.k; ++i)
    for (int c = 0; c < 2; ++c) {
      ev.cmax = std::max(ev.cmax, std::fabs(ev.vb[i].C[c]));
      ev.cnorm2 += ev.vb[i].C[c] * ev.vb[i].C[c];
    }
}

// Vertical ray cast into a heightfield at (x, y): the triangle of the grid
// cell containing (x, y) and the barycentrics of the point in it.
static bool hf_vertical_hit(const HField& H, double x, double y, Vtx& v) {
  double fx = (x - H.x0) / H.dx, fy = (y - H.y0) / H.dy;
  if (!(fx >= 0.0 && fy >= 0.0 && fx <= H.nx - 1 && fy <= H.ny - 1)) return false;
  int i = std::min((int)fx, H.nx - 2), j = std::min((int)fy, H.ny - 2);
  double u = fx - i, w = fy - j;
  int quad = j * (H.nx - 1) + i;
  if (u >= w) { v.prim = 2 * quad; v.b1 = u - w; v.b2 = w; }       // triangle (v00, v10, v11)
  else { v.prim = 2 * quad + 1; v.b1 = u; v.b2 = w - u; }          // triangle (v00, v11, v01)
  int vv[3]; H.tri_vertices(v.prim, vv);
  v.p = H.P[vv[0]] + (H.P[vv[1]] - H.P[vv[0]]) * v.b1 + (H.P[vv[2]] - H.P[vv[0]]) * v.b2;
  return true;
}

// Reprojection of a moved vertex onto its own surface by a ray cast along the
// surface's projection direction: from the centre (spheres and caps), along
// the normal (rectangles), vertically (heightfields).  Fails when the point
// leaves the surface (cap rim, rectangle border, heightfield domain).
static bool reproject_vertex(const Scene& S, const Vtx& cur, const V3d& target, Vtx& out) {
  const Surface& sf = S.surf[cur.surf];
  out = cur;
  if (sf.type == SURF_SPHERE || sf.type == SURF_CAP) {
    V3d d = target - sf.c;
    double l = norm(d);
    if (!(l > 0.0)) return false;
    out.p = sf.c + d * (sf.r / l);
    return sf.type == SURF_SPHERE || dot(out.p - sf.c, sf.axis) >= sf.r * sf.cap_cos;
  }
  if (sf.type == SURF_RECT) {
    out.p = target - sf.axis * dot(target - sf.c, sf.axis);
    V3d q = out.p - sf.c;
    return std::fabs(dot(q, sf.ex)) <= dot(sf.ex, sf.ex) && std::fabs(dot(q, sf.ey)) <= dot(sf.ey, sf.ey);
  }
  return hf_vertical_hit(S.hf[sf.hf], target.x, target.y, out);
}

// Move every vertex by beta * (dpdu du_0 + dpdv du_1) in its tangent plane and
// reproject it onto its surface.  Visibility along the chain is not enforced
// during the walk; the admissibility test of the converged chain checks it.
static bool propose(const Scene& S, const ChainIO& ch, const Frame<double>* f, const double* du,
                    double beta, ChainIO& out) {
  out = ch;
  for (int i = 1; i <= ch.k; ++i) {
    V3d target = ch.v[i].p + (f[i].dpdu * du[2 * (i - 1)] + f[i].dpdv * du[2 * (i - 1) + 1]) * beta;
    if (!reproject_vertex(S, ch.v[i], target, out.v[i])) return false;
  }
  return true;
}

static int walk_chain(const Scene& S, ChainIO& ch, const V3d& nD, const orc_params& prm, int& iters,
                      const double* off = nullptr) {
  EvalOut ev;
  for (int it = 0;; ++it) {
    iters = it;
    eval_chain(S, ch, nD, ev, off);
    if (!ev.ok) return ST_FAILED;
    if (ev.cmax < prm.tol) return ST_CONVERGED;
    if (it >= prm.max_iter) return ST_LIMIT;
    int k = ch.k;
    double rhs[2 * MAXK], du[2 * MAXK];
    for (int i = 0; i < k; ++i) { rhs[2 * i] = -ev.vb[i].C[0]; rhs[2 * i + 1] = -ev.vb[i].C[1]; }
    if (!block_thomas<double>(k, ev.vb, 1, rhs, du, prm.sing_eps)) return ST_FAILED;
    double beta = 1.0;
    bool accepted = false;
    for (int hv = 0; hv <= prm.max_halvings; ++hv, beta *= 0.5) {
      ChainIO cand;
      if (!propose(S, ch, ev.f, du, beta, cand)) continue;
      EvalOut ec;
      eval_chain(S, cand, nD, ec, off);
      if (ec.ok && ec.cnorm2 < ev.cnorm2) {
        ch = cand;
        accepted = true;
        break;
      }
    }
    if (!accepted) return ST_FAILED;
  }
}

// ---------------------------------------------------------------------------
// Contribution: admissibility (visibility, types, orientation), generalized
// geometry term G, scattering factor kappa, T = kappa G L_o (Eq. ThroughputEval).
// ---------------------------------------------------------------------------
// Unpolarised Fresnel reflectance for light meeting an interface from the side
// of index eta1 at incidence cosine cos1 (other side eta2); 1 under total
// internal reflection.
template <class T>
T fresnel(T cos1, T eta1, T eta2) {
  using std::sqrt;
  T s2 = (eta1 / eta2) * (eta1 / eta2) * (T(1.0) - cos1 * cos1);
  if (val(s2) >= 1.0) return T(1.0);
  T cos2 = sqrt(T(1.0) - s2);
  T rs = (eta1 * cos1 - eta2 * cos2) / (eta1 * cos1 + eta2 * cos2);
  T rp = (eta2 * cos1 - eta1 * cos2) / (eta2 * cos1 + eta1 * cos2);
  return T(0.5) * (rs * rs + rp * rp);
}

// kappa: product over vertices of the mirror factor (1), the Fresnel
// reflectance (dielectric reflection) or transmittance (dielectric
// refraction).  Under an area light the refraction factor also carries the
// radiance scaling (eta_i/eta_o)^2 (light travelling from the x_{i+1} side
// into the x_{i-1} side): there G = cos(theta_D) |d(w_D)/d(u_L)| integrates
// radiance over the receiver's solid angle, and radiance over eta^2 is what
// refraction keeps.  Under a point light G = |d(w_L)/d(u_D)| maps the emitted
// intensity's solid angle onto receiver area, so E = I kappa G conserves flux
// with the transmittance alone and the radiance scaling does not enter.
template <class T>
T chain_kappa(const Scene& S, int k, uint8_t tau, const Frame<T>* f, const int* surf,
              const VBlocks<T>* vb) {
  const bool point = S.light.type == LIGHT_POINT;
  T kap(1.0);
  for (int i = 1; i <= k; ++i) {
    const Surface& sf = S.surf[surf[i]];
    if (sf.mat == MAT_MIRROR) continue;
    V3<T> wi = normalize(f[i - 1].p - f[i].p);
    T ci = fabs(dot(wi, f[i].n));
    bool refract = (tau >> (i - 1)) & 1;
    T eta1 = vb[i - 1].eta_i;
    T eta2 = T(vb[i - 1].front ? sf.etaB : sf.etaF);
    T F = fresnel(ci, eta1, eta2);
    if (refract) {
      T r = point ? T(1.0) : vb[i - 1].eta_i / vb[i - 1].eta_o;
      kap = kap * (T(1.0) - F) * r * r;
    } else {
      kap = kap * F;
    }
  }
  return kap;
}

// Generalized geometry term by the implicit function theorem.  Area light:
// G = cos(theta_D) |det d(w_D)/d(u_L)|, u_L orthonormal coordinates on the
// emitter; point light: G = |det d(w_L)/d(u_D)|, u_D orthonormal coordinates on
// the receiver (irradiance per unit intensity).  dx/du of the moving end vertex
// comes from J Y = -dC/du_end, a 2-column block Thomas solve.
template <class T>
bool chain_ggt(int k, bool point_light, const Frame<T>* f, const VBlocks<T>* vb, double sing_eps,
               T& G) {
  std::vector<T> rhs((size_t)k * 4, T(0.0)), Y((size_t)k * 4, T(0.0));
  int row = point_light ? 0 : k - 1;
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c)
      rhs[((size_t)row * 2 + r) * 2 + c] = point_light ? -vb[0].A[r][c] : -vb[k - 1].Cc[r][c];
  if (!block_thomas<T>(k, vb, 2, rhs.data(), Y.data(), sing_eps)) return false;
  int vi = point_light ? k : 1;   // vertex whose motion moves the measured direction
  const Frame<T>& fv = f[vi];
  V3<T> anchor = point_light ? f[k + 1].p : f[0].p;
  V3<T> w = fv.p - anchor;
  T dist = norm(w);
  w = w / dist;
  V3<T> a, b;
  onb(w, a, b);
  T M[2][2];
  for (int c = 0; c < 2; ++c) {
    size_t base = (size_t)(vi - 1) * 4;
    V3<T> dx = fv.dpdu * Y[base + 0 * 2 + c] + fv.dpdv * Y[base + 1 * 2 + c];
    V3<T> dw = (dx - w * dot(w, dx)) / dist;
    M[0][c] = dot(a, dw);
    M[1][c] = dot(b, dw);
  }
  T det = fabs(M[0][0] * M[1][1] - M[0][1] * M[1][0]);
  if (point_light) {
    G = det;
  } else {
    T cosD = dot(f[0].n, w);
    G = cosD * det;
  }
  return true;
}

static bool segment_clear(const Scene& S, const V3d& a, const V3d& b, double ray_eps) {
  V3d d = b - a;
  double len = norm(d);
  if (!(len > 2.0 * ray_eps)) return true;
  Hit h = intersect(S, a, d / len, ray_eps, len - ray_eps);
  return !h.hit;
}

static bool admissible_chain(const Scene& S, const ChainIO& ch, const EvalOut& ev, double ray_eps) {
  int k = ch.k;
  for (int i = 1; i <= k; ++i) {
    V3d wi = normalize(ch.v[i - 1].p - ch.v[i].p), wo = normalize(ch.v[i + 1].p - ch.v[i].p);
    double si = dot(wi, ev.f[i].n), so = dot(wo, ev.f[i].n);
    bool refract = (ch.tau >> (i - 1)) & 1;
    if (refract ? !(si * so < 0.0) : !(si * so > 0.0)) return false;
  }
  V3d wD = normalize(ch.v[1].p - ch.v[0].p);
  if (!(dot(ev.f[0].n, wD) > 0.0)) return false;
  if (S.light.type == LIGHT_RECT) {
    V3d wL = normalize(ch.v[k].p - ch.v[k + 1].p);
    if (!(dot(S.light.n, wL) > 0.0)) return false;
  }
  for (int j = 0; j <= k; ++j)
    if (!segment_clear(S, ch.v[j].p, ch.v[j + 1].p, ray_eps)) return false;
  return true;
}

// Two converged chains are one solution when they have the same length,
// types and surfaces and every vertex lies within dedup_eps.
static bool same_solution(const ChainIO& a, const ChainIO& b, double eps) {
  if (a.k != b.k || a.tau != b.tau) return false;
  for (int i = 1; i <= a.k; ++i) {
    if (a.v[i].surf != b.v[i].surf) return false;
    if (norm(a.v[i].p - b.v[i].p) >= eps) return false;
  }
  return true;
}

// ---------------------------------------------------------------------------
// Array marshalling helpers
// ---------------------------------------------------------------------------
static void load_chain(const Scene& S, int b, int k, uint8_t tau, const double* xD, const double* xL,
                       const double* x, const int32_t* surf, const int32_t* prim, const double* bary,
                       int spq, ChainIO& ch) {
  (void)S;
  ch.k = k;
  ch.tau = tau;
  int q = b / spq;
  ch.v[0] = Vtx();
  ch.v[0].p = load3(xD + 3 * (size_t)q);
  for (int i = 1; i <= k; ++i) {
    size_t o = (size_t)b * MAXK + (i - 1);
    ch.v[i].p = load3(x + 3 * o);
    ch.v[i].surf = surf[o];
    ch.v[i].prim = prim ? prim[o] : -1;
    ch.v[i].b1 = bary ? bary[2 * o] : 0.0;
    ch.v[i].b2 = bary ? bary[2 * o + 1] : 0.0;
  }
  ch.v[k + 1] = Vtx();
  ch.v[k + 1].p = load3(xL + 3 * (size_t)b);
}

static void store_chain(const ChainIO& ch, int b, double* x, int32_t* surf, int32_t* prim,
                        double* bary) {
  for (int i = 1; i <= MAXK; ++i) {
    size_t o = (size_t)b * MAXK + (i - 1);
    if (i <= ch.k) {
      store3(x + 3 * o, ch.v[i].p);
      surf[o] = ch.v[i].surf;
      if (prim) prim[o] = ch.v[i].prim;
      if (bary) { bary[2 * o] = ch.v[i].b1; bary[2 * o + 1] = ch.v[i].b2; }
    } else {
      store3(x + 3 * o, V3d());
      surf[o] = -1;
      if (prim) prim[o] = -1;
      if (bary) { bary[2 * o] = 0.0; bary[2 * o + 1] = 0.0; }
    }
  }
}

template <class F>
static void parallel_for(int n, int n_threads, F fn) {
  if (n_threads <= 1 || n < 64) {
    for (int i = 0; i < n; ++i) fn(i);
    return;
  }
  std::vector<std::thread> th;
  int per = (n + n_threads - 1) / n_threads;
  for (int t = 0; t < n_threads; ++t) {
    int lo = t * per, hi = std::min(n, lo + per);
    if (lo >= hi) break;
    th.emplace_back([=]() { for (int i = lo; i < hi; ++i) fn(i); });
  }
  for (auto& x : th) x.join();
}

static orc_params default_check(const orc_params* p) { return *p; }

// ---------------------------------------------------------------------------
// Adjoint of the receiver irradiance with respect to heightfield heights
// (implicit function theorem on the converged constraint; <1/P> held fixed).
// For a converged chain with local coordinates u (2 per vertex) and heights
// theta: C(u*, theta) = 0 defines u*(theta), so
//   dT/dtheta = dT/dtheta|_u - lambda^T dC/dtheta,   J^T lambda = (dT/du)^T.
// All partial derivatives come from forward-mode dual numbers evaluated
// through the same primitives as the walk (frames, constraint blocks, G, kappa).
// ---------------------------------------------------------------------------
static const int ADJ_LANES = 8;
typedef Dual<ADJ_LANES> DN;

// Grid vertices whose heights move vertex `prim` of heightfield H (its three
// corners and the stencils of their normals).
static void triangle_params(const HField& H, int prim, std::vector<int>& out) {
  int v[3]; H.tri_vertices(prim, v);
  for (int c = 0; c < 3; ++c) {
    int i = v[c] % H.nx, j = v[c] / H.nx;
    int cand[5][2] = {{i, j}, {i - 1, j}, {i + 1, j}, {i, j - 1}, {i, j + 1}};
    for (auto& q : cand)
      if (q[0] >= 0 && q[0] < H.nx && q[1] >= 0 && q[1] < H.ny) {
        int id = q[1] * H.nx + q[0];
        if (std::find(out.begin(), out.end(), id) == out.end()) out.push_back(id);
      }
  }
}

// Throughput and constraints of the chain at local coordinates u and heights
// theta, as dual numbers; lane l carries direction dir0 + l of the list
// [u_1 .. u_2k, theta_params[0 .. m)].
static bool chain_value_dual(const Scene& S, const ChainIO& ch, const V3d& nD, const std::vector<int>& params,
                             const std::vector<std::array<double, 4>>& Dmat, int dir0, DN* C, DN& T) {
  int k = ch.k;
  const HField* H = nullptr;
  for (int i = 1; i <= k; ++i) {
    const Surface& sf = S.surf[ch.v[i].surf];
    if (sf.type != SURF_HEIGHTFIELD) return false;
    H = &S.hf[sf.hf];
  }
  auto seed_of = [&](int dir) { int l = dir - dir0; return (l >= 0 && l < ADJ_LANES) ? l : -1; };
  auto hgt = [&](int i, int j) {
    int id = j * H->nx + i;
    DN h(H->h[(size_t)id]);
    for (size_t p = 0; p < params.size(); ++p)
      if (params[p] == id) { int l = seed_of(2 * k + (int)p); if (l >= 0) h.d[l] = 1.0; }
    return h;
  };
  Frame<DN> f[MAXK + 2];
  Frame<double> f0 = receiver_frame(ch.v[0].p, nD), fL = light_frame(S.light, ch.v[k + 1].p);
  auto liftf = [](const Frame<double>& a) {
    Frame<DN> r;
    r.p = lift<DN>(a.p); r.n = lift<DN>(a.n); r.dpdu = lift<DN>(a.dpdu); r.dpdv = lift<DN>(a.dpdv);
    r.dndu = lift<DN>(a.dndu); r.dndv = lift<DN>(a.dndv);
    return r;
  };
  f[0] = liftf(f0);
  f[k + 1] = liftf(fL);
  for (int i = 1; i <= k; ++i) {
    int v[3]; H->tri_vertices(ch.v[i].prim, v);
    V3<DN> P[3], N[3];
    for (int c = 0; c < 3; ++c) {
      int gi = v[c] % H->nx, gj = v[c] / H->nx;
      P[c] = V3<DN>(DN(H->x0 + gi * H->dx), DN(H->y0 + gj * H->dy), hgt(gi, gj));
      N[c] = hf_normal<DN>(*H, gi, gj, hgt);
    }
    DN u0(0.0), u1(0.0);
    int l0 = seed_of(2 * (i - 1)), l1 = seed_of(2 * (i - 1) + 1);
    if (l0 >= 0) u0.d[l0] = 1.0;
    if (l1 >= 0) u1.d[l1] = 1.0;
    const std::array<double, 4>& D = Dmat[i - 1];
    DN b1 = DN(ch.v[i].b1) + u0 * DN(D[0]) + u1 * DN(D[1]);
    DN b2 = DN(ch.v[i].b2) + u0 * DN(D[2]) + u1 * DN(D[3]);
    f[i] = frame_triangle<DN>(P[0], P[1], P[2], N[0], N[1], N[2], b1, b2);
  }
  int surf[MAXK + 2];
  for (int i = 0; i <= k + 1; ++i) surf[i] = ch.v[i].surf;
  VBlocks<DN> vb[MAXK];
  if (!chain_blocks<DN>(S, k, ch.tau, f, surf, vb)) return false;
  for (int i = 0; i < k; ++i) { C[2 * i] = vb[i].C[0]; C[2 * i + 1] = vb[i].C[1]; }
  DN G;
  if (!chain_ggt<DN>(k, S.light.type == LIGHT_POINT, f, vb, 0.0, G)) return false;
  DN kap = chain_kappa<DN>(S, k, ch.tau, f, surf, vb);
  T = kap * G * DN(S.light.power);
  return true;
}

// Dense solve of A x = b (n <= 16) by Gaussian elimination with partial pivoting.
static bool dense_solve(int n, std::vector<double> A, std::vector<double>& b) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r) if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (!(std::fabs(A[piv * n + c]) > 0.0)) return false;
    if (piv != c) { for (int q = 0; q < n; ++q) std::swap(A[c * n + q], A[piv * n + q]); std::swap(b[c], b[piv]); }
    for (int r = c + 1; r < n; ++r) {
      double f = A[r * n + c] / A[c * n + c];
      for (int q = c; q < n; ++q) A[r * n + q] -= f * A[c * n + q];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double v = b[r];
    for (int q = r + 1; q < n; ++q) v -= A[r * n + q] * b[q];
    b[r] = v / A[r * n + r];
  }
  return true;
}

// dT/dtheta of one converged heightfield chain; returns false if the chain is
// not a heightfield chain or its Jacobian is singular.
static bool chain_adjoint(const Scene& S, const ChainIO& ch, const V3d& nD, std::vector<int>& params,
                          std::vector<double>& dT) {
  int k = ch.k;
  const HField* H = nullptr;
  params.clear();
  std::vector<std::array<double, 4>> Dmat(k);
  for (int i = 1; i <= k; ++i) {
    const Surface& sf = S.surf[ch.v[i].surf];
    if (sf.type != SURF_HEIGHTFIELD) return false;
    H = &S.hf[sf.hf];
    triangle_params(*H, ch.v[i].prim, params);
    // map from local coordinates (along dpdu, dpdv) to barycentric increments
    Frame<double> f = vertex_frame(S, ch.v[i]);
    int v[3]; H->tri_vertices(ch.v[i].prim, v);
    V3d e1 = H->P[v[1]] - H->P[v[0]], e2 = H->P[v[2]] - H->P[v[0]];
    double g11 = dot(e1, e1), g12 = dot(e1, e2), g22 = dot(e2, e2), gd = g11 * g22 - g12 * g12;
    V3d a[2] = {f.dpdu, f.dpdv};
    for (int q = 0; q < 2; ++q) {
      double r1 = dot(e1, a[q]), r2 = dot(e2, a[q]);
      Dmat[i - 1][q] = (g22 * r1 - g12 * r2) / gd;      // db1 / du_q
      Dmat[i - 1][2 + q] = (g11 * r2 - g12 * r1) / gd;  // db2 / du_q
    }
  }
  int n = 2 * k, m = (int)params.size(), nd = n + m;
  std::vector<double> dC((size_t)n * nd), dTd(nd);
  for (int d0 = 0; d0 < nd; d0 += ADJ_LANES) {
    DN C[2 * MAXK], T;
    if (!chain_value_dual(S, ch, nD, params, Dmat, d0, C, T)) return false;
    for (int l = 0; l < ADJ_LANES && d0 + l < nd; ++l) {
      for (int r = 0; r < n; ++r) dC[(size_t)r * nd + d0 + l] = C[r].d[l];
      dTd[d0 + l] = T.d[l];
    }
  }
  // J^T lambda = dT/du
  std::vector<double> JT((size_t)n * n), lam(n);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) JT[(size_t)r * n + c] = dC[(size_t)c * nd + r];
  for (int r = 0; r < n; ++r) lam[r] = dTd[r];
  if (!dense_solve(n, JT, lam)) return false;
  dT.assign(m, 0.0);
  for (int p = 0; p < m; ++p) {
    double v = dTd[n + p];
    for (int r = 0; r < n; ++r) v -= lam[r] * dC[(size_t)r * nd + n + p];
    dT[p] = v;
  }
  return true;
}

}  // namespace orc

using namespace orc;

// ---------------------------------------------------------------------------
// Glossy chains (Sec. 5.7): offset normals.  Every vertex of a glossy chain
// is a rough interface with an isotropic Beckmann microfacet distribution of
// roughness alpha.  An offset normal m_i is drawn per vertex before the walk;
// its tangential components o_i = (m_i.s, m_i.t) in the vertex's shading frame
// are the constraint's targets (C_i = o_i), and the walk then finds the
// chains whose half-vectors are the drawn normals, as in the specular case.
// The estimate of one found chain is the path integrand in area measure over
// the density of the offsets in the constraint's coordinates:
//   W = L_e prod_i [f_i |n_i.l_i|] prod_j [geometric factors]
//       / (|det dC/du| prod_i p(o_i)),
// dC/du the 2k x 2k Jacobian in orthonormal area coordinates of the surfaces,
// f_i the microfacet BSDF (Walter et al. 2007: reflection
// F D G2 / (4 |l.n||v.n|); transmission |l.m||v.m| / (|l.n||v.n|) *
// eta_v^2 (1 - F) D G2 / (eta_l l.m + eta_v v.m)^2), l toward the light and
// v toward the receiver, G2 the separable Smith term.  Drawing m with density
// D(m) (m.n) in solid angle gives o the density D(m) on the unit disk, since
// the disk's area element is (m.n) times the solid angle.
// ---------------------------------------------------------------------------
static double beckmann_D(double cos_m, double alpha) {
  if (!(cos_m > 0.0)) return 0.0;
  double c2 = cos_m * cos_m, t2 = (1.0 - c2) / c2;
  return std::exp(-t2 / (alpha * alpha)) / (PI * alpha * alpha * c2 * c2);
}

// Smith masking of one direction with cosine c to the macro normal and
// cosine cm to the microfacet normal (Beckmann, exact Lambda with erf).
static double smith_G1(double c, double cm, double alpha) {
  if (!(c * cm > 0.0)) return 0.0;
  double ac = std::fabs(c);
  if (ac >= 1.0) return 1.0;
  double tan_t = std::sqrt(1.0 - ac * ac) / ac;
  double a = 1.0 / (alpha * tan_t);
  double lambda = 0.5 * (std::erf(a) - 1.0) + std::exp(-a * a) / (2.0 * a * std::sqrt(PI));
  return 1.0 / (1.0 + lambda);
}

// Offset (tangential components) of a normal drawn with density D(m) (m.n):
// tan^2(theta) = -alpha^2 log(1 - u1), phi = 2 pi u2.
static void beckmann_offset(double alpha, double u1, double u2, double o[2]) {
  double t2 = -alpha * alpha * std::log(1.0 - u1);
  double c = 1.0 / std::sqrt(1.0 + t2), s = std::sqrt(t2) * c;
  double phi = 2.0 * PI * u2;
  o[0] = s * std::cos(phi);
  o[1] = s * std::sin(phi);
}

// Determinant of a dense n x n matrix by Gaussian elimination with partial
// pivoting (a different route from the block Thomas sweep).
static double dense_det(int n, std::vector<double> A) {
  double det = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r) if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return 0.0;
    if (piv != c) {
      for (int q = 0; q < n; ++q) std::swap(A[c * n + q], A[piv * n + q]);
      det = -det;
    }
    det *= A[c * n + c];
    for (int r = c + 1; r < n; ++r) {
      double f = A[r * n + c] / A[c * n + c];
      for (int q = c; q < n; ++q) A[r * n + q] -= f * A[c * n + q];
    }
  }
  return det;
}

struct GlossyTerms {
  double detJ = 0.0;    // |det dC/du|
  double bsdf = 1.0;    // prod_i f_i |n_i.l_i| / D(m_i)  (the BSDF's D divided out)
  double geom = 1.0;    // receiver cosine, area-measure factors, light factor
  double dens = 1.0;    // prod_i D(m_i): the offsets' density on the disk
  double W = 0.0;       // the estimate L_e bsdf geom / detJ (D cancels against dens)
};

// Terms of one converged glossy chain (alpha > 0) or, with alpha = 0, of the
// specular limit (D and G2 dropped: the terms then reproduce kappa G).
static bool glossy_terms(const Scene& S, const ChainIO& ch, const EvalOut& ev, double alpha, GlossyTerms& gt) {
  const int k = ch.k;
  std::vector<double> J((size_t)4 * k * k, 0.0);
  for (int i = 0; i < k; ++i)
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 2; ++c) {
        J[(size_t)(2 * i + r) * 2 * k + 2 * i + c] = ev.vb[i].B[r][c];
        if (i > 0) J[(size_t)(2 * i + r) * 2 * k + 2 * (i - 1) + c] = ev.vb[i].A[r][c];
        if (i < k - 1) J[(size_t)(2 * i + r) * 2 * k + 2 * (i + 1) + c] = ev.vb[i].Cc[r][c];
      }
  gt.detJ = std::fabs(dense_det(2 * k, J));
  if (!(gt.detJ > 0.0)) return false;
  gt.bsdf = gt.geom = gt.dens = 1.0;
  for (int i = 1; i <= k; ++i) {
    const Surface& sf = S.surf[ch.v[i].surf];
    const Frame<double>& f = ev.f[i];
    const VBlocks<double>& vb = ev.vb[i - 1];
    V3d v = normalize(ch.v[i - 1].p - f.p), l = normalize(ch.v[i + 1].p - f.p);
    double cv = dot(v, f.n), cl = dot(l, f.n);
    bool refract = (ch.tau >> (i - 1)) & 1;
    double ev_ = vb.eta_i, el = vb.eta_o;  // indices on the receiver and light sides
    V3d m = normalize(v * ev_ + l * el);
    if (dot(m, f.n) < 0.0) m = -m;
    double vm = dot(v, m), lm = dot(l, m), mn = dot(m, f.n);
    double F = 1.0;
    if (sf.mat != MAT_MIRROR) {
      double e2 = vb.front ? sf.etaB : sf.etaF;
      F = fresnel<double>(std::fabs(vm), ev_, e2);
    }
    double G2 = alpha > 0.0 ? smith_G1(cv, vm, alpha) * smith_G1(cl, lm, alpha) : 1.0;
    double fhat;  // f_i / D(m_i)
    if (refract) {
      double den = ev_ * vm + el * lm;
      fhat = std::fabs(lm) * std::fabs(vm) / (std::fabs(cl) * std::fabs(cv)) * ev_ * ev_ * (1.0 - F) * G2 /
             (den * den);
    } else {
      fhat = F * G2 / (4.0 * std::fabs(cl) * std::fabs(cv));
    }
    gt.bsdf *= fhat * std::fabs(cl);
    if (alpha > 0.0) gt.dens *= beckmann_D(mn, alpha);
    // area measure at x_i: |cos| to the surface's geometric normal over d^2
    V3d ng = normalize(cross(f.dpdu, f.dpdv));
    double d = norm(ch.v[i - 1].p - f.p);
    gt.geom *= std::fabs(dot(ng, v)) / (d * d);
  }
  V3d w0 = normalize(ch.v[1].p - ch.v[0].p);
  gt.geom *= std::fabs(dot(ev.f[0].n, w0));
  double dL = norm(ch.v[k + 1].p - ch.v[k].p);
  V3d wL = (ch.v[k].p - ch.v[k + 1].p) / dL;
  gt.geom *= (S.light.type == LIGHT_POINT ? 1.0 : std::fabs(dot(S.light.n, wL))) / (dL * dL);
  gt.W = S.light.power * gt.bsdf * gt.geom / gt.detJ;
  return true;
}

extern "C" {

void* orc_scene_create(const double* surfaces, int32_t n_surf, const double* hf_desc,
                       const double* hf_heights, int32_t n_hf, const double* targets,
                       int32_t n_targets, const double* light) {
  if (n_surf < 0 || n_hf < 0 || n_targets < 0 || !light) return nullptr;
  Scene* S = new Scene();
  size_t hoff = 0;
  for (int h = 0; h < n_hf; ++h) {
    HField H;
    const double* d = hf_desc + 6 * h;
    H.nx = (int)d[0]; H.ny = (int)d[1];
    H.x0 = d[2]; H.y0 = d[3]; H.x1 = d[4]; H.y1 = d[5];
    H.surf = -1;
    if (H.nx < 2 || H.ny < 2) { delete S; return nullptr; }
    H.h.assign(hf_heights + hoff, hf_heights + hoff + (size_t)H.nx * H.ny);
    hoff += (size_t)H.nx * H.ny;
    hf_build(H);
    S->hf.push_back(std::move(H));
  }
  for (int s = 0; s < n_surf; ++s) {
    const double* r = surfaces + 24 * s;
    Surface sf;
    sf.type = (int)r[0]; sf.mat = (int)r[1]; sf.etaF = r[2]; sf.etaB = r[3];
    sf.c = load3(r + 4); sf.r = r[7]; sf.axis = load3(r + 8); sf.cap_cos = r[11];
    sf.ex = load3(r + 12); sf.ey = load3(r + 15); sf.hf = (int)r[18];
    if (sf.type == SURF_RECT) sf.axis = normalize(sf.axis);
    if (sf.type == SURF_HEIGHTFIELD) {
      if (sf.hf < 0 || sf.hf >= n_hf) { delete S; return nullptr; }
      S->hf[sf.hf].surf = s;
    }
    S->surf.push_back(sf);
  }
  for (int t = 0; t < n_targets; ++t) {
    const double* r = targets + 16 * t;
    Target tg;
    tg.type = (int)r[0]; tg.c = load3(r + 1); tg.r = r[4]; tg.ex = load3(r + 5);
    tg.ey = load3(r + 8); tg.n = load3(r + 11);
    if (tg.type == TARGET_RECT) tg.n = normalize(tg.n);
    S->tg.push_back(tg);
  }
  Light& L = S->light;
  L.type = (int)light[0]; L.p = load3(light + 1); L.n = normalize(load3(light + 4));
  L.ex = load3(light + 7); L.ey = load3(light + 10); L.power = light[13];
  L.area = L.type == LIGHT_RECT ? 4.0 * norm(L.ex) * norm(L.ey) : 1.0;
  return S;
}

void orc_scene_destroy(void* scene) { delete (Scene*)scene; }

int32_t orc_intersect(void* scene, int32_t n, const double* o, const double* d, double tmin,
                      double tmax, int32_t brute, double* t, int32_t* surf, int32_t* prim,
                      double* bary) {
  if (!scene || n < 0) return -1;
  const Scene& S = *(Scene*)scene;
  for (int i = 0; i < n; ++i) {
    Hit h = intersect(S, load3(o + 3 * i), normalize(load3(d + 3 * i)), tmin, tmax, brute != 0);
    t[i] = h.hit ? h.t : -1.0;
    surf[i] = h.surf;
    prim[i] = h.prim;
    bary[2 * i] = h.b1;
    bary[2 * i + 1] = h.b2;
  }
  return 0;
}

int32_t orc_sample_seeds(void* scene, const orc_guide* guide, int32_t Q, const double* xD,
                         const double* nD, const uint32_t* cell, int32_t spq, const double* xL,
                         const uint8_t* k, const uint8_t* tau, int32_t tau_random,
                         uint64_t rng_seed, uint64_t rng_offset, uint32_t trial,
                         const orc_params* prm, double* x, int32_t* surf, int32_t* prim,
                         double* bary, uint8_t* tau_out, double* pdf, uint8_t* valid,
                         int32_t n_threads, const uint32_t* chain_cell) {
  if (!scene || !prm || Q < 0 || spq <= 0) return -1;
  const Scene& S = *(Scene*)scene;
  orc_params P = default_check(prm);
  GuideCDF cdf;
  bool g_ok = guide && (guide->counts || guide->vmf);
  if (g_ok && !guide->vmf) guide_cdf(*guide, cdf);
  int B = Q * spq;
  auto cell_of = [&](int b) { return chain_cell ? chain_cell[b] : (cell ? cell[b / spq] : 0u); };
  if (g_ok && guide->vmf)
    for (int b = 0; b < B; ++b)
      if ((int)cell_of(b) >= guide->vmf->n_cells) return -3;
  for (int b = 0; b < B; ++b)
    if (k[b] < 1 || k[b] > MAXK) return -2;
  parallel_for(B, n_threads, [&](int b) {
    int q = b / spq;
    SeedDraw sd = sample_seed(S, g_ok ? guide : nullptr, g_ok ? &cdf : nullptr, load3(xD + 3 * (size_t)q),
                              load3(nD + 3 * (size_t)q), cell_of(b), load3(xL + 3 * (size_t)b),
                              k[b], tau[b], tau_random != 0, rng_seed, (uint64_t)b + rng_offset, trial, P);
    valid[b] = sd.valid ? 1 : 0;
    pdf[b] = sd.valid ? sd.pdf : 0.0;
    tau_out[b] = sd.tau;
    if (!sd.valid) { sd.ch.k = 0; }
    store_chain(sd.ch, b, x, surf, prim, bary);
  });
  return 0;
}

int32_t orc_walk(void* scene, int32_t B, int32_t spq, const double* xD, const double* nD,
                 const double* xL, const uint8_t* k, const uint8_t* tau, const orc_params* prm,
                 const uint8_t* valid, double* x, int32_t* surf, int32_t* prim, double* bary,
                 uint8_t* status, uint8_t* iters, int32_t n_threads, const double* offset) {
  if (!scene || !prm || B < 0 || spq <= 0) return -1;
  const Scene& S = *(Scene*)scene;
  orc_params P = *prm;
  parallel_for(B, n_threads, [&](int b) {
    if (!valid[b] || k[b] < 1 || k[b] > MAXK) { status[b] = ST_INVALID; iters[b] = 0; return; }
    ChainIO ch;
    load_chain(S, b, k[b], tau[b], xD, xL, x, surf, prim, bary, spq, ch);
    int it = 0;
    int st = walk_chain(S, ch, load3(nD + 3 * (size_t)(b / spq)), P, it,
                        offset ? offset + (size_t)b * 2 * MAXK : nullptr);
    status[b] = (uint8_t)st;
    iters[b] = (uint8_t)it;
    store_chain(ch, b, x, surf, prim, bary);
  });
  return 0;
}

int32_t orc_contribution(void* scene, int32_t B, int32_t spq, const double* xD,
                         const double* nD, const double* xL, const uint8_t* k,
                         const uint8_t* tau, const double* x, const int32_t* surf,
                         const int32_t* prim, const double* bary, const uint8_t* status,
                         const orc_params* prm, double* G, double* kappa, double* T,
                         uint8_t* admissible, int32_t n_threads) {
  if (!scene || !prm || B < 0 || spq <= 0) return -1;
  const Scene& S = *(Scene*)scene;
  parallel_for(B, n_threads, [&](int b) {
    G[b] = kappa[b] = T[b] = 0.0;
    admissible[b] = 0;
    if (status[b] != ST_CONVERGED) return;
    ChainIO ch;
    load_chain(S, b, k[b], tau[b], xD, xL, x, surf, prim, bary, spq, ch);
    EvalOut ev;
    eval_chain(S, ch, load3(nD + 3 * (size_t)(b / spq)), ev);
    if (!ev.ok || !admissible_chain(S, ch, ev, prm->ray_eps)) return;
    int sid[MAXK + 2];
    for (int i = 0; i <= ch.k + 1; ++i) sid[i] = ch.v[i].surf;
    double g;
    if (!chain_ggt<double>(ch.k, S.light.type == LIGHT_POINT, ev.f, ev.vb, prm->sing_eps, g)) return;
    double kap = chain_kappa<double>(S, ch.k, ch.tau, ev.f, sid, ev.vb);
    admissible[b] = 1;
    G[b] = g;
    kappa[b] = kap;
    T[b] = kap * g * S.light.power;
  });
  return 0;
}

int32_t orc_bernoulli(void* scene, const orc_guide* guide, int32_t Q, const double* xD,
                      const double* nD, const uint32_t* cell, int32_t spq, const double* xL,
                      const uint8_t* k, const uint8_t* tau, int32_t tau_random,
                      uint64_t rng_seed, uint64_t rng_offset, const orc_params* prm,
                      const double* x, const int32_t* surf, const uint8_t* admissible,
                      uint32_t* N, uint8_t* capped, uint32_t* trial_walks, int32_t n_threads,
                      const uint32_t* chain_cell, const double* offset) {
  if (!scene || !prm || Q < 0 || spq <= 0) return -1;
  const Scene& S = *(Scene*)scene;
  orc_params P = *prm;
  GuideCDF cdf;
  bool g_ok = guide && (guide->counts || guide->vmf);
  if (g_ok && !guide->vmf) guide_cdf(*guide, cdf);
  int B = Q * spq;
  auto cell_of = [&](int b) { return chain_cell ? chain_cell[b] : (cell ? cell[b / spq] : 0u); };
  if (g_ok && guide->vmf)
    for (int b = 0; b < B; ++b)
      if ((int)cell_of(b) >= guide->vmf->n_cells) return -3;
  parallel_for(B, n_threads, [&](int b) {
    N[b] = 0;
    capped[b] = 0;
    if (trial_walks) trial_walks[b] = 0;
    if (!admissible[b]) return;
    int q = b / spq;
    ChainIO target;
    load_chain(S, b, k[b], tau[b], xD, xL, x, surf, nullptr, nullptr, spq, target);
    V3d xd = load3(xD + 3 * (size_t)q), nd = load3(nD + 3 * (size_t)q), xl = load3(xL + 3 * (size_t)b);
    const int repeats = P.bern_repeats > 1 ? P.bern_repeats : 1;
    for (int rep = 0; rep < repeats; ++rep) {
      bool hit = false;
      for (int t = 1; t <= P.max_trials && !hit; ++t) {
        SeedDraw sd = sample_seed(S, g_ok ? guide : nullptr, g_ok ? &cdf : nullptr, xd, nd,
                                  cell_of(b), xl, k[b], tau[b], tau_random != 0, rng_seed,
                                  (uint64_t)b + rng_offset, (uint32_t)t | ((uint32_t)rep << 24), P);
        if (!sd.valid) continue;
        int it = 0;
        if (walk_chain(S, sd.ch, nd, P, it, offset ? offset + (size_t)b * 2 * MAXK : nullptr) != ST_CONVERGED)
          continue;
        if (trial_walks) trial_walks[b]++;
        if (same_solution(sd.ch, target, P.dedup_eps)) {
          N[b] += (uint32_t)t;
          hit = true;
        }
      }
      if (!hit) {
        N[b] += (uint32_t)P.max_trials;
        capped[b] = 1;
      }
    }
  });
  return 0;
}

int32_t orc_vmf_build(int32_t n_cells, int32_t R, const uint32_t* cell, const float* omega,
                      const float* w, const uint8_t* k, const uint8_t* tau, int32_t weight_shift,
                      uint32_t* cell_start, uint32_t* key, double* lobe, uint64_t* prefix) {
  if (n_cells <= 0 || R < 0 || !cell_start) return -1;
  for (int r = 0; r < R; ++r) {
    if ((int64_t)cell[r] >= n_cells || k[r] < 1 || k[r] > MAXK || tau[r] >= (1u << k[r])) return -2;
  }
  // order: cell, then key (n, tau), then record index
  std::vector<int> ord(R);
  for (int r = 0; r < R; ++r) ord[r] = r;
  auto rkey = [&](int r) { return ((uint32_t)k[r] << 8) | tau[r]; };
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
    if (cell[a] != cell[b]) return cell[a] < cell[b];
    return rkey(a) < rkey(b);
  });
  for (int c = 0; c <= n_cells; ++c) cell_start[c] = 0;
  for (int r = 0; r < R; ++r) cell_start[cell[r] + 1]++;
  for (int c = 0; c < n_cells; ++c) cell_start[c + 1] += cell_start[c];
  for (int i = 0; i < R; ++i) {
    int r = ord[i];
    key[i] = rkey(r);
    for (int j = 0; j < 3; ++j) lobe[4 * (size_t)i + j] = (double)omega[3 * (size_t)r + j];
  }
  // kappa_i = sigma_i^-2, sigma_i the angle to the nearest other direction
  // of the same group (same cell and key; groups are contiguous)
  for (int i = 0; i < R; ++i) {
    uint32_t ci = cell[ord[i]];
    int g0 = i, g1 = i + 1;
    while (g0 > 0 && cell[ord[g0 - 1]] == ci && key[g0 - 1] == key[i]) --g0;
    while (g1 < R && cell[ord[g1]] == ci && key[g1] == key[i]) ++g1;
    V3d mi(lobe[4 * (size_t)i], lobe[4 * (size_t)i + 1], lobe[4 * (size_t)i + 2]);
    double sigma = PI;
    if (g1 - g0 > 1) {
      double best = std::numeric_limits<double>::infinity();
      for (int j = g0; j < g1; ++j) {
        if (j == i) continue;
        V3d d = mi - V3d(lobe[4 * (size_t)j], lobe[4 * (size_t)j + 1], lobe[4 * (size_t)j + 2]);
        best = std::min(best, dot(d, d));
      }
      sigma = 2.0 * std::asin(std::min(1.0, 0.5 * std::sqrt(best)));  // chord -> angle
    }
    sigma = std::max(sigma, VMF_SIGMA_MIN);
    lobe[4 * (size_t)i + 3] = 1.0 / (sigma * sigma);
  }
  // prefix sums of the quantised weights within each cell
  for (int c = 0; c < n_cells; ++c) {
    uint64_t acc = 0;
    for (uint32_t i = cell_start[c]; i < cell_start[c + 1]; ++i) {
      acc += quantise_weight(w[ord[i]], weight_shift);
      prefix[i] = acc;
    }
  }
  return 0;
}

int32_t orc_sample_lengths(const orc_guide* guide, int32_t Q, const uint32_t* cell, int32_t spq,
                           const uint32_t* p0w, uint64_t rng_seed, uint64_t rng_offset,
                           const orc_params* prm, uint8_t* k_out, double* pn_out, const uint32_t* chain_cell) {
  if (Q < 0 || spq <= 0 || !p0w || !prm) return -1;
  uint64_t W0 = 0;
  for (int n = 1; n <= MAXK; ++n) W0 += p0w[n - 1];
  if (W0 == 0) return -2;
  const orc_vmf* vm = guide ? guide->vmf : nullptr;
  uint32_t key[2] = {(uint32_t)rng_seed, (uint32_t)(rng_seed >> 32)};
  for (size_t b = 0; b < (size_t)Q * spq; ++b) {
    uint32_t c = chain_cell ? chain_cell[b] : (cell ? cell[b / spq] : 0u);
    if (vm && (int)c >= vm->n_cells) return -3;
    // W(n) of the chain's cell, n = 1..8
    uint64_t We[MAXK + 1] = {0}, Wc = 0;
    if (vm) {
      for (int n = 1; n <= MAXK; ++n) {
        We[n] = lobe_range(*vm, c, (uint32_t)n << 8, (uint32_t)(n + 1) << 8).total;
        Wc += We[n];
      }
    }
    uint64_t idx = (uint64_t)b + rng_offset;
    uint32_t ctr[4] = {(uint32_t)idx, (uint32_t)(idx >> 32), 0u, 2u}, r[4];
    philox4x32_10(ctr, key, r);
    bool pick_p0 = Wc == 0 || u01(r[0]) < prm->alpha;
    const uint64_t* Wt = pick_p0 ? nullptr : We;
    uint64_t total = pick_p0 ? W0 : Wc;
    uint64_t target = scaled_target(r[1], total);
    int n = 1;
    uint64_t acc = 0;
    for (; n <= MAXK; ++n) {
      acc += Wt ? Wt[n] : p0w[n - 1];
      if (acc > target) break;
    }
    n = std::min(n, MAXK);
    double P0 = (double)p0w[n - 1] / (double)W0;
    k_out[b] = (uint8_t)n;
    pn_out[b] = Wc == 0 ? P0 : prm->alpha * P0 + (1.0 - prm->alpha) * (double)We[n] / (double)Wc;
  }
  return 0;
}

double orc_vmf_pdf(const double* mu, double kappa, const double* w) {
  return vmf_pdf(load3(mu), kappa, load3(w));
}

void orc_vmf_sample(const double* mu, double kappa, double u1, double u2, double* w) {
  store3(w, vmf_sample(load3(mu), kappa, u1, u2));
}

int32_t orc_guide_bin(const orc_guide* guide, int32_t R, const float* omega, int32_t* bin) {
  if (!guide || R < 0) return -1;
  for (int r = 0; r < R; ++r) bin[r] = guide_bin(*guide, omega + 3 * (size_t)r);
  return 0;
}

int32_t orc_guide_update(const orc_guide* guide, uint64_t* counts, int32_t R,
                         const uint32_t* cell, const float* omega, const float* w,
                         int32_t weight_shift) {
  if (!guide || !counts || R < 0) return -1;
  int bins = guide->n_theta * guide->n_phi;
  for (int r = 0; r < R; ++r) {
    if ((int)cell[r] >= guide->n_cells) return -2;
    int b = guide_bin(*guide, omega + 3 * (size_t)r);
    counts[(size_t)cell[r] * bins + b] += quantise_weight(w[r], weight_shift);
  }
  return 0;
}

int32_t orc_constraint(void* scene, int32_t B, int32_t spq, const double* xD, const double* nD,
                       const double* xL, const uint8_t* k, const uint8_t* tau,
                       const double* x, const int32_t* surf, const int32_t* prim,
                       const double* bary, double* C, double* cmax) {
  if (!scene || B < 0 || spq <= 0) return -1;
  const Scene& S = *(Scene*)scene;
  for (int b = 0; b < B; ++b) {
    for (int i = 0; i < 2 * MAXK; ++i) C[(size_t)b * 2 * MAXK + i] = 0.0;
    cmax[b] = -1.0;
    bool ok = k[b] >= 1 && k[b] <= MAXK;
    for (int i = 0; ok && i < k[b]; ++i) {
      int s = surf[(size_t)b * MAXK + i];
      ok = s >= 0 && s < (int)S.surf.size();
    }
    if (!ok) continue;  // chain without vertices (invalid seed)
    ChainIO ch;
    load_chain(S, b, k[b], tau[b], xD, xL, x, surf, prim, bary, spq, ch);
    EvalOut ev;
    eval_chain(S, ch, load3(nD + 3 * (size_t)(b / spq)), ev);
    if (!ev.ok) { cmax[b] = -1.0; continue; }
    for (int i = 0; i < ch.k; ++i) {
      C[(size_t)b * 2 * MAXK + 2 * i] = ev.vb[i].C[0];
      C[(size_t)b * 2 * MAXK + 2 * i + 1] = ev.vb[i].C[1];
    }
    cmax[b] = ev.cmax;
  }
  return 0;
}

int32_t orc_shoot(void* scene, const double* xD, const double* omega, int32_t k, uint8_t tau,
                  double ray_eps, double* x, double* exit_dir) {
  if (!scene || k < 1 || k > MAXK) return -1;
  const Scene& S = *(Scene*)scene;
  V3d o = load3(xD), d = normalize(load3(omega));
  for (int i = 1; i <= k; ++i) {
    Hit h = intersect(S, o, d, ray_eps, std::numeric_limits<double>::infinity());
    if (!h.hit) return -2;
    Vtx v = hit_vertex(S, o, d, h);
    store3(x + 3 * (i - 1), v.p);
    Frame<double> f = vertex_frame(S, v);
    V3d dn;
    if (!scatter(S.surf[h.surf], f.n, d, (tau >> (i - 1)) & 1, dn)) return -3;
    o = v.p;
    d = dn;
  }
  store3(exit_dir, d);
  return 0;
}

int32_t orc_adjoint(void* scene, int32_t B, int32_t spq, const double* xD, const double* nD, const double* xL,
                    const uint8_t* k, const uint8_t* tau, const double* x, const int32_t* surf,
                    const int32_t* prim, const double* bary, const double* weight, double* dL_dtheta,
                    double* dT_out, int32_t n_threads) {
  if (!scene || B < 0 || spq <= 0) return -1;
  const Scene& S = *(Scene*)scene;
  if (S.hf.empty()) return -2;
  std::vector<std::vector<int>> P(B);
  std::vector<std::vector<double>> D(B);
  std::vector<uint8_t> ok(B, 0);
  parallel_for(B, n_threads, [&](int b) {
    if (weight[b] == 0.0) return;
    ChainIO ch;
    load_chain(S, b, k[b], tau[b], xD, xL, x, surf, prim, bary, spq, ch);
    ok[b] = chain_adjoint(S, ch, load3(nD + 3 * (size_t)(b / spq)), P[b], D[b]) ? 1 : 0;
  });
  for (int b = 0; b < B; ++b) {
    if (dT_out) dT_out[b] = ok[b] ? 1.0 : 0.0;
    if (!ok[b]) continue;
    for (size_t p = 0; p < P[b].size(); ++p) dL_dtheta[P[b][p]] += weight[b] * D[b][p];
  }
  return 0;
}

void orc_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  philox4x32_10(ctr, key, out);
}

static double tally_flops(const Tally& t) { return (double)(t.add + t.mul + t.div + t.sqrt); }

// Floating-point operations (add, mul, div, sqrt: one flop each) of one
// execution of each primitive, counted with the Counted scalar type on a
// representative configuration.  out[]: 0 sphere frame, 1 plane frame,
// 2 triangle frame, 3 sphere normal, 4 triangle normal, 5 vertex blocks (C and
// the three Jacobian blocks), 6 vertex constraint only, 7 Thomas first row,
// 8 Thomas further row (1 column), 9 geometry-term Thomas row (2 columns),
// 10 geometry-term projection and determinant, 11 ray/sphere roots,
// 12 ray/rectangle test, 13 ray/triangle test, 14 ray/box slab test,
// 15 kappa per dielectric vertex.
int32_t orc_unit_flops(double* out) {
  typedef Counted C;
  auto run = [](auto fn) { g_tally = Tally(); fn(); return tally_flops(g_tally); };
  V3<C> p(0.3, -0.4, 0.86602540378), c(0.0, 0.0, 0.0);
  out[0] = run([&] { frame_sphere<C>(p, c, C(1.0)); });
  out[1] = run([&] { frame_plane<C>(p, V3<C>(0.0, 0.0, 1.0)); });
  V3<C> P0(0.0, 0.0, 0.01), P1(0.02, 0.0, 0.012), P2(0.02, 0.02, 0.008);
  V3<C> N0(0.01, 0.02, 0.9997), N1(-0.01, 0.0, 0.99995), N2(0.0, -0.02, 0.9998);
  out[2] = run([&] { frame_triangle<C>(P0, P1, P2, N0, N1, N2, C(0.3), C(0.2)); });
  out[3] = run([&] { normalize(p - c); });
  out[4] = run([&] { normalize(N0 * (C(1.0) - C(0.3) - C(0.2)) + N1 * C(0.3) + N2 * C(0.2)); });
  Surface sf;
  sf.type = SURF_SPHERE; sf.mat = MAT_DIELECTRIC; sf.etaF = 1.0; sf.etaB = 1.5; sf.hf = -1;
  sf.r = 1.0; sf.cap_cos = -1.0;
  Frame<C> fp = frame_plane<C>(V3<C>(0.1, 0.2, -1.5), V3<C>(0.0, 0.0, 1.0));
  Frame<C> f = frame_sphere<C>(normalize(V3<C>(0.1, 0.1, -1.0)), c, C(1.0));
  Frame<C> fn = frame_sphere<C>(normalize(V3<C>(0.0, -0.2, 1.0)), c, C(1.0));
  VBlocks<C> vb;
  out[5] = run([&] { vertex_blocks<C>(fp, f, fn, sf, true, vb); });
  out[6] = run([&] { vertex_blocks<C>(fp, f, fn, sf, true, vb, true); });
  VBlocks<C> v8[8];
  for (int i = 0; i < 8; ++i) vertex_blocks<C>(fp, f, fn, sf, true, v8[i]);
  C rhs[32], x[32];
  for (int i = 0; i < 32; ++i) rhs[i] = C(0.01 * (i + 1));
  double t1 = run([&] { block_thomas<C>(1, v8, 1, rhs, x, 0.0); });
  double t8 = run([&] { block_thomas<C>(8, v8, 1, rhs, x, 0.0); });
  out[7] = t1;
  out[8] = (t8 - t1) / 7.0;
  double g1 = run([&] { block_thomas<C>(1, v8, 2, rhs, x, 0.0); });
  double g8 = run([&] { block_thomas<C>(8, v8, 2, rhs, x, 0.0); });
  out[9] = (g8 - g1) / 7.0;
  Frame<C> ff[3] = {fp, f, fn};
  double gg = run([&] { C G; chain_ggt<C>(1, false, ff, v8, 0.0, G); });
  out[10] = gg - g1;
  // The ray tests take a unit direction as input: it is normalised once per
  // ray (or is unit by construction), outside the counted test.
  C r0[2];
  const V3<C> d_sph = normalize(V3<C>(0.0, 0.1, 1.0)), d_tri = normalize(V3<C>(0.0, 0.0, 1.0));
  out[11] = run([&] { sphere_roots<C>(V3<C>(0.1, 0.2, -1.5), d_sph, c, C(1.0), r0); });
  out[12] = run([&] {  // plane t, hit point and two in-rectangle projections
    V3<C> o(0.1, 0.2, 1.0), d(0.0, 0.1, -1.0), n(0.0, 0.0, 1.0), ex(1.0, 0.0, 0.0), ey(0.0, 1.0, 0.0);
    C t = dot(c - o, n) / dot(d, n);
    V3<C> q = o + d * t - c;
    dot(q, ex); dot(q, ey); dot(ex, ex); dot(ey, ey);
  });
  C tt, bb1, bb2;
  out[13] = run([&] { tri_hit<C>(V3<C>(0.01, 0.005, -1.0), d_tri, P0, P1, P2, tt, bb1, bb2); });
  out[14] = 12.0;  // 6 subtractions and 6 divisions (or reciprocal products) of the slab test
  out[15] = run([&] {
    V3<C> wi = normalize(fp.p - f.p);
    C ci = fabs(dot(wi, f.n));
    C F = fresnel<C>(ci, C(1.0), C(1.5));
    C r = C(1.0) / C(1.5);
    C k = (C(1.0) - F) * r * r;
    (void)k;
  });
  return 0;
}



// Offset normals of glossy chains: for chain b (global index b + rng_offset)
// and vertex i < k[b], one Philox block with counter (index, i, 4) gives the
// two uniforms of the Beckmann draw; vertices i >= k[b] get zero offsets.
int32_t orc_sample_offsets(int32_t B, const uint8_t* k, double alpha, uint64_t rng_seed, uint64_t rng_offset,
                           double* offset) {
  if (B < 0 || !(alpha > 0.0)) return -1;
  uint32_t key[2] = {(uint32_t)rng_seed, (uint32_t)(rng_seed >> 32)};
  for (int b = 0; b < B; ++b) {
    uint64_t idx = (uint64_t)b + rng_offset;
    for (int i = 0; i < MAXK; ++i) {
      double* o = offset + ((size_t)b * MAXK + i) * 2;
      o[0] = o[1] = 0.0;
      if (i >= k[b]) continue;
      uint32_t ctr[4] = {(uint32_t)idx, (uint32_t)(idx >> 32), (uint32_t)i, 4u}, r[4];
      philox4x32_10(ctr, key, r);
      beckmann_offset(alpha, u01(r[0]), u01(r[1]), o);
    }
  }
  return 0;
}

// Terms of converged glossy chains: out [B][5] = |det dC/du|, the BSDF
// product with D divided out, the geometric factors, the offsets' density and
// the estimate W; admissible[b] as for orc_contribution.  alpha = 0 gives the
// specular limit.
int32_t orc_glossy(void* scene, int32_t B, int32_t spq, const double* xD, const double* nD, const double* xL,
                   const uint8_t* k, const uint8_t* tau, const double* x, const int32_t* surf, const int32_t* prim,
                   const double* bary, const uint8_t* status, const orc_params* prm, const double* offset,
                   double alpha, double* out, uint8_t* admissible, int32_t n_threads) {
  if (!scene || !prm || B < 0 || spq <= 0 || !(alpha >= 0.0)) return -1;
  const Scene& S = *(Scene*)scene;
  parallel_for(B, n_threads, [&](int b) {
    for (int j = 0; j < 5; ++j) out[(size_t)b * 5 + j] = 0.0;
    admissible[b] = 0;
    if (status[b] != ST_CONVERGED) return;
    ChainIO ch;
    load_chain(S, b, k[b], tau[b], xD, xL, x, surf, prim, bary, spq, ch);
    EvalOut ev;
    eval_chain(S, ch, load3(nD + 3 * (size_t)(b / spq)), ev, offset ? offset + (size_t)b * 2 * MAXK : nullptr);
    if (!ev.ok || !admissible_chain(S, ch, ev, prm->ray_eps)) return;
    GlossyTerms gt;
    if (!glossy_terms(S, ch, ev, alpha, gt)) return;
    admissible[b] = 1;
    double* o = out + (size_t)b * 5;
    o[0] = gt.detJ; o[1] = gt.bsdf; o[2] = gt.geom; o[3] = gt.dens; o[4] = gt.W;
  });
  return 0;
}

}  // extern "C"
