// vMF mixture guide of Sec. 5.5 (Eq. vMF) on the GPU: guide records in chain
// order, the lobe build from the records of the last pass (a stable radix
// sort by cell, length and types; cell starts; per-cell prefix sums of the
// quantised weights; kappa from the nearest direction of each group), and the
// chain-length sampler of the defensive mixture P(n) = alpha P_0(n) +
// (1 - alpha) P_e(n | cell).  Seed and trial directions are drawn by
// draw_seed (mpg_device.cuh).
#include <algorithm>
#include <utility>

#include "mpg_aux.cuh"

namespace mpg {

namespace {
constexpr unsigned FULL = 0xffffffffu;
constexpr int SCAN_THREADS = 1024;
constexpr int TILE_THREADS = 256;
constexpr int REC_TILE = 8 * TILE_THREADS;    // chains per CTA of the record compaction
constexpr int RADIX_TILE = 4 * TILE_THREADS;  // keys per CTA of a radix pass
constexpr float VMF_SIGMA_MIN = 1e-6f;        // identical directions
}  // namespace

__device__ __forceinline__ unsigned lanemask_lt() { return (1u << (threadIdx.x & 31)) - 1u; }

// Exclusive scan of a[0..n) in place by one CTA of SCAN_THREADS threads (each
// thread a contiguous chunk); *total (may be NULL) receives the sum.
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_exclusive(uint32_t* a, int n, int* total) {
  __shared__ uint32_t warp_sum[SCAN_THREADS / 32];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int chunk = (n + SCAN_THREADS - 1) / SCAN_THREADS;
  const int i0 = min(n, t * chunk), i1 = min(n, i0 + chunk);
  uint32_t s = 0;
  for (int i = i0; i < i1; ++i) s += a[i];
  // exclusive prefix of the chunk sums across the CTA
  uint32_t x = s;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t v = warp_sum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(FULL, v, o);
      if (lane >= o) v += y;
    }
    warp_sum[lane] = v;  // inclusive over warps
  }
  __syncthreads();
  uint32_t run = x - s + (wid > 0 ? warp_sum[wid - 1] : 0u);
  for (int i = i0; i < i1; ++i) {
    uint32_t v = a[i];
    a[i] = run;
    run += v;
  }
  if (total && t == SCAN_THREADS - 1) *total = (int)run;
}

// Exclusive scan of a long array over many CTAs: tiles of SCAN_TILE values,
// their sums (k_scan_tile_sums), the one-CTA scan of the sums, then every tile
// scanned with its offset (k_scan_tile_apply).  Loads and stores of a tile go
// through shared memory, coalesced; the one-CTA kernel above reads a thread's
// contiguous chunk and is kept for short arrays.
constexpr int SCAN_TILE_THREADS = 256, SCAN_PER = 16, SCAN_TILE = SCAN_TILE_THREADS * SCAN_PER;

__global__ void __launch_bounds__(SCAN_TILE_THREADS) k_scan_tile_sums(const uint32_t* a, int n, uint32_t* sums) {
  __shared__ uint32_t ws[SCAN_TILE_THREADS / 32];
  const int base = blockIdx.x * SCAN_TILE;
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < SCAN_PER; ++j) {
    const int i = base + j * SCAN_TILE_THREADS + threadIdx.x;
    if (i < n) s += a[i];
  }
  s = __reduce_add_sync(FULL, s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < SCAN_TILE_THREADS / 32; ++w) t += ws[w];
    sums[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(SCAN_TILE_THREADS) k_scan_tile_apply(uint32_t* a, int n, const uint32_t* offs) {
  __shared__ uint32_t tile[SCAN_TILE];
  __shared__ uint32_t ws[SCAN_TILE_THREADS / 32];
  const int base = blockIdx.x * SCAN_TILE;
#pragma unroll
  for (int j = 0; j < SCAN_PER; ++j) {
    const int k = j * SCAN_TILE_THREADS + threadIdx.x, i = base + k;
    tile[k] = i < n ? a[i] : 0u;
  }
  __syncthreads();
  // each thread scans its SCAN_PER consecutive values
  uint32_t v[SCAN_PER], s = 0;
#pragma unroll
  for (int j = 0; j < SCAN_PER; ++j) {
    v[j] = tile[threadIdx.x * SCAN_PER + j];
    s += v[j];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = s;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[wid] = x;
  __syncthreads();
  uint32_t before = 0;
  for (int w = 0; w < wid; ++w) before += ws[w];
  uint32_t run = offs[blockIdx.x] + before + x - s;
  __syncthreads();  // every thread has read its values from the tile
#pragma unroll
  for (int j = 0; j < SCAN_PER; ++j) {
    tile[threadIdx.x * SCAN_PER + j] = run;
    run += v[j];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < SCAN_PER; ++j) {
    const int k = j * SCAN_TILE_THREADS + threadIdx.x, i = base + k;
    if (i < n) a[i] = tile[k];
  }
}

// Exclusive scan of the digit-major tile counts cnt[d * tiles + t] over the
// tiles that hold records (t < used, the others take no part), by one CTA:
// the virtual index v = d * used + t runs over 256 * used entries.
__global__ void __launch_bounds__(SCAN_THREADS) k_radix_scan(uint32_t* cnt, int tiles, int R, const int* R_dev) {
  __shared__ uint32_t warp_sum[SCAN_THREADS / 32];
  const int nr = R_dev ? min(max(*R_dev, 0), R) : R;
  const int used = (nr + 4 * 256 - 1) / (4 * 256);
  const int n = 256 * used;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int chunk = (n + SCAN_THREADS - 1) / SCAN_THREADS;
  const int i0 = min(n, t * chunk), i1 = min(n, i0 + chunk);
  auto at = [&](int v) -> uint32_t& { return cnt[(size_t)(v / used) * tiles + v % used]; };
  uint32_t s = 0;
  for (int i = i0; i < i1; ++i) s += at(i);
  uint32_t x = s;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t v = warp_sum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(FULL, v, o);
      if (lane >= o) v += y;
    }
    warp_sum[lane] = v;
  }
  __syncthreads();
  uint32_t run = x - s + (wid > 0 ? warp_sum[wid - 1] : 0u);
  for (int i = i0; i < i1; ++i) {
    uint32_t v = at(i);
    at(i) = run;
    run += v;
  }
}

// ---------------------------------------------------------------------------
// Guide records in chain order (count per tile, scan, write)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TILE_THREADS) k_rec_count(const float* contrib, int B, uint32_t* cnt) {
  __shared__ int wsum[TILE_THREADS / 32];
  int n = 0;
  for (int r = 0; r < REC_TILE / TILE_THREADS; ++r) {
    int b = blockIdx.x * REC_TILE + r * TILE_THREADS + threadIdx.x;
    n += (b < B && contrib[b] > 0.0f) ? 1 : 0;
  }
  n = __reduce_add_sync(FULL, n);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < TILE_THREADS / 32; ++w) s += wsum[w];
    cnt[blockIdx.x] = (uint32_t)s;
  }
}

__global__ void __launch_bounds__(TILE_THREADS) k_rec_write(DChains c, const float* contrib, float inv_area,
                                                            const uint32_t* offs, uint32_t* cell_out, float* om_out,
                                                            float* w_out, uint8_t* k_out, uint8_t* tau_out,
                                                            int* chain_out) {
  __shared__ int wcount[TILE_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int run = (int)offs[blockIdx.x];
  for (int r = 0; r < REC_TILE / TILE_THREADS; ++r) {
    int b = blockIdx.x * REC_TILE + r * TILE_THREADS + threadIdx.x;
    bool f = b < c.B && contrib[b] > 0.0f;
    unsigned m = __ballot_sync(FULL, f);
    if (lane == 0) wcount[wid] = __popc(m);
    __syncthreads();
    int before = 0, all = 0;
    for (int w = 0; w < TILE_THREADS / 32; ++w) {
      before += w < wid ? wcount[w] : 0;
      all += wcount[w];
    }
    if (f) {
      int o = run + before + __popc(m & lanemask_lt());
      int q = b / c.spq;
      float3 xD = make_float3(c.xD[q], c.xD[c.Q + q], c.xD[2 * c.Q + q]);
      float3 x1 = make_float3(c.x[b], c.x[(size_t)c.B + b], c.x[2 * (size_t)c.B + b]);
      float3 w = unit(x1 - xD);
      cell_out[o] = cell_of(c, b);
      om_out[o] = w.x;
      om_out[c.B + o] = w.y;
      om_out[2 * (size_t)c.B + o] = w.z;
      w_out[o] = contrib[b] * inv_area;
      if (k_out) k_out[o] = c.k[b];
      if (tau_out) tau_out[o] = c.tau[b];
      if (chain_out) chain_out[o] = b;
    }
    run += all;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (key, value) pairs, 8 bits per pass
// ---------------------------------------------------------------------------
// Digit counts of each tile, stored digit-major: cnt[d * tiles + tile].
// Number of records to sort: the device count when given, else R.
__device__ __forceinline__ int sort_count(int R, const int* R_dev) { return R_dev ? min(max(*R_dev, 0), R) : R; }

__global__ void __launch_bounds__(TILE_THREADS) k_radix_hist(const uint32_t* keys, int R, const int* R_dev, int shift,
                                                             uint32_t* cnt) {
  __shared__ uint32_t h[256];
  const int n = sort_count(R, R_dev);
  if (blockIdx.x * RADIX_TILE >= n) return;  // past the records: this tile takes no part
  h[threadIdx.x] = 0;
  __syncthreads();
  for (int r = 0; r < RADIX_TILE / TILE_THREADS; ++r) {
    int i = blockIdx.x * RADIX_TILE + r * TILE_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  cnt[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// Scatter by digit: off = exclusive scan of the digit-major counts.  Within a
// tile the items go in index order (rounds of 256, warps in order, lanes in
// order: match-any ranks within a warp, per-warp digit counts across warps).
__global__ void __launch_bounds__(TILE_THREADS) k_radix_scatter(const uint32_t* kin, const uint32_t* vin,
                                                                uint32_t* kout, uint32_t* vout, int R,
                                                                const int* R_dev, int shift, const uint32_t* off) {
  constexpr int NW = TILE_THREADS / 32;
  __shared__ uint32_t base[256];
  __shared__ uint32_t wc[NW][256];
  const int n = sort_count(R, R_dev);
  if (blockIdx.x * RADIX_TILE >= n) return;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  base[t] = off[(size_t)t * gridDim.x + blockIdx.x];
  for (int r = 0; r < RADIX_TILE / TILE_THREADS; ++r) {
    for (int w = 0; w < NW; ++w) wc[w][t] = 0;
    __syncthreads();
    int i = blockIdx.x * RADIX_TILE + r * TILE_THREADS + t;
    bool valid = i < n;
    uint32_t key = valid ? kin[i] : 0u;
    int d = valid ? (int)((key >> shift) & 255u) : -1 - lane;  // past the end: a lane of its own
    unsigned peers = __match_any_sync(FULL, d);
    int rank = __popc(peers & lanemask_lt());
    if (valid && rank == 0) wc[wid][d] = __popc(peers);
    __syncthreads();
    // per digit: exclusive prefix over the warps, on top of the tile's running base
    uint32_t run = base[t];
    for (int w = 0; w < NW; ++w) {
      uint32_t v = wc[w][t];
      wc[w][t] = run;
      run += v;
    }
    base[t] = run;
    __syncthreads();
    if (valid) {
      uint32_t pos = wc[wid][d] + (uint32_t)rank;
      kout[pos] = key;
      vout[pos] = vin[i];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Lobe build
// ---------------------------------------------------------------------------
// Group key of each of the n records, cell << 11 | (n - 1) << 8 | tau (cell,
// then length, then types); invalid records get n_cells << 11 and sort after
// every valid one.  Entries past the record count are not sorted or read.
__global__ void k_vmf_keys(const uint32_t* cell, const uint8_t* k, const uint8_t* tau, int R, const int* R_dev,
                           int n_cells, uint32_t* keys, uint32_t* vals, int* err) {
  const int n = sort_count(R, R_dev);
  const uint32_t past = (uint32_t)n_cells << 11;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint32_t key = past;
    uint32_t c = cell[i], kk = k[i], tt = tau[i];
    if (c < (uint32_t)n_cells && kk >= 1 && kk <= MAXK && tt < (1u << kk)) key = (c << 11) | ((kk - 1) << 8) | tt;
    else atomicOr(err, 4);
    keys[i] = key;
    vals[i] = (uint32_t)i;
  }
}

// cell_start[c] = first sorted key >= c << 11, c = 0..n_cells (the last is the lobe count).
__global__ void k_vmf_cells(const uint32_t* keys, int R, const int* R_dev, int n_cells, uint32_t* cell_start) {
  const int n = sort_count(R, R_dev);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= n_cells; c += gridDim.x * blockDim.x) {
    uint32_t want = (uint32_t)c << 11;
    int a = 0, b = n;
    while (a < b) {
      int m = (a + b) >> 1;
      if (keys[m] < want) a = m + 1; else b = m;
    }
    cell_start[c] = (uint32_t)a;
  }
}

// Lobe i from the record sorted into place i: key, direction and quantised
// weight q = min(floor(w 2^S), 2^32 - 1) (exact in FP32: a power-of-two
// scaling and its floor), as the histogram update.
__global__ void k_vmf_lobes(const uint32_t* vals, const uint32_t* cell_start, int n_cells, const float* omega,
                            const float* w, const uint8_t* k, const uint8_t* tau, int R, int shift, uint32_t* lobe_key,
                            float4* lobe, uint64_t* prefix) {
  const int L = (int)cell_start[n_cells];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L; i += gridDim.x * blockDim.x) {
    uint32_t r = vals[i];
    lobe_key[i] = ((uint32_t)k[r] << 8) | tau[r];
    lobe[i] = make_float4(omega[r], omega[R + r], omega[2 * (size_t)R + r], 0.0f);
    float wr = w[r];
    uint64_t q = 0;
    if (wr > 0.0f) {
      float qf = floorf(ldexpf(wr, shift));
      q = qf >= 4294967295.0f ? 4294967295ull : (uint64_t)qf;
    }
    prefix[i] = q;
  }
}

// Inclusive prefix sums of the lobe weights within each cell, one CTA per cell.
__global__ void __launch_bounds__(TILE_THREADS) k_vmf_prefix(const uint32_t* cell_start, uint64_t* prefix) {
  __shared__ unsigned long long ws[TILE_THREADS / 32];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const uint32_t a = cell_start[blockIdx.x], b = cell_start[blockIdx.x + 1];
  unsigned long long carry = 0;
  for (uint32_t i0 = a; i0 < b; i0 += TILE_THREADS) {
    uint32_t i = i0 + t;
    unsigned long long v = i < b ? prefix[i] : 0ull, x = v;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    unsigned long long before = carry;
    for (int w = 0; w < wid; ++w) before += ws[w];
    if (i < b) prefix[i] = before + x;
    unsigned long long all = 0;
    for (int w = 0; w < TILE_THREADS / 32; ++w) all += ws[w];
    carry += all;
    __syncthreads();
  }
}

// kappa_i = sigma_i^-2, sigma_i the angle between mu_i and the nearest other
// direction of its group (same cell, length and types; the groups are runs of
// equal sorted keys): the smallest chord |mu_i - mu_j| converted to an angle,
// pi for a lone lobe, at least VMF_SIGMA_MIN.  Threads of a warp hold
// neighbouring lobes of one group, so the loads of mu_j are broadcasts.
// kappa goes to kap[i] (the lobes are read-only here) and k_vmf_kappa_store
// moves it into the lobes.
__global__ void __launch_bounds__(TILE_THREADS) k_vmf_kappa(const uint32_t* keys, const uint32_t* cell_start,
                                                            int n_cells, const float4* lobe, float* kap) {
  const int L = (int)cell_start[n_cells];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L; i += gridDim.x * blockDim.x) {
    const uint32_t key = keys[i];
    int g0 = 0, g1 = i;
    while (g0 < g1) {  // first index of the group
      int m = (g0 + g1) >> 1;
      if (keys[m] < key) g0 = m + 1; else g1 = m;
    }
    int h0 = i + 1, h1 = L;
    while (h0 < h1) {  // one past its last index
      int m = (h0 + h1) >> 1;
      if (keys[m] <= key) h0 = m + 1; else h1 = m;
    }
    const float4 me = __ldg(lobe + i);
    float sigma = 3.14159265358979323846f;
    if (h0 - g0 > 1) {
      float best = 3.0e38f;
      for (int j = g0; j < h0; ++j) {
        float4 o = __ldg(lobe + j);
        float dx = me.x - o.x, dy = me.y - o.y, dz = me.z - o.z;
        float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        best = j == i ? best : fminf(best, d2);
      }
      sigma = 2.0f * asinf(fminf(1.0f, 0.5f * sqrtf(best)));
    }
    sigma = fmaxf(sigma, VMF_SIGMA_MIN);
    kap[i] = 1.0f / (sigma * sigma);
  }
}

// Stores kappa into the lobes and the density coefficient of each lobe,
// q_i kappa_i / (2 pi (1 - e^{-2 kappa_i})), so that the mixture density is
// sum_i coef_i e^{-kappa_i |w - mu_i|^2 / 2} / Q.
__global__ void k_vmf_kappa_store(const uint32_t* cell_start, int n_cells, const float* kap,
                                  const uint64_t* prefix, float4* lobe, float* coef) {
  const int L = (int)cell_start[n_cells];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L; i += gridDim.x * blockDim.x) {
    const float k = kap[i];
    lobe[i].w = k;
    // the cell of lobe i: the last c with cell_start[c] <= i
    int a = 0, b = n_cells;
    while (b - a > 1) {
      int m = (a + b) >> 1;
      if ((int)cell_start[m] <= i) a = m; else b = m;
    }
    const uint64_t q = prefix[i] - ((uint32_t)i > cell_start[a] ? prefix[i - 1] : 0ull);
    coef[i] = (float)q * (k / (6.28318530717958647f * -expm1f(-2.0f * k)));
  }
}

// ---------------------------------------------------------------------------
// Chain lengths: P(n) = alpha P_0(n) + (1 - alpha) P_e(n | cell)
// ---------------------------------------------------------------------------
struct P0Table {
  uint32_t w[MAXK];
  uint64_t total;
};

__global__ void k_sample_lengths(DGuide g, int has_guide, DChains ch, P0Table p0, uint2 key, uint64_t offset,
                                 float alpha, DCtx ctx, uint8_t* k_out, float* pn_out) {
  offset = rng_offset(offset, ctx);
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < ch.B; b += gridDim.x * blockDim.x) {
    uint64_t idx = (uint64_t)b + offset;
    uint4 r = philox(make_uint4((uint32_t)idx, (uint32_t)(idx >> 32), 0u, 2u), key);
    uint32_t c = cell_of(ch, b);
    uint32_t cs = 0, ce = 0;
    uint64_t Wc = 0;
    if (has_guide) {
      if (c >= (uint32_t)g.n_cells) {
        atomicOr(ctx.err, 2);
      } else {
        cs = __ldg(g.cell_start + c);
        ce = __ldg(g.cell_start + c + 1);
        Wc = lobe_cum(g, cs, ce);
      }
    }
    const bool pick_p0 = Wc == 0 || u01(r.x) < alpha;
    int n = 1;
    if (pick_p0) {
      uint64_t target = scaled_target(r.y, p0.total), acc = 0;
      for (n = 1; n < MAXK; ++n) {
        acc += p0.w[n - 1];
        if (acc > target) break;
      }
    } else {
      // the lobe holding the target; lobes ascend in n, so its n is drawn
      // with probability W(n) / W
      VmfRange all;
      all.cs = cs; all.a = cs; all.b = ce; all.base = 0; all.total = Wc;
      n = (int)(__ldg(g.lobe_key + vmf_search(g, all, scaled_target(r.y, Wc))) >> 8);
    }
    float P0 = (float)p0.w[n - 1] / (float)p0.total;
    float pn = P0;
    if (Wc > 0) {
      uint32_t a = lobe_bound(g, cs, ce, (uint32_t)n << 8), bb = lobe_bound(g, a, ce, (uint32_t)(n + 1) << 8);
      float Pe = (float)(lobe_cum(g, cs, bb) - lobe_cum(g, cs, a)) / (float)Wc;
      pn = alpha * P0 + (1.0f - alpha) * Pe;
    }
    k_out[b] = (uint8_t)n;
    pn_out[b] = pn;
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
int rec_tiles(int B) { return (B + REC_TILE - 1) / REC_TILE; }

void launch_scan_exclusive(uint32_t* a, int n, int* total, cudaStream_t st) {
  k_scan_exclusive<<<1, SCAN_THREADS, 0, st>>>(a, n, total);
}

int scan_tiles(int n) { return (n + SCAN_TILE - 1) / SCAN_TILE; }

void launch_scan_exclusive_tiled(uint32_t* a, int n, uint32_t* sums, cudaStream_t st) {
  const int tiles = scan_tiles(n);
  if (tiles <= 1) {
    k_scan_exclusive<<<1, SCAN_THREADS, 0, st>>>(a, n, nullptr);
    return;
  }
  k_scan_tile_sums<<<tiles, SCAN_TILE_THREADS, 0, st>>>(a, n, sums);
  k_scan_exclusive<<<1, SCAN_THREADS, 0, st>>>(sums, tiles, nullptr);
  k_scan_tile_apply<<<tiles, SCAN_TILE_THREADS, 0, st>>>(a, n, sums);
}

void launch_guide_records_ordered(const DChains& c, const float* contrib, float inv_area, uint32_t* tile_scratch,
                                  uint32_t* cell_out, float* om_out, float* w_out, uint8_t* k_out, uint8_t* tau_out,
                                  int* chain_out, int* R, cudaStream_t st) {
  const int tiles = rec_tiles(c.B);
  if (tiles == 0) {
    cudaMemsetAsync(R, 0, sizeof(int), st);
    return;
  }
  k_rec_count<<<tiles, TILE_THREADS, 0, st>>>(contrib, c.B, tile_scratch);
  k_scan_exclusive<<<1, SCAN_THREADS, 0, st>>>(tile_scratch, tiles, R);
  k_rec_write<<<tiles, TILE_THREADS, 0, st>>>(c, contrib, inv_area, tile_scratch, cell_out, om_out, w_out, k_out,
                                              tau_out, chain_out);
}

int vmf_build_launches(int R, int n_cells) {
  int bits = 32 - __builtin_clz((unsigned)n_cells << 11);
  int passes = (bits + 7) / 8;
  return R == 0 ? 1 : 1 + 3 * passes + 5;
}

void launch_vmf_build(const DGuide& g, uint32_t* scratch, const uint32_t* cell, const float* omega, const float* w,
                      const uint8_t* k, const uint8_t* tau, int R, const int* R_dev, int shift, int* err, int sms,
                      cudaStream_t st) {
  uint32_t* cell_start = const_cast<uint32_t*>(g.cell_start);
  if (R == 0) {
    cudaMemsetAsync(cell_start, 0, sizeof(uint32_t) * (size_t)(g.n_cells + 1), st);
    return;
  }
  const int tiles = (R + RADIX_TILE - 1) / RADIX_TILE;  // tiles past the record count return at once
  uint32_t* ka = scratch;
  uint32_t* va = ka + R;
  uint32_t* kb = va + R;
  uint32_t* vb = kb + R;
  uint32_t* cnt = vb + R;
  const int grid = std::min(sms * 8, (R + 255) / 256);
  k_vmf_keys<<<grid, 256, 0, st>>>(cell, k, tau, R, R_dev, g.n_cells, ka, va, err);
  const int bits = 32 - __builtin_clz((unsigned)g.n_cells << 11);
  for (int shift = 0; shift < bits; shift += 8) {
    k_radix_hist<<<tiles, TILE_THREADS, 0, st>>>(ka, R, R_dev, shift, cnt);
    k_radix_scan<<<1, SCAN_THREADS, 0, st>>>(cnt, tiles, R, R_dev);
    k_radix_scatter<<<tiles, TILE_THREADS, 0, st>>>(ka, va, kb, vb, R, R_dev, shift, cnt);
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  k_vmf_cells<<<(g.n_cells + 256) / 256, 256, 0, st>>>(ka, R, R_dev, g.n_cells, cell_start);
  k_vmf_lobes<<<grid, 256, 0, st>>>(va, cell_start, g.n_cells, omega, w, k, tau, R, shift,
                                    const_cast<uint32_t*>(g.lobe_key), const_cast<float4*>(g.lobe),
                                    const_cast<uint64_t*>(g.lobe_prefix));
  k_vmf_prefix<<<g.n_cells, TILE_THREADS, 0, st>>>(cell_start, const_cast<uint64_t*>(g.lobe_prefix));
  float* kap = reinterpret_cast<float*>(kb);  // the sort's other key buffer is free now
  k_vmf_kappa<<<grid, TILE_THREADS, 0, st>>>(ka, cell_start, g.n_cells, g.lobe, kap);
  k_vmf_kappa_store<<<grid, 256, 0, st>>>(cell_start, g.n_cells, kap, g.lobe_prefix, const_cast<float4*>(g.lobe),
                                          const_cast<float*>(g.lobe_coef));
}

void launch_sample_lengths(const DGuide* g, const DChains& c, const uint32_t* p0w, uint2 key, uint64_t offset,
                           float alpha, DCtx ctx, uint8_t* k_out, float* pn_out, int sms, cudaStream_t st) {
  P0Table t;
  t.total = 0;
  for (int n = 0; n < MAXK; ++n) {
    t.w[n] = p0w[n];
    t.total += p0w[n];
  }
  DGuide gg = g ? *g : DGuide{};
  const int grid = std::max(1, std::min(sms * 8, (c.B + 255) / 256));
  k_sample_lengths<<<grid, 256, 0, st>>>(gg, g != nullptr, c, t, key, offset, alpha, ctx, k_out, pn_out);
}

}  // namespace mpg
