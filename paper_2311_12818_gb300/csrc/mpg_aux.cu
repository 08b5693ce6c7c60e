// Small kernels around the hot path: k-bucketing of the work list, the
// per-point irradiance reduction, the guide histogram (update, prefix sums;
// the records are compacted in mpg_vmf.cu), the end of a Bernoulli round, a
// standalone ray batch and the FP32 / FP64 peak probes.
#include "mpg_aux.cuh"

namespace mpg {

// ---------------------------------------------------------------------------
// k-bucketing (counting sort of chain indices by length)
// ---------------------------------------------------------------------------
__global__ void k_bucket_count(const uint8_t* k, const uint8_t* status, int filter, int B, int* count) {
  __shared__ int sh[MAXK + 1];
  if (threadIdx.x <= MAXK) sh[threadIdx.x] = 0;
  __syncthreads();
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    if (filter >= 0 && status[b] != filter) continue;
    int kk = k[b];
    if (kk >= 1 && kk <= MAXK) atomicAdd(&sh[kk], 1);
  }
  __syncthreads();
  if (threadIdx.x >= 1 && threadIdx.x <= MAXK && sh[threadIdx.x]) atomicAdd(&count[threadIdx.x], sh[threadIdx.x]);
}

__global__ void k_bucket_scan(const int* count, int* base, int* cursor) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int s = 0;
    for (int kk = 0; kk <= MAXK; ++kk) {
      base[kk] = s;
      cursor[kk] = s;
      s += kk >= 1 ? count[kk] : 0;
    }
  }
}

// Lanes of a warp with the same length share one atomic (match + popc), so
// the eight bucket cursors see one update per warp and length, not per chain.
__global__ void k_bucket_scatter(const uint8_t* k, const uint8_t* status, int filter, int B, int* cursor, int* order) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int stride = gridDim.x * blockDim.x;
  for (int b0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); b0 < B; b0 += stride) {  // warp-uniform
    int b = b0 + lane;
    int kk = 0;
    if (b < B && (filter < 0 || status[b] == filter)) {
      kk = k[b];
      if (kk < 1 || kk > MAXK) kk = 0;
    }
    unsigned same = __match_any_sync(FULL, kk);
    int leader = __ffs(same) - 1;
    int off = 0;
    if (kk && lane == leader) off = atomicAdd(&cursor[kk], __popc(same));
    off = __shfl_sync(FULL, off, leader);
    if (kk) order[off + __popc(same & ((1u << lane) - 1u))] = b;
  }
}

cudaError_t launch_bucket(const uint8_t* k, const uint8_t* status, int filter, int B, int* count, int* base,
                          int* cursor, int* order, int sms, cudaStream_t st) {
  const cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * (MAXK + 1), st);
  if (e != cudaSuccess) return e;  // the counting kernels need zeroed counts
  int grid = min(sms * 4, (B + 255) / 256 + 1);
  k_bucket_count<<<grid, 256, 0, st>>>(k, status, filter, B, count);
  k_bucket_scan<<<1, 32, 0, st>>>(count, base, cursor);
  k_bucket_scatter<<<grid, 256, 0, st>>>(k, status, filter, B, cursor, order);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Offset normals of glossy chains (Sec. 5.7): for chain b and vertex i < k[b]
// one Philox4x32-10 block with counter (b + offset, i, 4) gives u1 and u2; the
// normal is drawn from the Beckmann distribution with density D(m) (m.n):
// tan^2(theta) = -alpha^2 log(1 - u1), phi = 2 pi u2; its tangential part
// (sin theta cos phi, sin theta sin phi) is the offset.  Vertices past the
// chain's length get zeros.
// ---------------------------------------------------------------------------
__global__ void k_offsets(const uint8_t* k, int B, float alpha, uint2 key, uint64_t offset, DCtx ctx, float* out) {
  offset = rng_offset(offset, ctx);
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    const int kk = k[b];
    const uint64_t idx = (uint64_t)b + offset;
#pragma unroll
    for (int i = 0; i < MAXK; ++i) {
      float ox = 0.0f, oy = 0.0f;
      if (i < kk) {
        const uint4 r = philox(make_uint4((uint32_t)idx, (uint32_t)(idx >> 32), (uint32_t)i, 4u), key);
        const float u1 = u01(r.x), u2 = u01(r.y);
        const float t2 = -alpha * alpha * logf(1.0f - u1);
        const float c = 1.0f / sqrtf(1.0f + t2), sn = sqrtf(t2) * c;
        float sp, cp;
        sincospif(2.0f * u2, &sp, &cp);
        ox = sn * cp;
        oy = sn * sp;
      }
      out[(size_t)(2 * i + 0) * B + b] = ox;
      out[(size_t)(2 * i + 1) * B + b] = oy;
    }
  }
}

void launch_offsets(const DChains& c, float alpha, uint2 key, uint64_t offset, DCtx ctx, float* out, int sms,
                    cudaStream_t st) {
  const int grid = max(1, min(sms * 8, (c.B + 255) / 256));
  k_offsets<<<grid, 256, 0, st>>>(c.k, c.B, alpha, key, offset, ctx, out);
}

// ---------------------------------------------------------------------------
// E[q] = (1/spq) sum_j contrib[q*spq + j]   (Eq. ThroughputMC), fixed order.
// ---------------------------------------------------------------------------
__global__ void k_irradiance(const float* contrib, int Q, int spq, float* E) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < Q; q += gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int j = 0; j < spq; ++j) s += contrib[(size_t)q * spq + j];
    E[q] = s / (float)spq;
  }
}

void launch_irradiance(const float* contrib, int Q, int spq, float* E, int sms, cudaStream_t st) {
  int grid = min(sms * 8, (Q + 255) / 256 + 1);
  k_irradiance<<<grid, 256, 0, st>>>(contrib, Q, spq, E);
}

// ---------------------------------------------------------------------------
// Guide histogram
// ---------------------------------------------------------------------------
__global__ void k_guide_update(DGuide g, const uint32_t* cell, const float* omega, const float* w, int R,
                               const int* R_dev, int shift, int* err) {
  const int n = R_dev ? min(*R_dev, R) : R;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    uint32_t c = cell[r];
    if ((int)c >= g.n_cells) { atomicOr(err, 2); continue; }
    float wr = w[r];
    if (!(wr > 0.0f)) continue;
    // w 2^S is exact in FP32 (a power-of-two scaling; +inf past the range) and
    // so is its floor: q = min(floor(w 2^S), 2^32 - 1) with no rounding
    float qf = floorf(ldexpf(wr, shift));
    unsigned long long q = qf >= 4294967295.0f ? 4294967295ull : (unsigned long long)qf;
    if (q == 0) continue;
    float3 om = make_float3(omega[r], omega[R + r], omega[2 * (size_t)R + r]);
    int bin = guide_bin(g, om);
    atomicAdd(reinterpret_cast<unsigned long long*>(const_cast<uint64_t*>(g.counts)) + (size_t)c * g.bins + bin, q);
  }
}

// One block per cell: inclusive prefix sum of the cell's bins (uint64).
__global__ void k_guide_cdf(DGuide g, uint64_t* cdf) {
  extern __shared__ unsigned long long warp_sums[];
  const int c = blockIdx.x;
  const int bins = g.bins;
  const int per = (bins + blockDim.x - 1) / blockDim.x;
  const uint64_t* in = g.counts + (size_t)c * bins;
  uint64_t* out = cdf + (size_t)c * bins;
  int lo = threadIdx.x * per, hi = min(bins, lo + per);
  unsigned long long s = 0;
  for (int i = lo; i < hi; ++i) s += in[i];
  // inclusive warp scan of the thread sums
  unsigned long long v = s;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  if (lane == 31) warp_sums[wid] = v;
  __syncthreads();
  if (wid == 0) {
    int nw = blockDim.x >> 5;
    unsigned long long x = lane < nw ? warp_sums[lane] : 0ull;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long n = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += n;
    }
    if (lane < nw) warp_sums[lane] = x;
  }
  __syncthreads();
  unsigned long long run = v - s + (wid > 0 ? warp_sums[wid - 1] : 0ull);
  for (int i = lo; i < hi; ++i) {
    run += in[i];
    out[i] = run;
  }
}

void launch_guide_update(const DGuide& g, const uint32_t* cell, const float* omega, const float* w, int R,
                         const int* R_dev, int shift, int* err, int sms, cudaStream_t st) {
  if (R > 0) {
    int grid = min(sms * 8, (R + 255) / 256 + 1);
    k_guide_update<<<grid, 256, 0, st>>>(g, cell, omega, w, R, R_dev, shift, err);
  }
  k_guide_cdf<<<g.n_cells, 256, (256 / 32) * sizeof(unsigned long long), st>>>(g, const_cast<uint64_t*>(g.cdf));
}

// Records (cell, w_D, w = contrib / A_L) of chains with a contribution.
// ---------------------------------------------------------------------------
// Glossy separators (Sec. 5.7): a normalised Phong lobe around the mirror
// direction of the camera ray, applied to the contributions (radiance) and to
// the guide records' weights (product importance sampling, Eq. eq_weight_pis)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float phong_rho(float3 w_i, float3 n, float3 w, float e) {
  const float3 r = w_i - n * (2.0f * dot(w_i, n));
  return (e + 2.0f) * 0.15915494309189535f * powf(fmaxf(dot(r, w), 0.0f), e);
}

__device__ __forceinline__ float3 receiver_at(const float* a, int Q, int q) {
  return make_float3(a[q], a[Q + q], a[2 * Q + q]);
}

__global__ void k_separator_bsdf(DChains c, const float* contrib, float3 cam, float e, float* radiance) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < c.B; b += gridDim.x * blockDim.x) {
    const float cb = contrib[b];
    float out = 0.0f;
    if (cb > 0.0f) {
      const int q = b / c.spq;
      const float3 xD = receiver_at(c.xD, c.Q, q);
      const float3 x1 = make_float3(c.x[b], c.x[(size_t)c.B + b], c.x[2 * (size_t)c.B + b]);
      out = phong_rho(unit(xD - cam), receiver_at(c.nD, c.Q, q), unit(x1 - xD), e) * cb;
    }
    radiance[b] = out;
  }
}

__global__ void k_records_bsdf(DChains c, const int* rec_chain, const float* omega, float* w, int R, const int* R_dev,
                               float3 cam, float e) {
  const int n = R_dev ? min(max(*R_dev, 0), R) : R;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const int q = rec_chain[r] / c.spq;
    const float3 xD = receiver_at(c.xD, c.Q, q);
    const float3 om = make_float3(omega[r], omega[R + r], omega[2 * (size_t)R + r]);
    w[r] *= phong_rho(unit(xD - cam), receiver_at(c.nD, c.Q, q), om, e);
  }
}

void launch_separator_bsdf(const DChains& c, const float* contrib, float3 cam, float e, float* radiance, int sms,
                           cudaStream_t st) {
  k_separator_bsdf<<<std::max(1, std::min(sms * 8, (c.B + 255) / 256)), 256, 0, st>>>(c, contrib, cam, e, radiance);
}

void launch_records_bsdf(const DChains& c, const int* rec_chain, const float* omega, float* w, int R, const int* R_dev,
                         float3 cam, float e, int sms, cudaStream_t st) {
  k_records_bsdf<<<std::max(1, std::min(sms * 8, (R + 255) / 256)), 256, 0, st>>>(c, rec_chain, omega, w, R, R_dev,
                                                                                  cam, e);
}

// ---------------------------------------------------------------------------
// End of a Bernoulli trial round
// ---------------------------------------------------------------------------
__global__ void k_bern_finish(float area, DChains c, DOut o, const int* list, const int* n_list, const int* base,
                              unsigned* nbest, int t_end, int max_trials, int* next, int* n_next, DPairs pr,
                              unsigned long long* stats) {
  // converged walks to other solutions below each chain's first success
  const int cap = pairs_cap(pr);
  const int np = *pr.n;
  const uint2* P = pr.buf + (size_t)PAIRS_PER_CHAIN * *base;
  uint32_t below = 0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < min(np, cap); j += gridDim.x * blockDim.x) {
    uint2 p = P[j];
    below += p.y < nbest[p.x];
  }
  below = __reduce_add_sync(0xffffffffu, below);
  if (stats && (threadIdx.x & 31) == 0 && below) atomicAdd(stats + 10, (unsigned long long)below);
  if (stats && blockIdx.x == 0 && threadIdx.x == 0 && np > cap) atomicAdd(stats + 15, (unsigned long long)(np - cap));
  const int n = *n_list;
  const int* L = list + *base;
  int* Nx = next + *base;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    int b = L[j];
    unsigned nb = nbest[b];
    bool hit = nb != 0xffffffffu;
    bool cap = !hit && t_end >= max_trials;
    if (hit && stats) atomicAdd(stats + 10, 1ull);  // the walk of trial N converged
    if (hit || cap) {
      bern_write(area, c, o, b, o.T[b], hit ? nb : (uint32_t)max_trials, cap);
    } else {
      Nx[atomicAdd(n_next, 1)] = b;
    }
  }
}

void launch_bern_finish(const DScene& S, const DChains& c, DOut o, const int* list, const int* n_list,
                        const int* base, unsigned* nbest, int t_end, int max_trials, int* next, int* n_next,
                        DPairs pr, unsigned long long* stats, int sms, cudaStream_t st) {
  k_bern_finish<<<sms * 2, 256, 0, st>>>(S.L.area, c, o, list, n_list, base, nbest, t_end, max_trials, next, n_next,
                                         pr, stats);
}

// ---------------------------------------------------------------------------
// Standalone ray batch (BVH/analytic nearest hit)
// ---------------------------------------------------------------------------
template <bool kS>
__global__ void __launch_bounds__(128) k_trace(const __grid_constant__ DScene S, const float* o, const float* d, int n,
                                               float tmin, float tmax, float* t, int* surf, int* prim, float* bary,
                                               int* err, unsigned long long* stats) {
  Counters cnt = {};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float3 oo = make_float3(o[i], o[n + i], o[2 * (size_t)n + i]);
    float3 dd = unit(make_float3(d[i], d[n + i], d[2 * (size_t)n + i]));
    Hit h = intersect<kS, BVH_INLINE>(S, oo, dd, tmin, tmax, err, cnt);
    t[i] = h.surf >= 0 ? h.t : -1.0f;
    surf[i] = h.surf;
    prim[i] = h.prim;
    bary[i] = h.b1;
    bary[n + i] = h.b2;
  }
  if (kS) {
    __syncwarp();
    uint32_t v[5] = {cnt.casts, cnt.sphere, cnt.plane, cnt.node, cnt.tri};
    const int idx[5] = {4, 5, 6, 7, 8};
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      uint32_t s = __reduce_add_sync(0xffffffffu, v[j]);
      if ((threadIdx.x & 31) == 0 && s) atomicAdd(stats + idx[j], (unsigned long long)s);
    }
  }
}

void launch_trace(const DScene& S, const float* o, const float* d, int n, float tmin, float tmax, float* t, int* surf,
                  int* prim, float* bary, int* err, unsigned long long* stats, bool st_on, int sms, cudaStream_t st) {
  int grid = min(sms * 16, (n + 127) / 128 + 1);
  if (st_on) k_trace<true><<<grid, 128, 0, st>>>(S, o, d, n, tmin, tmax, t, surf, prim, bary, err, stats);
  else k_trace<false><<<grid, 128, 0, st>>>(S, o, d, n, tmin, tmax, t, surf, prim, bary, err, stats);
}

// ---------------------------------------------------------------------------
// FP32 peak probe: 8 independent FFMA chains per thread.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_ffma(float* out, int iters, float a, float b) {
  float x0 = threadIdx.x * 1e-3f, x1 = x0 + 1.f, x2 = x0 + 2.f, x3 = x0 + 3.f;
  float x4 = x0 + 4.f, x5 = x0 + 5.f, x6 = x0 + 6.f, x7 = x0 + 7.f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
      x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
    }
  }
  float s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == 1234.5f) out[0] = s;  // keeps the chains live
}

// FP64 peak probe: the same loop with DFMA.
__global__ void __launch_bounds__(256) k_dfma(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1.0, x2 = x0 + 2.0, x3 = x0 + 3.0;
  double x4 = x0 + 4.0, x5 = x0 + 5.0, x6 = x0 + 6.0, x7 = x0 + 7.0;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  double s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == 1234.5) out[0] = s;
}

double run_fp64_peak(float* scratch, int sms, cudaStream_t st) {
  const int block = 256, per_sm = 8, iters = 256;
  int grid = sms * per_sm;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_dfma<<<grid, block, 0, st>>>((double*)scratch, 8, 0.999, 1e-3);  // warm-up
  cudaEventRecord(e0, st);
  k_dfma<<<grid, block, 0, st>>>((double*)scratch, iters, 0.999, 1e-3);
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  double flops = (double)grid * block * iters * 16.0 * 8.0 * 2.0;
  return ms > 0.f ? flops / (ms * 1e-3) : 0.0;
}

// Advances a captured graph's random-number counter at the end of a replay.
__global__ void k_rng_advance(unsigned long long* counter, unsigned long long delta) { *counter += delta; }

void launch_rng_advance(unsigned long long* counter, unsigned long long delta, cudaStream_t st) {
  k_rng_advance<<<1, 1, 0, st>>>(counter, delta);
}

double run_fp32_peak(float* scratch, int sms, cudaStream_t st) {
  const int block = 256, per_sm = 8, iters = 4096;
  int grid = sms * per_sm;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_ffma<<<grid, block, 0, st>>>(scratch, 64, 0.999f, 1e-3f);  // warm-up
  cudaEventRecord(e0, st);
  k_ffma<<<grid, block, 0, st>>>(scratch, iters, 0.999f, 1e-3f);
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  double flops = (double)grid * block * iters * 16.0 * 8.0 * 2.0;
  return ms > 0.f ? flops / (ms * 1e-3) : 0.0;
}

}  // namespace mpg

// ---------------------------------------------------------------------------
// Heightfield heights replaced on the device (mpg_scene_set_heights)
// ---------------------------------------------------------------------------
namespace mpg {

// Vertex positions and interpolation normals of the grid: the same formulas,
// in the same FP64 operations, as the scene builder on the host (central
// differences inside, one-sided on the border; explicit round-to-nearest
// operations so that nothing is contracted into a fused multiply-add), so the
// two give the same FP32 arrays.
__global__ void k_hf_mesh(int nx, int ny, double x0, double y0, double dx, double dy, const float* __restrict__ h,
                          float4* P, float4* N) {
  const int n = nx * ny;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int i = v % nx, j = v / nx;
    auto H = [&](int a, int b) { return (double)h[(size_t)b * nx + a]; };
    double gx, gy;
    if (i == 0) gx = __ddiv_rn(__dsub_rn(H(1, j), H(0, j)), dx);
    else if (i == nx - 1) gx = __ddiv_rn(__dsub_rn(H(nx - 1, j), H(nx - 2, j)), dx);
    else gx = __ddiv_rn(__dsub_rn(H(i + 1, j), H(i - 1, j)), __dmul_rn(2.0, dx));
    if (j == 0) gy = __ddiv_rn(__dsub_rn(H(i, 1), H(i, 0)), dy);
    else if (j == ny - 1) gy = __ddiv_rn(__dsub_rn(H(i, ny - 1), H(i, ny - 2)), dy);
    else gy = __ddiv_rn(__dsub_rn(H(i, j + 1), H(i, j - 1)), __dmul_rn(2.0, dy));
    const double l = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(gx, gx), __dmul_rn(gy, gy)), 1.0));
    P[v] = make_float4((float)__dadd_rn(x0, __dmul_rn((double)i, dx)), (float)__dadd_rn(y0, __dmul_rn((double)j, dy)),
                       h[v], 0.0f);
    N[v] = make_float4((float)__ddiv_rn(-gx, l), (float)__ddiv_rn(-gy, l), (float)__ddiv_rn(1.0, l), 0.0f);
  }
}

// Leaf-ordered triangles (v0 with the triangle id in w, e1, e2) from the new
// positions; the id already in slot s's w gives the triangle.
__global__ void k_hf_tris(int nx, int n_tris, const float4* __restrict__ P, float4* tris) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_tris; s += gridDim.x * blockDim.x) {
    const int t = __float_as_int(tris[3 * (size_t)s].w);
    const int quad = t / 2, tt = t % 2, i = quad % (nx - 1), j = quad / (nx - 1);
    const int v00 = j * nx + i, v1 = tt == 0 ? v00 + 1 : v00 + nx + 1, v2 = tt == 0 ? v00 + nx + 1 : v00 + nx;
    const float4 a = P[v00], b = P[v1], c = P[v2];
    tris[3 * (size_t)s + 0] = make_float4(a.x, a.y, a.z, __int_as_float(t));
    tris[3 * (size_t)s + 1] = make_float4(__fsub_rn(b.x, a.x), __fsub_rn(b.y, a.y), __fsub_rn(b.z, a.z), 0.f);
    tris[3 * (size_t)s + 2] = make_float4(__fsub_rn(c.x, a.x), __fsub_rn(c.y, a.y), __fsub_rn(c.z, a.z), 0.f);
  }
}

struct Box3 {
  float lo[3], hi[3];
};

__device__ __forceinline__ void grow(Box3& b, float x, float y, float z) {
  b.lo[0] = fminf(b.lo[0], x); b.hi[0] = fmaxf(b.hi[0], x);
  b.lo[1] = fminf(b.lo[1], y); b.hi[1] = fmaxf(b.hi[1], y);
  b.lo[2] = fminf(b.lo[2], z); b.hi[2] = fmaxf(b.hi[2], z);
}

// Box of one child of a node: over the grid vertices of its triangles (a
// leaf; as the host builder) or over the two boxes stored in the child node
// (read through L2: another thread wrote them).
__device__ __forceinline__ Box3 child_box(const float4* nodes, const float4* tris, const float4* P, int nx, int idx,
                                          int count) {
  Box3 b = {{INFINITY, INFINITY, INFINITY}, {-INFINITY, -INFINITY, -INFINITY}};
  if (count > 0) {
    for (int s = idx; s < idx + count; ++s) {
      const int t = __float_as_int(tris[3 * (size_t)s].w);
      const int quad = t / 2, tt = t % 2, i = quad % (nx - 1), j = quad / (nx - 1);
      const int v00 = j * nx + i, v1 = tt == 0 ? v00 + 1 : v00 + nx + 1, v2 = tt == 0 ? v00 + nx + 1 : v00 + nx;
      const float4 p0 = P[v00], p1 = P[v1], p2 = P[v2];
      grow(b, p0.x, p0.y, p0.z);
      grow(b, p1.x, p1.y, p1.z);
      grow(b, p2.x, p2.y, p2.z);
    }
    return b;
  }
  const float4 na = __ldcg(nodes + 4 * (size_t)idx), nb = __ldcg(nodes + 4 * (size_t)idx + 1),
               nc = __ldcg(nodes + 4 * (size_t)idx + 2);
  b.lo[0] = fminf(na.x, nb.x); b.hi[0] = fmaxf(na.y, nb.y);
  b.lo[1] = fminf(na.z, nb.z); b.hi[1] = fmaxf(na.w, nb.w);
  b.lo[2] = fminf(nc.x, nc.z); b.hi[2] = fmaxf(nc.y, nc.w);
  return b;
}

// Bottom-up refit in one launch: a node whose children are all leaves starts
// at once; a node with inner children is taken by the thread that finishes
// its last inner child (counter per node).  No thread waits on another.
__global__ void k_hf_refit(int n_nodes, int nx, float4* nodes, const float4* __restrict__ tris,
                           const float4* __restrict__ P, const int* __restrict__ parent,
                           const int* __restrict__ ninner, int* count) {
  for (int v0 = blockIdx.x * blockDim.x + threadIdx.x; v0 < n_nodes; v0 += gridDim.x * blockDim.x) {
    if (ninner[v0] != 0) continue;
    int v = v0;
    while (true) {
      const int4 ch = __ldcg(reinterpret_cast<const int4*>(nodes + 4 * (size_t)v + 3));
      const Box3 L = child_box(nodes, tris, P, nx, ch.x, ch.z), R = child_box(nodes, tris, P, nx, ch.y, ch.w);
      nodes[4 * (size_t)v + 0] = make_float4(L.lo[0], L.hi[0], L.lo[1], L.hi[1]);
      nodes[4 * (size_t)v + 1] = make_float4(R.lo[0], R.hi[0], R.lo[1], R.hi[1]);
      nodes[4 * (size_t)v + 2] = make_float4(L.lo[2], L.hi[2], R.lo[2], R.hi[2]);
      __threadfence();
      const int p = parent[v];
      if (p < 0) break;
      if (atomicAdd(count + p, 1) + 1 < ninner[p]) break;  // the sibling subtree is not done yet
      __threadfence();
      v = p;
    }
  }
}

cudaError_t launch_hf_update(DHF H, const double* extent, const float* heights, int n_tris, const int* parent,
                             const int* ninner, int* count, cudaStream_t st) {
  const double dx = (extent[2] - extent[0]) / (H.nx - 1), dy = (extent[3] - extent[1]) / (H.ny - 1);
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)H.n_nodes, st);
  if (e != cudaSuccess) return e;
  const int nv = H.nx * H.ny;
  k_hf_mesh<<<(nv + 255) / 256, 256, 0, st>>>(H.nx, H.ny, extent[0], extent[1], dx, dy, heights,
                                               const_cast<float4*>(H.P), const_cast<float4*>(H.N));
  k_hf_tris<<<(n_tris + 255) / 256, 256, 0, st>>>(H.nx, n_tris, H.P, const_cast<float4*>(H.tris));
  k_hf_refit<<<(H.n_nodes + 127) / 128, 128, 0, st>>>(H.n_nodes, H.nx, const_cast<float4*>(H.nodes), H.tris, H.P,
                                                       parent, ninner, count);
  return cudaGetLastError();
}

}  // namespace mpg
