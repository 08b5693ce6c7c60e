// Declarations of the auxiliary kernels' host launchers.
#pragma once

#include <vector>

#include "mpg_kernels.cuh"

namespace mpg {

// Spatial tree of the guide samples, host side (mpg_stree.cu): per node the
// split axis (-1 for a leaf), split value, children (the leaf index in `left`
// for a leaf); per leaf member its leaf and record, leaf-major, ascending
// records within a leaf.
struct StreeHost {
  std::vector<int> axis, left, right, member_leaf, member_rec;
  std::vector<double> split;
  int n_leaves = 0, n_samples = 0;
};
void stree_build(const float* pos /* [6][n] host */, int n, double eps, double c, StreeHost& t);
// The same tree level by level (mpg_stree_level.cuh): on the host from host
// positions, or on the device from device positions d_pos [6][n] (consumed
// as scratch; synchronous on st).  Returns false on a CUDA error (message in err).
void stree_build_levels_host(const float* pos, int n, double eps, double c, StreeHost& t);
bool stree_build_levels_device(float* d_pos, int n, double eps, double c, StreeHost& t, cudaStream_t st,
                               const char** err);

// Counting sort of the chains with status `filter` (any status when < 0) by
// length into order[]; returns the first CUDA error of its calls.
cudaError_t launch_bucket(const uint8_t* k, const uint8_t* status, int filter, int B, int* count, int* base,
                          int* cursor, int* order, int sms, cudaStream_t st);
void launch_irradiance(const float* contrib, int Q, int spq, float* E, int sms, cudaStream_t st);
// New heights of a heightfield on the device: vertex positions and normals,
// the leaf-ordered triangles and a bottom-up refit of the BVH boxes (the tree's
// shape is kept).  `extent` = (x0, y0, x1, y1); parent / ninner describe the
// tree; count is scratch of one int per node.  Returns the first CUDA error.
cudaError_t launch_hf_update(DHF H, const double* extent, const float* heights, int n_tris, const int* parent,
                             const int* ninner, int* count, cudaStream_t st);
void launch_guide_update(const DGuide& g, const uint32_t* cell, const float* omega, const float* w, int R,
                         const int* R_dev, int shift, int* err, int sms, cudaStream_t st);
// Guide records in chain order (mpg_vmf.cu): tile_scratch holds rec_tiles(B) counts.
int rec_tiles(int B);
// Exclusive scan of a[0..n) in place by one CTA; *total (may be NULL) gets the sum.
void launch_scan_exclusive(uint32_t* a, int n, int* total, cudaStream_t st);
// The same over many CTAs for long arrays; sums holds scan_tiles(n) values.
int scan_tiles(int n);
void launch_scan_exclusive_tiled(uint32_t* a, int n, uint32_t* sums, cudaStream_t st);
void launch_guide_records_ordered(const DChains& c, const float* contrib, float inv_area, uint32_t* tile_scratch,
                                  uint32_t* cell_out, float* om_out, float* w_out, uint8_t* k_out, uint8_t* tau_out,
                                  int* chain_out, int* R, cudaStream_t st);
// vMF lobe build and chain-length sampler (mpg_vmf.cu).
int vmf_build_launches(int R, int n_cells);
void launch_vmf_build(const DGuide& g, uint32_t* scratch, const uint32_t* cell, const float* omega, const float* w,
                      const uint8_t* k, const uint8_t* tau, int R, const int* R_dev, int shift, int* err, int sms,
                      cudaStream_t st);
void launch_sample_lengths(const DGuide* g, const DChains& c, const uint32_t* p0w, uint2 key, uint64_t offset,
                           float alpha, DCtx ctx, uint8_t* k_out, float* pn_out, int sms, cudaStream_t st);
// Glossy separators (mpg_aux.cu).
void launch_separator_bsdf(const DChains& c, const float* contrib, float3 cam, float e, float* radiance, int sms,
                           cudaStream_t st);
void launch_records_bsdf(const DChains& c, const int* rec_chain, const float* omega, float* w, int R, const int* R_dev,
                         float3 cam, float e, int sms, cudaStream_t st);
// Spatial tree of the guide samples (mpg_stree.cu).
void launch_stree_gather(const DChains& c, const int* rec_chain, int n, float* pos, cudaStream_t st);
void launch_stree_records(const int* member_leaf, const int* member_rec, int M, const float* omega, const float* w,
                          const uint8_t* k, const uint8_t* tau, int R_in, uint32_t* cell_out, float* omega_out,
                          float* w_out, uint8_t* k_out, uint8_t* tau_out, int R_out, int* R_out_dev, int sms,
                          cudaStream_t st);
void launch_stree_query(const int* axis, const double* split, const int* left, const int* right, const DChains& c,
                        uint32_t* chain_cell, int sms, cudaStream_t st);
void launch_trace(const DScene& S, const float* o, const float* d, int n, float tmin, float tmax, float* t, int* surf,
                  int* prim, float* bary, int* err, unsigned long long* stats, bool st_on, int sms, cudaStream_t st);
double run_fp32_peak(float* scratch, int sms, cudaStream_t st);
double run_fp64_peak(float* scratch, int sms, cudaStream_t st);  // scratch: 8-byte aligned
void launch_rng_advance(unsigned long long* counter, unsigned long long delta, cudaStream_t st);

}  // namespace mpg
