/*
 * mpg.h -- C ABI of the GB300 (sm_103a) manifold-walk library libmpg.so.
 *
 * The library runs the data-parallel hot path of Manifold Path Guiding
 * (Fan, Hong, Guo, Zou, Guo, Yan; ACM TOG 42(6), 2023): guided seed chains
 * between two separators x_D and x_L, Newton manifold walks on the specular
 * constraints, the contribution T = kappa G L_o of each admissible chain, its
 * reciprocal probability by Bernoulli trials, the guide-histogram update, and
 * the adjoint of the receiver irradiance with respect to surface parameters;
 * and around it the paper's guiding machinery: the vMF mixture with sampled
 * chain lengths and types, the spatial tree of the guide samples, glossy
 * separators with product importance sampling, repeated reciprocal estimates,
 * selective activation and the online training schedule.
 *
 * Conventions for every entry point:
 *   - Return value: MPG_OK (0) or a negative mpg_status.  The message of the
 *     last failure on the calling host thread is returned by mpg_last_error().
 *     No C++ exception crosses this boundary.
 *   - Pointers inside mpg_chains, mpg_guide and the output arguments are DEVICE
 *     pointers, borrowed: the caller allocates and frees them (for example as
 *     PyTorch tensors) and keeps them alive until the stream work completes.
 *     All must be 16-byte aligned.  Arrays are structure-of-arrays with the
 *     chain index fastest: element (i, c, b) of x lives at x[(i*3 + c)*B + b].
 *   - Host pointers are used only during the call (scene and guide tables).
 *   - Every call is asynchronous on the given cudaStream_t (0 = legacy default
 *     stream); only mpg_ctx_sync() waits.  Device-side failures (for example a
 *     BVH traversal stack overflow) are recorded in the context and reported by
 *     the next mpg_ctx_sync().
 *   - Opaque handles come in create/destroy pairs; destroy accepts NULL.
 *   - A batch with B = Q = 0 is a valid no-op.
 *   - Chain b belongs to receiver point q = b / spq.  Vertex types: bit i-1 of
 *     tau[b] set means vertex i refracts (T), clear means it reflects (R).
 */
#ifndef MPG_H
#define MPG_H

#include <stdint.h>
#include <cuda_runtime.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mpg_status;
#define MPG_OK 0
#define MPG_ERR_INVALID_ARG (-1)
#define MPG_ERR_CUDA (-2)
#define MPG_ERR_OOM (-3)
#define MPG_ERR_LIMIT (-4)
#define MPG_ERR_UNSUPPORTED (-5)

#define MPG_MAXK 8

/* Per-chain status written by the walk (uint8). */
#define MPG_CHAIN_INVALID 0   /* seed could not be deduced (miss, TIR, wrong side) */
#define MPG_CHAIN_CONVERGED 1 /* max_i |C_i|_inf < tol */
#define MPG_CHAIN_FAILED 2    /* singular block, failed reprojection or line search */
#define MPG_CHAIN_LIMIT 3     /* max_iter Newton steps without convergence */
#define MPG_CHAIN_SEEDED 255  /* valid seed, not walked yet */

#define MPG_WALK_PLAIN 0      /* one launch per chain length k, no graph */
#define MPG_WALK_BATCHED 1    /* all k in one persistent launch, k-sorted work queue */

/* Solver constants.  The paper fixes none of them (it defers the walk to the
 * manifold-walk literature, Sec. 3); the values are the caller's. */
typedef struct mpg_params {
  float tol;            /* converged when max_i |C_i|_inf < tol                  */
  int32_t max_iter;     /* Newton steps per walk                                  */
  int32_t max_halvings; /* step halvings per Newton step                          */
  float ray_eps;        /* ray origin offset and shadow-segment shrink (scene units) */
  float sing_eps;       /* |det B'| <= sing_eps * max|B'|^2 => singular block      */
  float dedup_eps;      /* two chains are one solution when every vertex is closer */
  int32_t max_trials;   /* Bernoulli trial cap                                    */
  int32_t weight_shift; /* histogram weight quantisation q = floor(w * 2^S)        */
  float alpha;          /* defensive mixture weight of p_0 (Sec. 5.5, alpha = 0.5) */
  int32_t walk_mode;    /* MPG_WALK_PLAIN or MPG_WALK_BATCHED                     */
  int32_t block_threads;/* threads per block of the walk kernels (0 = 128; 32..128,
                           a multiple of 32)                                      */
  int32_t tau_random;   /* nonzero: draw tau_i ~ Bernoulli(0.5) per trial          */
  int32_t k_uniform;    /* 1..8: every chain has this length; 0: lengths vary      */
  float stall_tol;      /* FP32 resolution of C: a walk whose line search can no
                           longer reduce |C|, or that reaches max_iter, ends
                           CONVERGED when max_i |C_i|_inf < stall_tol (0 disables;
                           the FP64 oracle has no such rule)                      */
  float fp64_tol;       /* G is formed in FP32 from both chain ends (reciprocity);
                           when the two differ by more than this relative amount,
                           for k >= 6, or for a walk stopped by stall_tol, the
                           vertices are polished and G recomputed in FP64
                           (0: always FP64)                                     */
  /* Schedule of the batched mode.  Apart from fp64_k and walk_group none of
   * these changes a result: every chain is walked, and every trial drawn, with
   * the same arithmetic whatever the schedule (mpg_autotune picks them by
   * timing). */
  int32_t fp64_k;       /* chains of this length or longer always take the FP64
                           geometry term (0 = 6; 1..6 allowed, so the split can
                           only move toward more FP64)                         */
  int32_t ctas_per_sm;  /* resident CTAs per SM of the persistent kernels
                           (0 = the occupancy maximum)                          */
  int32_t refill_every; /* passes between work-queue refills of idle lanes in the
                           persistent kernels (0 or 1 = every pass; a warp whose
                           lanes are all idle refills at once)                  */
  int32_t trial_sync_rounds; /* Bernoulli: rounds that draw one trial per chain
                           before the parallel rounds (0 = 2; -1 = none; 1..8)   */
  int32_t trial_batch;  /* Bernoulli: parallel trials per chain in the first
                           parallel round (0 = 64; 1..4096), x4 each round after;
                           issued trial-major, so trials past a chain's first
                           success are mostly skipped                          */
  int32_t walk_group;   /* one chain per group of G lanes (G = 2, 4, 8 >= k; 128
                           threads per CTA) instead of one thread per chain:
                           bit 0 in the walks (primary and synchronous trial
                           walks), bit 1 in the parallel Bernoulli rounds.
                           Lane j owns vertex j, the blocks are staged in shared
                           memory.  Same per-vertex arithmetic; the compiler may
                           contract products differently in the two forms, so
                           results agree to FP32 rounding, not bit for bit    */
  int32_t bern_repeats; /* Bernoulli: independent reciprocal-probability
                           estimates averaged per chain (0 or 1 = one; up to 64;
                           the paper's repeated estimation, Sec. 6.5
                           performance analysis).  Repeat j draws trial t from counter
                           (b + offset, t | j << 24, block), so repeat 0 is the
                           single estimate; trials[b] is the sum of the N_j,
                           <1/P> = trials[b] / (repeats P(n)), capped is set when
                           any repeat ran out of trials                        */
  int32_t selective;    /* selective activation (Sec. 5.8): with a guide, seeds
                           of receiver points whose cell holds no samples (no
                           histogram weight; no lobes) are not drawn -- the
                           chain is MPG_CHAIN_INVALID at once and contributes
                           nothing; the paper hands such points to path
                           tracing, which this library does not do          */
  float roughness;      /* glossy chains (chains.offset set, Sec. 5.7): the
                           Beckmann roughness alpha of every vertex, used by
                           the shadowing term of the estimate (0..1; 0 = the
                           specular limit of the estimate)                   */
} mpg_params;

/* Chain batch: B = Q * spq chains of length k[b] <= 8 between x_D[q] and x_L[b]. */
typedef struct mpg_chains {
  int32_t B, Q, spq;
  const float* xD;      /* [3][Q] receiver points (separator x_D)                  */
  const float* nD;      /* [3][Q] receiver normals                                 */
  const uint32_t* cell; /* [Q] guide cell of each receiver point                   */
  const float* xL;      /* [3][B] light-side separator x_L of each chain           */
  const uint8_t* k;     /* [B] chain length n (1..8)                               */
  const float* pn;      /* [B] P(n) of the chain's length (NULL => 1)              */
  uint8_t* tau;         /* [B] vertex types (input; overwritten when tau_random)   */
  float* x;             /* [8][3][B] vertex positions                              */
  int32_t* surf;        /* [8][B] surface index of each vertex                     */
  int32_t* prim;        /* [8][B] triangle index (meshes) or -1                    */
  float* bary;          /* [8][2][B] barycentrics on triangles                     */
  float* pdf;           /* [B] solid-angle density of the seed direction           */
  uint8_t* status;      /* [B] MPG_CHAIN_* (valid seed => INVALID until walked)    */
  uint8_t* iters;       /* [B] Newton steps taken                                  */
  const uint32_t* chain_cell; /* [B] guide cell of each chain (a spatial tree's leaf,
                           mpg_stree_query), or NULL => cell[b / spq]             */
  const float* offset;  /* [8][2][B] offset normals of glossy chains
                           (mpg_sample_offsets), or NULL for specular chains:
                           the tangential components o_i of a microfacet normal
                           per vertex in the vertex's shading frame; the walk
                           then solves C_i = (h.s_i, h.t_i) - o_i (Sec. 5.7)  */
} mpg_chains;

/* Guide kinds (mpg_guide.kind). */
#define MPG_GUIDE_HISTOGRAM 0
#define MPG_GUIDE_VMF 1

/* Build scratch of a vMF guide of `capacity` lobes, in uint32 words. */
#define MPG_VMF_SCRATCH_WORDS(capacity) (4 * (size_t)(capacity) + 256 * (((size_t)(capacity) + 1023) / 1024) + 64)

/* Guide, caller-owned, one of two kinds.
 * MPG_GUIDE_HISTOGRAM (0): per cell a (theta, phi) histogram over world
 *   directions (theta from +z uniform over [0, pi], phi uniform over
 *   [0, 2 pi)).  The vMF fields are unused (zero).
 * MPG_GUIDE_VMF (1): the vMF mixture of Sec. 5.5 (Eq. vMF) built by
 *   mpg_vmf_build from the records of the last pass: one lobe per record, the
 *   lobes of a cell contiguous and ordered by key = (n << 8) | tau and, within
 *   a key, by record order.  The receiver cell stands for the spatial
 *   neighbourhood S(x_D, x_L).  Uses n_cells and the vMF fields; the histogram
 *   pointers are unused. */
typedef struct mpg_guide {
  int32_t n_cells, n_theta, n_phi;
  uint64_t* counts;        /* [n_cells][n_theta*n_phi] quantised weight sums      */
  uint64_t* cdf;           /* [n_cells][n_theta*n_phi] inclusive prefix sums      */
  const float* cos_theta;  /* [n_theta+1] FP32 edges cos(j pi/n_theta)            */
  const float* phi_cos;    /* [n_phi+1] FP32 cos(2 pi j/n_phi)                    */
  const float* phi_sin;    /* [n_phi+1] FP32 sin(2 pi j/n_phi)                    */
  int32_t kind;            /* MPG_GUIDE_HISTOGRAM or MPG_GUIDE_VMF                 */
  int32_t capacity;        /* vMF: lobes the arrays hold                           */
  uint32_t* cell_start;    /* vMF: [n_cells+1] first lobe of each cell             */
  uint32_t* lobe_key;      /* vMF: [capacity] (n << 8) | tau                       */
  float* lobe;             /* vMF: [capacity][4] mu_x, mu_y, mu_z, kappa           */
  uint64_t* lobe_prefix;   /* vMF: [capacity] inclusive prefix sums of the
                              quantised weights within the cell                    */
  float* lobe_coef;        /* vMF: [capacity] q_i kappa_i / (2 pi (1 - e^{-2 kappa_i})),
                              the lobe's factor in the mixture density             */
  uint32_t* scratch;       /* vMF: MPG_VMF_SCRATCH_WORDS(capacity) build scratch   */
} mpg_guide;

typedef struct mpg_ctx mpg_ctx;
typedef struct mpg_scene mpg_scene;

/* Work counters accumulated by the kernels since the last reset (device-side,
 * read back by mpg_ctx_stats): multiplied by per-unit operation counts they
 * give the algorithmic flop count of a run. */
typedef struct mpg_stats {
  uint64_t newton_steps;     /* Newton steps (one Thomas solve each)              */
  uint64_t thomas_rows;      /* block rows of those Thomas solves (k per step)    */
  uint64_t full_evals;       /* vertex evaluations with Jacobian blocks           */
  uint64_t c_evals;          /* constraint-only vertex evaluations (line search)  */
  uint64_t ray_casts;        /* nearest-hit ray queries                           */
  uint64_t sphere_tests;     /* ray/sphere and ray/cap tests                      */
  uint64_t plane_tests;      /* ray/rectangle tests                               */
  uint64_t node_tests;       /* BVH child-box tests                               */
  uint64_t tri_tests;        /* ray/triangle tests                                */
  uint64_t walks;            /* walks started                                     */
  uint64_t converged;        /* walks converged: first walks, and the trial walks
                                a sequential Bernoulli loop runs (up to each
                                chain's first recurrence), whatever the schedule */
  uint64_t ggt_rows;         /* block rows of the 2-column geometry-term solves   */
  uint64_t trials;           /* Bernoulli trials drawn                            */
  uint64_t seeds;            /* seed directions drawn (first draws and trials)    */
  uint64_t ggt_fp64;         /* geometry terms recomputed in FP64                 */
  uint64_t uncounted;        /* converged trial walks of the parallel Bernoulli
                                rounds left out of `converged` (their record
                                buffer of 8 entries per chain overflowed)      */
} mpg_stats;

/* Kernel families, for per-family counters and launch timings. */
#define MPG_KERNEL_SEED 0
#define MPG_KERNEL_WALK 1
#define MPG_KERNEL_CONTRIB 2
#define MPG_KERNEL_BERNOULLI 3
#define MPG_KERNEL_TRACE 4
#define MPG_KERNEL_AUX 5   /* bucketing, irradiance reduction, guide update/prefix sums/records */
#define MPG_KERNEL_KINDS 6

const char* mpg_last_error(void);
int32_t mpg_version(void);

/* Context on one CUDA device (made current by every call that takes it). */
mpg_status mpg_ctx_create(int32_t device, mpg_ctx** out);
void mpg_ctx_destroy(mpg_ctx* ctx);
/* Waits for `stream` and returns the first device-side error recorded since the
 * last sync (MPG_ERR_LIMIT for a traversal overflow), else MPG_OK. */
mpg_status mpg_ctx_sync(mpg_ctx* ctx, cudaStream_t stream);
/* Counters of one kernel family (kind = MPG_KERNEL_*) or of all (kind = -1);
 * waits for `stream`; reset != 0 clears them afterwards.  out may be NULL. */
mpg_status mpg_ctx_stats(mpg_ctx* ctx, int32_t kind, mpg_stats* out, int32_t reset, cudaStream_t stream);
/* Work counters on (default) or off; off skips writing them. */
mpg_status mpg_ctx_set_stats(mpg_ctx* ctx, int32_t on);
/* Launch timing: when on, every kernel launch of the library is bracketed by
 * CUDA events recorded on the stream it is launched on, and the per-length
 * launches of a batched call run one after another on the call's stream
 * (instead of on concurrent streams), so each bracket times its kernel alone.  mpg_ctx_profile sums
 * the elapsed times (ms) and counts the launches of a family (kind) since the
 * last reset; it synchronises on the recorded events. */
mpg_status mpg_ctx_set_profile(mpg_ctx* ctx, int32_t on);
mpg_status mpg_ctx_profile(mpg_ctx* ctx, int32_t kind, double* ms, int64_t* launches, int32_t reset);
/* Total kernel launches issued by the library on this context. */
mpg_status mpg_ctx_launches(mpg_ctx* ctx, int64_t* count);

/* Scene from the host tables (format: one row of 24 doubles per surface --
 * type, material, eta_front, eta_back, centre[3], radius, axis/normal[3],
 * cap_cos, e_x[3], e_y[3], heightfield index; heightfield descriptors of 6
 * doubles nx, ny, x0, y0, x1, y1 with heights concatenated row-major; seed
 * targets of 16 doubles; a light of 16 doubles).  Builds the triangle meshes,
 * interpolation normals and BVHs on the host and uploads them (library-owned
 * device memory, freed by mpg_scene_destroy).  Synchronous. */
mpg_status mpg_scene_create(mpg_ctx* ctx, const double* surfaces, int32_t n_surf,
                            const double* hf_desc, const double* hf_heights, int32_t n_hf,
                            const double* targets, int32_t n_targets, const double* light,
                            mpg_scene** out);
void mpg_scene_destroy(mpg_scene* scene);
/* Number of BVH nodes and triangles of heightfield h (for reports). */
mpg_status mpg_scene_info(const mpg_scene* scene, int32_t h, int32_t* n_nodes, int32_t* n_tris);
/* New heights of heightfield h, on the device: `heights` is a device array of
 * nx * ny floats (row-major, as hf_heights of mpg_scene_create), read only.
 * Recomputes the vertex positions and interpolation normals with the scene
 * builder's formulas and FP64 operations (so a scene built on the host from
 * the same FP32 heights has the same arrays), the leaf-ordered triangles, and
 * refits the boxes of the BVH bottom up while keeping its shape.  The
 * heightfield's parameters are what the adjoint (mpg_walk_adjoint, Sec. 5.2)
 * differentiates, so a gradient loop changes them without leaving the device.
 * Asynchronous on `stream`; calls on the scene queued after it on that stream
 * see the new surface, calls already running on other streams must be
 * finished first (the caller orders them).  Errors: MPG_ERR_INVALID_ARG for
 * a NULL or unaligned pointer or no heightfield h, MPG_ERR_CUDA for a launch
 * failure. */
mpg_status mpg_scene_set_heights(mpg_ctx* ctx, mpg_scene* scene, int32_t h, const float* heights,
                                 cudaStream_t stream);

/* S1 -- seed chains (Eq. deduction; Sec. 5.4 initialisation p_0; Sec. 5.5
 * guided sampling with the one-sample defensive mixture alpha p_0 + (1-alpha) p_e).
 * For each chain: draws from Philox4x32-10 keyed by rng_seed with counter
 * (b + rng_offset, trial 0, block), picks p_0 (a seed target, uniform visible cap
 * or rectangle) or the cell's guide (guide may be NULL => p_0 only), deduces
 * x_1 = r(x_D, w_D) and the next vertices by scattering with tau, and writes
 * x/surf/prim/bary/pdf/tau and status (MPG_CHAIN_INVALID on failure, else
 * MPG_CHAIN_SEEDED).
 * Histogram guide: tau is the input (or uniform when tau_random) and pdf the
 * solid-angle density of w_D.  vMF guide: given n = k[b], the guided component
 * draws a lobe of the cell with probability proportional to its weight among
 * the lobes of length n (of length n and type tau[b] unless tau_random) and
 * takes (w_D, tau) from it; p_0 draws tau uniformly (tau_random) or keeps the
 * input; pdf is the joint density p(w_D, tau | n) = alpha p_0(w_D) P_0(tau | n)
 * + (1 - alpha) sum_{lobes of (n, tau)} (q_i / Q) v(w_D; mu_i, kappa_i).  A
 * cell without lobes of the chain's length (and type) samples p_0 only. */
mpg_status mpg_sample_seeds(mpg_ctx* ctx, const mpg_scene* scene, const mpg_guide* guide,
                            mpg_chains* chains, uint64_t rng_seed, uint64_t rng_offset,
                            const mpg_params* params, cudaStream_t stream);

/* Sec. 5.7 -- offset normals of glossy chains: for chain b and vertex i <
 * k[b], a microfacet normal m drawn from the isotropic Beckmann distribution
 * of roughness alpha with density D(m) (m.n) (tan^2 theta = -alpha^2
 * log(1 - u1), phi = 2 pi u2, u1 and u2 from Philox4x32-10 counter
 * (b + rng_offset, i, 4)); offset[(2i + c) B + b] = its tangential components
 * (sin theta cos phi, sin theta sin phi), zeros for i >= k[b].  Uses B and k
 * of `chains`; offset is a device array of 16 B floats.  Errors: alpha outside
 * (0, 1], NULL or unaligned arrays (MPG_ERR_INVALID_ARG). */
mpg_status mpg_sample_offsets(mpg_ctx* ctx, const mpg_chains* chains, float alpha, uint64_t rng_seed,
                              uint64_t rng_offset, float* offset, cudaStream_t stream);

/* S2-S6 -- manifold walk (Sec. 3, "Manifold walks"): Newton's method on the
 * generalized half-vector constraints C_i = (h.s_i, h.t_i), h ~ eta_i w_i +
 * eta_o w_o, with the 2k x 2k block-tridiagonal Jacobian solved by a 2x2-block
 * Thomas sweep, step halving and reprojection of each moved vertex onto its own
 * surface by a ray cast along the surface's projection direction (from the
 * centre of spheres and caps, along the normal of rectangles, vertically into
 * heightfields).  Chain visibility is left to mpg_chain_contribution's
 * admissibility test.  Walks every chain whose status is MPG_CHAIN_SEEDED; writes x,
 * surf, prim, bary, status and iters in place.  Glossy chains (chains.offset
 * set) are walked to C_i = o_i by the plain kernels whatever walk_mode asks. */
mpg_status mpg_manifold_walk(mpg_ctx* ctx, const mpg_scene* scene, mpg_chains* chains,
                             const mpg_params* params, cudaStream_t stream);

/* Allocation-free variant of mpg_manifold_walk in the batched (persistent
 * work-queue) form; the paper has no counterpart -- it exists for callers that
 * must not allocate device memory during a call: renderers whose frame loop
 * forbids cudaMalloc (it synchronises the device and can stall the frame),
 * codes whose device memory is owned by their own pool allocator, and
 * callers that cannot touch the runtime allocator while another thread holds a
 * global-mode stream capture.  Same inputs, outputs and results (bit for
 * bit) as mpg_manifold_walk with walk_mode MPG_WALK_BATCHED and the same
 * schedule (walk_group, block_threads, ctas_per_sm, refill_every) on the
 * current device, with no context: work counters and launch timing are not
 * kept.  Unlike mpg_manifold_walk it waits for `stream` before returning, to
 * read the device-side error word it clears at the start of every call: a
 * BVH traversal stack overflow returns MPG_ERR_LIMIT.
 * Scratch: a fixed device array inside the library (about 4 MiB plus the
 * counters, held by every GPU that loads the library until the process exits),
 * so one call takes at most 1,048,576 chains; larger batches are rejected with
 * MPG_ERR_INVALID_ARG.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress); make that first call before any
 * stream capture.  It calls no cudaMalloc, cudaFree or allocating library
 * routine.  Every call shares the array and clears what must start at zero;
 * calls that overlap on the GPU (two streams, or two host threads) race on it.
 * The scene must live on the current device.  Glossy chains (chains.offset
 * set) are rejected with MPG_ERR_UNSUPPORTED. */
mpg_status mpg_manifold_walk_noalloc(const mpg_scene* scene, mpg_chains* chains,
                                     const mpg_params* params, cudaStream_t stream);

/* S7-S9 -- contribution of each converged chain (Eq. ThroughputEval):
 * admissibility (unoccluded segments, vertex types consistent with the sides,
 * positive end cosines), the generalized geometry term G by the implicit
 * function theorem (in FP64 for k >= 6 and ill-conditioned chains, see
 * fp64_tol), kappa (Fresnel / mirror and
 * radiance scaling), T = kappa G L_o; then Bernoulli trials (Sec. 5.8, reciprocal probability estimation): fresh
 * seeds with the same n are walked until one reaches the same solution (FP64
 * distance test), N = trial index, <1/P> = N / P(n) (capped at max_trials,
 * `capped` set).  Writes contrib[b] = A_L T <1/P> (A_L = light area, 1 for a
 * point light) and the irradiance estimate E[q] = sum_b contrib / spq
 * (Eq. ThroughputMC).  Outputs may be NULL except E; all are [B] unless noted.
 * Chains whose geometry term is formed in FP64 are first polished in FP64;
 * their x, prim and bary are updated in place with the polished vertices.
 * Glossy chains (chains.offset set; plain kernels): T is the estimate
 * W = L_e prod_i f_i |n_i.l_i| prod(area factors) / (|det dC/du| prod_i p(o_i))
 * of Sec. 5.7 in FP64 (f the microfacet BSDF of Walter et al. 2007 with the
 * Beckmann distribution of roughness params.roughness, p(o) = D(m) on the unit
 * disk, so D cancels; |det dC/du| as the product of the block elimination's
 * pivot determinants), G and kappa are 0, and the Bernoulli trials walk every
 * trial seed with the chain's own offsets. */
mpg_status mpg_chain_contribution(mpg_ctx* ctx, const mpg_scene* scene, const mpg_guide* guide,
                                  const mpg_chains* chains, uint64_t rng_seed, uint64_t rng_offset,
                                  const mpg_params* params, float* G, float* kappa, float* T,
                                  uint32_t* trials, uint8_t* capped, float* contrib,
                                  float* E /* [Q] */, cudaStream_t stream);

/* S10 -- guide update with sample weights w = T <1/P> (Eq. eq_weight): each
 * record r < n (n = *R_dev when R_dev is not NULL, else R) adds
 * q = min(floor(w[r] 2^S), 2^32-1) (0 unless w > 0) to counts[cell[r]][bin(omega)]
 * with 64-bit integer atomics (bit-exact, order independent), then rebuilds the
 * per-cell prefix sums used by the sampler.  omega is [3][R] SoA FP32 (R is the
 * row stride and the upper bound of n); R_dev is a device int32.  Histogram
 * guides only (a vMF guide is built by mpg_vmf_build). */
mpg_status mpg_guide_update(mpg_ctx* ctx, const mpg_guide* guide, const uint32_t* cell,
                            const float* omega, const float* w, int32_t R, const int32_t* R_dev,
                            int32_t weight_shift, cudaStream_t stream);
/* Empties the guide (counts and prefix sums to zero; a vMF guide: no lobes in
 * any cell) on `stream`, for a new
 * training pass (Sec. 5.8: the distributions are built from the last training iteration's samples only). */
mpg_status mpg_guide_clear(mpg_ctx* ctx, const mpg_guide* guide, cudaStream_t stream);
/* Records of the admissible chains of a batch for mpg_guide_update and
 * mpg_vmf_build: compacts (cell, w_D = unit(x_1 - x_D), w = contrib/A_L, and
 * when k_out / tau_out / chain_out are not NULL the chain's length, types and
 * index) of chains with contrib > 0 into cell_out[B], omega_out[3][B],
 * w_out[B], k_out[B], tau_out[B] and chain_out[B] (capacity B) in chain
 * order, and writes the record count to *R_dev (device int32).  The cell is
 * the chain's (chain_cell when set). */
mpg_status mpg_guide_records(mpg_ctx* ctx, const mpg_scene* scene, const mpg_chains* chains,
                             const float* contrib, uint32_t* cell_out, float* omega_out,
                             float* w_out, uint8_t* k_out, uint8_t* tau_out, int32_t* chain_out,
                             int32_t* R_dev, cudaStream_t stream);

/* Sec. 5.5 -- vMF mixture guide from the records of the last pass (Eq. vMF):
 * record r < n (n = *R_dev when R_dev is not NULL, else R) with cell[r],
 * direction omega[.][r] (SoA [3][R], R the row stride), weight w[r] (Eq.
 * eq_weight), length k[r] (1..8) and types tau[r] (< 2^k) becomes a lobe with
 * mu = omega, kappa = sigma^-2 where sigma is the angle to the nearest other
 * direction of the same cell, length and types (pi when there is none, at
 * least 1e-6), and weight q = min(floor(w 2^S), 2^32-1).  Lobes are sorted by
 * (cell, n, tau) keeping the record order (a stable radix sort), so a build
 * from the same records is bit-identical; cell_start, lobe_key, lobe,
 * lobe_prefix and lobe_coef are overwritten.  The work scales with the record
 * count (*R_dev), not with R.  Records with a cell, length or type out of
 * range are left out and flag the context error (reported by mpg_ctx_sync).
 * R must not exceed guide->capacity. */
mpg_status mpg_vmf_build(mpg_ctx* ctx, const mpg_guide* guide, const uint32_t* cell, const float* omega,
                         const float* w, const uint8_t* k, const uint8_t* tau, int32_t R,
                         const int32_t* R_dev, int32_t weight_shift, cudaStream_t stream);

/* Sec. 5.5 -- chain lengths by the defensive one-sample mixture
 * P(n) = alpha P_0(n) + (1 - alpha) P_e(n | cell), P_e(n | cell) = W(n) / W the
 * weight fraction of the cell's lobes of length n (guide of kind
 * MPG_GUIDE_VMF; NULL, or a cell without lobes => P_0 alone).  P_0 is given
 * by the integer weights p0_weights[n-1], n = 1..8 (host array, sum > 0).
 * Draws use Philox4x32-10 counter (b + rng_offset, 0, 2); writes k_out[b] and
 * pn_out[b] = P(k_out[b]) for the B chains of `chains` (which supplies Q, spq
 * and cell), to be used as chains->k and chains->pn. */
mpg_status mpg_sample_lengths(mpg_ctx* ctx, const mpg_guide* guide, const mpg_chains* chains,
                              const uint32_t* p0_weights, uint64_t rng_seed, uint64_t rng_offset,
                              const mpg_params* params, uint8_t* k_out, float* pn_out,
                              cudaStream_t stream);

/* S11 -- adjoint (the configuration's differentiable form, built on the
 * continuity of the specular manifold, Sec. 5.2): accumulates
 *   dL_dtheta[h] += sum_b dL_dE[q_b] * d(contrib_b / spq)/dtheta_h
 * for the heights theta of heightfield 0 (grid index j*nx + i, FP32,
 * accumulated with atomics), with <1/P> held constant so that
 * d contrib_b/dtheta = (contrib_b / T_b) dT_b/dtheta.  dT/dtheta comes from the
 * implicit function theorem on the converged constraint (J^T lambda = dT/du,
 * dT/dtheta = dT/dtheta|_u - lambda^T dC/dtheta); the Newton iterations are not
 * unrolled.  Chains of length 1..4 whose vertices all lie on heightfield 0 are
 * differentiated; other chains are skipped.  T and contrib are the outputs of
 * mpg_chain_contribution for the same chains. */
mpg_status mpg_walk_adjoint(mpg_ctx* ctx, const mpg_scene* scene, const mpg_chains* chains,
                            const float* T, const float* contrib, const float* dL_dE,
                            float* dL_dtheta, cudaStream_t stream);

/* K3 -- standalone BVH/analytic ray batch: nearest hit of rays (o[3][n], d[3][n])
 * in (tmin, tmax): t (or -1), surface, primitive and barycentrics [2][n]. */
mpg_status mpg_trace_rays(mpg_ctx* ctx, const mpg_scene* scene, const float* o, const float* d,
                          int32_t n, float tmin, float tmax, float* t, int32_t* surf,
                          int32_t* prim, float* bary, cudaStream_t stream);

/* FP32 peak probe: a dependent-FFMA loop over the whole GPU; writes the
 * achieved FP32 FLOP/s (host double) after synchronising `stream`. */
mpg_status mpg_fp32_peak(mpg_ctx* ctx, double* flops, cudaStream_t stream);
/* FP64 peak probe: the same loop with DFMA (FP64 FLOP/s). */
mpg_status mpg_fp64_peak(mpg_ctx* ctx, double* flops, cudaStream_t stream);

/* Captured steps.  The paper runs its chains one by one on CPU threads; on the
 * GPU a whole batched step (seeds, walk, contribution with its Bernoulli rounds,
 * records, guide update: several dozen launches over up to eight concurrent
 * streams) is recorded once as a CUDA graph and replayed with one launch.
 *
 * mpg_graph_begin starts a thread-local stream capture on `stream`: the library
 * calls that follow on that stream (from this thread, on this context) are
 * recorded, not run, until mpg_graph_end, which instantiates the graph.  Calls
 * recorded this way add the graph's device counter to their rng_offset; the
 * counter starts at 0 and the graph adds `rng_advance` to it at the end of each
 * replay, so replay r draws with rng_offset + r * rng_advance and a replayed
 * loop never repeats its random numbers.  Launch timing (mpg_ctx_set_profile)
 * is suspended while recording.  Capacity: the library's context buffers
 * grow only outside a capture, so run the same sequence once uncaptured first;
 * a recorded call that would have to grow them fails with MPG_ERR_INVALID_ARG.
 * After a failed recorded call, still end the capture with mpg_graph_end and
 * destroy the (incomplete) graph it returns.  Nothing may free device memory
 * while the capture is open (no *_destroy of a context, scene or graph from
 * this thread): cudaFree is not allowed then and invalidates the capture.  The device pointers of the
 * recorded calls are baked into the graph: keep them alive and in place.
 * Synchronous (allocates the counter). */
typedef struct mpg_graph mpg_graph;
mpg_status mpg_graph_begin(mpg_ctx* ctx, cudaStream_t stream, uint64_t rng_advance);
/* Lets another context (same device) record into the capture begun on `ctx`:
 * its calls on streams joined to the capture stream (by an event recorded on
 * it) are recorded too and share the graph's random-number counter, until
 * mpg_graph_end on `ctx`.  Two contexts with their own buffers make a graph
 * that advances two independent batches at once, so that the latency-bound
 * ends of one batch's kernels overlap the other's (double buffering). */
mpg_status mpg_graph_join(mpg_ctx* ctx, mpg_ctx* other);
mpg_status mpg_graph_end(mpg_ctx* ctx, cudaStream_t stream, mpg_graph** out);
/* Replays the graph on `stream` (asynchronous, one graph launch). */
mpg_status mpg_graph_launch(mpg_graph* graph, cudaStream_t stream);
/* Kernel launches inside one replay (of every context recorded). */
mpg_status mpg_graph_kernels(const mpg_graph* graph, int64_t* count);
void mpg_graph_destroy(mpg_graph* graph);

/* Sec. 5.6 -- spatial tree of the guide samples: a binary tree over the
 * 6-D positions (x_D, x_L) of the records of a pass, whose leaves stand for
 * the neighbourhood S(x_D, x_L) of the guiding distribution.  A node holding
 * more than T = floor(c sqrt(|S|)) of its own samples (c = 1 in the paper) is
 * split at the midpoint of its box along the axis of largest extent relative
 * to the root box (first such axis on ties; boxes and midpoints in FP64 from
 * the FP32 positions), samples below the midpoint going left; floor(eps k)
 * samples of each child nearest to the plane (k = the node's own samples;
 * eps = 0.1 in the paper; ties by record index) are copied into the other
 * child (spatial filtering) and are not passed on when that child splits in
 * turn; depth at most 48.  Leaves are numbered depth-first, left first; a
 * leaf's members are its own samples and the copies it received, ascending by
 * record index.
 * mpg_stree_build reads the record count (*R_dev, else R) and the records'
 * chain indices (rec_chain, from mpg_guide_records) back to the host,
 * gathers their positions from `chains` on the device and builds the tree
 * (library-owned; synchronous) by `method`:
 *   MPG_STREE_RECURSIVE: depth first on the host (threads for the subtrees
 *     near the root), after copying the positions back;
 *   MPG_STREE_LEVELS: level by level on the device -- each level partitions
 *     the samples of all its split nodes at once (stable, by prefix counts)
 *     and selects all their copies at once (the m-th smallest FP64 distance
 *     of each side by 8-bit digits of its bit pattern, ties by position,
 *     which is ascending record index); the host decides nodes and numbering.
 * Both give the same tree.  Errors: invalid arguments or method
 * (MPG_ERR_INVALID_ARG), a CUDA failure (MPG_ERR_CUDA). */
#define MPG_STREE_RECURSIVE 0
#define MPG_STREE_LEVELS 1
typedef struct mpg_stree mpg_stree;
mpg_status mpg_stree_build(mpg_ctx* ctx, const mpg_chains* chains, const int32_t* rec_chain, int32_t R,
                           const int32_t* R_dev, float epsilon, float c, int32_t method, mpg_stree** out,
                           cudaStream_t stream);
/* The same tree from host positions: pos [6][n] host FP32 (x_D then x_L,
 * coordinate-major; borrowed, read during the call), record r at column r.
 * Built on the host with no device copy and no CUDA call, so it needs no
 * GPU: MPG_STREE_RECURSIVE depth first, or MPG_STREE_LEVELS with the passes
 * of the device's level-by-level build run as plain loops (the same
 * decisions in the same order).  mpg_stree_info and mpg_stree_export work on
 * it, mpg_stree_records and mpg_stree_query reject it (MPG_ERR_INVALID_ARG).
 * Errors: pos NULL with n > 0, n < 0, epsilon outside [0, 0.5), c <= 0, an
 * unknown method or a non-finite position (MPG_ERR_INVALID_ARG). */
mpg_status mpg_stree_build_host(const float* pos, int32_t n, float epsilon, float c, int32_t method,
                                mpg_stree** out);
/* Sizes of a tree: samples, nodes, leaves and leaf members (own + copies). */
mpg_status mpg_stree_info(const mpg_stree* tree, int32_t* n_samples, int32_t* n_nodes, int32_t* n_leaves,
                          int32_t* n_members);
/* Host copies of the tree (for checks): per node axis (-1 for a leaf), split,
 * left child (the leaf index for a leaf) and right child [n_nodes]; per member
 * its leaf and record index [n_members].  Any pointer may be NULL. */
mpg_status mpg_stree_export(const mpg_stree* tree, int32_t* axis, double* split, int32_t* left, int32_t* right,
                            int32_t* member_leaf, int32_t* member_rec);
/* Guide records of the leaves: member m of leaf j becomes a record with cell
 * j and the direction, weight, length and types of its record in the input
 * (arrays of capacity R_in, omega SoA [3][R_in]); written in member order to
 * the outputs (capacity R_out >= n_members, omega [3][R_out]) with the count in
 * *R_out_dev.  A guide built from them has n_cells = n_leaves. */
mpg_status mpg_stree_records(mpg_ctx* ctx, const mpg_stree* tree, const float* omega, const float* w,
                             const uint8_t* k, const uint8_t* tau, int32_t R_in, uint32_t* cell_out,
                             float* omega_out, float* w_out, uint8_t* k_out, uint8_t* tau_out, int32_t R_out,
                             int32_t* R_out_dev, cudaStream_t stream);
/* Leaf of each chain of a batch by descending the tree with (x_D, x_L) (FP64
 * comparisons): chain_cell[b], to be set as chains->chain_cell. */
mpg_status mpg_stree_query(mpg_ctx* ctx, const mpg_stree* tree, const mpg_chains* chains, uint32_t* chain_cell,
                           cudaStream_t stream);
void mpg_stree_destroy(mpg_stree* tree);

/* Sec. 5.7 -- glossy separators.  The receiver's BSDF is a normalised Phong
 * lobe rho(w_i, w) = (e + 2) / (2 pi) max(0, r.w)^e around the mirror
 * direction r = w_i - 2 (w_i.n_D) n_D of the camera ray w_i = unit(x_D -
 * camera) (camera: host float[3]; exponent e > 0).
 * mpg_separator_bsdf: the radiance estimate toward the camera, radiance[b] =
 * rho(w_i, w_D) contrib[b] with w_D = unit(x_1 - x_D) (0 where contrib is 0),
 * and L[q] = sum over the point's seeds / spq.
 * mpg_records_bsdf: product importance sampling with the separator's BSDF
 * (Eq. eq_weight_pis): for the records r < n (n = *R_dev, else R) of
 * mpg_guide_records (chain index, omega SoA [3][R], weight), w[r] *=
 * rho(w_i(x_D of the record's chain), omega_r), in place, before the guide
 * update or build. */
mpg_status mpg_separator_bsdf(mpg_ctx* ctx, const mpg_chains* chains, const float* contrib, const float* camera,
                              float exponent, float* radiance, float* L, cudaStream_t stream);
mpg_status mpg_records_bsdf(mpg_ctx* ctx, const mpg_chains* chains, const int32_t* rec_chain, const float* omega,
                            float* w, int32_t R, const int32_t* R_dev, const float* camera, float exponent,
                            cudaStream_t stream);

/* Sample schedule of the progressive training (Sec. 5.8, online training and
 * rendering), in seeds per receiver point: training iterations of first_spp,
 * 2 first_spp, 4 first_spp, ... seeds; training never uses more than
 * floor(train_fraction * total_spp) seeds (an iteration that would pass it is
 * cut there); after an iteration a new one starts only while less than half
 * of the training budget is used, otherwise the current iteration continues
 * until the training budget is spent.  Writes the iterations' seed counts to
 * iter_spp[0 .. *n_iters) (room for max_iters) and the rendering budget
 * total_spp - (training seeds) to *render_spp.  Each iteration's guide is
 * built from its own samples only, and training samples are not splatted
 * into the image.  Host-only: no device or context. */
mpg_status mpg_training_plan(int32_t total_spp, int32_t first_spp, float train_fraction, int32_t max_iters,
                             int32_t* iter_spp, int32_t* n_iters, int32_t* render_spp);

/* Autotuner of the batched schedule (block_threads, ctas_per_sm, walk_group,
 * refill_every, trial_sync_rounds, trial_batch, fp64_k).  Times candidate
 * schedules by running the step seeds -> walk -> contribution on the given
 * batch (same rng_seed and rng_offset for every candidate, so each one does
 * the same work; the chain arrays are overwritten) and returns in *out the
 * input parameters with the fastest schedule, and in *best_ms its time.
 * Coordinate descent over one group at a time (tile shape, walk form, refill
 * cadence, Bernoulli rounds, FP64 split); each candidate is timed `repeats`
 * times (minimum) and replaces the best one only when more than 3 % faster.
 * The result is then timed three more times against the input schedule,
 * alternately, and the input schedule is returned if it is the faster.
 * The default schedule walks every length with one thread per chain; on
 * batches with chains of length 3 and more the lane-group form (walk_group)
 * is usually faster (the mixed k = 1..8 batch: about 2.5 times), which this
 * call finds.  The outputs of the step go to scratch the call allocates and
 * frees.  Synchronous; walk_mode must be MPG_WALK_BATCHED. */
mpg_status mpg_autotune(mpg_ctx* ctx, const mpg_scene* scene, const mpg_guide* guide,
                        mpg_chains* chains, uint64_t rng_seed, uint64_t rng_offset,
                        const mpg_params* in, int32_t repeats, mpg_params* out,
                        double* best_ms, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* MPG_H */
