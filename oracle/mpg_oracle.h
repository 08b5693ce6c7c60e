/*
 * FP64 CPU oracle of the batched manifold walk (Manifold Path Guiding,
 * Fan et al. 2023).  TEST INFRASTRUCTURE ONLY: the CUDA library never links,
 * includes or calls this code; only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark use it.
 *
 * Plain and slow on purpose: one chain at a time, FP64 throughout, the
 * method's steps in the paper's order:
 *   seed chain  = p_0 / guided mixture direction + deduction by ray casts (Eq. deduction, Sec. 5.3-5.5)
 *   manifold walk = Newton on the half-vector constraint + reprojection (Sec. 3, "Manifold walks")
 *   contribution T = kappa * G * L_o                                  (Eq. ThroughputEval)
 *   reciprocal probability by Bernoulli trials, n reused             (Sec. 5.8, reciprocal probability estimation)
 *   guide histogram update with w = T <1/P>                          (Eq. eq_weight)
 *   vMF mixture guide, P_e(n), P_e(tau | n), one-sample MIS          (Sec. 5.5, Eq. vMF)
 *
 * Arrays are caller-owned, array-of-structures, float64 unless stated:
 *   chain vertex positions x[B][8][3], surface ids surf[B][8], primitive ids
 *   prim[B][8], barycentrics bary[B][8][2] (triangles only), k[B], tau[B]
 *   (bit i-1 set => vertex i refracts).  Chain b belongs to receiver point
 *   q = b / spq.  All calls return 0 on success and a negative value on a
 *   bad argument; they never throw.
 */
#ifndef MPG_ORACLE_H
#define MPG_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_params {
  double tol;          /* converged when max_i |C_i|_inf < tol */
  int32_t max_iter;    /* Newton steps */
  int32_t max_halvings;/* step halvings per Newton step */
  double ray_eps;      /* ray origin offset and segment shrink */
  double sing_eps;     /* singular 2x2 block threshold (relative) */
  double dedup_eps;    /* same-solution distance */
  int32_t max_trials;  /* Bernoulli trial cap */
  int32_t weight_shift;/* histogram quantisation shift S */
  double alpha;        /* defensive mixture weight of p_0 */
  int32_t bern_repeats;/* independent Bernoulli estimates per chain (<= 1: one) */
  int32_t selective;   /* selective activation: with a guide, no seed in a cell without samples */
} orc_params;

/* vMF mixture guide (Sec. 5.5): one lobe per sample of the last pass.  The
 * lobes of a cell are contiguous, ordered by key = (n << 8) | tau and, within
 * a key, in record order. */
typedef struct orc_vmf {
  int32_t n_cells, n_lobes;
  const uint32_t* cell_start; /* [n_cells+1] first lobe of each cell */
  const uint32_t* key;        /* [n_lobes] (n << 8) | tau */
  const double* lobe;         /* [n_lobes][4] mu_x, mu_y, mu_z, kappa */
  const uint64_t* prefix;     /* [n_lobes] inclusive prefix sums of the quantised weights within the cell */
} orc_vmf;

typedef struct orc_guide {
  const uint64_t* counts; /* [n_cells][n_theta*n_phi]; NULL => p_0 only */
  int32_t n_cells, n_theta, n_phi;
  const float* cos_theta; /* [n_theta+1] bin edges in cos(theta), decreasing */
  const float* phi_cos;   /* [n_phi+1] cos of phi edges */
  const float* phi_sin;   /* [n_phi+1] sin of phi edges */
  const orc_vmf* vmf;     /* non-NULL => the vMF mixture replaces the histograms */
} orc_guide;

void* orc_scene_create(const double* surfaces, int32_t n_surf, const double* hf_desc,
                       const double* hf_heights, int32_t n_hf, const double* targets,
                       int32_t n_targets, const double* light);
void orc_scene_destroy(void* scene);

/* Nearest hit along each ray in (tmin, tmax); brute != 0 skips the BVH. */
int32_t orc_intersect(void* scene, int32_t n, const double* o, const double* d, double tmin,
                      double tmax, int32_t brute, double* t, int32_t* surf, int32_t* prim,
                      double* bary);

/* Seed chains (trial index `trial`, 0 for the first draw).  The guide cell of
 * chain b is chain_cell[b] when chain_cell is not NULL (a spatial tree's
 * leaf), else cell[b / spq]; the same holds for orc_bernoulli and
 * orc_sample_lengths. */
int32_t orc_sample_seeds(void* scene, const orc_guide* guide, int32_t Q, const double* xD,
                         const double* nD, const uint32_t* cell, int32_t spq, const double* xL,
                         const uint8_t* k, const uint8_t* tau, int32_t tau_random,
                         uint64_t rng_seed, uint64_t rng_offset, uint32_t trial,
                         const orc_params* prm, double* x, int32_t* surf, int32_t* prim,
                         double* bary, uint8_t* tau_out, double* pdf, uint8_t* valid,
                         int32_t n_threads, const uint32_t* chain_cell);

/* Manifold walk in place on chains with valid[b] != 0.  offset (may be NULL):
 * offset normals of glossy chains, [B][8][2] tangential components per vertex;
 * the walk then solves C_i = off_i (Sec. 5.7, glossy chains). */
int32_t orc_walk(void* scene, int32_t B, int32_t spq, const double* xD, const double* nD,
                 const double* xL, const uint8_t* k, const uint8_t* tau, const orc_params* prm,
                 const uint8_t* valid, double* x, int32_t* surf, int32_t* prim, double* bary,
                 uint8_t* status, uint8_t* iters, int32_t n_threads, const double* offset);

/* Admissibility, generalized geometry term, kappa, T = kappa G L_o. */
int32_t orc_contribution(void* scene, int32_t B, int32_t spq, const double* xD,
                         const double* nD, const double* xL, const uint8_t* k,
                         const uint8_t* tau, const double* x, const int32_t* surf,
                         const int32_t* prim, const double* bary, const uint8_t* status,
                         const orc_params* prm, double* G, double* kappa, double* T,
                         uint8_t* admissible, int32_t n_threads);

/* Bernoulli trials for admissible chains: N[b] = index of the first trial
 * that walks to the same solution, capped[b] = 1 when max_trials ran out,
 * trial_walks[b] (may be NULL) = trial walks that converged.  With
 * bern_repeats = r > 1 the estimate is repeated r times independently (repeat
 * j draws trial t with trial counter t | j << 24) and N[b] is the sum of the
 * r trial counts, so <1/P(x | n)> = N[b] / r; capped when any repeat capped.
 * offset (may be NULL): the offset normals of glossy chains ([B][8][2], as for
 * orc_walk); every trial of chain b walks with chain b's offsets, so N[b]
 * estimates 1/P(x | n, offsets). */
int32_t orc_bernoulli(void* scene, const orc_guide* guide, int32_t Q, const double* xD,
                      const double* nD, const uint32_t* cell, int32_t spq, const double* xL,
                      const uint8_t* k, const uint8_t* tau, int32_t tau_random,
                      uint64_t rng_seed, uint64_t rng_offset, const orc_params* prm,
                      const double* x, const int32_t* surf, const uint8_t* admissible,
                      uint32_t* N, uint8_t* capped, uint32_t* trial_walks, int32_t n_threads,
                      const uint32_t* chain_cell, const double* offset);

/* Histogram bin of each direction (theta-major index), and the update
 * counts[cell][bin] += q(w), q = min(floor(w 2^S), 2^32-1) (0 unless w > 0). */
int32_t orc_guide_bin(const orc_guide* guide, int32_t R, const float* omega, int32_t* bin);
int32_t orc_guide_update(const orc_guide* guide, uint64_t* counts, int32_t R,
                         const uint32_t* cell, const float* omega, const float* w,
                         int32_t weight_shift);

/* vMF mixture from guide records (cell, w_D [R][3], w, n, tau): lobes sorted
 * by (cell, n, tau) and record order, mu = w_D, kappa = sigma^-2 with sigma
 * the angle to the nearest other direction of the same cell, n and tau (pi
 * when there is none; at least 1e-6), prefix sums of q(w) within each cell.
 * Outputs are [n_cells+1], [R], [R][4] and [R]. */
int32_t orc_vmf_build(int32_t n_cells, int32_t R, const uint32_t* cell, const float* omega,
                      const float* w, const uint8_t* k, const uint8_t* tau, int32_t weight_shift,
                      uint32_t* cell_start, uint32_t* key, double* lobe, uint64_t* prefix);

/* Chain lengths from P(n) = alpha P_0(n) + (1 - alpha) P_e(n | cell) (Sec. 5.5,
 * defensive one-sample MIS; P_e from the vMF guide's weights, absent => P_0
 * only): k_out[b] and pn_out[b] = P(k_out[b]).  p0w[n-1] are integer weights
 * of P_0(n), n = 1..8. */
int32_t orc_sample_lengths(const orc_guide* guide, int32_t Q, const uint32_t* cell, int32_t spq,
                           const uint32_t* p0w, uint64_t rng_seed, uint64_t rng_offset,
                           const orc_params* prm, uint8_t* k_out, double* pn_out,
                           const uint32_t* chain_cell);

/* vMF lobe density (Eq. vMF) and inverse-CDF draw, exposed for the tests. */
double orc_vmf_pdf(const double* mu, double kappa, const double* w);
void orc_vmf_sample(const double* mu, double kappa, double u1, double u2, double* w);

/* Constraint values of a given chain (tests): C[b][2k] and max |C|. */
int32_t orc_constraint(void* scene, int32_t B, int32_t spq, const double* xD, const double* nD,
                       const double* xL, const uint8_t* k, const uint8_t* tau,
                       const double* x, const int32_t* surf, const int32_t* prim,
                       const double* bary, double* C, double* cmax);

/* Shooting map used by finite-difference tests: trace from x_D along omega
 * with the scattering types tau; returns the k vertices and the exit ray. */
int32_t orc_shoot(void* scene, const double* xD, const double* omega, int32_t k, uint8_t tau,
                  double ray_eps, double* x, double* exit_dir);

/* Adjoint: dL_dtheta[height] += sum_b weight[b] * dT_b/dtheta for heightfield
 * chains (T = kappa G L_o at the converged chain, implicit function theorem,
 * heights of heightfield 0 on its grid).  dT_out[b] (may be NULL) = 1 where a
 * gradient was formed. */
int32_t orc_adjoint(void* scene, int32_t B, int32_t spq, const double* xD, const double* nD, const double* xL,
                    const uint8_t* k, const uint8_t* tau, const double* x, const int32_t* surf,
                    const int32_t* prim, const double* bary, const double* weight, double* dL_dtheta,
                    double* dT_out, int32_t n_threads);

/* Glossy chains (Sec. 5.7): offset normals drawn from an isotropic Beckmann
 * distribution of roughness alpha > 0, [B][8][2] tangential components per
 * vertex (zero beyond k[b]); chain b uses Philox counter (b + rng_offset,
 * vertex, 4). */
int32_t orc_sample_offsets(int32_t B, const uint8_t* k, double alpha, uint64_t rng_seed, uint64_t rng_offset,
                           double* offset);

/* Terms of converged glossy chains walked with `offset` (may be NULL):
 * out [B][5] = |det dC/du| (orthonormal area coordinates), the microfacet
 * BSDF product with D divided out, the geometric factors, the offsets'
 * density prod D(m_i) on the disk, and the estimate W = L_e bsdf geom / det;
 * admissible[b] as for orc_contribution.  alpha = 0: the specular limit
 * (no D, no shadowing), whose W equals kappa G L_e. */
int32_t orc_glossy(void* scene, int32_t B, int32_t spq, const double* xD, const double* nD, const double* xL,
                   const uint8_t* k, const uint8_t* tau, const double* x, const int32_t* surf, const int32_t* prim,
                   const double* bary, const uint8_t* status, const orc_params* prm, const double* offset,
                   double alpha, double* out, uint8_t* admissible, int32_t n_threads);

/* Philox4x32-10 block: out = philox(ctr[4], key[2]). */
void orc_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out);

/* Flops of one execution of each primitive in the counted scalar type (16
 * values; the order is documented in the implementation). */
int32_t orc_unit_flops(double* out);



#ifdef __cplusplus
}
#endif
#endif
