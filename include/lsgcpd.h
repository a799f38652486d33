/*
 * lsgcpd.h -- C ABI of the GB300 (sm_103a) implementation of LSG-CPD:
 * "Coherent Point Drift with Local Surface Geometry for Point Cloud
 * Registration" (Liu, Wu, Chirikjian, ICCV 2021).
 *
 * Problem (Sec. 3.1): fix a target cloud Y (M points), align a source cloud X
 * (N points) by a rigid motion g = (R, t), maximising the likelihood of the
 * Gaussian mixture of Eq. (1) built on the target with the anisotropic
 * components of Eq. (2) and a uniform outlier term.  EM (Sec. 3.1): E step of
 * Eq. (5) / Eq. (9); M step by Newton on SE(3) (Eqs. (11)-(13)) and the
 * sigma^2 update.
 *
 * Conventions for every entry point:
 *  - Return value: an lsgcpd_status.  Nothing aborts or traps; on error the
 *    message is available from lsgcpd_last_error(ctx).
 *  - Point arrays are row-major N x 3 (or M x 3) FP32.  Unless stated
 *    otherwise they are DEVICE pointers on the context's device.
 *  - The caller owns every array passed in; the context owns all scratch
 *    memory, CUDA graphs and events.  Entry points never free caller memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls that return host values synchronise that stream.
 *  - A context serves one call at a time (not thread-safe).
 *  - Rotations are row-major 3x3 doubles, translations 3 doubles, in the
 *    caller's (uncentred) frame: y ~ R x + t.
 *  - Size limit: the E step's work tables count (source block x target tile)
 *    units in 32-bit integers; a problem (or a context's capacity) with more
 *    than 2^30 units in its finest tiling, sum over pairs of
 *    ceil(N_i / 128) ceil(M_i / 128), is rejected with EINVAL (a single pair
 *    of N = M = 4,000,000 is within the limit).
 */
#ifndef LSGCPD_H_
#define LSGCPD_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lsgcpd_ctx lsgcpd_ctx;

typedef enum {
  LSGCPD_OK = 0,
  LSGCPD_EINVAL = 1,   /* invalid argument (size, range, NaN/Inf, null pointer) */
  LSGCPD_ENOMEM = 2,   /* device allocation failed or above the context capacity */
  LSGCPD_ECUDA = 3,    /* a CUDA runtime call failed */
  LSGCPD_ETIMEOUT = 4, /* a bounded device wait expired; results are invalid */
  LSGCPD_ENUMERIC = 5  /* the posterior mass vanished (all sources outliers) */
} lsgcpd_status;

/* Per-iteration trace record (lsgcpd_register):
 * sigma2 (after the update), N_P = sum P, Q_d(g_new), Newton steps, damped
 * steps, motion of the iteration (max(rotation angle, |dt| / diag)),
 * negative log-likelihood of Eq. (4) at the E step, outlier mass sum P_out. */
#define LSGCPD_TRACE_WIDTH 8

/* Per-source E-step output width (lsgcpd_estep `per_n`, see there). */
#define LSGCPD_PER_N_WIDTH 16

/* Global E-step moments returned by lsgcpd_estep (doubles):
 *   [0]      N_P = sum_n Pbar_n
 *   [1]      sum_n D_n
 *   [2..13]  H1 (3x4 row-major) = sum_n h_n xt_n^T
 *   [14..73] G = sum_n A_n (x) xt_n xt_n^T, A_n = Pbar_n I + W_n, 60 unique
 *            entries ordered by A pair (00,01,02,11,12,22) major and
 *            xt pair (00,01,02,03,11,12,13,22,23,33) minor
 *   [74]     sum_n Pout_n
 *   [75]     sum_n -log p(z_n) (Eq. (4)) at (R, t, sigma2)
 * with xt_n = [x_n; 1] in the caller's frame.  Per-source moments are
 * defined under lsgcpd_estep. */
#define LSGCPD_MOMENTS 76

typedef struct {
  double w;           /* outlier weight w0 in [0, 1) of Eq. (1); uniform w_n = w          */
  double alpha_max;   /* upper bound of the penalty, Eq. (3)                               */
  double lambda;      /* sensitivity of the penalty, Eq. (3)                               */
  double tol;         /* EM stops when an iteration moves less than tol; 0 = never         */
  double volume;      /* V of p_o = 1/V; <= 0 -> target AABB volume, sides >= 1e-2 diag   */
  double sigma2_init; /* <= 0 -> CPD start sum |g0 x_n - y_m|^2 / (3 N M)                  */
  double init_R[9];   /* initial g0 (identity by default); resuming = passing a prior g   */
  double init_t[3];
  double newton_tol;  /* inner Newton stop on |xi| (default 1e-12)                         */
  double sigma2_floor_rel; /* sigma^2 floor relative to diag^2 (default 1e-10); hitting it ends EM */
  int32_t knn_k;      /* neighbourhood size for normals and surface variation (default 10) */
  int32_t max_iters;  /* EM iterations (default 50)                                        */
  int32_t include_alpha_norm; /* 0: Eq. (9) as printed; 1: component constant with sqrt(1+alpha) */
  int32_t newton_max; /* inner Newton steps per M step (default 20)                       */
  int32_t precision;  /* 0: FP32 E step; 1: FP32 residuals with packed f16x2 exponentials
                         (per-source shifts; posteriors to ~1e-3 relative); 2: FP32 residuals and
                         exponentials, exponentials truncated to TF32 and the moment sums of
                         Eq. (9) (a product over the targets) on the tensor cores (tcgen05, TF32
                         operands with hi + lo features, FP32 accumulation; per-source moments to
                         ~2e-3 relative; lsgcpd_posteriors stays FP32) */
  int32_t knn_method; /* neighbour search: 0 auto (uniform grid above 50,000 targets in the largest
                         pair, brute force below), 1 brute force, 2 uniform grid; all give the same lists */
  /* Outlier weight from the outlier ratio (Sec. 3.2): eta in (0, 1) sets
   * w0 = w_max = eta V S / ((1 - eta) + eta V S), S = sum_m pi(m) c_m with c_m
   * the peak of component m, evaluated once at sigma^2_0 (overrides w);
   * 0 = use w. */
  double eta;
  /* Confidence filtering (Sec. 3.3): with phi_y, pi(m) = phi(y_m) / sum phi(y);
   * with phi_x, w_n = 1 - (1 - w0) phi(x_n).  Points whose phi is below
   * cf_threshold (> 0) are removed from X and Y before anything else
   * (neighbourhoods, sigma^2_0, V and the priors are those of the kept points).
   * phi_x / phi_y: N / M floats in (0, 1], in the same memory (host or device)
   * and with the same offsets as X / Y, or NULL (phi = 1).  Registration calls
   * only (lsgcpd_register, lsgcpd_register_batch) and lsgcpd_estep (no
   * truncation there). */
  double cf_threshold;
  /* Termination on the log-likelihood (Eq. (4)): > 0 stops EM after the M step
   * of the first iteration i >= 1 whose E step changed the NLL by at most
   * nll_tol |NLL_i|; 0 = off. */
  double nll_tol;
  const float* phi_x;
  const float* phi_y;
} lsgcpd_params;

/* Result of a registration (host struct filled by lsgcpd_register). */
typedef struct {
  double R[9];
  double t[3];
  double sigma2;
  int32_t iters;      /* EM iterations run */
  int32_t mode;       /* 0: uniform shift; 1: per-source shift (w = 0, extreme V, the Gaussian-constant
                         option, confidences or f16 exponentials) */
  double ms_estep;    /* device time of the E-step kernels (only with timing enabled) */
  double ms_total;    /* device time of the whole call (only with timing enabled)     */
} lsgcpd_result;

/* Fill *p with the defaults: w 0.1, alpha_max 2, lambda 0.2, tol 0, volume 0,
 * sigma2_init 0, identity g0, newton_tol 1e-12, floor 1e-10, k 10, 50
 * iterations, Eq. (9) constant, 20 Newton steps, FP32. */
void lsgcpd_params_default(lsgcpd_params* p);

/* Create a context on `device` able to handle up to max_N sources and max_M
 * targets (both >= 1).  Allocates all scratch memory up front; later calls
 * allocate nothing unless a larger size is requested.  *out is set on success. */
lsgcpd_status lsgcpd_create(lsgcpd_ctx** out, int device, int64_t max_N, int64_t max_M);

/* Release every resource of the context (NULL is ignored). */
void lsgcpd_destroy(lsgcpd_ctx* ctx);

/* Message of the last failed call on ctx (never NULL; "" after success). */
const char* lsgcpd_last_error(const lsgcpd_ctx* ctx);

/* Enable (1) or disable (0) device timing with CUDA events; results appear in
 * lsgcpd_result.ms_* and lsgcpd_last_timing(). */
lsgcpd_status lsgcpd_set_timing(lsgcpd_ctx* ctx, int enable);

/* Figures of the last call.  Device times in ms (timing enabled only):
 * [0] total, [1] E-step kernels, [2] combine + reduction kernels, [3] M-step
 * kernels, [4] preprocessing and initialisation.  Always: [5] kernel launches,
 * [6] bytes copied host -> device, [7] bytes copied device -> host.
 * Returns EINVAL (after filling out) if timing is off. */
lsgcpd_status lsgcpd_last_timing(const lsgcpd_ctx* ctx, double out[8]);

/* Local surface geometry of the target (Sec. 3.1, Eqs. (2)-(3)): for every
 * target m, its k nearest targets (self included, ties to the lower index,
 * FP32 squared distances), the neighbourhood covariance about its mean, the
 * smallest eigenpair (FP64 Jacobi), the surface variation
 * kappa_m = lambda_min / trace in [0, 1/3] and the penalty
 * alpha_m = alpha_max tanh(lambda (1/kappa_m - 3) / 2) of Eq. (3).
 *   Y       device, M x 3 FP32 (input)
 *   normals device, M x 3 FP32 (output, unit; the sign is arbitrary) or NULL
 *   kappa   device, M FP32 (output) or NULL
 *   alpha   device, M FP32 (output) or NULL
 *   knn_idx device, M x k int32 (output, ascending distance) or NULL
 * Uses p->knn_k, p->alpha_max, p->lambda.  Requires 1 <= k <= min(M, 32). */
lsgcpd_status lsgcpd_preprocess(lsgcpd_ctx* ctx, const float* Y, int64_t M, const lsgcpd_params* p,
                                float* normals, float* kappa, float* alpha, int32_t* knn_idx,
                                void* stream);

/* One E step (Eq. (5), computed as Eq. (9) with gamma_n = w/(1-w) (2 pi s2)^{3/2} / V)
 * at z_n = R x_n + t for the given target geometry, followed by the per-source
 * normalisation and the FP64 moment reduction consumed by the M step.
 *   X       device, N x 3 FP32 sources;  Y, normals (unit), alpha: device, target side
 *   R, t    host, the pose at which the posteriors are evaluated
 *   sigma2  > 0;  volume > 0 (V of p_o = 1/V)
 *   moments host, LSGCPD_MOMENTS doubles (output) or NULL
 *   per_n   device, N x LSGCPD_PER_N_WIDTH FP32 (output) or NULL, per source n,
 *           with r_mn = z_n - y_m and Lambda_m = I + alpha_m n_m n_m^T:
 *           [0] Pbar = sum_m P_mn, [1..3] h = sum_m P_mn Lambda_m r_mn,
 *           [4..9] W = sum_m P_mn alpha_m n_m n_m^T (00,01,02,11,12,22),
 *           [10] D = sum_m P_mn d_mn, d = r^T Lambda_m r, [11] Pout,
 *           [12] 1 / (S0_n + gamma'_n), the normaliser of the kernel's shifted
 *           exponentials, [13] gamma'_n (shifted outlier term), [14..15] 0.
 * Uses p->w (0 allowed: no outlier term) as w0, p->include_alpha_norm and the
 * optional confidences p->phi_x / p->phi_y (DEVICE arrays of N / M floats;
 * Sec. 3.3: pi(m) = phi_m / sum phi, w_n = 1 - (1 - w0) phi_n; no truncation
 * and no eta here). */
lsgcpd_status lsgcpd_estep(lsgcpd_ctx* ctx, const float* X, int64_t N, const float* Y,
                           const float* normals, const float* alpha, int64_t M,
                           const lsgcpd_params* p, const double R[9], const double t[3],
                           double sigma2, double volume, double* moments, float* per_n,
                           void* stream);

/* The dense posteriors of one E step (Eq. (5)), for checking and debugging
 * small problems: the E step of lsgcpd_estep (same arguments and rules), then
 *   P  device, (M + 1) x N FP32, row-major: P[m][n] = P_mn for m < M (the
 *      E step's own exponentials over its per-source normaliser), P[M][n] the
 *      outlier posterior of source n.  Columns sum to 1 up to FP32 rounding.
 * EINVAL if (M + 1) N exceeds 4e9. */
lsgcpd_status lsgcpd_posteriors(lsgcpd_ctx* ctx, const float* X, int64_t N, const float* Y,
                                const float* normals, const float* alpha, int64_t M,
                                const lsgcpd_params* p, const double R[9], const double t[3],
                                double sigma2, double volume, float* P, void* stream);

/* M step from the global moments of one E step (Eqs. (11)-(13) and the
 * sigma^2 update): Newton on SE(3) with the posteriors fixed, starting at
 * (R, t), with the damping / halving rules of the parameter block; then
 * sigma2 = Q_d(g_new) / (3 N_P) (no floor).  All arguments are host memory.
 * info (4 int32, may be NULL): Newton steps, damped steps, halvings, 0. */
lsgcpd_status lsgcpd_mstep(lsgcpd_ctx* ctx, const double* moments, const double R[9],
                           const double t[3], const lsgcpd_params* p, double R_out[9],
                           double t_out[3], double* sigma2_out, int32_t* info, void* stream);

/* Full registration: preprocessing of the target, initial sigma^2 and V,
 * then p->max_iters EM iterations (E step, moment reduction, Newton M step,
 * sigma^2 update) captured once per problem shape in a CUDA graph and
 * replayed.  X and Y may be HOST or DEVICE pointers (detected per pointer);
 * host inputs are copied into the context.  The optional confidences
 * (p->phi_x / p->phi_y, same memory as X / Y), confidence truncation
 * (p->cf_threshold), outlier ratio (p->eta) and likelihood termination
 * (p->nll_tol) apply as described at lsgcpd_params.  out receives the result
 * in the caller's frame.  trace (host, max_iters x LSGCPD_TRACE_WIDTH doubles)
 * may be NULL.  Returns ENUMERIC if the posterior mass vanished (result = last
 * pose). */
lsgcpd_status lsgcpd_register(lsgcpd_ctx* ctx, const float* X, int64_t N, const float* Y, int64_t M,
                              const lsgcpd_params* p, lsgcpd_result* out, double* trace,
                              void* stream);

/* Autotuning of the E step's source tile (on by default).  The hot kernel can
 * give each thread 4, 2 or 1 sources (source blocks of 1024, 256 or 128
 * sources): fewer sources per thread waste less padding on small or uneven
 * pairs, more share each target tile among more sources.  With autotuning on,
 * the first lsgcpd_register / lsgcpd_register_batch call for a problem shape
 * (the list of N_i, M_i) whose E step has at most 1.5e10 pairs times three
 * E-step launches of each variant on the caller's data (after a warm-up
 * launch) and keeps the fastest, unless the fixed rule's choice is within 2%
 * of it; later calls with the same shape reuse the choice.
 * With it off (or above the size limit) a fixed rule chooses.  The choice
 * changes only the FP32 summation order, so results within one context are
 * reproducible; two contexts can differ at FP32 rounding level.  The paper
 * has no counterpart (a GB300 scheduling choice).  enable: 0 or 1. */
lsgcpd_status lsgcpd_set_autotune(lsgcpd_ctx* ctx, int enable);

/* The plan of the last registration call: info[0] sources per thread,
 * info[1] sources per block, info[2] E-step CTAs, info[3] = 1 if the source
 * tile was chosen by measurement (this call or an earlier one with the same
 * shape).  tune_ms (may be NULL): measured ms per E-step launch for 4, 2 and 1
 * sources per thread (0 where not measured).  Host memory. */
lsgcpd_status lsgcpd_plan_info(const lsgcpd_ctx* ctx, int32_t info[4], double tune_ms[3]);

/* Persistent autotune cache (no counterpart in the paper).  save writes the
 * context's measured choices (problem shape -> sources per thread and the three
 * trial times) to a text file at `path` (UTF-8, one entry per line after a
 * header line), keyed by this device's name and SM count; EINVAL if the file
 * cannot be written.  load reads such a file and adds the entries written on
 * a device with the same name and SM count (others, and malformed lines, are
 * skipped), so that later calls with those shapes skip the trial launches;
 * *count (may be NULL) receives the number of entries added; EINVAL if the
 * file cannot be read or its header is not that of this format. */
lsgcpd_status lsgcpd_autotune_save(const lsgcpd_ctx* ctx, const char* path);
lsgcpd_status lsgcpd_autotune_load(lsgcpd_ctx* ctx, const char* path, int32_t* count);

/* Diagnostic of the failure path of the E step's copy pipeline (no
 * counterpart in the paper): one kernel waits, with the same bounded wait the
 * E step uses on its target-tile barriers, on a shared-memory barrier that
 * nothing completes; after budget_cycles (1 .. 4e9 GPU clocks) it gives up and
 * records the timeout.  Returns LSGCPD_ETIMEOUT when the wait ran out (the
 * expected result) and leaves the context usable; LSGCPD_OK would mean the
 * barrier completed.  Nothing faults, traps or hangs. */
lsgcpd_status lsgcpd_selftest_timeout(lsgcpd_ctx* ctx, int64_t budget_cycles);

/* Largest num_pairs of lsgcpd_register_batch. */
#define LSGCPD_MAX_PAIRS 65535

/* Many independent registrations (Sec. 3, applied to each pair on its own)
 * in one pass: every stage runs once over the whole batch, the E step as one
 * persistent launch whose work units (source block x target tile) are split
 * evenly over the SMs whatever the pair sizes, so that small and uneven pairs
 * still fill the GPU.  Pair i has sources X[n_off[i] .. n_off[i+1]) and
 * targets Y[m_off[i] .. m_off[i+1]) (rows of 3 floats, HOST or DEVICE
 * pointers); n_off / m_off (host, num_pairs + 1 entries, n_off[0] = m_off[0]
 * = 0, strictly increasing) give the offsets.  Each pair gets exactly the
 * computation lsgcpd_register would give it alone (its own centring, kNN
 * among its own targets, sigma^2_0, V, floor and convergence test); p is
 * shared and p->knn_k must not exceed any M_i.  The shift mode (fixed or
 * per-source) is chosen once for the batch: fixed only where it is safe for
 * every pair.  Outputs (host): R_out (num_pairs x 9, row-major), t_out
 * (num_pairs x 3), sigma2_out and iters_out (num_pairs each, may be NULL),
 * trace (num_pairs x max_iters x LSGCPD_TRACE_WIDTH, may be NULL).  Returns
 * EINVAL for an empty pair, bad offsets or num_pairs outside
 * [1, LSGCPD_MAX_PAIRS]; ENUMERIC if the posterior mass of any pair vanished
 * (every pair's result is still written). */
lsgcpd_status lsgcpd_register_batch(lsgcpd_ctx* ctx, int32_t num_pairs, const float* X,
                                    const int64_t* n_off, const float* Y, const int64_t* m_off,
                                    const lsgcpd_params* p, double* R_out, double* t_out,
                                    double* sigma2_out, int32_t* iters_out, double* trace,
                                    void* stream);

/* Size limits and scratch size of lsgcpd_estep_noalloc. */
#define LSGCPD_NOALLOC_MAX_N 4096
#define LSGCPD_NOALLOC_MAX_M 4096
#define LSGCPD_NOALLOC_ARENA_BYTES (16u << 20)

/* The E step of lsgcpd_estep for callers that cannot allocate device memory.
 * The paper has no counterpart: this is a deployment variant of the same
 * computation (same kernels, same results as lsgcpd_estep).
 *
 * Who needs it: code that runs while another framework owns the device memory
 * pool, latency-critical loops in which cudaMalloc/cudaFree would synchronise
 * the device, and integrations that must keep a fixed, known footprint.  It
 * takes no context (creating one allocates) and calls no cudaMalloc, cudaFree
 * or allocating library routine.  All scratch memory lives in one
 * LSGCPD_NOALLOC_ARENA_BYTES static device array that every GPU which loads
 * the library holds until the process exits.
 *
 * Arguments and outputs are those of lsgcpd_estep (X, Y, normals, alpha,
 * per_n: device memory of the calling thread's current device; R, t, moments:
 * host).  moments must not be NULL.  Returns EINVAL if N or M exceeds
 * LSGCPD_NOALLOC_MAX_N / LSGCPD_NOALLOC_MAX_M or an argument is invalid;
 * no error message is kept (there is no context).
 *
 * The first call on a device looks the arena's device address up
 * (cudaGetSymbolAddress) for that device; make that first call before any
 * stream capture.  Every call shares the one arena and leaves its contents
 * behind: concurrent or overlapping calls (other threads, other streams whose
 * work has not finished) race on it and must be serialised by the caller.
 * The call synchronises `stream` before returning.  The confidence fields of
 * the parameter block (phi_x, phi_y, cf_threshold) and eta are not used here:
 * uniform priors and outlier weight w. */
lsgcpd_status lsgcpd_estep_noalloc(const float* X, int64_t N, const float* Y, const float* normals,
                                   const float* alpha, int64_t M, const lsgcpd_params* p,
                                   const double R[9], const double t[3], double sigma2, double volume,
                                   double* moments, float* per_n, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LSGCPD_H_ */
