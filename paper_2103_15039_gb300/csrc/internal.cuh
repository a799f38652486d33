// Internal declarations shared by the CUDA translation units of liblsgcpd.
//
// Every kernel works on a batch of P independent registration pairs (a single
// registration is a batch of one).  Pair i has N_i sources and M_i targets;
// the raw inputs are concatenated (offsets n_off / m_off), sources are padded
// per pair to whole source blocks of SB and targets to whole tiles of kTile.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace lsg {

// ---------------------------------------------------------------------------
// Target records (one per target y_m, in its pair's centred frame), stored
// tile-major and plane-minor so that a tile of kTile targets is one contiguous
// block that a single bulk copy moves into shared memory:
//   rec[tile][plane][kTile]
// planes 0-3 are rewritten before every E step for the current sigma^2 (the
// E step works in coordinates scaled by sqrt(c), c = log2(e) / (2 sigma^2), so
// that c d_mn is a plain sum of squares):
//   0-2  -sqrt(c) y
//   3    lambda_m: L - l_m with the uniform shift L, or -l_m with per-source shifts
//   4-6  a = sqrt(alpha) n
//   7-12 a a^T (00,01,02,11,12,22)
//   13-15 b = Lambda_m y = y + (a . y) a
// with l_m = log2 pi_m (+ 1/2 log2(1 + alpha_m) with the Gaussian constant).
// A padding target has lambda = kPadLambda, so it contributes exactly 0.
// The unscaled centred y and l_m of every record slot are kept in yl[slot]
// (float4; l = -inf marks padding).
// ---------------------------------------------------------------------------
constexpr int kPlanes = 16;
constexpr int kTile = 128;
constexpr int kTileFloats = kPlanes * kTile;
constexpr int kTileBytes = kTileFloats * 4;
constexpr float kPadLambda = 1e30f;

// Per-source raw E-step moments accumulated by the hot kernel (e = 2^-q,
// q = c d + lambda_m [+ L_n]):
//   S0 = sum e, B (3) = sum e b_m, W (6) = sum e a a^T, Dq = sum e q,
//   El = sum e lambda_m (per-source shift mode only)
constexpr int kMom = 12;

// Global moments per pair (see lsgcpd.h): N_P, sum D, H1 (12), G (60), sum Pout, NLL.
constexpr int kGlob = 76;

// Sources per combine CTA (a divisor of every source block size).
constexpr int kCombineSources = 128;

// Status bits written by kernels (never traps).
constexpr int kStatusTimeout = 1;
constexpr int kStatusNumeric = 2;

// Device-resident EM state of one pair.  Written by the initialisation and
// M-step kernels, read by the E step, so that a whole EM loop runs without the
// host.
struct EmState {
  double R[9];          // current g in the centred frame
  double t[3];
  double sigma2;
  double sigma2_floor;
  double V;             // volume of the outlier density
  double diag;          // target AABB diagonal
  double log2_wodds;    // log2(w / (1 - w)); -inf when w = 0
  double mu_x[3];       // source centroid
  double mu_y[3];       // target centroid
  double ylo[3];        // target AABB (caller's frame)
  double yhi[3];
  double nll_const;     // per-source constant of -log p: -ln((1-w) (2 pi s2)^(-3/2)) at the E step
  double log2_V;        // log2 V
  double ln_1mw;        // ln(1 - w)
  double log2_pi;       // -log2 sum_m phi_m: log2 pi_m = log2 phi_m + log2_pi (uniform: -log2 M)
  double w0;            // outlier weight w0 (given, or from the outlier ratio)
  double nll_prev;      // NLL of the previous E step (termination on the likelihood)
  int32_t done;         // EM finished (floor, tol or numeric failure)
  int32_t iter;         // iterations completed
  int32_t numeric_fail;
  int32_t pad0;
  // E-step constants for the current (R, t, sigma2):
  float Rf[9];
  float tf[3];
  float neg_c;          // -c = -log2(e) / (2 sigma2)
  float L;              // log2 gamma: the uniform log2 shift (-inf without outlier term)
  float sqc;            // sqrt(c): the E step's coordinate scale
  float lam;            // L - log2 pi: lambda_m of every target in the uniform-shift mode
  float Lb;             // 1.5 log2(2 pi s2) - log2 V: log2 gamma_n = log2(w_n / (1 - w_n)) + Lb
  float pad1;
};

// E-step constants for the current sigma2 (FP32: they feed FP32 arithmetic only).
__device__ inline void set_sigma_constants(EmState* st, float s2) {
  const float lg = log2f(6.2831853f * s2);
  const float Lb = 1.5f * lg - static_cast<float>(st->log2_V);
  const float L = static_cast<float>(st->log2_wodds) + Lb;
  st->Lb = Lb;
  const float c = 1.44269504f / (2.f * s2);  // log2(e) / (2 s2)
  st->neg_c = -c;
  st->L = L;
  st->sqc = sqrtf(c);
  st->lam = L - static_cast<float>(st->log2_pi);
  st->nll_const = -st->ln_1mw + 1.5 * 0.6931471805599453 * static_cast<double>(lg);
}

// The sigma-dependent planes 0-3 of record slot `lane` of tile `tile` (y scaled by
// -sqrt(c), lambda = L - l or -l): written by the prescale kernel, or by the M step of the
// previous iteration for small problems.
__device__ inline void prescale_slot(float* rec, const float4* yl, long long tile, int lane, float sqc, float L,
                                     int mode) {
  const float4 y = yl[tile * kTile + lane];
  const bool pad = y.w == -INFINITY;
  float* r = rec + static_cast<size_t>(tile) * kTileFloats + lane;
  r[0 * kTile] = pad ? 0.f : -sqc * y.x;
  r[1 * kTile] = pad ? 0.f : -sqc * y.y;
  r[2 * kTile] = pad ? 0.f : -sqc * y.z;
  r[3 * kTile] = pad ? kPadLambda : (mode ? -y.w : L - y.w);
}

// E-step constants for the current (R, t, sigma2) of the state.
__device__ inline void set_estep_constants(EmState* st) {
  for (int i = 0; i < 9; ++i) st->Rf[i] = static_cast<float>(st->R[i]);
  for (int i = 0; i < 3; ++i) st->tf[i] = static_cast<float>(st->t[i]);
  set_sigma_constants(st, static_cast<float>(st->sigma2));
}

// Scalar parameters the device needs (a subset of lsgcpd_params).
struct DevParams {
  double w;
  double volume;
  double sigma2_init;
  double init_R[9];
  double init_t[3];
  double newton_tol;
  double sigma2_floor_rel;
  double tol;
  int32_t newton_max;
  int32_t include_alpha_norm;
  int32_t max_iters;
  int32_t cf_x;         // per-source confidences phi_x present (carried in xs[n].w)
  double eta;           // > 0: w0 from the outlier ratio
  double nll_tol;       // > 0: stop on a small relative NLL change
};

// ---------------------------------------------------------------------------
// Batch geometry: sizes, layouts and the E step's stream-K work split.
//
// Work = (source block) x (target tile of the block's pair) units, ordered
// block-major, split into `grid` contiguous ranges (one per CTA).  A CTA
// flushes its partial moments into a new slot at every source-block boundary
// and every seg_cap tiles; slots are numbered CTA-major, so all slots of one
// source block are contiguous.
//
// Device int32 table (offsets in Geo):
//   blk_off[P+1]    first source block of each pair
//   tile_off[P+1]   first target tile of each pair
//   block_pair[B]   pair of each source block
//   unit_off[B+1]   first unit of each source block
//   cta_slot[G+1]   first partial slot of each CTA
//   cta_block[G]    source block of each CTA's first unit
//   block_slot[2B]  (first slot, slot count) of each source block
//   tile_pair[T]    pair of each target tile
// Device int64 table: n_off[P+1], m_off[P+1] (offsets of the raw inputs).
// ---------------------------------------------------------------------------
struct Geo {
  int P;
  int S;               // sources per thread of the E step
  int SB;              // sources per source block
  int B;               // source blocks
  int T;               // target tiles
  int grid;            // E-step CTAs
  int seg_cap;
  int max_tiles;       // largest tile count of one pair
  int max_blocks;      // largest source-block count of one pair
  long long U;         // units
  long long max_n;     // largest N_i
  long long max_m;     // largest M_i
  int o_blk_off, o_tile_off, o_block_pair, o_unit_off, o_cta_slot, o_cta_block, o_block_slot, o_tile_pair;
  int total_slots;
  int combine_ctas;    // B * SB / kCombineSources
};

struct BatchPlan {
  Geo g;
  std::vector<int> tab;
  std::vector<long long> off64;  // n_off[P+1], m_off[P+1]
  size_t smem_bytes;
};

// Upper limit of the plan's 32-bit tables: (source block x target tile) units and tiles.
constexpr long long kMaxPlanUnits = 1LL << 30;
// True when every pair has N, M >= 1 and the plan of the batch stays within kMaxPlanUnits
// for every source tile (a single pair of N = M = 4,000,000 fits; about 4.2 million does not).
bool plan_fits(const std::vector<long long>& N, const std::vector<long long>& M);
// Plan a batch (sizes N[i], M[i]); S_override in {1, 2, 4} forces the
// sources per thread, 0 chooses.  seg_cap: target tiles a CTA sums into one
// partial slot at most (the length of an FP32 accumulation run).
constexpr int kSegCap = 64;
BatchPlan plan_batch(const std::vector<long long>& N, const std::vector<long long>& M, int num_sms,
                     int S_override, int seg_cap = kSegCap);
size_t estep_partial_floats(const Geo& g);
// Resident CTAs per SM and warps per CTA of the FP32 E-step kernel with S sources per thread.
int estep_resident_ctas(int S);
int estep_warps(int S);
size_t estep_smem_bytes();  // dynamic shared memory of the FP32 E-step kernel

// ----- programmatic dependent launch (the captured EM loop) ----------------
// While the EM loop is captured, its kernels are launched with programmatic
// stream serialisation: a kernel may be scheduled while its predecessor
// finishes, and waits for the predecessor's completion (hence for everything
// before it) before its first memory access (pdl_wait).  Kernels launched
// without the attribute pass pdl_wait at once.
void set_pdl(bool on);  // launches of this host thread use the attribute while on
bool pdl_on();

template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  if (pdl_on()) {
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// let the next kernel of the stream be scheduled (it still waits in pdl_wait for this one)
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
#endif

// Device pointers of a batch.
struct Dev {
  const int* tab;
  const long long* off64;
  EmState* st;         // [P]
  int* done_count;     // number of pairs whose EM loop has finished
};

// ----- E step (estep.cu) --------------------------------------------------------
// Shift modes: 0 = uniform shift L (fixed), 1 = per-source shift L_n (shift pass).
// Rewrite the sigma-dependent record planes 0-3 from yl for the current state.
cudaError_t launch_prescale(const BatchPlan& p, const Dev& d, const float4* yl, int mode, float* rec,
                            cudaStream_t s);
// mode 1 only: L_n and gamma'_n of every source (cf_x: per-source w_n from xs[n].w): a
// max pass of the E-step kernel (partials in part, overwritten by the E step after it)
// and a per-source finalisation.
cudaError_t launch_shift(const BatchPlan& p, const Dev& d, const float4* xs, const float* rec, int cf_x,
                         float* part, int* status, float* ls_n, float* gam_n, cudaStream_t s);
// half (mode 1 only): exponentials as packed f16x2 (the mixed-precision variant).
cudaError_t launch_estep(const BatchPlan& p, const Dev& d, const float4* xs, const float* rec, int mode, int half,
                         const float* ls_n, float* part, int* status, cudaStream_t s);
// ----- E step with the moment contraction on tcgen05 (estep_tc.cu) -----------------
// Feature tiles (the B operand: b, a a^T, lambda split hi + lo in TF32) of every
// record slot, built once from the static record planes; floats for a plan.
size_t tc_feature_floats(const Geo& g);
cudaError_t launch_features(const BatchPlan& p, const float* rec, const float4* yl, float* feat, cudaStream_t s);
// Same partial moments as launch_estep with 4 sources per thread (p.g.SB must be
// 1024), exponentials truncated to TF32; mode 0 or 1 (after launch_shift).
cudaError_t launch_estep_tc(const BatchPlan& p, const Dev& d, const float4* xs, const float* rec, const float* feat,
                            int mode, const float* ls_n, float* part, int* status, cudaStream_t s);
cudaError_t launch_combine(const BatchPlan& p, const Dev& d, const float4* xs, const float* part, int mode,
                           int cf_x, const float* ls_n, const float* gam_n, double* rows, float* per_n,
                           cudaStream_t s);
// Dense posteriors (M + 1) x N of a single pair after its E step (per_n from the combine).
cudaError_t launch_posteriors(const float4* xs, const float* rec, const EmState* st, const float* ls_n, int mode,
                              int half, const float* per_n, long long N, long long M, float* P, cudaStream_t s);
// Diagnostic wait on a barrier nothing completes, bounded by `budget` cycles.
cudaError_t launch_wait_selftest(long long budget, int* status, cudaStream_t s);
// Sum each pair's combine rows (fixed order, FP64) into mom[P][kGlob]; one warp per moment.
cudaError_t launch_final_reduce(const BatchPlan& p, const Dev& d, const double* rows, double* mom,
                                cudaStream_t s);

// ----- M step (mstep.cu) -------------------------------------------------------
// Newton M step of every pair from mom[P][kGlob] and the state update; trace [P][iters][8].
// rows != nullptr: the kernel first sums each pair's combine rows itself (fixed order,
// FP64) into mom, in place of launch_final_reduce (for plans where mstep_sums_rows holds).
// yl != nullptr: the kernel also writes the next E step's sigma-dependent record planes
// (in place of launch_prescale; for plans where mstep_prescales holds).
cudaError_t launch_mstep(const BatchPlan& p, const Dev& d, const double* rows, double* mom, const DevParams& dp,
                         double* trace, int trace_iters, const float4* yl, int mode, float* rec, cudaStream_t s);
// Combine rows per pair small enough for the M-step kernel to sum them (a chain of at most
// kMaxFusedRows FP64 adds per moment costs less than one more kernel boundary per iteration).
constexpr int kMaxFusedRows = 32;
inline bool mstep_sums_rows(const Geo& g) { return g.max_blocks * (g.SB / kCombineSources) <= kMaxFusedRows; }
// Target tiles per pair small enough for the M-step CTA (one thread per slot) to prescale
// faster than a separate launch (measured: ahead at 8 tiles, behind at 32).
constexpr int kMaxFusedTiles = 16;
inline bool mstep_prescales(const Geo& g) { return mstep_sums_rows(g) && g.max_tiles <= kMaxFusedTiles; }
// Standalone M step: io[0..75] moments, io[80..91] starting pose (R, t);
// results R (9), t (3), sigma2, Q, newton steps, damped, halvings at io[96..112].
cudaError_t launch_mstep_standalone(double* io, const DevParams& dp, cudaStream_t s);
// E-step constants of pair 0 for a pose given in the caller's frame (centroids known).
cudaError_t launch_estep_constants(EmState* st, double sigma2, double w, double V, const double* R,
                                   const double* t, cudaStream_t s);

// ----- preprocessing / initialisation (prep.cu) ------------------------------
// Rows of the statistics reductions per pair.
int stats_chunks(const Geo& g);
// Centroids, AABB, V, floor and centred sources of every pair; with `full`, also
// sigma^2_0 and the initial EM state (otherwise only what the standalone E step
// and the preprocessing need).
// phi_x / phi_y (device, same offsets as X / Y) may be NULL (phi = 1); phi_x goes
// to xs[n].w, sum phi_y sets the normalisation of pi(m).
cudaError_t launch_init(const BatchPlan& p, const Dev& d, const float* X, const float* Y, const float* phi_x,
                        const float* phi_y, const DevParams& dp, bool full, double* red, float4* xs,
                        cudaStream_t s);
int knn_splits(const Geo& g, int num_sms);
// Exact kNN through a uniform grid per pair (same lists as launch_knn: FP32
// distances, (distance, index) order).  Cells of pair i occupy
// [4 m_off[i] + 64 i, 4 m_off[i+1] + 64 (i+1)) of the cell arrays.
long long knn_grid_cells(long long Mtot, int P);
struct GridBufs {
  int* count;      // [cells] points per cell
  int* start;      // [cells + 1] exclusive prefix of count (global sorted position)
  int* fill;       // [cells] scatter cursor
  int* cell_of;    // [Mtot] cell of every target
  float4* sorted;  // [Mtot] targets sorted by cell, w = pair-local index (bits)
  int* scan_tmp;   // [scan blocks] block sums
  double* info;    // [P][8] grid origin (3), cell edge, dims (3)
};
size_t knn_grid_scan_blocks(long long cells);
cudaError_t launch_knn_grid(const BatchPlan& p, const Dev& d, const float* Y, int k, const GridBufs& gb,
                            int* idx_out, cudaStream_t s);
cudaError_t launch_knn(const BatchPlan& p, const Dev& d, const float* Y, int k, int splits, float4* y4,
                       float* part_d, int* part_i, int* idx_out, cudaStream_t s);
// Outlier weight from the outlier ratio (per pair, after the records exist):
// w0 = eta V S / ((1 - eta) + eta V S), S = c0 sum_m 2^(l_m), then the E-step constants.
cudaError_t launch_eta(const BatchPlan& p, const Dev& d, const float4* yl, double eta, cudaStream_t s);
// Stable per-pair compaction of rows (x, y, z) whose phi >= threshold.  Pass 1
// counts kept rows per (pair, chunk) into cnt[P][chunks]; pass 2 scatters with
// the exclusive per-pair chunk offsets coff[P][chunks] (from the host) into
// out rows at out_off[pair] + coff + rank, and phi into phi_out.
int compact_chunks(long long max_rows);
cudaError_t launch_compact_count(const float* phi, const long long* off, int P, int chunks, float threshold,
                                 int* cnt, cudaStream_t s);
cudaError_t launch_compact_scatter(const float* rows, const float* phi, const long long* off,
                                   const long long* out_off, const int* coff, int P, int chunks, float threshold,
                                   float* rows_out, float* phi_out, cudaStream_t s);
// Both write the static record planes 4-15 and yl.
cudaError_t launch_geometry(const BatchPlan& p, const Dev& d, const float* Y, const float* phi_y, const int* idx,
                            int k, double alpha_max, double lambda, int alpha_norm, float* rec, float4* yl,
                            float* normals, float* kappa, float* alpha, cudaStream_t s);
cudaError_t launch_pack(const BatchPlan& p, const Dev& d, const float* Y, const float* phi_y, const float* normals,
                        const float* alpha, int alpha_norm, float* rec, float4* yl, cudaStream_t s);

}  // namespace lsg
