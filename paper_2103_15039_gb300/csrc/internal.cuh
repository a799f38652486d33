// Internal declarations shared by the CUDA translation units of liblsgcpd.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace lsg {

// ---------------------------------------------------------------------------
// Target records (one per target y_m, in the centred frame), stored tile-major
// and plane-minor so that a tile of kTile targets is one contiguous block that
// a single bulk copy moves into shared memory:
//   rec[tile][plane][kTile]
// planes: -y (3), a = sqrt(alpha) n (3), a a^T (00,01,02,11,12,22), l
// with l = log2 pi_m (+ 1/2 log2(1 + alpha_m) with the Gaussian constant).
// A padding target has l = -inf, so it contributes exactly 0.
// ---------------------------------------------------------------------------
constexpr int kPlanes = 13;
constexpr int kTile = 128;
constexpr int kTileFloats = kPlanes * kTile;
constexpr int kTileBytes = kTileFloats * 4;

// Per-source raw E-step moments accumulated by the hot kernel:
//   S0 = sum e, h (3) = sum e Lambda_m r (Lambda_m = I + a a^T), W (6) = sum e a a^T,
//   D' = sum e (d + kappa_n)
constexpr int kMom = 11;

// Global moments (see lsgcpd.h): N_P, sum D, H1 (12), G (60), sum Pout, NLL part.
constexpr int kGlob = 76;

// Status bits written by kernels (never traps).
constexpr int kStatusTimeout = 1;
constexpr int kStatusNumeric = 2;

// Device-resident EM state.  Written by the initialisation and M-step kernels,
// read by the E step, so that a whole EM loop runs without the host.
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
  double nll_const;     // per-source constant of -log p: -ln((1-w) (2 pi s2)^(-3/2)) at the E step
  double log2_V;        // log2 V
  double ln_1mw;        // ln(1 - w)
  int32_t done;         // EM finished (floor, tol or numeric failure)
  int32_t iter;         // iterations completed
  int32_t numeric_fail;
  int32_t pad0;
  // E-step constants for the current (R, t, sigma2):
  float Rf[9];
  float tf[3];
  float neg_c;          // -log2(e) / (2 sigma2)
  float kap;            // uniform shift in distance units, L / c  (fixed-shift mode)
  float L;              // uniform log2 shift (fixed-shift mode): log2 gamma
  float pad1;
};

// E-step constants for the current (R, t, sigma2) of the state.  The shift L
// and the logarithms feed FP32 arithmetic only, so they are evaluated in FP32.
__device__ inline void set_estep_constants(EmState* st) {
  const float s2 = static_cast<float>(st->sigma2);
  const float lg = log2f(6.2831853f * s2);
  const float L = static_cast<float>(st->log2_wodds) + 1.5f * lg - static_cast<float>(st->log2_V);
  for (int i = 0; i < 9; ++i) st->Rf[i] = static_cast<float>(st->R[i]);
  for (int i = 0; i < 3; ++i) st->tf[i] = static_cast<float>(st->t[i]);
  st->neg_c = -1.44269504f / (2.f * s2);  // -log2(e) / (2 s2)
  st->L = L;
  st->kap = L * (2.f * s2) * 0.69314718f;  // L / c
  st->nll_const = -st->ln_1mw + 1.5 * 0.6931471805599453 * static_cast<double>(lg);
}

// Scalar parameters the device needs (a subset of lsgcpd_params, plus sizes).
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
  int32_t pad;
};

// Launch plan of the hot E-step kernel: a stream-K style split of
// (source block) x (target tile) units over a grid sized to the SM count.
// A CTA flushes its partial moments into a new slot at every source-block
// boundary and every seg_cap tiles.  Slots are numbered CTA-major, so all
// slots of one source block are contiguous.  `table` holds, for the device:
//   [0, grid]                first slot of every CTA (prefix sums)
//   [grid+1, grid+1+2*blocks) (first slot, slot count) of every source block
struct EstepPlan {
  int S;               // sources per thread
  int NW;              // warps per CTA
  int SB;              // sources per block = NW * 32 * S
  int num_blocks;      // ceil(N / SB)
  int num_tiles;       // ceil(M / kTile)
  long long units;     // num_blocks * num_tiles
  int grid;            // CTAs (<= units)
  int seg_cap;         // flush after this many tiles (FP32 sums stay short)
  int total_slots;
  size_t smem_bytes;
  std::vector<int> table;
};

// ----- kernels / launchers (estep.cu) -------------------------------------
EstepPlan plan_estep(int64_t N, int64_t M, int num_sms, int S_override);
size_t estep_partial_floats(const EstepPlan& p);
cudaError_t launch_estep(const EstepPlan& p, const float4* xs, const float* rec, const EmState* st,
                         const float* kap_n, float* part, const int* table, int* status,
                         cudaStream_t s);
cudaError_t launch_shift(const EstepPlan& p, const float4* xs, const float* rec, const EmState* st,
                         int64_t N, float* kap_n, float* gam_n, cudaStream_t s);
// rows of FP64 partial global moments written by the combine kernel
int combine_rows(int64_t N, int num_sms);
cudaError_t launch_combine(const EstepPlan& p, const float4* xs, int64_t N, const float* part,
                           const int* table, const EmState* st, const float* kap_n,
                           const float* gam_n, double* rows, int nrows, float* per_n,
                           cudaStream_t s);
// Sum the rows (fixed order, FP64) into kGlob moments; one warp per moment.
cudaError_t launch_final_reduce(const double* rows, int nrows, double* mom, const EmState* st,
                                cudaStream_t s);

// ----- M step (mstep.cu) -------------------------------------------------------
// Newton M step from the kGlob global moments `mom` and the state update.
cudaError_t launch_mstep(const double* mom, EmState* st, const DevParams& dp, double* trace,
                         cudaStream_t s);
// Standalone M step: io[0..75] moments, io[80..91] starting pose (R, t);
// results R (9), t (3), sigma2, Q, newton steps, damped, halvings at io[96..112].
cudaError_t launch_mstep_standalone(double* io, const DevParams& dp, cudaStream_t s);

// ----- preprocessing / initialisation (prep.cu) ------------------------------
int stats_blocks(int64_t n);
cudaError_t launch_init(const float* X, int64_t N, const float* Y, int64_t M, const DevParams& dp,
                        double* red, EmState* st, float4* xs, int64_t n_pad, cudaStream_t s);
cudaError_t launch_center_only(const float* X, int64_t N, const float* Y, int64_t M, double* red,
                               EmState* st, float4* xs, int64_t n_pad, cudaStream_t s);
cudaError_t launch_knn(const float* Y, int64_t M, int k, float4* y4, float* part_d, int* part_i,
                       int* idx_out, int splits, cudaStream_t s);
int knn_splits(int64_t M, int num_sms);
cudaError_t launch_geometry(const float* Y, int64_t M, const int* idx, int k, double alpha_max,
                            double lambda, int alpha_norm, const EmState* st, float* rec,
                            int num_tiles, float* normals, float* kappa, float* alpha,
                            cudaStream_t s);
cudaError_t launch_pack(const float* Y, const float* normals, const float* alpha, int64_t M,
                        int alpha_norm, const EmState* st, float* rec, int num_tiles,
                        cudaStream_t s);
cudaError_t launch_estep_constants(EmState* st, double sigma2, double w, double V,
                                   const double* R, const double* t, cudaStream_t s);

}  // namespace lsg
