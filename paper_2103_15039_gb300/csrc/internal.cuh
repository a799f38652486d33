// Internal declarations shared by the CUDA translation units of liblsgcpd.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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
//   S0 = sum e, rho (3) = sum e r, W (6) = sum e a a^T, beta (3) = sum e (a.r) a,
//   D' = sum e (d + kappa_n)
constexpr int kMom = 14;

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
struct EstepPlan {
  int S;               // sources per thread
  int NW;              // warps per CTA
  int SB;              // sources per block = NW * 32 * S
  int num_blocks;      // ceil(N / SB)
  int num_tiles;       // ceil(M / kTile)
  int64_t units;       // num_blocks * num_tiles
  int grid;            // CTAs (<= units)
  int seg_cap;         // flush after this many tiles (FP32 sums stay short)
  int segs_max;        // partial slots per CTA
  size_t smem_bytes;
};

// ----- kernels / launchers (estep.cu) -------------------------------------
EstepPlan plan_estep(int64_t N, int64_t M, int num_sms, int S_override);
size_t estep_partial_floats(const EstepPlan& p);
cudaError_t launch_estep(const EstepPlan& p, const float4* xs, const float* rec, const EmState* st,
                         const float* kap_n, float* part, int* part_meta, int* status,
                         cudaStream_t s);
cudaError_t launch_shift(const EstepPlan& p, const float4* xs, const float* rec, const EmState* st,
                         int64_t N, float* kap_n, float* gam_n, cudaStream_t s);
int combine_blocks(int64_t N);
cudaError_t launch_combine(const EstepPlan& p, const float4* xs, int64_t N, const float* part,
                           const int* part_meta, const EmState* st, const float* kap_n,
                           const float* gam_n, double* blk, float* per_n, cudaStream_t s);

// ----- M step (mstep.cu) -------------------------------------------------------
// Reduce `nblk` partial moment rows, run the Newton M step and update the state.
// mode_tail: 1 = full EM iteration (update state, trace, E-step constants);
//            0 = standalone M step (write results to `out`).
cudaError_t launch_mstep(const double* blk, int nblk, EmState* st, const DevParams& dp,
                         double* trace, double* out, int standalone, cudaStream_t s);
// Sum `nblk` partial moment rows into `out` (kGlob doubles), fixed order.
cudaError_t launch_reduce_moments(const double* blk, int nblk, double* out, cudaStream_t s);

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
