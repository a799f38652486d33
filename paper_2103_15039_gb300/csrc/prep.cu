// Preprocessing and initialisation kernels of LSG-CPD on sm_103a.
//
//  * statistics + centring: FP64 centroids of both clouds, the target's axis-
//    aligned box (V of the outlier density p_o = 1/V, sides clamped below at
//    1e-2 of the diagonal), the CPD start value of sigma^2
//    sum_mn |g0 x_n - y_m|^2 / (3 N M) in closed form, and FP32 centred copies;
//  * k nearest neighbours of every target (self included): exact brute force
//    over shared-memory candidate tiles, FP32 squared distances
//    fma(dz, dz, fma(dy, dy, dx * dx)), ties to the lower index, the candidate
//    range split over several CTAs and the sorted partial lists merged;
//  * local surface geometry (Sec. 3.1, Eqs. (2)-(3)): FP64 covariance of the
//    neighbourhood about its mean, cyclic Jacobi for the smallest eigenpair,
//    surface variation kappa = lambda_min / trace, penalty
//    alpha = alpha_max tanh(lambda (1/kappa - 3) / 2), packed into the
//    E step's tile-major target records.
#include <math.h>

#include "internal.cuh"

namespace lsg {
namespace {

constexpr int kStatThreads = 256;
constexpr int kStatChunk = kStatThreads * 2;  // points per statistics CTA

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block reduction of NV values with per-value operation op (0 sum, 1 min, 2 max).
template <int NV>
__device__ void block_reduce(double (&v)[NV], const int (&op)[NV], double* out_row) {
  __shared__ double sh[kStatThreads / 32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double x = v[j];
    x = op[j] == 0 ? warp_sum_d(x) : (op[j] == 1 ? warp_min_d(x) : warp_max_d(x));
    if (lane == 0) sh[warp][j] = x;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    const int j = threadIdx.x;
    double x = sh[0][j];
    for (int w = 1; w < kStatThreads / 32; ++w)
      x = op[j] == 0 ? x + sh[w][j] : (op[j] == 1 ? fmin(x, sh[w][j]) : fmax(x, sh[w][j]));
    out_row[j] = x;
  }
}

// Pass 1 (per pair, per chunk of kStatChunk points): sum x (3), sum y (3),
// min y (3), max y (3), sum phi_y.  grid = (chunks, P).
constexpr int kRaw = 13;
__global__ void __launch_bounds__(kStatThreads) raw_stats_kernel(const float* __restrict__ X, const float* __restrict__ Y,
                                                                 const float* __restrict__ phi_y,
                                                                 const long long* __restrict__ off64, int P,
                                                                 double* __restrict__ red) {
  const int pair = blockIdx.y;
  const long long n0 = off64[pair], N = off64[pair + 1] - n0;
  const long long m0 = off64[P + 1 + pair], M = off64[P + 1 + pair + 1] - m0;
  const long long c0 = static_cast<long long>(blockIdx.x) * kStatChunk;
  if (c0 >= (N > M ? N : M)) return;
  double v[kRaw];
  const int op[kRaw] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 2, 2, 2, 0};
  for (int j = 0; j < 6; ++j) v[j] = 0.0;
  for (int j = 6; j < 9; ++j) v[j] = INFINITY;
  for (int j = 9; j < 12; ++j) v[j] = -INFINITY;
  v[12] = 0.0;
  for (long long i = c0 + threadIdx.x; i < c0 + kStatChunk; i += kStatThreads) {
    if (i < N) {
      const float* x = X + 3 * (n0 + i);
      v[0] += x[0];
      v[1] += x[1];
      v[2] += x[2];
    }
    if (i < M) {
      const float* y = Y + 3 * (m0 + i);
      const double a = y[0], b = y[1], c = y[2];
      v[3] += a;
      v[4] += b;
      v[5] += c;
      v[6] = fmin(v[6], a);
      v[7] = fmin(v[7], b);
      v[8] = fmin(v[8], c);
      v[9] = fmax(v[9], a);
      v[10] = fmax(v[10], b);
      v[11] = fmax(v[11], c);
      v[12] += phi_y ? static_cast<double>(phi_y[m0 + i]) : 1.0;
    }
  }
  block_reduce<kRaw>(v, op, red + (static_cast<size_t>(pair) * gridDim.x + blockIdx.x) * kRaw);
}

// Finalise pass 1 per pair (grid = P, one warp per value): centroids, V,
// diagonal and sigma^2 floor.
__global__ void finalize_raw_kernel(const double* __restrict__ red, int chunks, const long long* __restrict__ off64,
                                    int P, double volume, double floor_rel, EmState* __restrict__ st_all) {
  __shared__ double v[kRaw];
  const int pair = blockIdx.x;
  const long long N = off64[pair + 1] - off64[pair];
  const long long M = off64[P + 1 + pair + 1] - off64[P + 1 + pair];
  const long long big = N > M ? N : M;
  const int nchunk = static_cast<int>((big + kStatChunk - 1) / kStatChunk);
  const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (j < kRaw) {
    const int op = (j < 6 || j == 12) ? 0 : (j < 9 ? 1 : 2);
    double x = op == 0 ? 0.0 : (op == 1 ? INFINITY : -INFINITY);
    for (int b = lane; b < nchunk; b += 32) {
      const double r = red[(static_cast<size_t>(pair) * chunks + b) * kRaw + j];
      x = op == 0 ? x + r : (op == 1 ? fmin(x, r) : fmax(x, r));
    }
    x = op == 0 ? warp_sum_d(x) : (op == 1 ? warp_min_d(x) : warp_max_d(x));
    if (lane == 0) v[j] = x;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  EmState* st = st_all + pair;
  for (int c = 0; c < 3; ++c) {
    st->mu_x[c] = v[c] / static_cast<double>(N);
    st->mu_y[c] = v[3 + c] / static_cast<double>(M);
  }
  double s[3], d2 = 0.0;
  for (int c = 0; c < 3; ++c) {
    s[c] = v[9 + c] - v[6 + c];
    d2 += s[c] * s[c];
  }
  const double diag = sqrt(d2);
  double V = 1.0;
  for (int c = 0; c < 3; ++c) V *= fmax(s[c], 1e-2 * diag);
  st->diag = diag;
  for (int c = 0; c < 3; ++c) {
    st->ylo[c] = v[6 + c];
    st->yhi[c] = v[9 + c];
  }
  st->log2_pi = -log2(v[12]);  // pi(m) = phi_m / sum phi (phi = 1: 1 / M)
  st->V = volume > 0.0 ? volume : V;
  st->sigma2_floor = floor_rel * diag * diag;
}

// Pass 2 (grid = (chunks, P)): centred FP32 sources as float4 (zero padding up
// to the pair's whole source blocks) and sums of the centred clouds:
// sum xc (3), sum |xc|^2, sum yc (3), sum |yc|^2.
__global__ void __launch_bounds__(kStatThreads) center_kernel(const float* __restrict__ X, const float* __restrict__ Y,
                                                              const float* __restrict__ phi_x,
                                                              const long long* __restrict__ off64,
                                                              const int* __restrict__ tab, Geo g,
                                                              const EmState* __restrict__ st_all,
                                                              float4* __restrict__ xs, double* __restrict__ red) {
  const int pair = blockIdx.y;
  const int P = g.P;
  const long long n0 = off64[pair], N = off64[pair + 1] - n0;
  const long long m0 = off64[P + 1 + pair], M = off64[P + 1 + pair + 1] - m0;
  const long long xb = static_cast<long long>(tab[g.o_blk_off + pair]) * g.SB;
  const long long npad = static_cast<long long>(tab[g.o_blk_off + pair + 1]) * g.SB - xb;
  const long long big = npad > M ? npad : M;
  const long long c0 = static_cast<long long>(blockIdx.x) * kStatChunk;
  if (c0 >= big) return;
  const EmState* st = st_all + pair;
  double v[8];
  const int op[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int j = 0; j < 8; ++j) v[j] = 0.0;
  const double mx0 = st->mu_x[0], mx1 = st->mu_x[1], mx2 = st->mu_x[2];
  const double my0 = st->mu_y[0], my1 = st->mu_y[1], my2 = st->mu_y[2];
  for (long long i = c0 + threadIdx.x; i < c0 + kStatChunk; i += kStatThreads) {
    if (i < npad) {
      if (i < N) {
        const float* x = X + 3 * (n0 + i);
        const float fa = static_cast<float>(x[0] - mx0), fb = static_cast<float>(x[1] - mx1),
                    fc = static_cast<float>(x[2] - mx2);
        xs[xb + i] = make_float4(fa, fb, fc, phi_x ? phi_x[n0 + i] : 1.f);
        v[0] += fa;
        v[1] += fb;
        v[2] += fc;
        v[3] += static_cast<double>(fa) * fa + static_cast<double>(fb) * fb + static_cast<double>(fc) * fc;
      } else {
        xs[xb + i] = make_float4(0.f, 0.f, 0.f, 1.f);
      }
    }
    if (i < M) {
      const float* y = Y + 3 * (m0 + i);
      const float fa = static_cast<float>(y[0] - my0), fb = static_cast<float>(y[1] - my1),
                  fc = static_cast<float>(y[2] - my2);
      v[4] += fa;
      v[5] += fb;
      v[6] += fc;
      v[7] += static_cast<double>(fa) * fa + static_cast<double>(fb) * fb + static_cast<double>(fc) * fc;
    }
  }
  block_reduce<8>(v, op, red + (static_cast<size_t>(pair) * gridDim.x + blockIdx.x) * 8);
}

// Finalise pass 2 per pair (grid = P): initial pose in the centred frame,
// sigma^2_0, E-step constants.  t_c = R0 mu_x + t0 - mu_y;  with z = R0 xc + t_c:
//   sum z = R0 sum xc + N t_c,  sum |z|^2 = sum |xc|^2 + 2 t_c . (R0 sum xc) + N |t_c|^2,
//   sigma^2_0 = (M sum|z|^2 + N sum|yc|^2 - 2 sum z . sum yc) / (3 N M).
__global__ void finalize_init_kernel(const double* __restrict__ red, int chunks, const long long* __restrict__ off64,
                                     const int* __restrict__ tab, Geo g, DevParams dp, EmState* __restrict__ st_all,
                                     int* __restrict__ done_count) {
  __shared__ double v[8];
  const int pair = blockIdx.x;
  const int P = g.P;
  const long long N = off64[pair + 1] - off64[pair];
  const long long M = off64[P + 1 + pair + 1] - off64[P + 1 + pair];
  const long long npad = static_cast<long long>(tab[g.o_blk_off + pair + 1] - tab[g.o_blk_off + pair]) * g.SB;
  const long long big = npad > M ? npad : M;
  const int nchunk = static_cast<int>((big + kStatChunk - 1) / kStatChunk);
  {
    const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (j < 8) {
      double x = 0.0;
      for (int b = lane; b < nchunk; b += 32) x += red[(static_cast<size_t>(pair) * chunks + b) * 8 + j];
      x = warp_sum_d(x);
      if (lane == 0) v[j] = x;
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  if (pair == 0) *done_count = 0;
  EmState* st = st_all + pair;
  const double* R = dp.init_R;
  double tc[3], Rsx[3];
  for (int i = 0; i < 3; ++i) {
    tc[i] = R[3 * i] * st->mu_x[0] + R[3 * i + 1] * st->mu_x[1] + R[3 * i + 2] * st->mu_x[2] + dp.init_t[i] -
            st->mu_y[i];
    Rsx[i] = R[3 * i] * v[0] + R[3 * i + 1] * v[1] + R[3 * i + 2] * v[2];
  }
  const double Nd = static_cast<double>(N), Md = static_cast<double>(M);
  double sz[3], zz = v[3] + Nd * (tc[0] * tc[0] + tc[1] * tc[1] + tc[2] * tc[2]);
  for (int i = 0; i < 3; ++i) {
    sz[i] = Rsx[i] + Nd * tc[i];
    zz += 2.0 * tc[i] * Rsx[i];
  }
  const double cross = sz[0] * v[4] + sz[1] * v[5] + sz[2] * v[6];
  const double s20 = (Md * zz + Nd * v[7] - 2.0 * cross) / (3.0 * Nd * Md);
  for (int i = 0; i < 9; ++i) st->R[i] = R[i];
  for (int i = 0; i < 3; ++i) st->t[i] = tc[i];
  double s2 = dp.sigma2_init > 0.0 ? dp.sigma2_init : s20;
  if (!(s2 > st->sigma2_floor)) s2 = st->sigma2_floor > 0.0 ? st->sigma2_floor : 1e-30;
  st->sigma2 = s2;
  st->log2_wodds = dp.w > 0.0 ? log2(dp.w) - log2(1.0 - dp.w) : -INFINITY;
  st->log2_V = log2(st->V);
  st->ln_1mw = log1p(-dp.w);
  st->w0 = dp.w;
  st->nll_prev = 0.0;
  st->done = 0;
  st->iter = 0;
  st->numeric_fail = 0;
  set_estep_constants(st);
}

// ---------------------------------------------------------------------------
// kNN
// ---------------------------------------------------------------------------
constexpr int kKnnThreads = 128;
constexpr int kKnnTile = 512;

__global__ void to_float4_kernel(const float* __restrict__ Y, long long M, float4* __restrict__ y4) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < M) y4[i] = make_float4(Y[3 * i], Y[3 * i + 1], Y[3 * i + 2], 0.f);
}

// Insert (d, ci) into the sorted first k entries of (bd, bi); an equal distance
// already present (lower index) stays first.  Fully unrolled over KMAX.  The new
// threshold is min(k-th entry, cap) (cap bounds the k-th distance from above).
template <int KMAX>
__device__ __forceinline__ void knn_insert(float (&bd)[KMAX], int (&bi)[KMAX], float& thr, int k, float d,
                                           int ci, float cap) {
#pragma unroll
  for (int s = KMAX - 1; s >= 0; --s) {
    if (s < k) {
      if (s > 0 && bd[s - 1] > d) {
        bd[s] = bd[s - 1];
        bi[s] = bi[s - 1];
      } else if (bd[s] > d) {
        bd[s] = d;
        bi[s] = ci;
      }
    }
  }
#pragma unroll
  for (int s = 0; s < KMAX; ++s)
    if (s == k - 1) thr = fminf(bd[s], cap);
}

// An upper bound of the k-th nearest distance of query q: the largest distance
// to k targets with indices next to q (scanned clouds keep neighbours close in
// index, so the bound is tight there; it is valid for any order).  Returned just
// above that distance, so that a strict comparison keeps every candidate with
// d <= bound.  Same FP32 formula as the scan.
__device__ __forceinline__ float knn_seed_bound(const float4* __restrict__ y, long long M, long long q, int k,
                                                float4 p) {
  long long s0 = q - k / 2;
  if (s0 > M - k) s0 = M - k;
  if (s0 < 0) s0 = 0;
  float b = 0.f;
  for (int j = 0; j < k; ++j) {
    const float4 c = y[s0 + j];
    const float dx = p.x + (-c.x), dy = p.y + (-c.y), dz = p.z + (-c.z);
    b = fmaxf(b, fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
  }
  return b < INFINITY ? __uint_as_float(__float_as_uint(b) + 1u) : INFINITY;
}

// Two queries per thread (q and q + kKnnThreads), packed FP32x2 distances:
// with the candidate stored negated, p + (-c) is exactly p - c, and
// fma(dz, dz, fma(dy, dy, dx * dx)) per half is the scalar formula.
// grid = (query blocks of the largest pair, P, splits); candidates are the
// split's share of the query's own pair.
// KFIX > 0: k == KFIX is a compile-time constant (lists stay in registers);
// KFIX == 0: runtime k <= KMAX.
template <int KMAX, int KFIX>
__global__ void __launch_bounds__(kKnnThreads) knn_partial_kernel(const float4* __restrict__ y4,
                                                                  const long long* __restrict__ off64, int P,
                                                                  long long Mtot, int k_rt, int splits,
                                                                  float* __restrict__ part_d,
                                                                  int* __restrict__ part_i) {
  const int k = KFIX > 0 ? KFIX : k_rt;
  __shared__ float4 cxy[kKnnTile];  // (-x, -x, -y, -y)
  __shared__ float2 cz[kKnnTile];   // (-z, -z)
  const int pair = blockIdx.y;
  const long long m0 = off64[P + 1 + pair];
  const long long M = off64[P + 1 + pair + 1] - m0;
  const long long qb = static_cast<long long>(blockIdx.x) * (2 * kKnnThreads);
  if (qb >= M) return;
  const long long q0 = qb + threadIdx.x;
  const long long q1 = q0 + kKnnThreads;
  const int split = blockIdx.z;
  const long long per = (M + splits - 1) / splits;
  const long long c_lo = split * per;
  long long c_hi = c_lo + per;
  if (c_hi > M) c_hi = M;
  const bool v0 = q0 < M, v1 = q1 < M;
  const float4 p0 = v0 ? y4[m0 + q0] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 p1 = v1 ? y4[m0 + q1] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float2 px = make_float2(p0.x, p1.x), py = make_float2(p0.y, p1.y), pz = make_float2(p0.z, p1.z);
  float bd0[KMAX], bd1[KMAX];
  int bi0[KMAX], bi1[KMAX];
#pragma unroll
  for (int j = 0; j < KMAX; ++j) {
    bd0[j] = bd1[j] = INFINITY;
    bi0[j] = bi1[j] = 0x7fffffff;
  }
  // candidates above the seed bound can never enter the list: skipping them keeps the
  // (divergent) insertions to the few near candidates
  const float cap0 = v0 ? knn_seed_bound(y4 + m0, M, q0, k, p0) : INFINITY;
  const float cap1 = v1 ? knn_seed_bound(y4 + m0, M, q1, k, p1) : INFINITY;
  float thr0 = cap0, thr1 = cap1;
  for (long long base = c_lo; base < c_hi; base += kKnnTile) {
    const int cnt = static_cast<int>((c_hi - base) < kKnnTile ? (c_hi - base) : kKnnTile);
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += kKnnThreads) {
      const float4 c = y4[m0 + base + j];
      cxy[j] = make_float4(-c.x, -c.x, -c.y, -c.y);
      cz[j] = make_float2(-c.z, -c.z);
    }
    __syncthreads();
    // eight candidates per step: independent distance chains, one branch per query
    // unless a candidate passes (then the eight are inserted in index order)
    int j = 0;
    for (; j + 8 <= cnt; j += 8) {
      float2 d[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float4 a = cxy[j + u];
        const float2 dx = __fadd2_rn(px, make_float2(a.x, a.y));
        const float2 dy = __fadd2_rn(py, make_float2(a.z, a.w));
        const float2 dz = __fadd2_rn(pz, cz[j + u]);
        d[u] = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
      }
      const int ci = static_cast<int>(base + j);
      if (fminf(fminf(fminf(d[0].x, d[1].x), fminf(d[2].x, d[3].x)), fminf(fminf(d[4].x, d[5].x), fminf(d[6].x, d[7].x))) < thr0) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (d[u].x < thr0) knn_insert<KMAX>(bd0, bi0, thr0, k, d[u].x, ci + u, cap0);
      }
      if (fminf(fminf(fminf(d[0].y, d[1].y), fminf(d[2].y, d[3].y)), fminf(fminf(d[4].y, d[5].y), fminf(d[6].y, d[7].y))) < thr1) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (d[u].y < thr1) knn_insert<KMAX>(bd1, bi1, thr1, k, d[u].y, ci + u, cap1);
      }
    }
    for (; j < cnt; ++j) {
      const float4 a = cxy[j];
      const float2 dx = __fadd2_rn(px, make_float2(a.x, a.y));
      const float2 dy = __fadd2_rn(py, make_float2(a.z, a.w));
      const float2 dz = __fadd2_rn(pz, cz[j]);
      const float2 d = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
      const int ci = static_cast<int>(base + j);
      if (d.x < thr0) knn_insert<KMAX>(bd0, bi0, thr0, k, d.x, ci, cap0);
      if (d.y < thr1) knn_insert<KMAX>(bd1, bi1, thr1, k, d.y, ci, cap1);
    }
  }
  if (v0) {
    float* od = part_d + (static_cast<size_t>(split) * Mtot + m0 + q0) * k;
    int* oi = part_i + (static_cast<size_t>(split) * Mtot + m0 + q0) * k;
#pragma unroll
    for (int s = 0; s < KMAX; ++s)
      if (s < k) {
        od[s] = bd0[s];
        oi[s] = bi0[s];
      }
  }
  if (v1) {
    float* od = part_d + (static_cast<size_t>(split) * Mtot + m0 + q1) * k;
    int* oi = part_i + (static_cast<size_t>(split) * Mtot + m0 + q1) * k;
#pragma unroll
    for (int s = 0; s < KMAX; ++s)
      if (s < k) {
        od[s] = bd1[s];
        oi[s] = bi1[s];
      }
  }
}

// Merge the sorted partial lists of every split by (distance, index).
__global__ void knn_merge_kernel(const float* __restrict__ part_d, const int* __restrict__ part_i, long long Mtot,
                                 int k, int splits, int* __restrict__ idx) {
  const long long q = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= Mtot) return;
  int head[64];
  for (int s = 0; s < splits; ++s) head[s] = 0;
  for (int r = 0; r < k; ++r) {
    int best = -1;
    float bd = INFINITY;
    int bi = 0x7fffffff;
    for (int s = 0; s < splits; ++s) {
      if (head[s] >= k) continue;
      const size_t o = (static_cast<size_t>(s) * Mtot + q) * k + head[s];
      const float d = part_d[o];
      const int i = part_i[o];
      if (d < bd || (d == bd && i < bi)) {
        bd = d;
        bi = i;
        best = s;
      }
    }
    if (best < 0) break;
    ++head[best];
    idx[q * k + r] = bi;
  }
}

// ---------------------------------------------------------------------------
// Local geometry + record packing
// ---------------------------------------------------------------------------

// Cyclic Jacobi for a symmetric 3x3 matrix (FP64); returns the eigenvalues and
// the eigenvectors (columns of V).
__device__ void jacobi_sym3(double A[3][3], double V[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 32; ++sweep) {
    const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    const double dg = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off == 0.0 || off <= 1e-34 * dg) break;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0;
      const int q = pq == 0 ? 1 : 2;
      const double apq = A[p][q];
      if (apq == 0.0) continue;
      const double th = (A[q][q] - A[p][p]) / (2.0 * apq);
      const double t = copysign(1.0, th) / (fabs(th) + sqrt(th * th + 1.0));
      const double c = rsqrt(t * t + 1.0);
      const double s = t * c;
      // A' = J^T A J with J = [[c, s], [-s, c]] acting on (p, q)
      const double app = A[p][p] - t * apq;
      const double aqq = A[q][q] + t * apq;
      const int r = 3 - p - q;
      const double arp = A[r][p], arq = A[r][q];
      A[r][p] = A[p][r] = c * arp - s * arq;
      A[r][q] = A[q][r] = s * arp + c * arq;
      A[p][p] = app;
      A[q][q] = aqq;
      A[p][q] = A[q][p] = 0.0;
      for (int i = 0; i < 3; ++i) {
        const double vip = V[i][p], viq = V[i][q];
        V[i][p] = c * vip - s * viq;
        V[i][q] = s * vip + c * viq;
      }
    }
  }
}

// Static planes 4-15 of a record slot and its yl entry (see internal.cuh).
__device__ __forceinline__ void write_record(float* rec, float4* yl, long long slot, float y0, float y1, float y2,
                                             float a0, float a1, float a2, float b0, float b1, float b2, float l) {
  const long long tile = slot / kTile;
  const int j = static_cast<int>(slot % kTile);
  float* r = rec + tile * kTileFloats + j;
  const float v[12] = {a0, a1, a2, a0 * a0, a0 * a1, a0 * a2, a1 * a1, a1 * a2, a2 * a2, b0, b1, b2};
#pragma unroll
  for (int p = 0; p < 12; ++p) r[(4 + p) * kTile] = v[p];
  yl[slot] = make_float4(y0, y1, y2, l);
}

__device__ __forceinline__ void write_padding(float* rec, float4* yl, long long slot) {
  write_record(rec, yl, slot, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, -INFINITY);
}

// Record of target y (caller's frame) with normal n and penalty alpha: centred
// coordinates, a = sqrt(alpha) n, b = Lambda y_c = y_c + (a . y_c) a (FP64, then FP32).
__device__ __forceinline__ void pack_target(float* rec, float4* yl, long long slot, const float* y,
                                            const EmState* st, double nx, double ny, double nz, double alpha,
                                            double phi, int alpha_norm) {
  const double sa = sqrt(alpha > 0.0 ? alpha : 0.0);
  // l_m = log2 pi(m) (+ 1/2 log2(1 + alpha_m)), pi(m) = phi_m / sum phi
  const double l = (phi == 1.0 ? 0.0 : log2(phi)) + st->log2_pi + (alpha_norm ? 0.5 * log2(1.0 + alpha) : 0.0);
  const double c0 = y[0] - st->mu_y[0], c1 = y[1] - st->mu_y[1], c2 = y[2] - st->mu_y[2];
  const double a0 = sa * nx, a1 = sa * ny, a2 = sa * nz;
  const double ay = a0 * c0 + a1 * c1 + a2 * c2;
  write_record(rec, yl, slot, static_cast<float>(c0), static_cast<float>(c1), static_cast<float>(c2),
               static_cast<float>(a0), static_cast<float>(a1), static_cast<float>(a2),
               static_cast<float>(c0 + ay * a0), static_cast<float>(c1 + ay * a1), static_cast<float>(c2 + ay * a2),
               static_cast<float>(l));
}

// grid = (largest tile count, P), kTile threads: target m = tile * kTile + tid of
// the pair; its record slot is (tile_off[pair] + tile) * kTile + tid.
__global__ void __launch_bounds__(kTile) geometry_kernel(const float* __restrict__ Y,
                                                         const float* __restrict__ phi_y,
                                                         const long long* __restrict__ off64,
                                                         const int* __restrict__ tab, Geo g,
                                                         const int* __restrict__ idx, int k, double alpha_max,
                                                         double lambda, int alpha_norm,
                                                         const EmState* __restrict__ st_all,
                                                         float* __restrict__ rec, float4* __restrict__ yl,
                                                         float* __restrict__ normals, float* __restrict__ kappa,
                                                         float* __restrict__ alpha_out) {
  const int pair = blockIdx.y;
  const int t0 = tab[g.o_tile_off + pair], t1 = tab[g.o_tile_off + pair + 1];
  if (static_cast<int>(blockIdx.x) >= t1 - t0) return;
  const long long m0 = off64[g.P + 1 + pair];
  const long long M = off64[g.P + 1 + pair + 1] - m0;
  const long long m = static_cast<long long>(blockIdx.x) * kTile + threadIdx.x;
  const long long slot = static_cast<long long>(t0 + blockIdx.x) * kTile + threadIdx.x;
  if (m >= M) {
    write_padding(rec, yl, slot);
    return;
  }
  const long long gm = m0 + m;
  // FP64 throughput is the bound of this kernel on GB300 (a division costs about a dozen
  // FP64 instructions): the six distinct sums of the covariance are scaled once by 1/k
  const double inv_k = 1.0 / k;
  double mean[3] = {0.0, 0.0, 0.0};
  for (int j = 0; j < k; ++j) {
    const long long q = m0 + idx[gm * k + j];
    mean[0] += Y[3 * q];
    mean[1] += Y[3 * q + 1];
    mean[2] += Y[3 * q + 2];
  }
  for (int c = 0; c < 3; ++c) mean[c] *= inv_k;
  double s00 = 0.0, s01 = 0.0, s02 = 0.0, s11 = 0.0, s12 = 0.0, s22 = 0.0;
  for (int j = 0; j < k; ++j) {
    const long long q = m0 + idx[gm * k + j];
    const double d0 = Y[3 * q] - mean[0], d1 = Y[3 * q + 1] - mean[1], d2 = Y[3 * q + 2] - mean[2];
    s00 = fma(d0, d0, s00);
    s01 = fma(d0, d1, s01);
    s02 = fma(d0, d2, s02);
    s11 = fma(d1, d1, s11);
    s12 = fma(d1, d2, s12);
    s22 = fma(d2, d2, s22);
  }
  double C[3][3] = {{s00 * inv_k, s01 * inv_k, s02 * inv_k},
                    {s01 * inv_k, s11 * inv_k, s12 * inv_k},
                    {s02 * inv_k, s12 * inv_k, s22 * inv_k}};
  double V[3][3];
  jacobi_sym3(C, V);
  int i0 = 0;
  if (C[1][1] < C[i0][i0]) i0 = 1;
  if (C[2][2] < C[i0][i0]) i0 = 2;
  const double l0 = fmax(C[i0][i0], 0.0);
  const double tr = fmax(C[0][0], 0.0) + fmax(C[1][1], 0.0) + fmax(C[2][2], 0.0);
  double kap, n0, n1, n2;
  if (tr > 0.0) {
    kap = l0 / tr;
    n0 = V[0][i0];
    n1 = V[1][i0];
    n2 = V[2][i0];
  } else {
    kap = 1.0 / 3.0;
    n0 = 0.0;
    n1 = 0.0;
    n2 = 1.0;
  }
  double a = kap > 0.0 ? alpha_max * tanh(0.5 * lambda * (1.0 / kap - 3.0)) : alpha_max;
  if (a < 0.0) a = 0.0;
  pack_target(rec, yl, slot, Y + 3 * gm, st_all + pair, n0, n1, n2, a, phi_y ? phi_y[gm] : 1.0, alpha_norm);
  if (normals) {
    normals[3 * gm] = static_cast<float>(n0);
    normals[3 * gm + 1] = static_cast<float>(n1);
    normals[3 * gm + 2] = static_cast<float>(n2);
  }
  if (kappa) kappa[gm] = static_cast<float>(kap);
  if (alpha_out) alpha_out[gm] = static_cast<float>(a);
}

__global__ void __launch_bounds__(kTile) pack_kernel(const float* __restrict__ Y, const float* __restrict__ phi_y,
                                                     const long long* __restrict__ off64,
                                                     const int* __restrict__ tab, Geo g,
                                                     const float* __restrict__ normals, const float* __restrict__ alpha,
                                                     int alpha_norm, const EmState* __restrict__ st_all,
                                                     float* __restrict__ rec, float4* __restrict__ yl) {
  const int pair = blockIdx.y;
  const int t0 = tab[g.o_tile_off + pair], t1 = tab[g.o_tile_off + pair + 1];
  if (static_cast<int>(blockIdx.x) >= t1 - t0) return;
  const long long m0 = off64[g.P + 1 + pair];
  const long long M = off64[g.P + 1 + pair + 1] - m0;
  const long long m = static_cast<long long>(blockIdx.x) * kTile + threadIdx.x;
  const long long slot = static_cast<long long>(t0 + blockIdx.x) * kTile + threadIdx.x;
  if (m >= M) {
    write_padding(rec, yl, slot);
    return;
  }
  const long long gm = m0 + m;
  pack_target(rec, yl, slot, Y + 3 * gm, st_all + pair, normals[3 * gm], normals[3 * gm + 1], normals[3 * gm + 2],
              alpha[gm], phi_y ? phi_y[gm] : 1.0, alpha_norm);
}

// Outlier weight from the outlier ratio (Sec. 3.2), one CTA per pair:
// S = sum_m pi(m) c_m = c0 sum_m 2^(l_m) with c0 = (2 pi sigma^2_0)^(-3/2) (l_m
// already holds log2 pi(m) and, with the Gaussian constant, 1/2 log2(1 + alpha_m)),
// w0 = eta V S / ((1 - eta) + eta V S), then the E-step constants of the pair.
constexpr int kEtaThreads = 256;
__global__ void __launch_bounds__(kEtaThreads) eta_kernel(const float4* __restrict__ yl, const int* __restrict__ tab,
                                                          Geo g, double eta, EmState* __restrict__ st_all) {
  __shared__ double sh[kEtaThreads / 32];
  const int pair = blockIdx.x;
  const long long s0 = static_cast<long long>(tab[g.o_tile_off + pair]) * kTile;
  const long long s1 = static_cast<long long>(tab[g.o_tile_off + pair + 1]) * kTile;
  double acc = 0.0;
  for (long long i = s0 + threadIdx.x; i < s1; i += kEtaThreads) acc += exp2(static_cast<double>(yl[i].w));
  acc = warp_sum_d(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x != 0) return;
  double sum = 0.0;
  for (int w = 0; w < kEtaThreads / 32; ++w) sum += sh[w];
  EmState* st = st_all + pair;
  const double S = pow(2.0 * 3.14159265358979323846 * st->sigma2, -1.5) * sum;
  const double a = eta * st->V * S;
  const double w = a / ((1.0 - eta) + a);
  st->w0 = w;
  st->log2_wodds = w > 0.0 ? log2(w) - log2(1.0 - w) : -INFINITY;
  st->ln_1mw = log1p(-w);
  set_estep_constants(st);
}

// Stable compaction (confidence truncation, Sec. 3.3).  grid = (chunks, P),
// kStatThreads threads, kStatChunk rows per CTA: each thread owns two
// consecutive rows, so ranks follow from one block-wide exclusive scan.
__device__ __forceinline__ int block_exclusive_scan(int v, int* total) {
  __shared__ int wsum[kStatThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  int before = 0, all = 0;
  for (int w = 0; w < kStatThreads / 32; ++w) {
    if (w < warp) before += wsum[w];
    all += wsum[w];
  }
  __syncthreads();
  *total = all;
  return before + x - v;
}

__global__ void __launch_bounds__(kStatThreads) compact_count_kernel(const float* __restrict__ phi,
                                                                     const long long* __restrict__ off, float thr,
                                                                     int* __restrict__ cnt) {
  const int pair = blockIdx.y;
  const long long r0 = off[pair], n = off[pair + 1] - r0;
  const long long i0 = static_cast<long long>(blockIdx.x) * kStatChunk + 2 * threadIdx.x;
  int v = 0;
  for (int j = 0; j < 2; ++j)
    if (i0 + j < n && phi[r0 + i0 + j] >= thr) ++v;
  int total = 0;
  block_exclusive_scan(v, &total);
  if (threadIdx.x == 0) cnt[static_cast<size_t>(pair) * gridDim.x + blockIdx.x] = total;
}

__global__ void __launch_bounds__(kStatThreads) compact_scatter_kernel(
    const float* __restrict__ rows, const float* __restrict__ phi, const long long* __restrict__ off,
    const long long* __restrict__ out_off, const int* __restrict__ coff, float thr, float* __restrict__ rows_out,
    float* __restrict__ phi_out) {
  const int pair = blockIdx.y;
  const long long r0 = off[pair], n = off[pair + 1] - r0;
  const long long i0 = static_cast<long long>(blockIdx.x) * kStatChunk + 2 * threadIdx.x;
  bool keep[2];
  int v = 0;
  for (int j = 0; j < 2; ++j) {
    keep[j] = i0 + j < n && phi[r0 + i0 + j] >= thr;
    v += keep[j];
  }
  int total = 0;
  int rank = block_exclusive_scan(v, &total);
  const long long o0 = out_off[pair] + coff[static_cast<size_t>(pair) * gridDim.x + blockIdx.x];
  for (int j = 0; j < 2; ++j)
    if (keep[j]) {
      const long long src = r0 + i0 + j, dst = o0 + rank++;
      rows_out[3 * dst] = rows[3 * src];
      rows_out[3 * dst + 1] = rows[3 * src + 1];
      rows_out[3 * dst + 2] = rows[3 * src + 2];
      phi_out[dst] = phi[src];
    }
}

}  // namespace

int stats_chunks(const Geo& g) {
  const long long big_n = static_cast<long long>(g.max_blocks) * g.SB;
  const long long big = big_n > g.max_m ? big_n : g.max_m;
  return static_cast<int>((big + kStatChunk - 1) / kStatChunk);
}

cudaError_t launch_init(const BatchPlan& p, const Dev& d, const float* X, const float* Y, const float* phi_x,
                        const float* phi_y, const DevParams& dp, bool full, double* red, float4* xs,
                        cudaStream_t s) {
  const Geo& g = p.g;
  const int chunks = stats_chunks(g);
  dim3 grid(static_cast<unsigned>(chunks), static_cast<unsigned>(g.P));
  raw_stats_kernel<<<grid, kStatThreads, 0, s>>>(X, Y, phi_y, d.off64, g.P, red);
  finalize_raw_kernel<<<g.P, kRaw * 32, 0, s>>>(red, chunks, d.off64, g.P, full ? dp.volume : 0.0,
                                              full ? dp.sigma2_floor_rel : 0.0, d.st);
  double* red2 = red + static_cast<size_t>(g.P) * chunks * kRaw;
  center_kernel<<<grid, kStatThreads, 0, s>>>(X, Y, phi_x, d.off64, d.tab, g, d.st, xs, red2);
  if (full) finalize_init_kernel<<<g.P, 8 * 32, 0, s>>>(red2, chunks, d.off64, d.tab, g, dp, d.st, d.done_count);
  return cudaGetLastError();
}

int knn_splits(const Geo& g, int num_sms) {
  long long qblocks = 0;  // total query blocks over the batch is approximated by P x the largest pair
  qblocks = static_cast<long long>(g.P) * ((g.max_m + 2 * kKnnThreads - 1) / (2 * kKnnThreads));
  long long sp = (4LL * num_sms + qblocks - 1) / qblocks;
  if (sp < 1) sp = 1;
  if (sp > 32) sp = 32;
  // at least 64 candidates per split in the largest pair
  while (sp > 1 && g.max_m / sp < 64) --sp;
  return static_cast<int>(sp);
}

cudaError_t launch_knn(const BatchPlan& p, const Dev& d, const float* Y, int k, int splits, float4* y4,
                       float* part_d, int* part_i, int* idx_out, cudaStream_t s) {
  const Geo& g = p.g;
  const long long Mtot = p.off64[2 * g.P + 1];
  to_float4_kernel<<<static_cast<unsigned>((Mtot + 255) / 256), 256, 0, s>>>(Y, Mtot, y4);
  dim3 grid(static_cast<unsigned>((g.max_m + 2 * kKnnThreads - 1) / (2 * kKnnThreads)), static_cast<unsigned>(g.P),
            static_cast<unsigned>(splits));
  switch (k) {
#define LSG_KNN_CASE(K) \
  case K:               \
    knn_partial_kernel<K, K><<<grid, kKnnThreads, 0, s>>>(y4, d.off64, g.P, Mtot, k, splits, part_d, part_i); \
    break;
    LSG_KNN_CASE(1) LSG_KNN_CASE(2) LSG_KNN_CASE(3) LSG_KNN_CASE(4) LSG_KNN_CASE(5) LSG_KNN_CASE(6)
    LSG_KNN_CASE(7) LSG_KNN_CASE(8) LSG_KNN_CASE(9) LSG_KNN_CASE(10) LSG_KNN_CASE(11) LSG_KNN_CASE(12)
    LSG_KNN_CASE(13) LSG_KNN_CASE(14) LSG_KNN_CASE(15) LSG_KNN_CASE(16)
#undef LSG_KNN_CASE
    default:
      knn_partial_kernel<32, 0><<<grid, kKnnThreads, 0, s>>>(y4, d.off64, g.P, Mtot, k, splits, part_d, part_i);
  }
  knn_merge_kernel<<<static_cast<unsigned>((Mtot + 127) / 128), 128, 0, s>>>(part_d, part_i, Mtot, k, splits,
                                                                            idx_out);
  return cudaGetLastError();
}

cudaError_t launch_geometry(const BatchPlan& p, const Dev& d, const float* Y, const float* phi_y, const int* idx,
                            int k, double alpha_max, double lambda, int alpha_norm, float* rec, float4* yl,
                            float* normals, float* kappa, float* alpha, cudaStream_t s) {
  dim3 grid(static_cast<unsigned>(p.g.max_tiles), static_cast<unsigned>(p.g.P));
  geometry_kernel<<<grid, kTile, 0, s>>>(Y, phi_y, d.off64, d.tab, p.g, idx, k, alpha_max, lambda, alpha_norm, d.st, rec,
                                         yl, normals, kappa, alpha);
  return cudaGetLastError();
}

cudaError_t launch_pack(const BatchPlan& p, const Dev& d, const float* Y, const float* phi_y, const float* normals,
                        const float* alpha, int alpha_norm, float* rec, float4* yl, cudaStream_t s) {
  dim3 grid(static_cast<unsigned>(p.g.max_tiles), static_cast<unsigned>(p.g.P));
  pack_kernel<<<grid, kTile, 0, s>>>(Y, phi_y, d.off64, d.tab, p.g, normals, alpha, alpha_norm, d.st, rec, yl);
  return cudaGetLastError();
}

cudaError_t launch_eta(const BatchPlan& p, const Dev& d, const float4* yl, double eta, cudaStream_t s) {
  eta_kernel<<<p.g.P, kEtaThreads, 0, s>>>(yl, d.tab, p.g, eta, d.st);
  return cudaGetLastError();
}

int compact_chunks(long long max_rows) { return static_cast<int>((max_rows + kStatChunk - 1) / kStatChunk); }

cudaError_t launch_compact_count(const float* phi, const long long* off, int P, int chunks, float threshold,
                                 int* cnt, cudaStream_t s) {
  dim3 grid(static_cast<unsigned>(chunks), static_cast<unsigned>(P));
  compact_count_kernel<<<grid, kStatThreads, 0, s>>>(phi, off, threshold, cnt);
  return cudaGetLastError();
}

cudaError_t launch_compact_scatter(const float* rows, const float* phi, const long long* off,
                                   const long long* out_off, const int* coff, int P, int chunks, float threshold,
                                   float* rows_out, float* phi_out, cudaStream_t s) {
  dim3 grid(static_cast<unsigned>(chunks), static_cast<unsigned>(P));
  compact_scatter_kernel<<<grid, kStatThreads, 0, s>>>(rows, phi, off, out_off, coff, threshold, rows_out, phi_out);
  return cudaGetLastError();
}

}  // namespace lsg
