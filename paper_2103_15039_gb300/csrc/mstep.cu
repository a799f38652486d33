// M step of LSG-CPD (Sec. 3.5, Eqs. (11)-(13)) and the sigma^2 update, from
// the global moments of one E step.
//
// With the posteriors fixed, sum_m P_mn d_mn is an exact quadratic function
// of the moved source point, and the moved point is affine in T = [R | t]
// (3x4).  With x~ = [x; 1] and the transform T_o used by the E step,
//   Q_d(T) = SD + 2 <H1, T - T_o> + <T - T_o, G (T - T_o)>,
//   H1 = sum_n h_n x~_n^T,  G_(ik),(jl) = A^{kl}_ij = sum_n A_n,ij x~_nk x~_nl,
// (h_n = sum_m P_mn Lambda_m r_mn, A_n = Pbar_n I + W_n), so the inner Newton loop of
// Eq. (13) costs O(1) per step, independent of N and M.
//
// Newton on SE(3): right perturbation T o exp(xi^), basis order rotations
// about x, y, z then translations.  With M1 = H1 + G (T - T_o),
// N = R^T M1[:, :3], m = R^T M1[:, 3] and C^{kl} = R^T A^{kl} R:
//   grad_rot a  = 2 <N, [e_a]x>,             grad_tr c = 2 m_c
//   H_rot a,rot b = 2 sum eps_aik eps_bjl C^{kl}_ij + N_ab + N_ba - 2 delta_ab tr N
//   H_rot a,tr c  = -2 sum eps_aik C^{k3}_ic + m . (e_a x e_c)
//   H_tr c,tr d   = 2 C^{33}_cd
// which is the symmetrised Hessian (H + H^T)/2 of Eq. (12) at the current iterate.
// Step rule (same as the FP64 reference): xi = -(H_s)^{-1} grad; if H_s is not
// positive definite it is damped by mu I (mu = 1e-6 tr/6, x10); a step that
// raises Q_d is halved up to 10 times; stop when |xi| < newton_tol, after
// newton_max steps, or when no halving lowers Q_d.
//
// Precision (GB300 issues one FP64 warp instruction per ~64 cycles per SM
// sub-partition, and the loop is a chain of dependent operations): the residual
// M1, the gradient, the objective change dQ = 2 <M1, D> + <D, G D> of a trial
// step D, the transform and Q_d are double-float values (pairs of FP32 numbers,
// about 48 significant bits) computed lane-parallel on the FP32 pipe; the model
// arrives in FP64 and is split once, with integer bit operations (an FP64
// instruction has ~80 cycles of latency on GB300, a conversion chain several times
// that).  The Hessian and the 6x6 solve for the
// Newton direction (LDL^T) are FP32: an inexact direction only changes the path,
// not the fixed point, which is set by the double-float residual (iterative
// refinement).
#include <math.h>

#include "internal.cuh"

namespace lsg {
namespace {

constexpr int kMThreads = 128;

// ---------------------------------------------------------------------------
// Double-float arithmetic for the Newton loop: a value is hi + lo (|lo| at most
// half an ulp of hi), about 48 significant bits, computed on the FP32 pipe with
// the error-free transformations of Knuth (TwoSum), Dekker (FastTwoSum) and the
// FMA-based exact product.  GB300 issues FP64 instructions far more slowly than
// FP32 ones and the loop is a chain of dependent operations, so its state, the
// model it needs for the objective change, and every operation on them use
// these pairs; the Hessian only steers the direction and is FP32.
// ---------------------------------------------------------------------------
struct dd {
  float hi, lo;
};

__device__ __forceinline__ dd dd_from(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - static_cast<double>(h))};
}
__device__ __forceinline__ double dd_to(dd a) { return static_cast<double>(a.hi) + static_cast<double>(a.lo); }
// The same split with integer operations only (FP64 instructions have a latency of ~80
// cycles on GB300, and a conversion chain several times that): hi = x truncated to 24
// significant bits (exact bit surgery), lo = the remaining 29 bits rounded to FP32, so
// hi + lo carries about 48 bits of x.  Magnitudes below 2^-126 flush to zero, above the
// FP32 range hi is an infinity; infinities and NaN pass through in hi.
__device__ __forceinline__ dd dd_split(double x) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned sign = static_cast<unsigned>(u >> 32) & 0x80000000u;
  const int e = static_cast<int>((u >> 52) & 0x7ffu);
  const unsigned long long m = u & 0xfffffffffffffULL;
  if (e == 0x7ff) return {__uint_as_float(sign | 0x7f800000u | (m ? 0x400000u : 0u)), 0.f};
  const int ef = e - 1023 + 127;
  if (ef <= 0) return {__uint_as_float(sign), 0.f};
  if (ef >= 255) return {__uint_as_float(sign | 0x7f800000u), 0.f};
  const float hi = __uint_as_float(sign | (static_cast<unsigned>(ef) << 23) | static_cast<unsigned>(m >> 29));
  const float lo = ldexpf(static_cast<float>(static_cast<unsigned>(m & 0x1fffffffu)), e - 1075);
  return {hi, sign ? -lo : lo};
}
__device__ __forceinline__ float dd_f(dd a) { return __fadd_rn(a.hi, a.lo); }

__device__ __forceinline__ dd two_sum(float a, float b) {  // s + e = a + b exactly
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ dd fast_two_sum(float a, float b) {  // |a| >= |b| or a = 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dd two_prod(float a, float b) {  // p + e = a b exactly
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  const dd t = two_sum(a.lo, b.lo);
  s = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ dd dd_neg(dd a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ dd dd_mulf(dd a, float b) {  // b exact in FP32
  dd p = two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ dd dd_fma(dd a, dd b, dd c) { return dd_add(dd_mul(a, b), c); }
__device__ __forceinline__ dd dd_scale2(dd a, float s) { return {a.hi * s, a.lo * s}; }  // s a power of two
__device__ __forceinline__ bool dd_le0(dd a) { return a.hi < 0.f || (a.hi == 0.f && a.lo <= 0.f); }

// Power-series coefficients (-1)^k / (2k + o)! of sin(th)/th (o = 1), (1 - cos th)/th^2
// (o = 2) and (th - sin th)/th^3 (o = 3) in powers of th^2, k = 0..8; the truncation
// error is below 1e-19 for th^2 <= 1/4.
constexpr double kExpSeries[3][9] = {
    {1.0, -0.16666666666666666, 0.008333333333333333, -0.0001984126984126984, 2.7557319223985893e-06, -2.505210838544172e-08, 1.6059043836821613e-10, -7.647163731819816e-13, 2.8114572543455206e-15},
    {0.5, -0.041666666666666664, 0.001388888888888889, -2.48015873015873e-05, 2.755731922398589e-07, -2.08767569878681e-09, 1.1470745597729725e-11, -4.779477332387385e-14, 1.5619206968586225e-16},
    {0.16666666666666666, -0.008333333333333333, 0.0001984126984126984, -2.7557319223985893e-06, 2.505210838544172e-08, -1.6059043836821613e-10, 7.647163731819816e-13, -2.8114572543455206e-15, 8.22063524662433e-18}};

// The same coefficients as double-float pairs (hi = the FP32 rounding, lo = the FP32
// rounding of the rest), split at compile time.
struct SeriesTab {
  dd c[3][9];
};
__host__ __device__ constexpr SeriesTab make_series_tab() {
  SeriesTab t{};
  for (int o = 0; o < 3; ++o)
    for (int k = 0; k < 9; ++k) {
      const float hi = static_cast<float>(kExpSeries[o][k]);
      t.c[o][k] = dd{hi, static_cast<float>(kExpSeries[o][k] - static_cast<double>(hi))};
    }
  return t;
}
__device__ const SeriesTab c_series = make_series_tab();

// Gradient and symmetrised Hessian entries as fixed linear combinations of the
// entries of C (10 pairs x 9) and of NM = R^T M1 (3 x 4):
//   entry e = sum_t cc[e][t] * C_flat[ic[e][t]] + sum_t cn[e][t] * NM[in[e][t]]
// e = 0..5: gradient; e = 6..26: upper triangle of H_s in row-major order.
// Built at compile time from the closed forms in the file comment.
struct HessTab {
  int ic[27][4];
  float cc[27][4];
  int in[27][3];
  float cn[27][3];
};

__host__ __device__ constexpr int pair_q_c(int k, int l) {
  return k > l ? pair_q_c(l, k) : (k == 0 ? l : (k == 1 ? 3 + l : (k == 2 ? 5 + l : 9)));
}
__host__ __device__ constexpr int cflat(int k, int l, int i, int j) { return pair_q_c(k, l) * 9 + 3 * i + j; }
__host__ __device__ constexpr float eps_c(int a, int b, int c) {
  return (a == b || b == c || a == c) ? 0.f : (((b - a + 3) % 3 == 1) ? 1.f : -1.f);
}

__host__ __device__ constexpr HessTab make_hess_tab() {
  HessTab h{};
  for (int e = 0; e < 27; ++e)
    for (int t = 0; t < 4; ++t) {
      h.ic[e][t] = 0;
      h.cc[e][t] = 0.f;
      if (t < 3) {
        h.in[e][t] = 0;
        h.cn[e][t] = 0.f;
      }
    }
  for (int a = 0; a < 6; ++a) {  // gradient
    if (a < 3) {
      const int a1 = (a + 1) % 3, a2 = (a + 2) % 3;
      h.in[a][0] = 4 * a2 + a1;
      h.cn[a][0] = 2.f;
      h.in[a][1] = 4 * a1 + a2;
      h.cn[a][1] = -2.f;
    } else {
      h.in[a][0] = 4 * (a - 3) + 3;
      h.cn[a][0] = 2.f;
    }
  }
  int e = 6;
  for (int a = 0; a < 6; ++a)
    for (int b = a; b < 6; ++b, ++e) {
      const int a1 = (a + 1) % 3, a2 = (a + 2) % 3;
      if (b < 3) {
        const int b1 = (b + 1) % 3, b2 = (b + 2) % 3;
        h.ic[e][0] = cflat(a2, b2, a1, b1);
        h.cc[e][0] = 2.f;
        h.ic[e][1] = cflat(a2, b1, a1, b2);
        h.cc[e][1] = -2.f;
        h.ic[e][2] = cflat(a1, b2, a2, b1);
        h.cc[e][2] = -2.f;
        h.ic[e][3] = cflat(a1, b1, a2, b2);
        h.cc[e][3] = 2.f;
        if (a != b) {  // N_ab + N_ba
          h.in[e][0] = 4 * a + b;
          h.cn[e][0] = 1.f;
          h.in[e][1] = 4 * b + a;
          h.cn[e][1] = 1.f;
        } else {  // 2 N_aa - 2 tr N
          for (int i = 0; i < 3; ++i) {
            h.in[e][i] = 5 * i;
            h.cn[e][i] = (i == a) ? 0.f : -2.f;
          }
        }
      } else if (a < 3) {
        const int c = b - 3;
        h.ic[e][0] = cflat(a1, 3, a2, c);
        h.cc[e][0] = 2.f;
        h.ic[e][1] = cflat(a2, 3, a1, c);
        h.cc[e][1] = -2.f;
        if (c != a) {
          const int i = 3 - a - c;
          h.in[e][0] = 4 * i + 3;
          h.cn[e][0] = eps_c(a, c, i);
        }
      } else {
        h.ic[e][0] = cflat(3, 3, a - 3, b - 3);
        h.cc[e][0] = 2.f;
      }
    }
  return h;
}

__device__ const HessTab c_hess = make_hess_tab();

// theta^2 = w . w for a rotation part given exactly in FP32
__device__ __forceinline__ dd theta2(const float* w) {
  return dd_add(dd_add(two_prod(w[0], w[0]), two_prod(w[1], w[1])), two_prod(w[2], w[2]));
}

struct Shared {
  double SD, NP;
  double R[9], t[3];  // the result of the Newton loop in FP64
  double Q;
  float gHf[27];  // gradient (6) then the upper triangle of H_s (21), FP32 for the direction solve
  float xf[6];    // Newton direction (FP32)
  float wv[6];    // step * xi (exact in FP32)
  float Af[10][6];  // model in FP32 for the Hessian: A^{q}, q = xt pair (00,01,02,03,11,12,13,22,23,33),
                    // entries (00,01,02,11,12,22)
  float Cf[10][9];  // C^{kl} = R^T A^{kl} R (FP32, Hessian only)
  float NMf[12];
  int iters, damped, halvings;
  int go;          // loop control
  int accepted;
  HessTab hess;    // per-lane divergent lookups: shared, not constant, memory
  // double-float state of the loop (hi, lo pairs)
  dd Ad[10][6];  // the model for G D
  dd Rd[9], td[3], M1d[12], NMd[12], Qd, dQd;
  dd Rod[9], tod[3];  // the E step's pose T_o
  dd coefd[3], Ed[9], Vvd[3], Tcd[12], dld[12], Gdd[12], dqv[12];
  SeriesTab series;
};

// position of (a, b), a <= b, in the row-major upper triangle of a 6x6 matrix
__host__ __device__ constexpr int tri_index(int a, int b) { return a * 6 - a * (a - 1) / 2 + (b - a); }

__device__ __forceinline__ int pair_q(int k, int l) {
  if (k > l) {
    const int t = k;
    k = l;
    l = t;
  }
  // (0,0)0 (0,1)1 (0,2)2 (0,3)3 (1,1)4 (1,2)5 (1,3)6 (2,2)7 (2,3)8 (3,3)9
  return k == 0 ? l : (k == 1 ? 3 + l : (k == 2 ? 5 + l : 9));
}

__device__ __forceinline__ int sym_p(int i, int j) {
  if (i > j) {
    const int t = i;
    i = j;
    j = t;
  }
  return i == 0 ? j : (i == 1 ? 2 + j : 5);
}

// Levi-Civita symbol for indices in {0, 1, 2}
__device__ __forceinline__ double eps3(int a, int b, int c) {
  if (a == b || b == c || a == c) return 0.0;
  return ((b - a + 3) % 3 == 1) ? 1.0 : -1.0;
}

// Constant tables of the Newton loop (Hessian index table, exp-map series) into
// shared memory.  They do not depend on the E step, so the kernels load them before
// waiting for their predecessor.
__device__ void load_tables(Shared& s) {
  const int tid = threadIdx.x;
  // global (not constant) memory: every lane reads a different word, so the loads coalesce
  const int* src = reinterpret_cast<const int*>(&c_hess);
  int* dst = reinterpret_cast<int*>(&s.hess);
  constexpr int kWords = static_cast<int>(sizeof(HessTab) / sizeof(int));
#pragma unroll
  for (int r = 0; r < (kWords + kMThreads - 1) / kMThreads; ++r) {  // all loads in flight at once
    const int i = tid + r * kMThreads;
    if (i < kWords) dst[i] = __ldg(src + i);
  }
  constexpr int kSeriesWords = static_cast<int>(sizeof(SeriesTab) / sizeof(int));
  static_assert(kSeriesWords <= kMThreads, "one word per thread");
  if (tid < kSeriesWords)
    reinterpret_cast<int*>(&s.series)[tid] = __ldg(reinterpret_cast<const int*>(&c_series) + tid);
}

// Model, start pose and loop state of the Newton loop from the global moments (FP64)
// and the pose T_o = (R, t) (FP64), all lanes in parallel and without FP64
// instructions; the caller synchronises before newton().
__device__ void setup_newton(Shared& s, const double* mom, const double* R, const double* t) {
  const int tid = threadIdx.x;
  if (tid < 60) {
    const int p = tid / 10, q = tid % 10;  // moments are ordered A pair major, xt pair minor
    const dd a = dd_split(mom[14 + tid]);
    s.Ad[q][p] = a;
    s.Af[q][p] = dd_f(a);
  } else if (tid >= 64 && tid < 76) {
    s.M1d[tid - 64] = dd_split(mom[2 + tid - 64]);  // M1 = H1 at T = T_o
  } else if (tid >= 76 && tid < 85) {
    const dd r = dd_split(R[tid - 76]);
    s.Rd[tid - 76] = r;
    s.Rod[tid - 76] = r;
  } else if (tid >= 85 && tid < 88) {
    const dd v = dd_split(t[tid - 85]);
    s.td[tid - 85] = v;
    s.tod[tid - 85] = v;
  } else if (tid == 96) {
    s.NP = mom[0];
    s.SD = mom[1];
    s.Qd = dd_split(mom[1]);
    s.iters = s.damped = s.halvings = 0;
    s.go = 1;
  }
}

// FP32 LDL^T solve of the symmetric 6x6 H x = b; false if a pivot is not positive.
// Every loop has a constant trip count and is fully unrolled (triangular ranges are
// masked), so that all arrays stay in registers.
__device__ __forceinline__ bool ldl_solve6(const float (&H)[36], const float (&b)[6], float (&x)[6]) {
  float L[36], D[6], Dinv[6];
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    float d = H[7 * j];
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (k < j) d -= L[6 * j + k] * L[6 * j + k] * D[k];
    ok = ok && (d > 0.f);
    D[j] = d;
    Dinv[j] = __frcp_rn(d);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      if (i > j) {
        float v = H[6 * i + j];
#pragma unroll
        for (int k = 0; k < 6; ++k)
          if (k < j) v -= L[6 * i + k] * L[6 * j + k] * D[k];
        L[6 * i + j] = v * Dinv[j];
      }
    }
  }
  float y[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    float v = b[i];
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (k < i) v -= L[6 * i + k] * y[k];
    y[i] = v;
  }
#pragma unroll
  for (int ii = 0; ii < 6; ++ii) {
    const int i = 5 - ii;
    float v = y[i] * Dinv[i];
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (k > i) v -= L[6 * k + i] * x[k];
    x[i] = v;
  }
  return ok;
}

// Newton loop on the model in shared memory (set up by setup_newton, synchronised);
// T starts at T_o.  Ends with s.R, s.t and s.Q (FP64) set from the double-float state.
__device__ void newton(Shared& s, int newton_max, double newton_tol) {
  const int tid = threadIdx.x;
  for (int it = 0; it < newton_max; ++it) {
    // --- C^{kl} = R^T A^{kl} R (FP32: Hessian only) and N, m = R^T M1 (double-float) ---
    if (tid < 60) {
      const int q = tid / 6, p = tid % 6;
      const int i = p < 3 ? 0 : (p < 5 ? 1 : 2);
      const int j = p < 3 ? p : (p < 5 ? p - 2 : 2);
      const float* Aq = s.Af[q];
      // u = A^q R e_j, then v = (R e_i) . u
      const float r0 = s.Rd[j].hi, r1 = s.Rd[3 + j].hi, r2 = s.Rd[6 + j].hi;
      const float u0 = fmaf(Aq[0], r0, fmaf(Aq[1], r1, Aq[2] * r2));
      const float u1 = fmaf(Aq[1], r0, fmaf(Aq[3], r1, Aq[4] * r2));
      const float u2 = fmaf(Aq[2], r0, fmaf(Aq[4], r1, Aq[5] * r2));
      const float v = fmaf(s.Rd[i].hi, u0, fmaf(s.Rd[3 + i].hi, u1, s.Rd[6 + i].hi * u2));
      s.Cf[q][3 * i + j] = v;
      s.Cf[q][3 * j + i] = v;
    } else if (tid >= 64 && tid < 76) {
      const int e = tid - 64, i = e / 4, k = e % 4;
      dd v = dd_mul(s.Rd[i], s.M1d[k]);
      v = dd_fma(s.Rd[3 + i], s.M1d[4 + k], v);
      v = dd_fma(s.Rd[6 + i], s.M1d[8 + k], v);
      s.NMd[e] = v;
      s.NMf[e] = dd_f(v);
    }
    __syncthreads();
    // --- gradient (6, double-float, rounded for the FP32 solve) and the upper triangle of
    // H_s (21, FP32): branch-free table form ---
    if (tid < 6) {
      dd v{0.f, 0.f};
#pragma unroll
      for (int t = 0; t < 3; ++t) v = dd_add(v, dd_scale2(s.NMd[s.hess.in[tid][t]], s.hess.cn[tid][t]));
      s.gHf[tid] = dd_f(v);
    } else if (tid < 27) {
      float v = 0.f;
#pragma unroll
      for (int t = 0; t < 4; ++t) v = fmaf(s.hess.cc[tid][t], (&s.Cf[0][0])[s.hess.ic[tid][t]], v);
#pragma unroll
      for (int t = 0; t < 3; ++t) v = fmaf(s.hess.cn[tid][t], s.NMf[s.hess.in[tid][t]], v);
      s.gHf[tid] = v;
    }
    __syncthreads();
    // --- Newton direction (FP32 LDL^T, damped if not positive definite) ---
    if (tid == 0) {
      // attempt 0 undamped; then mu = 1e-6 tr/6, x10 per attempt (a single call site
      // with compile-time indices keeps every array of the solve in registers)
      float mg[6], x[6];
      float tr = 0.f;
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        mg[a] = -s.gHf[a];
        tr += fabsf(s.gHf[6 + tri_index(a, a)]);
      }
      const float mu0 = 1e-6f * (tr > 0.f ? tr / 6.f : 1.f);
      bool ok = false;
      float mu = 0.f;
      for (int k = 0; k <= 40 && !ok; ++k) {
        float Dm[36];
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int b = 0; b < 6; ++b)
            Dm[6 * a + b] = s.gHf[6 + (a <= b ? tri_index(a, b) : tri_index(b, a))] + (a == b ? mu : 0.f);
        ok = ldl_solve6(Dm, mg, x);
        if (k == 1) ++s.damped;
        mu = (k == 0) ? mu0 : mu * 10.f;
      }
      if (!ok) {
        s.go = 0;
      } else {
        ++s.iters;
        float nx = 0.f;
#pragma unroll
        for (int a = 0; a < 6; ++a) {
          s.xf[a] = x[a];
          nx += x[a] * x[a];
        }
        // a step below the tolerance changes the transform by less than the tolerance:
        // the iteration has converged, so it is not evaluated
        if (nx < static_cast<float>(newton_tol) * static_cast<float>(newton_tol)) s.go = 0;
      }
      s.accepted = 0;
    }
    __syncthreads();
    if (!s.go) break;
    // --- backtracking on the exact change of Q_d (double-float) ---
    float step = 1.f;  // a power of two: step * xi is exact in FP32
    for (int bt = 0; bt <= 10; ++bt, step *= 0.5f) {
      if (tid < 6) s.wv[tid] = step * s.xf[tid];
      __syncthreads();
      if (tid < 3) {
        // exp coefficients A = sin(th)/th, B = (1 - cos th)/th^2, C = (th - sin th)/th^3 as
        // power series in th^2 (Horner, with as many terms as th^2 needs for 2^-48), else from sincos
        const dd x = theta2(s.wv);
        dd cf;
        if (x.hi <= 0.25f) {
          const dd* c = s.series.c[tid];
          const int top = x.hi < 1e-6f ? 3 : (x.hi < 1e-3f ? 5 : 8);
          dd r = c[top];
          for (int k = top - 1; k >= 0; --k) r = dd_fma(r, x, c[k]);
          cf = r;
        } else {
          const double xd = dd_to(x);
          const double th = sqrt(xd);
          double sh, ch;
          sincos(0.5 * th, &sh, &ch);
          const double sn = 2.0 * sh * ch;
          cf = dd_from(tid == 0 ? sn / th : (tid == 1 ? 2.0 * sh * sh / xd : (th - sn) / (xd * th)));
        }
        s.coefd[tid] = cf;
      }
      __syncthreads();
      // E = I + A W + B W^2 and V v = v + B W v + C W^2 v with W = [w]x, W^2 = w w^T - th^2 I
      if (tid < 9) {
        const int k = tid / 3, j = tid % 3;
        const float* w = s.wv;
        // ([w]x)_kj = -eps_kjm w_m (m = 3 - k - j; zero on the diagonal), exact in FP32
        const float Wkj = (k == j) ? 0.f : -static_cast<float>(eps3(k, j, 3 - k - j)) * w[3 - k - j];
        dd W2kj = two_prod(w[k], w[j]);
        if (k == j) W2kj = dd_sub(W2kj, theta2(w));
        dd E = dd_add(dd_mulf(s.coefd[0], Wkj), dd_mul(s.coefd[1], W2kj));
        if (k == j) E = dd_add(E, dd{1.f, 0.f});
        s.Ed[tid] = E;
      } else if (tid >= 32 && tid < 35) {
        const int i = tid - 32;
        const float* w = s.wv;
        const float* v = s.wv + 3;
        const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
        const dd Wv = dd_sub(two_prod(w[i1], v[i2]), two_prod(w[i2], v[i1]));  // (w x v)_i
        const dd wdv = dd_add(dd_add(two_prod(w[0], v[0]), two_prod(w[1], v[1])), two_prod(w[2], v[2]));
        const dd W2v = dd_sub(dd_mulf(wdv, w[i]), dd_mulf(theta2(w), v[i]));
        s.Vvd[i] = dd_add(dd_add(dd{v[i], 0.f}, dd_mul(s.coefd[1], Wv)), dd_mul(s.coefd[2], W2v));
      }
      __syncthreads();
      if (tid < 12) {  // candidate T o exp(step xi) and the difference D = T_c - T
        const int i = tid / 4, k = tid % 4;
        dd v;
        if (k < 3) {
          v = dd_mul(s.Rd[3 * i], s.Ed[k]);
          v = dd_fma(s.Rd[3 * i + 1], s.Ed[3 + k], v);
          v = dd_fma(s.Rd[3 * i + 2], s.Ed[6 + k], v);
        } else {
          v = dd_fma(s.Rd[3 * i], s.Vvd[0], s.td[i]);
          v = dd_fma(s.Rd[3 * i + 1], s.Vvd[1], v);
          v = dd_fma(s.Rd[3 * i + 2], s.Vvd[2], v);
        }
        s.Tcd[tid] = v;
        s.dld[tid] = dd_sub(v, k < 3 ? s.Rd[3 * i + k] : s.td[i]);
      }
      __syncthreads();
      if (tid < 32) {  // G D and dQ = 2 <M1, D> + <D, G D>
        if (tid < 12) {
          const dd* Af = &s.Ad[0][0];
          // lane tid owns (G D)_ik, i = tid / 4, k = tid % 4, from the model entries
          // A^{q(k,l)}_{i j} (j = 0..2, l = 0..3) (offsets from integer arithmetic: an
          // array kept across the loop spills)
          int gidx[12];
          {
            const int i = tid / 4, k = tid % 4;
#pragma unroll
            for (int l = 0; l < 4; ++l)
#pragma unroll
              for (int j = 0; j < 3; ++j) gidx[3 * l + j] = pair_q(k, l) * 6 + sym_p(i, j);
          }
          dd gl[4];
#pragma unroll
          for (int l = 0; l < 4; ++l) {  // four independent chains of three
            gl[l] = dd_mul(Af[gidx[3 * l]], s.dld[l]);
            gl[l] = dd_fma(Af[gidx[3 * l + 1]], s.dld[4 + l], gl[l]);
            gl[l] = dd_fma(Af[gidx[3 * l + 2]], s.dld[8 + l], gl[l]);
          }
          const dd g = dd_add(dd_add(gl[0], gl[1]), dd_add(gl[2], gl[3]));
          s.Gdd[tid] = g;
          s.dqv[tid] = dd_mul(s.dld[tid], dd_add(dd_scale2(s.M1d[tid], 2.f), g));
        }
        // fixed-order tree over the 12 terms in shared memory (a warp-shuffle tree of the
        // pairs measured several times slower here)
        __syncwarp();
        if (tid < 6) s.dqv[tid] = dd_add(s.dqv[tid], s.dqv[tid + 6]);
        __syncwarp();
        if (tid < 3) s.dqv[tid] = dd_add(s.dqv[tid], s.dqv[tid + 3]);
        __syncwarp();
        if (tid == 0) s.dQd = dd_add(dd_add(s.dqv[0], s.dqv[1]), s.dqv[2]);
      }
      __syncthreads();
      const bool acc = dd_le0(s.dQd);
      if (acc) {
        if (tid < 12) {
          const int i = tid / 4, k = tid % 4;
          if (k < 3)
            s.Rd[3 * i + k] = s.Tcd[tid];
          else
            s.td[i] = s.Tcd[tid];
          s.M1d[tid] = dd_add(s.M1d[tid], s.Gdd[tid]);
        }
        if (tid == 0) {
          s.Qd = dd_add(s.Qd, s.dQd);
          s.accepted = 1;
        }
        __syncthreads();
        break;
      }
      if (tid == 0) ++s.halvings;
      __syncthreads();
    }
    if (tid == 0) {
      float nx = 0.f;  // |step xi|^2 of the accepted step (FP32 suffices for the test)
#pragma unroll
      for (int a = 0; a < 6; ++a) nx += (step * s.xf[a]) * (step * s.xf[a]);
      if (!s.accepted || nx < static_cast<float>(newton_tol) * static_cast<float>(newton_tol)) s.go = 0;
    }
    __syncthreads();
    if (!s.go) break;
  }
  // the pose and objective in FP64 for the caller
  if (tid < 9) {
    s.R[tid] = dd_to(s.Rd[tid]);
  } else if (tid < 12) {
    s.t[tid - 9] = dd_to(s.td[tid - 9]);
  } else if (tid == 32) {
    s.Q = dd_to(s.Qd);
  }
  __syncthreads();
}

// One CTA per pair: its Newton M step, sigma^2 update, trace and E-step constants.
// Global memory is touched in three rounds: the constant tables (before the wait for
// the predecessor), then the moments, the counter and a copy of the pair's state (one
// coalesced read), and at the end the updated state (one coalesced write); every
// scalar of the epilogue is worked on in shared memory.
constexpr int kStateWords = static_cast<int>(sizeof(EmState) / sizeof(int));
static_assert(sizeof(EmState) % sizeof(int) == 0 && kStateWords <= kMThreads, "one word of the state per thread");

// rows != nullptr: the pair's combine rows [blk_off[pair] * per_block, blk_off[pair + 1] *
// per_block) are summed here (in row order, FP64) into mom_all first, in place of the
// cross-block reduction kernel.
// yl != nullptr: the epilogue also writes the sigma-dependent record planes of the pair's
// tiles [tile_off[pair], tile_off[pair + 1]) for the next E step (one thread per slot), in
// place of the prescale kernel.
static_assert(kMThreads == kTile, "one thread per record slot");
__global__ void __launch_bounds__(kMThreads) mstep_em_kernel(const double* __restrict__ rows,
                                                              const int* __restrict__ blk_off, int per_block,
                                                              double* __restrict__ mom_all,
                                                              EmState* __restrict__ st_all, DevParams dp,
                                                              double* __restrict__ trace_all, int trace_iters,
                                                              int* __restrict__ done_count, int P,
                                                              const float4* __restrict__ yl,
                                                              const int* __restrict__ tile_off, int mode,
                                                              float* __restrict__ rec) {
  __shared__ Shared s;
  __shared__ EmState es;
  __shared__ double mom_sh[kGlob];
  __shared__ double nll_sh, pout_sh;
  __shared__ float dmot[12];
  __shared__ int finish_sh, nll_stop_sh;  // written by different lanes in the same phase
  const int tid = threadIdx.x;
  load_tables(s);
  pdl_wait();
  pdl_launch_dependents();
  const int pair = blockIdx.x;
  EmState* st = st_all + pair;
  const double* mom = mom_all + static_cast<size_t>(pair) * kGlob;
  if (rows) {
    if (tid < kGlob) {
      const int r0 = blk_off[pair] * per_block, r1 = blk_off[pair + 1] * per_block;
      double v = 0.0;
      for (int r = r0; r < r1; ++r) v += rows[static_cast<size_t>(r) * kGlob + tid];
      mom_sh[tid] = v;
      mom_all[static_cast<size_t>(pair) * kGlob + tid] = v;
    }
    __syncthreads();
    mom = mom_sh;
  }
  const int finished = *done_count;
  if (tid < kStateWords) reinterpret_cast<int*>(&es)[tid] = reinterpret_cast<const int*>(st)[tid];
  setup_newton(s, mom, st->R, st->t);
  if (tid == 97) {
    nll_sh = mom[75];
    pout_sh = mom[74];
  }
  __syncthreads();
  if (finished >= P || es.done) return;  // uniform over the CTA
  if (!(s.NP > 0.0)) {
    if (tid == 0) {
      st->numeric_fail = 1;
      st->done = 1;
      atomicAdd(done_count, 1);
    }
    return;
  }
  newton(s, dp.newton_max, dp.newton_tol);
  // --- epilogue, lane-parallel on the shared copy of the state ---
  const int it = es.iter;
  if (tid < 9) {  // rotation change (FP32 suffices for the motion test)
    dmot[tid] = dd_f(dd_sub(s.Rd[tid], s.Rod[tid]));
  } else if (tid < 12) {  // translation change of the source centroid: dt - dR mu_x
    const int i = tid - 9;
    float d = dd_f(dd_sub(s.td[i], s.tod[i]));
    for (int j = 0; j < 3; ++j)
      d -= dd_f(dd_sub(s.Rd[3 * i + j], s.Rod[3 * i + j])) * static_cast<float>(es.mu_x[j]);
    dmot[tid] = d;
  } else if (tid == 32) {  // sigma^2 and the E-step constants it sets
    const double s2 = s.Q * __drcp_rn(3.0 * s.NP);
    const bool at_floor = !(s2 > es.sigma2_floor);
    const double s2c = at_floor ? es.sigma2_floor : s2;
    es.sigma2 = s2c;
    set_sigma_constants(&es, static_cast<float>(s2c));
    finish_sh = (at_floor || it + 1 >= dp.max_iters) ? 1 : 0;
  } else if (tid >= 64 && tid < 76) {  // new pose (FP64) and its FP32 copies for the next E step
    const int e = tid - 64;
    if (e < 9) {
      es.R[e] = s.R[e];
      es.Rf[e] = static_cast<float>(s.R[e]);
    } else {
      es.t[e - 9] = s.t[e - 9];
      es.tf[e - 9] = static_cast<float>(s.t[e - 9]);
    }
  } else if (tid == 96) {  // termination on the log-likelihood of Eq. (4): change since the previous E step
    const double nll = nll_sh;
    nll_stop_sh = dp.nll_tol > 0.0 && it > 0 && fabs(nll - es.nll_prev) <= dp.nll_tol * fabs(nll);
    es.nll_prev = nll;
  }
  __syncthreads();
  if (tid == 0) {
    float fro = 0.f;
    for (int i = 0; i < 9; ++i) fro += dmot[i] * dmot[i];
    const float ang = 2.f * asinf(fminf(1.f, sqrtf(fro) * 0.35355339f));
    const float dtr = sqrtf(dmot[9] * dmot[9] + dmot[10] * dmot[10] + dmot[11] * dmot[11]);
    const float motion = fmaxf(ang, dtr / static_cast<float>(es.diag > 0 ? es.diag : 1.0));
    if (trace_all) {
      double* tr = trace_all + (static_cast<size_t>(pair) * trace_iters + it) * 8;
      tr[0] = es.sigma2;
      tr[1] = s.NP;
      tr[2] = s.Q;
      tr[3] = s.iters;
      tr[4] = s.damped;
      tr[5] = motion;
      tr[6] = nll_sh;
      tr[7] = pout_sh;
    }
    es.iter = it + 1;
    if (finish_sh || nll_stop_sh || (dp.tol > 0.0 && motion < dp.tol)) {
      es.done = 1;
      atomicAdd(done_count, 1);
    }
  }
  __syncthreads();
  if (yl && !es.done)
    for (int t = tile_off[pair]; t < tile_off[pair + 1]; ++t) prescale_slot(rec, yl, t, tid, es.sqc, es.L, mode);
  if (tid < kStateWords) reinterpret_cast<int*>(st)[tid] = reinterpret_cast<const int*>(&es)[tid];
}

__global__ void __launch_bounds__(kMThreads) mstep_standalone_kernel(double* __restrict__ io, DevParams dp) {
  __shared__ Shared s;
  const int tid = threadIdx.x;
  load_tables(s);
  setup_newton(s, io, io + 80, io + 89);
  __syncthreads();
  newton(s, dp.newton_max, dp.newton_tol);
  if (tid != 0) return;
  double* out = io + 96;
  for (int i = 0; i < 9; ++i) out[i] = s.R[i];
  for (int i = 0; i < 3; ++i) out[9 + i] = s.t[i];
  out[12] = s.NP > 0.0 ? s.Q / (3.0 * s.NP) : 0.0;
  out[13] = s.Q;
  out[14] = s.iters;
  out[15] = s.damped;
  out[16] = s.halvings;
}

struct PoseArg {
  double R[9];
  double t[3];
};

// E-step constants for a pose given in the caller's frame: the centred
// translation is t_c = R mu_x + t - mu_y (centroids already in the state).
__global__ void constants_kernel(EmState* st, double sigma2, double w, double V, PoseArg pose) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = 0; i < 9; ++i) st->R[i] = pose.R[i];
  for (int i = 0; i < 3; ++i)
    st->t[i] = pose.R[3 * i] * st->mu_x[0] + pose.R[3 * i + 1] * st->mu_x[1] + pose.R[3 * i + 2] * st->mu_x[2] +
               pose.t[i] - st->mu_y[i];
  st->sigma2 = sigma2;
  st->V = V;
  st->log2_V = log2(V);
  st->log2_wodds = w > 0.0 ? log2(w) - log2(1.0 - w) : -INFINITY;
  st->ln_1mw = log1p(-w);
  st->w0 = w;
  st->nll_prev = 0.0;
  st->done = 0;
  st->iter = 0;
  st->numeric_fail = 0;
  set_estep_constants(st);
}

}  // namespace

cudaError_t launch_mstep(const BatchPlan& p, const Dev& d, const double* rows, double* mom, const DevParams& dp,
                         double* trace, int trace_iters, const float4* yl, int mode, float* rec, cudaStream_t s) {
  return launch_k(mstep_em_kernel, dim3(p.g.P), dim3(kMThreads), 0, s, rows, d.tab + p.g.o_blk_off,
                  p.g.SB / kCombineSources, mom, d.st, dp, trace, trace_iters, d.done_count, p.g.P, yl,
                  d.tab + p.g.o_tile_off, mode, rec);
}

cudaError_t launch_mstep_standalone(double* io, const DevParams& dp, cudaStream_t s) {
  mstep_standalone_kernel<<<1, kMThreads, 0, s>>>(io, dp);
  return cudaGetLastError();
}

cudaError_t launch_estep_constants(EmState* st, double sigma2, double w, double V, const double* R,
                                   const double* t, cudaStream_t s) {
  PoseArg pa;
  for (int i = 0; i < 9; ++i) pa.R[i] = R[i];
  for (int i = 0; i < 3; ++i) pa.t[i] = t[i];
  constants_kernel<<<1, 32, 0, s>>>(st, sigma2, w, V, pa);
  return cudaGetLastError();
}

}  // namespace lsg
