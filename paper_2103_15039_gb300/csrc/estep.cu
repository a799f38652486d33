// E step of LSG-CPD on sm_103a (Eq. (5) evaluated in the form of Eq. (9)).
//
// For every source n and every target m (Eq. (2)):
//   r_mn = z_n - y_m,  d_mn = |r|^2 + alpha_m (n_m . r)^2 = |r|^2 + (a_m . r)^2,  a = sqrt(alpha) n,
//   P_mn = pi_m e^{-d/(2 s2)} / (sum_k pi_k e^{-d_k/(2 s2)} + gamma_n),
//   gamma_n = w/(1-w) (2 pi s2)^{3/2} / V.
// The kernel never forms P.  With c = log2(e)/(2 s2) and coordinates scaled by
// sqrt(c) (z^ = sqrt(c) z, y^ = sqrt(c) y, so that c d = |z^ - y^|^2 + (a . (z^ - y^))^2)
// it evaluates e_mn = 2^-q_mn with
//   q_mn = c d_mn + lambda_m (+ L_n),   lambda_m = L - l_m  (or -l_m with per-source shifts),
// l_m = log2 pi_m and L (L_n) the log2 shift, and accumulates per source
//   S0 = sum e,  B = sum e b_m (b_m = Lambda_m y_m),  W = sum e a a^T,  Dq = sum e q
// (+ El = sum e lambda_m with per-source shifts).  The combine turns them into
// the M step's statistics with one division per source:
//   sum_m e Lambda_m r_mn = S0 z + W z - B  (Lambda_m = I + a a^T),
//   sum_m e d_mn = (Dq - lambda S0) / c     (lambda uniform; else Dq - L_n S0 - El).
// Per pair that is 21 packed-FP32 operations for two targets at once (3 adds,
// 3 for a . r, 4 for q, 11 accumulations) and two MUFU.EX2.
//
// Hot-loop layout (GB300):
//  * a CTA = 8 warps (S = 4) or 4 warps; each thread owns S sources (z^_n duplicated into both
//    halves of an FP32x2 register) and 11 (12) FP32x2 accumulators per source;
//  * the two halves of every packed register belong to two consecutive
//    targets, so every operation of the pair update is one packed
//    FADD2/FMUL2/FFMA2;
//  * target tiles (kTile records, 8 KB) stream into a 4-stage shared-memory
//    ring by cp.async.bulk (TMA bulk copy) completing on mbarriers; every warp
//    reads the tile with broadcast shared loads;
//  * the sigma-dependent record planes are rewritten once per EM iteration by a
//    small O(M) pass (prescale), so the hot loop needs no per-target setup;
//  * work = (source block) x (target tile) units split stream-K style over a
//    grid of (SM count x resident CTAs); a CTA flushes its FP32 partial
//    moments at block boundaries and every seg_cap tiles, so FP32 sums stay
//    short; the combine adds the pieces (compensated) in a fixed order.
// Kernel variants (MODE): 0 uniform shift; 1 per-source shift L_n; 2 per-source
// shift with packed f16x2 exponentials; 3 the max pass that finds L_n.
// No tensor cores: the contraction depth is 3, so the work is FP32-pipe bound.
#include <math.h>

#include "estep_common.cuh"
#include "internal.cuh"
#include "pipeline.cuh"

namespace lsg {
namespace {

constexpr int kStages = 4;
// warps per CTA of the hot kernel: with 4 sources per thread (190 registers) one
// 8-warp CTA per SM shares each tile among 1024 sources; narrower variants run
// several 4-warp CTAs per SM
template <int S>
__host__ __device__ constexpr int warps_for() { return S >= 4 ? 8 : 4; }
template <int S>
__host__ __device__ constexpr int min_ctas_for() { return S >= 4 ? 1 : 3; }

// 2^-q for both halves through one packed f16x2 MUFU.EX2 (the mixed-precision
// variant): -q is rounded to f16 (11-bit significand), the result widened back.
__device__ __forceinline__ float2 ex2_neg_f16x2(float2 q) {
  uint32_t h;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(-q.y), "f"(-q.x));  // upper = y, lower = x
  asm("ex2.approx.f16x2 %0, %1;" : "=r"(h) : "r"(h));
  float2 e;
  asm("{ .reg .f16 lo, hi; mov.b32 {lo, hi}, %2; cvt.f32.f16 %0, lo; cvt.f32.f16 %1, hi; }"
      : "=f"(e.x), "=f"(e.y)
      : "r"(h));
  return e;
}

struct Src {
  float2 z0, z1, z2;  // z^_n in both halves
  float2 ls;          // L_n in both halves (per-source shift mode)
};

struct Acc {
  float2 s0, b0, b1, b2, w00, w01, w02, w11, w12, w22, d, el;
};

struct Tgt {  // two consecutive targets, one per half
  float2 ny0, ny1, ny2, lam, a0, a1, a2, q00, q01, q02, q11, q12, q22, b0, b1, b2;
};


// One source against two targets: 21 packed FP32 operations (22 + 1 with
// per-source shifts) and 2 EX2 (one packed f16x2 EX2 with MODE 2).
// MODE: 0 uniform shift, 1 per-source shift, 2 per-source shift + f16x2 exponentials.
template <int MODE>
__device__ __forceinline__ void pair_update(Acc& A, const Src& s, const Tgt& g) {
  constexpr bool MAXS = MODE == 1 || MODE == 2;
  const float2 r0 = __fadd2_rn(s.z0, g.ny0);
  const float2 r1 = __fadd2_rn(s.z1, g.ny1);
  const float2 r2 = __fadd2_rn(s.z2, g.ny2);
  float2 v = __fmul2_rn(g.a0, r0);  // v = a . r^
  v = __ffma2_rn(g.a1, r1, v);
  v = __ffma2_rn(g.a2, r2, v);
  float2 q = MAXS ? __fadd2_rn(g.lam, s.ls) : g.lam;  // q = c d + lambda_m (+ L_n)
  q = __ffma2_rn(r0, r0, q);
  q = __ffma2_rn(r1, r1, q);
  q = __ffma2_rn(r2, r2, q);
  q = __ffma2_rn(v, v, q);
  if (MODE == 3) {  // max pass (records hold lambda_m = -l_m): running min of q = c d - l_m
    A.s0.x = fminf(A.s0.x, q.x);
    A.s0.y = fminf(A.s0.y, q.y);
    return;
  }
  float2 e;
  if (MODE == 2) {
    e = ex2_neg_f16x2(q);
  } else {
    e.x = ex2_neg(q.x);
    e.y = ex2_neg(q.y);
  }
  A.s0 = __fadd2_rn(A.s0, e);
  A.b0 = __ffma2_rn(e, g.b0, A.b0);
  A.b1 = __ffma2_rn(e, g.b1, A.b1);
  A.b2 = __ffma2_rn(e, g.b2, A.b2);
  A.w00 = __ffma2_rn(e, g.q00, A.w00);
  A.w01 = __ffma2_rn(e, g.q01, A.w01);
  A.w02 = __ffma2_rn(e, g.q02, A.w02);
  A.w11 = __ffma2_rn(e, g.q11, A.w11);
  A.w12 = __ffma2_rn(e, g.q12, A.w12);
  A.w22 = __ffma2_rn(e, g.q22, A.w22);
  A.d = __ffma2_rn(e, q, A.d);
  if (MAXS) A.el = __ffma2_rn(e, g.lam, A.el);
}

// All pairs of one tile: every thread walks the tile two targets at a time
// (broadcast 64-bit shared loads of the 16 planes).
template <int S, int MODE>
__device__ __forceinline__ void tile_compute(const float* tile, const Src (&src)[S], Acc (&acc)[S]) {
  const float2* T2 = reinterpret_cast<const float2*>(tile);
  constexpr int H = kTile / 2;
#pragma unroll 2
  for (int q = 0; q < H; ++q) {
    Tgt g;
    g.ny0 = T2[0 * H + q];
    g.ny1 = T2[1 * H + q];
    g.ny2 = T2[2 * H + q];
    g.lam = T2[3 * H + q];
    g.a0 = T2[4 * H + q];
    g.a1 = T2[5 * H + q];
    g.a2 = T2[6 * H + q];
    g.q00 = T2[7 * H + q];
    g.q01 = T2[8 * H + q];
    g.q02 = T2[9 * H + q];
    g.q11 = T2[10 * H + q];
    g.q12 = T2[11 * H + q];
    g.q22 = T2[12 * H + q];
    g.b0 = T2[13 * H + q];
    g.b1 = T2[14 * H + q];
    g.b2 = T2[15 * H + q];
#pragma unroll
    for (int s = 0; s < S; ++s) pair_update<MODE>(acc[s], src[s], g);
  }
}

template <int MODE>
__device__ __forceinline__ void store_acc(float* dst, int SB, int nl, const Acc& a) {
  constexpr bool MAXS = MODE == 1 || MODE == 2;
  if (MODE == 3) {
    dst[nl] = fminf(a.s0.x, a.s0.y);
    return;
  }
  dst[0 * SB + nl] = a.s0.x + a.s0.y;
  dst[1 * SB + nl] = a.b0.x + a.b0.y;
  dst[2 * SB + nl] = a.b1.x + a.b1.y;
  dst[3 * SB + nl] = a.b2.x + a.b2.y;
  dst[4 * SB + nl] = a.w00.x + a.w00.y;
  dst[5 * SB + nl] = a.w01.x + a.w01.y;
  dst[6 * SB + nl] = a.w02.x + a.w02.y;
  dst[7 * SB + nl] = a.w11.x + a.w11.y;
  dst[8 * SB + nl] = a.w12.x + a.w12.y;
  dst[9 * SB + nl] = a.w22.x + a.w22.y;
  dst[10 * SB + nl] = a.d.x + a.d.y;
  if (MAXS) dst[11 * SB + nl] = a.el.x + a.el.y;
}

template <int S, int MODE>
__global__ void __launch_bounds__(warps_for<S>() * 32, min_ctas_for<S>())
    estep_kernel(const float4* __restrict__ xs, const float* __restrict__ rec, const EmState* __restrict__ st,
                 const float* __restrict__ ls_n, float* __restrict__ part, const int* __restrict__ tab,
                 const int* __restrict__ done_count, int* __restrict__ status, Geo g) {
  constexpr int SB = warps_for<S>() * 32 * S;
  constexpr bool MAXS = MODE == 1 || MODE == 2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* tiles = reinterpret_cast<float*>(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + kStages * kTileBytes);

  pdl_wait();
  if (*done_count >= g.P) return;
  const int* tile_off = tab + g.o_tile_off;
  const int* block_pair = tab + g.o_block_pair;
  const int* unit_off = tab + g.o_unit_off;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const long long G = gridDim.x;
  const long long u0 = static_cast<long long>(blockIdx.x) * g.U / G;
  const long long u1 = static_cast<long long>(blockIdx.x + 1) * g.U / G;
  const int n_units = static_cast<int>(u1 - u0);
  if (n_units <= 0) return;
  const int first_block = tab[g.o_cta_block + blockIdx.x];
  const int first_slot = tab[g.o_cta_slot + blockIdx.x];

  Cursor prod{first_block};  // used by thread 0 only
  auto tile_of = [&](long long u) -> long long {
    const int b = prod.advance(unit_off, u);
    return static_cast<long long>(tile_off[block_pair[b]]) + (u - unit_off[b]);
  };
  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) mbar_init(&full[i], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    for (int i = 0; i < kStages && i < n_units; ++i)
      bulk_load(tiles + i * kTileFloats, rec + tile_of(u0 + i) * kTileFloats, kTileBytes, &full[i]);
  }

  bool abort = false;
  int seg = 0;
  int i = 0;  // units consumed by this CTA
  long long u = u0;
  Cursor cons{first_block};
  while (u < u1) {
    const int b = cons.advance(unit_off, u);
    const EmState* sp = st + block_pair[b];
    const long long block_end = unit_off[b + 1];
    long long seg_end = u + g.seg_cap;
    if (seg_end > block_end) seg_end = block_end;
    if (seg_end > u1) seg_end = u1;

    // a pair whose EM loop has finished keeps its tiles flowing through the ring but is not computed
    const bool live = !sp->done;
    const float sqc = sp->sqc;
    float Rm[9], tv[3];
#pragma unroll
    for (int q = 0; q < 9; ++q) Rm[q] = sp->Rf[q];
#pragma unroll
    for (int q = 0; q < 3; ++q) tv[q] = sp->tf[q];
    Src src[S];
    Acc acc[S];
#pragma unroll
    for (int s2 = 0; s2 < S; ++s2) {
      const int nl = warp * 32 * S + s2 * 32 + lane;
      const long long n = static_cast<long long>(b) * SB + nl;
      const float4 x = xs[n];
      // z = R x + t in FP32 (centred frame of the pair)
      const float z0 = fmaf(Rm[0], x.x, fmaf(Rm[1], x.y, fmaf(Rm[2], x.z, tv[0])));
      const float z1 = fmaf(Rm[3], x.x, fmaf(Rm[4], x.y, fmaf(Rm[5], x.z, tv[1])));
      const float z2 = fmaf(Rm[6], x.x, fmaf(Rm[7], x.y, fmaf(Rm[8], x.z, tv[2])));
      src[s2].z0 = dup(sqc * z0);
      src[s2].z1 = dup(sqc * z1);
      src[s2].z2 = dup(sqc * z2);
      src[s2].ls = dup(MAXS ? ls_n[n] : 0.f);
      const float2 zero = make_float2(0.f, 0.f);
      acc[s2] = Acc{MODE == 3 ? make_float2(INFINITY, INFINITY) : zero, zero, zero, zero, zero, zero, zero, zero,
                    zero, zero, zero, zero};
    }

    for (; u < seg_end; ++u, ++i) {
      const int stage = i % kStages;
      const uint32_t parity = static_cast<uint32_t>(i / kStages) & 1u;
      const bool ok = mbar_wait(&full[stage], parity);
      if (!ok && lane == 0) atomicOr(status, kStatusTimeout);
      if (live) tile_compute<S, MODE>(tiles + stage * kTileFloats, src, acc);
      if (__syncthreads_or(!ok)) {
        abort = true;
        break;
      }
      if (tid == 0 && i + kStages < n_units)
        bulk_load(tiles + stage * kTileFloats, rec + tile_of(u0 + i + kStages) * kTileFloats, kTileBytes,
                  &full[stage]);
    }
    if (abort) break;
    float* dst = part + static_cast<size_t>(first_slot + seg) * kMom * SB;
#pragma unroll
    for (int s2 = 0; s2 < S; ++s2) store_acc<MODE>(dst, SB, warp * 32 * S + s2 * 32 + lane, acc[s2]);
    ++seg;
  }
  if (abort && tid == 0) {
    // let copies still in flight land before the CTA's shared memory is released
    for (int k = 0; k < kStages; ++k) {  // units i .. i + kStages - 1 were issued
      const int j = i + k;
      if (j < n_units) mbar_wait(&full[j % kStages], static_cast<uint32_t>(j / kStages) & 1u);
    }
  }
}

// ---------------------------------------------------------------------------
// Prescale: the sigma-dependent planes of every record slot for the current
// state of its pair: -sqrt(c) y (3) and lambda_m (L - l_m, or -l_m with
// per-source shifts; kPadLambda for padding).  One thread per slot.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kTile)
    prescale_kernel(const float4* __restrict__ yl, const EmState* __restrict__ st, const int* __restrict__ tab,
                    const int* __restrict__ done_count, int mode, float* __restrict__ rec, Geo g) {
  pdl_wait();
  pdl_launch_dependents();
  if (*done_count >= g.P) return;
  const int tile = blockIdx.x;
  const EmState* sp = st + tab[g.o_tile_pair + tile];
  if (sp->done) return;
  prescale_slot(rec, yl, tile, threadIdx.x, sp->sqc, sp->L, mode);
}

// ---------------------------------------------------------------------------
// Per-source shift for the max-shift mode (used when w = 0, when a fixed shift
// could overflow FP32, when l_m or w_n vary, and with f16 exponentials):
// L_n = max(log2 gamma_n, max_m (l_m - c d_mn)) over the targets of the
// source's pair.  The max itself comes from a pass of the E-step kernel in
// MODE 3 (records prescaled with lambda_m = -l_m: l_m - c d = -q), which leaves
// min_m q per source in every partial slot; this kernel takes the minimum over
// the source block's slots and forms L_n and gamma'_n.
// ---------------------------------------------------------------------------
constexpr int kShiftThreads = 128;

__global__ void __launch_bounds__(kShiftThreads)
    shift_kernel(const float4* __restrict__ xs, const float* __restrict__ part, const EmState* __restrict__ st,
                 const int* __restrict__ tab, const int* __restrict__ done_count, int cf_x,
                 float* __restrict__ ls_n, float* __restrict__ gam_n, Geo g) {
  pdl_wait();
  pdl_launch_dependents();
  if (*done_count >= g.P) return;
  // every CTA covers kShiftThreads sources of one source block (SB is a multiple)
  const long long n = static_cast<long long>(blockIdx.x) * kShiftThreads + threadIdx.x;
  const int b = static_cast<int>(n / g.SB);
  const int nl = static_cast<int>(n - static_cast<long long>(b) * g.SB);
  const EmState* sp = st + tab[g.o_block_pair + b];
  if (sp->done) return;
  const int first = tab[g.o_block_slot + 2 * b];
  const int count = tab[g.o_block_slot + 2 * b + 1];
  float best = INFINITY;  // min_m q
  for (int j = first; j < first + count; ++j) best = fminf(best, part[static_cast<size_t>(j) * kMom * g.SB + nl]);
  // log2 gamma_n (-inf without outlier term); per source with confidences: w_n = 1 - (1 - w0) phi_n
  float Lg = sp->L;
  if (cf_x) {
    const float wn = 1.f - static_cast<float>(1.0 - sp->w0) * xs[n].w;
    Lg = (wn > 0.f ? log2f(wn) - log2f(1.f - wn) : -INFINITY) + sp->Lb;
  }
  const float L = fmaxf(-best, Lg);  // padding sources (zero x) get finite values too; never read back
  ls_n[n] = L;
  gam_n[n] = exp2f(Lg - L);  // gamma'_n = 2^(log2 gamma - L_n)
}

// ---------------------------------------------------------------------------
// Combine: per source, add the FP32 pieces with compensated summation,
// normalise by S0 + gamma'_n, and form the 76 contributions to the global
// moments of the M step (FP32 products).  Each warp transposes its 32 x 76
// contributions through shared memory; lane l then sums columns l, l+32, l+64
// over the 32 sources with Neumaier's compensated summation (an error-free
// TwoSum per add), and the CTA adds its warps in FP64.  A CTA covers
// kCombineSources sources of one source block (hence of one pair) and writes
// one row of kGlob doubles; FP64 appears only there and in the per-pair
// cross-row reduction.
// ---------------------------------------------------------------------------
constexpr int kCombineThreads = kCombineSources;
constexpr int kCombineUnroll = 4;
constexpr int kCombineWarps = kCombineThreads / 32;
constexpr int kCPad = kGlob + 1;  // odd row pitch: conflict-free transposition

__global__ void __launch_bounds__(kCombineThreads)
    combine_kernel(const float4* __restrict__ xs, const float* __restrict__ part, const int* __restrict__ tab,
                   const long long* __restrict__ off64, const EmState* __restrict__ st,
                   const int* __restrict__ done_count, int mode, int cf_x, const float* __restrict__ ls_n,
                   const float* __restrict__ gam_n, double* __restrict__ rows, float* __restrict__ per_n, Geo g) {
  __shared__ float buf[kCombineWarps][32 * kCPad];
  __shared__ double acc[kCombineWarps][kGlob];
  pdl_wait();
  pdl_launch_dependents();
  if (*done_count >= g.P) return;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const long long n = static_cast<long long>(blockIdx.x) * kCombineThreads + tid;
  const int b = static_cast<int>(n / g.SB);
  const int pair = tab[g.o_block_pair + b];
  const EmState* sp = st + pair;
  if (sp->done) return;  // uniform over the CTA: its rows are not read again
  const long long local = n - static_cast<long long>(tab[g.o_blk_off + pair]) * g.SB;
  const long long Np = off64[pair + 1] - off64[pair];
  const bool valid = local < Np;
  const int nl = static_cast<int>(n - static_cast<long long>(b) * g.SB);
  const int nmom = mode ? kMom : kMom - 1;
  float m[kMom], cmp[kMom];
#pragma unroll
  for (int k = 0; k < kMom; ++k) m[k] = cmp[k] = 0.f;
  float x0 = 0.f, x1 = 0.f, x2 = 0.f, xw = 1.f, gp = 0.f, L = 0.f, lam = 0.f;
  if (valid) {
    const int first = tab[g.o_block_slot + 2 * b];
    const int count = tab[g.o_block_slot + 2 * b + 1];
    // Kahan summation of the pieces, in slot order; the loads of up to kCombineUnroll slots
    // are issued before they are summed (the sums are latency-bound on L2 otherwise)
    for (int j0 = first; j0 < first + count; j0 += kCombineUnroll) {
      float v[kCombineUnroll][kMom];
#pragma unroll
      for (int jj = 0; jj < kCombineUnroll; ++jj) {
        const bool in = j0 + jj < first + count;
        const float* src = part + static_cast<size_t>(in ? j0 + jj : first) * kMom * g.SB + nl;
#pragma unroll
        for (int k = 0; k < kMom; ++k) v[jj][k] = (in && k < nmom) ? __ldg(src + static_cast<size_t>(k) * g.SB) : 0.f;
      }
#pragma unroll
      for (int jj = 0; jj < kCombineUnroll; ++jj) {
        if (j0 + jj < first + count) {
#pragma unroll
          for (int k = 0; k < kMom; ++k) {
            const float y = v[jj][k] - cmp[k];
            const float t = m[k] + y;
            cmp[k] = (t - m[k]) - y;
            m[k] = t;
          }
        }
      }
    }
    const float4 x = xs[n];
    x0 = x.x;
    x1 = x.y;
    x2 = x.z;
    xw = x.w;
    if (mode) {
      L = ls_n[n];
      gp = gam_n[n];
      lam = L;  // sum e c d = Dq - L_n S0 - El
    } else {
      L = sp->L;
      gp = (sp->log2_wodds > -INFINITY) ? 1.f : 0.f;
      lam = sp->lam;  // sum e c d = Dq - lambda S0
    }
  }
  const float S0 = m[0];
  // z = R x + t (centred frame), h = S0 z + W z - B = sum e Lambda_m r_mn
  const float* Rr = sp->Rf;
  const float z0 = fmaf(Rr[0], x0, fmaf(Rr[1], x1, fmaf(Rr[2], x2, sp->tf[0])));
  const float z1 = fmaf(Rr[3], x0, fmaf(Rr[4], x1, fmaf(Rr[5], x2, sp->tf[1])));
  const float z2 = fmaf(Rr[6], x0, fmaf(Rr[7], x1, fmaf(Rr[8], x2, sp->tf[2])));
  const float hr0 = fmaf(S0 + m[4], z0, fmaf(m[5], z1, fmaf(m[6], z2, -m[1])));
  const float hr1 = fmaf(m[5], z0, fmaf(S0 + m[7], z1, fmaf(m[8], z2, -m[2])));
  const float hr2 = fmaf(m[6], z0, fmaf(m[8], z1, fmaf(S0 + m[9], z2, -m[3])));
  const float cD = fmaf(-lam, S0, m[10]) - (mode ? m[11] : 0.f);  // sum e c d
  const float D = cD / -sp->neg_c;
  const float denom = S0 + gp;
  const float inv = denom > 0.f ? 1.f / denom : 0.f;
  const float Pb = S0 * inv;
  const float h[3] = {hr0 * inv, hr1 * inv, hr2 * inv};
  const float W00 = m[4] * inv, W01 = m[5] * inv, W02 = m[6] * inv, W11 = m[7] * inv, W12 = m[8] * inv,
              W22 = m[9] * inv;
  const float Dn = D * inv;
  const float Pout = gp * inv;
  // -ln((1 - w_n) (2 pi s2)^(-3/2)): the pair's constant, or per source with confidences
  float nll_c = static_cast<float>(sp->nll_const);
  if (cf_x && valid) {
    const float wn = 1.f - static_cast<float>(1.0 - sp->w0) * xw;
    nll_c += static_cast<float>(sp->ln_1mw) - log1pf(-wn);
  }
  const float nll = (valid && denom > 0.f) ? nll_c - (L * 0.6931471805599453f + logf(denom)) : 0.f;
  if (valid && per_n) {
    float4* o = reinterpret_cast<float4*>(per_n + (off64[pair] + local) * 16);
    o[0] = make_float4(Pb, h[0], h[1], h[2]);
    o[1] = make_float4(W00, W01, W02, W11);
    o[2] = make_float4(W12, W22, Dn, Pout);
    o[3] = make_float4(inv, gp, 0.f, 0.f);  // the normaliser of the shifted exponentials, gamma'_n
  }
  const float A[6] = {Pb + W00, W01, W02, Pb + W11, W12, Pb + W22};
  const float xt[4] = {x0, x1, x2, valid ? 1.f : 0.f};
  float* row = buf[warp] + lane * kCPad;
  row[0] = Pb;
  row[1] = Dn;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) row[2 + 4 * i + k] = h[i] * xt[k];
  {
    int j = 14;
#pragma unroll
    for (int p = 0; p < 6; ++p)
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int l = k; l < 4; ++l) row[j++] = A[p] * (xt[k] * xt[l]);
  }
  row[74] = Pout;
  row[75] = nll;
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int col = lane + 32 * i;
    if (col < kGlob) {
      float sum = 0.f, comp = 0.f;
#pragma unroll 8
      for (int r = 0; r < 32; ++r) {  // Neumaier: sum + comp is the exact running sum
        const float v = buf[warp][r * kCPad + col];
        const float t = sum + v;
        comp += (fabsf(sum) >= fabsf(v)) ? ((sum - t) + v) : ((v - t) + sum);
        sum = t;
      }
      acc[warp][col] = static_cast<double>(sum) + static_cast<double>(comp);
    }
  }
  __syncthreads();
  if (tid < kGlob) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kCombineWarps; ++w) s += acc[w][tid];
    rows[static_cast<size_t>(blockIdx.x) * kGlob + tid] = s;
  }
}

// One warp per (pair, moment): lanes take strided rows of the pair, then a
// shuffle tree (FP64).
constexpr int kReduceWarps = 4;

__global__ void final_reduce_kernel(const double* __restrict__ rows, const int* __restrict__ tab,
                                    const EmState* __restrict__ st, const int* __restrict__ done_count,
                                    double* __restrict__ mom, Geo g) {
  pdl_wait();
  pdl_launch_dependents();
  if (*done_count >= g.P) return;
  const int pair = blockIdx.y;
  if (st[pair].done) return;
  const int j = blockIdx.x * kReduceWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= kGlob) return;
  const int per_block = g.SB / kCombineSources;
  const int r0 = tab[g.o_blk_off + pair] * per_block;
  const int r1 = tab[g.o_blk_off + pair + 1] * per_block;
  double v = 0.0;
  for (int r = r0 + lane; r < r1; r += 32) v += rows[static_cast<size_t>(r) * kGlob + j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) mom[static_cast<size_t>(pair) * kGlob + j] = v;
}

template <int S, int MODE>
cudaError_t launch_estep_t(const BatchPlan& p, const Dev& d, const float4* xs, const float* rec,
                           const float* ls_n, float* part, int* status, cudaStream_t s) {
  return launch_k(estep_kernel<S, MODE>, dim3(p.g.grid), dim3(warps_for<S>() * 32), p.smem_bytes, s, xs, rec, d.st,
                  ls_n, part, d.tab, d.done_count, status, p.g);
}

int resident_ctas(int S) {
  int occ = 1;
  const size_t smem = kStages * kTileBytes + kStages * sizeof(uint64_t);
  cudaError_t e = cudaSuccess;
  if (S == 4)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, estep_kernel<4, 0>, warps_for<4>() * 32, smem);
  else if (S == 2)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, estep_kernel<2, 0>, warps_for<2>() * 32, smem);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, estep_kernel<1, 0>, warps_for<1>() * 32, smem);
  if (e != cudaSuccess || occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  return occ;
}

int warps_of(int S) { return S >= 4 ? warps_for<4>() : (S == 2 ? warps_for<2>() : warps_for<1>()); }

// Dense posteriors of one pair (a debugging aid for small problems): thread per
// source, P[m][n] = e_mn / (S0_n + gamma'_n) with e_mn recomputed exactly as the
// E step computes it (same FP32 operations, same exponential), the outlier row
// P[M][n] = Pout_n.  Needs the per-source output of the combine (per_n).
__global__ void __launch_bounds__(128)
    posterior_kernel(const float4* __restrict__ xs, const float* __restrict__ rec, const EmState* __restrict__ st,
                     const float* __restrict__ ls_n, int mode, int half, const float* __restrict__ per_n,
                     long long N, long long M, float* __restrict__ P) {
  const long long n = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const float4 x = xs[n];
  const float* R = st->Rf;
  const float sqc = st->sqc;
  const float z0 = sqc * fmaf(R[0], x.x, fmaf(R[1], x.y, fmaf(R[2], x.z, st->tf[0])));
  const float z1 = sqc * fmaf(R[3], x.x, fmaf(R[4], x.y, fmaf(R[5], x.z, st->tf[1])));
  const float z2 = sqc * fmaf(R[6], x.x, fmaf(R[7], x.y, fmaf(R[8], x.z, st->tf[2])));
  const float Ln = mode ? ls_n[n] : 0.f;
  const float inv = per_n[n * 16 + 12];
  for (long long m = 0; m < M; ++m) {
    const float* r = rec + (m / kTile) * kTileFloats + (m % kTile);
    const float r0 = z0 + r[0 * kTile], r1 = z1 + r[1 * kTile], r2 = z2 + r[2 * kTile];
    float v = r[4 * kTile] * r0;
    v = fmaf(r[5 * kTile], r1, v);
    v = fmaf(r[6 * kTile], r2, v);
    float q = mode ? r[3 * kTile] + Ln : r[3 * kTile];
    q = fmaf(r0, r0, q);
    q = fmaf(r1, r1, q);
    q = fmaf(r2, r2, q);
    q = fmaf(v, v, q);
    const float e = half ? ex2_neg_f16x2(make_float2(q, q)).x : ex2_neg(q);
    P[m * N + n] = e * inv;
  }
  P[M * N + n] = per_n[n * 16 + 11];
}

}  // namespace

cudaError_t launch_posteriors(const float4* xs, const float* rec, const EmState* st, const float* ls_n, int mode,
                              int half, const float* per_n, long long N, long long M, float* P, cudaStream_t s) {
  posterior_kernel<<<static_cast<unsigned>((N + 127) / 128), 128, 0, s>>>(xs, rec, st, ls_n, mode, half, per_n,
                                                                           N, M, P);
  return cudaGetLastError();
}

// Occupancy and CTA shape of the FP32 kernel for the batch planner (plan.cu).
int estep_resident_ctas(int S) { return resident_ctas(S); }
int estep_warps(int S) { return warps_of(S); }
size_t estep_smem_bytes() { return kStages * kTileBytes + kStages * sizeof(uint64_t); }

cudaError_t launch_estep(const BatchPlan& p, const Dev& d, const float4* xs, const float* rec, int mode, int half,
                         const float* ls_n, float* part, int* status, cudaStream_t s) {
  if (mode && half) {
    switch (p.g.S) {
      case 4: return launch_estep_t<4, 2>(p, d, xs, rec, ls_n, part, status, s);
      case 2: return launch_estep_t<2, 2>(p, d, xs, rec, ls_n, part, status, s);
      default: return launch_estep_t<1, 2>(p, d, xs, rec, ls_n, part, status, s);
    }
  }
  if (mode) {
    switch (p.g.S) {
      case 4: return launch_estep_t<4, 1>(p, d, xs, rec, ls_n, part, status, s);
      case 2: return launch_estep_t<2, 1>(p, d, xs, rec, ls_n, part, status, s);
      default: return launch_estep_t<1, 1>(p, d, xs, rec, ls_n, part, status, s);
    }
  }
  switch (p.g.S) {
    case 4: return launch_estep_t<4, 0>(p, d, xs, rec, nullptr, part, status, s);
    case 2: return launch_estep_t<2, 0>(p, d, xs, rec, nullptr, part, status, s);
    default: return launch_estep_t<1, 0>(p, d, xs, rec, nullptr, part, status, s);
  }
}

cudaError_t launch_prescale(const BatchPlan& p, const Dev& d, const float4* yl, int mode, float* rec,
                            cudaStream_t s) {
  return launch_k(prescale_kernel, dim3(p.g.T), dim3(kTile), 0, s, yl, d.st, d.tab, d.done_count, mode, rec, p.g);
}

cudaError_t launch_shift(const BatchPlan& p, const Dev& d, const float4* xs, const float* rec, int cf_x,
                         float* part, int* status, float* ls_n, float* gam_n, cudaStream_t s) {
  cudaError_t e;
  switch (p.g.S) {
    case 4: e = launch_estep_t<4, 3>(p, d, xs, rec, nullptr, part, status, s); break;
    case 2: e = launch_estep_t<2, 3>(p, d, xs, rec, nullptr, part, status, s); break;
    default: e = launch_estep_t<1, 3>(p, d, xs, rec, nullptr, part, status, s);
  }
  if (e != cudaSuccess) return e;
  const long long blocks = static_cast<long long>(p.g.B) * p.g.SB / kShiftThreads;
  return launch_k(shift_kernel, dim3(static_cast<unsigned>(blocks)), dim3(kShiftThreads), 0, s, xs, part, d.st, d.tab,
                  d.done_count, cf_x, ls_n, gam_n, p.g);
}

cudaError_t launch_combine(const BatchPlan& p, const Dev& d, const float4* xs, const float* part, int mode,
                           int cf_x, const float* ls_n, const float* gam_n, double* rows, float* per_n,
                           cudaStream_t s) {
  return launch_k(combine_kernel, dim3(p.g.combine_ctas), dim3(kCombineThreads), 0, s, xs, part, d.tab, d.off64, d.st,
                  d.done_count, mode, cf_x, ls_n, gam_n, rows, per_n, p.g);
}

cudaError_t launch_final_reduce(const BatchPlan& p, const Dev& d, const double* rows, double* mom, cudaStream_t s) {
  dim3 grid((kGlob + kReduceWarps - 1) / kReduceWarps, static_cast<unsigned>(p.g.P));
  return launch_k(final_reduce_kernel, grid, dim3(32 * kReduceWarps), 0, s, rows, d.tab, d.st, d.done_count, mom, p.g);
}

}  // namespace lsg
