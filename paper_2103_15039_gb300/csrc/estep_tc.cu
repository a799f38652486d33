// E step of LSG-CPD with the moment contraction on the tensor cores
// (precision = 2), sm_103a.
//
// The moments of the E step (Eq. (9)) are a product over the targets:
//   [S0, B, W, El]_n = sum_m e_mn f_m,   f_m = [1, b_m, a_m a_m^T, lambda_m],
// the N x M matrix of shifted exponentials e_mn = 2^-q_mn times an M x F matrix
// of target features that do not change during a registration.  That product
// has contraction depth M and runs here on tcgen05; the residual, the
// anisotropic distance and the exponential stay on the FP32 pipe (depth 3, no
// tensor-core form), with the same scaled coordinates and shifts as the FP32
// kernel.  Per pair the FP32 pipe does 10 operations for q and 1 for
// Dq = sum e q (21 in the FP32 kernel).
//
// Precision: e is truncated to TF32 (10 fraction bits) before it is used
// anywhere, so S0, B, W, El and Dq are exact-arithmetic moments of one set of
// weights e' = e (1 - delta), 0 <= delta < 2^-10, accumulated in FP32.  The
// features are split hi + lo in TF32 (about 21 significant bits).  Relative to
// the FP32 kernel, per-source normalised moments move by at most ~2^-9.
//
// CTA (one per SM; all 512 TMEM columns; 1024 sources = 8 matrices of 128 rows):
//   warps 0-15 compute, 2 sources per thread.  Thread (w, l) owns sources
//              w*64 + s*32 + l (s = 0, 1) of the source block; source s of
//              warp w is row 32 (w % 4) + l of matrix mi = 2 (w / 4) + s (a
//              warp reaches only its quarter of the TMEM lanes).  Warps 0-7
//              form half 0 (matrices 0-3), warps 8-15 half 1 (matrices 4-7);
//              the halves never wait for each other.  For every chunk of 32
//              targets a thread writes its 2 x 32 exponentials into TMEM (the
//              A operand), 16 at a time.
//   warps 16, 17  MMA issuer of half 0 (also TMEM owner) and of half 1: one
//              thread each issues the MMAs of its 4 matrices (M = 128 sources,
//              N = 32 features, K = 8 targets per instruction) and commits.
//   warp 18    producer: bulk copies (cp.async.bulk) of each target tile:
//              16 KB of features in the canonical K-major core-matrix layout
//              (the B operand) and the 7 record planes q needs.
// TMEM columns: accumulators D of matrix mi at 32 mi (F32), the A chunk buffer
// of matrix mi (32 TF32 columns) at 256 + 32 mi.
// mbarriers (every wait is bounded; a timeout sets ETIMEOUT, lets the copies
// and MMAs in flight finish, frees TMEM and returns):
//   full[stage]  tile landed              empty[stage]  16 compute warps + both MMA commits
//   a_full[h]    8 warps wrote A of half h   a_empty[h]  MMA commit (A of half h consumed)
//   d_full[h]    segment's MMAs of half h done   d_empty[h]  8 warps read D of half h
// The MMAs of chunk c run while the compute warps compute the first 16 targets
// of chunk c + 1; the buffer is reused only after they complete.
// Segments (FP32 flush points) and partial slots are those of the FP32 kernel
// with 4 sources per thread (source blocks of 1024), so the combine is shared.
#include <math.h>

#include "estep_common.cuh"
#include "internal.cuh"
#include "pipeline.cuh"

namespace lsg {
namespace {

constexpr int kTcSB = 1024;   // sources per block (the plan with 4 sources per thread)
constexpr int kTcS = 2;        // sources per compute thread
constexpr int kTcCW = kTcSB / (32 * kTcS);  // 16 compute warps: two halves of 8 (4 matrices of 128 sources each)
constexpr int kHalfWarps = kTcCW / 2;
constexpr int kMmaWarp0 = kTcCW;            // warps 16, 17: TMEM owner / MMA issuer of half 0, MMA issuer of half 1
constexpr int kProducerWarp = kTcCW + 2;    // warp 18: bulk copies
constexpr int kTcThreads = (kTcCW + 3) * 32;
constexpr int kTcStages = 6;  // 6 x 19.5 KB: also keeps the CTA alone on its SM
constexpr int kFeatRows = 32;
constexpr int kFeatFloats = kFeatRows * kTile;  // per tile
constexpr int kQPlanes = 7;                     // -sqrt(c) y (3), lambda, a (3): record planes 0-6
constexpr int kQBytes = kQPlanes * kTile * 4;
constexpr int kStageBytes = kFeatFloats * 4 + kQBytes;
constexpr int kChunk = 32;  // targets per A buffer (one buffer per matrix)
constexpr int kChunks = kTile / kChunk;
constexpr uint32_t kDCol = 0;
constexpr uint32_t kACol = 256;
constexpr size_t kTcSmem = static_cast<size_t>(kTcStages) * kStageBytes + (2 * kTcStages + 10) * 8 + 16;

static_assert(kStageBytes % 128 == 0, "stages stay 128-byte aligned");

// Feature rows (B operand, one row per feature, K = target):
//   0 one | 1-3 b hi | 4-9 a a^T hi | 10-12 b lo | 13-18 a a^T lo | 19 lambda hi | 20 lambda lo | 21-31 zero
// Layout of a tile: core matrix (g, kc) = rows 8g..8g+7 x targets 4kc..4kc+3 at
// floats (32 g + kc) * 32, row r at +4 r, target at +k % 4.
__host__ __device__ constexpr int feat_index(int f, int k) { return ((f / 8) * 32 + k / 4) * 32 + (f % 8) * 4 + k % 4; }

// tcgen05.mma kind::tf32 instruction descriptor: F32 accumulator (bits 4-5 = 1), A and B TF32
// (bits 7-9 and 10-12 = 2), both K-major, N = 32 (bits 17-22 = N / 8), M = 128 (bits 24-28 = M / 16)
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

// Shared-memory descriptor of 8 targets x 32 features starting at byte address `a` (canonical K-major
// layout without swizzle: leading byte offset 128 B between cores adjacent in K, stride byte offset
// 32 x 128 B between 8-row groups, descriptor version 1 at bit 46).
__device__ __forceinline__ uint64_t feat_desc(uint32_t a) {
  return static_cast<uint64_t>((a >> 4) & 0x3FFFu) | (static_cast<uint64_t>(128u >> 4) << 16) |
         (static_cast<uint64_t>(4096u >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ float tf32_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }



// Bounded wait that also gives up once another role of the CTA has aborted.  The
// producer and MMA threads (`idle_role`) pass a suspend-time hint to try_wait, so that
// while they wait they take fewer issue slots from the compute warps of their
// schedulers; the compute warps poll without one.
constexpr uint32_t kSuspendHintNs = 20000;

__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, const volatile int* abort_flag,
                                        bool idle_role = false) {
  const uint32_t a = smem_addr(bar);
  long long t0 = -1;
  while (true) {
    uint32_t ok;
    if (idle_role) {
      asm volatile(
          "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
          : "=r"(ok)
          : "r"(a), "r"(parity), "r"(kSuspendHintNs)
          : "memory");
    } else {
      asm volatile(
          "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
          : "=r"(ok)
          : "r"(a), "r"(parity)
          : "memory");
    }
    if (ok) return true;
    if (*abort_flag) return false;
    const long long now = clock64();
    if (t0 < 0) t0 = now;
    if (now - t0 > kWaitBudgetCycles) return false;
  }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p; }" ::"r"(d),
      "r"(a), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

// 16 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tc_st16(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]), "f"(v[9]),
      "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15])
      : "memory");
}

__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&d)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3]), "=f"(d[4]), "=f"(d[5]), "=f"(d[6]), "=f"(d[7]), "=f"(d[8]),
        "=f"(d[9]), "=f"(d[10]), "=f"(d[11]), "=f"(d[12]), "=f"(d[13]), "=f"(d[14]), "=f"(d[15]), "=f"(d[16]),
        "=f"(d[17]), "=f"(d[18]), "=f"(d[19]), "=f"(d[20]), "=f"(d[21]), "=f"(d[22]), "=f"(d[23]), "=f"(d[24]),
        "=f"(d[25]), "=f"(d[26]), "=f"(d[27]), "=f"(d[28]), "=f"(d[29]), "=f"(d[30]), "=f"(d[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}


// MODE: 0 uniform shift, 1 per-source shift L_n (El accumulated through the lambda feature).
template <int MODE>
__global__ void __launch_bounds__(kTcThreads, 1)
    estep_tc_kernel(const float4* __restrict__ xs, const float* __restrict__ rec, const float* __restrict__ feat,
                    const EmState* __restrict__ st, const float* __restrict__ ls_n, float* __restrict__ part,
                    const int* __restrict__ tab, const int* __restrict__ done_count, int* __restrict__ status,
                    Geo g) {
  constexpr int SB = kTcSB;
  constexpr int S = kTcS;
  constexpr int H = kTile / 2;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + kTcStages * kStageBytes);
  uint64_t* empty = full + kTcStages;
  uint64_t* a_full = empty + kTcStages;  // [half]
  uint64_t* a_empty = a_full + 2;        // [half]
  uint64_t* d_full = a_empty + 2;        // [half]
  uint64_t* d_empty = d_full + 2;        // [half]
  uint64_t* drain = d_empty + 2;         // [half]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

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

  if (tid == 0) {
    for (int i = 0; i < kTcStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kTcCW + 2);  // every compute warp and both MMA threads release a stage
    }
    for (int h = 0; h < 2; ++h) {
      mbar_init(&a_full[h], kHalfWarps);
      mbar_init(&a_empty[h], 1);
      mbar_init(&d_full[h], 1);
      mbar_init(&d_empty[h], kHalfWarps);
      mbar_init(&drain[h], 1);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == kMmaWarp0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_addr(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == kProducerWarp) {
    // ---------------- producer ----------------
    if (lane == 0) {
      Cursor cur{first_block};
      int issued = 0;
      for (int i = 0; i < n_units; ++i) {
        const int stage = i % kTcStages;
        if (i >= kTcStages &&
            !tc_wait(&empty[stage], static_cast<uint32_t>(i / kTcStages - 1) & 1u, abort_flag, true)) {
          atomicOr(status, kStatusTimeout);
          *abort_flag = 1;
          break;
        }
        const long long u = u0 + i;
        const int b = cur.advance(unit_off, u);
        const long long tile = static_cast<long long>(tile_off[block_pair[b]]) + (u - unit_off[b]);
        unsigned char* dst = smem_raw + stage * kStageBytes;
        arrive_expect_tx(&full[stage], kStageBytes);
        bulk_copy(dst, feat + tile * kFeatFloats, kFeatFloats * 4, &full[stage]);
        bulk_copy(dst + kFeatFloats * 4, rec + tile * kTileFloats, kQBytes, &full[stage]);
        ++issued;
      }
      // copies in flight land before the CTA's shared memory is released
      for (int j = issued > kTcStages ? issued - kTcStages : 0; j < issued; ++j)
        mbar_wait(&full[j % kTcStages], static_cast<uint32_t>(j / kTcStages) & 1u);
    }
    __syncwarp();
  } else if (warp >= kMmaWarp0) {
    // ---------------- MMA issuer of one half ----------------
    const int h = warp - kMmaWarp0;
    if (lane == 0) {
      Cursor cur{first_block};
      long long u = u0;
      int i = 0, cc = 0, seg = 0;
      bool ok = true;
      while (ok && u < u1) {
        const int b = cur.advance(unit_off, u);
        const bool live = !st[block_pair[b]].done;
        long long seg_end = u + g.seg_cap;
        if (seg_end > unit_off[b + 1]) seg_end = unit_off[b + 1];
        if (seg_end > u1) seg_end = u1;
        // the compute warps of this half have read the previous segment's accumulators
        if (seg > 0 && !tc_wait(&d_empty[h], static_cast<uint32_t>(seg - 1) & 1u, abort_flag, true)) {
          ok = false;
          break;
        }
        tc_fence_after();
        bool first = true;
        for (; u < seg_end; ++u, ++i) {
          const int stage = i % kTcStages;
          if (!tc_wait(&full[stage], static_cast<uint32_t>(i / kTcStages) & 1u, abort_flag, true)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_addr(smem_raw + stage * kStageBytes);
          for (int c = 0; c < kChunks; ++c, ++cc) {
            if (!tc_wait(&a_full[h], static_cast<uint32_t>(cc) & 1u, abort_flag, true)) {
              ok = false;
              break;
            }
            tc_fence_after();
            if (live) {
#pragma unroll
              for (int j = 0; j < kChunk / 8; ++j) {
                const uint64_t bd = feat_desc(fb + static_cast<uint32_t>(kChunk / 4 * c + 2 * j) * 128u);
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                  const uint32_t mi = 4u * h + m;
                  tc_mma(tmem + kDCol + 32u * mi, tmem + kACol + 32u * mi + 8u * j, bd, (first && j == 0) ? 0u : 1u);
                }
              }
              first = false;
            }
            tc_commit(&a_empty[h]);
          }
          if (!ok) break;
          tc_commit(&empty[stage]);
        }
        if (!ok) break;
        tc_commit(&d_full[h]);
        ++seg;
      }
      if (!ok) {
        atomicOr(status, kStatusTimeout);
        *abort_flag = 1;
      }
      // every MMA of this thread has completed before TMEM is released
      tc_commit(&drain[h]);
      mbar_wait(&drain[h], 0);
    }
    __syncwarp();
  } else {
    // ---------------- compute warps ----------------
    // Half h = warp / 8 (matrices 4h .. 4h+3).  A chunk of 32 targets is computed and
    // stored 16 at a time (two tensor-memory stores per source); the wait for the MMAs
    // that read the buffer before comes after the first 16 are computed.
    const int h = warp / kHalfWarps;
    const uint32_t lane_base = static_cast<uint32_t>((warp & 3) * 32) << 16;
    const uint32_t mi0 = static_cast<uint32_t>(S * (warp >> 2));
    Cursor cur{first_block};
    long long u = u0;
    int i = 0, cc = 0, seg = 0;
    bool ok = true;
    while (ok && u < u1) {
      const int b = cur.advance(unit_off, u);
      const EmState* sp = st + block_pair[b];
      const bool live = !sp->done;
      long long seg_end = u + g.seg_cap;
      if (seg_end > unit_off[b + 1]) seg_end = unit_off[b + 1];
      if (seg_end > u1) seg_end = u1;
      const float sqc = sp->sqc;
      float Rm[9], tv[3];
#pragma unroll
      for (int q = 0; q < 9; ++q) Rm[q] = sp->Rf[q];
#pragma unroll
      for (int q = 0; q < 3; ++q) tv[q] = sp->tf[q];
      float2 z0[S], z1[S], z2[S], ls[S], dq[S];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const long long n = static_cast<long long>(b) * SB + warp * 32 * S + s * 32 + lane;
        const float4 x = xs[n];
        // z = R x + t in FP32 (centred frame of the pair), scaled by sqrt(c)
        const float a0 = fmaf(Rm[0], x.x, fmaf(Rm[1], x.y, fmaf(Rm[2], x.z, tv[0])));
        const float a1 = fmaf(Rm[3], x.x, fmaf(Rm[4], x.y, fmaf(Rm[5], x.z, tv[1])));
        const float a2 = fmaf(Rm[6], x.x, fmaf(Rm[7], x.y, fmaf(Rm[8], x.z, tv[2])));
        z0[s] = dup(sqc * a0);
        z1[s] = dup(sqc * a1);
        z2[s] = dup(sqc * a2);
        ls[s] = dup(MODE ? ls_n[n] : 0.f);
        dq[s] = make_float2(0.f, 0.f);
      }
      for (; u < seg_end; ++u, ++i) {
        const int stage = i % kTcStages;
        if (!__all_sync(0xffffffffu, tc_wait(&full[stage], static_cast<uint32_t>(i / kTcStages) & 1u, abort_flag))) {
          ok = false;
          break;
        }
        const float2* T2 = reinterpret_cast<const float2*>(smem_raw + stage * kStageBytes + kFeatFloats * 4);
        for (int c = 0; c < kChunks; ++c, ++cc) {
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            float ev[S][16];
            if (live) {
#pragma unroll
              for (int p = 0; p < 8; ++p) {
                const int q = c * (kChunk / 2) + half * 8 + p;
                const float2 ny0 = T2[0 * H + q], ny1 = T2[1 * H + q], ny2 = T2[2 * H + q];
                const float2 lam = T2[3 * H + q];
                const float2 ta0 = T2[4 * H + q], ta1 = T2[5 * H + q], ta2 = T2[6 * H + q];
#pragma unroll
                for (int s = 0; s < S; ++s) {
                  const float2 r0 = __fadd2_rn(z0[s], ny0);
                  const float2 r1 = __fadd2_rn(z1[s], ny1);
                  const float2 r2 = __fadd2_rn(z2[s], ny2);
                  float2 v = __fmul2_rn(ta0, r0);  // v = a . r^
                  v = __ffma2_rn(ta1, r1, v);
                  v = __ffma2_rn(ta2, r2, v);
                  float2 qq = MODE ? __fadd2_rn(lam, ls[s]) : lam;  // q = c d + lambda_m (+ L_n)
                  qq = __ffma2_rn(r0, r0, qq);
                  qq = __ffma2_rn(r1, r1, qq);
                  qq = __ffma2_rn(r2, r2, qq);
                  qq = __ffma2_rn(v, v, qq);
                  float2 e;
                  e.x = tf32_trunc(ex2_neg(qq.x));
                  e.y = tf32_trunc(ex2_neg(qq.y));
                  dq[s] = __ffma2_rn(e, qq, dq[s]);
                  ev[s][2 * p] = e.x;
                  ev[s][2 * p + 1] = e.y;
                }
              }
            }
            if (half == 0 && cc > 0) {
              // the buffer is free once the MMAs of the previous chunk have completed (also
              // waited for when nothing is stored, so that the arrivals on a_full stay one
              // phase ahead of the MMA thread at most)
              if (!__all_sync(0xffffffffu,
                              tc_wait(&a_empty[h], static_cast<uint32_t>(cc - 1) & 1u, abort_flag))) {
                ok = false;
                break;
              }
            }
            if (live) {
              if (half == 0) tc_fence_after();
#pragma unroll
              for (int s = 0; s < S; ++s)
                tc_st16(tmem + lane_base + kACol + 32u * (mi0 + s) + 16u * half, ev[s]);
            }
          }
          if (!ok) break;
          if (live) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&a_full[h]);
        }
        if (!ok) break;
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[stage]);  // the record planes of this tile are no longer read
      }
      if (!ok) break;
      // segment end: the accumulators of this thread's sources
      if (!__all_sync(0xffffffffu, tc_wait(&d_full[h], static_cast<uint32_t>(seg) & 1u, abort_flag))) {
        ok = false;
        break;
      }
      tc_fence_after();
      if (live) {
        float* dst = part + static_cast<size_t>(first_slot + seg) * kMom * SB;
#pragma unroll
        for (int s = 0; s < S; ++s) {
          float d[32];
          tc_ld32(tmem + lane_base + kDCol + 32u * (mi0 + s), d);
          const int nl = warp * 32 * S + s * 32 + lane;
          dst[0 * SB + nl] = d[0];
#pragma unroll
          for (int k = 0; k < 3; ++k) dst[(1 + k) * SB + nl] = d[1 + k] + d[10 + k];
#pragma unroll
          for (int k = 0; k < 6; ++k) dst[(4 + k) * SB + nl] = d[4 + k] + d[13 + k];
          dst[10 * SB + nl] = dq[s].x + dq[s].y;
          if (MODE) dst[11 * SB + nl] = d[19] + d[20];
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&d_empty[h]);
      ++seg;
    }
    if (!ok) {
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");  // no store of this thread in flight
      if (lane == 0) {
        atomicOr(status, kStatusTimeout);
        *abort_flag = 1;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// Feature tile of every record slot (one thread per slot): rows as listed above,
// hi = the value truncated to TF32, lo = the remainder truncated to TF32; zero
// for padding.  lambda is -l_m (the per-source-shift plane of the record).
__global__ void __launch_bounds__(kTile) feature_kernel(const float* __restrict__ rec, const float4* __restrict__ yl,
                                                        float* __restrict__ feat) {
  const int tile = blockIdx.x;
  const int k = threadIdx.x;
  const float* r = rec + static_cast<size_t>(tile) * kTileFloats + k;
  const float4 y = yl[static_cast<size_t>(tile) * kTile + k];
  const bool pad = y.w == -INFINITY;
  float v[21];
  v[0] = 1.f;
#pragma unroll
  for (int j = 0; j < 3; ++j) v[1 + j] = r[(13 + j) * kTile];  // b = Lambda y
#pragma unroll
  for (int j = 0; j < 6; ++j) v[4 + j] = r[(7 + j) * kTile];  // a a^T
  v[19] = -y.w;
  float* o = feat + static_cast<size_t>(tile) * kFeatFloats;
#pragma unroll
  for (int f = 0; f < kFeatRows; ++f) {
    float x = 0.f;
    if (!pad) {
      if (f == 0) {
        x = 1.f;
      } else if (f < 10) {
        x = tf32_trunc(v[f]);
      } else if (f < 19) {
        const float w = v[f - 9];
        x = tf32_trunc(w - tf32_trunc(w));
      } else if (f == 19) {
        x = tf32_trunc(v[19]);
      } else if (f == 20) {
        x = tf32_trunc(v[19] - tf32_trunc(v[19]));
      }
    }
    o[feat_index(f, k)] = x;
  }
}

}  // namespace

size_t tc_feature_floats(const Geo& g) { return static_cast<size_t>(g.T) * kFeatFloats; }

cudaError_t launch_features(const BatchPlan& p, const float* rec, const float4* yl, float* feat, cudaStream_t s) {
  feature_kernel<<<p.g.T, kTile, 0, s>>>(rec, yl, feat);
  return cudaGetLastError();
}

namespace {
template <int MODE>
cudaError_t launch_tc_t(const BatchPlan& p, const Dev& d, const float4* xs, const float* rec, const float* feat,
                        const float* ls_n, float* part, int* status, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(estep_tc_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(kTcSmem));
  if (e != cudaSuccess) return e;
  return launch_k(estep_tc_kernel<MODE>, dim3(p.g.grid), dim3(kTcThreads), kTcSmem, s, xs, rec, feat, d.st, ls_n, part,
                  d.tab, d.done_count, status, p.g);
}
}  // namespace

cudaError_t launch_estep_tc(const BatchPlan& p, const Dev& d, const float4* xs, const float* rec, const float* feat,
                            int mode, const float* ls_n, float* part, int* status, cudaStream_t s) {
  if (p.g.SB != kTcSB) return cudaErrorInvalidValue;
  if (mode) return launch_tc_t<1>(p, d, xs, rec, feat, ls_n, part, status, s);
  return launch_tc_t<0>(p, d, xs, rec, feat, nullptr, part, status, s);
}

}  // namespace lsg
