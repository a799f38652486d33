// Exact k-nearest-neighbour search through a uniform grid (Sec. 3.1: the
// neighbourhood of every target for its normal and surface variation).
//
// The result is the brute-force result of launch_knn, bit for bit: the same
// FP32 squared distances (fma(dz, dz, fma(dy, dy, dx * dx))) and the same
// (distance, index) order.  Only the candidates change: the targets of each
// pair are bucketed into a uniform grid (counting sort), and every query
// visits cubic shells of cells around its own cell until the k-th distance is
// below the squared distance from the query to the boundary of the visited
// cube (with a relative margin of 1e-5, far above FP32 rounding of a squared
// distance), so no unvisited point can enter or tie the list.
//
// Cells of pair i live at [4 m_off[i] + 64 i, 4 m_off[i+1] + 64 (i+1)) of the
// cell arrays (at most 4 M_i + 64 cells per pair), so the host sizes them from
// the offsets alone.  Per pair the cell edge starts at diag sqrt(k / M) (about
// k points per occupied cell on a surface) and grows until the grid fits.
#include <math.h>

#include "internal.cuh"

namespace lsg {
namespace {

constexpr int kGridThreads = 256;
constexpr int kQueryThreads = 128;
constexpr int kScanElems = 1024;  // per scan block (4 per thread)

__device__ __forceinline__ long long cell_base(const long long* off64, int P, int pair) {
  return 4 * off64[P + 1 + pair] + 64LL * pair;
}

// Grid of every pair: origin, cell edge, dims (doubles), from the target AABB.
__global__ void grid_setup_kernel(const long long* __restrict__ off64, int P, int k,
                                  const EmState* __restrict__ st_all, double* __restrict__ info) {
  const int pair = blockIdx.x;
  if (threadIdx.x != 0) return;
  const EmState* st = st_all + pair;
  const long long M = off64[P + 1 + pair + 1] - off64[P + 1 + pair];
  const double cap = 4.0 * static_cast<double>(M) + 64.0;
  double ext[3], dims[3];
  for (int a = 0; a < 3; ++a) ext[a] = st->yhi[a] - st->ylo[a];
  double h = st->diag * sqrt(static_cast<double>(k) / static_cast<double>(M));
  if (!(h > 0.0)) h = 1.0;
  for (int it = 0; it < 200; ++it) {
    double prod = 1.0;
    bool ok = true;
    for (int a = 0; a < 3; ++a) {
      dims[a] = floor(ext[a] / h) + 1.0;
      prod *= dims[a];
      ok = ok && dims[a] <= 1024.0;
    }
    if (ok && prod <= cap) break;
    h *= fmax(1.05, 1.01 * cbrt(prod / cap));
  }
  if (dims[0] * dims[1] * dims[2] > cap || dims[0] > 1024.0 || dims[1] > 1024.0 || dims[2] > 1024.0) {
    h = 2.0 * fmax(fmax(ext[0], ext[1]), fmax(ext[2], 1.0));  // one cell: always within the bound
    dims[0] = dims[1] = dims[2] = 1.0;
  }
  double* o = info + 8 * pair;
  for (int a = 0; a < 3; ++a) {
    o[a] = st->ylo[a];
    o[4 + a] = dims[a];
  }
  o[3] = h;
  o[7] = cap;
}

__device__ __forceinline__ int cell_coord(double v, double lo, double h, int dim) {
  int c = static_cast<int>(floor((v - lo) / h));
  return c < 0 ? 0 : (c >= dim ? dim - 1 : c);
}

// Cell of every target and the per-cell counts.  grid = (target blocks of the largest pair, P).
__global__ void __launch_bounds__(kGridThreads)
    cell_count_kernel(const float* __restrict__ Y, const long long* __restrict__ off64, int P,
                      const double* __restrict__ info, int* __restrict__ count, int* __restrict__ cell_of) {
  const int pair = blockIdx.y;
  const long long m0 = off64[P + 1 + pair], M = off64[P + 1 + pair + 1] - m0;
  const long long m = static_cast<long long>(blockIdx.x) * kGridThreads + threadIdx.x;
  if (m >= M) return;
  const double* g = info + 8 * pair;
  const int dx = static_cast<int>(g[4]), dy = static_cast<int>(g[5]), dz = static_cast<int>(g[6]);
  const float* y = Y + 3 * (m0 + m);
  const int cx = cell_coord(y[0], g[0], g[3], dx);
  const int cy = cell_coord(y[1], g[1], g[3], dy);
  const int cz = cell_coord(y[2], g[2], g[3], dz);
  const int cid = (cz * dy + cy) * dx + cx;
  cell_of[m0 + m] = cid;
  atomicAdd(count + cell_base(off64, P, pair) + cid, 1);
}

// Exclusive prefix sum of the counts (three passes: blocks, block sums, add).
__global__ void __launch_bounds__(kGridThreads)
    scan_blocks_kernel(const int* __restrict__ in, long long n, int* __restrict__ out, int* __restrict__ sums) {
  __shared__ int sh[kGridThreads];
  const long long base = static_cast<long long>(blockIdx.x) * kScanElems + 4 * threadIdx.x;
  int v[4], t = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    v[j] = base + j < n ? in[base + j] : 0;
    t += v[j];
  }
  sh[threadIdx.x] = t;
  __syncthreads();
  for (int o = 1; o < kGridThreads; o <<= 1) {  // inclusive Hillis-Steele scan of the thread totals
    const int x = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += x;
    __syncthreads();
  }
  int run = sh[threadIdx.x] - t;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (base + j < n) out[base + j] = run;
    run += v[j];
  }
  if (threadIdx.x == kGridThreads - 1) sums[blockIdx.x] = sh[threadIdx.x];
}

// One CTA: exclusive scan of the block sums in place (sequential over chunks of the CTA width).
__global__ void __launch_bounds__(kGridThreads) scan_sums_kernel(int* __restrict__ sums, int nb) {
  __shared__ int sh[kGridThreads];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nb; b0 += kGridThreads) {
    const int i = b0 + threadIdx.x;
    const int v = i < nb ? sums[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kGridThreads; o <<= 1) {
      const int x = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += x;
      __syncthreads();
    }
    if (i < nb) sums[i] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == kGridThreads - 1) carry += sh[threadIdx.x];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kGridThreads)
    scan_add_kernel(int* __restrict__ out, long long n, const int* __restrict__ sums, int total) {
  const long long i = static_cast<long long>(blockIdx.x) * kGridThreads + threadIdx.x;
  if (i < n) out[i] += sums[i / kScanElems];
  if (i == n) out[n] = total;
}

// Targets sorted by cell (order inside a cell does not matter: ties are broken by index).
__global__ void __launch_bounds__(kGridThreads)
    cell_fill_kernel(const float* __restrict__ Y, const long long* __restrict__ off64, int P,
                     const int* __restrict__ cell_of, const int* __restrict__ start, int* __restrict__ fill,
                     float4* __restrict__ sorted) {
  const int pair = blockIdx.y;
  const long long m0 = off64[P + 1 + pair], M = off64[P + 1 + pair + 1] - m0;
  const long long m = static_cast<long long>(blockIdx.x) * kGridThreads + threadIdx.x;
  if (m >= M) return;
  const long long c = cell_base(off64, P, pair) + cell_of[m0 + m];
  const int pos = start[c] + atomicAdd(fill + c, 1);
  const float* y = Y + 3 * (m0 + m);
  sorted[pos] = make_float4(y[0], y[1], y[2], __int_as_float(static_cast<int>(m)));
}

// (d, i) < (d', i')
__device__ __forceinline__ bool before(float d, int i, float d2, int i2) { return d < d2 || (d == d2 && i < i2); }

template <int KMAX>
__device__ __forceinline__ void insert_sorted(float (&bd)[KMAX], int (&bi)[KMAX], int k, float d, int ci) {
#pragma unroll
  for (int s = KMAX - 1; s >= 0; --s) {
    if (s < k) {
      if (s > 0 && before(d, ci, bd[s - 1], bi[s - 1])) {
        bd[s] = bd[s - 1];
        bi[s] = bi[s - 1];
      } else if (before(d, ci, bd[s], bi[s])) {
        bd[s] = d;
        bi[s] = ci;
      }
    }
  }
}

// One query per thread.  grid = (query blocks of the largest pair, P).
template <int KMAX, int KFIX>
__global__ void __launch_bounds__(kQueryThreads)
    grid_knn_kernel(const float* __restrict__ Y, const long long* __restrict__ off64, int P, int k_rt,
                    const double* __restrict__ info, const int* __restrict__ count, const int* __restrict__ start,
                    const float4* __restrict__ sorted, int* __restrict__ idx_out) {
  const int k = KFIX > 0 ? KFIX : k_rt;
  const int pair = blockIdx.y;
  const long long m0 = off64[P + 1 + pair], M = off64[P + 1 + pair + 1] - m0;
  const long long q = static_cast<long long>(blockIdx.x) * kQueryThreads + threadIdx.x;
  if (q >= M) return;
  const double* g = info + 8 * pair;
  const double lo[3] = {g[0], g[1], g[2]};
  const double h = g[3];
  const int dim[3] = {static_cast<int>(g[4]), static_cast<int>(g[5]), static_cast<int>(g[6])};
  const long long cb = cell_base(off64, P, pair);
  const float qx = Y[3 * (m0 + q)], qy = Y[3 * (m0 + q) + 1], qz = Y[3 * (m0 + q) + 2];
  const double qv[3] = {qx, qy, qz};
  int c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) c[a] = cell_coord(qv[a], lo[a], h, dim[a]);
  float bd[KMAX];
  int bi[KMAX];
#pragma unroll
  for (int j = 0; j < KMAX; ++j) {
    bd[j] = INFINITY;
    bi[j] = 0x7fffffff;
  }
  int found = 0;
  float kd = INFINITY;  // the k-th entry of the list
  int ki = 0x7fffffff;
  for (int r = 0;; ++r) {
    for (int z = c[2] - r; z <= c[2] + r; ++z) {
      if (z < 0 || z >= dim[2]) continue;
      for (int y = c[1] - r; y <= c[1] + r; ++y) {
        if (y < 0 || y >= dim[1]) continue;
        const bool face = z == c[2] - r || z == c[2] + r || y == c[1] - r || y == c[1] + r;
        const int step = (face || r == 0) ? 1 : 2 * r;  // interior rows of the shell: only x = c -+ r
        for (int x = c[0] - r; x <= c[0] + r; x += step) {
          if (x < 0 || x >= dim[0]) continue;
          const long long cc = cb + (static_cast<long long>(z) * dim[1] + y) * dim[0] + x;
          const int j0 = start[cc], j1 = j0 + count[cc];
          for (int j = j0; j < j1; ++j) {
            const float4 p = sorted[j];
            const float dx = qx - p.x, dy = qy - p.y, dz = qz - p.z;
            const float d = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const int ci = __float_as_int(p.w);
            if (before(d, ci, kd, ki)) {
              insert_sorted<KMAX>(bd, bi, k, d, ci);
              ++found;
#pragma unroll
              for (int t = 0; t < KMAX; ++t)
                if (t == k - 1) {
                  kd = bd[t];
                  ki = bi[t];
                }
            }
          }
        }
      }
    }
    bool all = true;
    double bound = 1e300;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (c[a] - r > 0) {
        all = false;
        bound = fmin(bound, qv[a] - (lo[a] + (c[a] - r) * h));
      }
      if (c[a] + r < dim[a] - 1) {
        all = false;
        bound = fmin(bound, (lo[a] + (c[a] + r + 1) * h) - qv[a]);
      }
    }
    if (all) break;
    if (found >= k && bound > 0.0 && static_cast<double>(kd) < bound * bound * (1.0 - 1e-5)) break;
  }
  int* out = idx_out + (m0 + q) * k;
#pragma unroll
  for (int j = 0; j < KMAX; ++j)
    if (j < k) out[j] = bi[j];
}

}  // namespace

long long knn_grid_cells(long long Mtot, int P) { return 4 * Mtot + 64LL * P; }

size_t knn_grid_scan_blocks(long long cells) { return static_cast<size_t>((cells + kScanElems - 1) / kScanElems); }

cudaError_t launch_knn_grid(const BatchPlan& p, const Dev& d, const float* Y, int k, const GridBufs& gb,
                            int* idx_out, cudaStream_t s) {
  const Geo& g = p.g;
  const int P = g.P;
  const long long Mtot = p.off64[2 * P + 1];
  const long long cells = knn_grid_cells(Mtot, P);
  cudaError_t e = cudaMemsetAsync(gb.count, 0, sizeof(int) * cells, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(gb.fill, 0, sizeof(int) * cells, s);
  if (e != cudaSuccess) return e;
  grid_setup_kernel<<<P, 32, 0, s>>>(d.off64, P, k, d.st, gb.info);
  dim3 tgrid(static_cast<unsigned>((g.max_m + kGridThreads - 1) / kGridThreads), static_cast<unsigned>(P));
  cell_count_kernel<<<tgrid, kGridThreads, 0, s>>>(Y, d.off64, P, gb.info, gb.count, gb.cell_of);
  const int nb = static_cast<int>(knn_grid_scan_blocks(cells));
  scan_blocks_kernel<<<nb, kGridThreads, 0, s>>>(gb.count, cells, gb.start, gb.scan_tmp);
  scan_sums_kernel<<<1, kGridThreads, 0, s>>>(gb.scan_tmp, nb);
  scan_add_kernel<<<static_cast<unsigned>((cells + 1 + kGridThreads - 1) / kGridThreads), kGridThreads, 0, s>>>(
      gb.start, cells, gb.scan_tmp, static_cast<int>(Mtot));
  cell_fill_kernel<<<tgrid, kGridThreads, 0, s>>>(Y, d.off64, P, gb.cell_of, gb.start, gb.fill, gb.sorted);
  dim3 qgrid(static_cast<unsigned>((g.max_m + kQueryThreads - 1) / kQueryThreads), static_cast<unsigned>(P));
  switch (k) {
#define LSG_GKNN_CASE(K)                                                                                 \
  case K:                                                                                                \
    grid_knn_kernel<K, K><<<qgrid, kQueryThreads, 0, s>>>(Y, d.off64, P, k, gb.info, gb.count, gb.start, \
                                                          gb.sorted, idx_out);                           \
    break;
    LSG_GKNN_CASE(1) LSG_GKNN_CASE(2) LSG_GKNN_CASE(4) LSG_GKNN_CASE(8) LSG_GKNN_CASE(10) LSG_GKNN_CASE(16)
#undef LSG_GKNN_CASE
    default:
      grid_knn_kernel<32, 0><<<qgrid, kQueryThreads, 0, s>>>(Y, d.off64, P, k, gb.info, gb.count, gb.start,
                                                             gb.sorted, idx_out);
  }
  return cudaGetLastError();
}

}  // namespace lsg
