// C ABI of liblsgcpd (declared in include/lsgcpd.h): context, argument
// validation, scratch memory, the batch plan, the CUDA-graph-captured EM loop
// and the conversions between the centred working frame and the caller's frame.
// A single registration is a batch of one pair.
#include <math.h>
#include <nvtx3/nvToolsExt.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <vector>

#include "internal.cuh"
#include "lsgcpd.h"

using namespace lsg;

namespace {

constexpr int kMaxK = 32;
// problems up to this many pairs per E step (about 12 ms) are autotuned on first sight
constexpr double kTuneMaxPairs = 1.5e10;

template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t cap = 0;  // elements
};

// Identity of a captured EM graph: the sizes of every pair, the shift mode, the
// iteration count, what the graph records and the parameters its kernels take
// by value.
struct GraphKey {
  std::vector<long long> sizes;
  std::vector<unsigned char> params;
  int iters = -1, mode = -1, prec = -1, S = -1, timing = -1, trace = -1;
  bool operator==(const GraphKey& o) const {
    return sizes == o.sizes && params == o.params && iters == o.iters && mode == o.mode && prec == o.prec &&
           S == o.S && timing == o.timing && trace == o.trace;
  }
};

}  // namespace

struct lsgcpd_ctx {
  int device = 0;
  int num_sms = 0;
  std::string err;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  DevBuf<float> X_in, Y_in, rec, part, knn_d, ls_n, gam_n;
  DevBuf<float> feat;  // feature tiles of the tensor-core E step (precision 2)
  DevBuf<float> phx_in, phy_in, Xc, Yc, phxc, phyc;  // confidences; truncated clouds
  DevBuf<float> pern_tmp;                             // per-source output for the dense posteriors
  DevBuf<int> cnt, coff;
  DevBuf<int> g_count, g_start, g_fill, g_cellof, g_scan;  // grid kNN
  DevBuf<float4> g_sorted;
  DevBuf<double> g_info;
  DevBuf<long long> toff;
  DevBuf<float4> xs, y4, yl;
  DevBuf<int> knn_i, knn_idx, tab;
  DevBuf<long long> off64;
  DevBuf<double> rows, red, trace, io, mom;
  DevBuf<EmState> st;
  int* status = nullptr;
  int* done_count = nullptr;
  // graph of the EM loop
  cudaGraphExec_t gexec = nullptr;
  GraphKey gkey;
  // timing
  int timing = 0;
  cudaEvent_t t_begin = nullptr, t_prep = nullptr, t_end = nullptr;
  cudaEvent_t* t_iter = nullptr;  // 4 per iteration
  int t_iter_cap = 0;
  double last_timing[5] = {0, 0, 0, 0, 0};
  int64_t launches = 0;
  int64_t h2d_bytes = 0, d2h_bytes = 0;
  // autotuning of the E step's source tile (sources per thread), per problem shape
  int autotune = 1;
  struct Tuned {
    std::vector<long long> sizes;
    int S;
    double ms[3];  // measured ms per E-step launch for S = 4, 2, 1 (0: not measured)
  };
  std::vector<Tuned> tuned;
  cudaEvent_t tune_ev[2] = {nullptr, nullptr};
  int32_t last_plan[4] = {0, 0, 0, 0};  // S, SB, grid, chosen by measurement
  double last_tune_ms[3] = {0, 0, 0};
};

namespace {

// Message of the size limit of the plan tables (lsg::plan_fits).
constexpr const char* kTooLarge =
    "problem too large: more than 2^30 (source block x target tile) units (a single pair of N = M = 4,000,000 "
    "is within the limit)";

lsgcpd_status fail(lsgcpd_ctx* c, lsgcpd_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

lsgcpd_status cuda_fail(lsgcpd_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return fail(c, LSGCPD_ECUDA, m);
}

#define LSG_CUDA(call, where)                              \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
  } while (0)

template <class T>
cudaError_t ensure(DevBuf<T>& b, size_t n) {
  if (n == 0) n = 1;
  if (b.cap >= n) return cudaSuccess;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
  cudaError_t e = cudaMalloc(&b.p, n * sizeof(T));
  if (e == cudaSuccess) b.cap = n;
  return e;
}

bool is_finite_d(double v) { return isfinite(v) != 0; }

lsgcpd_status check_params(lsgcpd_ctx* c, const lsgcpd_params* p) {
  if (!p) return fail(c, LSGCPD_EINVAL, "params is NULL");
  if (!(p->w >= 0.0 && p->w < 1.0)) return fail(c, LSGCPD_EINVAL, "w must be in [0, 1)");
  if (!is_finite_d(p->alpha_max) || p->alpha_max < 0.0) return fail(c, LSGCPD_EINVAL, "alpha_max must be finite and >= 0");
  if (!is_finite_d(p->lambda) || p->lambda < 0.0) return fail(c, LSGCPD_EINVAL, "lambda must be finite and >= 0");
  if (!is_finite_d(p->tol) || p->tol < 0.0) return fail(c, LSGCPD_EINVAL, "tol must be finite and >= 0");
  if (!is_finite_d(p->volume) || !is_finite_d(p->sigma2_init))
    return fail(c, LSGCPD_EINVAL, "volume/sigma2_init must be finite");
  for (int i = 0; i < 9; ++i)
    if (!is_finite_d(p->init_R[i])) return fail(c, LSGCPD_EINVAL, "init_R must be finite");
  for (int i = 0; i < 3; ++i)
    if (!is_finite_d(p->init_t[i])) return fail(c, LSGCPD_EINVAL, "init_t must be finite");
  if (!is_finite_d(p->newton_tol) || p->newton_tol < 0.0) return fail(c, LSGCPD_EINVAL, "newton_tol must be >= 0");
  if (!is_finite_d(p->sigma2_floor_rel) || p->sigma2_floor_rel < 0.0)
    return fail(c, LSGCPD_EINVAL, "sigma2_floor_rel must be >= 0");
  if (p->max_iters < 0 || p->max_iters > 100000) return fail(c, LSGCPD_EINVAL, "max_iters out of range");
  if (p->newton_max < 1 || p->newton_max > 1000) return fail(c, LSGCPD_EINVAL, "newton_max out of range");
  if (p->precision < 0 || p->precision > 2)
    return fail(c, LSGCPD_EINVAL,
                "precision must be 0 (FP32), 1 (f16x2 exponentials) or 2 (tensor-core moments)");
  if (!(p->eta >= 0.0 && p->eta < 1.0)) return fail(c, LSGCPD_EINVAL, "eta must be in [0, 1)");
  if (!is_finite_d(p->cf_threshold) || p->cf_threshold < 0.0)
    return fail(c, LSGCPD_EINVAL, "cf_threshold must be finite and >= 0");
  if (!is_finite_d(p->nll_tol) || p->nll_tol < 0.0) return fail(c, LSGCPD_EINVAL, "nll_tol must be finite and >= 0");
  if (p->knn_method < 0 || p->knn_method > 2) return fail(c, LSGCPD_EINVAL, "knn_method must be 0, 1 or 2");
  return LSGCPD_OK;
}

DevParams dev_params(const lsgcpd_params* p) {
  DevParams d{};
  d.w = p->w;
  d.volume = p->volume;
  d.sigma2_init = p->sigma2_init;
  for (int i = 0; i < 9; ++i) d.init_R[i] = p->init_R[i];
  for (int i = 0; i < 3; ++i) d.init_t[i] = p->init_t[i];
  d.newton_tol = p->newton_tol;
  d.sigma2_floor_rel = p->sigma2_floor_rel;
  d.tol = p->tol;
  d.newton_max = p->newton_max;
  d.include_alpha_norm = p->include_alpha_norm;
  d.max_iters = p->max_iters;
  d.cf_x = p->phi_x ? 1 : 0;
  d.eta = p->eta;
  d.nll_tol = p->nll_tol;
  return d;
}

// Fixed-shift mode (L = log2 gamma for every source) is safe when no term can
// overflow FP32: l_max - L_min + log2(M) stays well below 127.
int choose_mode(double w, double sigma2_min, double V, int64_t M, double l_extra) {
  if (!(w > 0.0) || !(sigma2_min > 0.0) || !(V > 0.0)) return 1;
  const double L_min = log2(w) - log2(1.0 - w) + 1.5 * log2(2.0 * M_PI * sigma2_min) - log2(V);
  const double l_max = -log2(static_cast<double>(M)) + l_extra;
  const double x_max = l_max - L_min;
  return (x_max + log2(static_cast<double>(M)) + 12.0 < 126.0) ? 0 : 1;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

__global__ void check_finite_kernel(const float* p, long long n, int* status) {
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  bool bad = false;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
    bad |= !isfinite(p[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, 8);
}

// Confidences must lie in (0, 1] (NaN fails too): status bit 16.
__global__ void check_conf_kernel(const float* p, long long n, int* status) {
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  bool bad = false;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
    bad |= !(p[i] > 0.f && p[i] <= 1.f);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, 16);
}

cudaError_t check_conf(const float* p, long long n, int* status, cudaStream_t s) {
  long long b = (n + 255) / 256;
  if (b > 1024) b = 1024;
  if (b < 1) b = 1;
  check_conf_kernel<<<static_cast<unsigned>(b), 256, 0, s>>>(p, n, status);
  return cudaGetLastError();
}

cudaError_t check_finite(const float* p, long long n, int* status, cudaStream_t s) {
  long long b = (n + 255) / 256;
  if (b > 1024) b = 1024;
  if (b < 1) b = 1;
  check_finite_kernel<<<static_cast<unsigned>(b), 256, 0, s>>>(p, n, status);
  return cudaGetLastError();
}

// Make the context's stream wait for the caller's stream (inputs ready).
cudaError_t enter(lsgcpd_ctx* c, void* stream) {
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(c->ev_in, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return e;
  return cudaStreamWaitEvent(c->stream, c->ev_in, 0);
}

// Make the caller's stream wait for the context's stream (outputs ready).
cudaError_t leave(lsgcpd_ctx* c, void* stream) {
  cudaError_t e = cudaEventRecord(c->ev_out, c->stream);
  if (e != cudaSuccess) return e;
  return cudaStreamWaitEvent(static_cast<cudaStream_t>(stream), c->ev_out, 0);
}

// Scratch for a plan; k = 0 skips the neighbour buffers.  A buffer that has to
// grow moves, so the captured graph (which holds the old addresses) is dropped.
lsgcpd_status reserve(lsgcpd_ctx* c, const BatchPlan& p, int k, int iters, bool host_inputs, bool tc = false) {
  const Geo& g = p.g;
  const size_t n_pad = static_cast<size_t>(g.B) * g.SB;
  const size_t m_pad = static_cast<size_t>(g.T) * kTile;
  const long long Ntot = p.off64[g.P], Mtot = p.off64[2 * g.P + 1];
  const int chunks = stats_chunks(g);
  bool grew = false, ok = true;
  auto grow = [&](auto& buf, size_t n) {
    if (!ok || buf.cap >= (n ? n : 1)) return;
    grew = true;
    ok = ensure(buf, n) == cudaSuccess;
  };
  grow(c->xs, n_pad);
  grow(c->rec, m_pad * kPlanes);
  if (tc) grow(c->feat, tc_feature_floats(g));
  grow(c->yl, m_pad);
  grow(c->part, estep_partial_floats(g));
  grow(c->rows, static_cast<size_t>(g.combine_ctas) * kGlob);
  grow(c->ls_n, n_pad);
  grow(c->gam_n, n_pad);
  grow(c->tab, p.tab.size());
  grow(c->off64, p.off64.size());
  grow(c->st, static_cast<size_t>(g.P));
  grow(c->mom, static_cast<size_t>(g.P) * kGlob);
  grow(c->red, static_cast<size_t>(g.P) * chunks * 24);
  grow(c->trace, static_cast<size_t>(g.P) * (iters > 0 ? iters : 1) * LSGCPD_TRACE_WIDTH);
  if (k > 0) {
    const int splits = knn_splits(g, c->num_sms);
    grow(c->y4, static_cast<size_t>(Mtot));
    grow(c->knn_d, static_cast<size_t>(splits) * Mtot * k);
    grow(c->knn_i, static_cast<size_t>(splits) * Mtot * k);
    grow(c->knn_idx, static_cast<size_t>(Mtot) * k);
  }
  if (host_inputs) {
    grow(c->X_in, static_cast<size_t>(Ntot) * 3);
    grow(c->Y_in, static_cast<size_t>(Mtot) * 3);
  }
  if (grew && c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->gkey = GraphKey();
  }
  if (!ok) {
    cudaGetLastError();
    return fail(c, LSGCPD_ENOMEM, "device allocation failed");
  }
  return LSGCPD_OK;
}

Dev dev_of(lsgcpd_ctx* c) { return Dev{c->tab.p, c->off64.p, c->st.p, c->done_count}; }

// One E-step launch for the precision: 0 FP32, 1 f16x2 exponentials, 2 moments on the tensor cores.
cudaError_t estep_launch(lsgcpd_ctx* c, const BatchPlan& plan, const Dev& d, int mode, int prec, cudaStream_t s) {
  if (prec == 2)
    return launch_estep_tc(plan, d, c->xs.p, c->rec.p, c->feat.p, mode, c->ls_n.p, c->part.p, c->status, s);
  return launch_estep(plan, d, c->xs.p, c->rec.p, mode, prec == 1 ? 1 : 0, c->ls_n.p, c->part.p, c->status, s);
}

// k nearest targets of every target (needs the pair AABBs from launch_init for the grid).
cudaError_t run_knn(lsgcpd_ctx* c, const BatchPlan& plan, const Dev& d, const float* Y, int k, int method,
                    int* idx, int64_t* launches, cudaStream_t s) {
  const bool grid = method == 2 || (method == 0 && plan.g.max_m > 50000);
  if (!grid) {
    *launches += 2;
    return launch_knn(plan, d, Y, k, knn_splits(plan.g, c->num_sms), c->y4.p, c->knn_d.p, c->knn_i.p, idx, s);
  }
  const int P = plan.g.P;
  const long long Mtot = plan.off64[2 * P + 1];
  const long long cells = knn_grid_cells(Mtot, P);
  cudaError_t e = ensure(c->g_count, static_cast<size_t>(cells));
  if (e == cudaSuccess) e = ensure(c->g_fill, static_cast<size_t>(cells));
  if (e == cudaSuccess) e = ensure(c->g_start, static_cast<size_t>(cells) + 1);
  if (e == cudaSuccess) e = ensure(c->g_cellof, static_cast<size_t>(Mtot));
  if (e == cudaSuccess) e = ensure(c->g_sorted, static_cast<size_t>(Mtot));
  if (e == cudaSuccess) e = ensure(c->g_scan, knn_grid_scan_blocks(cells));
  if (e == cudaSuccess) e = ensure(c->g_info, 8 * static_cast<size_t>(P));
  if (e != cudaSuccess) return e;
  const GridBufs gb{c->g_count.p, c->g_start.p, c->g_fill.p, c->g_cellof.p, c->g_sorted.p, c->g_scan.p, c->g_info.p};
  *launches += 7;
  return launch_knn_grid(plan, d, Y, k, gb, idx, s);
}

// The plan's tables and the finished-pair count (zero) for this call.  The
// status word is cleared separately, before the input checks that set it.
cudaError_t upload_plan(lsgcpd_ctx* c, const BatchPlan& p, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(c->tab.p, p.tab.data(), sizeof(int) * p.tab.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->off64.p, p.off64.data(), sizeof(long long) * p.off64.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->done_count, 0, sizeof(int), s);
  return e;
}

cudaError_t ensure_iter_events(lsgcpd_ctx* c, int iters) {
  if (c->t_iter_cap >= iters) return cudaSuccess;
  if (c->t_iter) {
    for (int i = 0; i < 4 * c->t_iter_cap; ++i) cudaEventDestroy(c->t_iter[i]);
    delete[] c->t_iter;
  }
  c->t_iter = new cudaEvent_t[4 * iters];
  c->t_iter_cap = iters;
  for (int i = 0; i < 4 * iters; ++i) {
    cudaError_t e = cudaEventCreate(&c->t_iter[i]);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Elapsed ms between two recorded events; 0 (and the error cleared) if unavailable.
double elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
    cudaGetLastError();
    return 0.0;
  }
  return ms;
}

// Centred-frame moments -> caller's frame (x~_raw = T x~_c, T = [[I, mu_x], [0, 1]]).
void moments_to_raw(const double* mc, const double mu[3], double* mr) {
  for (int j = 0; j < LSGCPD_MOMENTS; ++j) mr[j] = mc[j];
  double T[4][4] = {{1, 0, 0, mu[0]}, {0, 1, 0, mu[1]}, {0, 0, 1, mu[2]}, {0, 0, 0, 1}};
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 4; ++k) {
      double s = 0;
      for (int l = 0; l < 4; ++l) s += mc[2 + 4 * i + l] * T[k][l];
      mr[2 + 4 * i + k] = s;
    }
  int pidx[4][4];
  int q = 0;
  for (int k = 0; k < 4; ++k)
    for (int l = k; l < 4; ++l, ++q) pidx[k][l] = pidx[l][k] = q;
  for (int p = 0; p < 6; ++p) {
    double Gc[4][4];
    for (int k = 0; k < 4; ++k)
      for (int l = 0; l < 4; ++l) Gc[k][l] = mc[14 + p * 10 + pidx[k][l]];
    for (int k = 0; k < 4; ++k)
      for (int l = k; l < 4; ++l) {
        double s = 0;
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) s += T[k][a] * T[l][b] * Gc[a][b];
        mr[14 + p * 10 + pidx[k][l]] = s;
      }
  }
}

// One or more registrations: X and Y are the concatenated clouds (host or
// device), sizes N[i], M[i].  Results per pair in the caller's frame.
// Inputs of a registration on the device: host arrays copied in, confidences
// checked, and (Sec. 3.3) the points below the confidence threshold removed.
struct Staged {
  const float* X = nullptr;
  const float* Y = nullptr;
  const float* phx = nullptr;
  const float* phy = nullptr;
  std::vector<long long> N, M;
  int64_t h2d = 0;
  int64_t launches = 0;
};

// Stable per-pair removal of the rows whose confidence is below the threshold
// (one host round trip for the kept counts).
lsgcpd_status compact_side(lsgcpd_ctx* c, const float* rows, const float* phi, std::vector<long long>& sizes,
                           float thr, DevBuf<float>& rows_out, DevBuf<float>& phi_out, int64_t* launches) {
  cudaStream_t s = c->stream;
  const int P = static_cast<int>(sizes.size());
  long long big = 1;
  std::vector<long long> off(P + 1, 0);
  for (int i = 0; i < P; ++i) {
    off[i + 1] = off[i] + sizes[i];
    big = std::max(big, sizes[i]);
  }
  const int chunks = compact_chunks(big);
  LSG_CUDA(ensure(c->cnt, static_cast<size_t>(P) * chunks), "alloc");
  LSG_CUDA(ensure(c->coff, static_cast<size_t>(P) * chunks), "alloc");
  LSG_CUDA(ensure(c->toff, 2 * static_cast<size_t>(P + 1)), "alloc");
  LSG_CUDA(cudaMemcpyAsync(c->toff.p, off.data(), sizeof(long long) * (P + 1), cudaMemcpyHostToDevice, s), "copy");
  LSG_CUDA(launch_compact_count(phi, c->toff.p, P, chunks, thr, c->cnt.p, s), "compact");
  std::vector<int> cnt(static_cast<size_t>(P) * chunks);
  int status = 0;
  LSG_CUDA(cudaMemcpyAsync(cnt.data(), c->cnt.p, sizeof(int) * cnt.size(), cudaMemcpyDeviceToHost, s), "copy");
  LSG_CUDA(cudaMemcpyAsync(&status, c->status, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
  LSG_CUDA(cudaStreamSynchronize(s), "sync");
  if (status & 8) return fail(c, LSGCPD_EINVAL, "inputs contain NaN or Inf");
  if (status & 16) return fail(c, LSGCPD_EINVAL, "confidences must lie in (0, 1]");
  std::vector<int> coff(cnt.size());
  std::vector<long long> out_off(P + 1, 0);
  for (int i = 0; i < P; ++i) {
    long long run = 0;
    for (int j = 0; j < chunks; ++j) {
      coff[static_cast<size_t>(i) * chunks + j] = static_cast<int>(run);
      run += cnt[static_cast<size_t>(i) * chunks + j];
    }
    sizes[i] = run;
    out_off[i + 1] = out_off[i] + run;
  }
  LSG_CUDA(ensure(rows_out, static_cast<size_t>(out_off[P]) * 3), "alloc");
  LSG_CUDA(ensure(phi_out, static_cast<size_t>(out_off[P])), "alloc");
  LSG_CUDA(cudaMemcpyAsync(c->coff.p, coff.data(), sizeof(int) * coff.size(), cudaMemcpyHostToDevice, s), "copy");
  LSG_CUDA(cudaMemcpyAsync(c->toff.p + (P + 1), out_off.data(), sizeof(long long) * (P + 1), cudaMemcpyHostToDevice,
                           s),
           "copy");
  LSG_CUDA(launch_compact_scatter(rows, phi, c->toff.p, c->toff.p + (P + 1), c->coff.p, P, chunks, thr, rows_out.p,
                                  phi_out.p, s),
           "compact");
  *launches += 2;
  // the host vectors above are staged by the copies before these calls return
  return LSGCPD_OK;
}

lsgcpd_status stage(lsgcpd_ctx* c, const float* X, const float* Y, const std::vector<long long>& N,
                    const std::vector<long long>& M, const lsgcpd_params* p, bool xd, bool yd, Staged* in) {
  cudaStream_t s = c->stream;
  if (!plan_fits(N, M)) return fail(c, LSGCPD_EINVAL, kTooLarge);
  long long Ntot = 0, Mtot = 0;
  for (long long v : N) Ntot += v;
  for (long long v : M) Mtot += v;
  in->N = N;
  in->M = M;
  in->X = X;
  in->Y = Y;
  in->phx = p->phi_x;
  in->phy = p->phi_y;
  auto up = [&](DevBuf<float>& buf, const float* h, long long n) -> cudaError_t {
    cudaError_t e = ensure(buf, static_cast<size_t>(n));
    if (e == cudaSuccess) e = cudaMemcpyAsync(buf.p, h, sizeof(float) * n, cudaMemcpyHostToDevice, s);
    in->h2d += 4 * n;
    return e;
  };
  if (!xd) {
    LSG_CUDA(up(c->X_in, X, 3 * Ntot), "copy X");
    in->X = c->X_in.p;
  }
  if (!yd) {
    LSG_CUDA(up(c->Y_in, Y, 3 * Mtot), "copy Y");
    in->Y = c->Y_in.p;
  }
  if (p->phi_x && !xd) {
    LSG_CUDA(up(c->phx_in, p->phi_x, Ntot), "copy phi_x");
    in->phx = c->phx_in.p;
  }
  if (p->phi_y && !yd) {
    LSG_CUDA(up(c->phy_in, p->phi_y, Mtot), "copy phi_y");
    in->phy = c->phy_in.p;
  }
  LSG_CUDA(cudaMemsetAsync(c->status, 0, sizeof(int), s), "memset");
  LSG_CUDA(check_finite(in->X, Ntot * 3, c->status, s), "check");
  LSG_CUDA(check_finite(in->Y, Mtot * 3, c->status, s), "check");
  in->launches += 2;
  if (in->phx) {
    LSG_CUDA(check_conf(in->phx, Ntot, c->status, s), "check");
    ++in->launches;
  }
  if (in->phy) {
    LSG_CUDA(check_conf(in->phy, Mtot, c->status, s), "check");
    ++in->launches;
  }
  const float thr = static_cast<float>(p->cf_threshold);
  if (p->cf_threshold > 0.0 && in->phx) {
    lsgcpd_status r = compact_side(c, in->X, in->phx, in->N, thr, c->Xc, c->phxc, &in->launches);
    if (r != LSGCPD_OK) return r;
    in->X = c->Xc.p;
    in->phx = c->phxc.p;
  }
  if (p->cf_threshold > 0.0 && in->phy) {
    lsgcpd_status r = compact_side(c, in->Y, in->phy, in->M, thr, c->Yc, c->phyc, &in->launches);
    if (r != LSGCPD_OK) return r;
    in->Y = c->Yc.p;
    in->phy = c->phyc.p;
  }
  for (size_t i = 0; i < in->N.size(); ++i) {
    if (in->N[i] < 1 || in->M[i] < 1)
      return fail(c, LSGCPD_EINVAL, "confidence truncation left a pair without points");
    if (p->knn_k > in->M[i]) return fail(c, LSGCPD_EINVAL, "knn_k must not exceed the target count of any pair");
  }
  return LSGCPD_OK;
}

// One or more registrations: X and Y are the concatenated clouds (host or
// device), sizes N[i], M[i].  Results per pair in the caller's frame.
}  // namespace

namespace lsg {
static thread_local bool t_pdl = false;
void set_pdl(bool on) { t_pdl = on; }
bool pdl_on() { return t_pdl; }
}  // namespace lsg

namespace {

// NVTX range over a host phase (a no-op unless a profiler is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// LSGCPD_LOG=1: print every pair's per-iteration trace to stderr after a registration.
bool log_enabled() {
  const char* v = getenv("LSGCPD_LOG");
  return v && v[0] && strcmp(v, "0") != 0;
}

void print_trace(const double* trace, int P, int iters, const std::vector<EmState>& hs) {
  for (int i = 0; i < P; ++i)
    for (int it = 0; it < hs[i].iter && it < iters; ++it) {
      const double* r = trace + (static_cast<size_t>(i) * iters + it) * LSGCPD_TRACE_WIDTH;
      fprintf(stderr,
              "lsgcpd pair %d iter %d: sigma2 %.9g N_P %.9g Q %.9g newton %d damped %d motion %.3g nll %.12g "
              "outlier mass %.6g\n",
              i, it, r[0], r[1], r[2], static_cast<int>(r[3]), static_cast<int>(r[4]), r[5], r[6], r[7]);
    }
}

lsgcpd_status run_registration(lsgcpd_ctx* c, const float* X, const float* Y, const std::vector<long long>& N_in,
                               const std::vector<long long>& M_in, const lsgcpd_params* p, double* R_out,
                               double* t_out, double* sigma2_out, int32_t* iters_out, int32_t* mode_out,
                               double* trace, void* stream) {
  NvtxRange range_all("lsgcpd registration");
  const int P = static_cast<int>(N_in.size());
  const int k = p->knn_k;
  // with LSGCPD_LOG the trace is recorded into a host buffer of our own if the caller did not ask for it
  std::vector<double> log_trace;
  const bool log = log_enabled() && p->max_iters > 0;
  if (log && !trace) {
    log_trace.assign(static_cast<size_t>(P) * p->max_iters * LSGCPD_TRACE_WIDTH, 0.0);
    trace = log_trace.data();
  }
  LSG_CUDA(enter(c, stream), "stream");
  cudaStream_t s = c->stream;
  const bool xd = is_device_ptr(X), yd = is_device_ptr(Y);
  const int iters = p->max_iters;
  if (c->timing) {
    LSG_CUDA(ensure_iter_events(c, iters > 0 ? iters : 1), "events");
    LSG_CUDA(cudaEventRecord(c->t_begin, s), "event");
  }
  Staged in;
  lsgcpd_status rs;
  {
    NvtxRange r("lsgcpd stage inputs");
    rs = stage(c, X, Y, N_in, M_in, p, xd, yd, &in);
  }
  if (rs != LSGCPD_OK) {
    leave(c, stream);
    return rs;
  }
  const std::vector<long long>& N = in.N;
  const std::vector<long long>& M = in.M;
  const float* Xd = in.X;
  const float* Yd = in.Y;
  // source tile: measured once per problem shape (cached), else the plan's heuristic
  std::vector<long long> skey = N;
  skey.insert(skey.end(), M.begin(), M.end());
  const lsgcpd_ctx::Tuned* hit = nullptr;
  if (c->autotune)
    for (const auto& t : c->tuned)
      if (t.sizes == skey) hit = &t;
  double pairs = 0;
  for (int i = 0; i < P; ++i) pairs += static_cast<double>(N[i]) * static_cast<double>(M[i]);
  // the tensor-core E step has one source tile (4 sources per thread): nothing to tune
  const bool tc = p->precision == 2;
  const bool tune = c->autotune && iters > 0 && !hit && pairs <= kTuneMaxPairs && !tc;
  BatchPlan plan = plan_batch(N, M, c->num_sms, tc ? 4 : (hit ? hit->S : 0));
  std::vector<BatchPlan> cands;
  if (tune)
    for (int S : {4, 2, 1}) cands.push_back(S == plan.g.S ? plan : plan_batch(N, M, c->num_sms, S));
  rs = reserve(c, plan, k, iters, false, tc);
  for (size_t i = 0; i < cands.size() && rs == LSGCPD_OK; ++i) rs = reserve(c, cands[i], k, iters, false);
  if (rs != LSGCPD_OK) return rs;
  const Dev d = dev_of(c);
  int64_t launches = in.launches;
  const DevParams dp = dev_params(p);
  // the EM state of every pair: centring, V, sigma^2_0, then w0 from the outlier ratio if asked
  auto init_state = [&](const BatchPlan& pl) -> cudaError_t {
    cudaError_t e = launch_init(pl, d, Xd, Yd, in.phx, in.phy, dp, true, c->red.p, c->xs.p, s);
    if (e == cudaSuccess && p->eta > 0.0) e = launch_eta(pl, d, c->yl.p, p->eta, s);
    launches += 4 + (p->eta > 0.0 ? 1 : 0);
    return e;
  };
  LSG_CUDA(upload_plan(c, plan, s), "plan");
  LSG_CUDA(launch_init(plan, d, Xd, Yd, in.phx, in.phy, dp, true, c->red.p, c->xs.p, s), "init");
  LSG_CUDA(run_knn(c, plan, d, Yd, k, p->knn_method, c->knn_idx.p, &launches, s), "knn");
  LSG_CUDA(launch_geometry(plan, d, Yd, in.phy, c->knn_idx.p, k, p->alpha_max, p->lambda, p->include_alpha_norm,
                           c->rec.p, c->yl.p, nullptr, nullptr, nullptr, s),
           "geometry");
  launches += 4 + 1;
  if (p->eta > 0.0) {
    LSG_CUDA(launch_eta(plan, d, c->yl.p, p->eta, s), "eta");
    ++launches;
  }
  if (tc) {
    LSG_CUDA(launch_features(plan, c->rec.p, c->yl.p, c->feat.p, s), "features");
    ++launches;
  }
  if (c->timing) LSG_CUDA(cudaEventRecord(c->t_prep, s), "event");
  std::vector<EmState> hs(P);
  int status = 0;
  LSG_CUDA(cudaMemcpyAsync(hs.data(), c->st.p, sizeof(EmState) * P, cudaMemcpyDeviceToHost, s), "copy");
  LSG_CUDA(cudaMemcpyAsync(&status, c->status, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
  LSG_CUDA(cudaStreamSynchronize(s), "sync");
  if (status & (8 | 16)) {
    leave(c, stream);
    return fail(c, LSGCPD_EINVAL, (status & 8) ? "inputs contain NaN or Inf" : "confidences must lie in (0, 1]");
  }
  // one shift mode for the whole batch: fixed shift only if it is safe for every pair, l_m is
  // uniform (the uniform-shift moments assume one l) and w_n is uniform
  const double l_extra = p->include_alpha_norm ? 0.5 * log2(1.0 + p->alpha_max) : 0.0;
  int mode = (p->include_alpha_norm || in.phx || in.phy || p->precision == 1) ? 1 : 0;
  const int prec = p->precision;
  for (int i = 0; i < P; ++i) mode |= choose_mode(hs[i].w0, hs[i].sigma2_floor, hs[i].V, M[i], l_extra);
  const int cfx = in.phx ? 1 : 0;
  if (tune) {
    // time three back-to-back E-step launches (after a warm-up launch) for every source tile; the
    // fastest wins unless the rule's own choice is within 2% of it (noise must not flip the plan);
    // the target records do not depend on the tile, the source layout and the EM state are rebuilt
    const int rule_S = plan.g.S;
    lsgcpd_ctx::Tuned rec{skey, plan.g.S, {0, 0, 0}};
    for (const BatchPlan& pc : cands) {
      LSG_CUDA(upload_plan(c, pc, s), "plan");
      LSG_CUDA(init_state(pc), "init");
      LSG_CUDA(launch_prescale(pc, d, c->yl.p, mode, c->rec.p, s), "prescale");
      if (mode) LSG_CUDA(launch_shift(pc, d, c->xs.p, c->rec.p, cfx, c->part.p, c->status, c->ls_n.p, c->gam_n.p, s), "shift");
      LSG_CUDA(estep_launch(c, pc, d, mode, prec, s), "estep");
      LSG_CUDA(cudaEventRecord(c->tune_ev[0], s), "event");
      for (int r = 0; r < 3; ++r) LSG_CUDA(estep_launch(c, pc, d, mode, prec, s), "estep");
      LSG_CUDA(cudaEventRecord(c->tune_ev[1], s), "event");
      LSG_CUDA(cudaEventSynchronize(c->tune_ev[1]), "sync");
      rec.ms[pc.g.S == 4 ? 0 : (pc.g.S == 2 ? 1 : 2)] = elapsed_ms(c->tune_ev[0], c->tune_ev[1]) / 3.0;
      launches += (mode ? 5 : 3) + 2;
    }
    const auto slot = [](int S) { return S == 4 ? 0 : (S == 2 ? 1 : 2); };
    double best = 1e300;
    for (const BatchPlan& pc : cands) {
      const double ms = rec.ms[slot(pc.g.S)];
      if (ms > 0 && ms < best) {
        best = ms;
        rec.S = pc.g.S;
      }
    }
    const double rule_ms = rec.ms[slot(rule_S)];
    if (rule_ms > 0 && rule_ms <= 1.02 * best) rec.S = rule_S;
    for (const BatchPlan& pc : cands)
      if (pc.g.S == rec.S) plan = pc;
    c->tuned.push_back(rec);
    hit = &c->tuned.back();
    LSG_CUDA(upload_plan(c, plan, s), "plan");
    LSG_CUDA(init_state(plan), "init");
  }
  const Geo& g = plan.g;
  c->last_plan[0] = g.S;
  c->last_plan[1] = g.SB;
  c->last_plan[2] = g.grid;
  c->last_plan[3] = hit ? 1 : 0;
  for (int i = 0; i < 3; ++i) c->last_tune_ms[i] = hit ? hit->ms[i] : 0.0;
  if (iters > 0) {
    GraphKey key;
    key.sizes = N;
    key.sizes.insert(key.sizes.end(), M.begin(), M.end());
    key.params.assign(reinterpret_cast<const unsigned char*>(&dp),
                      reinterpret_cast<const unsigned char*>(&dp) + sizeof(dp));
    key.iters = iters;
    key.mode = mode;
    key.prec = prec;
    key.S = g.S;
    key.timing = c->timing;
    key.trace = trace ? 1 : 0;
    if (!(c->gexec && key == c->gkey)) {
      cudaGraph_t gr = nullptr;
      LSG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "capture");
      set_pdl(true);  // consecutive kernels of the loop overlap their launch with the predecessor's tail
      const bool fused = mstep_sums_rows(g);
      const bool fused_prescale = mstep_prescales(g);  // the M step prescales the next E step's records
      cudaError_t ce = cudaSuccess;
      for (int it = 0; it < iters && ce == cudaSuccess; ++it) {
        if (c->timing) ce = cudaEventRecordWithFlags(c->t_iter[4 * it], s, cudaEventRecordExternal);
        if (ce == cudaSuccess && (it == 0 || !fused_prescale))
          ce = launch_prescale(plan, d, c->yl.p, mode, c->rec.p, s);
        if (ce == cudaSuccess && mode == 1)
          ce = launch_shift(plan, d, c->xs.p, c->rec.p, cfx, c->part.p, c->status, c->ls_n.p, c->gam_n.p, s);
        if (ce == cudaSuccess) ce = estep_launch(c, plan, d, mode, prec, s);
        if (ce == cudaSuccess && c->timing)
          ce = cudaEventRecordWithFlags(c->t_iter[4 * it + 1], s, cudaEventRecordExternal);
        if (ce == cudaSuccess)
          ce = launch_combine(plan, d, c->xs.p, c->part.p, mode, cfx, c->ls_n.p, c->gam_n.p, c->rows.p, nullptr,
                              s);
        // small problems: the M-step kernel sums the combine rows itself (one boundary less)
        if (ce == cudaSuccess && !fused) ce = launch_final_reduce(plan, d, c->rows.p, c->mom.p, s);
        if (ce == cudaSuccess && c->timing)
          ce = cudaEventRecordWithFlags(c->t_iter[4 * it + 2], s, cudaEventRecordExternal);
        if (ce == cudaSuccess)
          ce = launch_mstep(plan, d, fused ? c->rows.p : nullptr, c->mom.p, dp, trace ? c->trace.p : nullptr, iters,
                            fused_prescale && it + 1 < iters ? c->yl.p : nullptr, mode, c->rec.p, s);
        if (ce == cudaSuccess && c->timing)
          ce = cudaEventRecordWithFlags(c->t_iter[4 * it + 3], s, cudaEventRecordExternal);
      }
      set_pdl(false);
      cudaError_t ee = cudaStreamEndCapture(s, &gr);
      if (ce != cudaSuccess || ee != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        return cuda_fail(c, ce != cudaSuccess ? ce : ee, "graph capture");
      }
      // the same loop for another problem (same node sequence, other sizes and launch
      // shapes): update the executable graph's parameters in place, a fraction of the cost
      // of instantiating it; anything the update cannot express is instantiated afresh
      bool updated = false;
      if (c->gexec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(c->gexec, gr, &info) == cudaSuccess) {
          updated = true;
        } else {
          cudaGetLastError();
          cudaGraphExecDestroy(c->gexec);
          c->gexec = nullptr;
        }
      }
      cudaError_t ie = updated ? cudaSuccess : cudaGraphInstantiate(&c->gexec, gr, 0);
      cudaGraphDestroy(gr);
      if (ie != cudaSuccess) {
        c->gexec = nullptr;
        return cuda_fail(c, ie, "graph instantiate");
      }
      c->gkey = key;
    }
    NvtxRange r("lsgcpd EM loop (graph)");
    LSG_CUDA(cudaGraphLaunch(c->gexec, s), "graph launch");
    launches += static_cast<int64_t>(iters) * ((mode ? 7 : 5) - (mstep_sums_rows(g) ? 1 : 0)) -
                (mstep_prescales(g) ? iters - 1 : 0);
  }
  if (c->timing) LSG_CUDA(cudaEventRecord(c->t_end, s), "event");
  LSG_CUDA(cudaMemcpyAsync(hs.data(), c->st.p, sizeof(EmState) * P, cudaMemcpyDeviceToHost, s), "copy");
  LSG_CUDA(cudaMemcpyAsync(&status, c->status, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
  if (trace && iters > 0)
    LSG_CUDA(cudaMemcpyAsync(trace, c->trace.p, sizeof(double) * LSGCPD_TRACE_WIDTH * iters * P,
                             cudaMemcpyDeviceToHost, s),
             "copy trace");
  LSG_CUDA(cudaStreamSynchronize(s), "sync");
  LSG_CUDA(leave(c, stream), "stream");
  if (log && iters > 0) print_trace(trace, P, iters, hs);
  c->launches = launches;
  c->h2d_bytes = in.h2d +
                 static_cast<int64_t>(sizeof(int) * plan.tab.size() + sizeof(long long) * plan.off64.size());
  c->d2h_bytes = 2 * static_cast<int64_t>(sizeof(EmState) * P + sizeof(int)) +
                 (trace && iters > 0 ? static_cast<int64_t>(sizeof(double)) * LSGCPD_TRACE_WIDTH * iters * P : 0);
  bool numeric = false;
  for (int i = 0; i < P; ++i) {
    const EmState& h = hs[i];
    // result in the caller's frame: t = t_c + mu_y - R mu_x
    for (int q = 0; q < 9; ++q) R_out[9 * i + q] = h.R[q];
    for (int q = 0; q < 3; ++q)
      t_out[3 * i + q] =
          h.t[q] + h.mu_y[q] - (h.R[3 * q] * h.mu_x[0] + h.R[3 * q + 1] * h.mu_x[1] + h.R[3 * q + 2] * h.mu_x[2]);
    if (sigma2_out) sigma2_out[i] = h.sigma2;
    if (iters_out) iters_out[i] = h.iter;
    numeric = numeric || h.numeric_fail;
  }
  if (mode_out) *mode_out = mode;
  if (c->timing) {
    double es = 0, cb = 0, ms = 0;
    for (int it = 0; it < iters; ++it) {
      es += elapsed_ms(c->t_iter[4 * it], c->t_iter[4 * it + 1]);
      cb += elapsed_ms(c->t_iter[4 * it + 1], c->t_iter[4 * it + 2]);
      ms += elapsed_ms(c->t_iter[4 * it + 2], c->t_iter[4 * it + 3]);
    }
    c->last_timing[0] = elapsed_ms(c->t_begin, c->t_end);
    c->last_timing[1] = es;
    c->last_timing[2] = cb;
    c->last_timing[3] = ms;
    c->last_timing[4] = elapsed_ms(c->t_begin, c->t_prep);
  }
  if (status & kStatusTimeout) return fail(c, LSGCPD_ETIMEOUT, "E-step tile wait timed out");
  if (numeric) return fail(c, LSGCPD_ENUMERIC, "posterior mass vanished (N_P = 0)");
  return LSGCPD_OK;
}

}  // namespace

extern "C" {

void lsgcpd_params_default(lsgcpd_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->w = 0.1;
  p->alpha_max = 2.0;
  p->lambda = 0.2;
  for (int i = 0; i < 9; ++i) p->init_R[i] = (i % 4 == 0) ? 1.0 : 0.0;
  p->newton_tol = 1e-12;
  p->sigma2_floor_rel = 1e-10;
  p->knn_k = 10;
  p->max_iters = 50;
  p->newton_max = 20;
}

lsgcpd_status lsgcpd_create(lsgcpd_ctx** out, int device, int64_t max_N, int64_t max_M) {
  if (!out) return LSGCPD_EINVAL;
  *out = nullptr;
  if (max_N < 1 || max_M < 1 || !lsg::plan_fits({max_N}, {max_M})) return LSGCPD_EINVAL;
  lsgcpd_ctx* c = new lsgcpd_ctx();
  c->device = device;
  auto bail = [&](lsgcpd_status s) {
    lsgcpd_destroy(c);
    return s;
  };
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return bail(LSGCPD_ECUDA);
  }
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    return bail(LSGCPD_ECUDA);
  }
  if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&c->t_begin) != cudaSuccess || cudaEventCreate(&c->t_prep) != cudaSuccess ||
      cudaEventCreate(&c->t_end) != cudaSuccess || cudaEventCreate(&c->tune_ev[0]) != cudaSuccess ||
      cudaEventCreate(&c->tune_ev[1]) != cudaSuccess) {
    cudaGetLastError();
    return bail(LSGCPD_ECUDA);
  }
  if (cudaMalloc(&c->status, sizeof(int)) != cudaSuccess || cudaMalloc(&c->done_count, sizeof(int)) != cudaSuccess ||
      ensure(c->io, 128) != cudaSuccess) {
    cudaGetLastError();
    return bail(LSGCPD_ENOMEM);
  }
  cudaMemset(c->status, 0, sizeof(int));
  cudaMemset(c->done_count, 0, sizeof(int));
  const BatchPlan p = plan_batch({max_N}, {max_M}, c->num_sms, 0);
  if (reserve(c, p, 10, 50, false) != LSGCPD_OK) return bail(LSGCPD_ENOMEM);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return bail(LSGCPD_ECUDA);
  }
  *out = c;
  return LSGCPD_OK;
}

void lsgcpd_destroy(lsgcpd_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  void* bufs2[] = {c->pern_tmp.p, c->phx_in.p, c->phy_in.p, c->Xc.p,      c->Yc.p,       c->phxc.p,    c->phyc.p,   c->cnt.p,
                   c->coff.p,   c->toff.p,   c->g_count.p, c->g_start.p,  c->g_fill.p,  c->g_cellof.p,
                   c->g_scan.p, c->g_sorted.p, c->g_info.p, c->feat.p};
  for (void* q : bufs2)
    if (q) cudaFree(q);
  void* bufs[] = {c->X_in.p, c->Y_in.p,    c->rec.p, c->part.p,  c->knn_d.p, c->ls_n.p, c->gam_n.p,
                  c->xs.p,   c->y4.p,  c->yl.p,      c->knn_i.p, c->knn_idx.p, c->tab.p, c->off64.p, c->rows.p,
                  c->red.p,  c->trace.p,   c->io.p,  c->mom.p,   c->st.p,    c->status,  c->done_count};
  for (void* q : bufs)
    if (q) cudaFree(q);
  if (c->t_iter) {
    for (int i = 0; i < 4 * c->t_iter_cap; ++i) cudaEventDestroy(c->t_iter[i]);
    delete[] c->t_iter;
  }
  cudaEvent_t evs[] = {c->ev_in, c->ev_out, c->t_begin, c->t_prep, c->t_end, c->tune_ev[0], c->tune_ev[1]};
  for (cudaEvent_t e : evs)
    if (e) cudaEventDestroy(e);
  if (c->stream) cudaStreamDestroy(c->stream);
  cudaGetLastError();
  delete c;
}

const char* lsgcpd_last_error(const lsgcpd_ctx* c) { return c ? c->err.c_str() : "null context"; }

lsgcpd_status lsgcpd_set_timing(lsgcpd_ctx* c, int enable) {
  if (!c) return LSGCPD_EINVAL;
  c->timing = enable ? 1 : 0;
  return LSGCPD_OK;
}

lsgcpd_status lsgcpd_set_autotune(lsgcpd_ctx* c, int enable) {
  if (!c) return LSGCPD_EINVAL;
  c->autotune = enable ? 1 : 0;
  return LSGCPD_OK;
}

namespace {
// Key of this context's device in the autotune file: its name (spaces as '_') and SM count.
std::string device_key(const lsgcpd_ctx* c) {
  cudaDeviceProp prop;
  std::string name = "unknown";
  if (cudaGetDeviceProperties(&prop, c->device) == cudaSuccess) name = prop.name;
  else cudaGetLastError();
  for (char& ch : name)
    if (ch == ' ' || ch == '\t' || ch == '\n') ch = '_';
  return name + ":" + std::to_string(c->num_sms);
}
const char kTuneHeader[] = "lsgcpd-autotune 1";
}  // namespace

lsgcpd_status lsgcpd_autotune_save(const lsgcpd_ctx* c, const char* path) {
  if (!c || !path) return LSGCPD_EINVAL;
  FILE* f = fopen(path, "w");
  if (!f) return LSGCPD_EINVAL;
  const std::string key = device_key(c);
  fprintf(f, "%s\n", kTuneHeader);
  // line: device-key S ms4 ms2 ms1 n_sizes sizes...
  for (const auto& t : c->tuned) {
    fprintf(f, "%s %d %.17g %.17g %.17g %zu", key.c_str(), t.S, t.ms[0], t.ms[1], t.ms[2], t.sizes.size());
    for (long long v : t.sizes) fprintf(f, " %lld", v);
    fprintf(f, "\n");
  }
  const bool ok = fclose(f) == 0;
  return ok ? LSGCPD_OK : LSGCPD_EINVAL;
}

lsgcpd_status lsgcpd_autotune_load(lsgcpd_ctx* c, const char* path, int32_t* count) {
  if (!c || !path) return LSGCPD_EINVAL;
  if (count) *count = 0;
  FILE* f = fopen(path, "r");
  if (!f) return fail(c, LSGCPD_EINVAL, "autotune file cannot be read");
  const std::string key = device_key(c);
  std::vector<char> line(1 << 20);
  int added = 0;
  bool header = false;
  while (fgets(line.data(), static_cast<int>(line.size()), f)) {
    if (!header) {
      header = strncmp(line.data(), kTuneHeader, sizeof(kTuneHeader) - 1) == 0;
      if (!header) break;
      continue;
    }
    char dev[256];
    int S = 0, used = 0;
    size_t n = 0;
    double ms[3];
    if (sscanf(line.data(), "%255s %d %lf %lf %lf %zu%n", dev, &S, &ms[0], &ms[1], &ms[2], &n, &used) != 6) continue;
    if (key != dev || (S != 1 && S != 2 && S != 4) || n == 0 || n % 2 != 0 || n > 2 * LSGCPD_MAX_PAIRS) continue;
    lsgcpd_ctx::Tuned t;
    t.S = S;
    for (int i = 0; i < 3; ++i) t.ms[i] = ms[i];
    const char* q = line.data() + used;
    bool good = true;
    for (size_t i = 0; i < n && good; ++i) {
      long long v = 0;
      int u = 0;
      good = sscanf(q, "%lld%n", &v, &u) == 1 && v > 0;
      q += u;
      t.sizes.push_back(v);
    }
    if (!good) continue;
    bool dup = false;
    for (auto& e : c->tuned)
      if (e.sizes == t.sizes) {
        e = t;
        dup = true;
      }
    if (!dup) c->tuned.push_back(t);
    ++added;
  }
  fclose(f);
  if (!header) return fail(c, LSGCPD_EINVAL, "not an autotune file");
  if (count) *count = added;
  return LSGCPD_OK;
}

lsgcpd_status lsgcpd_plan_info(const lsgcpd_ctx* c, int32_t info[4], double tune_ms[3]) {
  if (!c || !info) return LSGCPD_EINVAL;
  for (int i = 0; i < 4; ++i) info[i] = c->last_plan[i];
  if (tune_ms)
    for (int i = 0; i < 3; ++i) tune_ms[i] = c->last_tune_ms[i];
  return LSGCPD_OK;
}

lsgcpd_status lsgcpd_selftest_timeout(lsgcpd_ctx* c, int64_t budget_cycles) {
  if (!c) return LSGCPD_EINVAL;
  c->err.clear();
  if (budget_cycles < 1 || budget_cycles > 4000000000LL) return fail(c, LSGCPD_EINVAL, "budget out of range");
  LSG_CUDA(cudaSetDevice(c->device), "device");
  cudaStream_t s = c->stream;
  int status = 0;
  LSG_CUDA(cudaMemsetAsync(c->status, 0, sizeof(int), s), "memset");
  LSG_CUDA(launch_wait_selftest(budget_cycles, c->status, s), "selftest");
  LSG_CUDA(cudaMemcpyAsync(&status, c->status, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
  LSG_CUDA(cudaStreamSynchronize(s), "sync");
  if (status & kStatusTimeout) return fail(c, LSGCPD_ETIMEOUT, "bounded wait gave up (expected)");
  return LSGCPD_OK;
}

lsgcpd_status lsgcpd_last_timing(const lsgcpd_ctx* c, double out[8]) {
  if (!c || !out) return LSGCPD_EINVAL;
  for (int i = 0; i < 5; ++i) out[i] = c->last_timing[i];
  out[5] = static_cast<double>(c->launches);
  out[6] = static_cast<double>(c->h2d_bytes);
  out[7] = static_cast<double>(c->d2h_bytes);
  return c->timing ? LSGCPD_OK : LSGCPD_EINVAL;
}

lsgcpd_status lsgcpd_preprocess(lsgcpd_ctx* c, const float* Y, int64_t M, const lsgcpd_params* p, float* normals,
                                float* kappa, float* alpha, int32_t* knn_idx, void* stream) {
  if (!c) return LSGCPD_EINVAL;
  c->err.clear();
  if (!Y || M < 1) return fail(c, LSGCPD_EINVAL, "Y must be non-NULL with M >= 1");
  lsgcpd_status ps = check_params(c, p);
  if (ps != LSGCPD_OK) return ps;
  const int k = p->knn_k;
  if (k < 1 || k > kMaxK || k > M) return fail(c, LSGCPD_EINVAL, "knn_k must satisfy 1 <= k <= min(M, 32)");
  if (!plan_fits({M}, {M})) return fail(c, LSGCPD_EINVAL, kTooLarge);
  LSG_CUDA(enter(c, stream), "stream");
  // a batch of one whose source cloud is Y itself (only the target side is used)
  const BatchPlan plan = plan_batch({M}, {M}, c->num_sms, 1);
  lsgcpd_status rs = reserve(c, plan, k, 1, false);
  if (rs != LSGCPD_OK) return rs;
  cudaStream_t s = c->stream;
  const Dev d = dev_of(c);
  LSG_CUDA(upload_plan(c, plan, s), "plan");
  LSG_CUDA(cudaMemsetAsync(c->status, 0, sizeof(int), s), "memset");
  LSG_CUDA(check_finite(Y, M * 3, c->status, s), "check");
  const DevParams dp = dev_params(p);
  LSG_CUDA(launch_init(plan, d, Y, Y, nullptr, nullptr, dp, false, c->red.p, c->xs.p, s), "center");
  int* idx = knn_idx ? knn_idx : c->knn_idx.p;
  int64_t launches = 5;
  LSG_CUDA(run_knn(c, plan, d, Y, k, p->knn_method, idx, &launches, s), "knn");
  LSG_CUDA(launch_geometry(plan, d, Y, nullptr, idx, k, p->alpha_max, p->lambda, p->include_alpha_norm, c->rec.p,
                           c->yl.p,
                           normals, kappa, alpha, s),
           "geometry");
  c->launches = launches;
  int status = 0;
  LSG_CUDA(cudaMemcpyAsync(&status, c->status, sizeof(int), cudaMemcpyDeviceToHost, s), "status");
  LSG_CUDA(cudaStreamSynchronize(s), "sync");
  LSG_CUDA(leave(c, stream), "stream");
  if (status & 8) return fail(c, LSGCPD_EINVAL, "Y contains NaN or Inf");
  return LSGCPD_OK;
}

}  // extern "C"

namespace {

// One E step at (R, t, sigma2) with optional per-source output and, for small
// problems, the dense posteriors (P: device, (M + 1) x N, outlier row last).
lsgcpd_status estep_impl(lsgcpd_ctx* c, const float* X, int64_t N, const float* Y, const float* normals,
                         const float* alpha, int64_t M, const lsgcpd_params* p, const double R[9], const double t[3],
                         double sigma2, double volume, double* moments, float* per_n, float* P, void* stream) {
  if (!c) return LSGCPD_EINVAL;
  c->err.clear();
  if (!X || !Y || !normals || !alpha || !R || !t) return fail(c, LSGCPD_EINVAL, "NULL input");
  if (N < 1 || M < 1) return fail(c, LSGCPD_EINVAL, "N and M must be >= 1");
  lsgcpd_status ps = check_params(c, p);
  if (ps != LSGCPD_OK) return ps;
  if (!(sigma2 > 0.0) || !is_finite_d(sigma2)) return fail(c, LSGCPD_EINVAL, "sigma2 must be finite and > 0");
  if (!(volume > 0.0) || !is_finite_d(volume)) return fail(c, LSGCPD_EINVAL, "volume must be finite and > 0");
  for (int i = 0; i < 9; ++i)
    if (!is_finite_d(R[i])) return fail(c, LSGCPD_EINVAL, "R must be finite");
  for (int i = 0; i < 3; ++i)
    if (!is_finite_d(t[i])) return fail(c, LSGCPD_EINVAL, "t must be finite");
  if (!plan_fits({N}, {M})) return fail(c, LSGCPD_EINVAL, kTooLarge);
  LSG_CUDA(enter(c, stream), "stream");
  const bool tc = p->precision == 2;
  const BatchPlan plan = plan_batch({N}, {M}, c->num_sms, tc ? 4 : 0);
  lsgcpd_status rs = reserve(c, plan, 0, 1, false, tc);
  if (rs != LSGCPD_OK) return rs;
  cudaStream_t s = c->stream;
  const Dev d = dev_of(c);
  LSG_CUDA(upload_plan(c, plan, s), "plan");
  LSG_CUDA(cudaMemsetAsync(c->status, 0, sizeof(int), s), "memset");
  LSG_CUDA(check_finite(X, N * 3, c->status, s), "check");
  LSG_CUDA(check_finite(Y, M * 3, c->status, s), "check");
  LSG_CUDA(check_finite(normals, M * 3, c->status, s), "check");
  LSG_CUDA(check_finite(alpha, M, c->status, s), "check");
  int64_t launches = 10;
  if (p->phi_x) {
    LSG_CUDA(check_conf(p->phi_x, N, c->status, s), "check");
    ++launches;
  }
  if (p->phi_y) {
    LSG_CUDA(check_conf(p->phi_y, M, c->status, s), "check");
    ++launches;
  }
  const DevParams dp = dev_params(p);
  LSG_CUDA(launch_init(plan, d, X, Y, p->phi_x, p->phi_y, dp, false, c->red.p, c->xs.p, s), "center");
  LSG_CUDA(launch_estep_constants(c->st.p, sigma2, p->w, volume, R, t, s), "constants");
  LSG_CUDA(launch_pack(plan, d, Y, p->phi_y, normals, alpha, p->include_alpha_norm, c->rec.p, c->yl.p, s), "pack");
  if (tc) {
    LSG_CUDA(launch_features(plan, c->rec.p, c->yl.p, c->feat.p, s), "features");
    ++launches;
  }
  const int cfx = p->phi_x ? 1 : 0;
  const int mode = (p->include_alpha_norm || p->phi_x || p->phi_y || p->precision == 1)
                       ? 1
                       : choose_mode(p->w, sigma2, volume, M, 0.0);
  const int half = p->precision == 1 ? 1 : 0;  // the dense posteriors of precision 2 are FP32
  if (c->timing) LSG_CUDA(cudaEventRecord(c->t_begin, s), "event");
  LSG_CUDA(launch_prescale(plan, d, c->yl.p, mode, c->rec.p, s), "prescale");
  if (mode == 1) {
    LSG_CUDA(launch_shift(plan, d, c->xs.p, c->rec.p, cfx, c->part.p, c->status, c->ls_n.p, c->gam_n.p, s), "shift");
    launches += 2;
  }
  LSG_CUDA(estep_launch(c, plan, d, mode, p->precision, s), "estep");
  if (c->timing) LSG_CUDA(cudaEventRecord(c->t_prep, s), "event");
  float* pn = per_n;
  if (P && !pn) {
    LSG_CUDA(ensure(c->pern_tmp, static_cast<size_t>(N) * LSGCPD_PER_N_WIDTH), "alloc");
    pn = c->pern_tmp.p;
  }
  LSG_CUDA(launch_combine(plan, d, c->xs.p, c->part.p, mode, cfx, c->ls_n.p, c->gam_n.p, c->rows.p, pn, s),
           "combine");
  if (P) {
    LSG_CUDA(launch_posteriors(c->xs.p, c->rec.p, c->st.p, c->ls_n.p, mode, half, pn, N, M, P, s), "posteriors");
    ++launches;
  }
  LSG_CUDA(launch_final_reduce(plan, d, c->rows.p, c->mom.p, s), "reduce");
  launches += 3;
  if (c->timing) LSG_CUDA(cudaEventRecord(c->t_end, s), "event");
  double mom[LSGCPD_MOMENTS];
  EmState hs;
  int status = 0;
  LSG_CUDA(cudaMemcpyAsync(mom, c->mom.p, sizeof(mom), cudaMemcpyDeviceToHost, s), "copy");
  LSG_CUDA(cudaMemcpyAsync(&hs, c->st.p, sizeof(EmState), cudaMemcpyDeviceToHost, s), "copy");
  LSG_CUDA(cudaMemcpyAsync(&status, c->status, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
  LSG_CUDA(cudaStreamSynchronize(s), "sync");
  LSG_CUDA(leave(c, stream), "stream");
  c->launches = launches;
  if (c->timing) {
    const double a = elapsed_ms(c->t_begin, c->t_prep);
    const double b = elapsed_ms(c->t_prep, c->t_end);
    c->last_timing[0] = a + b;
    c->last_timing[1] = a;
    c->last_timing[2] = b;
    c->last_timing[3] = 0;
    c->last_timing[4] = 0;
  }
  if (status & 8) return fail(c, LSGCPD_EINVAL, "inputs contain NaN or Inf");
  if (status & 16) return fail(c, LSGCPD_EINVAL, "confidences must lie in (0, 1]");
  if (status & kStatusTimeout) return fail(c, LSGCPD_ETIMEOUT, "E-step tile wait timed out");
  if (moments) moments_to_raw(mom, hs.mu_x, moments);
  return LSGCPD_OK;
}

}  // namespace

extern "C" {

lsgcpd_status lsgcpd_estep(lsgcpd_ctx* c, const float* X, int64_t N, const float* Y, const float* normals,
                           const float* alpha, int64_t M, const lsgcpd_params* p, const double R[9], const double t[3],
                           double sigma2, double volume, double* moments, float* per_n, void* stream) {
  return estep_impl(c, X, N, Y, normals, alpha, M, p, R, t, sigma2, volume, moments, per_n, nullptr, stream);
}

lsgcpd_status lsgcpd_posteriors(lsgcpd_ctx* c, const float* X, int64_t N, const float* Y, const float* normals,
                                const float* alpha, int64_t M, const lsgcpd_params* p, const double R[9],
                                const double t[3], double sigma2, double volume, float* P, void* stream) {
  if (!c) return LSGCPD_EINVAL;
  if (!P) return fail(c, LSGCPD_EINVAL, "P is NULL");
  if (N > 0 && M > 0 && static_cast<double>(N) * static_cast<double>(M + 1) > 4.0e9)
    return fail(c, LSGCPD_EINVAL, "(M + 1) N above 4e9: the dense posteriors are for small problems");
  return estep_impl(c, X, N, Y, normals, alpha, M, p, R, t, sigma2, volume, nullptr, nullptr, P, stream);
}

lsgcpd_status lsgcpd_mstep(lsgcpd_ctx* c, const double* moments, const double R[9], const double t[3],
                           const lsgcpd_params* p, double R_out[9], double t_out[3], double* sigma2_out, int32_t* info,
                           void* stream) {
  if (!c) return LSGCPD_EINVAL;
  c->err.clear();
  if (!moments || !R || !t || !R_out || !t_out) return fail(c, LSGCPD_EINVAL, "NULL argument");
  lsgcpd_status ps = check_params(c, p);
  if (ps != LSGCPD_OK) return ps;
  for (int i = 0; i < LSGCPD_MOMENTS; ++i)
    if (!is_finite_d(moments[i])) return fail(c, LSGCPD_EINVAL, "moments must be finite");
  LSG_CUDA(enter(c, stream), "stream");
  cudaStream_t s = c->stream;
  double host[128];
  memset(host, 0, sizeof(host));
  // io layout: [0..75] moments, [80..91] pose, [96..112] results
  memcpy(host, moments, sizeof(double) * LSGCPD_MOMENTS);
  memcpy(host + 80, R, sizeof(double) * 9);
  memcpy(host + 89, t, sizeof(double) * 3);
  LSG_CUDA(cudaMemcpyAsync(c->io.p, host, sizeof(host), cudaMemcpyHostToDevice, s), "copy");
  DevParams dp = dev_params(p);
  LSG_CUDA(launch_mstep_standalone(c->io.p, dp, s), "mstep");
  LSG_CUDA(cudaMemcpyAsync(host, c->io.p, sizeof(host), cudaMemcpyDeviceToHost, s), "copy");
  LSG_CUDA(cudaStreamSynchronize(s), "sync");
  LSG_CUDA(leave(c, stream), "stream");
  c->launches = 1;
  const double* r = host + 96;
  memcpy(R_out, r, sizeof(double) * 9);
  memcpy(t_out, r + 9, sizeof(double) * 3);
  if (sigma2_out) *sigma2_out = r[12];
  if (info) {
    info[0] = static_cast<int32_t>(r[14]);
    info[1] = static_cast<int32_t>(r[15]);
    info[2] = static_cast<int32_t>(r[16]);
    info[3] = 0;
  }
  return moments[0] > 0.0 ? LSGCPD_OK : fail(c, LSGCPD_ENUMERIC, "N_P is zero");
}

lsgcpd_status lsgcpd_register(lsgcpd_ctx* c, const float* X, int64_t N, const float* Y, int64_t M,
                              const lsgcpd_params* p, lsgcpd_result* out, double* trace, void* stream) {
  if (!c) return LSGCPD_EINVAL;
  c->err.clear();
  if (!X || !Y || !out) return fail(c, LSGCPD_EINVAL, "NULL argument");
  if (N < 1 || M < 1) return fail(c, LSGCPD_EINVAL, "N and M must be >= 1");
  lsgcpd_status ps = check_params(c, p);
  if (ps != LSGCPD_OK) return ps;
  const int k = p->knn_k;
  if (k < 1 || k > kMaxK || k > M) return fail(c, LSGCPD_EINVAL, "knn_k must satisfy 1 <= k <= min(M, 32)");
  double s2 = 0;
  int32_t iters = 0, mode = 0;
  lsgcpd_status rs = run_registration(c, X, Y, {N}, {M}, p, out->R, out->t, &s2, &iters, &mode, trace, stream);
  out->sigma2 = s2;
  out->iters = iters;
  out->mode = mode;
  out->ms_estep = c->timing ? c->last_timing[1] : 0.0;
  out->ms_total = c->timing ? c->last_timing[0] : 0.0;
  return rs;
}

lsgcpd_status lsgcpd_register_batch(lsgcpd_ctx* c, int32_t num_pairs, const float* X, const int64_t* n_off,
                                    const float* Y, const int64_t* m_off, const lsgcpd_params* p, double* R_out,
                                    double* t_out, double* sigma2_out, int32_t* iters_out, double* trace,
                                    void* stream) {
  if (!c) return LSGCPD_EINVAL;
  c->err.clear();
  if (num_pairs < 1 || num_pairs > LSGCPD_MAX_PAIRS) return fail(c, LSGCPD_EINVAL, "num_pairs out of range");
  if (!X || !Y || !n_off || !m_off || !R_out || !t_out) return fail(c, LSGCPD_EINVAL, "NULL argument");
  lsgcpd_status ps = check_params(c, p);
  if (ps != LSGCPD_OK) return ps;
  const int k = p->knn_k;
  if (k < 1 || k > kMaxK) return fail(c, LSGCPD_EINVAL, "knn_k must satisfy 1 <= k <= 32");
  if (n_off[0] != 0 || m_off[0] != 0) return fail(c, LSGCPD_EINVAL, "offsets must start at 0");
  std::vector<long long> N(num_pairs), M(num_pairs);
  for (int i = 0; i < num_pairs; ++i) {
    N[i] = n_off[i + 1] - n_off[i];
    M[i] = m_off[i + 1] - m_off[i];
    if (N[i] < 1 || M[i] < 1) return fail(c, LSGCPD_EINVAL, "every pair needs N >= 1 and M >= 1");
  }
  return run_registration(c, X, Y, N, M, p, R_out, t_out, sigma2_out, iters_out, nullptr, trace, stream);
}

}  // extern "C"
