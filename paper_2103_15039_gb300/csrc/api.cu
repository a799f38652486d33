// C ABI of liblsgcpd (declared in include/lsgcpd.h): context, argument
// validation, scratch memory, the CUDA-graph-captured EM loop and the
// conversions between the centred working frame and the caller's frame.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>

#include "internal.cuh"
#include "lsgcpd.h"

using namespace lsg;

namespace {

constexpr int kMaxK = 32;

struct GraphKey {
  int64_t N = -1, M = -1;
  int iters = -1, mode = -1, S = -1, timing = -1;
  bool operator==(const GraphKey& o) const {
    return N == o.N && M == o.M && iters == o.iters && mode == o.mode && S == o.S && timing == o.timing;
  }
};

template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t cap = 0;  // elements
};

}  // namespace

struct lsgcpd_ctx {
  int device = 0;
  int num_sms = 0;
  std::string err;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  DevBuf<float> X_in, Y_in, rec, part, knn_d, kap_n, gam_n;
  DevBuf<float4> xs, y4;
  DevBuf<int> knn_i, knn_idx, segtab;
  DevBuf<double> rows, red, trace, io;
  EmState* st = nullptr;
  int* status = nullptr;
  // graph of the EM loop
  cudaGraphExec_t gexec = nullptr;
  GraphKey gkey;
  // timing
  int timing = 0;
  cudaEvent_t t_begin = nullptr, t_prep = nullptr, t_end = nullptr;
  cudaEvent_t* t_iter = nullptr;  // 4 per iteration
  int t_iter_cap = 0;
  double last_timing[6] = {0, 0, 0, 0, 0, 0};
  int64_t launches = 0;
  int64_t h2d_bytes = 0, d2h_bytes = 0;
};

namespace {

lsgcpd_status fail(lsgcpd_ctx* c, lsgcpd_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

lsgcpd_status cuda_fail(lsgcpd_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return fail(c, LSGCPD_ECUDA, m);
}

#define LSG_CUDA(call, where)                       \
  do {                                              \
    cudaError_t e_ = (call);                        \
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
  if (!is_finite_d(p->volume) || !is_finite_d(p->sigma2_init)) return fail(c, LSGCPD_EINVAL, "volume/sigma2_init must be finite");
  for (int i = 0; i < 9; ++i)
    if (!is_finite_d(p->init_R[i])) return fail(c, LSGCPD_EINVAL, "init_R must be finite");
  for (int i = 0; i < 3; ++i)
    if (!is_finite_d(p->init_t[i])) return fail(c, LSGCPD_EINVAL, "init_t must be finite");
  if (!is_finite_d(p->newton_tol) || p->newton_tol < 0.0) return fail(c, LSGCPD_EINVAL, "newton_tol must be >= 0");
  if (!is_finite_d(p->sigma2_floor_rel) || p->sigma2_floor_rel < 0.0)
    return fail(c, LSGCPD_EINVAL, "sigma2_floor_rel must be >= 0");
  if (p->max_iters < 0 || p->max_iters > 100000) return fail(c, LSGCPD_EINVAL, "max_iters out of range");
  if (p->newton_max < 1 || p->newton_max > 1000) return fail(c, LSGCPD_EINVAL, "newton_max out of range");
  if (p->precision != 0) return fail(c, LSGCPD_EINVAL, "only precision 0 (FP32 E step) is implemented");
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

// Scratch sizes for a problem (N, M, k) with plan p.
lsgcpd_status reserve(lsgcpd_ctx* c, int64_t N, int64_t M, int k, const EstepPlan& p, int iters,
                      bool host_inputs) {
  const size_t n_pad = static_cast<size_t>(p.num_blocks) * p.SB;
  const size_t m_pad = static_cast<size_t>(p.num_tiles) * kTile;
  const int splits = knn_splits(M, c->num_sms);
  bool grew = false;
  auto grow = [&](auto& buf, size_t n) -> cudaError_t {
    if (buf.cap >= (n ? n : 1)) return cudaSuccess;
    grew = true;
    return ensure(buf, n);
  };
  cudaError_t e = cudaSuccess;
  if (grow(c->xs, n_pad) != cudaSuccess || grow(c->rec, m_pad * kPlanes) != cudaSuccess ||
      grow(c->part, estep_partial_floats(p)) != cudaSuccess ||
      grow(c->rows, static_cast<size_t>(combine_rows(N, c->num_sms)) * kGlob) != cudaSuccess ||
      grow(c->segtab, p.table.size()) != cudaSuccess ||
      grow(c->kap_n, n_pad) != cudaSuccess || grow(c->gam_n, n_pad) != cudaSuccess ||
      grow(c->trace, static_cast<size_t>(iters > 0 ? iters : 1) * LSGCPD_TRACE_WIDTH) != cudaSuccess)
    e = cudaErrorMemoryAllocation;
  if (e == cudaSuccess && k > 0) {
    if (grow(c->y4, static_cast<size_t>(M)) != cudaSuccess ||
        grow(c->knn_d, static_cast<size_t>(splits) * M * k) != cudaSuccess ||
        grow(c->knn_i, static_cast<size_t>(splits) * M * k) != cudaSuccess ||
        grow(c->knn_idx, static_cast<size_t>(M) * k) != cudaSuccess)
      e = cudaErrorMemoryAllocation;
  }
  if (e == cudaSuccess && host_inputs) {
    if (grow(c->X_in, static_cast<size_t>(N) * 3) != cudaSuccess ||
        grow(c->Y_in, static_cast<size_t>(M) * 3) != cudaSuccess)
      e = cudaErrorMemoryAllocation;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, LSGCPD_ENOMEM, "device allocation failed");
  }
  if (grew && c->gexec) {  // buffers moved: the captured graph is stale
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->gkey = GraphKey();
  }
  return LSGCPD_OK;
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
  if (max_N < 1 || max_M < 1) return LSGCPD_EINVAL;
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
      cudaEventCreate(&c->t_end) != cudaSuccess) {
    cudaGetLastError();
    return bail(LSGCPD_ECUDA);
  }
  if (cudaMalloc(&c->st, sizeof(EmState)) != cudaSuccess || cudaMalloc(&c->status, sizeof(int)) != cudaSuccess ||
      ensure(c->red, 1024 * 20) != cudaSuccess || ensure(c->io, 128) != cudaSuccess) {
    cudaGetLastError();
    return bail(LSGCPD_ENOMEM);
  }
  cudaMemset(c->st, 0, sizeof(EmState));
  cudaMemset(c->status, 0, sizeof(int));
  const EstepPlan p = plan_estep(max_N, max_M, c->num_sms, 0);
  if (reserve(c, max_N, max_M, 10, p, 50, false) != LSGCPD_OK) return bail(LSGCPD_ENOMEM);
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
  float* fb[] = {c->X_in.p, c->Y_in.p, c->rec.p, c->part.p, c->knn_d.p, c->kap_n.p, c->gam_n.p};
  for (float* p : fb)
    if (p) cudaFree(p);
  if (c->xs.p) cudaFree(c->xs.p);
  if (c->y4.p) cudaFree(c->y4.p);
  if (c->knn_i.p) cudaFree(c->knn_i.p);
  if (c->knn_idx.p) cudaFree(c->knn_idx.p);
  if (c->segtab.p) cudaFree(c->segtab.p);
  double* db[] = {c->rows.p, c->red.p, c->trace.p, c->io.p};
  for (double* p : db)
    if (p) cudaFree(p);
  if (c->st) cudaFree(c->st);
  if (c->status) cudaFree(c->status);
  if (c->t_iter) {
    for (int i = 0; i < 4 * c->t_iter_cap; ++i) cudaEventDestroy(c->t_iter[i]);
    delete[] c->t_iter;
  }
  cudaEvent_t evs[] = {c->ev_in, c->ev_out, c->t_begin, c->t_prep, c->t_end};
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

lsgcpd_status lsgcpd_last_timing(const lsgcpd_ctx* c, double out[8]) {
  if (!c || !out) return LSGCPD_EINVAL;
  for (int i = 0; i < 5; ++i) out[i] = c->last_timing[i];
  out[5] = static_cast<double>(c->launches);
  out[6] = static_cast<double>(c->h2d_bytes);
  out[7] = static_cast<double>(c->d2h_bytes);
  return c->timing ? LSGCPD_OK : LSGCPD_EINVAL;
}

lsgcpd_status lsgcpd_preprocess(lsgcpd_ctx* c, const float* Y, int64_t M, const lsgcpd_params* p,
                                float* normals, float* kappa, float* alpha, int32_t* knn_idx, void* stream) {
  if (!c) return LSGCPD_EINVAL;
  c->err.clear();
  if (!Y || M < 1) return fail(c, LSGCPD_EINVAL, "Y must be non-NULL with M >= 1");
  lsgcpd_status ps = check_params(c, p);
  if (ps != LSGCPD_OK) return ps;
  const int k = p->knn_k;
  if (k < 1 || k > kMaxK || k > M) return fail(c, LSGCPD_EINVAL, "knn_k must satisfy 1 <= k <= min(M, 32)");
  LSG_CUDA(enter(c, stream), "stream");
  const EstepPlan plan = plan_estep(M, M, c->num_sms, 1);
  lsgcpd_status rs = reserve(c, M, M, k, plan, 1, false);
  if (rs != LSGCPD_OK) return rs;
  cudaStream_t s = c->stream;
  c->launches = 0;
  LSG_CUDA(cudaMemsetAsync(c->status, 0, sizeof(int), s), "memset");
  LSG_CUDA(check_finite(Y, M * 3, c->status, s), "check");
  const int64_t n_pad = static_cast<int64_t>(plan.num_blocks) * plan.SB;
  LSG_CUDA(launch_center_only(Y, M, Y, M, c->red.p, c->st, c->xs.p, n_pad, s), "center");
  const int splits = knn_splits(M, c->num_sms);
  int* idx = knn_idx ? knn_idx : c->knn_idx.p;
  LSG_CUDA(launch_knn(Y, M, k, c->y4.p, c->knn_d.p, c->knn_i.p, idx, splits, s), "knn");
  LSG_CUDA(launch_geometry(Y, M, idx, k, p->alpha_max, p->lambda, p->include_alpha_norm, c->st, c->rec.p,
                           plan.num_tiles, normals, kappa, alpha, s),
           "geometry");
  c->launches = 7;
  int status = 0;
  LSG_CUDA(cudaMemcpyAsync(&status, c->status, sizeof(int), cudaMemcpyDeviceToHost, s), "status");
  LSG_CUDA(cudaStreamSynchronize(s), "sync");
  LSG_CUDA(leave(c, stream), "stream");
  if (status & 8) return fail(c, LSGCPD_EINVAL, "Y contains NaN or Inf");
  return LSGCPD_OK;
}

lsgcpd_status lsgcpd_estep(lsgcpd_ctx* c, const float* X, int64_t N, const float* Y, const float* normals,
                           const float* alpha, int64_t M, const lsgcpd_params* p, const double R[9],
                           const double t[3], double sigma2, double volume, double* moments, float* per_n,
                           void* stream) {
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
  LSG_CUDA(enter(c, stream), "stream");
  const EstepPlan plan = plan_estep(N, M, c->num_sms, 0);
  lsgcpd_status rs = reserve(c, N, M, 0, plan, 1, false);
  if (rs != LSGCPD_OK) return rs;
  cudaStream_t s = c->stream;
  const int64_t n_pad = static_cast<int64_t>(plan.num_blocks) * plan.SB;
  LSG_CUDA(cudaMemsetAsync(c->status, 0, sizeof(int), s), "memset");
  LSG_CUDA(check_finite(X, N * 3, c->status, s), "check");
  LSG_CUDA(check_finite(Y, M * 3, c->status, s), "check");
  LSG_CUDA(check_finite(normals, M * 3, c->status, s), "check");
  LSG_CUDA(check_finite(alpha, M, c->status, s), "check");
  LSG_CUDA(launch_center_only(X, N, Y, M, c->red.p, c->st, c->xs.p, n_pad, s), "center");
  LSG_CUDA(launch_estep_constants(c->st, sigma2, p->w, volume, R, t, s), "constants");
  LSG_CUDA(launch_pack(Y, normals, alpha, M, p->include_alpha_norm, c->st, c->rec.p, plan.num_tiles, s), "pack");
  const int mode = choose_mode(p->w, sigma2, volume, M, p->include_alpha_norm ? 12.0 : 0.0);
  int64_t launches = 11;
  LSG_CUDA(cudaMemcpyAsync(c->segtab.p, plan.table.data(), sizeof(int) * plan.table.size(),
                           cudaMemcpyHostToDevice, s),
           "table");
  const int nrows = combine_rows(N, c->num_sms);
  if (c->timing) LSG_CUDA(cudaEventRecord(c->t_begin, s), "event");
  if (mode == 1) {
    LSG_CUDA(launch_shift(plan, c->xs.p, c->rec.p, c->st, N, c->kap_n.p, c->gam_n.p, s), "shift");
    ++launches;
  }
  LSG_CUDA(launch_estep(plan, c->xs.p, c->rec.p, c->st, mode ? c->kap_n.p : nullptr, c->part.p, c->segtab.p,
                        c->status, s),
           "estep");
  if (c->timing) LSG_CUDA(cudaEventRecord(c->t_prep, s), "event");
  LSG_CUDA(launch_combine(plan, c->xs.p, N, c->part.p, c->segtab.p, c->st, mode ? c->kap_n.p : nullptr,
                          mode ? c->gam_n.p : nullptr, c->rows.p, nrows, per_n, s),
           "combine");
  LSG_CUDA(launch_final_reduce(c->rows.p, nrows, c->io.p, nullptr, s), "reduce");
  launches += 3;
  if (c->timing) LSG_CUDA(cudaEventRecord(c->t_end, s), "event");
  double mom[LSGCPD_MOMENTS];
  EmState hs;
  int status = 0;
  LSG_CUDA(cudaMemcpyAsync(mom, c->io.p, sizeof(mom), cudaMemcpyDeviceToHost, s), "copy");
  LSG_CUDA(cudaMemcpyAsync(&hs, c->st, sizeof(EmState), cudaMemcpyDeviceToHost, s), "copy");
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
  if (status & kStatusTimeout) return fail(c, LSGCPD_ETIMEOUT, "E-step tile wait timed out");
  if (moments) moments_to_raw(mom, hs.mu_x, moments);
  return LSGCPD_OK;
}

lsgcpd_status lsgcpd_mstep(lsgcpd_ctx* c, const double* moments, const double R[9], const double t[3],
                           const lsgcpd_params* p, double R_out[9], double t_out[3], double* sigma2_out,
                           int32_t* info, void* stream) {
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
  LSG_CUDA(enter(c, stream), "stream");
  const bool xd = is_device_ptr(X), yd = is_device_ptr(Y);
  const EstepPlan plan = plan_estep(N, M, c->num_sms, 0);
  const int iters = p->max_iters;
  lsgcpd_status rs = reserve(c, N, M, k, plan, iters, !xd || !yd);
  if (rs != LSGCPD_OK) return rs;
  cudaStream_t s = c->stream;
  if (c->timing) {
    LSG_CUDA(ensure_iter_events(c, iters > 0 ? iters : 1), "events");
    LSG_CUDA(cudaEventRecord(c->t_begin, s), "event");
  }
  const float* Xd = X;
  const float* Yd = Y;
  if (!xd) {
    LSG_CUDA(cudaMemcpyAsync(c->X_in.p, X, sizeof(float) * 3 * N, cudaMemcpyHostToDevice, s), "copy X");
    Xd = c->X_in.p;
  }
  if (!yd) {
    LSG_CUDA(cudaMemcpyAsync(c->Y_in.p, Y, sizeof(float) * 3 * M, cudaMemcpyHostToDevice, s), "copy Y");
    Yd = c->Y_in.p;
  }
  int64_t launches = 0;
  LSG_CUDA(cudaMemsetAsync(c->status, 0, sizeof(int), s), "memset");
  LSG_CUDA(check_finite(Xd, N * 3, c->status, s), "check");
  LSG_CUDA(check_finite(Yd, M * 3, c->status, s), "check");
  const DevParams dp = dev_params(p);
  const int64_t n_pad = static_cast<int64_t>(plan.num_blocks) * plan.SB;
  LSG_CUDA(launch_init(Xd, N, Yd, M, dp, c->red.p, c->st, c->xs.p, n_pad, s), "init");
  const int splits = knn_splits(M, c->num_sms);
  LSG_CUDA(launch_knn(Yd, M, k, c->y4.p, c->knn_d.p, c->knn_i.p, c->knn_idx.p, splits, s), "knn");
  LSG_CUDA(launch_geometry(Yd, M, c->knn_idx.p, k, p->alpha_max, p->lambda, p->include_alpha_norm, c->st,
                           c->rec.p, plan.num_tiles, nullptr, nullptr, nullptr, s),
           "geometry");
  launches += 2 + 4 + 3 + 1;
  if (c->timing) LSG_CUDA(cudaEventRecord(c->t_prep, s), "event");
  EmState hs;
  int status = 0;
  LSG_CUDA(cudaMemcpyAsync(&hs, c->st, sizeof(EmState), cudaMemcpyDeviceToHost, s), "copy");
  LSG_CUDA(cudaMemcpyAsync(&status, c->status, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
  LSG_CUDA(cudaStreamSynchronize(s), "sync");
  if (status & 8) {
    leave(c, stream);
    return fail(c, LSGCPD_EINVAL, "inputs contain NaN or Inf");
  }
  const double l_extra = p->include_alpha_norm ? 0.5 * log2(1.0 + p->alpha_max) : 0.0;
  const int mode = choose_mode(p->w, hs.sigma2_floor, hs.V, M, l_extra);
  const int nrows = combine_rows(N, c->num_sms);
  LSG_CUDA(cudaMemcpyAsync(c->segtab.p, plan.table.data(), sizeof(int) * plan.table.size(),
                           cudaMemcpyHostToDevice, s),
           "table");
  if (iters > 0) {
    GraphKey key;
    key.N = N;
    key.M = M;
    key.iters = iters;
    key.mode = mode;
    key.S = plan.S;
    key.timing = c->timing;
    if (!(c->gexec && key == c->gkey)) {
      if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
      }
      cudaGraph_t g = nullptr;
      LSG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "capture");
      cudaError_t ce = cudaSuccess;
      for (int it = 0; it < iters && ce == cudaSuccess; ++it) {
        if (c->timing) ce = cudaEventRecordWithFlags(c->t_iter[4 * it], s, cudaEventRecordExternal);
        if (ce == cudaSuccess && mode == 1)
          ce = launch_shift(plan, c->xs.p, c->rec.p, c->st, N, c->kap_n.p, c->gam_n.p, s);
        if (ce == cudaSuccess)
          ce = launch_estep(plan, c->xs.p, c->rec.p, c->st, mode ? c->kap_n.p : nullptr, c->part.p,
                            c->segtab.p, c->status, s);
        if (ce == cudaSuccess && c->timing)
          ce = cudaEventRecordWithFlags(c->t_iter[4 * it + 1], s, cudaEventRecordExternal);
        if (ce == cudaSuccess)
          ce = launch_combine(plan, c->xs.p, N, c->part.p, c->segtab.p, c->st, mode ? c->kap_n.p : nullptr,
                              mode ? c->gam_n.p : nullptr, c->rows.p, nrows, nullptr, s);
        if (ce == cudaSuccess) ce = launch_final_reduce(c->rows.p, nrows, c->io.p, c->st, s);
        if (ce == cudaSuccess && c->timing)
          ce = cudaEventRecordWithFlags(c->t_iter[4 * it + 2], s, cudaEventRecordExternal);
        if (ce == cudaSuccess) ce = launch_mstep(c->io.p, c->st, dp, c->trace.p, s);
        if (ce == cudaSuccess && c->timing)
          ce = cudaEventRecordWithFlags(c->t_iter[4 * it + 3], s, cudaEventRecordExternal);
      }
      cudaError_t ee = cudaStreamEndCapture(s, &g);
      if (ce != cudaSuccess || ee != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(c, ce != cudaSuccess ? ce : ee, "graph capture");
      }
      cudaError_t ie = cudaGraphInstantiate(&c->gexec, g, 0);
      cudaGraphDestroy(g);
      if (ie != cudaSuccess) {
        c->gexec = nullptr;
        return cuda_fail(c, ie, "graph instantiate");
      }
      c->gkey = key;
    }
    LSG_CUDA(cudaGraphLaunch(c->gexec, s), "graph launch");
    launches += static_cast<int64_t>(iters) * (mode ? 5 : 4);
  }
  if (c->timing) LSG_CUDA(cudaEventRecord(c->t_end, s), "event");
  LSG_CUDA(cudaMemcpyAsync(&hs, c->st, sizeof(EmState), cudaMemcpyDeviceToHost, s), "copy");
  LSG_CUDA(cudaMemcpyAsync(&status, c->status, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
  if (trace && iters > 0)
    LSG_CUDA(cudaMemcpyAsync(trace, c->trace.p, sizeof(double) * LSGCPD_TRACE_WIDTH * iters,
                             cudaMemcpyDeviceToHost, s),
             "copy trace");
  LSG_CUDA(cudaStreamSynchronize(s), "sync");
  LSG_CUDA(leave(c, stream), "stream");
  c->launches = launches;
  c->h2d_bytes = (xd ? 0 : 12 * N) + (yd ? 0 : 12 * M) + static_cast<int64_t>(sizeof(int) * plan.table.size());
  c->d2h_bytes = 2 * static_cast<int64_t>(sizeof(EmState) + sizeof(int)) +
                 (trace && iters > 0 ? static_cast<int64_t>(sizeof(double)) * LSGCPD_TRACE_WIDTH * iters : 0);
  // result in the caller's frame: t = t_c + mu_y - R mu_x
  for (int i = 0; i < 9; ++i) out->R[i] = hs.R[i];
  for (int i = 0; i < 3; ++i)
    out->t[i] = hs.t[i] + hs.mu_y[i] - (hs.R[3 * i] * hs.mu_x[0] + hs.R[3 * i + 1] * hs.mu_x[1] + hs.R[3 * i + 2] * hs.mu_x[2]);
  out->sigma2 = hs.sigma2;
  out->iters = hs.iter;
  out->mode = mode;
  out->ms_estep = 0;
  out->ms_total = 0;
  if (c->timing) {
    const double tot = elapsed_ms(c->t_begin, c->t_end);
    const double prep = elapsed_ms(c->t_begin, c->t_prep);
    double es = 0, cb = 0, ms = 0;
    for (int it = 0; it < iters; ++it) {
      es += elapsed_ms(c->t_iter[4 * it], c->t_iter[4 * it + 1]);
      cb += elapsed_ms(c->t_iter[4 * it + 1], c->t_iter[4 * it + 2]);
      ms += elapsed_ms(c->t_iter[4 * it + 2], c->t_iter[4 * it + 3]);
    }
    c->last_timing[0] = tot;
    c->last_timing[1] = es;
    c->last_timing[2] = cb;
    c->last_timing[3] = ms;
    c->last_timing[4] = prep;
    out->ms_estep = es;
    out->ms_total = tot;
  }
  if (status & kStatusTimeout) return fail(c, LSGCPD_ETIMEOUT, "E-step tile wait timed out");
  if (hs.numeric_fail) return fail(c, LSGCPD_ENUMERIC, "posterior mass vanished (N_P = 0)");
  return LSGCPD_OK;
}

}  // extern "C"
