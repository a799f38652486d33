// lsgcpd_estep_noalloc: the E step of lsgcpd_estep with every piece of scratch
// memory taken from one fixed, file-scope device array instead of a context.
//
// Some callers cannot allocate device memory when they call us: code that runs
// while another framework owns the device memory pool (its caching allocator
// holds the memory, and a cudaMalloc of ours could fail or fragment it),
// latency-critical loops where cudaMalloc / cudaFree would synchronise the
// device, and embedded integrations that must keep a fixed, known footprint.
// This entry point needs no context (creating one allocates) and never calls
// cudaMalloc, cudaFree or any allocating library routine.  The price is a fixed
// size limit and a shared arena (see the declaration in lsgcpd.h).
#include <math.h>
#include <string.h>

#include <mutex>

#include "internal.cuh"
#include "lsgcpd.h"

namespace {

// The scratch arena.  Every GPU that loads the library holds it until the
// process exits.  Its size is stated in lsgcpd.h (LSGCPD_NOALLOC_ARENA_BYTES).
constexpr size_t kArenaBytes = static_cast<size_t>(LSGCPD_NOALLOC_ARENA_BYTES);
static __device__ __align__(256) unsigned char g_noalloc_arena[kArenaBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_arena_ptr[kMaxDevices] = {nullptr};

// Device address of the arena on the current device; looked up once per device.
cudaError_t arena_address(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_arena_ptr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_arena);
    if (e != cudaSuccess) return e;
    g_arena_ptr[device] = p;
  }
  *out = static_cast<unsigned char*>(g_arena_ptr[device]);
  return cudaSuccess;
}

size_t align256(size_t n) { return (n + 255) & ~static_cast<size_t>(255); }

// Carve the arena; returns false if the problem does not fit.
struct Carve {
  lsg::EmState* st;
  int* status;
  int* done_count;
  int* tab;
  long long* off64;
  double* red;
  double* rows;
  double* mom;
  float4* xs;
  float4* yl;
  float* rec;
  float* ls;
  float* gam;
  float* part;
};

bool carve(unsigned char* base, const lsg::BatchPlan& p, Carve* c) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* q = base + off;
    off += align256(bytes);
    return q;
  };
  const lsg::Geo& g = p.g;
  const size_t n_pad = static_cast<size_t>(g.B) * g.SB;
  const size_t m_pad = static_cast<size_t>(g.T) * lsg::kTile;
  c->st = reinterpret_cast<lsg::EmState*>(take(sizeof(lsg::EmState)));
  c->status = reinterpret_cast<int*>(take(sizeof(int)));
  c->done_count = reinterpret_cast<int*>(take(sizeof(int)));
  c->tab = reinterpret_cast<int*>(take(sizeof(int) * p.tab.size()));
  c->off64 = reinterpret_cast<long long*>(take(sizeof(long long) * p.off64.size()));
  c->red = reinterpret_cast<double*>(take(sizeof(double) * static_cast<size_t>(lsg::stats_chunks(g)) * 24));
  c->rows = reinterpret_cast<double*>(take(sizeof(double) * static_cast<size_t>(g.combine_ctas) * lsg::kGlob));
  c->mom = reinterpret_cast<double*>(take(sizeof(double) * lsg::kGlob));
  c->xs = reinterpret_cast<float4*>(take(sizeof(float4) * n_pad));
  c->rec = reinterpret_cast<float*>(take(sizeof(float) * m_pad * lsg::kPlanes));
  c->yl = reinterpret_cast<float4*>(take(sizeof(float4) * m_pad));
  c->ls = reinterpret_cast<float*>(take(sizeof(float) * n_pad));
  c->gam = reinterpret_cast<float*>(take(sizeof(float) * n_pad));
  c->part = reinterpret_cast<float*>(take(sizeof(float) * lsg::estep_partial_floats(g)));
  return off <= kArenaBytes;
}

// Moments of the centred working frame -> the caller's frame (xt_raw = T xt_c,
// T = [[I, mu_x], [0, 1]]).
void to_caller_frame(const double* mc, const double mu[3], double* mr) {
  for (int j = 0; j < LSGCPD_MOMENTS; ++j) mr[j] = mc[j];
  const double T[4][4] = {{1, 0, 0, mu[0]}, {0, 1, 0, mu[1]}, {0, 0, 1, mu[2]}, {0, 0, 0, 1}};
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
  for (int p = 0; p < 6; ++p)
    for (int k = 0; k < 4; ++k)
      for (int l = k; l < 4; ++l) {
        double s = 0;
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) s += T[k][a] * T[l][b] * mc[14 + p * 10 + pidx[a][b]];
        mr[14 + p * 10 + pidx[k][l]] = s;
      }
}

bool finite_d(double v) { return isfinite(v) != 0; }

}  // namespace

extern "C" lsgcpd_status lsgcpd_estep_noalloc(const float* X, int64_t N, const float* Y, const float* normals,
                                              const float* alpha, int64_t M, const lsgcpd_params* p,
                                              const double R[9], const double t[3], double sigma2, double volume,
                                              double* moments, float* per_n, void* stream) {
  if (!X || !Y || !normals || !alpha || !R || !t || !p || !moments) return LSGCPD_EINVAL;
  if (N < 1 || M < 1 || N > LSGCPD_NOALLOC_MAX_N || M > LSGCPD_NOALLOC_MAX_M) return LSGCPD_EINVAL;
  if (!(p->w >= 0.0 && p->w < 1.0) || p->precision != 0) return LSGCPD_EINVAL;  // FP32 only
  if (!(sigma2 > 0.0) || !finite_d(sigma2) || !(volume > 0.0) || !finite_d(volume)) return LSGCPD_EINVAL;
  for (int i = 0; i < 9; ++i)
    if (!finite_d(R[i])) return LSGCPD_EINVAL;
  for (int i = 0; i < 3; ++i)
    if (!finite_d(t[i])) return LSGCPD_EINVAL;
  int device = 0, sms = 0;
  if (cudaGetDevice(&device) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    return LSGCPD_ECUDA;
  }
  unsigned char* base = nullptr;
  if (arena_address(device, &base) != cudaSuccess) {
    cudaGetLastError();
    return LSGCPD_ECUDA;
  }
  const lsg::BatchPlan plan = lsg::plan_batch({N}, {M}, sms, 0);
  Carve c;
  if (!carve(base, plan, &c)) return LSGCPD_ENOMEM;  // cannot happen within the stated limits
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const lsg::Dev d{c.tab, c.off64, c.st, c.done_count};
  // the arena keeps the previous call's contents: the status word and the
  // finished-pair count must start at zero, everything else below is written
  // before it is read
  cudaError_t e = cudaMemsetAsync(c.status, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.done_count, 0, sizeof(int), s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c.tab, plan.tab.data(), sizeof(int) * plan.tab.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c.off64, plan.off64.data(), sizeof(long long) * plan.off64.size(), cudaMemcpyHostToDevice,
                        s);
  lsg::DevParams dp{};
  dp.w = p->w;
  dp.volume = volume;
  if (e == cudaSuccess) e = lsg::launch_init(plan, d, X, Y, nullptr, nullptr, dp, false, c.red, c.xs, s);
  if (e == cudaSuccess) e = lsg::launch_estep_constants(c.st, sigma2, p->w, volume, R, t, s);
  if (e == cudaSuccess) e = lsg::launch_pack(plan, d, Y, nullptr, normals, alpha, p->include_alpha_norm, c.rec, c.yl, s);
  // fixed shift unless the outlier term is absent, a term could overflow FP32 or l_m varies
  int mode = 1;
  if (p->w > 0.0 && !p->include_alpha_norm) {
    const double L = log2(p->w) - log2(1.0 - p->w) + 1.5 * log2(2.0 * M_PI * sigma2) - log2(volume);
    const double l_max = -log2(static_cast<double>(M));
    mode = (l_max - L + log2(static_cast<double>(M)) + 12.0 < 126.0) ? 0 : 1;
  }
  if (e == cudaSuccess) e = lsg::launch_prescale(plan, d, c.yl, mode, c.rec, s);
  if (e == cudaSuccess && mode == 1) e = lsg::launch_shift(plan, d, c.xs, c.rec, 0, c.part, c.status, c.ls, c.gam, s);
  if (e == cudaSuccess) e = lsg::launch_estep(plan, d, c.xs, c.rec, mode, 0, c.ls, c.part, c.status, s);
  if (e == cudaSuccess) e = lsg::launch_combine(plan, d, c.xs, c.part, mode, 0, c.ls, c.gam, c.rows, per_n, s);
  if (e == cudaSuccess) e = lsg::launch_final_reduce(plan, d, c.rows, c.mom, s);
  double mom[LSGCPD_MOMENTS];
  double mu[3];
  int status = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(mom, c.mom, sizeof(mom), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(mu, reinterpret_cast<unsigned char*>(c.st) + offsetof(lsg::EmState, mu_x), sizeof(mu),
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, c.status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LSGCPD_ECUDA;
  }
  if (status & lsg::kStatusTimeout) return LSGCPD_ETIMEOUT;
  to_caller_frame(mom, mu, moments);
  return LSGCPD_OK;
}
