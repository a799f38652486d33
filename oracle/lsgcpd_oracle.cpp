// LSG-CPD oracle: a plain, slow, FP64 CPU restatement of the method of
// "LSG-CPD: Coherent Point Drift with Local Surface Geometry for Point Cloud
// Registration" (Liu, Wu, Chirikjian, ICCV 2021).
//
// TEST INFRASTRUCTURE ONLY.  This file is the correctness reference for the
// CUDA library; only the test suite, the smoke check and the CPU-baseline leg
// of the benchmark may load it.  It shares no code with the CUDA path.
//
// Every function states the passage of the paper it follows.  Where the paper
// is silent or ambiguous the reading used is stated beside the code:
//   R1  Eq. (9) as printed: c_m = (2 pi sigma^2)^(-3/2) with no sqrt(1+alpha_m)
//       factor, unless include_alpha_norm (then c_m is the Gaussian constant of
//       the anisotropic covariance of Eq. (2)).
//   R2  p_o = 1/V everywhere (Eq. (9) uses a constant gamma).
//   R3  V = volume of the target's axis-aligned bounding box, each side clamped
//       below at 1e-2 of the box diagonal, unless the caller gives V.
//   R4  sigma^2 starts at the CPD value sum ||g0(x_n) - y_m||^2 / (3 N M).
//   R5  neighbourhood = k nearest targets (self included), ties to the lower
//       index; distance decisions in FP32 with a fixed operation order
//       (the same decision the GPU takes).  Covariance about the neighbourhood
//       mean with factor 1/k.  Zero trace -> kappa = 1/3, n = (0,0,1).
//   R6  Newton (Eq. (13)) is iterated with P fixed: xi = -(H_s)^(-1) grad with
//       H_s = (H + H^T)/2, until ||xi|| < newton_tol or newton_max steps.  If
//       H_s is not positive definite it is damped by mu I, mu starting at
//       1e-6 tr(H_s)/6 and growing x10.  A step that raises Q is halved (up to
//       10 times); if none lowers Q the inner loop stops.
//   R7  sigma^2 = sum_mn P_mn d_mn(g_new) / (3 sum_mn P_mn) (dQ/dsigma^2 = 0 of
//       Eq. (6)), floored at 1e-10 * diag^2; reaching the floor ends the EM loop.
//   R8  The M-step objective is Q_d(g) = sum_mn P_mn d_mn(g) with
//       d_mn = (z_n - y_m)^T (I + alpha_m n_m n_m^T)(z_n - y_m); it differs from
//       Eq. (6) by the factor 1/(2 sigma^2) and a constant, which changes neither
//       the Newton step nor its minimiser.  Gradient and Hessian follow Eqs.
//       (11)-(12) with the same scaling.
//   R9  se(3) basis order: E1..E3 rotations about x, y, z; E4..E6 translations.
//   R14 Outlier weight from the outlier ratio eta (Sec. 3.2): w0 = w_max =
//       eta V S / ((1 - eta) + eta V S), S = sum_m pi(m) c_m, with c_m the peak
//       of component m (R1) evaluated once, at sigma^2_0.
//   R15 Confidence filtering (Sec. 3.3): pi(m) = phi(y_m) / sum phi(y),
//       w_n = 1 - (1 - w0) phi(x_n); truncation removes the points with
//       phi < threshold from X and Y before anything else (neighbourhoods,
//       sigma^2_0, V and the priors are those of the kept points).
//   R16 Termination on the log-likelihood (Eq. (4)): after the E step of an
//       iteration i >= 1, if |NLL_i - NLL_{i-1}| <= nll_tol |NLL_i| the M step of
//       that iteration still runs and EM stops.
//
// Build:  g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared -pthread
// (-ffp-contract=off keeps every product separately rounded, so the only fused
// operations are the explicit fmaf calls of the kNN distance.)
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

namespace {

constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// small dense helpers (3x3 row-major, vectors of 3)
// ---------------------------------------------------------------------------
struct V3 {
  double x, y, z;
};
inline V3 v3(double a, double b, double c) { return V3{a, b, c}; }
inline V3 operator+(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
inline V3 operator-(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
inline V3 operator*(double s, V3 a) { return v3(s * a.x, s * a.y, s * a.z); }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
  return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
inline double comp(V3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }
inline V3 unit(int i) { return v3(i == 0, i == 1, i == 2); }

struct M3 {
  double a[9];
};
inline V3 mul(const M3& R, V3 v) {
  return v3(R.a[0] * v.x + R.a[1] * v.y + R.a[2] * v.z, R.a[3] * v.x + R.a[4] * v.y + R.a[5] * v.z,
            R.a[6] * v.x + R.a[7] * v.y + R.a[8] * v.z);
}
inline M3 mul(const M3& A, const M3& B) {
  M3 C;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += A.a[3 * i + k] * B.a[3 * k + j];
      C.a[3 * i + j] = s;
    }
  return C;
}
inline M3 load_m3(const double* p) {
  M3 m;
  std::memcpy(m.a, p, sizeof(m.a));
  return m;
}

// Rigid transform g = (R, t): g(x) = R x + t.
struct Rigid {
  M3 R;
  V3 t;
};
inline V3 apply(const Rigid& g, V3 x) { return mul(g.R, x) + g.t; }
inline Rigid compose(const Rigid& a, const Rigid& b) {  // (a o b)(x) = a(b(x))
  return Rigid{mul(a.R, b.R), mul(a.R, b.t) + a.t};
}

int thread_count(int requested) {
  if (requested > 0) return requested;
  unsigned h = std::thread::hardware_concurrency();
  return h ? static_cast<int>(h) : 1;
}

template <class F>
void parallel_for(int64_t n, int threads, F f) {
  threads = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(threads, std::max<int64_t>(n, 1))));
  if (threads == 1) {
    f(0, n, 0);
    return;
  }
  std::vector<std::thread> pool;
  for (int w = 0; w < threads; ++w) {
    int64_t lo = n * w / threads, hi = n * (w + 1) / threads;
    pool.emplace_back([=] { f(lo, hi, w); });
  }
  for (auto& th : pool) th.join();
}

// ---------------------------------------------------------------------------
// se(3) exponential (closed form, Murray, Li and Sastry), xi = (omega, v)
// ---------------------------------------------------------------------------
Rigid se3_exp(const double xi[6]) {
  V3 w = v3(xi[0], xi[1], xi[2]);
  V3 v = v3(xi[3], xi[4], xi[5]);
  double th2 = dot(w, w);
  double th = std::sqrt(th2);
  double A, B, C;  // sin(th)/th, (1-cos th)/th^2, (th - sin th)/th^3
  if (th < 1e-4) {
    A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
    B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
    C = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
  } else {
    A = std::sin(th) / th;
    B = (1.0 - std::cos(th)) / th2;
    C = (th - std::sin(th)) / (th2 * th);
  }
  // W = [w]_x ; W2 = W W
  double W[9] = {0, -w.z, w.y, w.z, 0, -w.x, -w.y, w.x, 0};
  double W2[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += W[3 * i + k] * W[3 * k + j];
      W2[3 * i + j] = s;
    }
  Rigid g;
  M3 Vm;
  for (int i = 0; i < 9; ++i) {
    double I = (i % 4 == 0) ? 1.0 : 0.0;
    g.R.a[i] = I + A * W[i] + B * W2[i];
    Vm.a[i] = I + B * W[i] + C * W2[i];
  }
  g.t = mul(Vm, v);
  return g;
}

// ---------------------------------------------------------------------------
// Cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix (textbook method).
// Returns eigenvalues ascending and the matching unit eigenvectors (columns).
// ---------------------------------------------------------------------------
void jacobi3(const double Cin[9], double evals[3], double evecs[9]) {
  double a[3][3], v[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      a[i][j] = 0.5 * (Cin[3 * i + j] + Cin[3 * j + i]);
      v[i][j] = (i == j) ? 1.0 : 0.0;
    }
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    double diag = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
    if (off == 0.0 || off <= 1e-34 * diag) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (a[p][q] == 0.0) continue;
        // rotation angle that zeroes a[p][q]
        double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0);
        double s = t * c;
        for (int k = 0; k < 3; ++k) {  // A <- A J (columns p, q)
          double akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - s * akq;
          a[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {  // A <- J^T A (rows p, q)
          double apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - s * aqk;
          a[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {  // V <- V J
          double vkp = v[k][p], vkq = v[k][q];
          v[k][p] = c * vkp - s * vkq;
          v[k][q] = s * vkp + c * vkq;
        }
        a[p][q] = a[q][p] = 0.0;  // annihilated by construction
      }
  }
  int order[3] = {0, 1, 2};
  std::sort(order, order + 3, [&](int i, int j) { return a[i][i] < a[j][j]; });
  for (int c = 0; c < 3; ++c) {
    evals[c] = a[order[c]][order[c]];
    for (int r = 0; r < 3; ++r) evecs[3 * r + c] = v[r][order[c]];
  }
}

// Eq. (3): alpha = alpha_max (1 - exp(lambda (3 - 1/kappa))) / (1 + exp(lambda (3 - 1/kappa))).
double penalty_from_kappa(double kappa, double alpha_max, double lambda) {
  if (kappa <= 0.0) return alpha_max;  // 1/kappa -> infinity: exp(-inf) = 0
  double e = std::exp(lambda * (3.0 - 1.0 / kappa));
  double a = alpha_max * (1.0 - e) / (1.0 + e);
  return a < 0.0 ? 0.0 : a;  // kappa <= 1/3 up to rounding
}

// ---------------------------------------------------------------------------
// Per-source sufficient statistics of the E step (absolute form in y):
//   Pbar = sum_m P_mn, ybar = sum_m P y_m, W = sum_m P alpha n n^T,
//   b = sum_m P alpha (n.y) n, f = sum_m P (|y|^2 + alpha (n.y)^2).
// With A = Pbar I + W and e = ybar + b:  sum_m P_mn d_mn(z) = z^T A z - 2 e^T z + f.
// Layout per source (15 doubles): Pbar, ybar[3], W00 W01 W02 W11 W12 W22, b[3], f, Pout
// ---------------------------------------------------------------------------
constexpr int kStat = 15;

struct SrcStat {
  double A[9];
  V3 e;
  double f, Pbar;
};

SrcStat unpack_stat(const double* s) {
  SrcStat q;
  q.Pbar = s[0];
  double W[6] = {s[4], s[5], s[6], s[7], s[8], s[9]};
  q.A[0] = s[0] + W[0];
  q.A[1] = W[1];
  q.A[2] = W[2];
  q.A[3] = W[1];
  q.A[4] = s[0] + W[3];
  q.A[5] = W[4];
  q.A[6] = W[2];
  q.A[7] = W[4];
  q.A[8] = s[0] + W[5];
  q.e = v3(s[1] + s[10], s[2] + s[11], s[3] + s[12]);
  q.f = s[13];
  return q;
}

inline V3 mulA(const double A[9], V3 v) {
  return v3(A[0] * v.x + A[1] * v.y + A[2] * v.z, A[3] * v.x + A[4] * v.y + A[5] * v.z,
            A[6] * v.x + A[7] * v.y + A[8] * v.z);
}

// Q_d(g) = sum_n (z^T A z - 2 e^T z + f), z = g(x_n)   (reading R8)
double objective(const std::vector<SrcStat>& st, const std::vector<V3>& X, const Rigid& g) {
  double Q = 0.0;
  for (size_t n = 0; n < X.size(); ++n) {
    V3 z = apply(g, X[n]);
    Q += dot(z, mulA(st[n].A, z)) - 2.0 * dot(st[n].e, z) + st[n].f;
  }
  return Q;
}

// (E_i x~)_{1:3}: rotations give e_i x x, translations give e_i.
inline V3 gen_apply(int i, V3 x) { return i < 3 ? cross(unit(i), x) : unit(i - 3); }
// (E_j E_i x~)_{1:3}: E_i x~ = [u; 0];  E_j [u; 0] = [e_j x u; 0] for a rotation j, 0 otherwise.
inline V3 gen2_apply(int j, int i, V3 x) {
  if (j >= 3) return v3(0, 0, 0);
  return cross(unit(j), gen_apply(i, x));
}

// Eqs. (11)-(12) from the per-source statistics: with r_n = A_n z_n - e_n
// (= sum_m P_mn Lambda_m (z_n - y_m)), J_{n,i} = R (E_i x~_n)_{1:3}:
//   grad_i = 2 sum_n r_n^T J_{n,i}
//   H_ij   = 2 sum_n [ J_{n,j}^T A_n J_{n,i} + r_n^T R (E_j E_i x~_n)_{1:3} ]
void grad_hess(const std::vector<SrcStat>& st, const std::vector<V3>& X, const Rigid& g,
               double grad[6], double H[36]) {
  for (int i = 0; i < 6; ++i) grad[i] = 0.0;
  for (int i = 0; i < 36; ++i) H[i] = 0.0;
  for (size_t n = 0; n < X.size(); ++n) {
    V3 z = apply(g, X[n]);
    V3 r = mulA(st[n].A, z) - st[n].e;
    V3 J[6], AJ[6];
    for (int i = 0; i < 6; ++i) {
      J[i] = mul(g.R, gen_apply(i, X[n]));
      AJ[i] = mulA(st[n].A, J[i]);
    }
    for (int i = 0; i < 6; ++i) {
      grad[i] += 2.0 * dot(r, J[i]);
      for (int j = 0; j < 6; ++j) {
        double h = dot(J[j], AJ[i]) + dot(r, mul(g.R, gen2_apply(j, i, X[n])));
        H[6 * i + j] += 2.0 * h;
      }
    }
  }
}

// Cholesky solve of the symmetric 6x6 S x = b; returns false if S is not positive definite.
bool chol_solve6(const double S[36], const double b[6], double x[6]) {
  double L[36] = {0};
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = S[6 * i + j];
      for (int k = 0; k < j; ++k) s -= L[6 * i + k] * L[6 * j + k];
      if (i == j) {
        if (!(s > 0.0)) return false;
        L[6 * i + i] = std::sqrt(s);
      } else {
        L[6 * i + j] = s / L[6 * j + j];
      }
    }
  double y[6];
  for (int i = 0; i < 6; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[6 * i + k] * y[k];
    y[i] = s / L[6 * i + i];
  }
  for (int i = 5; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < 6; ++k) s -= L[6 * k + i] * x[k];
    x[i] = s / L[6 * i + i];
  }
  return true;
}

struct MStepOut {
  Rigid g;
  double Q;
  int newton_iters;
  int damped;
  int halvings;
};

// Newton on SE(3) with P fixed (Eq. (13), readings R6, R9).
MStepOut mstep(const std::vector<SrcStat>& st, const std::vector<V3>& X, const Rigid& g0,
               int newton_max, double newton_tol) {
  MStepOut o{g0, objective(st, X, g0), 0, 0, 0};
  for (int it = 0; it < newton_max; ++it) {
    double grad[6], H[36], Hs[36];
    grad_hess(st, X, o.g, grad, H);
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) Hs[6 * i + j] = 0.5 * (H[6 * i + j] + H[6 * j + i]);
    double minus_grad[6], xi[6];
    for (int i = 0; i < 6; ++i) minus_grad[i] = -grad[i];
    if (!chol_solve6(Hs, minus_grad, xi)) {
      double tr = 0;
      for (int i = 0; i < 6; ++i) tr += std::fabs(Hs[7 * i]);
      double mu = 1e-6 * (tr > 0 ? tr / 6.0 : 1.0);
      bool ok = false;
      for (int k = 0; k < 40 && !ok; ++k, mu *= 10.0) {
        double D[36];
        std::memcpy(D, Hs, sizeof(D));
        for (int i = 0; i < 6; ++i) D[7 * i] += mu;
        ok = chol_solve6(D, minus_grad, xi);
      }
      ++o.damped;
      if (!ok) break;
    }
    ++o.newton_iters;
    double step = 1.0;
    bool accepted = false;
    double nx = 0;
    for (int bt = 0; bt <= 10; ++bt, step *= 0.5) {
      double s[6];
      for (int i = 0; i < 6; ++i) s[i] = step * xi[i];
      Rigid cand = compose(o.g, se3_exp(s));
      double Qc = objective(st, X, cand);
      if (Qc <= o.Q) {
        o.g = cand;
        o.Q = Qc;
        accepted = true;
        nx = 0;
        for (int i = 0; i < 6; ++i) nx += s[i] * s[i];
        nx = std::sqrt(nx);
        break;
      }
      ++o.halvings;
    }
    if (!accepted || nx < newton_tol) break;
  }
  return o;
}

std::vector<V3> to_v3(const float* P, int64_t n) {
  std::vector<V3> out(static_cast<size_t>(n));
  for (int64_t i = 0; i < n; ++i) out[i] = v3(P[3 * i], P[3 * i + 1], P[3 * i + 2]);
  return out;
}

}  // namespace

extern "C" {

// Parameters of a registration (mirrors the CUDA library's parameter block in
// meaning; it is declared here separately).
struct oracle_params {
  double w;             // outlier weight w0 in [0, 1) of Eq. (1)
  double alpha_max;     // Eq. (3)
  double lambda;        // Eq. (3)
  double tol;           // EM stop on the per-iteration motion; 0 = run max_iters
  double volume;        // V of the outlier density; <= 0 -> reading R3
  double sigma2_init;   // <= 0 -> reading R4
  double init_R[9];
  double init_t[3];
  double newton_tol;    // reading R6
  double sigma2_floor_rel;  // reading R7
  int32_t knn_k;
  int32_t max_iters;
  int32_t include_alpha_norm;  // reading R1
  int32_t newton_max;
  int32_t threads;      // 0 = all hardware threads
  int32_t pad_;
  double eta;           // > 0: w0 = w_max of Sec. 3.2 at sigma^2_0 (reading R14); else w
  double cf_threshold;  // Sec. 3.3 truncation: points with phi < cf_threshold are dropped (R15)
  double nll_tol;       // > 0: stop when the NLL of Eq. (4) changes by <= nll_tol relative (R16)
  const float* phi_x;   // confidence phi of every source (Sec. 3.3), NULL = 1
  const float* phi_y;   // confidence phi of every target, NULL = 1
};

// --- kNN (reading R5): k nearest targets of every target, FP32 distance decisions.
int oracle_knn(const float* Y, int64_t M, int32_t k, int32_t threads, int32_t* idx) {
  if (M <= 0 || k <= 0 || k > M) return 1;
  parallel_for(M, thread_count(threads), [&](int64_t lo, int64_t hi, int) {
    std::vector<std::pair<float, int32_t>> d(static_cast<size_t>(M));
    for (int64_t q = lo; q < hi; ++q) {
      float qx = Y[3 * q], qy = Y[3 * q + 1], qz = Y[3 * q + 2];
      for (int64_t m = 0; m < M; ++m) {
        float dx = qx - Y[3 * m], dy = qy - Y[3 * m + 1], dz = qz - Y[3 * m + 2];
        float s = std::fmaf(dz, dz, std::fmaf(dy, dy, dx * dx));
        d[m] = {s, static_cast<int32_t>(m)};
      }
      std::partial_sort(d.begin(), d.begin() + k, d.end());  // (distance, index) order
      for (int j = 0; j < k; ++j) idx[q * k + j] = d[j].second;
    }
  });
  return 0;
}

// Brute-force k nearest targets of the listed queries only (rows of oracle_knn).
int oracle_knn_subset(const float* Y, int64_t M, const int64_t* queries, int64_t nq, int32_t k, int32_t threads,
                      int32_t* idx) {
  if (M <= 0 || k <= 0 || k > M || nq < 0) return 1;
  for (int64_t i = 0; i < nq; ++i)
    if (queries[i] < 0 || queries[i] >= M) return 1;
  parallel_for(nq, thread_count(threads), [&](int64_t lo, int64_t hi, int) {
    std::vector<std::pair<float, int32_t>> d(static_cast<size_t>(M));
    for (int64_t i = lo; i < hi; ++i) {
      const int64_t q = queries[i];
      float qx = Y[3 * q], qy = Y[3 * q + 1], qz = Y[3 * q + 2];
      for (int64_t m = 0; m < M; ++m) {
        float dx = qx - Y[3 * m], dy = qy - Y[3 * m + 1], dz = qz - Y[3 * m + 2];
        d[m] = {std::fmaf(dz, dz, std::fmaf(dy, dy, dx * dx)), static_cast<int32_t>(m)};
      }
      std::partial_sort(d.begin(), d.begin() + k, d.end());
      for (int j = 0; j < k; ++j) idx[i * k + j] = d[j].second;
    }
  });
  return 0;
}

// The same k nearest neighbours as oracle_knn (same FP32 distances, same
// (distance, index) order), found through a uniform grid so that clouds of
// 10^5..10^6 points finish in seconds.  Cells are visited in growing cubic
// shells around the query's cell; the search stops once the k-th distance is
// below the squared distance from the query to the boundary of the visited
// cube (with a relative margin of 1e-5, far above FP32 rounding of a squared
// distance), so every point that could enter or tie the list was examined.
int oracle_knn_grid(const float* Y, int64_t M, int32_t k, int32_t threads, int32_t* idx) {
  if (M <= 0 || k <= 0 || k > M) return 1;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t m = 0; m < M; ++m)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], static_cast<double>(Y[3 * m + a]));
      hi[a] = std::max(hi[a], static_cast<double>(Y[3 * m + a]));
    }
  double diag = 0;
  for (int a = 0; a < 3; ++a) diag += (hi[a] - lo[a]) * (hi[a] - lo[a]);
  diag = std::sqrt(diag);
  // cell edge for about k points per cell on a surface-like cloud; at most 256 cells per axis
  double h = diag * std::sqrt(static_cast<double>(k) / static_cast<double>(M));
  int64_t dim[3];
  for (int pass = 0; pass < 64; ++pass) {
    bool ok = true;
    for (int a = 0; a < 3; ++a) {
      dim[a] = h > 0 ? static_cast<int64_t>(std::floor((hi[a] - lo[a]) / h)) + 1 : 1;
      if (dim[a] > 256) ok = false;
    }
    if (ok) break;
    h *= 1.5;
  }
  if (!(h > 0)) h = 1.0;
  const int64_t ncell = dim[0] * dim[1] * dim[2];
  auto cell_of = [&](double v, int a) {
    int64_t c = static_cast<int64_t>(std::floor((v - lo[a]) / h));
    return std::min<int64_t>(std::max<int64_t>(c, 0), dim[a] - 1);
  };
  std::vector<int64_t> start(static_cast<size_t>(ncell + 1), 0);
  std::vector<int64_t> cid(static_cast<size_t>(M));
  for (int64_t m = 0; m < M; ++m) {
    cid[m] = (cell_of(Y[3 * m + 2], 2) * dim[1] + cell_of(Y[3 * m + 1], 1)) * dim[0] + cell_of(Y[3 * m], 0);
    ++start[cid[m] + 1];
  }
  for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
  std::vector<int32_t> order(static_cast<size_t>(M));
  {
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for (int64_t m = 0; m < M; ++m) order[fill[cid[m]]++] = static_cast<int32_t>(m);
  }
  parallel_for(M, thread_count(threads), [&](int64_t q0, int64_t q1, int) {
    std::vector<std::pair<float, int32_t>> best;
    for (int64_t q = q0; q < q1; ++q) {
      const float qx = Y[3 * q], qy = Y[3 * q + 1], qz = Y[3 * q + 2];
      const int64_t c[3] = {cell_of(qx, 0), cell_of(qy, 1), cell_of(qz, 2)};
      best.clear();
      for (int64_t r = 0;; ++r) {
        for (int64_t z = c[2] - r; z <= c[2] + r; ++z) {
          if (z < 0 || z >= dim[2]) continue;
          for (int64_t y = c[1] - r; y <= c[1] + r; ++y) {
            if (y < 0 || y >= dim[1]) continue;
            for (int64_t x = c[0] - r; x <= c[0] + r; ++x) {
              if (x < 0 || x >= dim[0]) continue;
              const bool shell = std::llabs(z - c[2]) == r || std::llabs(y - c[1]) == r || std::llabs(x - c[0]) == r;
              if (!shell) continue;
              const int64_t cc = (z * dim[1] + y) * dim[0] + x;
              for (int64_t j = start[cc]; j < start[cc + 1]; ++j) {
                const int32_t m = order[j];
                float dx = qx - Y[3 * m], dy = qy - Y[3 * m + 1], dz = qz - Y[3 * m + 2];
                best.push_back({std::fmaf(dz, dz, std::fmaf(dy, dy, dx * dx)), m});
              }
            }
          }
        }
        const bool all = c[0] - r <= 0 && c[1] - r <= 0 && c[2] - r <= 0 && c[0] + r >= dim[0] - 1 &&
                         c[1] + r >= dim[1] - 1 && c[2] + r >= dim[2] - 1;
        if (static_cast<int64_t>(best.size()) >= k) {
          std::partial_sort(best.begin(), best.begin() + k, best.end());
          best.resize(static_cast<size_t>(k));
          // distance from the query to the boundary of the visited cube of cells
          double bound = 1e300;
          const double qv[3] = {qx, qy, qz};
          for (int a = 0; a < 3; ++a) {
            if (c[a] - r > 0) bound = std::min(bound, qv[a] - (lo[a] + (c[a] - r) * h));
            if (c[a] + r < dim[a] - 1) bound = std::min(bound, (lo[a] + (c[a] + r + 1) * h) - qv[a]);
          }
          if (all || (bound > 0 && static_cast<double>(best[k - 1].first) < bound * bound * (1.0 - 1e-5))) break;
        } else if (all) {
          break;
        }
      }
      for (int j = 0; j < k; ++j) idx[q * k + j] = best[j].second;
    }
  });
  return 0;
}

// Eigen-decomposition exposed for the tests (ascending eigenvalues, eigenvectors in columns).
void oracle_jacobi3(const double* C, double* evals, double* evecs) { jacobi3(C, evals, evecs); }

double oracle_penalty(double kappa, double alpha_max, double lambda) {
  return penalty_from_kappa(kappa, alpha_max, lambda);
}

// --- Local surface geometry (Sec. 3.1, Eqs. (2)-(3), reading R5): for every target,
// the neighbourhood covariance, its smallest eigenpair, the surface variation
// kappa = lambda_min / trace and the penalty alpha of Eq. (3).
int oracle_local_geometry(const float* Y, int64_t M, const int32_t* idx, int32_t k,
                          double alpha_max, double lambda, double* normals, double* kappa,
                          double* alpha) {
  if (M <= 0 || k <= 0) return 1;
  for (int64_t m = 0; m < M; ++m) {
    V3 mean = v3(0, 0, 0);
    for (int j = 0; j < k; ++j) {
      int64_t q = idx[m * k + j];
      mean = mean + v3(Y[3 * q], Y[3 * q + 1], Y[3 * q + 2]);
    }
    mean = (1.0 / k) * mean;
    double C[9] = {0};
    for (int j = 0; j < k; ++j) {
      int64_t q = idx[m * k + j];
      V3 d = v3(Y[3 * q], Y[3 * q + 1], Y[3 * q + 2]) - mean;
      double dv[3] = {d.x, d.y, d.z};
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) C[3 * r + c] += dv[r] * dv[c] / k;
    }
    double ev[3], vec[9];
    jacobi3(C, ev, vec);
    double l0 = std::max(ev[0], 0.0), l1 = std::max(ev[1], 0.0), l2 = std::max(ev[2], 0.0);
    double tr = l0 + l1 + l2;
    double kap;
    V3 nrm;
    if (tr > 0.0) {
      kap = l0 / tr;
      nrm = v3(vec[0], vec[3], vec[6]);
    } else {
      kap = 1.0 / 3.0;
      nrm = v3(0, 0, 1);
    }
    normals[3 * m] = nrm.x;
    normals[3 * m + 1] = nrm.y;
    normals[3 * m + 2] = nrm.z;
    kappa[m] = kap;
    alpha[m] = penalty_from_kappa(kap, alpha_max, lambda);
  }
  return 0;
}

// --- Volume of the working space (reading R3) and the target box diagonal.
double oracle_volume(const float* Y, int64_t M, double* diag_out) {
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t m = 0; m < M; ++m)
    for (int c = 0; c < 3; ++c) {
      lo[c] = std::min(lo[c], static_cast<double>(Y[3 * m + c]));
      hi[c] = std::max(hi[c], static_cast<double>(Y[3 * m + c]));
    }
  double s[3], diag2 = 0;
  for (int c = 0; c < 3; ++c) {
    s[c] = hi[c] - lo[c];
    diag2 += s[c] * s[c];
  }
  double diag = std::sqrt(diag2);
  if (diag_out) *diag_out = diag;
  double V = 1.0;
  for (int c = 0; c < 3; ++c) V *= std::max(s[c], 1e-2 * diag);
  return V;
}

// --- sigma^2 start value (reading R4), closed form
//   (M sum|z|^2 + N sum|y|^2 - 2 (sum z).(sum y)) / (3 N M),  z = R x + t.
double oracle_sigma2_init(const float* X, int64_t N, const float* Y, int64_t M, const double* R,
                          const double* t) {
  Rigid g{load_m3(R), v3(t[0], t[1], t[2])};
  double zz = 0, yy = 0;
  V3 sz = v3(0, 0, 0), sy = v3(0, 0, 0);
  for (int64_t n = 0; n < N; ++n) {
    V3 z = apply(g, v3(X[3 * n], X[3 * n + 1], X[3 * n + 2]));
    zz += dot(z, z);
    sz = sz + z;
  }
  for (int64_t m = 0; m < M; ++m) {
    V3 y = v3(Y[3 * m], Y[3 * m + 1], Y[3 * m + 2]);
    yy += dot(y, y);
    sy = sy + y;
  }
  return (M * zz + N * yy - 2.0 * dot(sz, sy)) / (3.0 * N * M);
}

// --- E step (Eq. (5) with the mixture of Eq. (1) and the component density of
// Eq. (2)), by Bayes' rule in the log domain:
//   l_mn = log((1 - w_n) pi_m c_m) - d_mn / (2 sigma^2),  l_on = log(w_n p_o),
//   P_mn = exp(l_mn - LSE_n),  P_on = exp(l_on - LSE_n),  -log p(z_n) = -LSE_n,
// with c_m from reading R1 and p_o = 1/V (reading R2).
// Outputs: stats [N x 15] (see kStat layout), optional dense P [M x N], optional
// negative log-likelihood of Eq. (4) at (g, sigma^2).
int oracle_estep(const float* X, int64_t N, const float* Y, int64_t M, const double* normals,
                 const double* alpha, const double* pi_m, const double* w_n, double w, double V,
                 const double* R, const double* t, double sigma2, int32_t include_alpha_norm,
                 int32_t threads, double* stats, double* P_dense, double* nll_out) {
  if (N <= 0 || M <= 0 || !(sigma2 > 0) || !(V > 0)) return 1;
  Rigid g{load_m3(R), v3(t[0], t[1], t[2])};
  std::vector<V3> Yv = to_v3(Y, M);
  std::vector<V3> Nv(static_cast<size_t>(M));
  std::vector<double> logpc(static_cast<size_t>(M));
  for (int64_t m = 0; m < M; ++m) {
    Nv[m] = v3(normals[3 * m], normals[3 * m + 1], normals[3 * m + 2]);
    double pi = pi_m ? pi_m[m] : 1.0 / static_cast<double>(M);
    double logc = -1.5 * std::log(2.0 * kPi * sigma2);
    if (include_alpha_norm) logc += 0.5 * std::log(1.0 + alpha[m]);
    logpc[m] = std::log(pi) + logc;
  }
  int T = thread_count(threads);
  std::vector<double> nll_part(static_cast<size_t>(T), 0.0);
  parallel_for(N, T, [&](int64_t lo, int64_t hi, int wid) {
    std::vector<double> l(static_cast<size_t>(M));
    double nll = 0.0;
    for (int64_t n = lo; n < hi; ++n) {
      double wn = w_n ? w_n[n] : w;
      V3 z = apply(g, v3(X[3 * n], X[3 * n + 1], X[3 * n + 2]));
      double lmax = -std::numeric_limits<double>::infinity();
      for (int64_t m = 0; m < M; ++m) {
        V3 r = z - Yv[m];
        double s = dot(Nv[m], r);
        double d = dot(r, r) + alpha[m] * s * s;
        l[m] = std::log(1.0 - wn) + logpc[m] - d / (2.0 * sigma2);
        lmax = std::max(lmax, l[m]);
      }
      double lo_ = (wn > 0.0) ? std::log(wn / V) : -std::numeric_limits<double>::infinity();
      lmax = std::max(lmax, lo_);
      double sum = (wn > 0.0) ? std::exp(lo_ - lmax) : 0.0;
      for (int64_t m = 0; m < M; ++m) sum += std::exp(l[m] - lmax);
      double lse = lmax + std::log(sum);
      nll -= lse;
      double* s = stats + n * kStat;
      for (int c = 0; c < kStat; ++c) s[c] = 0.0;
      for (int64_t m = 0; m < M; ++m) {
        double P = std::exp(l[m] - lse);
        if (P_dense) P_dense[m * N + n] = P;
        V3 y = Yv[m];
        V3 nm = Nv[m];
        double am = alpha[m];
        double ny = dot(nm, y);
        s[0] += P;
        s[1] += P * y.x;
        s[2] += P * y.y;
        s[3] += P * y.z;
        s[4] += P * am * nm.x * nm.x;
        s[5] += P * am * nm.x * nm.y;
        s[6] += P * am * nm.x * nm.z;
        s[7] += P * am * nm.y * nm.y;
        s[8] += P * am * nm.y * nm.z;
        s[9] += P * am * nm.z * nm.z;
        s[10] += P * am * ny * nm.x;
        s[11] += P * am * ny * nm.y;
        s[12] += P * am * ny * nm.z;
        s[13] += P * (dot(y, y) + am * ny * ny);
      }
      s[14] = (wn > 0.0) ? std::exp(lo_ - lse) : 0.0;
    }
    nll_part[wid] = nll;
  });
  if (nll_out) {
    double s = 0;
    for (double v : nll_part) s += v;
    *nll_out = s;
  }
  return 0;
}

// --- Q_d(g) of reading R8 from the per-source statistics.
double oracle_objective(const double* stats, const float* X, int64_t N, const double* R,
                        const double* t) {
  std::vector<SrcStat> st(static_cast<size_t>(N));
  for (int64_t n = 0; n < N; ++n) st[n] = unpack_stat(stats + n * kStat);
  return objective(st, to_v3(X, N), Rigid{load_m3(R), v3(t[0], t[1], t[2])});
}

// --- Gradient and (asymmetric) Hessian of Eqs. (11)-(12) from the statistics (reading R8).
void oracle_grad_hess(const double* stats, const float* X, int64_t N, const double* R,
                      const double* t, double* grad, double* H) {
  std::vector<SrcStat> st(static_cast<size_t>(N));
  for (int64_t n = 0; n < N; ++n) st[n] = unpack_stat(stats + n * kStat);
  grad_hess(st, to_v3(X, N), Rigid{load_m3(R), v3(t[0], t[1], t[2])}, grad, H);
}

// --- Eqs. (11)-(12) evaluated literally as double sums over (m, n) with 4x4
// homogeneous matrices g~, E_i, x~, y~ and Sigma~^{-1} = Sigma^{-1} (+) 0, where
// Sigma_m^{-1} = (alpha_m n_m n_m^T + I) / sigma^2 (Eq. (2)).  For small inputs only.
void oracle_grad_hess_direct(const float* X, int64_t N, const float* Y, int64_t M,
                             const double* normals, const double* alpha, const double* P,
                             const double* R, const double* t, double sigma2, double* grad,
                             double* H) {
  double g4[16] = {R[0], R[1], R[2], t[0], R[3], R[4], R[5], t[1],
                   R[6], R[7], R[8], t[2], 0, 0, 0, 1};
  double E[6][16];
  for (int i = 0; i < 6; ++i) {
    for (int c = 0; c < 16; ++c) E[i][c] = 0.0;
    if (i < 3) {  // [e_i]_x in the top-left block
      int a = (i + 1) % 3, b = (i + 2) % 3;
      E[i][4 * b + a] = 1.0;
      E[i][4 * a + b] = -1.0;
    } else {
      E[i][4 * (i - 3) + 3] = 1.0;
    }
  }
  auto mv4 = [](const double* A, const double* x, double* y) {
    for (int r = 0; r < 4; ++r) {
      double s = 0;
      for (int c = 0; c < 4; ++c) s += A[4 * r + c] * x[c];
      y[r] = s;
    }
  };
  for (int i = 0; i < 6; ++i) grad[i] = 0.0;
  for (int i = 0; i < 36; ++i) H[i] = 0.0;
  for (int64_t m = 0; m < M; ++m) {
    double S[16] = {0};
    const double* nm = normals + 3 * m;
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) S[4 * r + c] = (alpha[m] * nm[r] * nm[c] + (r == c)) / sigma2;
    double yt[4] = {Y[3 * m], Y[3 * m + 1], Y[3 * m + 2], 1.0};
    for (int64_t n = 0; n < N; ++n) {
      double p = P[m * N + n];
      double xt[4] = {X[3 * n], X[3 * n + 1], X[3 * n + 2], 1.0};
      double gx[4], diff[4], Sd[4];
      mv4(g4, xt, gx);
      for (int r = 0; r < 4; ++r) diff[r] = gx[r] - yt[r];
      mv4(S, diff, Sd);  // Sigma~^{-1} (g~x~ - y~) (symmetric Sigma~^{-1})
      double Ex[6][4], gEx[6][4], SgEx[6][4];
      for (int i = 0; i < 6; ++i) {
        mv4(E[i], xt, Ex[i]);
        mv4(g4, Ex[i], gEx[i]);
        mv4(S, gEx[i], SgEx[i]);
      }
      for (int i = 0; i < 6; ++i) {
        double gi = 0;
        for (int r = 0; r < 4; ++r) gi += Sd[r] * gEx[i][r];
        grad[i] += 2.0 * p * gi;
        for (int j = 0; j < 6; ++j) {
          double EjEix[4], gEjEix[4];
          mv4(E[j], Ex[i], EjEix);
          mv4(g4, EjEix, gEjEix);
          double h1 = 0, h2 = 0;
          for (int r = 0; r < 4; ++r) {
            h1 += gEx[j][r] * SgEx[i][r];
            h2 += Sd[r] * gEjEix[r];
          }
          H[6 * i + j] += 2.0 * p * (h1 + h2);
        }
      }
    }
  }
}

// --- se(3) exponential exposed for the tests: T = [[R, t], [0, 1]] row-major 4x4.
void oracle_se3_exp(const double* xi, double* T) {
  Rigid g = se3_exp(xi);
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) T[4 * r + c] = g.R.a[3 * r + c];
    T[4 * r + 3] = comp(g.t, r);
  }
  T[12] = T[13] = T[14] = 0.0;
  T[15] = 1.0;
}

// --- M step: Newton on SE(3) with P fixed (Eq. (13), readings R6, R8), then the
// sigma^2 update (reading R7, without the floor).  info = {newton_iters, damped, halvings}.
int oracle_mstep(const double* stats, const float* X, int64_t N, const double* R_in,
                 const double* t_in, int32_t newton_max, double newton_tol, double* R_out,
                 double* t_out, double* sigma2_out, double* Q_out, int32_t* info) {
  if (N <= 0) return 1;
  std::vector<SrcStat> st(static_cast<size_t>(N));
  double NP = 0;
  for (int64_t n = 0; n < N; ++n) {
    st[n] = unpack_stat(stats + n * kStat);
    NP += st[n].Pbar;
  }
  std::vector<V3> Xv = to_v3(X, N);
  MStepOut o = mstep(st, Xv, Rigid{load_m3(R_in), v3(t_in[0], t_in[1], t_in[2])}, newton_max,
                     newton_tol);
  std::memcpy(R_out, o.g.R.a, sizeof(double) * 9);
  t_out[0] = o.g.t.x;
  t_out[1] = o.g.t.y;
  t_out[2] = o.g.t.z;
  if (Q_out) *Q_out = o.Q;
  if (sigma2_out) *sigma2_out = NP > 0 ? o.Q / (3.0 * NP) : 0.0;
  if (info) {
    info[0] = o.newton_iters;
    info[1] = o.damped;
    info[2] = o.halvings;
  }
  return NP > 0 ? 0 : 2;
}

// --- Full registration (Sec. 3): preprocessing of the target, then EM iterations
// E step -> Newton M step -> sigma^2 update.  Per-iteration trace (8 doubles):
// sigma2 after the update, N_P, Q_d(g_new), newton_iters, damped, motion, NLL at
// the E step, outlier mass.  Returns 0, or 2 if N_P vanished.
// Sec. 3.2 (reading R14): the largest outlier weight for which the expected
// number of outliers, with every component density at its peak c_m, does not
// exceed eta N.  pi_m NULL = uniform 1/M.
double oracle_w_from_eta(double eta, double V, double sigma2, const double* alpha, const double* pi_m, int64_t M,
                         int32_t include_alpha_norm) {
  if (!(eta > 0.0)) return 0.0;
  if (!(eta < 1.0)) return 1.0;
  double S = 0.0;
  const double c0 = std::pow(2.0 * kPi * sigma2, -1.5);
  for (int64_t m = 0; m < M; ++m) {
    double pi = pi_m ? pi_m[m] : 1.0 / static_cast<double>(M);
    double c = c0 * (include_alpha_norm ? std::sqrt(1.0 + alpha[m]) : 1.0);
    S += pi * c;
  }
  const double a = eta * V * S;
  return a / ((1.0 - eta) + a);
}

int oracle_register(const float* X, int64_t N, const float* Y, int64_t M, const oracle_params* p,
                    double* R_out, double* t_out, double* sigma2_out, int32_t* iters_out,
                    double* trace, double* normals_out, double* alpha_out) {
  if (N <= 0 || M <= 0 || p->knn_k <= 0 || !(p->w >= 0.0 && p->w < 1.0) || !(p->eta >= 0.0 && p->eta < 1.0))
    return 1;
  // confidence truncation (Sec. 3.3, reading R15): keep the points with phi >= threshold
  std::vector<float> Xk, Yk;
  std::vector<double> phx, phy;
  std::vector<int64_t> ykeep;
  for (int64_t n = 0; n < N; ++n) {
    const double ph = p->phi_x ? p->phi_x[n] : 1.0;
    if (p->phi_x && p->cf_threshold > 0 && ph < p->cf_threshold) continue;
    for (int c = 0; c < 3; ++c) Xk.push_back(X[3 * n + c]);
    phx.push_back(ph);
  }
  for (int64_t m = 0; m < M; ++m) {
    const double ph = p->phi_y ? p->phi_y[m] : 1.0;
    if (p->phi_y && p->cf_threshold > 0 && ph < p->cf_threshold) continue;
    for (int c = 0; c < 3; ++c) Yk.push_back(Y[3 * m + c]);
    phy.push_back(ph);
    ykeep.push_back(m);
  }
  const int64_t M_all = M;
  N = static_cast<int64_t>(phx.size());
  M = static_cast<int64_t>(phy.size());
  X = Xk.data();
  Y = Yk.data();
  if (N <= 0 || M <= 0 || p->knn_k > M) return 1;
  int k = p->knn_k;
  std::vector<int32_t> idx(static_cast<size_t>(M * k));
  if (M > 20000)
    oracle_knn_grid(Y, M, k, p->threads, idx.data());
  else
    oracle_knn(Y, M, k, p->threads, idx.data());
  std::vector<double> nrm(static_cast<size_t>(3 * M)), kap(static_cast<size_t>(M)),
      alp(static_cast<size_t>(M));
  oracle_local_geometry(Y, M, idx.data(), k, p->alpha_max, p->lambda, nrm.data(), kap.data(),
                        alp.data());
  // outputs in the caller's target indexing; truncated targets get NaN
  for (int64_t m = 0; m < M_all && (normals_out || alpha_out); ++m) {
    if (normals_out) normals_out[3 * m] = normals_out[3 * m + 1] = normals_out[3 * m + 2] = std::nan("");
    if (alpha_out) alpha_out[m] = std::nan("");
  }
  for (int64_t j = 0; j < M; ++j) {
    if (normals_out)
      for (int c = 0; c < 3; ++c) normals_out[3 * ykeep[j] + c] = nrm[3 * j + c];
    if (alpha_out) alpha_out[ykeep[j]] = alp[j];
  }
  double diag = 0;
  double Vbox = oracle_volume(Y, M, &diag);
  double V = p->volume > 0 ? p->volume : Vbox;
  Rigid g{load_m3(p->init_R), v3(p->init_t[0], p->init_t[1], p->init_t[2])};
  double sigma2 = p->sigma2_init > 0 ? p->sigma2_init
                                     : oracle_sigma2_init(X, N, Y, M, p->init_R, p->init_t);
  double floor = p->sigma2_floor_rel * diag * diag;
  // priors and outlier weights (Secs. 3.2-3.3)
  std::vector<double> pim, wn;
  if (p->phi_y) {
    double sum = 0;
    for (double v : phy) sum += v;
    for (double v : phy) pim.push_back(v / sum);
  }
  const double w0 = p->eta > 0 ? oracle_w_from_eta(p->eta, V, sigma2, alp.data(), p->phi_y ? pim.data() : nullptr, M,
                                                   p->include_alpha_norm)
                               : p->w;
  if (p->phi_x)
    for (double v : phx) wn.push_back(1.0 - (1.0 - w0) * v);
  double nll_prev = 0;
  std::vector<double> stats(static_cast<size_t>(N * kStat));
  std::vector<V3> Xv = to_v3(X, N);
  int it = 0;
  int rc = 0;
  for (; it < p->max_iters; ++it) {
    double nll = 0;
    oracle_estep(X, N, Y, M, nrm.data(), alp.data(), p->phi_y ? pim.data() : nullptr,
                 p->phi_x ? wn.data() : nullptr, w0, V, g.R.a, &g.t.x, sigma2, p->include_alpha_norm,
                 p->threads, stats.data(), nullptr, &nll);
    const bool nll_stop = p->nll_tol > 0 && it > 0 && std::fabs(nll - nll_prev) <= p->nll_tol * std::fabs(nll);
    nll_prev = nll;
    std::vector<SrcStat> st(static_cast<size_t>(N));
    double NP = 0, Pout = 0;
    for (int64_t n = 0; n < N; ++n) {
      st[n] = unpack_stat(stats.data() + n * kStat);
      NP += st[n].Pbar;
      Pout += stats[n * kStat + 14];
    }
    if (!(NP > 0)) {
      rc = 2;
      break;
    }
    MStepOut o = mstep(st, Xv, g, p->newton_max, p->newton_tol);
    // motion of this iteration: rotation angle and translation / diag of g_old^{-1} g_new
    M3 dR;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s = 0;
        for (int c = 0; c < 3; ++c) s += g.R.a[3 * c + i] * o.g.R.a[3 * c + j];
        dR.a[3 * i + j] = s;
      }
    double fro = 0;
    for (int i = 0; i < 9; ++i) {
      double d = dR.a[i] - ((i % 4 == 0) ? 1.0 : 0.0);
      fro += d * d;
    }
    double ang = 2.0 * std::asin(std::min(1.0, std::sqrt(fro) / (2.0 * std::sqrt(2.0))));
    V3 dt = o.g.t - g.t;
    double motion = std::max(ang, std::sqrt(dot(dt, dt)) / (diag > 0 ? diag : 1.0));
    g = o.g;
    double s2 = o.Q / (3.0 * NP);
    bool at_floor = !(s2 > floor);
    sigma2 = at_floor ? floor : s2;
    if (trace) {
      double* tr = trace + 8 * it;
      tr[0] = sigma2;
      tr[1] = NP;
      tr[2] = o.Q;
      tr[3] = o.newton_iters;
      tr[4] = o.damped;
      tr[5] = motion;
      tr[6] = nll;
      tr[7] = Pout;
    }
    if (at_floor || nll_stop || (p->tol > 0 && motion < p->tol)) {
      ++it;
      break;
    }
  }
  std::memcpy(R_out, g.R.a, sizeof(double) * 9);
  t_out[0] = g.t.x;
  t_out[1] = g.t.y;
  t_out[2] = g.t.z;
  *sigma2_out = sigma2;
  *iters_out = it;
  return rc;
}

}  // extern "C"
