// M step of LSG-CPD (Sec. 3.5, Eqs. (11)-(13)) and the sigma^2 update, in FP64,
// from the global moments of one E step.
//
// With the posteriors fixed, sum_m P_mn d_mn is a quadratic function of the
// moved source point, and the moved point z' = g_old Delta x is affine in
// U = [Delta_R - I | Delta_t] (3x4).  Writing x~ = [x; 1],
//   Q_d(Delta) = sum_n D_n + 2 <H1', U> + sum_{i,k,j,l} U_ik U_jl B^{kl}_ij,
//   H1' = R_old^T sum_n h_n x~_n^T,   B^{kl} = R_old^T (sum_n A_n x~_nk x~_nl) R_old,
// exactly (h_n = rho_n + beta_n, A_n = Pbar_n I + W_n).  The Newton iteration
// of Eq. (13) on SE(3) (right perturbation Delta o exp(xi^), basis order
// rotations x, y, z then translations) needs the gradient and the symmetrised
// Hessian (H + H^T)/2 of xi -> Q_d(Delta o exp(xi^)) at xi = 0, which follow
// from the first and second derivatives of U(xi):
//   dU/dw_a = [Delta_R [e_a]x | 0],  dU/dv_a = [0 | Delta_R e_a],
//   d2U/dw_a dw_b = [Delta_R ([e_a]x[e_b]x + [e_b]x[e_a]x)/2 | 0],
//   d2U/dw_a dv_b = [0 | Delta_R [e_a]x e_b / 2].
// So the whole inner Newton loop is O(1) work on 76 numbers, independent of N and M.
// Step rule: xi = -(H_s)^{-1} grad by Cholesky; if H_s is not positive definite
// it is damped by mu I (mu from 1e-6 tr/6, x10); a step that raises Q_d is halved
// up to 10 times; stop when |xi| < newton_tol, after newton_max steps, or when no
// halving lowers Q_d.  sigma^2 = Q_d(g_new) / (3 N_P) (dQ/dsigma^2 = 0 of Eq. (6)).
#include <math.h>

#include "internal.cuh"

namespace lsg {
namespace {

constexpr int kRedThreads = 256;

struct NewtonOut {
  double dR[9], dt[3];
  double Q;
  int iters, damped, halvings;
};

// Q model data
struct QModel {
  double SD;
  double H1[3][4];
  double B[4][4][3][3];  // B[k][l][i][j]
};

__device__ void build_model(const double* mom, const double* Ro, QModel& q) {
  q.SD = mom[1];
  double H1[3][4];
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 4; ++k) H1[i][k] = mom[2 + 4 * i + k];
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 4; ++k) {
      double s = 0;
      for (int a = 0; a < 3; ++a) s += Ro[3 * a + i] * H1[a][k];
      q.H1[i][k] = s;
    }
  // xt pair index of (k, l), k <= l
  int qi = 0;
  for (int k = 0; k < 4; ++k)
    for (int l = k; l < 4; ++l, ++qi) {
      double A[3][3];
      const double* g = mom + 14;  // g[p * 10 + qi], p = (00,01,02,11,12,22)
      A[0][0] = g[0 * 10 + qi];
      A[0][1] = A[1][0] = g[1 * 10 + qi];
      A[0][2] = A[2][0] = g[2 * 10 + qi];
      A[1][1] = g[3 * 10 + qi];
      A[1][2] = A[2][1] = g[4 * 10 + qi];
      A[2][2] = g[5 * 10 + qi];
      double T[3][3], Bm[3][3];
      for (int a = 0; a < 3; ++a)
        for (int j = 0; j < 3; ++j) {
          double s = 0;
          for (int b = 0; b < 3; ++b) s += A[a][b] * Ro[3 * b + j];
          T[a][j] = s;
        }
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          double s = 0;
          for (int a = 0; a < 3; ++a) s += Ro[3 * a + i] * T[a][j];
          Bm[i][j] = s;
        }
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          q.B[k][l][i][j] = Bm[i][j];
          q.B[l][k][i][j] = Bm[i][j];
        }
    }
}

// GU[i][k] = sum_{j,l} B[k][l][i][j] U[j][l]
__device__ void apply_G(const QModel& q, const double U[3][4], double GU[3][4]) {
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 4; ++k) {
      double s = 0;
      for (int j = 0; j < 3; ++j)
        for (int l = 0; l < 4; ++l) s += q.B[k][l][i][j] * U[j][l];
      GU[i][k] = s;
    }
}

__device__ double frob(const double A[3][4], const double B[3][4]) {
  double s = 0;
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 4; ++k) s += A[i][k] * B[i][k];
  return s;
}

__device__ double q_value(const QModel& q, const double U[3][4]) {
  double GU[3][4];
  apply_G(q, U, GU);
  return q.SD + 2.0 * frob(q.H1, U) + frob(U, GU);
}

__device__ void make_U(const double dR[9], const double dt[3], double U[3][4]) {
  for (int i = 0; i < 3; ++i) {
    for (int k = 0; k < 3; ++k) U[i][k] = dR[3 * i + k] - (i == k ? 1.0 : 0.0);
    U[i][3] = dt[i];
  }
}

// hat(e_a) applied: ([e_a]x)[r][c]
__device__ __forceinline__ double hat_e(int a, int r, int c) {
  // [e]_x = [[0,-e2,e1],[e2,0,-e0],[-e1,e0,0]]
  if (a == 0) return (r == 2 && c == 1) ? 1.0 : ((r == 1 && c == 2) ? -1.0 : 0.0);
  if (a == 1) return (r == 0 && c == 2) ? 1.0 : ((r == 2 && c == 0) ? -1.0 : 0.0);
  return (r == 1 && c == 0) ? 1.0 : ((r == 0 && c == 1) ? -1.0 : 0.0);
}

// closed-form exponential of se(3): xi = (w, v) -> (R, t)
__device__ void se3_exp_dev(const double xi[6], double R[9], double t[3]) {
  const double w0 = xi[0], w1 = xi[1], w2 = xi[2];
  const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
  const double th = sqrt(th2);
  double a, b, c;
  if (th < 1e-4) {
    a = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
    b = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
    c = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
  } else {
    const double sn = sin(th), cs = cos(th);
    a = sn / th;
    b = (1.0 - cs) / th2;
    c = (th - sn) / (th2 * th);
  }
  const double K[9] = {0.0, -w2, w1, w2, 0.0, -w0, -w1, w0, 0.0};
  double K2[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      K2[3 * i + j] = K[3 * i] * K[j] + K[3 * i + 1] * K[3 + j] + K[3 * i + 2] * K[6 + j];
  double V[9];
  for (int i = 0; i < 9; ++i) {
    const double I = (i % 4 == 0) ? 1.0 : 0.0;
    R[i] = I + a * K[i] + b * K2[i];
    V[i] = I + b * K[i] + c * K2[i];
  }
  for (int i = 0; i < 3; ++i) t[i] = V[3 * i] * xi[3] + V[3 * i + 1] * xi[4] + V[3 * i + 2] * xi[5];
}

__device__ bool cholesky_solve6(const double S[36], const double b[6], double x[6]) {
  double L[36];
  for (int i = 0; i < 36; ++i) L[i] = 0.0;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = S[6 * i + j];
      for (int k = 0; k < j; ++k) s -= L[6 * i + k] * L[6 * j + k];
      if (i == j) {
        if (!(s > 0.0)) return false;
        L[6 * i + i] = sqrt(s);
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

__device__ void newton(const QModel& q, int newton_max, double newton_tol, NewtonOut& o) {
  for (int i = 0; i < 9; ++i) o.dR[i] = (i % 4 == 0) ? 1.0 : 0.0;
  o.dt[0] = o.dt[1] = o.dt[2] = 0.0;
  o.Q = q.SD;
  o.iters = o.damped = o.halvings = 0;
  for (int it = 0; it < newton_max; ++it) {
    double U[3][4], GU[3][4], M1[3][4];
    make_U(o.dR, o.dt, U);
    apply_G(q, U, GU);
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 4; ++k) M1[i][k] = q.H1[i][k] + GU[i][k];
    double Ua[6][3][4];
    for (int a = 0; a < 6; ++a)
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 4; ++k) {
          double v = 0.0;
          if (a < 3) {
            if (k < 3)
              for (int j = 0; j < 3; ++j) v += o.dR[3 * i + j] * hat_e(a, j, k);
          } else if (k == 3) {
            v = o.dR[3 * i + (a - 3)];
          }
          Ua[a][i][k] = v;
        }
    double grad[6], Hs[36];
    double GUa[6][3][4];
    for (int a = 0; a < 6; ++a) {
      grad[a] = 2.0 * frob(M1, Ua[a]);
      apply_G(q, Ua[a], GUa[a]);
    }
    for (int a = 0; a < 6; ++a)
      for (int b = a; b < 6; ++b) {
        double h = 2.0 * frob(Ua[a], GUa[b]);
        double sec = 0.0;
        if (a < 3 && b < 3) {
          // Delta_R (hat_a hat_b + hat_b hat_a) / 2 in the rotation block
          for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) {
              double s = 0.0;
              for (int j = 0; j < 3; ++j) {
                double Sjk = 0.0;
                for (int m = 0; m < 3; ++m)
                  Sjk += 0.5 * (hat_e(a, j, m) * hat_e(b, m, k) + hat_e(b, j, m) * hat_e(a, m, k));
                s += o.dR[3 * i + j] * Sjk;
              }
              sec += M1[i][k] * s;
            }
        } else if (a < 3 && b >= 3) {
          for (int i = 0; i < 3; ++i) {
            double s = 0.0;
            for (int j = 0; j < 3; ++j) s += o.dR[3 * i + j] * 0.5 * hat_e(a, j, b - 3);
            sec += M1[i][3] * s;
          }
        }
        h += 2.0 * sec;
        Hs[6 * a + b] = h;
        Hs[6 * b + a] = h;
      }
    double mg[6], xi[6];
    for (int a = 0; a < 6; ++a) mg[a] = -grad[a];
    if (!cholesky_solve6(Hs, mg, xi)) {
      double tr = 0.0;
      for (int a = 0; a < 6; ++a) tr += fabs(Hs[7 * a]);
      double mu = 1e-6 * (tr > 0.0 ? tr / 6.0 : 1.0);
      bool ok = false;
      for (int k = 0; k < 40 && !ok; ++k, mu *= 10.0) {
        double D[36];
        for (int e = 0; e < 36; ++e) D[e] = Hs[e];
        for (int a = 0; a < 6; ++a) D[7 * a] += mu;
        ok = cholesky_solve6(D, mg, xi);
      }
      ++o.damped;
      if (!ok) break;
    }
    ++o.iters;
    double step = 1.0;
    bool accepted = false;
    double nx = 0.0;
    for (int bt = 0; bt <= 10; ++bt, step *= 0.5) {
      double s[6], eR[9], et[3], cR[9], ct[3];
      for (int a = 0; a < 6; ++a) s[a] = step * xi[a];
      se3_exp_dev(s, eR, et);
      for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j)
          cR[3 * i + j] = o.dR[3 * i] * eR[j] + o.dR[3 * i + 1] * eR[3 + j] + o.dR[3 * i + 2] * eR[6 + j];
        ct[i] = o.dR[3 * i] * et[0] + o.dR[3 * i + 1] * et[1] + o.dR[3 * i + 2] * et[2] + o.dt[i];
      }
      double Uc[3][4];
      make_U(cR, ct, Uc);
      const double Qc = q_value(q, Uc);
      if (Qc <= o.Q) {
        for (int e = 0; e < 9; ++e) o.dR[e] = cR[e];
        for (int e = 0; e < 3; ++e) o.dt[e] = ct[e];
        o.Q = Qc;
        accepted = true;
        for (int a = 0; a < 6; ++a) nx += s[a] * s[a];
        nx = sqrt(nx);
        break;
      }
      ++o.halvings;
    }
    if (!accepted || nx < newton_tol) break;
  }
}

// Sum the partial moment rows (fixed order: deterministic) into mom[kGlob].
__device__ void reduce_rows(const double* blk, int nblk, double* part /*[8][kGlob]*/, double* mom) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nw = blockDim.x >> 5;
  for (int c = lane; c < kGlob; c += 32) {
    double s = 0.0;
    for (int r = warp; r < nblk; r += nw) s += blk[static_cast<size_t>(r) * kGlob + c];
    part[warp * kGlob + c] = s;
  }
  __syncthreads();
  if (tid < kGlob) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += part[w * kGlob + tid];
    mom[tid] = s;
  }
  __syncthreads();
}

__device__ void set_constants(EmState* st, double w) {
  const double s2 = st->sigma2;
  const double c = 1.4426950408889634 / (2.0 * s2);  // log2(e) / (2 s2)
  const double L = st->log2_wodds + 1.5 * log2(2.0 * 3.14159265358979323846 * s2) - log2(st->V);
  for (int i = 0; i < 9; ++i) st->Rf[i] = static_cast<float>(st->R[i]);
  for (int i = 0; i < 3; ++i) st->tf[i] = static_cast<float>(st->t[i]);
  st->neg_c = static_cast<float>(-c);
  st->L = static_cast<float>(L);
  st->kap = static_cast<float>(L / c);
  st->nll_const = -log1p(-w) + 1.5 * log(2.0 * 3.14159265358979323846 * s2);
}

__global__ void __launch_bounds__(kRedThreads) mstep_em_kernel(const double* __restrict__ blk, int nblk,
                                                                EmState* __restrict__ st, DevParams dp,
                                                                double* __restrict__ trace) {
  __shared__ double part[(kRedThreads / 32) * kGlob];
  __shared__ double mom[kGlob];
  if (st->done) return;
  reduce_rows(blk, nblk, part, mom);
  if (threadIdx.x != 0) return;
  const double NP = mom[0];
  if (!(NP > 0.0)) {
    st->numeric_fail = 1;
    st->done = 1;
    return;
  }
  QModel q;
  build_model(mom, st->R, q);
  NewtonOut o;
  newton(q, dp.newton_max, dp.newton_tol, o);
  double Rn[9], tn[3];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j)
      Rn[3 * i + j] = st->R[3 * i] * o.dR[j] + st->R[3 * i + 1] * o.dR[3 + j] + st->R[3 * i + 2] * o.dR[6 + j];
    tn[i] = st->R[3 * i] * o.dt[0] + st->R[3 * i + 1] * o.dt[1] + st->R[3 * i + 2] * o.dt[2] + st->t[i];
  }
  // motion in the caller's frame: rotation angle of Delta_R and the change of
  // t_raw = t + mu_y - R mu_x, relative to the target diagonal
  double fro = 0.0;
  for (int i = 0; i < 9; ++i) {
    const double d = o.dR[i] - ((i % 4 == 0) ? 1.0 : 0.0);
    fro += d * d;
  }
  const double ang = 2.0 * asin(fmin(1.0, sqrt(fro) / (2.0 * sqrt(2.0))));
  double dtr2 = 0.0;
  for (int i = 0; i < 3; ++i) {
    const double to = st->t[i] - (st->R[3 * i] * st->mu_x[0] + st->R[3 * i + 1] * st->mu_x[1] + st->R[3 * i + 2] * st->mu_x[2]);
    const double tw = tn[i] - (Rn[3 * i] * st->mu_x[0] + Rn[3 * i + 1] * st->mu_x[1] + Rn[3 * i + 2] * st->mu_x[2]);
    dtr2 += (tw - to) * (tw - to);
  }
  const double motion = fmax(ang, sqrt(dtr2) / (st->diag > 0 ? st->diag : 1.0));
  const double s2 = o.Q / (3.0 * NP);
  const bool at_floor = !(s2 > st->sigma2_floor);
  for (int i = 0; i < 9; ++i) st->R[i] = Rn[i];
  for (int i = 0; i < 3; ++i) st->t[i] = tn[i];
  st->sigma2 = at_floor ? st->sigma2_floor : s2;
  const int it = st->iter;
  if (trace) {
    double* tr = trace + static_cast<size_t>(it) * 8;
    tr[0] = st->sigma2;
    tr[1] = NP;
    tr[2] = o.Q;
    tr[3] = o.iters;
    tr[4] = o.damped;
    tr[5] = motion;
    tr[6] = mom[75];
    tr[7] = mom[74];
  }
  st->iter = it + 1;
  if (at_floor || (dp.tol > 0.0 && motion < dp.tol) || st->iter >= dp.max_iters) st->done = 1;
  set_constants(st, dp.w);
}

// Standalone M step: moments and the starting pose are given; results go to `out`:
// R (9), t (3), sigma2, Q, newton_iters, damped, halvings.
__global__ void mstep_standalone_kernel(const double* __restrict__ mom, const double* __restrict__ pose,
                                        DevParams dp, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  QModel q;
  build_model(mom, pose, q);
  NewtonOut o;
  newton(q, dp.newton_max, dp.newton_tol, o);
  const double* R = pose;
  const double* t = pose + 9;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j)
      out[3 * i + j] = R[3 * i] * o.dR[j] + R[3 * i + 1] * o.dR[3 + j] + R[3 * i + 2] * o.dR[6 + j];
    out[9 + i] = R[3 * i] * o.dt[0] + R[3 * i + 1] * o.dt[1] + R[3 * i + 2] * o.dt[2] + t[i];
  }
  out[12] = mom[0] > 0.0 ? o.Q / (3.0 * mom[0]) : 0.0;
  out[13] = o.Q;
  out[14] = o.iters;
  out[15] = o.damped;
  out[16] = o.halvings;
}

__global__ void __launch_bounds__(kRedThreads) reduce_kernel(const double* __restrict__ blk, int nblk,
                                                             double* __restrict__ out) {
  __shared__ double part[(kRedThreads / 32) * kGlob];
  __shared__ double mom[kGlob];
  reduce_rows(blk, nblk, part, mom);
  if (threadIdx.x < kGlob) out[threadIdx.x] = mom[threadIdx.x];
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
    st->t[i] = pose.R[3 * i] * st->mu_x[0] + pose.R[3 * i + 1] * st->mu_x[1] +
               pose.R[3 * i + 2] * st->mu_x[2] + pose.t[i] - st->mu_y[i];
  st->sigma2 = sigma2;
  st->V = V;
  st->log2_wodds = w > 0.0 ? log2(w) - log2(1.0 - w) : -INFINITY;
  st->done = 0;
  st->iter = 0;
  st->numeric_fail = 0;
  set_constants(st, w);
}

}  // namespace

cudaError_t launch_mstep(const double* blk, int nblk, EmState* st, const DevParams& dp, double* trace,
                         double* out, int standalone, cudaStream_t s) {
  if (standalone) {
    // blk holds the kGlob moments; out[0..11] holds the starting pose (R, t) and
    // receives the results at out[16..32]
    mstep_standalone_kernel<<<1, 32, 0, s>>>(blk, out, dp, out + 16);
  } else {
    mstep_em_kernel<<<1, kRedThreads, 0, s>>>(blk, nblk, st, dp, trace);
  }
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

cudaError_t launch_reduce_moments(const double* blk, int nblk, double* out, cudaStream_t s) {
  reduce_kernel<<<1, kRedThreads, 0, s>>>(blk, nblk, out);
  return cudaGetLastError();
}

}  // namespace lsg
