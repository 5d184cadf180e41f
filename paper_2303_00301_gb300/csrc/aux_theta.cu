// aux_theta.cu — the stochastic-volatility parameterisation behind the C ABI:
// theta = (mu, phi, L = chol Sigma) -> (m0, P0, F, b, Q) on the device, and the
// gradient-based theta-update inside the Gibbs sweep.
//
// Model (Section 4.1): F = diag(phi), b = (1 - phi) mu, Q = L L^T, p_0 the
// stationary law (m0 = mu, P0_ij = Q_ij / (1 - phi_i phi_j)). The handle keeps
// theta in the head of its FP64 gradient constants [mu, phi, L, Q, Q^{-1},
// P0^{-1}] (unpadded), which aux_loglik_grad reads; one warp rebuilds every
// constant and the padded compute-type model from theta, so that a sweep
// aux_kalman_step -> aux_loglik_grad -> aux_sv_theta_step stays on the device.
//
// The update (the paper updates its static parameters inside the sampler,
// Section 4.3, without stating a rule): one projected gradient-ascent step on the
// mean over the chains of log p(ytilde_c | theta),
//   mu  <- mu + lr mean_c g_mu[c],   phi <- clip(phi + lr mean_c g_phi[c], +-0.999),
//   L   <- tril(L + lr mean_c g_L[c]) with diag(L) >= 1e-6.
#include <cmath>
#include <vector>

#include "aux_device.cuh"
#include "aux_internal.h"

namespace auxk {

constexpr double THETA_PHI_MAX = 0.999;
constexpr double THETA_L_MIN = 1e-6;

template <typename Real> struct ThetaArgs {
  double* gc;                  // [mu d][phi d][L d^2][Q d^2][Q^-1 d^2][P0^-1 d^2]
  Real *F, *b, *Q, *P0, *m0;   // padded device model (compute type)
  const double *g_mu, *g_phi, *g_L;   // [C][d], [C][d], [C][d][d], or null: no update
  int C, d;
  double lr;
  int32_t* status;             // [1]: ST_NOT_PD when chol(P0) failed
};

// one warp; lane i owns row i of every d x d matrix
template <typename Real, int DP>
__global__ void __launch_bounds__(32, 1) k_sv_theta(ThetaArgs<Real> a) {
  using L_ = Lay<double, DP>;
  constexpr int MAT = L_::MAT, VEC = L_::VEC, LD = L_::LD;
  __shared__ __align__(16) double sm[4 * MAT + 3 * VEC];
  double* SL = sm;           // L rows, then P0's factor (LS form)
  double* SLS = SL + MAT;    // L in LS form (L[k + m][k] at [k][m])
  double* SW = SLS + MAT;    // L^{-1}, then chol(P0)^{-1}
  double* SX = SW + MAT;     // scratch rows
  double* sphi = SX + MAT;
  double* vinv = sphi + VEC;
  double* vinv2 = vinv + VEC;
  const int lane = threadIdx.x, d = a.d;
  const bool act = lane < DP, in = lane < d;
  const int row = act ? lane : 0;
  const long dd = (long)d * d;
  double* gmu = a.gc;
  double* gphi = gmu + d;
  double* gL = gphi + d;
  double* gQ = gL + dd;
  double* gQi = gQ + dd;
  double* gP0i = gQi + dd;
  // theta of this lane's row, updated when gradients are given
  double mu = in ? gmu[lane] : 0.0, phi = in ? gphi[lane] : 0.0;
  double l[DP];
#pragma unroll
  for (int j = 0; j < DP; ++j) l[j] = (in && j <= lane && j < d) ? gL[(long)lane * d + j] : 0.0;
  if (a.g_mu && in) {
    double sm_ = 0.0, sp = 0.0;
    for (int c = 0; c < a.C; ++c) {
      sm_ += a.g_mu[(long)c * d + lane];
      sp += a.g_phi[(long)c * d + lane];
    }
    mu += a.lr * sm_ / a.C;
    phi = fmin(THETA_PHI_MAX, fmax(-THETA_PHI_MAX, phi + a.lr * sp / a.C));
#pragma unroll
    for (int j = 0; j < DP; ++j) {
      if (j <= lane && j < d) {
        double sg = 0.0;
        for (int c = 0; c < a.C; ++c) sg += a.g_L[((long)c * d + lane) * d + j];
        l[j] += a.lr * sg / a.C;
      }
    }
#pragma unroll
    for (int j = 0; j < DP; ++j)
      if (j == lane) l[j] = fmax(l[j], THETA_L_MIN);
  }
  if (in) {
    gmu[lane] = mu;
    gphi[lane] = phi;
#pragma unroll
    for (int j = 0; j < DP; ++j)
      if (j < d) gL[(long)lane * d + j] = l[j];
  }
  // L rows, its LS form and 1/L_kk; phi as a broadcast vector
  st_row<double, DP>(SL, row, l, act);
  if (act) {
    sphi[lane] = in ? phi : 0.0;
#pragma unroll
    for (int k = 0; k < DP; ++k)
      if (k <= lane) SLS[k * LD + (lane - k)] = (k < d || k == lane) ? l[k] : 0.0;
    double diag = 1.0;
#pragma unroll
    for (int j = 0; j < DP; ++j)
      if (j == lane && lane < d) diag = l[j];
    vinv[lane] = 1.0 / diag;
  }
  __syncwarp();
  // Q = L L^T and P0_ij = Q_ij / (1 - phi_i phi_j) for the lane's row
  double q[DP], p0[DP], ph[DP];
  row_matT<double, DP>(l, SL, q);
  ld_vec<double, DP>(sphi, ph);
#pragma unroll
  for (int j = 0; j < DP; ++j) p0[j] = (in && j < d) ? q[j] / (1.0 - phi * ph[j]) : 0.0;
  // Q^{-1} = W^T W with W = L^{-1} (column `lane` of W from L w = e_lane)
  {
    double r[DP];
#pragma unroll
    for (int j = 0; j < DP; ++j) r[j] = (j == lane) ? 1.0 : 0.0;
    fsolve_rot<double, DP, true>(SLS, vinv, r, SW, lane);
  }
  __syncwarp();
  double qi[DP];
  mm_col<double, DP>(SW, row, SW, qi);
  // P0^{-1} the same way from chol(P0) (the padded rows get unit pivots)
  int bad = 0;
  {
    double a_[DP];
#pragma unroll
    for (int j = 0; j < DP; ++j) a_[j] = p0[j];
    __syncwarp();
    chol_rot<double, DP>(a_, SL, nullptr, nullptr, vinv2, nullptr, d, lane, &bad);
    double r[DP];
#pragma unroll
    for (int j = 0; j < DP; ++j) r[j] = (j == lane) ? 1.0 : 0.0;
    __syncwarp();
    fsolve_rot<double, DP, true>(SL, vinv2, r, SX, lane);
  }
  __syncwarp();
  double pi[DP];
  mm_col<double, DP>(SX, row, SX, pi);
  if (in) {
#pragma unroll
    for (int j = 0; j < DP; ++j) {
      if (j < d) {
        gQ[(long)lane * d + j] = q[j];
        gQi[(long)lane * d + j] = qi[j];
        gP0i[(long)lane * d + j] = pi[j];
      }
    }
  }
  // the padded compute-type model
  if (act) {
#pragma unroll
    for (int j = 0; j < DP; ++j) {
      const bool v = in && j < d;
      a.F[lane * DP + j] = (Real)((v && j == lane) ? phi : 0.0);
      a.Q[lane * DP + j] = (Real)(v ? q[j] : 0.0);
      a.P0[lane * DP + j] = (Real)(v ? p0[j] : 0.0);
    }
    a.b[lane] = (Real)(in ? (1.0 - phi) * mu : 0.0);
    a.m0[lane] = (Real)(in ? mu : 0.0);
  }
  if (bad && lane == 0 && a.status) atomicOr(a.status, 1);
}

template <typename Real>
int launch_theta(aux_model* m, const double* g_mu, const double* g_phi, const double* g_L, double lr,
                 cudaStream_t st) {
  ThetaArgs<Real> a{};
  a.gc = m->gconst;
  a.F = (Real*)m->F; a.b = (Real*)m->b; a.Q = (Real*)m->Q; a.P0 = (Real*)m->P0; a.m0 = (Real*)m->m0;
  a.g_mu = g_mu; a.g_phi = g_phi; a.g_L = g_L;
  a.C = m->C; a.d = m->d; a.lr = lr;
  a.status = m->cov_status ? m->cov_status : nullptr;
  switch (m->DP) {
    case 4: k_sv_theta<Real, 4><<<1, 32, 0, st>>>(a); break;
    case 8: k_sv_theta<Real, 8><<<1, 32, 0, st>>>(a); break;
    case 16: k_sv_theta<Real, 16><<<1, 32, 0, st>>>(a); break;
    case 32: k_sv_theta<Real, 32><<<1, 32, 0, st>>>(a); break;
    default: return AUX_E_UNSUPPORTED;
  }
  return cudaGetLastError() == cudaSuccess ? AUX_OK : AUX_E_CUDA;
}

}  // namespace auxk

namespace {
bool theta_handle_ok(const aux_model* m) {
  return m && !m->fact && !m->tv && m->DP <= 32 && m->gconst;
}
}  // namespace

extern "C" int aux_set_sv_theta(aux_model* m, const double* mu, const double* phi, const double* L,
                                double delta) {
  if (!m || !mu || !phi || !L) return AUX_E_INVALID_ARG;
  if (!theta_handle_ok(m)) return AUX_E_UNSUPPORTED;
  if (!(delta > 0.0) || !std::isfinite(delta)) return AUX_E_INVALID_ARG;
  const int d = m->d;
  std::vector<double> th((size_t)2 * d + (size_t)d * d, 0.0);
  for (int i = 0; i < d; ++i) {
    if (!std::isfinite(mu[i]) || !std::isfinite(phi[i])) return AUX_E_NONFINITE;
    if (!(std::fabs(phi[i]) < 1.0)) return AUX_E_INVALID_ARG;
    th[i] = mu[i];
    th[d + i] = phi[i];
    for (int j = 0; j <= i; ++j) {
      const double v = L[(size_t)i * d + j];
      if (!std::isfinite(v)) return AUX_E_NONFINITE;
      th[2 * d + (size_t)i * d + j] = v;
    }
    if (!(L[(size_t)i * d + i] > 0.0)) return AUX_E_NOT_PD;
  }
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return AUX_E_CUDA;
  if (cudaMemcpy(m->gconst, th.data(), th.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return AUX_E_CUDA;
  const int rc = m->dtype == AUX_F64
                     ? auxk::launch_theta<double>(m, nullptr, nullptr, nullptr, 0.0, m->stream)
                     : auxk::launch_theta<float>(m, nullptr, nullptr, nullptr, 0.0, m->stream);
  if (rc) return rc;
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return AUX_E_CUDA;
  m->delta = delta;
  m->grad_ok = 1;
  m->cov_valid = 0;
  m->br_valid = 0;
  return AUX_OK;
}

extern "C" int aux_sv_theta_step(aux_model* m, const double* g_mu, const double* g_phi, const double* g_L,
                                 double lr, void* stream) {
  if (!m || !g_mu || !g_phi || !g_L || !std::isfinite(lr)) return AUX_E_INVALID_ARG;
  if (!theta_handle_ok(m) || !m->grad_ok) return AUX_E_UNSUPPORTED;
  if (m->mode == AUX_MODE_CACHED_COV) return AUX_E_UNSUPPORTED;   // the cached tables would go stale
  m->stream = (cudaStream_t)stream;
  const int rc = m->dtype == AUX_F64 ? auxk::launch_theta<double>(m, g_mu, g_phi, g_L, lr, m->stream)
                                     : auxk::launch_theta<float>(m, g_mu, g_phi, g_L, lr, m->stream);
  if (rc) return rc;
  m->cov_valid = 0;
  m->br_valid = 0;
  return AUX_OK;
}

extern "C" int aux_get_sv_theta(aux_model* m, double* mu, double* phi, double* L) {
  if (!m || !mu || !phi || !L) return AUX_E_INVALID_ARG;
  if (!theta_handle_ok(m) || !m->grad_ok) return AUX_E_UNSUPPORTED;
  const int d = m->d;
  std::vector<double> th((size_t)2 * d + (size_t)d * d);
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return AUX_E_CUDA;
  if (cudaMemcpy(th.data(), m->gconst, th.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return AUX_E_CUDA;
  for (int i = 0; i < d; ++i) {
    mu[i] = th[i];
    phi[i] = th[d + i];
  }
  for (size_t q = 0; q < (size_t)d * d; ++q) L[q] = th[2 * d + q];
  return AUX_OK;
}
