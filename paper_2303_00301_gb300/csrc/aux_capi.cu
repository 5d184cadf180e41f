// aux_capi.cu — the C ABI declared in include/aux_kalman.h: argument checks,
// model upload, workspace ownership and dispatch to the per-precision kernels.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "aux_internal.h"

namespace {

int pick_dp(int d) {
  if (d <= 4) return 4;
  if (d <= 8) return 8;
  if (d <= 16) return 16;
  if (d <= 32) return 32;
  if (d <= 64) return 64;    // the wide table-mode kernels (aux_wide.cuh), single precision
  if (d <= 128) return 128;
  return 0;
}

// the wide kernels: table modes only, first-order proposal, (G, U) scan sampler
bool wide(const aux_model* m) { return m->DP > 32; }

bool all_finite(const double* a, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

// lower Cholesky of a symmetric d x d matrix (row-major), false if not SPD
bool host_cholesky(const double* A, int d, std::vector<double>& L) {
  L.assign((size_t)d * d, 0.0);
  for (int j = 0; j < d; ++j) {
    double s = A[j * d + j];
    for (int k = 0; k < j; ++k) s -= L[j * d + k] * L[j * d + k];
    if (!(s > 0.0)) return false;
    const double ljj = std::sqrt(s);
    L[j * d + j] = ljj;
    for (int i = j + 1; i < d; ++i) {
      double t = A[i * d + j];
      for (int k = 0; k < j; ++k) t -= L[i * d + k] * L[j * d + k];
      L[i * d + j] = t / ljj;
    }
  }
  return true;
}

bool is_symmetric(const double* A, int d) {
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < i; ++j) {
      const double a = A[i * d + j], b = A[j * d + i];
      if (std::fabs(a - b) > 1e-12 * (std::fabs(a) + std::fabs(b) + 1e-300)) return false;
    }
  return true;
}

// inverse of an SPD matrix from its Cholesky factor
std::vector<double> spd_inverse(const std::vector<double>& L, int d) {
  std::vector<double> inv((size_t)d * d, 0.0), col(d);
  for (int c = 0; c < d; ++c) {
    for (int i = 0; i < d; ++i) col[i] = (i == c) ? 1.0 : 0.0;
    for (int i = 0; i < d; ++i) {  // L y = e_c
      double s = col[i];
      for (int k = 0; k < i; ++k) s -= L[i * d + k] * col[k];
      col[i] = s / L[i * d + i];
    }
    for (int i = d - 1; i >= 0; --i) {  // L^T x = y
      double s = col[i];
      for (int k = i + 1; k < d; ++k) s -= L[k * d + i] * col[k];
      col[i] = s / L[i * d + i];
    }
    for (int i = 0; i < d; ++i) inv[i * d + c] = col[i];
  }
  return inv;
}

template <typename Real>
std::vector<unsigned char> pad_matrix(const double* A, int d, int DP) {
  std::vector<unsigned char> out((size_t)DP * DP * sizeof(Real), 0);
  Real* o = reinterpret_cast<Real*>(out.data());
  if (A)
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) o[i * DP + j] = (Real)A[i * d + j];
  return out;
}

template <typename Real>
std::vector<unsigned char> pad_vector(const double* a, int d, int DP) {
  std::vector<unsigned char> out((size_t)DP * sizeof(Real), 0);
  Real* o = reinterpret_cast<Real*>(out.data());
  if (a)
    for (int i = 0; i < d; ++i) o[i] = (Real)a[i];
  return out;
}

template <typename Real>
std::vector<unsigned char> convert(const double* a, size_t n) {
  std::vector<unsigned char> out(n * sizeof(Real));
  Real* o = reinterpret_cast<Real*>(out.data());
  for (size_t i = 0; i < n; ++i) o[i] = (Real)a[i];
  return out;
}

int dev_alloc(aux_model* m, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return AUX_E_OOM;
  }
  m->allocs.push_back(*p);
  return AUX_OK;
}

int upload(aux_model* m, void** p, const std::vector<unsigned char>& h) {
  int rc = dev_alloc(m, p, h.size());
  if (rc) return rc;
  return cudaMemcpy(*p, h.data(), h.size(), cudaMemcpyHostToDevice) == cudaSuccess ? AUX_OK
                                                                                  : AUX_E_CUDA;
}

void release(aux_model* m) {
  if (!m) return;
  cudaDeviceSynchronize();
  for (auto& r : m->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto& r : m->pool) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (void* p : m->allocs) cudaFree(p);
  m->allocs.clear();
  delete m;
}

int put(aux_model* m, void** p, const std::vector<unsigned char>& h, bool alloc) {
  if (alloc) return upload(m, p, h);
  return cudaMemcpy(*p, h.data(), h.size(), cudaMemcpyHostToDevice) == cudaSuccess ? AUX_OK
                                                                                  : AUX_E_CUDA;
}

// time-varying dynamics: the T - 1 transitions in the per-chain kernels' shared-memory
// slot layout (row stride DP + 16 bytes of padding, zero padded), F^T beside F
template <typename Real>
std::vector<unsigned char> slot_stack(const double* A, int n, int d, int DP, bool transpose) {
  const int LD = DP + (int)(16 / sizeof(Real));
  std::vector<unsigned char> out((size_t)std::max(n, 1) * DP * LD * sizeof(Real), 0);
  Real* o = reinterpret_cast<Real*>(out.data());
  for (int t = 0; t < n; ++t)
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j)
        o[(size_t)t * DP * LD + (size_t)i * LD + j] = (Real)A[(size_t)t * d * d + (transpose ? j * d + i : i * d + j)];
  return out;
}
template <typename Real>
std::vector<unsigned char> vec_stack(const double* a, int n, int d, int DP) {
  const int VEC = (DP + (int)(16 / sizeof(Real)) - 1) / (int)(16 / sizeof(Real)) * (int)(16 / sizeof(Real));
  std::vector<unsigned char> out((size_t)std::max(n, 1) * VEC * sizeof(Real), 0);
  Real* o = reinterpret_cast<Real*>(out.data());
  for (int t = 0; t < n; ++t)
    for (int i = 0; i < d; ++i) o[(size_t)t * VEC + i] = (Real)a[(size_t)t * d + i];
  return out;
}

template <typename Real>
int upload_model(aux_model* m, const aux_model_desc* d, const std::vector<double>& Ryinv,
                 bool alloc) {
  const int dd = m->d, DP = m->DP;
  int rc;
  if (m->tv) {   // the stacks, and the first transition as the homogeneous model slots
    const int n = m->T - 1;
    if ((rc = put(m, &m->Ftv, slot_stack<Real>(d->F, n, dd, DP, false), alloc))) return rc;
    if ((rc = put(m, &m->FTtv, slot_stack<Real>(d->F, n, dd, DP, true), alloc))) return rc;
    if ((rc = put(m, &m->Qtv, slot_stack<Real>(d->Q, n, dd, DP, false), alloc))) return rc;
    if ((rc = put(m, &m->btv, vec_stack<Real>(d->b, n, dd, DP), alloc))) return rc;
  }
  if ((rc = put(m, &m->F, pad_matrix<Real>(d->F, dd, DP), alloc))) return rc;
  if ((rc = put(m, &m->Q, pad_matrix<Real>(d->Q, dd, DP), alloc))) return rc;
  if ((rc = put(m, &m->P0, pad_matrix<Real>(d->P0, dd, DP), alloc))) return rc;
  if ((rc = put(m, &m->m0, pad_vector<Real>(d->m0, dd, DP), alloc))) return rc;
  if ((rc = put(m, &m->b, pad_vector<Real>(d->b, dd, DP), alloc))) return rc;
  if ((rc = put(m, &m->Ryinv, pad_matrix<Real>(Ryinv.empty() ? nullptr : Ryinv.data(), dd, DP), alloc))) return rc;
  const size_t ny = (size_t)(m->y_per_chain ? m->C : 1) * m->T * dd;
  if ((rc = put(m, &m->y, convert<Real>(d->y, ny), alloc))) return rc;
  return AUX_OK;
}

// Host validation shared by aux_init_model and aux_set_model_params; fills Ryinv.
int validate_desc(const aux_model_desc* desc, std::vector<double>& Ryinv) {
  if (!desc) return AUX_E_INVALID_ARG;
  if (desc->abi_version != AUX_ABI_VERSION) return AUX_E_INVALID_ARG;
  if (desc->dtype != AUX_F32 && desc->dtype != AUX_F64 && desc->dtype != AUX_MIXED) return AUX_E_INVALID_ARG;
  if (desc->emis_kind != AUX_EMIS_LINEAR_GAUSSIAN && desc->emis_kind != AUX_EMIS_SV &&
      desc->emis_kind != AUX_EMIS_STUDENT_T)
    return AUX_E_INVALID_ARG;
  const int d = desc->d_x, T = desc->T, C = desc->n_chains;
  const bool st = desc->emis_kind == AUX_EMIS_STUDENT_T;
  if (d < 1 || T < 1 || C < 1 || desc->block_len < 0) return AUX_E_INVALID_ARG;
  if (!desc->m0 || !desc->P0 || !desc->F || !desc->b || !desc->Q || !desc->y)
    return AUX_E_INVALID_ARG;
  if ((desc->emis_kind == AUX_EMIS_LINEAR_GAUSSIAN || st) && !desc->R_y) return AUX_E_INVALID_ARG;
  if (!(desc->delta > 0.0) || !std::isfinite(desc->delta)) return AUX_E_INVALID_ARG;
  if (st && (!(desc->nu > 0.0) || !std::isfinite(desc->nu))) return AUX_E_INVALID_ARG;
  if (desc->dyn_kind != AUX_DYN_HOMOGENEOUS && desc->dyn_kind != AUX_DYN_TIME_VARYING) return AUX_E_INVALID_ARG;
  const bool tvd = desc->dyn_kind == AUX_DYN_TIME_VARYING;
  if (tvd && (st || desc->dtype == AUX_MIXED || pick_dp(d) == 0 || pick_dp(d) > 32)) return AUX_E_UNSUPPORTED;
  if (st) {
    if (d > 1024 || desc->dtype == AUX_MIXED) return AUX_E_UNSUPPORTED;
    for (int i = 0; i < d; ++i)   // the factorised path needs diagonal F, Q, P0
      for (int j = 0; j < d; ++j)
        if (i != j && (desc->F[i * d + j] != 0.0 || desc->Q[i * d + j] != 0.0 || desc->P0[i * d + j] != 0.0))
          return AUX_E_UNSUPPORTED;
  } else {
    const int DP = pick_dp(d);
    if (DP == 0) return AUX_E_UNSUPPORTED;
    if (desc->dtype == AUX_F64 && DP > 32) return AUX_E_UNSUPPORTED;
    if (desc->dtype == AUX_MIXED && DP <= 32) return AUX_E_UNSUPPORTED;   // the wide widths only
  }
  if ((long long)C * T * d > (1LL << 31)) return AUX_E_UNSUPPORTED;
  const size_t dd = (size_t)d * d;
  const size_t ny = (size_t)(desc->y_per_chain ? C : 1) * T * d;
  const size_t ntr = tvd ? (size_t)(T - 1) : 1;   // transitions given
  if (!all_finite(desc->m0, d) || !all_finite(desc->P0, dd) || !all_finite(desc->F, ntr * dd) ||
      !all_finite(desc->b, ntr * d) || !all_finite(desc->Q, ntr * dd) || !all_finite(desc->y, ny))
    return AUX_E_NONFINITE;
  if (desc->R_y && desc->emis_kind != AUX_EMIS_SV && !all_finite(desc->R_y, dd))
    return AUX_E_NONFINITE;
  std::vector<double> L;
  if (!is_symmetric(desc->P0, d) || !host_cholesky(desc->P0, d, L)) return AUX_E_NOT_PD;
  for (size_t t = 0; t < (tvd ? ntr : 1); ++t)
    if (!is_symmetric(desc->Q + t * dd, d) || !host_cholesky(desc->Q + t * dd, d, L)) return AUX_E_NOT_PD;
  Ryinv.clear();
  if (desc->emis_kind != AUX_EMIS_SV) {
    if (!is_symmetric(desc->R_y, d) || !host_cholesky(desc->R_y, d, L)) return AUX_E_NOT_PD;
    Ryinv = spd_inverse(L, d);
  }
  return AUX_OK;
}

// The SV parameterisation needed by aux_loglik_grad: F = diag(phi) with |phi| < 1,
// m0 = mu = b / (1 - phi), P0_ij = Q_ij / (1 - phi_i phi_j). Fills the FP64 constants
// [mu, phi, L, Q, Q^{-1}, P0^{-1}] when it holds.
bool theta_constants(const aux_model_desc* desc, std::vector<double>& gc) {
  const int d = desc->d_x;
  std::vector<double> mu(d), phi(d), L, LP;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      if (i != j && desc->F[i * d + j] != 0.0) return false;
  for (int i = 0; i < d; ++i) {
    phi[i] = desc->F[i * d + i];
    if (!(std::fabs(phi[i]) < 1.0)) return false;
    mu[i] = desc->b[i] / (1.0 - phi[i]);
    if (std::fabs(desc->m0[i] - mu[i]) > 1e-9 * (1.0 + std::fabs(mu[i]))) return false;
  }
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      const double st = desc->Q[i * d + j] / (1.0 - phi[i] * phi[j]);
      if (std::fabs(desc->P0[i * d + j] - st) > 1e-9 * (1.0 + std::fabs(st))) return false;
    }
  if (!host_cholesky(desc->Q, d, L) || !host_cholesky(desc->P0, d, LP)) return false;
  const std::vector<double> Qi = spd_inverse(L, d), P0i = spd_inverse(LP, d);
  gc.clear();
  gc.insert(gc.end(), mu.begin(), mu.end());
  gc.insert(gc.end(), phi.begin(), phi.end());
  gc.insert(gc.end(), L.begin(), L.end());
  gc.insert(gc.end(), desc->Q, desc->Q + (size_t)d * d);
  gc.insert(gc.end(), Qi.begin(), Qi.end());
  gc.insert(gc.end(), P0i.begin(), P0i.end());
  return true;
}

int diag_flag(const aux_model_desc* desc) {
  const int d = desc->d_x;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      if (i != j && desc->F[i * d + j] != 0.0) return 0;
  return 1;
}

// the emission's Hessian in x_t is diagonal: SV, or linear-Gaussian with diagonal R_y
int hess_diag_flag(const aux_model_desc* desc) {
  if (desc->emis_kind == AUX_EMIS_SV) return 1;
  const int d = desc->d_x;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      if (i != j && desc->R_y[i * d + j] != 0.0) return 0;
  return 1;
}

// factorised-prior handle (Student-t emission): diagonal model vectors, the
// inverse scale matrix, observations and the scalar tables and workspaces
template <typename Real>
int fact_upload(aux_model* m, const aux_model_desc* desc, const std::vector<double>& Lam) {
  const int d = m->d;
  std::vector<Real> mod(5 * (size_t)d), lam((size_t)d * d);
  for (int i = 0; i < d; ++i) {
    mod[i] = (Real)desc->F[i * d + i];
    mod[d + i] = (Real)desc->b[i];
    mod[2 * d + i] = (Real)desc->Q[i * d + i];
    mod[3 * d + i] = (Real)desc->P0[i * d + i];
    mod[4 * d + i] = (Real)desc->m0[i];
  }
  for (size_t q = 0; q < (size_t)d * d; ++q) lam[q] = (Real)Lam[q];
  const size_t ny = (size_t)(m->y_per_chain ? m->C : 1) * m->T * d;
  std::vector<Real> yv(ny);
  for (size_t q = 0; q < ny; ++q) yv[q] = (Real)desc->y[q];
  auto bytes = [](const auto& v) {
    std::vector<unsigned char> h(v.size() * sizeof(v[0]));
    std::memcpy(h.data(), v.data(), h.size());
    return h;
  };
  int rc = upload(m, &m->fmodel, bytes(mod));
  if (!rc) rc = upload(m, &m->flam, bytes(lam));
  if (!rc) rc = upload(m, &m->y, bytes(yv));
  return rc;
}

int fact_init(aux_model* m, const aux_model_desc* desc, const std::vector<double>& Lam) {
  m->fact = 1;
  m->nu = desc->nu;
  int rc = m->dtype == AUX_F32 ? fact_upload<float>(m, desc, Lam) : fact_upload<double>(m, desc, Lam);
  if (!rc && desc->obs_mask) {
    std::vector<unsigned char> mk(desc->obs_mask, desc->obs_mask + m->T);
    rc = upload(m, (void**)&m->mask, mk);
  }
  const size_t es = m->esz, d = m->d, T = m->T, C = m->C, nb = m->nb;
  const size_t path = C * T * d * es, blk = C * nb * d;
  if (!rc) rc = dev_alloc(m, &m->u, path);
  if (!rc) rc = dev_alloc(m, &m->v, path);
  if (!rc) rc = dev_alloc(m, &m->yt, path);
  if (!rc) rc = dev_alloc(m, &m->xs, path);
  if (!rc) rc = dev_alloc(m, &m->yts, path);
  if (!rc) rc = dev_alloc(m, &m->U, path);
  if (!rc) rc = dev_alloc(m, &m->ftab, 4 * T * d * es);
  if (!rc) rc = dev_alloc(m, &m->fbt, 2 * nb * d * es);
  if (!rc) rc = dev_alloc(m, (void**)&m->fldb, nb * d * sizeof(double));
  if (!rc) rc = dev_alloc(m, &m->fz, blk * es);
  if (!rc) rc = dev_alloc(m, &m->fms, blk * es);
  if (!rc) rc = dev_alloc(m, &m->fub, blk * es);
  if (!rc) rc = dev_alloc(m, (void**)&m->ffq, blk * sizeof(double));
  if (!rc) rc = dev_alloc(m, (void**)&m->flz, blk * sizeof(double));
  if (!rc) rc = dev_alloc(m, (void**)&m->fgam, C * T * sizeof(double));
  if (!rc) rc = dev_alloc(m, (void**)&m->fmh, C * T * sizeof(double));
  if (!rc) rc = dev_alloc(m, (void**)&m->status, C * sizeof(int32_t));
  if (!rc) rc = dev_alloc(m, (void**)&m->status_iter, C * sizeof(int32_t));
  if (!rc) rc = dev_alloc(m, (void**)&m->accept, C * sizeof(int32_t));
  if (!rc) rc = dev_alloc(m, (void**)&m->la_all, C * sizeof(double));
  if (!rc && (cudaMemset(m->status, 0, C * sizeof(int32_t)) != cudaSuccess)) rc = AUX_E_CUDA;
  if (!rc) rc = aux_fact_prepare(m);
  return rc;
}


// buffers of the bridging sampler for the handle's current mode (aux_set_sampler)
int br_alloc(aux_model* m) {
  if (m->sampler != AUX_SAMPLER_BRIDGING) return AUX_OK;
  if (m->T - 1 > (1 << 29)) return AUX_E_UNSUPPORTED;   // tree depth beyond the kernel's level table
  const size_t es = m->esz, DP = (size_t)m->DP, DD = DP * DP;
  const int n = m->T - 1;
  int NN = 0;
  for (int c = n; c > 1;) { c = (c + 1) / 2; NN += c; }
  m->br_NN = NN;
  const size_t nn = (size_t)std::max(NN, 1);
  int rc = AUX_OK;
  if (!m->br_g) rc = dev_alloc(m, &m->br_g, (size_t)m->C * nn * DP * es);
  if (!rc && m->mode != AUX_MODE_PER_CHAIN) {
    if (!m->br_L0) rc = dev_alloc(m, &m->br_L0, (size_t)std::max(n, 1) * DD * es);
    if (!rc && !m->br_tree) rc = dev_alloc(m, &m->br_tree, 5 * nn * DD * es);
  }
  if (!rc && m->mode == AUX_MODE_PER_CHAIN) {
    if (!m->Sig) rc = dev_alloc(m, &m->Sig, (size_t)m->C * m->T * DD * es);
    if (!rc && !m->br_ctree) rc = dev_alloc(m, &m->br_ctree, (size_t)m->C * 5 * nn * DD * es);
  }
  return rc;
}

}  // namespace

extern "C" {

const char* aux_status_string(int code) {
  switch (code) {
    case AUX_OK: return "ok";
    case AUX_E_INVALID_ARG: return "invalid argument";
    case AUX_E_NOT_PD: return "matrix not positive definite";
    case AUX_E_NONFINITE: return "non-finite value";
    case AUX_E_CUDA: return "CUDA runtime error";
    case AUX_E_TIMEOUT: return "device wait timed out";
    case AUX_E_OOM: return "out of device memory";
    case AUX_E_UNSUPPORTED: return "unsupported configuration";
    case AUX_E_TOO_LARGE: return "problem exceeds the fixed scratch of aux_loglik_noalloc";
    default: return "unknown status";
  }
}

int aux_init_model(const aux_model_desc* desc, uint64_t seed, void* stream, aux_model** out) {
  if (!desc || !out) return AUX_E_INVALID_ARG;
  *out = nullptr;
  std::vector<double> Ryinv;
  const int vrc = validate_desc(desc, Ryinv);
  if (vrc) return vrc;
  const int d = desc->d_x, T = desc->T, C = desc->n_chains;
  const bool fact = desc->emis_kind == AUX_EMIS_STUDENT_T;
  const int DP = fact ? 0 : pick_dp(d);

  aux_model* m = new (std::nothrow) aux_model();
  if (!m) return AUX_E_OOM;
  m->dtype = desc->dtype; m->d = d; m->DP = DP; m->T = T; m->C = C;
  m->emis = desc->emis_kind; m->y_per_chain = desc->y_per_chain ? 1 : 0;
  int L_blk = desc->block_len;
  if (L_blk == 0) L_blk = std::max(1, (int)std::ceil(std::sqrt((double)T)));
  if (L_blk > T) L_blk = T;
  m->L = L_blk;
  m->nb = (T + L_blk - 1) / L_blk;
  m->delta = desc->delta;
  m->seed = seed;
  m->tv = desc->dyn_kind == AUX_DYN_TIME_VARYING ? 1 : 0;
  m->fdiag = m->tv ? 0 : diag_flag(desc);   // the time-varying kernels take the dense-F path
  m->diag_hess = hess_diag_flag(desc);
  m->stream = (cudaStream_t)stream;
  m->esz = desc->dtype == AUX_F64 ? sizeof(double) : sizeof(float);   // AUX_MIXED stores FP32
  cudaGetDevice(&m->device);
  if (cudaDeviceGetAttribute(&m->n_sm, cudaDevAttrMultiProcessorCount, m->device) != cudaSuccess ||
      m->n_sm < 1) {
    release(m);
    return AUX_E_CUDA;
  }
  if (fact) {
    const int rc = fact_init(m, desc, Ryinv);
    if (rc) { release(m); return rc; }
    *out = m;
    return AUX_OK;
  }
  if (desc->dtype == AUX_MIXED) m->ops = aux_ops_mixed_wide(DP);
  else m->ops = desc->dtype == AUX_F32 ? (DP > 32 ? aux_ops_f32_wide(DP) : aux_ops_f32(DP)) : aux_ops_f64(DP);
  if (!m->ops) { release(m); return AUX_E_UNSUPPORTED; }

  int rc = desc->dtype != AUX_F64 ? upload_model<float>(m, desc, Ryinv, true)
                                  : upload_model<double>(m, desc, Ryinv, true);
  std::vector<double> gc;
  m->grad_ok = (!m->tv && theta_constants(desc, gc)) ? 1 : 0;
  if (!rc) {   // always allocated (sized for d), rewritten by aux_set_model_params
    std::vector<unsigned char> h((size_t)(2 * d + 4 * d * d) * sizeof(double), 0);
    if (m->grad_ok) std::memcpy(h.data(), gc.data(), gc.size() * sizeof(double));
    rc = upload(m, (void**)&m->gconst, h);
  }
  if (!rc && desc->obs_mask) {
    std::vector<unsigned char> mk(desc->obs_mask, desc->obs_mask + T);
    rc = upload(m, (void**)&m->mask, mk);
  }
  const size_t es = m->esz;
  const size_t path = (size_t)C * T * d * es;
  const size_t nbC = (size_t)C * m->nb;
  if (!rc) rc = dev_alloc(m, &m->u, path);
  if (!rc) rc = dev_alloc(m, &m->v, path);
  if (!rc) rc = dev_alloc(m, &m->yt, path);
  if (!rc) rc = dev_alloc(m, &m->xs, path);
  if (!rc) rc = dev_alloc(m, &m->yts, path);
  if (DP <= 32) {   // the per-chain element scan (not offered by the wide kernels)
    if (!rc) rc = dev_alloc(m, &m->agg0, nbC * aux_es(DP) * es);
    if (!rc) rc = dev_alloc(m, &m->agg1, nbC * aux_es(DP) * es);
    if (!rc) rc = dev_alloc(m, &m->G, (size_t)C * T * DP * DP * es);
    if (!rc) rc = dev_alloc(m, &m->gum, nbC * DP * DP * es);
  }
  if (!rc) rc = dev_alloc(m, &m->U, (size_t)C * T * DP * es);
  if (!rc) rc = dev_alloc(m, &m->guv, nbC * DP * es);
  if (!rc) rc = dev_alloc(m, (void**)&m->fq, (size_t)C * T * sizeof(double));
  if (!rc) rc = dev_alloc(m, (void**)&m->fld, (size_t)C * T * sizeof(double));
  if (!rc) rc = dev_alloc(m, (void**)&m->mh_part, nbC * sizeof(double));
  if (!rc) rc = dev_alloc(m, (void**)&m->lz_part, nbC * sizeof(double));
  if (!rc) rc = dev_alloc(m, (void**)&m->status_iter, (size_t)C * sizeof(int32_t));
  if (!rc) rc = dev_alloc(m, (void**)&m->status, (size_t)C * sizeof(int32_t));
  if (!rc) rc = dev_alloc(m, (void**)&m->accept, (size_t)C * sizeof(int32_t));
  if (!rc) rc = dev_alloc(m, (void**)&m->la_all, (size_t)C * sizeof(double));
  if (!rc && (cudaMemset(m->status, 0, (size_t)C * sizeof(int32_t)) != cudaSuccess ||
              cudaMemset(m->status_iter, 0, (size_t)C * sizeof(int32_t)) != cudaSuccess))
    rc = AUX_E_CUDA;
  if (!rc) rc = m->ops->prepare();
  if (rc) { release(m); return rc; }
  *out = m;
  return AUX_OK;
}

int aux_kalman_step(aux_model* m, void* x, int32_t n_iters, uint64_t iter0,
                    uint32_t* accept_count, double* log_alpha, void* stream) {
  if (!m || !x || n_iters < 0) return AUX_E_INVALID_ARG;
  m->stream = (cudaStream_t)stream;
  if (n_iters == 0) return AUX_OK;
  if (m->fact) return aux_fact_kalman_step(m, x, n_iters, iter0, accept_count, log_alpha, m->stream);
  return m->ops->kalman_step(m, x, n_iters, iter0, accept_count, log_alpha, m->stream);
}

int aux_loglik(aux_model* m, const void* ytilde, double* logZ, void* mf, void* Pf, void* stream) {
  if (!m || !ytilde || !logZ) return AUX_E_INVALID_ARG;
  m->stream = (cudaStream_t)stream;
  if (m->fact) return Pf ? AUX_E_UNSUPPORTED : aux_fact_loglik(m, ytilde, logZ, mf, m->stream);
  return m->ops->loglik(m, ytilde, logZ, mf, Pf, m->stream);
}

int aux_sample_path(aux_model* m, const void* ytilde, const void* eps, uint64_t iteration,
                    void* xstar, double* logZ, void* stream) {
  if (!m || !ytilde || !xstar) return AUX_E_INVALID_ARG;
  m->stream = (cudaStream_t)stream;
  if (m->fact) return aux_fact_sample_path(m, ytilde, eps, iteration, xstar, logZ, m->stream);
  return m->ops->sample_path(m, ytilde, eps, iteration, xstar, logZ, m->stream);
}

// longest block of the covariance scan of the table modes: short blocks put
// most of its critical path into the O(log T) Hillis-Steele rounds; the
// block length divides the means block length so that each means block is a
// whole number of covariance blocks
constexpr int kCovBlockLen = 4;

int aux_set_mode(aux_model* m, int32_t mode) {
  if (!m || (mode != AUX_MODE_PER_CHAIN && mode != AUX_MODE_SHARED_COV && mode != AUX_MODE_CACHED_COV))
    return AUX_E_INVALID_ARG;
  if (m->fact) { m->mode = mode; return AUX_OK; }   // the factorised path has one execution
  if (m->tv && mode != AUX_MODE_PER_CHAIN) return AUX_E_UNSUPPORTED;   // homogeneous tables only
  if (mode != AUX_MODE_PER_CHAIN && !m->tab) {
    const size_t es = m->esz, DD = (size_t)m->DP * m->DP;
    m->Lc = 1;   // the largest divisor of the means block length that is <= kCovBlockLen
    for (int c = std::min(kCovBlockLen, m->L); c >= 1; --c)
      if (m->L % c == 0) { m->Lc = c; break; }
    m->nbc = (m->T + m->Lc - 1) / m->Lc;
    int rc = dev_alloc(m, &m->tab, (size_t)6 * m->T * DD * es);
    if (wide(m)) {   // E^(2^k), double-buffered; per-CTA scratch of the dense routines
      if (!rc) rc = dev_alloc(m, &m->cagg0, (size_t)6 * DD * es);
      if (!rc) rc = dev_alloc(m, &m->cagg1, aux_wide_scratch_elems(m->DP, m->n_sm) * es);
    } else {
      // the covariance scan's buffers; at least the doubling's two powers (A, C, J, chol C)
      if (!rc) rc = dev_alloc(m, &m->cagg0, (size_t)std::max(3 * m->nbc, 8) * DD * es);
      if (!rc) rc = dev_alloc(m, &m->cagg1, (size_t)m->nbc * 3 * DD * es);
    }
    if (!rc) rc = dev_alloc(m, (void**)&m->cov_ldt, (size_t)m->T * sizeof(double));
    // block products, and their group prefixes for the two-level cross-block composition
    if (!rc) rc = dev_alloc(m, &m->btab, (size_t)4 * m->nb * DD * es);
    if (!rc) rc = dev_alloc(m, &m->zb, (size_t)m->C * m->nb * m->DP * es);
    if (!rc) rc = dev_alloc(m, &m->ms, (size_t)m->C * m->nb * m->DP * es);
    if (!rc) rc = dev_alloc(m, (void**)&m->cov_ld, (size_t)m->nb * sizeof(double));
    if (!rc) rc = dev_alloc(m, (void**)&m->cov_status, sizeof(int32_t));
    if (!rc) rc = dev_alloc(m, (void**)&m->cov_kmap, 3 * sizeof(int));
    if (!rc) {
      const int km[3] = {0, 1, m->nbc - 1};
      if (cudaMemcpy(m->cov_kmap, km, sizeof(km), cudaMemcpyHostToDevice) != cudaSuccess) rc = AUX_E_CUDA;
    }
    if (rc) {
      m->tab = m->btab = m->zb = m->ms = m->cagg0 = m->cagg1 = nullptr;
      m->cov_ld = m->cov_ldt = nullptr;
      m->cov_status = nullptr;
      m->cov_kmap = nullptr;
      return rc;
    }
  }
  const int old = m->mode;
  m->mode = mode;
  const int rc = br_alloc(m);
  if (rc) { m->mode = old; return rc; }
  m->cov_valid = 0;
  m->br_valid = 0;
  return AUX_OK;
}

int aux_set_filter_form(aux_model* m, int32_t form) {
  if (!m || (form != AUX_FILTER_COVARIANCE && form != AUX_FILTER_SQUARE_ROOT)) return AUX_E_INVALID_ARG;
  if (m->fact || wide(m) || m->tv) return form == AUX_FILTER_COVARIANCE ? AUX_OK : AUX_E_UNSUPPORTED;
  const int f = form == AUX_FILTER_SQUARE_ROOT ? 1 : 0;
  if (f != m->sqrt_form) {   // the cached tables were made by the other form
    m->cov_valid = 0;
    m->br_valid = 0;
  }
  m->sqrt_form = f;
  return AUX_OK;
}

int aux_set_sampler(aux_model* m, int32_t sampler) {
  if (!m || (sampler != AUX_SAMPLER_SCAN && sampler != AUX_SAMPLER_BRIDGING)) return AUX_E_INVALID_ARG;
  if (m->fact || wide(m) || m->tv) return sampler == AUX_SAMPLER_SCAN ? AUX_OK : AUX_E_UNSUPPORTED;
  const int old = m->sampler;
  m->sampler = sampler;
  const int rc = br_alloc(m);
  if (rc) { m->sampler = old; return rc; }
  m->br_valid = 0;
  return AUX_OK;
}

int aux_set_proposal(aux_model* m, int32_t order) {
  if (!m || (order != AUX_PROPOSAL_FIRST_ORDER && order != AUX_PROPOSAL_SECOND_ORDER))
    return AUX_E_INVALID_ARG;
  if (order == AUX_PROPOSAL_SECOND_ORDER) {
    if (!m->diag_hess || m->fact || wide(m)) return AUX_E_UNSUPPORTED;
    if (!m->rho) {
      const size_t path = (size_t)m->C * m->T * m->d * m->esz;
      int rc = dev_alloc(m, &m->rho, path);
      if (!rc) rc = dev_alloc(m, &m->rhos, path);
      if (rc) { m->rho = m->rhos = nullptr; return rc; }
    }
  }
  m->order = order;
  return AUX_OK;
}

int aux_set_delta_adaptation(aux_model* m, int32_t enable, double target, double gain) {
  if (!m) return AUX_E_INVALID_ARG;
  if (enable) {
    if (!(target > 0.0 && target < 1.0) || !(gain > 0.0) || !std::isfinite(gain)) return AUX_E_INVALID_ARG;
    if (!m->delta_dev) {
      int rc = dev_alloc(m, (void**)&m->delta_dev, 4 * sizeof(double));
      if (!rc) rc = dev_alloc(m, (void**)&m->adapt_count, sizeof(int32_t));
      if (rc) { m->delta_dev = nullptr; m->adapt_count = nullptr; return rc; }
    }
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return AUX_E_CUDA;
    const int32_t zero = 0;
    double w[4];
    delta_words(m->delta, w);
    if (cudaMemcpy(m->delta_dev, w, sizeof(w), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->adapt_count, &zero, sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess)
      return AUX_E_CUDA;
    m->adapt_target = target;
    m->adapt_gain = gain;
    m->adapt = 1;
  } else if (m->adapt) {
    // freeze at the adapted value
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return AUX_E_CUDA;
    if (cudaMemcpy(&m->delta, m->delta_dev, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      return AUX_E_CUDA;
    m->adapt = 0;
  }
  m->cov_valid = 0;
  return AUX_OK;
}

int aux_set_device_iteration(aux_model* m, int32_t enable, uint64_t start) {
  if (!m) return AUX_E_INVALID_ARG;
  if (enable) {
    if (!m->iter_dev) {
      const int rc = dev_alloc(m, (void**)&m->iter_dev, sizeof(uint64_t));
      if (rc) { m->iter_dev = nullptr; return rc; }
    }
    if (cudaStreamSynchronize(m->stream) != cudaSuccess ||
        cudaMemcpy(m->iter_dev, &start, sizeof(uint64_t), cudaMemcpyHostToDevice) != cudaSuccess)
      return AUX_E_CUDA;
  }
  m->dev_iter = enable ? 1 : 0;
  return AUX_OK;
}

int aux_get_device_iteration(aux_model* m, uint64_t* iteration) {
  if (!m || !iteration || !m->iter_dev) return AUX_E_INVALID_ARG;
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return AUX_E_CUDA;
  return cudaMemcpy(iteration, m->iter_dev, sizeof(uint64_t), cudaMemcpyDeviceToHost) == cudaSuccess
             ? AUX_OK
             : AUX_E_CUDA;
}

int aux_get_delta(aux_model* m, double* delta) {
  if (!m || !delta) return AUX_E_INVALID_ARG;
  if (!m->adapt) { *delta = m->delta; return AUX_OK; }
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return AUX_E_CUDA;
  return cudaMemcpy(delta, m->delta_dev, sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess ? AUX_OK
                                                                                              : AUX_E_CUDA;
}

int aux_set_model_params(aux_model* m, const aux_model_desc* desc) {
  if (!m || !desc) return AUX_E_INVALID_ARG;
  if (m->fact) return AUX_E_UNSUPPORTED;
  if (desc->dtype != m->dtype || desc->d_x != m->d || desc->T != m->T || desc->n_chains != m->C ||
      desc->emis_kind != m->emis || (desc->y_per_chain ? 1 : 0) != m->y_per_chain ||
      (desc->dyn_kind == AUX_DYN_TIME_VARYING ? 1 : 0) != m->tv)
    return AUX_E_INVALID_ARG;
  std::vector<double> Ryinv;
  const int vrc = validate_desc(desc, Ryinv);
  if (vrc) return vrc;
  if (m->order == AUX_PROPOSAL_SECOND_ORDER && !hess_diag_flag(desc)) return AUX_E_UNSUPPORTED;
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return AUX_E_CUDA;
  const int rc = m->dtype != AUX_F64 ? upload_model<float>(m, desc, Ryinv, false)
                                     : upload_model<double>(m, desc, Ryinv, false);
  if (rc) return rc;
  m->delta = desc->delta;
  m->fdiag = m->tv ? 0 : diag_flag(desc);
  m->diag_hess = hess_diag_flag(desc);
  m->cov_valid = 0;
  if (m->adapt) {   // a new delta restarts the adaptation from it
    const int32_t zero = 0;
    double w[4];
    delta_words(m->delta, w);
    if (cudaMemcpy(m->delta_dev, w, sizeof(w), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->adapt_count, &zero, sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess)
      return AUX_E_CUDA;
  }
  std::vector<double> gc;
  m->grad_ok = (!m->tv && theta_constants(desc, gc)) ? 1 : 0;
  if (m->grad_ok &&
      cudaMemcpy(m->gconst, gc.data(), gc.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return AUX_E_CUDA;
  return AUX_OK;
}

int aux_loglik_grad(aux_model* m, const void* ytilde, double* logZ, double* g_mu, double* g_Phi,
                    double* g_cholSigma, double* g_delta, void* stream) {
  if (!m || !g_mu || !g_Phi || !g_cholSigma || !g_delta) return AUX_E_INVALID_ARG;
  if (!m->grad_ok || m->fact || wide(m)) return AUX_E_UNSUPPORTED;
  if (m->dtype == AUX_F64 && m->DP > 16) return AUX_E_UNSUPPORTED;   // smoother staging > 227 KB
  if (!ytilde) ytilde = m->yt;   // the last aux_kalman_step's pseudo-observations
  m->stream = (cudaStream_t)stream;
  const size_t es = m->esz, DP = m->DP, nbC = (size_t)m->C * m->nb;
  int rc = AUX_OK;
  // G_t, Sigma_t, U_t of every (chain, step), or of a chunk of blocks (recompute)
  const size_t per_step = (2 * DP * DP + DP) * es;
  m->grad_kc = 0;
  if (m->grad_mem && (size_t)m->C * m->T * per_step > m->grad_mem) {
    const size_t per_block = (size_t)m->C * m->L * per_step;
    m->grad_kc = (int)std::min<size_t>((size_t)m->nb, std::max<size_t>(1, m->grad_mem / per_block));
    const size_t need = (size_t)m->grad_kc * per_block;
    if (m->gscr_bytes < need) {
      rc = dev_alloc(m, &m->gscr, need);
      m->gscr_bytes = rc ? 0 : need;
    }
  } else if (!m->Sig) {
    rc = dev_alloc(m, &m->Sig, (size_t)m->C * m->T * DP * DP * es);
  }
  if (!rc && !m->sgu) rc = dev_alloc(m, &m->sgu, nbC * (2 * DP * DP + DP) * es);
  if (!rc && !m->gpart) rc = dev_alloc(m, &m->gpart, nbC * (2 * DP * DP + DP) * es);
  if (!rc && !m->opart) rc = dev_alloc(m, (void**)&m->opart, nbC * sizeof(double));
  if (!rc && !m->s0) rc = dev_alloc(m, &m->s0, (size_t)m->C * (DP * DP + DP) * es);
  if (rc) return rc;
  return m->ops->loglik_grad(m, ytilde, logZ, g_mu, g_Phi, g_cholSigma, g_delta, m->stream);
}

int aux_set_grad_memory(aux_model* m, uint64_t max_bytes) {
  if (!m) return AUX_E_INVALID_ARG;
  if (m->fact || wide(m)) return AUX_E_UNSUPPORTED;
  m->grad_mem = (size_t)max_bytes;
  return AUX_OK;
}

int aux_get_status(aux_model* m, int32_t* per_chain_status) {
  if (!m) return AUX_E_INVALID_ARG;
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return AUX_E_CUDA;
  std::vector<int32_t> st(m->C);
  if (cudaMemcpy(st.data(), m->status, m->C * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return AUX_E_CUDA;
  if (cudaMemset(m->status, 0, m->C * sizeof(int32_t)) != cudaSuccess) return AUX_E_CUDA;
  int first = AUX_OK;
  for (int c = 0; c < m->C; ++c) {
    int code = AUX_OK;
    if (st[c] & 1) code = AUX_E_NOT_PD;
    else if (st[c] & 2) code = AUX_E_NONFINITE;
    if (per_chain_status) per_chain_status[c] = code;
    if (first == AUX_OK) first = code;
  }
  return first;
}

int aux_set_profiling(aux_model* m, int32_t enable) {
  if (!m) return AUX_E_INVALID_ARG;
  m->profiling = enable != 0;
  return AUX_OK;
}

int aux_read_profile(aux_model* m, double* ms_per_kind, int32_t* launches_per_kind, int32_t n_kinds) {
  if (!m || n_kinds < 0 || (n_kinds > 0 && (!ms_per_kind || !launches_per_kind)))
    return AUX_E_INVALID_ARG;
  for (int k = 0; k < n_kinds; ++k) { ms_per_kind[k] = 0.0; launches_per_kind[k] = 0; }
  int rc = AUX_OK;
  for (auto& r : m->recs) {
    float ms = 0.0f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess)
      rc = AUX_E_CUDA;
    if (r.kind < n_kinds) { ms_per_kind[r.kind] += ms; launches_per_kind[r.kind] += r.n; }
    m->pool.push_back(r);
  }
  m->recs.clear();
  return rc;
}

void aux_free_model(aux_model* m) { release(m); }

}  // extern "C"
