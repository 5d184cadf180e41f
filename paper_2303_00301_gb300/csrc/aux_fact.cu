// aux_fact.cu — the auxiliary Kalman sampler for models whose prior factorises
// over the coordinates (F, Q, P0 diagonal), with the multivariate Student-t
// observation model of Section 4.2, which does not factorise.
//
// With R = (delta/2) I the auxiliary LGSSM of Eq. (2.7) then splits into d_x
// independent one-dimensional LGSSMs (Section 4.2): every filtering, gain and
// backward-sampling quantity is a scalar per coordinate, and the covariance
// recursion (a scalar Riccati recursion per coordinate) does not depend on
// the chain. Layout: coordinates are the fastest index everywhere ([.][T][d]
// paths, [T][d] tables), so the d threads of one (chain, block) read and
// write consecutive words.
//   k_fc_cov     per coordinate, sequentially in t: K'_t = r / S_t, G_t,
//                sqrt(Sigma_t), block prefix products of G, block products
//                of K'_t f (the mean's linear part) and sum log S_t;
//   k_fl_lin     one warp per (chain, t): e = y - x, q = e^T Lambda e,
//                v = (nu + d) Lambda e / (nu + q), u, ytilde, gamma_t;
//   k_fm_reduce / k_fm_cross / k_fm_apply / k_fm_back: the blocked scans of
//                the filter means and of the (G, U) backward sampler
//                (Appendix A.2, Proposition A.1) with one thread per
//                (chain, block, coordinate);
//   k_fl_lin_rev one warp per (chain, t): the gradient at x*, ytilde*, and
//                the MH terms of step t;
//   k_fm_mh      log alpha and the MH test per chain.
#include <cmath>
#include <cstring>
#include <vector>

#include "aux_kernels.cuh"

namespace auxk {
namespace {

template <typename Real> struct FP {
  int C, nT, d, L, nb, y_per_chain;
  Real r, sqrt_r, nu;
  uint64_t seed;
  const Real *f, *b, *q, *p0, *m0;   // [d] diagonal model
  const Real* lam;                   // [d][d] precision of the Student-t scale
  const Real* y;                     // [T][d] or [C][T][d]
  const uint8_t* mask;               // [T] or null
  const double* delta_dev;           // adapted delta, or null
  const uint64_t* iter_dev;          // MCMC iteration on the device, or null
};

template <typename Real>
__device__ __forceinline__ uint64_t fiter(const FP<Real>& p, uint64_t iter) {
  return p.iter_dev ? *p.iter_dev : iter;
}

template <typename Real>
__device__ __forceinline__ void fp_refresh(FP<Real>& p) {
  if (p.delta_dev) {   // the device words of delta (refresh_delta)
    if constexpr (sizeof(Real) == 4) {
      const float2 f = *reinterpret_cast<const float2*>(p.delta_dev + 3);
      p.r = f.x;
      p.sqrt_r = f.y;
    } else {
      p.r = (Real)p.delta_dev[1];
      p.sqrt_r = (Real)p.delta_dev[2];
    }
  }
}

enum { FK = 0, FG, FLS, FGP, NFT };   // per-step tables [NFT][T][d]
enum { FAH = 0, FGH };                // per-block tables [2][nb][d]

// ---------------------------------------------------------------------------
// Covariance pass: the scalar Kalman filter and backward-sampling variances of
// coordinate i (Appendix A.1 with H = 1, R = r), one thread per coordinate.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void k_fc_cov(FP<Real> p, Real* __restrict__ tab, Real* __restrict__ bt,
                         double* __restrict__ ldb) {
  fp_refresh(p);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.d) return;
  const long TD = (long)p.nT * p.d;
  const Real f = p.f[i], q = p.q[i];
  Real Pf = 0, GP = 1, AH = 1;
  double ld = 0.0;
  for (int t = 0; t < p.nT; ++t) {
    const int k = t / p.L;
    const bool start = t == k * p.L;
    const Real Pp = (t == 0) ? p.p0[i] : f * f * Pf + q;
    if (t > 0) {   // G_{t-1} = P^f_{t-1} f / P^p_t, Sigma_{t-1} = P^f_{t-1} - G_{t-1}^2 P^p_t
      const Real G = Pf * f / Pp;
      const Real Sig = Pf - G * G * Pp;
      tab[FG * TD + (long)(t - 1) * p.d + i] = G;
      tab[FLS * TD + (long)(t - 1) * p.d + i] = sqrt(Sig > (Real)0 ? Sig : (Real)0);
      if (start) bt[((long)FGH * p.nb + (k - 1)) * p.d + i] = GP * G;
      else GP *= G;
    }
    if (start) { GP = 1; AH = 1; ld = 0.0; }
    tab[FGP * TD + (long)t * p.d + i] = GP;
    const Real S = Pp + p.r;
    const Real Kp = p.r / S;
    tab[FK * TD + (long)t * p.d + i] = Kp;
    Pf = Pp * Kp;
    ld += log((double)S);
    AH *= Kp * f;
    if (t == min(p.nT, (k + 1) * p.L) - 1) {
      bt[((long)FAH * p.nb + k) * p.d + i] = AH;
      ldb[(long)k * p.d + i] = ld;
    }
  }
  tab[FG * TD + (long)(p.nT - 1) * p.d + i] = 0;
  tab[FLS * TD + (long)(p.nT - 1) * p.d + i] = sqrt(Pf);
  bt[((long)FGH * p.nb + (p.nb - 1)) * p.d + i] = 0;
}

// ---------------------------------------------------------------------------
// Emission gradient at x (one warp per (chain, t)): e = y_t - x_t,
// q = e^T Lambda e, v = (nu + d) Lambda e / (nu + q); the auxiliary draw
// u = x + sqrt(r) eps; ytilde = u + r v; gamma_t = -(nu + d)/2 log(1 + q / nu)
// (up to a constant that cancels in log alpha). Zero where t is not observed.
// ---------------------------------------------------------------------------
template <typename Real>
__device__ __forceinline__ double st_grad(const FP<Real>& p, const Real* __restrict__ xr,
                                         const Real* __restrict__ yr, Real* es, Real* vout, int lane) {
  for (int j = lane; j < p.d; j += 32) es[j] = yr[j] - xr[j];
  __syncwarp();
  double qa = 0.0;
  for (int i = lane; i < p.d; i += 32) {
    const Real* lrow = p.lam + (long)i * p.d;
    Real acc = 0;
    for (int j = 0; j < p.d; ++j) acc = fma(__ldg(lrow + j), es[j], acc);
    vout[i] = acc;                               // (Lambda e)_i, scaled below
    qa += (double)es[i] * (double)acc;
  }
  const double qd = warp_sum<double>(qa);
  const Real sc = (Real)(((double)p.nu + p.d) / ((double)p.nu + qd));
  __syncwarp();
  for (int i = lane; i < p.d; i += 32) vout[i] *= sc;
  __syncwarp();
  return -0.5 * ((double)p.nu + p.d) * log1p(qd / (double)p.nu);
}

template <typename Real>
__global__ void k_fl_lin(FP<Real> p, const Real* __restrict__ x, Real* __restrict__ u,
                         Real* __restrict__ v, Real* __restrict__ yt, double* __restrict__ gam,
                         uint64_t iter) {
  fp_refresh(p);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpc = blockDim.x >> 5;
  Real* es = reinterpret_cast<Real*>(smem_raw) + warp * 2 * p.d;
  Real* vs = es + p.d;
  const long item = (long)blockIdx.x * wpc + warp;
  if (item >= (long)p.C * p.nT) return;
  const int c = (int)(item / p.nT), t = (int)(item % p.nT);
  const long ct = item;
  const Real* xr = x + ct * p.d;
  const Real* yr = p.y + (p.y_per_chain ? ct : (long)t) * p.d;
  const bool obs = !p.mask || p.mask[t];
  double g = 0.0;
  if (obs) g = st_grad<Real>(p, xr, yr, es, vs, lane);
  for (int i = lane; i < p.d; i += 32) {
    const Real vi = obs ? vs[i] : (Real)0;
    const Real ep = philox_normal<Real>(p.seed, (uint32_t)c, fiter(p, iter), PURPOSE_AUX, (uint32_t)t, i);
    const Real ui = xr[i] + p.sqrt_r * ep;
    u[ct * p.d + i] = ui;
    v[ct * p.d + i] = vi;
    yt[ct * p.d + i] = ui + p.r * vi;
  }
  if (lane == 0) gam[ct] = g;
}

// the gradient at x*, ytilde* = u + r v*, and the step-t MH terms
// gamma*_t - gamma_t + sum_i [v_i (u_i - x*_i) + r v_i^2 / 2 - v*_i (u_i - x_i) - r v*_i^2 / 2]
template <typename Real>
__global__ void k_fl_lin_rev(FP<Real> p, const Real* __restrict__ xs, const Real* __restrict__ x,
                             const Real* __restrict__ u, const Real* __restrict__ v,
                             const double* __restrict__ gam, Real* __restrict__ yts,
                             double* __restrict__ mh) {
  fp_refresh(p);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpc = blockDim.x >> 5;
  Real* es = reinterpret_cast<Real*>(smem_raw) + warp * 2 * p.d;
  Real* vs = es + p.d;
  const long item = (long)blockIdx.x * wpc + warp;
  if (item >= (long)p.C * p.nT) return;
  const int t = (int)(item % p.nT);
  const long ct = item;
  const Real* xsr = xs + ct * p.d;
  const Real* yr = p.y + (p.y_per_chain ? ct : (long)t) * p.d;
  const bool obs = !p.mask || p.mask[t];
  double g = 0.0;
  if (obs) g = st_grad<Real>(p, xsr, yr, es, vs, lane);
  double acc = 0.0;
  for (int i = lane; i < p.d; i += 32) {
    const long idx = ct * p.d + i;
    const Real vsi = obs ? vs[i] : (Real)0;
    const Real ui = u[idx], vi = v[idx], xo = x[idx], xi = xsr[i];
    const Real fwd = vi * (ui - xi) + (Real)0.5 * p.r * vi * vi;
    const Real rev = vsi * (ui - xo) + (Real)0.5 * p.r * vsi * vsi;
    acc += (double)fwd - (double)rev;
    yts[idx] = ui + p.r * vsi;
  }
  acc = warp_sum<double>(acc);
  if (lane == 0) mh[ct] = acc + g - gam[ct];
}

// ---------------------------------------------------------------------------
// Filter means, one thread per (chain, block, coordinate); index i fastest.
// ---------------------------------------------------------------------------
struct FItem { int c, k, i, s, e; };
template <typename Real>
__device__ __forceinline__ bool fitem(const FP<Real>& p, FItem& it) {
  const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long)p.C * p.nb * p.d) return false;
  it.i = (int)(id % p.d);
  it.k = (int)((id / p.d) % p.nb);
  it.c = (int)(id / ((long)p.d * p.nb));
  it.s = it.k * p.L;
  it.e = min(p.nT, it.s + p.L) - 1;
  return true;
}

// block-local means from a zero start (block 0 from m0): z[c][k][i] = m^f_e
template <typename Real>
__global__ void k_fm_reduce(FP<Real> p, const Real* __restrict__ tab, const Real* __restrict__ yt,
                            Real* __restrict__ z) {
  fp_refresh(p);
  FItem it;
  if (!fitem(p, it)) return;
  const long TD = (long)p.nT * p.d;
  const Real f = p.f[it.i], b = p.b[it.i];
  Real m = 0;
  for (int t = it.s; t <= it.e; ++t) {
    const Real mp = (t == 0) ? p.m0[it.i] : fma(f, m, b);
    const Real y = yt[((long)it.c * p.nT + t) * p.d + it.i];
    m = y - tab[FK * TD + (long)t * p.d + it.i] * (y - mp);
  }
  z[((long)it.c * p.nb + it.k) * p.d + it.i] = m;
}

// composition over the blocks, one thread per (chain, coordinate):
//   forward:  out[c][k] = m^f_{e_{k-1}} from m^f_{e_k} = AH_k m^f_{e_{k-1}} + z_k;
//   backward: out[c][k] = x*_{e_k + 1} from x*_{s_k} = GH_k x*_{e_k + 1} + Ubar_k.
template <typename Real>
__global__ void k_fm_cross(FP<Real> p, const Real* __restrict__ mats, const Real* __restrict__ in,
                           Real* __restrict__ out, int backward) {
  const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long)p.C * p.d) return;
  const int i = (int)(id % p.d), c = (int)(id / p.d);
  const long cb = (long)c * p.nb;
  if (backward) {
    Real xn = 0;
    for (int k = p.nb - 1; k >= 0; --k) {
      out[(cb + k) * p.d + i] = xn;
      xn = mats[(long)k * p.d + i] * xn + in[(cb + k) * p.d + i];
    }
  } else {
    Real m = in[cb * p.d + i];
    for (int k = 1; k < p.nb; ++k) {
      out[(cb + k) * p.d + i] = m;
      m = mats[(long)k * p.d + i] * m + in[(cb + k) * p.d + i];
    }
  }
}

// means from the true start, likelihood terms, and (APPLY_EPI) the backward
// elements U_t = m^f_t - G_t m^p_{t+1} + sqrt(Sigma_t) eps_t with the block
// aggregate sum_t (G_s ... G_{t-1}) U_t
template <typename Real>
__global__ void k_fm_apply(FP<Real> p, const Real* __restrict__ tab, const double* __restrict__ ldb,
                           const Real* __restrict__ yt, const Real* __restrict__ mstart,
                           const Real* __restrict__ eps, Real* __restrict__ U, Real* __restrict__ ub,
                           double* __restrict__ fq, double* __restrict__ lz, Real* __restrict__ mf,
                           int flags, uint64_t iter) {
  fp_refresh(p);
  FItem it;
  if (!fitem(p, it)) return;
  const long TD = (long)p.nT * p.d;
  const Real f = p.f[it.i], b = p.b[it.i];
  const long cki = ((long)it.c * p.nb + it.k) * p.d + it.i;
  Real mp = (it.k == 0) ? p.m0[it.i] : fma(f, mstart[cki], b);
  double qa = 0.0;
  Real ubar = 0;
  const bool epi = flags & APPLY_EPI;
  for (int t = it.s; t <= it.e; ++t) {
    const long idx = ((long)it.c * p.nT + t) * p.d + it.i;
    const Real y = yt[idx];
    const Real Kp = tab[FK * TD + (long)t * p.d + it.i];
    const Real e = y - mp;
    qa += (double)e * (double)e * (double)Kp;    // e^2 / S_t = e^2 K'_t / r
    const Real m = y - Kp * e;
    if (mf) mf[idx] = m;
    const Real mpn = (t < p.nT - 1) ? fma(f, m, b) : (Real)0;
    if (epi) {
      const Real ep = eps ? eps[idx]
                          : philox_normal<Real>(p.seed, (uint32_t)it.c, fiter(p, iter), PURPOSE_BACKWARD, (uint32_t)t, it.i);
      const Real u = m - tab[FG * TD + (long)t * p.d + it.i] * mpn + tab[FLS * TD + (long)t * p.d + it.i] * ep;
      U[idx] = u;
      ubar = fma(tab[FGP * TD + (long)t * p.d + it.i], u, ubar);
    }
    mp = mpn;
  }
  const double q = qa / (double)p.r;
  if (flags & APPLY_STORE_Q) fq[cki] = q;
  if (flags & APPLY_REV_DIFF) lz[cki] = -0.5 * (fq[cki] - q);
  if (flags & APPLY_LOGZ)
    lz[cki] = -0.5 * ((double)(it.e - it.s + 1) * 1.8378770664093454835606594728112 +
                      ldb[(long)it.k * p.d + it.i] + q);
  if (epi) ub[cki] = ubar;
}

// x*_t = G_t x*_{t+1} + U_t inside each block, from x*_{e+1}
template <typename Real>
__global__ void k_fm_back(FP<Real> p, const Real* __restrict__ tab, const Real* __restrict__ U,
                          const Real* __restrict__ xnext, Real* __restrict__ xs) {
  FItem it;
  if (!fitem(p, it)) return;
  const long TD = (long)p.nT * p.d;
  Real xn = xnext[((long)it.c * p.nb + it.k) * p.d + it.i];
  for (int t = it.e; t >= it.s; --t) {
    const long idx = ((long)it.c * p.nT + t) * p.d + it.i;
    xn = fma(tab[FG * TD + (long)t * p.d + it.i], xn, U[idx]);
    xs[idx] = xn;
  }
}

// per chain: log alpha = sum_t mh_t + sum_{k,i} lz, the MH test (Algorithm 2)
template <typename Real>
__global__ void k_fm_mh(FP<Real> p, const double* __restrict__ mh, const double* __restrict__ lz,
                        uint64_t iter, uint32_t* acc_count, double* log_alpha, int32_t* status,
                        int32_t* __restrict__ accept, double* __restrict__ la_all) {
  const int c = blockIdx.x;
  __shared__ double red[32];
  double s = 0.0;
  for (int t = threadIdx.x; t < p.nT; t += blockDim.x) s += mh[(long)c * p.nT + t];
  const long nz = (long)p.nb * p.d;
  for (long q = threadIdx.x; q < nz; q += blockDim.x) s += lz[(long)c * nz + q];
  s = warp_sum<double>(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double la = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) la += red[w];
    int st = 0;
    if (!isfinite(la)) st |= ST_NONFINITE;
    const uint4 r = philox_word(p.seed, (uint32_t)c, fiter(p, iter), PURPOSE_MH, 0, 0);
    const double lu = log(u01<double>(r.x));
    const int acc = (st == 0) && (lu < la);
    accept[c] = acc;
    status[c] |= st;
    la_all[c] = la;
    if (log_alpha) log_alpha[c] = la;
    if (acc_count && acc) acc_count[c] += 1;
  }
}

template <typename Real>
__global__ void k_fm_commit(long per_chain, long n, Real* __restrict__ x, const Real* __restrict__ xs,
                            const int32_t* __restrict__ accept) {
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x)
    if (accept[q / per_chain]) x[q] = xs[q];
}

__global__ void k_fm_sum(const double* __restrict__ part, long n, double* __restrict__ out) {
  const int c = blockIdx.x;
  __shared__ double red[32];
  double s = 0.0;
  for (long q = threadIdx.x; q < n; q += blockDim.x) s += part[(long)c * n + q];
  s = warp_sum<double>(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) a += red[w];
    out[c] = a;
  }
}

inline int ok(cudaError_t e) { return e == cudaSuccess ? AUX_OK : AUX_E_CUDA; }

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename Real>
struct Fact {
  static FP<Real> params(const aux_model* m) {
    FP<Real> p{};
    p.C = m->C; p.nT = m->T; p.d = m->d; p.L = m->L; p.nb = m->nb; p.y_per_chain = m->y_per_chain;
    p.r = (Real)(0.5 * m->delta); p.sqrt_r = (Real)std::sqrt(0.5 * m->delta); p.nu = (Real)m->nu;
    p.seed = m->seed;
    const Real* base = (const Real*)m->fmodel;
    p.f = base; p.b = base + m->d; p.q = base + 2 * m->d; p.p0 = base + 3 * m->d; p.m0 = base + 4 * m->d;
    p.lam = (const Real*)m->flam;
    p.y = (const Real*)m->y;
    p.mask = m->mask;
    p.delta_dev = m->adapt ? m->delta_dev : nullptr;
    p.iter_dev = nullptr;
    return p;
  }
  static int grid(long n, int bs) { return (int)((n + bs - 1) / bs); }
  static size_t lin_smem(const aux_model* m) { return (size_t)4 * 2 * m->d * sizeof(Real); }

  static void cov(aux_model* m, const FP<Real>& p, cudaStream_t st) {
    ProfScope ps(m, PK_COV_APPLY, st);
    k_fc_cov<Real><<<grid(m->d, 64), 64, 0, st>>>(p, (Real*)m->ftab, (Real*)m->fbt, m->fldb);
  }
  static void ensure_cov(aux_model* m, const FP<Real>& p, cudaStream_t st) {
    if (m->cov_valid && !m->adapt) return;
    cov(m, p, st);
    m->cov_valid = 1;
  }

  // filter on yt: reduce, composition, apply
  static void filter(aux_model* m, const FP<Real>& p, const Real* yt, int flags, const Real* eps,
                     Real* mf, uint64_t iter, cudaStream_t st) {
    const long nk = (long)m->C * m->nb * m->d, nc = (long)m->C * m->d;
    { ProfScope ps(m, PK_REDUCE, st);
      k_fm_reduce<Real><<<grid(nk, 128), 128, 0, st>>>(p, (const Real*)m->ftab, yt, (Real*)m->fz); }
    { ProfScope ps(m, PK_SCAN, st);
      k_fm_cross<Real><<<grid(nc, 128), 128, 0, st>>>(p, (const Real*)m->fbt + (long)FAH * m->nb * m->d,
                                                      (const Real*)m->fz, (Real*)m->fms, 0); }
    { ProfScope ps(m, PK_APPLY, st);
      k_fm_apply<Real><<<grid(nk, 128), 128, 0, st>>>(p, (const Real*)m->ftab, m->fldb, yt,
                                                      (const Real*)m->fms, eps, (Real*)m->U,
                                                      (Real*)m->fub, m->ffq, m->flz, mf, flags, iter); }
  }
  static void backward(aux_model* m, const FP<Real>& p, Real* xs, cudaStream_t st) {
    const long nk = (long)m->C * m->nb * m->d, nc = (long)m->C * m->d;
    ProfScope ps(m, PK_BACKWARD, st, 2);
    k_fm_cross<Real><<<grid(nc, 128), 128, 0, st>>>(p, (const Real*)m->fbt + (long)FGH * m->nb * m->d,
                                                    (const Real*)m->fub, (Real*)m->fz, 1);
    k_fm_back<Real><<<grid(nk, 128), 128, 0, st>>>(p, (const Real*)m->ftab, (const Real*)m->U,
                                                   (const Real*)m->fz, xs);
  }

  static int kalman_step(aux_model* m, void* xv, int n_iters, uint64_t iter0, uint32_t* acc,
                         double* log_alpha, cudaStream_t st) {
    FP<Real> p = params(m);
    if (m->dev_iter) p.iter_dev = m->iter_dev;
    Real* x = (Real*)xv;
    const long CT = (long)m->C * m->T, n = CT * m->d;
    for (int it = 0; it < n_iters; ++it) {
      const uint64_t iter = iter0 + (uint64_t)it;
      ensure_cov(m, p, st);
      { ProfScope ps(m, PK_LINEARISE, st);
        k_fl_lin<Real><<<grid(CT, 4), 128, lin_smem(m), st>>>(p, x, (Real*)m->u, (Real*)m->v,
                                                               (Real*)m->yt, m->fgam, iter); }
      filter(m, p, (const Real*)m->yt, APPLY_EPI | APPLY_STORE_Q, nullptr, nullptr, iter, st);
      backward(m, p, (Real*)m->xs, st);
      { ProfScope ps(m, PK_LINEARISE, st);
        k_fl_lin_rev<Real><<<grid(CT, 4), 128, lin_smem(m), st>>>(
            p, (const Real*)m->xs, x, (const Real*)m->u, (const Real*)m->v, m->fgam, (Real*)m->yts,
            m->fmh); }
      filter(m, p, (const Real*)m->yts, APPLY_REV_DIFF, nullptr, nullptr, iter, st);
      { ProfScope ps(m, PK_MH, st, 2 + (m->adapt ? 1 : 0) + (m->dev_iter ? 1 : 0));
        k_fm_mh<Real><<<m->C, 256, 0, st>>>(p, m->fmh, m->flz, iter, acc, log_alpha, m->status, m->accept,
                                            m->la_all);
        k_fm_commit<Real><<<(int)std::min<long>(grid(n, 256), (long)m->n_sm * 8), 256, 0, st>>>(
            (long)m->T * m->d, n, x, (const Real*)m->xs, m->accept);
        if (m->adapt)
          k_adapt_delta<<<1, 256, 0, st>>>(m->la_all, m->C, m->delta_dev, m->adapt_count, m->adapt_target,
                                           m->adapt_gain);
        if (m->dev_iter) k_iter_next<<<1, 1, 0, st>>>(m->iter_dev);
      }
    }
    return ok(cudaGetLastError());
  }

  static int loglik(aux_model* m, const void* yt, double* logZ, void* mf, cudaStream_t st) {
    const FP<Real> p = params(m);
    ensure_cov(m, p, st);
    filter(m, p, (const Real*)yt, APPLY_LOGZ, nullptr, (Real*)mf, 0, st);
    ProfScope ps(m, PK_SUM, st);
    k_fm_sum<<<m->C, 256, 0, st>>>(m->flz, (long)m->nb * m->d, logZ);
    return ok(cudaGetLastError());
  }

  static int sample_path(aux_model* m, const void* yt, const void* eps, uint64_t iter, void* xs,
                         double* logZ, cudaStream_t st) {
    const FP<Real> p = params(m);
    ensure_cov(m, p, st);
    filter(m, p, (const Real*)yt, APPLY_EPI | APPLY_LOGZ, (const Real*)eps, nullptr, iter, st);
    backward(m, p, (Real*)xs, st);
    if (logZ) {
      ProfScope ps(m, PK_SUM, st);
      k_fm_sum<<<m->C, 256, 0, st>>>(m->flz, (long)m->nb * m->d, logZ);
    }
    return ok(cudaGetLastError());
  }

  static int prepare(const aux_model* m) {
    const size_t sm = lin_smem(m);
    if (sm > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k_fl_lin<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fl_lin_rev<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      return ok(e);
    }
    return AUX_OK;
  }
};

}  // namespace
}  // namespace auxk

int aux_fact_prepare(aux_model* m) {
  return m->dtype == AUX_F32 ? auxk::Fact<float>::prepare(m) : auxk::Fact<double>::prepare(m);
}
int aux_fact_kalman_step(aux_model* m, void* x, int n_iters, uint64_t iter0, uint32_t* acc,
                         double* log_alpha, cudaStream_t st) {
  return m->dtype == AUX_F32 ? auxk::Fact<float>::kalman_step(m, x, n_iters, iter0, acc, log_alpha, st)
                             : auxk::Fact<double>::kalman_step(m, x, n_iters, iter0, acc, log_alpha, st);
}
int aux_fact_loglik(aux_model* m, const void* yt, double* logZ, void* mf, cudaStream_t st) {
  return m->dtype == AUX_F32 ? auxk::Fact<float>::loglik(m, yt, logZ, mf, st)
                             : auxk::Fact<double>::loglik(m, yt, logZ, mf, st);
}
int aux_fact_sample_path(aux_model* m, const void* yt, const void* eps, uint64_t iter, void* xs,
                         double* logZ, cudaStream_t st) {
  return m->dtype == AUX_F32 ? auxk::Fact<float>::sample_path(m, yt, eps, iter, xs, logZ, st)
                             : auxk::Fact<double>::sample_path(m, yt, eps, iter, xs, logZ, st);
}
