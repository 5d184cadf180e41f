// aux_kernels.cuh — kernels of one auxiliary Kalman MH step (Algorithm 2 with
// Gaussian dynamics, first-order linearisation, Sigma_t = I).
//
// Per step, for C chains of T states in dimension d (padded to DP <= 32):
//   k_linearise          v_t = grad log h(y_t|x_t), u_t = x_t + sqrt(delta/2) eps_t,
//                        ytilde_t = u_t + (delta/2) v_t                    (Eq. (2.7))
//   parallel filter      blocked associative scan of the filtering elements
//                        (Appendix A.2.1): each block of L steps is reduced
//                        with the operator (k_filter_reduce, in a form
//                        specialised to raw elements), the block
//                        aggregates are scanned with Hillis-Steele rounds
//                        (the Hillis-Steele algorithm of Appendix A.2.1, k_filter_scan_level), and each block
//                        then applies its elements in order from the incoming
//                        prefix (k_filter_apply), which also emits the
//                        predictive log-likelihood terms (Kalman filter algorithm, Appendix A.1) and
//                        the backward elements (G_t, U_t) of Eq. (A.14).
//   backward scan        the (G, U) suffix scan of Proposition A.1, blocked the
//                        same way (block aggregates are built in k_filter_apply,
//                        k_sample_backward applies them), fused with the
//                        linearisation at x* and the MH partial sums.
//   reverse filter       the same filter on ytilde* (log-likelihood terms only).
//   k_mh, k_commit       log alpha and the MH test; x <- x* for the accepted chains.
//
// The element operator is evaluated in a Cholesky form: with C_i = U U^T and
// N = I + U^T J_j U = L L^T (SPD, eigenvalues >= 1), B = U L^{-T}:
//   C_ij = (A_j B)(A_j B)^T + C_j,           A_ij = A_j A_i - (A_j B)(B^T J_j A_i),
//   b_ij = A_j b_i + (A_j B) B^T r + b_j,    r = eta_j - J_j b_i,
//   eta_ij = A_i^T (r - J_j B B^T r) + eta_i,
//   J_ij = A_i^T J_j A_i - (B^T J_j A_i)^T (B^T J_j A_i) + J_i,
// which equals the operator with M = I + C_i J_j (M^{-1} = I - B B^T J_j) and
// keeps C symmetric positive definite by construction.
#pragma once
#include "aux_device.cuh"
#include "aux_internal.h"

namespace auxk {

template <typename Real> struct KP {
  int C, nT, d, DP, L, nb;
  Real r;        // delta / 2
  Real sqrt_r;   // sqrt(delta / 2)
  int emis, y_per_chain;
  int fdiag;     // F is diagonal: F C, F C F^T and F A are elementwise
  uint64_t seed;
  const Real *F, *Q, *P0, *m0, *b, *Ryinv;  // [DP*DP] / [DP], zero padded
  const Real* y;                             // [T][d] or [C][T][d]
  const uint8_t* mask;                       // [T] or null
  int32_t* status_iter;                      // [C], this step's status bits
  int order;                                 // proposal: 1 first order, 2 second order
  const Real* rho;   // [C][T][d] diagonal pseudo-observation variance (second order), or null: r
  const double* delta_dev;   // adapted delta on the device ([4] words, refresh_delta), or null: r and sqrt_r as given
  const uint64_t* iter_dev;  // MCMC iteration on the device (graph replay), or null: as passed
  // time-varying dynamics (AUX_DYN_TIME_VARYING; per-chain path, dense F): the
  // transition into x_t is (F_{t-1}, b_{t-1}, Q_{t-1}), stored per transition in
  // the shared-memory slot layout (row stride Lay::LD), F^T beside F; null: F, b, Q
  int tv;
  const Real *Ftv, *FTtv, *Qtv, *btv;   // [T-1][DP * LD] x 3, [T-1][VEC]
};

// the dynamics of transition tt (into x_{tt+1}): the CTA's model slots, or the
// time-varying stacks
template <typename Real, int DP> struct Dyn {
  const Real *F, *FT, *Q, *b;
};
template <typename Real, int DP>
__device__ __forceinline__ Dyn<Real, DP> dyn_at(const KP<Real>& p, int tt, const Real* sF, const Real* sFT,
                                                const Real* sQ, const Real* sb) {
  if (!p.tv) return Dyn<Real, DP>{sF, sFT, sQ, sb};
  constexpr long MAT = Lay<Real, DP>::MAT, VEC = Lay<Real, DP>::VEC;
  return Dyn<Real, DP>{p.Ftv + tt * MAT, p.FTtv + tt * MAT, p.Qtv + tt * MAT, p.btv + tt * VEC};
}

// the MCMC iteration that keys the Philox streams of this step
template <typename Real>
__device__ __forceinline__ uint64_t iter_of(const KP<Real>& p, uint64_t iter) {
  return p.iter_dev ? *p.iter_dev : iter;
}

// advance the device iteration counter (last launch of an MCMC iteration)
static __global__ void k_iter_next(uint64_t* iter_dev) {
  pdl_wait();
  pdl_trigger();
  *iter_dev += 1;
}

// With on-device delta adaptation the kernels take r = delta / 2 and sqrt(r)
// from device memory, written by k_adapt_delta of the previous iteration as
// four words: delta, r and sqrt(r) in FP64, and (r, sqrt r) rounded to FP32,
// so that no kernel spends FP64 operations (a sqrt is a dozen) on them.
template <typename Real>
__device__ __forceinline__ void refresh_delta(KP<Real>& p) {
  if (p.delta_dev) {
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

// the four device words of delta (see refresh_delta)
__device__ __forceinline__ void store_delta_words(double* w, double delta) {
  const double r = 0.5 * delta, sr = sqrt(r);
  w[0] = delta;
  w[1] = r;
  w[2] = sr;
  *reinterpret_cast<float2*>(w + 3) = make_float2((float)r, (float)sr);
}

// the lane's diagonal entry of the pseudo-observation covariance at (chain, t)
template <typename Real>
__device__ __forceinline__ Real obs_var(const KP<Real>& p, int c, int t, int lane) {
  if (lane >= p.d) return (Real)0;
  return p.rho ? p.rho[((long)c * p.nT + t) * p.d + lane] : p.r;
}

enum : int { ST_NOT_PD = 1, ST_NONFINITE = 2 };

enum : int {
  APPLY_EPI = 1,       // backward elements G_t, U_t and their block aggregates
  APPLY_STORE_Q = 2,   // store per-step quadratic form and log-determinant
  APPLY_REV_DIFF = 4,  // accumulate log-likelihood differences against stored terms
  APPLY_LOGZ = 8,      // accumulate log-likelihood terms
  APPLY_SMOOTH = 16    // noise-free U_t and Sigma_t stored (RTS smoother quantities)
};

template <typename Real, int DP> struct Sizes {
  static constexpr int MAT = Lay<Real, DP>::MAT;
  static constexpr int VEC = Lay<Real, DP>::VEC;
  static constexpr int ES = 3 * DP * DP + 2 * DP;   // global element: A, C, J, b, eta

  static constexpr size_t SMEM_MAX = 227 * 1024;
  static constexpr size_t MODEL = (3 * MAT + 2 * VEC) * sizeof(Real);   // F, F^T, Q, b, diag F
  static constexpr int cap(size_t fixed, size_t per_warp, int want) {
    return (SMEM_MAX - fixed) / per_warp >= (size_t)want ? want : (int)((SMEM_MAX - fixed) / per_warp);
  }
  // phase 1: SA SC SX SY SW SL + 5 vectors
  static constexpr int RED_WARP_ELEMS = 6 * MAT + 5 * VEC;
  static constexpr int RED_WPC = cap(MODEL, RED_WARP_ELEMS * sizeof(Real), 8);
  static constexpr size_t RED_SMEM = MODEL + RED_WPC * RED_WARP_ELEMS * sizeof(Real);
  // phase 2: SA SC SU S2 S3 S4 SAe SCe SJe + 9 vectors
  static constexpr int SCAN_WARP_ELEMS = 9 * MAT + 9 * VEC;
  static constexpr int SCAN_WPC = cap(0, SCAN_WARP_ELEMS * sizeof(Real), 8);
  static constexpr size_t SCAN_SMEM = SCAN_WPC * SCAN_WARP_ELEMS * sizeof(Real);
  // phase 3: SP SX SL SLR SY SG + 8 vectors
  static constexpr int APP_WARP_ELEMS = 6 * MAT + 8 * VEC;
  static constexpr int APP_WPC = cap(MODEL, APP_WARP_ELEMS * sizeof(Real), 8);
  static constexpr size_t APP_SMEM = MODEL + APP_WPC * APP_WARP_ELEMS * sizeof(Real);
  // backward sampler
  static constexpr int BWD_WPC = 8;
  static constexpr size_t BWD_SMEM = (MAT + BWD_WPC * 3 * VEC) * sizeof(Real);
  static_assert(RED_WPC >= 1 && SCAN_WPC >= 1 && APP_WPC >= 1, "shared memory budget");
};

// Diagonal of the Hessian of log h(y_t | x_t) at coordinate i (0 where t is not
// observed): SV -y_i^2 exp(-x_i) / 2; linear-Gaussian -(R_y^{-1})_ii (R_y diagonal).
template <typename Real>
__device__ __forceinline__ Real second_order_hess(const KP<Real>& p, Real yi, int i, Real xi, int t) {
  if (p.mask && !p.mask[t]) return (Real)0;
  if (p.emis == AUX_EMIS_SV) return (Real)-0.5 * yi * yi * exp(-xi);
  return -p.Ryinv[i * p.DP + i];
}

// ---------------------------------------------------------------------------
// k_linearise: A1 + A2 at the current state.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void k_linearise(KP<Real> p, const Real* __restrict__ x, Real* __restrict__ u,
                            Real* __restrict__ v, Real* __restrict__ yt, Real* __restrict__ rho,
                            uint64_t iter) {
  refresh_delta(p);
  const long n = (long)p.C * p.nT * p.d;
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % p.d);
    const long ct = idx / p.d;
    const int t = (int)(ct % p.nT);
    const int c = (int)(ct / p.nT);
    const Real* xr = x + ct * p.d;
    const Real* yr = p.y + (p.y_per_chain ? ct : (long)t) * p.d;
    Real vi = 0;
    if (!p.mask || p.mask[t]) {
      if (p.emis == AUX_EMIS_SV) {
        vi = (Real)-0.5 + (Real)0.5 * yr[i] * yr[i] * exp(-xr[i]);
      } else {
        Real acc = 0;
        for (int j = 0; j < p.d; ++j) acc = fma(p.Ryinv[i * p.DP + j], yr[j] - xr[j], acc);
        vi = acc;
      }
    }
    const Real e = philox_normal<Real>(p.seed, (uint32_t)c, iter_of(p, iter), PURPOSE_AUX, (uint32_t)t, i);
    const Real ui = xr[i] + p.sqrt_r * e;
    u[idx] = ui;
    v[idx] = vi;
    if (p.order == 2) {
      // second order (Eqs. (2.8)-(2.9)): Omega = (I / r - Lambda)^{-1}, omega = Omega (u / r + v - Lambda x)
      const Real li = second_order_hess(p, yr[i], i, xr[i], t);
      const Real om = (Real)1 / ((Real)1 / p.r - li);
      rho[idx] = om;
      yt[idx] = om * (ui / p.r + vi - li * xr[i]);
    } else {
      yt[idx] = ui + p.r * vi;
    }
    if (t == 0 && i == 0) p.status_iter[c] = 0;
  }
}

// ---------------------------------------------------------------------------
// Element operator a_i (x) a_j in Cholesky form (see the header comment), in
// three parts so that the matrix parts and the per-chain vector part can run
// on different warps (combine_general runs all three on one warp).
// Aggregate i: SA (A), SC (C), jreg (row `lane` of J), vb, veta  (in/out).
// Element j:   SAe, SCe, SJe slots and vbe, vetae vectors (read only).
// Scratch: SU, S2, S3, S4 slots, vt (4 vectors), vdiag.
// ---------------------------------------------------------------------------

// matrix part 1: U = chol(C_i) (rows in SU), N = I + U^T J_j U, B = U L_N^{-T}
// (rows in S2), P = A_j B (transposed in S3)
template <typename Real, int DP>
__device__ void combine_matrix_1(const Real* SC, const Real* SAe, const Real* SJe, Real* SU,
                                 Real* S2, Real* S3, Real* S4, Real* vdiag, int d, int lane,
                                 int* bad) {
  constexpr int LD = Lay<Real, DP>::LD;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  __syncwarp();
  {
    Real a[DP];
    ld_row<Real, DP>(SC, row, a);
    chol_ur<Real, DP>(a, S2, SU, nullptr, vdiag, nullptr, d, lane, bad);
  }
  {
    Real t1[DP];
    mm_row<Real, DP>(SJe + row * LD, SU, t1);
    st_row<Real, DP>(S3, row, t1, act);
  }
  __syncwarp();
  {
    Real n[DP];
    mm_col<Real, DP>(SU, row, S3, n);
#pragma unroll
    for (int j = 0; j < DP; ++j) n[j] += (j == lane) ? (Real)1 : (Real)0;
    chol_ur<Real, DP>(n, S4, nullptr, nullptr, vdiag, nullptr, d, lane, bad);
  }
  {
    Real r[DP];
    ld_row<Real, DP>(SU, row, r);
    fsolve_rot<Real, DP, false>(S4, vdiag, r, S2, lane);
  }
  __syncwarp();
  {
    Real pr[DP];
    mm_row<Real, DP>(SAe + row * LD, S2, pr);
    __syncwarp();
    st_col<Real, DP>(S3, row, pr, act);
  }
  __syncwarp();
}

// vector part (one chain): r = eta_j - J_j b_i, s = B^T r, b_new = A_j b_i + P s + b_j,
// w = B s, rq = r - J_j w, eta_new = A_i^T rq + eta_i. Reads SJe, S2 (B), SAe, S3 (P^T),
// SA (A_i, before matrix part 2 overwrites it); writes vb, veta (via the vt scratch).
template <typename Real, int DP>
__device__ void combine_vectors(const Real* SA, const Real* SAe, const Real* SJe, const Real* S2,
                                const Real* S3, Real* vb, Real* veta, const Real* vbe,
                                const Real* vetae, Real* vt, int lane) {
  constexpr int VEC = Lay<Real, DP>::VEC, LD = Lay<Real, DP>::LD;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  Real* vr = vt;
  Real* vs = vt + VEC;
  Real* vw = vt + 2 * VEC;
  Real* vrq = vt + 3 * VEC;
  const Real ri = vetae[row] - dot_row_vec<Real, DP>(SJe + row * LD, vb);
  __syncwarp();
  if (act) vr[lane] = ri;
  __syncwarp();
  {
    const Real si = dot_col_vec<Real, DP>(S2, row, vr);
    if (act) vs[lane] = si;
  }
  __syncwarp();
  const Real bnew = dot_row_vec<Real, DP>(SAe + row * LD, vb) +
                    dot_col_vec<Real, DP>(S3, row, vs) + vbe[row];
  {
    const Real wi = dot_row_vec<Real, DP>(S2 + row * LD, vs);
    if (act) vw[lane] = wi;
  }
  __syncwarp();
  {
    const Real rqi = ri - dot_row_vec<Real, DP>(SJe + row * LD, vw);
    if (act) vrq[lane] = rqi;
  }
  __syncwarp();
  const Real etanew = dot_col_vec<Real, DP>(SA, row, vrq) + veta[row];
  __syncwarp();
  if (act) {
    vb[lane] = bnew;
    veta[lane] = etanew;
  }
  __syncwarp();
}

// matrix part 2: X1 = J_j A_i, Z = B^T X1, J_new = A_i^T X1 - Z^T Z + J_i,
// A_new = A_j A_i - P Z (-> SA), C_new = P P^T + C_j (-> SC), J symmetrised.
template <typename Real, int DP>
__device__ void combine_matrix_2(Real* SA, Real* SC, Real (&jreg)[DP], const Real* SAe,
                                 const Real* SCe, const Real* SJe, Real* SU, const Real* S2,
                                 const Real* S3, Real* S4, int lane) {
  constexpr int LD = Lay<Real, DP>::LD;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  {
    Real x1[DP];
    mm_row<Real, DP>(SJe + row * LD, SA, x1);
    __syncwarp();
    st_row<Real, DP>(S4, row, x1, act);
  }
  __syncwarp();
  {
    Real z[DP];
    mm_col<Real, DP>(S2, row, S4, z);
    __syncwarp();
    st_row<Real, DP>(SU, row, z, act);
  }
  __syncwarp();
  mm_col<Real, DP, true>(SA, row, S4, jreg);
  mm_col<Real, DP, true, true>(SU, row, SU, jreg);
  __syncwarp();
  {
    Real an[DP];
    mm_row<Real, DP>(SAe + row * LD, SA, an);
    mm_col<Real, DP, true, true>(S3, row, SU, an);
    __syncwarp();
    st_row<Real, DP>(SA, row, an, act);
  }
  {
    Real cn[DP];
    ld_row<Real, DP>(SCe, row, cn);
    mm_col<Real, DP, true>(S3, row, S3, cn);
    st_row<Real, DP>(S4, row, jreg, act);
    __syncwarp();
    st_row<Real, DP>(SC, row, cn, act);
  }
  {
    Real jc[DP];
    ld_col<Real, DP>(S4, row, jc);
#pragma unroll
    for (int j = 0; j < DP; ++j) jreg[j] = (Real)0.5 * (jreg[j] + jc[j]);
  }
  __syncwarp();
}

template <typename Real, int DP>
__device__ void combine_general(Real* SA, Real* SC, Real (&jreg)[DP], Real* vb, Real* veta,
                                const Real* SAe, const Real* SCe, const Real* SJe,
                                const Real* vbe, const Real* vetae, Real* SU, Real* S2, Real* S3,
                                Real* S4, Real* vt, Real* vdiag, int d, int lane, int* bad) {
  combine_matrix_1<Real, DP>(SC, SAe, SJe, SU, S2, S3, S4, vdiag, d, lane, bad);
  combine_vectors<Real, DP>(SA, SAe, SJe, S2, S3, vb, veta, vbe, vetae, vt, lane);
  combine_matrix_2<Real, DP>(SA, SC, jreg, SAe, SCe, SJe, SU, S2, S3, S4, lane);
}

// symmetrise a register row through a slot: r <- (r + column of the stored matrix) / 2
template <typename Real, int DP>
__device__ __forceinline__ void symmetrise_store(Real* S, Real (&r)[DP], int lane) {
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  __syncwarp();
  st_row<Real, DP>(S, row, r, act);
  __syncwarp();
  Real c[DP];
  ld_col<Real, DP>(S, row, c);
#pragma unroll
  for (int j = 0; j < DP; ++j) r[j] = (Real)0.5 * (r[j] + c[j]);
  __syncwarp();
}

// CTA-shared model rows: F, F^T, Q (slots) and b
template <typename Real, int DP>
__device__ __forceinline__ void load_model_slots(const KP<Real>& p, Real* sF, Real* sFT, Real* sQ,
                                                 Real* sb) {
  constexpr int LD = Lay<Real, DP>::LD;
  for (int q = threadIdx.x; q < DP * DP; q += blockDim.x) {
    const int i = q / DP, j = q % DP;
    sF[i * LD + j] = p.F[q];
    sFT[j * LD + i] = p.F[q];
    sQ[i * LD + j] = p.Q[q];
  }
  if (threadIdx.x < DP) {
    sb[threadIdx.x] = p.b[threadIdx.x];
    sb[Lay<Real, DP>::VEC + threadIdx.x] = p.F[threadIdx.x * DP + threadIdx.x];   // diag F
  }
}

// global element <-> warp slots
template <typename Real, int DP>
__device__ __forceinline__ void store_element(Real* g, const Real* SA, const Real* SC,
                                              const Real (&jreg)[DP], const Real* vb,
                                              const Real* veta, int lane) {
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  Real r[DP];
  ld_row<Real, DP>(SA, row, r);
  if (act) st_vec<Real, DP>(g + row * DP, r);
  ld_row<Real, DP>(SC, row, r);
  if (act) st_vec<Real, DP>(g + DP * DP + row * DP, r);
  if (act) st_vec<Real, DP>(g + 2 * DP * DP + row * DP, jreg);
  if (act) {
    g[3 * DP * DP + lane] = vb[lane];
    g[3 * DP * DP + DP + lane] = veta[lane];
  }
}

template <typename Real, int DP>
__device__ __forceinline__ void load_element(const Real* g, Real* SA, Real* SC, Real (&jreg)[DP],
                                             Real* vb, Real* veta, int lane) {
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  Real r[DP];
  ld_vec<Real, DP>(g + row * DP, r);
  st_row<Real, DP>(SA, row, r, act);
  ld_vec<Real, DP>(g + DP * DP + row * DP, r);
  st_row<Real, DP>(SC, row, r, act);
  ld_vec<Real, DP>(g + 2 * DP * DP + row * DP, jreg);
  if (act) {
    vb[lane] = g[3 * DP * DP + lane];
    veta[lane] = g[3 * DP * DP + DP + lane];
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Phase 1: block aggregates a_s (x) ... (x) a_e, one warp per (chain, block).
// Applying the operator to a raw element a_t (t >= 1) is the Kalman recursion
// conditional on the block's entry state x_{s-1}: with the aggregate
// (A, b, C, eta, J) so far,
//   P^p = F C F^T + Q,  m^p = F b + b_dyn,  S = P^p + R = L L^T,
//   Y = L^{-1} P^p,  W = L^{-1} F A,  z = L^{-1} (ytilde_t - m^p),
//   C <- P^p - Y^T Y,  A <- F A - Y^T W,  b <- m^p + Y^T z,
//   J <- J + W^T W,    eta <- eta + W^T z,
// starting from the identity (A = I, b = 0, C = 0, eta = 0, J = 0) so that the
// first step reproduces a_s itself; block 0 starts from the prior (t = 0 uses
// P^p = P0, m^p = m0, A = 0). One Cholesky factorisation per step.
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __launch_bounds__(32 * Sizes<Real, DP>::RED_WPC, 1)
    k_filter_reduce(KP<Real> p, const Real* __restrict__ yt, Real* __restrict__ agg) {
  refresh_delta(p);
  using Z = Sizes<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC, LD = Lay<Real, DP>::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  Real* sF = sm;
  Real* sFT = sF + MAT;
  Real* sQ = sFT + MAT;
  Real* sb = sQ + MAT;
  load_model_slots<Real, DP>(p, sF, sFT, sQ, sb);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = blockIdx.x * Z::RED_WPC + warp;
  if (item >= p.C * p.nb) return;
  const int c = item / p.nb, k = item % p.nb;
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  const Real* sphi = sb + VEC;
  Real* SA = sb + 2 * VEC + warp * Z::RED_WARP_ELEMS;
  Real* SC = SA + MAT;
  Real* SX = SC + MAT;
  Real* SY = SX + MAT;
  Real* SW = SY + MAT;
  Real* SL = SW + MAT;
  Real* vb = SL + MAT;
  Real* veta = vb + VEC;
  Real* vr = veta + VEC;
  Real* vz = vr + VEC;
  Real* vdiag = vz + VEC;
  const Real* ytc = yt + (long)c * p.nT * p.d;
  int bad = 0;
  Real jreg[DP];
  zero<Real, DP>(jreg);
  constexpr int JTR = DP >= 16 ? Tile<Real, DP>::TR : 1, JTC = DP >= 16 ? Tile<Real, DP>::TC : 1;
  Real jtile[JTR][JTC];
#pragma unroll
  for (int i = 0; i < JTR; ++i)
#pragma unroll
    for (int j = 0; j < JTC; ++j) jtile[i][j] = (Real)0;
  {
    Real r[DP];
#pragma unroll
    for (int j = 0; j < DP; ++j) r[j] = (k > 0 && j == lane) ? (Real)1 : (Real)0;
    st_row<Real, DP>(SA, row, r, act);
    zero<Real, DP>(r);
    st_row<Real, DP>(SC, row, r, act);
    if (act) { vb[lane] = (Real)0; veta[lane] = (Real)0; }
  }
  __syncwarp();
  for (int t = s; t <= e; ++t) {
    Real pprow[DP];
    Real mpi;
    if (t == 0) {
      ld_vec<Real, DP>(p.P0 + row * DP, pprow);
      mpi = p.m0[row];
      Real z0[DP];
      zero<Real, DP>(z0);
      st_row<Real, DP>(SX, row, z0, act);          // F A = 0 for the prior
    } else if (p.fdiag) {
      // diagonal F: P^p_ij = C_ij phi_i phi_j + Q_ij, (F A)_ij = phi_i A_ij
      Real cr[DP], ph[DP], qr[DP], ar[DP];
      ld_row<Real, DP>(SC, row, cr);
      ld_vec<Real, DP>(sphi, ph);
      ld_row<Real, DP>(sQ, row, qr);
      ld_row<Real, DP>(SA, row, ar);
      const Real phi = sphi[row];
#pragma unroll
      for (int j = 0; j < DP; ++j) {
        pprow[j] = fma(cr[j], phi * ph[j], qr[j]);
        ar[j] *= phi;
      }
      mpi = phi * vb[row] + sb[row];
      __syncwarp();
      st_row<Real, DP>(SX, row, ar, act);
    } else {
      const Dyn<Real, DP> dy = dyn_at<Real, DP>(p, t - 1, sF, sFT, sQ, sb);
      Real xr[DP];
      mm_row<Real, DP>(dy.F + row * LD, SC, xr);      // X = F C
      __syncwarp();
      st_row<Real, DP>(SX, row, xr, act);
      __syncwarp();
      mm_row<Real, DP>(SX + row * LD, dy.FT, pprow);  // P^p = X F^T + Q
      Real qr[DP];
      ld_row<Real, DP>(dy.Q, row, qr);
#pragma unroll
      for (int j = 0; j < DP; ++j) pprow[j] += qr[j];
      symmetrise_store<Real, DP>(SY, pprow, lane);
      mpi = dot_row_vec<Real, DP>(dy.F + row * LD, vb) + dy.b[row];
      Real fa[DP];
      mm_row<Real, DP>(dy.F + row * LD, SA, fa);      // F A
      __syncwarp();
      st_row<Real, DP>(SX, row, fa, act);
    }
    __syncwarp();
    {
      Real s_[DP];
      const Real rl = obs_var<Real>(p, c, t, lane);
#pragma unroll
      for (int j = 0; j < DP; ++j) s_[j] = pprow[j] + (j == lane ? rl : (Real)0);
      chol_ur<Real, DP>(s_, SL, nullptr, nullptr, vdiag, nullptr, p.d, lane, &bad);
    }
    const Real rres = (lane < p.d) ? ytc[(long)t * p.d + lane] - mpi : (Real)0;
    if (act) vr[lane] = rres;
    __syncwarp();
    {
      // Y = L^{-1} P^p, W = L^{-1} F A (as columns) and z = L^{-1} r in one pass
      Real r1[DP], r2[DP], rv[DP];
#pragma unroll
      for (int j = 0; j < DP; ++j) r1[j] = pprow[j];
      ld_col<Real, DP>(SX, row, r2);
      ld_vec<Real, DP>(vr, rv);
      fsolve_multi<Real, DP, true>(SL, vdiag, r1, SY, r2, SW, rv, vz, lane);
    }
    __syncwarp();
    if constexpr (DP >= 16) {
      // register-tiled: C = P^p - Y^T Y, A = F A - Y^T W, J += W^T W
      st_row<Real, DP>(SC, row, pprow, act);
      __syncwarp();
      mm_tile_to_slot<Real, DP, true, true>(SY, SY, SC, SC, lane);
      mm_tile_to_slot<Real, DP, true, true>(SY, SW, SX, SA, lane);
      mm_tile_regs<Real, DP, true, false>(SW, SW, jtile, lane);
    } else {
      Real cn[DP];
#pragma unroll
      for (int j = 0; j < DP; ++j) cn[j] = pprow[j];
      mm_col<Real, DP, true, true>(SY, row, SY, cn);
      st_row<Real, DP>(SC, row, cn, act);
      Real an[DP];
      ld_row<Real, DP>(SX, row, an);
      mm_col<Real, DP, true, true>(SY, row, SW, an);
      st_row<Real, DP>(SA, row, an, act);
      mm_col<Real, DP, true>(SW, row, SW, jreg);
    }
    const Real bnew = mpi + dot_col_vec<Real, DP>(SY, row, vz);
    const Real etanew = veta[row] + dot_col_vec<Real, DP>(SW, row, vz);
    __syncwarp();
    if (act) {
      vb[lane] = bnew;
      veta[lane] = etanew;
    }
    __syncwarp();
  }
  if constexpr (DP >= 16) {
    __syncwarp();
    tile_store<Real, DP>(SY, jtile, lane);
    __syncwarp();
    ld_row<Real, DP>(SY, row, jreg);
  }
  store_element<Real, DP>(agg + (long)item * Z::ES, SA, SC, jreg, vb, veta, lane);
  if (bad && lane == 0) atomicOr(&p.status_iter[c], ST_NOT_PD);
}

// ---------------------------------------------------------------------------
// Phase 2: one Hillis-Steele round over the block aggregates of each chain
// (the prefix-sum algorithm of Appendix A.2.1):
// out_k = in_{k-off} (x) in_k for k >= off, else out_k = in_k.
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __launch_bounds__(32 * Sizes<Real, DP>::SCAN_WPC, 1)
    k_filter_scan_level(KP<Real> p, const Real* __restrict__ in, Real* __restrict__ out, int off) {
  using Z = Sizes<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = blockIdx.x * Z::SCAN_WPC + warp;
  if (item >= p.C * p.nb) return;
  const int c = item / p.nb, k = item % p.nb;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  Real* g_out = out + (long)item * Z::ES;
  const Real* g_in = in + (long)item * Z::ES;
  if (k < off) {
    for (int q = row; q < Z::ES / DP; q += DP) {
      if (!act) break;
      Real r[DP];
      ld_vec<Real, DP>(g_in + q * DP, r);
      st_vec<Real, DP>(g_out + q * DP, r);
    }
    return;
  }
  Real* SA = sm + warp * Z::SCAN_WARP_ELEMS;
  Real* SC = SA + MAT;
  Real* SU = SC + MAT;
  Real* S2 = SU + MAT;
  Real* S3 = S2 + MAT;
  Real* S4 = S3 + MAT;
  Real* SAe = S4 + MAT;
  Real* SCe = SAe + MAT;
  Real* SJe = SCe + MAT;
  Real* vb = SJe + MAT;
  Real* veta = vb + VEC;
  Real* vbe = veta + VEC;
  Real* vetae = vbe + VEC;
  Real* vt = vetae + VEC;
  Real* vdiag = vt + 4 * VEC;
  int bad = 0;
  Real jreg[DP], je[DP];
  load_element<Real, DP>(in + (long)(item - off) * Z::ES, SA, SC, jreg, vb, veta, lane);
  load_element<Real, DP>(g_in, SAe, SCe, je, vbe, vetae, lane);
  st_row<Real, DP>(SJe, row, je, act);
  __syncwarp();
  combine_general<Real, DP>(SA, SC, jreg, vb, veta, SAe, SCe, SJe, vbe, vetae, SU, S2, S3, S4, vt,
                            vdiag, p.d, lane, &bad);
  store_element<Real, DP>(g_out, SA, SC, jreg, vb, veta, lane);
  if (bad && lane == 0) atomicOr(&p.status_iter[c], ST_NOT_PD);
}

// ---------------------------------------------------------------------------
// Phase 3: per block, apply the elements in order from the incoming prefix
// (a marginal N(m^f_{s-1}, P^f_{s-1})): the Kalman filter algorithm of
// Appendix A.1 on the block, giving m^f_t, P^f_t and the predictive terms.
// With APPLY_EPI it also forms (G_t, U_t) of Eq. (A.14) and the block's
// backward aggregate (G_s ... G_e, U_s + G_s U_{s+1} + ...). The predicted
// covariance P^p_{t+1} is factorised once for both uses (G_t needs its
// factor, the update at t+1 needs that of P^p_{t+1} + R): a dual Cholesky.
// ---------------------------------------------------------------------------
// A range of scan blocks for the kernels that can run on part of the blocks
// (the gradient's recompute-not-store path): blocks k_lo .. k_lo + k_cnt - 1
// of every chain (k_cnt = 0: all blocks), with the per-step backward arrays
// (G_t, Sigma_t, U_t) of (c, t) at index c * cs + t - t_lo (cs = 0: nT), so that a
// chunk of blocks fills a scratch of C * cs steps instead of C * T.
struct BlockRange {
  int k_lo = 0, k_cnt = 0;
  long t_lo = 0, cs = 0;
  __device__ __forceinline__ int count(int nb) const { return k_cnt ? k_cnt : nb; }
  __device__ __forceinline__ void item(int it, int nb, int& c, int& k) const {
    const int n = count(nb);
    c = it / n;
    k = k_lo + it % n;
  }
  __device__ __forceinline__ long ct(int c, int t, int nT) const { return (long)c * (cs ? cs : nT) + (t - t_lo); }
};

template <typename Real> struct ApplyArgs {
  const Real* yt;
  const Real* prefix;   // inclusive block prefixes [C][nb][ES] (marginals), null if nb == 1
  int flags;
  Real* G;              // [C][T][DP*DP]
  Real* U;              // [C][T][DP]
  Real* gum;            // [C][nb][DP*DP] block aggregates G_s ... G_e
  Real* guv;            // [C][nb][DP]    block aggregates U_s + G_s U_{s+1} + ...
  double* fq;           // [C][T]
  double* fld;          // [C][T]
  double* lz_part;      // [C][nb]
  Real* mf;             // [C][T][d] or null
  Real* Pf;             // [C][T][d][d] or null
  const Real* eps;      // [C][T][d] or null
  uint64_t iter;
  Real* Sig;            // [C][T][DP*DP] backward covariances (APPLY_SMOOTH) or null
  BlockRange rg;        // blocks to run; indexing of G, U, Sig
};

template <typename Real, int DP>
__global__ void __launch_bounds__(32 * Sizes<Real, DP>::APP_WPC, 1)
    k_filter_apply(KP<Real> p, ApplyArgs<Real> a) {
  refresh_delta(p);
  using Z = Sizes<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC, LD = Lay<Real, DP>::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  Real* sF = sm;
  Real* sFT = sF + MAT;
  Real* sQ = sFT + MAT;
  Real* sb = sQ + MAT;
  load_model_slots<Real, DP>(p, sF, sFT, sQ, sb);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  const int item = blockIdx.x * Z::APP_WPC + warp;
  if (item >= p.C * a.rg.count(p.nb)) return;
  int c, k;
  a.rg.item(item, p.nb, c, k);
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  const Real* sphi = sb + VEC;
  Real* SP = sb + 2 * VEC + warp * Z::APP_WARP_ELEMS;
  Real* SX = SP + MAT;
  Real* SL = SX + MAT;
  Real* SLR = SL + MAT;
  Real* SY = SLR + MAT;
  Real* SG = SY + MAT;
  Real* vm = SG + MAT;
  Real* vmp = vm + VEC;
  Real* vr = vmp + VEC;
  Real* vz = vr + VEC;
  Real* veps = vz + VEC;
  Real* vU = veps + VEC;
  Real* vdA = vU + VEC;
  Real* vdB = vdA + VEC;
  const Real* ytc = a.yt + (long)c * p.nT * p.d;
  const bool epi = a.flags & APPLY_EPI;
  int bad = 0;
  double lz_acc = 0.0;
  const double half_dlog2pi = 0.5 * p.d * 1.8378770664093454835606594728112;
  Real pprow[DP];     // row of P^p_t
  Real ghat[DP];      // row of the running backward aggregate G_s ... G_t
  Real uhat = 0;
#pragma unroll
  for (int j = 0; j < DP; ++j) ghat[j] = (j == lane) ? (Real)1 : (Real)0;

  // X = F P^f (slot SX), P^p = X F^T + Q (symmetrised, pprow), m^p = F m^f + b (vmp),
  // with the dynamics of transition tt
  auto predict = [&](int tt) {
    if (p.fdiag) {
      Real pr[DP], ph[DP], qr[DP];
      ld_row<Real, DP>(SP, row, pr);
      ld_vec<Real, DP>(sphi, ph);
      ld_row<Real, DP>(sQ, row, qr);
      const Real phi = sphi[row];
      const Real mpi = phi * vm[row] + sb[row];
#pragma unroll
      for (int j = 0; j < DP; ++j) {
        pprow[j] = fma(pr[j], phi * ph[j], qr[j]);
        pr[j] *= phi;                                   // X = F P^f
      }
      __syncwarp();
      st_row<Real, DP>(SX, row, pr, act);
      if (act) vmp[lane] = mpi;
      __syncwarp();
      return;
    }
    const Dyn<Real, DP> dy = dyn_at<Real, DP>(p, tt, sF, sFT, sQ, sb);
    Real xr[DP];
    mm_row<Real, DP>(dy.F + row * LD, SP, xr);
    const Real mpi = dot_row_vec<Real, DP>(dy.F + row * LD, vm) + dy.b[row];
    __syncwarp();
    st_row<Real, DP>(SX, row, xr, act);
    if (act) vmp[lane] = mpi;
    __syncwarp();
    mm_row<Real, DP>(SX + row * LD, dy.FT, pprow);
    Real qr[DP];
    ld_row<Real, DP>(dy.Q, row, qr);
#pragma unroll
    for (int j = 0; j < DP; ++j) pprow[j] += qr[j];
    symmetrise_store<Real, DP>(SY, pprow, lane);
  };

  auto backward_noise = [&](int t) {
    Real ei = 0;
    if (lane < p.d && !(a.flags & APPLY_SMOOTH)) {
      ei = a.eps ? a.eps[((long)c * p.nT + t) * p.d + lane]
                 : philox_normal<Real>(p.seed, (uint32_t)c, iter_of(p, a.iter), PURPOSE_BACKWARD, (uint32_t)t, lane);
    }
    __syncwarp();
    if (act) veps[lane] = ei;
    __syncwarp();
  };

  // G row in SX (row-major), U_t -> global and the running aggregate
  auto store_backward = [&](int t, Real ui) {
    Real grow[DP];
    ld_row<Real, DP>(SX, row, grow);
    if (act) {
      st_vec<Real, DP>(a.G + a.rg.ct(c, t, p.nT) * DP * DP + row * DP, grow);
      a.U[a.rg.ct(c, t, p.nT) * DP + lane] = ui;
      vU[lane] = ui;
    }
    __syncwarp();
    {
      Real uu[DP];
      ld_vec<Real, DP>(vU, uu);
      uhat += dot_rr<Real, DP>(ghat, uu);
    }
    st_row<Real, DP>(SY, row, ghat, act);
    __syncwarp();
    mm_row<Real, DP>(SY + row * LD, SX, ghat);
    __syncwarp();
  };

  // epilogue for state t, after P^p_{t+1} has been factorised (LS in SL, LR in SLR,
  // inverse diagonal in vdA); uses X = F P^f_t (SX), m^p_{t+1} (vmp), m^f_t (vm), P^f_t (SP):
  // Y = L_p^{-1} X, Sigma_t = P^f - Y^T Y, G_t^T = L_p^{-T} Y, U_t = m^f - G m^p + chol(Sigma) eps.
  auto epilogue = [&](int t) {
    {
      Real rr[DP];
      ld_col<Real, DP>(SX, row, rr);
      fsolve_rot<Real, DP, true>(SL, vdA, rr, SY, lane);   // SY = Y (columns)
    }
    __syncwarp();
    Real sig[DP];
    if constexpr (DP >= 16) {
      mm_tile_to_slot<Real, DP, true, true>(SY, SY, SP, SL, lane);   // Sigma = P^f - Y^T Y
      __syncwarp();
      ld_row<Real, DP>(SL, row, sig);
    } else {
      ld_row<Real, DP>(SP, row, sig);
      mm_col<Real, DP, true, true>(SY, row, SY, sig);
    }
    if ((a.flags & APPLY_SMOOTH) && act)
      st_vec<Real, DP>(a.Sig + a.rg.ct(c, t, p.nT) * DP * DP + row * DP, sig);
    {
      Real rr[DP];
      ld_col<Real, DP>(SY, row, rr);
      bsolve_rot<Real, DP>(SLR, vdA, rr, SX, lane);       // SX = G (rows); X is dead
    }
    backward_noise(t);
    const Real le = chol_ur<Real, DP>(sig, SL, nullptr, nullptr, vdA, veps, p.d, lane, &bad);
    const Real ui = vm[row] - dot_row_vec<Real, DP>(SX + row * LD, vmp) + le;
    store_backward(t, ui);
  };

  // measurement update at t from (vmp, pprow), with the factor of P^p + R in SG / vdB
  auto update = [&](int t) {
    const Real rres = (lane < p.d) ? ytc[(long)t * p.d + lane] - vmp[lane] : (Real)0;
    __syncwarp();
    if (act) vr[lane] = rres;
    __syncwarp();
    {
      // Y_s = L_S^{-1} P^p (columns of SY) and z = L_S^{-1} r in one pass
      Real r1[DP], rv[DP];
#pragma unroll
      for (int j = 0; j < DP; ++j) r1[j] = pprow[j];
      ld_vec<Real, DP>(vr, rv);
      fsolve_multi<Real, DP, false>(SG, vdB, r1, SY, r1, nullptr, rv, vz, lane);
    }
    __syncwarp();
    const Real mfi = vmp[row] + dot_col_vec<Real, DP>(SY, row, vz);
    Real qz;
    {
      Real zz[DP];
      ld_vec<Real, DP>(vz, zz);
      qz = dot_rr<Real, DP>(zz, zz);
    }
    Real lg = (lane < p.d) ? -log(vdB[lane]) : (Real)0;
    lg = warp_sum<Real>(lg);
    Real pf[DP];
    if constexpr (DP >= 16) {
      __syncwarp();
      st_row<Real, DP>(SP, row, pprow, act);
      __syncwarp();
      mm_tile_to_slot<Real, DP, true, true>(SY, SY, SP, SP, lane);   // P^f = P^p - Y_s^T Y_s
      if (act) vm[lane] = mfi;
      __syncwarp();
      ld_row<Real, DP>(SP, row, pf);
    } else {
#pragma unroll
      for (int j = 0; j < DP; ++j) pf[j] = pprow[j];
      mm_col<Real, DP, true, true>(SY, row, SY, pf);
      __syncwarp();
      st_row<Real, DP>(SP, row, pf, act);
      if (act) vm[lane] = mfi;
      __syncwarp();
    }
    const double q = (double)qz, ld = 2.0 * (double)lg;
    const long ct = (long)c * p.nT + t;
    if (lane == 0) {
      if (a.flags & APPLY_STORE_Q) { a.fq[ct] = q; a.fld[ct] = ld; }
      if (a.flags & APPLY_REV_DIFF) lz_acc += -0.5 * ((a.fld[ct] - ld) + (a.fq[ct] - q));
      if (a.flags & APPLY_LOGZ) lz_acc += -(half_dlog2pi + 0.5 * (ld + q));
    }
    if (a.mf && lane < p.d) a.mf[ct * p.d + lane] = mfi;
    if (a.Pf && lane < p.d) {
      for (int j = 0; j < p.d; ++j) a.Pf[(ct * p.d + lane) * p.d + j] = pf[j];
    }
  };

  // factor of S = P^p + R_t only (SG / vdB)
  auto factor_S = [&](int t) {
    Real s_[DP];
    const Real rl = obs_var<Real>(p, c, t, lane);
#pragma unroll
    for (int j = 0; j < DP; ++j) s_[j] = pprow[j] + (j == lane ? rl : (Real)0);
    chol_ur<Real, DP>(s_, SG, nullptr, nullptr, vdB, nullptr, p.d, lane, &bad);
  };

  // ---- block start
  if (k == 0) {
    ld_vec<Real, DP>(p.P0 + row * DP, pprow);
    if (act) vmp[lane] = p.m0[lane];
    __syncwarp();
  } else {
    const Real* pre = a.prefix + ((long)c * p.nb + (k - 1)) * Z::ES;
    Real r[DP];
    ld_vec<Real, DP>(pre + DP * DP + row * DP, r);        // C of the prefix = P^f_{s-1}
    st_row<Real, DP>(SP, row, r, act);
    if (act) vm[lane] = pre[3 * DP * DP + lane];          // b of the prefix = m^f_{s-1}
    __syncwarp();
    predict(s - 1);
  }
  factor_S(s);
  update(s);
  for (int t = s + 1; t <= e; ++t) {
    predict(t - 1);
    if (epi) {
      Real a_[DP], s_[DP];
      const Real rl = obs_var<Real>(p, c, t, lane);
#pragma unroll
      for (int j = 0; j < DP; ++j) {
        a_[j] = pprow[j];
        s_[j] = pprow[j] + (j == lane ? rl : (Real)0);
      }
      chol_rot2<Real, DP>(a_, SL, SLR, vdA, s_, SG, vdB, p.d, lane, &bad);
      epilogue(t - 1);
    } else {
      factor_S(t);
    }
    update(t);
  }
  if (epi) {
    if (e < p.nT - 1) {
      predict(e);
      Real a_[DP];
#pragma unroll
      for (int j = 0; j < DP; ++j) a_[j] = pprow[j];
      chol_ur<Real, DP>(a_, SL, nullptr, SLR, vdA, nullptr, p.d, lane, &bad);
      epilogue(e);
    } else {
      // last state: G_{T-1} = 0, U_{T-1} = m^f + chol(P^f) eps
      Real pf[DP];
      ld_row<Real, DP>(SP, row, pf);
      if ((a.flags & APPLY_SMOOTH) && act)
        st_vec<Real, DP>(a.Sig + a.rg.ct(c, e, p.nT) * DP * DP + row * DP, pf);
      backward_noise(e);
      const Real le = chol_ur<Real, DP>(pf, SL, nullptr, nullptr, vdA, veps, p.d, lane, &bad);
      Real g0[DP];
      zero<Real, DP>(g0);
      __syncwarp();
      st_row<Real, DP>(SX, row, g0, act);
      __syncwarp();
      store_backward(e, vm[row] + le);
    }
    if (act) {
      st_vec<Real, DP>(a.gum + ((long)c * p.nb + k) * DP * DP + row * DP, ghat);
      a.guv[((long)c * p.nb + k) * DP + lane] = uhat;
    }
  }
  if ((a.flags & (APPLY_REV_DIFF | APPLY_LOGZ)) && lane == 0) a.lz_part[(long)c * p.nb + k] = lz_acc;
  if (bad && lane == 0) atomicOr(&p.status_iter[c], ST_NOT_PD);
}

// ---------------------------------------------------------------------------
// Backward sampling (Proposition A.1), blocked: x*_{s_{k+1}} from the later
// blocks' aggregates, then x*_t = G_t x*_{t+1} + U_t down the block.
// With mh != 0 also: v*_t, ytilde*_t = u_t + (delta/2) v*_t and the MH partial
// sum of gamma(x*) - gamma(x) + sum_t [v.(u - x*) + r|v|^2/2] - [v*.(u - x) + r|v*|^2/2].
// ---------------------------------------------------------------------------
template <typename Real> struct BackArgs {
  const Real* G;        // G_t at G + c * g_cs + t * DP*DP
  const Real* U;        // [C][T][DP]
  const Real* gum;      // block aggregate matrices at gum + c * gm_cs + k * DP*DP
  const Real* guv;      // [C][nb][DP]
  long g_cs, gm_cs;     // chain strides (0 when the matrices are shared by all chains)
  Real* xs;
  int mh;
  const Real* x;
  const Real* u;
  const Real* v;
  Real* yts;
  double* mh_part;
  // second-order proposal: forward pseudo-observations and variances, reverse variances out
  const Real* yt;
  const Real* rho;
  Real* rhos;
};

// The per-step inputs of mh_step_terms for the lane's coordinate (lane < d):
// x_t, u_t, v_t and y_t, loaded separately so that callers can fetch them early.
template <typename Real> struct MhIn {
  Real xo, ui, vi, yi;
  Real om, rh;   // second order: omega_t and Omega_t (diagonal) at the current state
};

template <typename Real>
__device__ __forceinline__ MhIn<Real> mh_load(const KP<Real>& p, const BackArgs<Real>& a, long ct,
                                              int t, int lane) {
  MhIn<Real> q{(Real)0, (Real)0, (Real)0, (Real)0, (Real)0, (Real)1};
  if (lane < p.d) {
    const long idx = ct * p.d + lane;
    q.xo = a.x[idx];
    q.ui = a.u[idx];
    q.vi = a.v[idx];
    q.yi = p.y[(p.y_per_chain ? ct : (long)t) * p.d + lane];
    if (p.order == 2) {
      q.om = a.yt[idx];
      q.rh = a.rho[idx];
    }
  }
  return q;
}

// The step-t terms of log alpha for the lane's coordinate (simplified form of
// Algorithm 2's ratio): gamma(x*) - gamma(x) + v (u - x*) + (r/2) v^2
// - v* (u - x) - (r/2) v*^2, with v* = grad log h at x*; also writes
// ytilde*_t = u_t + r v*_t. sRy: R_y^{-1} rows (linear-Gaussian emission),
// vxs: a warp-private vector slot. All lanes of the warp call it.
template <typename Real, int DP>
__device__ __forceinline__ void mh_step_terms(const KP<Real>& p, const BackArgs<Real>& a, long ct,
                                              int t, Real xi, const MhIn<Real>& in,
                                              const Real* sRy, Real* vxs, int lane, int row,
                                              TermSum<Real>& acc) {
  const bool act = lane < DP;
  const bool obs = !p.mask || p.mask[t];
  Real vsi = 0;
  if (p.emis == AUX_EMIS_LINEAR_GAUSSIAN) {
    __syncwarp();
    if (act) vxs[lane] = (lane < p.d) ? in.yi - xi : (Real)0;
    __syncwarp();
    Real ry[DP];
    ld_row<Real, DP>(sRy, row, ry);
    vsi = dot_rv<Real, DP>(ry, vxs);
  }
  if (lane < p.d) {
    const Real xo = in.xo, ui = in.ui, vi = in.vi, yi = in.yi;
    Real gdiff = 0;
    if (obs) {
      if (p.emis == AUX_EMIS_SV) {
        vsi = (Real)-0.5 + (Real)0.5 * yi * yi * exp(-xi);
        gdiff = (Real)-0.5 * (xi - xo) - (Real)0.5 * yi * yi * (exp(-xi) - exp(-xo));
      } else {
        gdiff = (Real)-0.5 * (yi - xi) * vsi + (Real)0.5 * (yi - xo) * vi;
      }
    } else {
      vsi = 0;
    }
    if (p.order == 2) {
      // log N(u; x*, r) - log N(u; x, r) + log N(omega*; x, Omega*) - log N(omega; x*, Omega)
      const Real ls = second_order_hess(p, yi, lane, xi, t);
      const Real rs = (Real)1 / ((Real)1 / p.r - ls);
      const Real oms = rs * (ui / p.r + vsi - ls * xi);
      const double du = (double)(ui - xo), dus = (double)(ui - xi);
      const double d1 = (double)(oms - xo), d0 = (double)(in.om - xi);
      acc.add_f64((double)gdiff + (du * du - dus * dus) / (2.0 * (double)p.r) +
                  0.5 * (log((double)in.rh) - log((double)rs)) - d1 * d1 / (2.0 * (double)rs) +
                  d0 * d0 / (2.0 * (double)in.rh));
      a.yts[ct * p.d + lane] = oms;
      a.rhos[ct * p.d + lane] = rs;
    } else {
      const Real fwd = vi * (ui - xi) + (Real)0.5 * p.r * vi * vi;
      const Real rev = vsi * (ui - xo) + (Real)0.5 * p.r * vsi * vsi;
      if constexpr (sizeof(Real) == 4) {
        acc.add(gdiff);
        acc.add(fwd);
        acc.add(-rev);
      } else {
        acc.add((double)gdiff + (double)fwd - (double)rev);
      }
      a.yts[ct * p.d + lane] = ui + p.r * vsi;
    }
  }
}

template <typename Real, int DP>
__global__ void __launch_bounds__(32 * Sizes<Real, DP>::BWD_WPC)
    k_sample_backward(KP<Real> p, BackArgs<Real> a) {
  refresh_delta(p);
  using Z = Sizes<Real, DP>;
  constexpr int VEC = Z::VEC, LD = Lay<Real, DP>::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  Real* sRy = sm;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int q = threadIdx.x; q < DP * DP; q += blockDim.x) sRy[(q / DP) * LD + q % DP] = p.Ryinv[q];
  __syncthreads();
  const int item = blockIdx.x * Z::BWD_WPC + warp;
  if (item >= p.C * p.nb) return;
  const int c = item / p.nb, k = item % p.nb;
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  Real* vx = sm + Z::MAT + warp * 3 * VEC;
  Real* vxs = vx + VEC;
  Real xi = 0;
  if (k < p.nb - 1) {
    xi = a.guv[((long)c * p.nb + (p.nb - 1)) * DP + row];
    for (int kk = p.nb - 2; kk > k; --kk) {
      __syncwarp();
      if (act) vx[lane] = xi;
      __syncwarp();
      Real g[DP];
      ld_vec<Real, DP>(a.gum + (long)c * a.gm_cs + (long)kk * DP * DP + row * DP, g);
      xi = dot_rv<Real, DP>(g, vx) + a.guv[((long)c * p.nb + kk) * DP + row];
    }
  }
  TermSum<Real> acc;
  for (int t = e; t >= s; --t) {
    const long ct = (long)c * p.nT + t;
    if (t == p.nT - 1) {
      xi = a.U[ct * DP + row];
    } else {
      __syncwarp();
      if (act) vx[lane] = xi;
      __syncwarp();
      Real g[DP];
      ld_vec<Real, DP>(a.G + (long)c * a.g_cs + (long)t * DP * DP + row * DP, g);
      xi = dot_rv<Real, DP>(g, vx) + a.U[ct * DP + row];
    }
    if (lane < p.d) a.xs[ct * p.d + lane] = xi;
    if (a.mh) mh_step_terms<Real, DP>(p, a, ct, t, xi, mh_load<Real>(p, a, ct, t, lane), sRy, vxs, lane, row, acc);
  }
  if (a.mh) {
    const double sum = warp_sum<double>(acc.value());
    if (lane == 0) a.mh_part[(long)c * p.nb + k] = sum;
  }
}

// ---------------------------------------------------------------------------
// MH test, one CTA per chain: log alpha from the partial sums, the Philox
// uniform of the (chain, iteration), the accept flag for k_commit.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void k_mh(KP<Real> p, const double* __restrict__ mh_part,
                     const double* __restrict__ lz_part, uint64_t iter, uint32_t* acc_count,
                     double* log_alpha, int32_t* status, int32_t* __restrict__ accept,
                     double* __restrict__ la_all) {
  pdl_wait();
  pdl_trigger();
  const int c = blockIdx.x;
  __shared__ double red[32];
  double sacc = 0.0;
  for (int k = threadIdx.x; k < p.nb; k += blockDim.x)
    sacc += mh_part[(long)c * p.nb + k] + lz_part[(long)c * p.nb + k];
  sacc = warp_sum<double>(sacc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sacc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double la = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) la += red[w];
    int st = p.status_iter[c];
    if (!isfinite(la)) st |= ST_NONFINITE;
    const uint4 r = philox_word(p.seed, (uint32_t)c, iter_of(p, iter), PURPOSE_MH, 0, 0);
    const double lu = log(u01<double>(r.x));
    const int acc = (st == 0) && (lu < la);
    accept[c] = acc;
    status[c] |= st;
    la_all[c] = la;
    if (log_alpha) log_alpha[c] = la;
    if (acc_count && acc) acc_count[c] += 1;
  }
}

// ---------------------------------------------------------------------------
// State update x <- x* for the accepted chains, over the whole grid.
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// On-line delta adaptation (Robbins-Monro on log delta): with a_k the mean over
// the chains of min(1, exp(log alpha)) (0 for a non-finite log alpha),
// log delta <- log delta + gain k^{-0.6} (a_k - target), k = 1, 2, ...; log delta
// is kept in [-40, 40]. One CTA.
// ---------------------------------------------------------------------------
static __global__ void k_adapt_delta(const double* __restrict__ la_all, int C, double* __restrict__ delta,
                                     int* __restrict__ count, double target, double gain) {
  pdl_wait();
  pdl_trigger();
  __shared__ double red[32];
  double s = 0.0;
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    const double la = la_all[c];
    s += isfinite(la) ? exp(fmin(0.0, la)) : 0.0;
  }
  s = warp_sum<double>(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) a += red[w];
    a /= (double)C;
    const int k = *count + 1;
    double ld = log(*delta) + gain * pow((double)k, -0.6) * (a - target);
    ld = fmin(40.0, fmax(-40.0, ld));
    store_delta_words(delta, exp(ld));
    *count = k;
  }
}

template <typename Real>
__global__ void k_commit(KP<Real> p, Real* __restrict__ x, const Real* __restrict__ xs,
                         const int32_t* __restrict__ accept) {
  pdl_wait();
  pdl_trigger();
  const long per_chain = (long)p.nT * p.d;
  const long n = (long)p.C * per_chain;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    if (accept[i / per_chain]) x[i] = xs[i];
}

}  // namespace auxk
