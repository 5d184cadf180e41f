// aux_kernels.cuh — kernels of one auxiliary Kalman MH step (Algorithm 2 with
// Gaussian dynamics, first-order linearisation, Sigma_t = I).
//
// Per step, for C chains of T states in dimension d (padded to DP <= 32):
//   k_linearise          v_t = grad log h(y_t|x_t), u_t = x_t + sqrt(delta/2) eps_t,
//                        ytilde_t = u_t + (delta/2) v_t                    (Eq. (2.7))
//   parallel filter      blocked associative scan of the filtering elements
//                        (Appendix A.2.1): each block of L steps is reduced
//                        with the operator (k_filter_reduce), the block
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
//   k_mh                 log alpha, the MH test and the state update.
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
  uint64_t seed;
  const Real *F, *Q, *P0, *m0, *b, *Ryinv;  // [DP*DP] / [DP], zero padded
  const Real* y;                             // [T][d] or [C][T][d]
  const uint8_t* mask;                       // [T] or null
  int32_t* status_iter;                      // [C], this step's status bits
};

enum : int { ST_NOT_PD = 1, ST_NONFINITE = 2 };

enum : int {
  APPLY_EPI = 1,       // backward elements G_t, U_t and their block aggregates
  APPLY_STORE_Q = 2,   // store per-step quadratic form and log-determinant
  APPLY_REV_DIFF = 4,  // accumulate log-likelihood differences against stored terms
  APPLY_LOGZ = 8       // accumulate log-likelihood terms
};

template <typename Real, int DP> struct Sizes {
  static constexpr int MAT = Lay<Real, DP>::MAT;
  static constexpr int VEC = Lay<Real, DP>::VEC;
  static constexpr int ES = 3 * DP * DP + 2 * DP;   // global element: A, C, J, b, eta
  static constexpr int GS = DP * DP + DP;           // global backward aggregate: G, U
  static constexpr size_t SMEM_MAX = 227 * 1024;
  // phase 1
  static constexpr size_t RED_CTA = (5 * MAT + VEC) * sizeof(Real);
  static constexpr size_t RED_WARP = (5 * MAT + 9 * VEC) * sizeof(Real);
  static constexpr int RED_WPC = (SMEM_MAX - RED_CTA) / RED_WARP >= 8 ? 8 : (int)((SMEM_MAX - RED_CTA) / RED_WARP);
  static constexpr size_t RED_SMEM = RED_CTA + RED_WPC * RED_WARP;
  // phase 2
  static constexpr size_t SCAN_WARP = (8 * MAT + 9 * VEC) * sizeof(Real);
  static constexpr int SCAN_WPC = SMEM_MAX / SCAN_WARP >= 4 ? 4 : (int)(SMEM_MAX / SCAN_WARP);
  static constexpr size_t SCAN_SMEM = SCAN_WPC * SCAN_WARP;
  // phase 3
  static constexpr size_t APP_CTA = (3 * MAT + VEC) * sizeof(Real);
  static constexpr size_t APP_WARP = (4 * MAT + 7 * VEC) * sizeof(Real);
  static constexpr int APP_WPC = (SMEM_MAX - APP_CTA) / APP_WARP >= 8 ? 8 : (int)((SMEM_MAX - APP_CTA) / APP_WARP);
  static constexpr size_t APP_SMEM = APP_CTA + APP_WPC * APP_WARP;
  // backward sampler
  static constexpr int BWD_WPC = 8;
  static constexpr size_t BWD_SMEM = (MAT + BWD_WPC * 3 * VEC) * sizeof(Real);
  static_assert(RED_WPC >= 1 && SCAN_WPC >= 1 && APP_WPC >= 1, "shared memory budget");
};

// ---------------------------------------------------------------------------
// k_linearise: A1 + A2 at the current state.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void k_linearise(KP<Real> p, const Real* __restrict__ x, Real* __restrict__ u,
                            Real* __restrict__ v, Real* __restrict__ yt, uint64_t iter) {
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
    const Real e = philox_normal<Real>(p.seed, (uint32_t)c, iter, PURPOSE_AUX, (uint32_t)t, i);
    const Real ui = xr[i] + p.sqrt_r * e;
    u[idx] = ui;
    v[idx] = vi;
    yt[idx] = ui + p.r * vi;
    if (t == 0 && i == 0) p.status_iter[c] = 0;
  }
}

// ---------------------------------------------------------------------------
// Element operator a_i (x) a_j (Cholesky form, see header comment).
// Aggregate i: SA (A), SC (C), jreg (row `lane` of J), vb, veta.
// Element j:   Ae, Ce, Je slots and vbe, vetae vectors (read only).
// Scratch: S2, S3, S4 slots, vt (4 vectors), vdiag.
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__device__ void combine_general(Real* SA, Real* SC, Real (&jreg)[DP], Real* vb, Real* veta,
                                const Real* Ae, const Real* Ce, const Real* Je,
                                const Real* vbe, const Real* vetae, Real* S2, Real* S3,
                                Real* S4, Real* vt, Real* vdiag, int d, int lane, int* bad) {
  constexpr int VEC = Lay<Real, DP>::VEC;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  Real* vr = vt;
  Real* vs = vt + VEC;
  Real* vw = vt + 2 * VEC;
  Real* vrq = vt + 3 * VEC;
  __syncwarp();
  // 1. U = chol(C_i), stored as U^T in SC
  {
    Real a[DP];
    ld_row<Real, DP>(SC, row, a);
    chol_rows<Real, DP>(a, SC, vdiag, d, lane, bad);
  }
  // 2. T1 = J_j U: lane i forms column i of T1, (U^T J_j)_i = (U^T row i) J_j
  //    (J_j symmetric), and stores it as column i, so S2 holds T1 row-major
  Real ut[DP];
  ld_row<Real, DP>(SC, row, ut);
  {
    Real t1c[DP];
    row_mat<Real, DP>(ut, Je, t1c);
    st_col<Real, DP>(S2, row, t1c, act);
  }
  __syncwarp();
  // 3-4. N = I + U^T T1, L = chol(N) -> L^T in S3
  {
    Real n[DP];
    row_mat<Real, DP>(ut, S2, n);
#pragma unroll
    for (int j = 0; j < DP; ++j) n[j] += (j == lane) ? (Real)1 : (Real)0;
    chol_rows<Real, DP>(n, S3, vdiag, d, lane, bad);
  }
  // 5. B = U L^{-T}: row i solves L b^T = (row i of U)^T = column i of U^T
  {
    Real rhs[DP], bro[DP];
    ld_col<Real, DP>(SC, row, rhs);
    fwd_subst<Real, DP>(S3, vdiag, rhs, bro);
    __syncwarp();
    st_row<Real, DP>(S2, row, bro, act);
  }
  __syncwarp();
  // 6. P = A_j B, kept transposed in SC (U^T is dead): row i of P is column i of SC
  {
    Real ae[DP], prow[DP];
    ld_row<Real, DP>(Ae, row, ae);
    row_mat<Real, DP>(ae, S2, prow);
    st_col<Real, DP>(SC, row, prow, act);
  }
  // vector parts: r = eta_j - J_j b_i, s = B^T r, b_new, w = B s, rq = r - J_j w
  Real ri, bnew;
  {
    Real je[DP];
    ld_row<Real, DP>(Je, row, je);
    ri = vetae[row] - dot_rv<Real, DP>(je, vb);
  }
  if (act) vr[lane] = ri;
  __syncwarp();
  {
    Real bcol[DP];
    ld_col<Real, DP>(S2, row, bcol);
    const Real si = dot_rv<Real, DP>(bcol, vr);
    if (act) vs[lane] = si;
  }
  __syncwarp();
  {
    Real ae[DP];
    ld_row<Real, DP>(Ae, row, ae);
    Real prow[DP];
    ld_col<Real, DP>(SC, row, prow);
    bnew = dot_rv<Real, DP>(ae, vb) + dot_rv<Real, DP>(prow, vs) + vbe[row];
  }
  {
    Real bro[DP];
    ld_row<Real, DP>(S2, row, bro);
    const Real wi = dot_rv<Real, DP>(bro, vs);
    if (act) vw[lane] = wi;
  }
  __syncwarp();
  {
    Real je[DP];
    ld_row<Real, DP>(Je, row, je);
    const Real rqi = ri - dot_rv<Real, DP>(je, vw);
    if (act) vrq[lane] = rqi;
  }
  // 7. X1 = J_j A_i -> S3 (L^T is dead)
  {
    Real je[DP], x1[DP];
    ld_row<Real, DP>(Je, row, je);
    row_mat<Real, DP>(je, SA, x1);
    __syncwarp();
    st_row<Real, DP>(S3, row, x1, act);
  }
  __syncwarp();
  // 8. Z = B^T X1 -> S4
  {
    Real bcol[DP], z[DP];
    ld_col<Real, DP>(S2, row, bcol);
    row_mat<Real, DP>(bcol, S3, z);
    st_row<Real, DP>(S4, row, z, act);
  }
  __syncwarp();
  // eta_new and 9. J_new = A_i^T X1 - Z^T Z + J_i (accumulated into jreg; uses the old A_i)
  Real etanew;
  {
    Real acol[DP];
    ld_col<Real, DP>(SA, row, acol);
    etanew = dot_rv<Real, DP>(acol, vrq) + veta[row];
    row_mat<Real, DP, true>(acol, S3, jreg);
  }
  {
    Real zc[DP];
    ld_col<Real, DP>(S4, row, zc);
    row_mat<Real, DP, true, true>(zc, S4, jreg);
  }
  __syncwarp();   // also keeps the scheduler from interleaving steps 9 and 10
  // 10. A_new = A_j A_i - P Z -> SA once every lane is done reading A_i
  {
    Real an[DP];
    {
      Real ae[DP];
      ld_row<Real, DP>(Ae, row, ae);
      row_mat<Real, DP>(ae, SA, an);
    }
    {
      Real prow[DP];
      ld_col<Real, DP>(SC, row, prow);
      row_mat<Real, DP, true, true>(prow, S4, an);
    }
    __syncwarp();
    st_row<Real, DP>(SA, row, an, act);
  }
  // 11. C_new = P P^T + C_j (P^T is in SC); J symmetrised through S3
  st_row<Real, DP>(S3, row, jreg, act);
  __syncwarp();
  {
    Real cn[DP];
    {
      Real prow[DP];
      ld_col<Real, DP>(SC, row, prow);
      ld_row<Real, DP>(Ce, row, cn);
      row_mat<Real, DP, true>(prow, SC, cn);
    }
    Real jc[DP];
    ld_col<Real, DP>(S3, row, jc);
#pragma unroll
    for (int j = 0; j < DP; ++j) jreg[j] = (Real)0.5 * (jreg[j] + jc[j]);
    __syncwarp();
    st_row<Real, DP>(SC, row, cn, act);
  }
  if (act) {
    vb[lane] = bnew;
    veta[lane] = etanew;
  }
  __syncwarp();
}

// symmetrise a slot in place: S <- (S + S^T) / 2, given own row in r
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
  st_row<Real, DP>(S, row, r, act);
  __syncwarp();
}

// Matrix parts of the elements (one warp, written to global memory once per
// filter pass): for t >= 1, S = Q + R, K = Q S^{-1}, H = F^T S^{-1},
// A_e = F - K F, C_e = Q - K Q, J_e = H F (vector parts b_e = b + K (ytilde_t - b),
// eta_e = H (ytilde_t - b)); for t = 0, K0 = P0 (P0 + R)^{-1}, C0 = P0 - K0 P0.
// Layout of the template: [A_e][C_e][J_e][K][H][C0][K0], DP*DP each, row-major.
template <typename Real, int DP>
__global__ void __launch_bounds__(32) k_element_template(KP<Real> p, Real* __restrict__ tmpl) {
  constexpr int MAT = Lay<Real, DP>::MAT, VEC = Lay<Real, DP>::VEC;
  __shared__ __align__(16) Real W1[MAT], W2[MAT], W3[MAT], vdiag[VEC];
  const int lane = threadIdx.x & 31;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  int bad = 0;
  Real* gAe = tmpl;
  Real* gCe = gAe + DP * DP;
  Real* gJe = gCe + DP * DP;
  Real* gK = gJe + DP * DP;
  Real* gH = gK + DP * DP;
  Real* gC0 = gH + DP * DP;
  Real* gK0 = gC0 + DP * DP;
  Real q[DP], f[DP];
  ld_vec<Real, DP>(p.Q + row * DP, q);
  ld_vec<Real, DP>(p.F + row * DP, f);
  {
    Real s_[DP];
#pragma unroll
    for (int j = 0; j < DP; ++j) s_[j] = q[j] + ((j == lane && j < p.d) ? p.r : (Real)0);
    chol_rows<Real, DP>(s_, W1, vdiag, p.d, lane, &bad);
  }
  Real kr[DP], hr[DP];
  {
    Real rhs[DP], y[DP];
#pragma unroll
    for (int j = 0; j < DP; ++j) rhs[j] = q[j];
    fwd_subst<Real, DP>(W1, vdiag, rhs, y);
    bwd_subst<Real, DP>(W1, vdiag, y, kr);
#pragma unroll
    for (int k = 0; k < DP; ++k) rhs[k] = p.F[k * DP + row];
    fwd_subst<Real, DP>(W1, vdiag, rhs, y);
    bwd_subst<Real, DP>(W1, vdiag, y, hr);
  }
  if (act) { st_vec<Real, DP>(gK + row * DP, kr); st_vec<Real, DP>(gH + row * DP, hr); }
  __syncwarp();
  st_row<Real, DP>(W1, row, f, act);
  st_row<Real, DP>(W2, row, q, act);
  __syncwarp();
  {
    Real a_[DP];
#pragma unroll
    for (int j = 0; j < DP; ++j) a_[j] = f[j];
    row_mat<Real, DP, true, true>(kr, W1, a_);
    if (act) st_vec<Real, DP>(gAe + row * DP, a_);
  }
  {
    Real cc[DP];
#pragma unroll
    for (int j = 0; j < DP; ++j) cc[j] = q[j];
    row_mat<Real, DP, true, true>(kr, W2, cc);
    symmetrise_store<Real, DP>(W3, cc, lane);
    if (act) st_vec<Real, DP>(gCe + row * DP, cc);
  }
  {
    Real jj[DP];
    row_mat<Real, DP>(hr, W1, jj);
    symmetrise_store<Real, DP>(W3, jj, lane);
    if (act) st_vec<Real, DP>(gJe + row * DP, jj);
  }
  // t = 0
  Real pr[DP];
  ld_vec<Real, DP>(p.P0 + row * DP, pr);
  {
    Real s_[DP];
#pragma unroll
    for (int j = 0; j < DP; ++j) s_[j] = pr[j] + ((j == lane && j < p.d) ? p.r : (Real)0);
    __syncwarp();
    chol_rows<Real, DP>(s_, W1, vdiag, p.d, lane, &bad);
  }
  Real k0[DP];
  {
    Real rhs[DP], y[DP];
#pragma unroll
    for (int j = 0; j < DP; ++j) rhs[j] = pr[j];
    fwd_subst<Real, DP>(W1, vdiag, rhs, y);
    bwd_subst<Real, DP>(W1, vdiag, y, k0);
  }
  if (act) st_vec<Real, DP>(gK0 + row * DP, k0);
  __syncwarp();
  st_row<Real, DP>(W2, row, pr, act);
  __syncwarp();
  {
    Real cc[DP];
#pragma unroll
    for (int j = 0; j < DP; ++j) cc[j] = pr[j];
    row_mat<Real, DP, true, true>(k0, W2, cc);
    symmetrise_store<Real, DP>(W3, cc, lane);
    if (act) st_vec<Real, DP>(gC0 + row * DP, cc);
  }
  if (bad && lane < p.C) {
    for (int c = lane; c < p.C; c += 32) atomicOr(&p.status_iter[c], ST_NOT_PD);
  }
}

// vector parts of element t >= 1 into vbe, vetae (uses vr as scratch)
template <typename Real, int DP>
__device__ __forceinline__ void element_vectors(const KP<Real>& p, const Real* ytc, int t,
                                                const Real* tK, const Real* tH, const Real* tb,
                                                Real* vbe, Real* vetae, Real* vr, int lane) {
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  const Real ri = (lane < p.d) ? ytc[(long)t * p.d + lane] - tb[lane] : (Real)0;
  __syncwarp();
  if (act) vr[lane] = ri;
  __syncwarp();
  Real kr[DP], hr[DP];
  ld_row<Real, DP>(tK, row, kr);
  ld_row<Real, DP>(tH, row, hr);
  const Real be = tb[row] + dot_rv<Real, DP>(kr, vr);
  const Real ee = dot_rv<Real, DP>(hr, vr);
  if (act) {
    vbe[lane] = be;
    vetae[lane] = ee;
  }
  __syncwarp();
}

// The t = 0 element: A = 0, J = 0, eta = 0, C = C0, b = m0 + K0 (ytilde_0 - m0).
template <typename Real, int DP>
__device__ void element_zero(const KP<Real>& p, const Real* ytc, const Real* gC0, const Real* gK0,
                             Real* SA, Real* SC, Real (&jreg)[DP], Real* vb, Real* veta, Real* vr,
                             int lane) {
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  Real r[DP];
  ld_vec<Real, DP>(gC0 + row * DP, r);
  st_row<Real, DP>(SC, row, r, act);
  zero<Real, DP>(r);
  st_row<Real, DP>(SA, row, r, act);
#pragma unroll
  for (int j = 0; j < DP; ++j) jreg[j] = (Real)0;
  const Real ri = (lane < p.d) ? ytc[lane] - p.m0[lane] : (Real)0;
  __syncwarp();
  if (act) vr[lane] = ri;
  __syncwarp();
  ld_vec<Real, DP>(gK0 + row * DP, r);
  const Real b0 = p.m0[row] + dot_rv<Real, DP>(r, vr);
  if (act) {
    vb[lane] = b0;
    veta[lane] = (Real)0;
  }
  __syncwarp();
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
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __launch_bounds__(32 * Sizes<Real, DP>::RED_WPC, 1)
    k_filter_reduce(KP<Real> p, const Real* __restrict__ tmpl, const Real* __restrict__ yt,
                    Real* __restrict__ agg) {
  using Z = Sizes<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  Real* tAe = sm;
  Real* tCe = tAe + MAT;
  Real* tJe = tCe + MAT;
  Real* tK = tJe + MAT;
  Real* tH = tK + MAT;
  Real* tb = tH + MAT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Real* SA = tb + VEC + warp * (5 * MAT + 9 * VEC);
  Real* SC = SA + MAT;
  Real* S2 = SC + MAT;
  Real* S3 = S2 + MAT;
  Real* S4 = S3 + MAT;
  Real* vb = S4 + MAT;
  Real* veta = vb + VEC;
  Real* vbe = veta + VEC;
  Real* vetae = vbe + VEC;
  Real* vt = vetae + VEC;
  Real* vdiag = vt + 4 * VEC;
  int bad = 0;
  for (int q = threadIdx.x; q < 5 * DP * DP; q += blockDim.x) {
    const int m = q / (DP * DP), rr = (q / DP) % DP, cc = q % DP;
    tAe[m * MAT + rr * Lay<Real, DP>::LD + cc] = tmpl[q];
  }
  if (threadIdx.x < DP) tb[threadIdx.x] = p.b[threadIdx.x];
  __syncthreads();
  const int item = blockIdx.x * Z::RED_WPC + warp;
  if (item >= p.C * p.nb) return;
  const int c = item / p.nb, k = item % p.nb;
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  const Real* ytc = yt + (long)c * p.nT * p.d;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  Real jreg[DP];
  if (k == 0) {
    element_zero<Real, DP>(p, ytc, tmpl + 5 * DP * DP, tmpl + 6 * DP * DP, SA, SC, jreg, vb, veta,
                           vt, lane);
  } else {
    Real r[DP];
    ld_row<Real, DP>(tAe, row, r);
    st_row<Real, DP>(SA, row, r, act);
    ld_row<Real, DP>(tCe, row, r);
    st_row<Real, DP>(SC, row, r, act);
    ld_row<Real, DP>(tJe, row, jreg);
    element_vectors<Real, DP>(p, ytc, s, tK, tH, tb, vb, veta, vt, lane);
  }
  for (int t = s + 1; t <= e; ++t) {
    element_vectors<Real, DP>(p, ytc, t, tK, tH, tb, vbe, vetae, vt, lane);
    combine_general<Real, DP>(SA, SC, jreg, vb, veta, tAe, tCe, tJe, vbe, vetae, S2, S3, S4, vt,
                              vdiag, p.d, lane, &bad);
  }
  store_element<Real, DP>(agg + (long)item * Z::ES, SA, SC, jreg, vb, veta, lane);
  if (bad && lane == 0) atomicOr(&p.status_iter[c], ST_NOT_PD);
}

// ---------------------------------------------------------------------------
// Phase 2: one Hillis-Steele round over the block aggregates of each chain
// (Hillis-Steele algorithm, Appendix A.2.1): out_k = in_{k-off} (x) in_k for k >= off, else out_k = in_k.
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
  Real* SA = sm + warp * (8 * MAT + 9 * VEC);
  Real* SC = SA + MAT;
  Real* S2 = SC + MAT;
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
  combine_general<Real, DP>(SA, SC, jreg, vb, veta, SAe, SCe, SJe, vbe, vetae, S2, S3, S4, vt,
                            vdiag, p.d, lane, &bad);
  store_element<Real, DP>(g_out, SA, SC, jreg, vb, veta, lane);
  if (bad && lane == 0) atomicOr(&p.status_iter[c], ST_NOT_PD);
}

// ---------------------------------------------------------------------------
// Phase 3: per block, apply the elements in order from the incoming prefix
// (a marginal N(m^f_{s-1}, P^f_{s-1})): this is the Kalman recursion of
// the Kalman filter algorithm (Appendix A.1) on the block, giving m^f_t, P^f_t and the predictive terms.
// With APPLY_EPI it also forms (G_t, U_t) of Eq. (A.14) and the block's
// backward aggregate (G_s ... G_e, U_s + G_s U_{s+1} + ...).
// ---------------------------------------------------------------------------
template <typename Real> struct ApplyArgs {
  const Real* yt;
  const Real* prefix;   // inclusive block prefixes [C][nb][ES] (marginals), null if nb == 1
  int flags;
  Real* G;              // [C][T][DP*DP]
  Real* U;              // [C][T][DP]
  Real* gu;             // [C][nb][GS]
  double* fq;           // [C][T]
  double* fld;          // [C][T]
  double* lz_part;      // [C][nb]
  Real* mf;             // [C][T][d] or null
  Real* Pf;             // [C][T][d][d] or null
  const Real* eps;      // [C][T][d] or null
  uint64_t iter;
};

template <typename Real, int DP>
__global__ void __launch_bounds__(32 * Sizes<Real, DP>::APP_WPC, 1)
    k_filter_apply(KP<Real> p, ApplyArgs<Real> a) {
  using Z = Sizes<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  Real* sF = sm;
  Real* sFT = sF + MAT;
  Real* sQ = sFT + MAT;
  Real* sb = sQ + MAT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  for (int q = threadIdx.x; q < DP * DP; q += blockDim.x) {
    sF[(q / DP) * Lay<Real, DP>::LD + q % DP] = p.F[q];
    sFT[(q % DP) * Lay<Real, DP>::LD + q / DP] = p.F[q];
    sQ[(q / DP) * Lay<Real, DP>::LD + q % DP] = p.Q[q];
  }
  if (threadIdx.x < DP) sb[threadIdx.x] = p.b[threadIdx.x];
  __syncthreads();
  const int item = blockIdx.x * Z::APP_WPC + warp;
  if (item >= p.C * p.nb) return;
  const int c = item / p.nb, k = item % p.nb;
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  Real* SP = sb + VEC + warp * (4 * MAT + 7 * VEC);
  Real* SX = SP + MAT;
  Real* SL = SX + MAT;
  Real* SY = SL + MAT;
  Real* vm = SY + MAT;
  Real* vmp = vm + VEC;
  Real* vr = vmp + VEC;
  Real* veps = vr + VEC;
  Real* vU = veps + VEC;
  Real* vdiag = vU + VEC;
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

  // X = F P^f (slot SX), P^p = X F^T + Q (symmetrised, pprow), m^p = F m^f + b (vmp)
  auto predict = [&]() {
    Real fr[DP], xr[DP];
    ld_row<Real, DP>(sF, row, fr);
    row_mat<Real, DP>(fr, SP, xr);
    const Real mpi = dot_rv<Real, DP>(fr, vm) + sb[row];
    __syncwarp();
    st_row<Real, DP>(SX, row, xr, act);
    if (act) vmp[lane] = mpi;
    __syncwarp();
    row_mat<Real, DP>(xr, sFT, pprow);
    Real qr[DP];
    ld_row<Real, DP>(sQ, row, qr);
#pragma unroll
    for (int j = 0; j < DP; ++j) pprow[j] += qr[j];
    symmetrise_store<Real, DP>(SY, pprow, lane);
  };

  auto store_backward = [&](int t, const Real (&grow)[DP], Real ui) {
    Real* Gt = a.G + ((long)c * p.nT + t) * DP * DP;
    if (act) {
      st_vec<Real, DP>(Gt + row * DP, grow);
      a.U[((long)c * p.nT + t) * DP + lane] = ui;
    }
    __syncwarp();
    if (act) vU[lane] = ui;
    __syncwarp();
    uhat += dot_rv<Real, DP>(ghat, vU);
    st_row<Real, DP>(SY, row, grow, act);
    __syncwarp();
    Real gn[DP];
    row_mat<Real, DP>(ghat, SY, gn);
#pragma unroll
    for (int j = 0; j < DP; ++j) ghat[j] = gn[j];
    __syncwarp();
  };

  auto backward_noise = [&](int t) {
    Real ei = 0;
    if (lane < p.d) {
      ei = a.eps ? a.eps[((long)c * p.nT + t) * p.d + lane]
                 : philox_normal<Real>(p.seed, (uint32_t)c, a.iter, PURPOSE_BACKWARD, (uint32_t)t, lane);
    }
    __syncwarp();
    if (act) veps[lane] = ei;
    __syncwarp();
  };

  // epilogue for state t (uses X = F P^f_t in SX, P^p_{t+1} in pprow, m^p_{t+1} in vmp,
  // m^f_t in vm, P^f_t in SP): G_t = P^f F^T (P^p)^{-1}, Sigma_t = P^f - G P^p G^T,
  // U_t = m^f_t - G_t m^p_{t+1} + chol(Sigma_t) eps_t.
  auto epilogue = [&](int t) {
    {
      Real a_[DP];
#pragma unroll
      for (int j = 0; j < DP; ++j) a_[j] = pprow[j];
      chol_rows<Real, DP>(a_, SL, vdiag, p.d, lane, &bad);   // L_p^T
    }
    Real ytr[DP];   // row j of Y^T, Y = L_p^{-1} X
    {
      Real xc[DP];
      ld_col<Real, DP>(SX, row, xc);
      fwd_subst<Real, DP>(SL, vdiag, xc, ytr);
    }
    __syncwarp();
    st_col<Real, DP>(SY, row, ytr, act);     // SY = Y row-major
    __syncwarp();
    Real sig[DP];
    ld_row<Real, DP>(SP, row, sig);
    row_mat<Real, DP, true, true>(ytr, SY, sig);   // Sigma = P^f - Y^T Y
    Real grow[DP];
    bwd_subst<Real, DP>(SL, vdiag, ytr, grow);                // row of G = (L_p^{-T} Y)^T
    chol_rows<Real, DP>(sig, SX, vdiag, p.d, lane, &bad);     // L_Sigma^T (X is dead)
    backward_noise(t);
    Real lc[DP];
    ld_col<Real, DP>(SX, row, lc);
    const Real ui = vm[row] - dot_rv<Real, DP>(grow, vmp) + dot_rv<Real, DP>(lc, veps);
    store_backward(t, grow, ui);
  };

  // measurement update at t from (vmp, pprow): m^f, P^f, predictive terms
  auto update = [&](int t) {
    {
      Real s_[DP];
#pragma unroll
      for (int j = 0; j < DP; ++j) s_[j] = pprow[j] + ((j == lane && j < p.d) ? p.r : (Real)0);
      chol_rows<Real, DP>(s_, SL, vdiag, p.d, lane, &bad);   // L_S^T
    }
    const Real rres = (lane < p.d) ? ytc[(long)t * p.d + lane] - vmp[lane] : (Real)0;
    __syncwarp();
    if (act) vr[lane] = rres;
    __syncwarp();
    Real z[DP];
    {
      Real rr[DP];
      ld_vec<Real, DP>(vr, rr);
      fwd_subst<Real, DP>(SL, vdiag, rr, z);
    }
    Real ys[DP];
    {
      Real rhs[DP];
#pragma unroll
      for (int j = 0; j < DP; ++j) rhs[j] = pprow[j];
      fwd_subst<Real, DP>(SL, vdiag, rhs, ys);
    }
    const Real mfi = vmp[row] + dot_rr<Real, DP>(ys, z);
    const Real qz = dot_rr<Real, DP>(z, z);
    Real lg = (lane < p.d) ? log(SL[lane * Lay<Real, DP>::LD + lane]) : (Real)0;
    lg = warp_sum<Real>(lg);
    __syncwarp();
    st_col<Real, DP>(SY, row, ys, act);      // SY = Y_s row-major
    __syncwarp();
    Real pf[DP];
#pragma unroll
    for (int j = 0; j < DP; ++j) pf[j] = pprow[j];
    row_mat<Real, DP, true, true>(ys, SY, pf);     // P^f = P^p - Y_s^T Y_s
    __syncwarp();
    st_row<Real, DP>(SP, row, pf, act);
    if (act) vm[lane] = mfi;
    __syncwarp();
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
    predict();
  }
  update(s);
  for (int t = s + 1; t <= e; ++t) {
    predict();
    if (epi) epilogue(t - 1);
    update(t);
  }
  if (epi) {
    if (e < p.nT - 1) {
      predict();
      epilogue(e);
    } else {
      // last state: G_{T-1} = 0, U_{T-1} = m^f + chol(P^f) eps
      Real pf[DP];
      ld_row<Real, DP>(SP, row, pf);
      chol_rows<Real, DP>(pf, SX, vdiag, p.d, lane, &bad);
      backward_noise(e);
      Real lc[DP];
      ld_col<Real, DP>(SX, row, lc);
      const Real ui = vm[row] + dot_rv<Real, DP>(lc, veps);
      Real g0[DP];
      zero<Real, DP>(g0);
      store_backward(e, g0, ui);
    }
    Real* gk = a.gu + ((long)c * p.nb + k) * Z::GS;
    if (act) {
      st_vec<Real, DP>(gk + row * DP, ghat);
      gk[DP * DP + lane] = uhat;
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
  const Real* G;
  const Real* U;
  const Real* gu;
  Real* xs;
  int mh;
  const Real* x;
  const Real* u;
  const Real* v;
  Real* yts;
  double* mh_part;
};

template <typename Real, int DP>
__global__ void __launch_bounds__(32 * Sizes<Real, DP>::BWD_WPC)
    k_sample_backward(KP<Real> p, BackArgs<Real> a) {
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
    const Real* gl = a.gu + ((long)c * p.nb + (p.nb - 1)) * Z::GS;
    xi = gl[DP * DP + row];
    for (int kk = p.nb - 2; kk > k; --kk) {
      const Real* gk = a.gu + ((long)c * p.nb + kk) * Z::GS;
      __syncwarp();
      if (act) vx[lane] = xi;
      __syncwarp();
      Real g[DP];
      ld_vec<Real, DP>(gk + row * DP, g);
      xi = dot_rv<Real, DP>(g, vx) + gk[DP * DP + row];
    }
  }
  double acc = 0.0;
  for (int t = e; t >= s; --t) {
    const long ct = (long)c * p.nT + t;
    if (t == p.nT - 1) {
      xi = a.U[ct * DP + row];
    } else {
      __syncwarp();
      if (act) vx[lane] = xi;
      __syncwarp();
      Real g[DP];
      ld_vec<Real, DP>(a.G + ct * DP * DP + row * DP, g);
      xi = dot_rv<Real, DP>(g, vx) + a.U[ct * DP + row];
    }
    if (lane < p.d) a.xs[ct * p.d + lane] = xi;
    if (a.mh) {
      const Real* yr = p.y + (p.y_per_chain ? ct : (long)t) * p.d;
      const bool obs = !p.mask || p.mask[t];
      Real vsi = 0;
      if (p.emis == AUX_EMIS_LINEAR_GAUSSIAN) {
        __syncwarp();
        if (act) vxs[lane] = (lane < p.d) ? yr[lane] - xi : (Real)0;
        __syncwarp();
        Real ry[DP];
        ld_row<Real, DP>(sRy, row, ry);
        vsi = dot_rv<Real, DP>(ry, vxs);
      }
      if (lane < p.d) {
        const long idx = ct * p.d + lane;
        const Real xo = a.x[idx], ui = a.u[idx], vi = a.v[idx];
        const Real yi = yr[lane];
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
        const Real fwd = vi * (ui - xi) + (Real)0.5 * p.r * vi * vi;
        const Real rev = vsi * (ui - xo) + (Real)0.5 * p.r * vsi * vsi;
        acc += (double)gdiff + (double)fwd - (double)rev;
        a.yts[idx] = ui + p.r * vsi;
      }
    }
  }
  if (a.mh) {
    acc = warp_sum<double>(acc);
    if (lane == 0) a.mh_part[(long)c * p.nb + k] = acc;
  }
}

// ---------------------------------------------------------------------------
// MH test and state update, one CTA per chain.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void k_mh(KP<Real> p, Real* __restrict__ x, const Real* __restrict__ xs,
                     const double* __restrict__ mh_part, const double* __restrict__ lz_part,
                     uint64_t iter, uint32_t* acc_count, double* log_alpha, int32_t* status) {
  const int c = blockIdx.x;
  __shared__ double red[32];
  __shared__ int accept;
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
    const uint4 r = philox_word(p.seed, (uint32_t)c, iter, PURPOSE_MH, 0, 0);
    const double lu = log(u01<double>(r.x));
    accept = (st == 0) && (lu < la);
    status[c] |= st;
    if (log_alpha) log_alpha[c] = la;
    if (acc_count && accept) acc_count[c] += 1;
  }
  __syncthreads();
  if (accept) {
    const long n = (long)p.nT * p.d;
    Real* xc = x + (long)c * n;
    const Real* xsc = xs + (long)c * n;
    for (long q = threadIdx.x; q < n; q += blockDim.x) xc[q] = xsc[q];
  }
}

}  // namespace auxk
