// aux_cov.cuh — tables of the covariance pass and two of its building blocks.
//
// With the first-order proposal and Gaussian dynamics the pseudo-observation
// model is ytilde_t = x_t + N(0, R), R = (delta/2) I (Eq. (2.7)), so the
// covariance part of every filtering element (Appendix A.2.1), every
// predictive and filtering covariance, every gain and every backward-sampling
// matrix of Eq. (A.14) is a function of (m0, P0, F, Q, delta) alone: it is the
// same for every chain and every MCMC iteration. The covariance pass
// (aux_cov2.cuh for the covariance form, aux_sqrt.cuh for the square-root
// form) writes, per step t,
//   tab[TK][t]  = K'_t = r S_t^{-1} = I - K_t,  S_t = P^p_t + R   (symmetric)
//   tab[TG][t]  = G_t = P^f_t F^T (P^p_{t+1})^{-1}          (G_{T-1} = 0)
//   tab[TLS][t] = chol(Sigma_t), Sigma_t = P^f_t - G_t P^p_{t+1} G_t^T
//                 (chol(P^f_{T-1}) at t = T-1)
//   tab[TPF][t] = P^f_t,   ldt[t] = log det S_t (FP64);
// and, for the blocks s..e of the per-chain means pass,
//   tab[TGP][t]  = G_s G_{s+1} ... G_{t-1}  (identity at t = s)
//   btab[BAH][k] = (I - K_e) F ... (I - K_s) F,  K_t = P^p_t S_t^{-1}
//                  (the linear part of m^f_e as a function of m^f_{s-1})
//   btab[BGH][k] = G_s ... G_e,   ld[k] = sum over the block of ldt[t].
// Because R = r I, I - K_t = r S_t^{-1} = K'_t, so the filtering mean update
// is m^f_t = ytilde_t - K'_t (ytilde_t - m^p_t) and the predictive likelihood
// term uses (ytilde_t - m^p_t)^T S_t^{-1} (ytilde_t - m^p_t) = r^{-1} e^T K'_t e
// and log det S_t: the per-chain work that remains (aux_means.cuh) is
// matrix-vector only, one product per step for the filter.
// This file holds the element operator's matrix part on one CTA
// (cov_combine_mw, the squaring of the doubling levels) and the composition of
// the square-root pass's covariance-block products into the means partition
// (k_cov_products, k_cov_gp_fix).
#pragma once
#include "aux_kernels.cuh"

namespace auxk {

enum { TK = 0, TG, TLS, TGP, TPF, NTAB };
// block products of the means partition, and (XPA, XPG) their prefix products
// within the groups of XGS consecutive maps of the two-level cross-block
// composition (aux_means.cuh, k_mean_cross2)
enum { BAH = 0, BGH, XPA, XPG, NBTAB };

template <typename Real> struct CovArgs {
  const Real* prefix;   // scan result [nbc][3 DP^2] (A, C, J); null when nbc == 1
  Real* tab;            // [NTAB][T][DP][DP]
  Real* btab;           // [NBTAB][nb][DP][DP] (means partition)
  double* ld;           // [nb] (means partition)
  double* ldt;          // [T]
  int32_t* status;      // [1]: ST_NOT_PD when a factorisation failed
  Real* cblk;           // [3][nbc][DP][DP]: per covariance block G_s..G_e, M_e..M_s, and the
                        // product of the earlier covariance blocks of its means block
  int R;                // covariance blocks per means block (means L / Lc)
};

template <typename Real, int DP> struct CovSizes {
  static constexpr int MAT = Lay<Real, DP>::MAT, VEC = Lay<Real, DP>::VEC;
  static constexpr int FIX_WPC = 8;
  static constexpr size_t PROD_SMEM = (2 * MAT) * sizeof(Real);
  static constexpr size_t FIX_SMEM = FIX_WPC * 2 * MAT * sizeof(Real);
};

// ---------------------------------------------------------------------------
// The matrix part (A, C, J) of the element operator (Appendix A.2.1) on one CTA
// of CW_SCAN warps: the ten d x d products are split by output columns across
// the warps, the two Cholesky factorisations and the triangular solve run on
// warp 0.
// ---------------------------------------------------------------------------
constexpr int CW_SCAN = 4;

template <typename Real, int DP> struct CovScanMW {
  static constexpr int MAT = Lay<Real, DP>::MAT, VEC = Lay<Real, DP>::VEC;
  static constexpr int NC = DP / CW_SCAN;   // output columns per warp
  // SA SC SJ SU S2 S3 S4 SN SAe SCe SJe + 2 vectors
  static constexpr size_t SMEM = (11 * MAT + 2 * VEC) * sizeof(Real);
};

// (A, C, J) of left (x) right into out (one CTA of CW_SCAN warps; products split
// by columns, Cholesky factorisations and solves on warp 0)
template <typename Real, int DP>
__device__ void cov_combine_mw(const KP<Real>& p, const Real* __restrict__ left,
                               const Real* __restrict__ right, Real* __restrict__ out,
                               int32_t* __restrict__ status) {
  using Z = CovScanMW<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC, LD = Lay<Real, DP>::LD, NC = Z::NC;
  constexpr long DD = (long)DP * DP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nth = blockDim.x;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  const int c0 = warp * NC;
  Real* SA = sm;
  Real* SC = SA + MAT;
  Real* SJ = SC + MAT;
  Real* SU = SJ + MAT;
  Real* S2 = SU + MAT;
  Real* S3 = S2 + MAT;
  Real* S4 = S3 + MAT;
  Real* SN = S4 + MAT;
  Real* SAe = SN + MAT;
  Real* SCe = SAe + MAT;
  Real* SJe = SCe + MAT;
  Real* vd1 = SJe + MAT;
  Real* vd2 = vd1 + VEC;
  // (A, C, J) of both operands straight into the padded slots (SA SC SJ and SAe SCe SJe
  // are consecutive), all copies in flight at once
  stage_mats<Real, DP>(SA, left, DD, 3);
  stage_mats<Real, DP>(SAe, right, DD, 3);
  cp_async_wait<0>();
  __syncthreads();
  int bad = 0;
  auto put = [&](Real* S, const Real (&v)[NC]) {   // the warp's column slice of row `row`
    if (act) stn<Real, NC>(S + row * LD + c0, v);
  };
  // U = chol(C_i): LS form in S2, rows in SU
  if (warp == 0) {
    Real a[DP];
    ld_row<Real, DP>(SC, row, a);
    chol_la<Real, DP>(a, S2, SU, nullptr, vd1, nullptr, p.d, lane, &bad);
  }
  __syncthreads();
  Real t1[NC];
  mm_row_c<Real, DP, NC>(SJe + row * LD, SU, c0, t1);   // J_e U
  put(S3, t1);
  __syncthreads();
  mm_col_c<Real, DP, NC>(SU, row, S3, c0, t1);          // N = I + U^T J_e U
#pragma unroll
  for (int j = 0; j < NC; ++j) t1[j] += (c0 + j == lane) ? (Real)1 : (Real)0;
  put(SN, t1);
  __syncthreads();
  if (warp == 0) {   // L_N = chol(N) (LS form in S4); B = U L_N^{-T} (rows in S2)
    Real a[DP];
    ld_row<Real, DP>(SN, row, a);
    chol_la<Real, DP>(a, S4, nullptr, nullptr, vd2, nullptr, p.d, lane, &bad);
    Real r[DP];
    ld_row<Real, DP>(SU, row, r);
    fsolve_pf<Real, DP, false>(S4, vd2, r, S2, lane);
  }
  __syncthreads();
  mm_row_c<Real, DP, NC>(SAe + row * LD, S2, c0, t1);   // P = A_e B, stored transposed in S3
  if (act) {
#pragma unroll
    for (int j = 0; j < NC; ++j) S3[(c0 + j) * LD + row] = t1[j];
  }
  mm_row_c<Real, DP, NC>(SJe + row * LD, SA, c0, t1);   // X1 = J_e A_i
  put(S4, t1);
  __syncthreads();
  mm_col_c<Real, DP, NC>(S2, row, S4, c0, t1);          // Z = B^T X1
  put(SU, t1);
  __syncthreads();
  Real jn[NC], an[NC], cn[NC];
  ldn<Real, NC>(SJ + row * LD + c0, jn);                // J = J_i + A_i^T X1 - Z^T Z
  mm_col_c<Real, DP, NC, true>(SA, row, S4, c0, jn);
  mm_col_c<Real, DP, NC, true, true>(SU, row, SU, c0, jn);
  mm_row_c<Real, DP, NC>(SAe + row * LD, SA, c0, an);   // A = A_e A_i - P Z
  mm_col_c<Real, DP, NC, true, true>(S3, row, SU, c0, an);
  ldn<Real, NC>(SCe + row * LD + c0, cn);               // C = C_e + P P^T
  mm_col_c<Real, DP, NC, true>(S3, row, S3, c0, cn);
  __syncthreads();
  put(SA, an);
  put(SC, cn);
  put(SJ, jn);
  __syncthreads();
  {   // J symmetrised
    Real jc[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) jc[j] = SJ[(c0 + j) * LD + row];
#pragma unroll
    for (int j = 0; j < NC; ++j) jn[j] = (Real)0.5 * (jn[j] + jc[j]);
  }
  __syncthreads();
  put(SJ, jn);
  __syncthreads();
  {   // SA SC SJ -> (A, C, J), 16-byte chunks
    using V = typename Vec16<Real>::V;
    constexpr int N = Vec16<Real>::N, CPR = DP / N, PER = DP * CPR;
    V* g = reinterpret_cast<V*>(out);
    for (int q = threadIdx.x; q < 3 * PER; q += nth) {
      const int m = q / PER, rem = q - m * PER, r = rem / CPR, cc = rem - r * CPR;
      g[q] = *reinterpret_cast<const V*>(SA + m * MAT + r * LD + cc * N);
    }
  }
  if (bad && lane == 0 && warp == 0) atomicOr(status, ST_NOT_PD);
}

// ---------------------------------------------------------------------------
// Block products of the means partition (p.L, p.nb; kc = covariance blocks,
// a.R per means block), one warp per means block k: over its covariance
// blocks j in order, the exclusive products E_j = GHc_0 ... GHc_{j-1} (to
// cblk[2]), GH_k = GHc_0 ... GHc_{R-1}, AH_k = AHc_{R-1} ... AHc_0, and
// ld[k] = sum of log det S_t over the block.
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __launch_bounds__(32) k_cov_products(KP<Real> p, CovArgs<Real> a, int nbc) {
  pdl_wait();
  pdl_trigger();
  constexpr int MAT = CovSizes<Real, DP>::MAT, LD = Lay<Real, DP>::LD;
  constexpr long DD = (long)DP * DP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* SX = reinterpret_cast<Real*>(smem_raw);
  Real* SY = SX + MAT;
  const int lane = threadIdx.x & 31, k = blockIdx.x;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  const int j0 = k * a.R, j1 = min(nbc, j0 + a.R) - 1;
  Real P[DP], Q[DP];
#pragma unroll
  for (int j = 0; j < DP; ++j) P[j] = Q[j] = (j == lane) ? (Real)1 : (Real)0;
  auto load_slot = [&](Real* S, const Real* g) {
    __syncwarp();
    Real r[DP];
    ld_vec<Real, DP>(g + row * DP, r);
    st_row<Real, DP>(S, row, r, act);
    __syncwarp();
  };
  for (int j = j0; j <= j1; ++j) {
    if (act) st_vec<Real, DP>(a.cblk + (2L * nbc + j) * DD + row * DP, P);
    // P <- P GHc_j
    __syncwarp();
    st_row<Real, DP>(SX, row, P, act);
    load_slot(SY, a.cblk + (long)j * DD);
    mm_row<Real, DP>(SX + row * LD, SY, P);
    // Q <- AHc_j Q
    __syncwarp();
    st_row<Real, DP>(SX, row, Q, act);
    load_slot(SY, a.cblk + ((long)nbc + j) * DD);
    mm_row<Real, DP>(SY + row * LD, SX, Q);
  }
  if (act) {
    st_vec<Real, DP>(a.btab + ((long)BGH * p.nb + k) * DD + row * DP, P);
    st_vec<Real, DP>(a.btab + ((long)BAH * p.nb + k) * DD + row * DP, Q);
  }
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  double acc = 0.0;
  for (int t = s + lane; t <= e; t += 32) acc += a.ldt[t];
  acc = warp_sum<double>(acc);
  if (lane == 0) a.ld[k] = acc;
}

// ---------------------------------------------------------------------------
// G_s ... G_{t-1} from the covariance-block-local prefix: tab[TGP][t] <-
// E_j tab[TGP][t] for the steps of covariance block j (not the first of its
// means block), one warp per step.
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __launch_bounds__(32 * CovSizes<Real, DP>::FIX_WPC)
    k_cov_gp_fix(KP<Real> p, CovArgs<Real> a, int Lc, int nbc) {
  pdl_wait();
  pdl_trigger();
  constexpr int MAT = CovSizes<Real, DP>::MAT, LD = Lay<Real, DP>::LD;
  constexpr int WPC = CovSizes<Real, DP>::FIX_WPC;
  constexpr long DD = (long)DP * DP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * WPC + warp;
  if (t >= p.nT) return;
  const int j = t / Lc;
  if (j % a.R == 0) return;
  Real* SX = reinterpret_cast<Real*>(smem_raw) + warp * 2 * MAT;
  Real* SY = SX + MAT;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  Real* gp = a.tab + ((long)TGP * p.nT + t) * DD;
  Real r[DP];
  ld_vec<Real, DP>(a.cblk + (2L * nbc + j) * DD + row * DP, r);
  st_row<Real, DP>(SX, row, r, act);
  ld_vec<Real, DP>(gp + row * DP, r);
  st_row<Real, DP>(SY, row, r, act);
  __syncwarp();
  mm_row<Real, DP>(SX + row * LD, SY, r);
  if (act) st_vec<Real, DP>(gp + row * DP, r);
}

}  // namespace auxk
