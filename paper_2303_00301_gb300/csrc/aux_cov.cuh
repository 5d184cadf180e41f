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
// This file holds the table layout, the CTA shape of the operators of the
// doubling levels (CovScanMW, cov_fw) and the composition of the square-root pass's
// covariance-block products into the means partition (k_cov_products,
// k_cov_gp_fix).
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
// One CTA of CW_SCAN warps per element operator of the doubling levels
// (aux_cov2.cuh): the d x d products are split by output columns across the
// warps and the Cholesky factorisations and triangular solves run on one warp,
// fw. The SM runs warp w of a CTA on its sub-partition w mod 4, so with several
// CTAs on one SM a fixed fw would queue all of their (latency-bound)
// factorisations on one sub-partition while the other three idle at the
// barrier; cov_fw spreads fw over the CTAs.
// ---------------------------------------------------------------------------
constexpr int CW_SCAN = 4;

// Factorising warp of CTA b when CTAs are dispatched breadth-first over nsm
// SMs: the CTAs that share an SM (b, b + nsm, b + 2 nsm, ...) get different
// warps, and so different sub-partitions, whenever nsm is a multiple of 4.
__device__ __forceinline__ int cov_fw(int b, int nsm) { return (b + b / nsm) & (CW_SCAN - 1); }

template <typename Real, int DP> struct CovScanMW {
  static constexpr int MAT = Lay<Real, DP>::MAT, VEC = Lay<Real, DP>::VEC;
  static constexpr int NC = DP / CW_SCAN;   // output columns per warp
  static constexpr size_t SMEM = (11 * MAT + 2 * VEC) * sizeof(Real);
};

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
