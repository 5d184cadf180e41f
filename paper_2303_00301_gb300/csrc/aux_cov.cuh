// aux_cov.cuh — the covariance pass of the parallel filter.
//
// With the first-order proposal and Gaussian dynamics the pseudo-observation
// model is ytilde_t = x_t + N(0, R), R = (delta/2) I (Eq. (2.7)), so the
// covariance part of every filtering element (Appendix A.2.1), every
// predictive and filtering covariance, every gain and every backward-sampling
// matrix of Eq. (A.14) is a function of (m0, P0, F, Q, delta) alone: it is the
// same for every chain and every MCMC iteration. This pass runs the matrix half
// of the blocked scan once, with its own short block length Lc (one warp per
// scan block: conditional-filter block reduction, Hillis-Steele rounds over
// the block aggregates, in-block filter from the prefix), and writes, per step t,
//   tab[TK][t]  = K'_t = r S_t^{-1} = I - K_t,  S_t = P^p_t + R   (symmetric)
//   tab[TG][t]  = G_t = P^f_t F^T (P^p_{t+1})^{-1}          (G_{T-1} = 0)
//   tab[TLS][t] = chol(Sigma_t), Sigma_t = P^f_t - G_t P^p_{t+1} G_t^T
//                 (chol(P^f_{T-1}) at t = T-1)
//   tab[TPF][t] = P^f_t,   ldt[t] = log det S_t (FP64);
// and, for the blocks s..e of the per-chain means pass (each a whole number of
// covariance blocks: local products in k_cov_apply, composed by k_cov_products
// and k_cov_gp_fix),
//   tab[TGP][t]  = G_s G_{s+1} ... G_{t-1}  (identity at t = s)
//   btab[BAH][k] = (I - K_e) F ... (I - K_s) F,  K_t = P^p_t S_t^{-1}
//                  (the linear part of m^f_e as a function of m^f_{s-1})
//   btab[BGH][k] = G_s ... G_e,   ld[k] = sum over the block of ldt[t].
// Because R = r I, I - K_t = r S_t^{-1} = K'_t, so the filtering mean update
// is m^f_t = ytilde_t - K'_t (ytilde_t - m^p_t) and the predictive likelihood
// term uses (ytilde_t - m^p_t)^T S_t^{-1} (ytilde_t - m^p_t) = r^{-1} e^T K'_t e
// and log det S_t: the per-chain work that remains (aux_means.cuh) is
// matrix-vector only, one product per step for the filter.
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
  static constexpr size_t MODEL = (3 * MAT + 2 * VEC) * sizeof(Real);
  static constexpr size_t RED_SMEM = MODEL + (6 * MAT + 3 * VEC) * sizeof(Real);
  static constexpr size_t SCAN_SMEM = (9 * MAT + VEC) * sizeof(Real);
  static constexpr size_t APP_SMEM = MODEL + (13 * MAT + 2 * VEC) * sizeof(Real);
  static constexpr int FIX_WPC = 8;
  static constexpr size_t PROD_SMEM = (2 * MAT) * sizeof(Real);
  static constexpr size_t FIX_SMEM = FIX_WPC * 2 * MAT * sizeof(Real);
};

// ---------------------------------------------------------------------------
// Block reduction: the conditional Kalman recursion of k_filter_reduce
// (identity element in, raw elements applied in order), matrix part only.
// aggm: [nb][3 DP^2] (A, C, J).
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __launch_bounds__(32, 1) k_cov_reduce(KP<Real> p, Real* __restrict__ aggm,
                                                     int32_t* __restrict__ status,
                                                     const int* __restrict__ kmap, Real* __restrict__ dst1,
                                                     Real* __restrict__ dst2) {
  pdl_wait();
  pdl_trigger();
  refresh_delta(p);
  using Z = CovSizes<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC, LD = Lay<Real, DP>::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  Real* sF = sm;
  Real* sFT = sF + MAT;
  Real* sQ = sFT + MAT;
  Real* sb = sQ + MAT;
  load_model_slots<Real, DP>(p, sF, sFT, sQ, sb);
  const Real* sphi = sb + VEC;
  Real* SA = sb + 2 * VEC;
  Real* SC = SA + MAT;
  Real* SX = SC + MAT;
  Real* SY = SX + MAT;
  Real* SW = SY + MAT;
  Real* SL = SW + MAT;
  Real* vdiag = SL + MAT;
  Real* vdummy = vdiag + VEC;
  // kmap (optional): CTA b reduces block kmap[b]; CTA 1 writes to dst1, CTA 2 to dst2
  // (the distinct aggregates of the doubling scan), else CTA b reduces block b into aggm
  const int lane = threadIdx.x & 31, k = kmap ? kmap[blockIdx.x] : blockIdx.x;
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
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
  }
  __syncwarp();
  for (int t = s; t <= e; ++t) {
    Real pprow[DP];
    if (t == 0) {
      ld_vec<Real, DP>(p.P0 + row * DP, pprow);
      Real z0[DP];
      zero<Real, DP>(z0);
      st_row<Real, DP>(SX, row, z0, act);
    } else if (p.fdiag) {
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
      __syncwarp();
      st_row<Real, DP>(SX, row, ar, act);
    } else {
      Real xr[DP];
      mm_row<Real, DP>(sF + row * LD, SC, xr);
      __syncwarp();
      st_row<Real, DP>(SX, row, xr, act);
      __syncwarp();
      mm_row<Real, DP>(SX + row * LD, sFT, pprow);
      Real qr[DP];
      ld_row<Real, DP>(sQ, row, qr);
#pragma unroll
      for (int j = 0; j < DP; ++j) pprow[j] += qr[j];
      symmetrise_store<Real, DP>(SY, pprow, lane);
      Real fa[DP];
      mm_row<Real, DP>(sF + row * LD, SA, fa);
      __syncwarp();
      st_row<Real, DP>(SX, row, fa, act);
    }
    __syncwarp();
    {
      Real s_[DP];
#pragma unroll
      for (int j = 0; j < DP; ++j) s_[j] = pprow[j] + ((j == lane && j < p.d) ? p.r : (Real)0);
      chol_rot<Real, DP>(s_, SL, nullptr, nullptr, vdiag, nullptr, p.d, lane, &bad);
    }
    {
      Real r1[DP], r2[DP], rv[DP];
#pragma unroll
      for (int j = 0; j < DP; ++j) r1[j] = pprow[j];
      ld_col<Real, DP>(SX, row, r2);
      zero<Real, DP>(rv);
      fsolve_multi<Real, DP, true>(SL, vdiag, r1, SY, r2, SW, rv, vdummy, lane);
    }
    __syncwarp();
    st_row<Real, DP>(SC, row, pprow, act);
    if constexpr (DP >= 16) {
      __syncwarp();
      mm_tile_to_slot<Real, DP, true, true>(SY, SY, SC, SC, lane);   // C = P^p - Y^T Y
      mm_tile_to_slot<Real, DP, true, true>(SY, SW, SX, SA, lane);   // A = F A - Y^T W
      mm_tile_regs<Real, DP, true, false>(SW, SW, jtile, lane);       // J += W^T W
    } else {
      __syncwarp();
      Real cn[DP];
      ld_row<Real, DP>(SC, row, cn);
      mm_col<Real, DP, true, true>(SY, row, SY, cn);
      Real an[DP];
      ld_row<Real, DP>(SX, row, an);
      mm_col<Real, DP, true, true>(SY, row, SW, an);
      __syncwarp();
      st_row<Real, DP>(SC, row, cn, act);
      st_row<Real, DP>(SA, row, an, act);
      mm_col<Real, DP, true>(SW, row, SW, jreg);
    }
    __syncwarp();
  }
  if constexpr (DP >= 16) {
    tile_store<Real, DP>(SY, jtile, lane);
    __syncwarp();
    ld_row<Real, DP>(SY, row, jreg);
  }
  if (act) {
    Real* g = !kmap || blockIdx.x == 0 ? aggm + (long)k * 3 * DP * DP : (blockIdx.x == 1 ? dst1 : dst2);
    Real r[DP];
    ld_row<Real, DP>(SA, row, r);
    st_vec<Real, DP>(g + row * DP, r);
    ld_row<Real, DP>(SC, row, r);
    st_vec<Real, DP>(g + DP * DP + row * DP, r);
    st_vec<Real, DP>(g + 2 * DP * DP + row * DP, jreg);
  }
  if (bad && lane == 0) atomicOr(status, ST_NOT_PD);
}

// ---------------------------------------------------------------------------
// One Hillis-Steele round over the block aggregates (matrix part of the
// element operator, Appendix A.2.1).
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __launch_bounds__(32, 1)
    k_cov_scan_level(KP<Real> p, const Real* __restrict__ in_m, Real* __restrict__ out_m, int off,
                     int32_t* __restrict__ status) {
  using Z = CovSizes<Real, DP>;
  constexpr int MAT = Z::MAT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const int lane = threadIdx.x & 31, k = blockIdx.x;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  if (k < off) {
    if (act) {
      for (int q = row; q < 3 * DP; q += DP) {
        Real r[DP];
        ld_vec<Real, DP>(in_m + (long)k * 3 * DP * DP + q * DP, r);
        st_vec<Real, DP>(out_m + (long)k * 3 * DP * DP + q * DP, r);
      }
    }
    return;
  }
  Real* SA = sm;
  Real* SC = SA + MAT;
  Real* SU = SC + MAT;
  Real* S2 = SU + MAT;
  Real* S3 = S2 + MAT;
  Real* S4 = S3 + MAT;
  Real* SAe = S4 + MAT;
  Real* SCe = SAe + MAT;
  Real* SJe = SCe + MAT;
  Real* vdiag = SJe + MAT;
  int bad = 0;
  Real jreg[DP];
  {
    const Real* gi = in_m + (long)(k - off) * 3 * DP * DP;
    const Real* gj = in_m + (long)k * 3 * DP * DP;
    Real r[DP];
    ld_vec<Real, DP>(gi + row * DP, r);
    st_row<Real, DP>(SA, row, r, act);
    ld_vec<Real, DP>(gi + DP * DP + row * DP, r);
    st_row<Real, DP>(SC, row, r, act);
    ld_vec<Real, DP>(gi + 2 * DP * DP + row * DP, jreg);
    ld_vec<Real, DP>(gj + row * DP, r);
    st_row<Real, DP>(SAe, row, r, act);
    ld_vec<Real, DP>(gj + DP * DP + row * DP, r);
    st_row<Real, DP>(SCe, row, r, act);
    ld_vec<Real, DP>(gj + 2 * DP * DP + row * DP, r);
    st_row<Real, DP>(SJe, row, r, act);
  }
  __syncwarp();
  combine_matrix_1<Real, DP>(SC, SAe, SJe, SU, S2, S3, S4, vdiag, p.d, lane, &bad);
  combine_matrix_2<Real, DP>(SA, SC, jreg, SAe, SCe, SJe, SU, S2, S3, S4, lane);
  if (act) {
    Real* g = out_m + (long)k * 3 * DP * DP;
    Real r[DP];
    ld_row<Real, DP>(SA, row, r);
    st_vec<Real, DP>(g + row * DP, r);
    ld_row<Real, DP>(SC, row, r);
    st_vec<Real, DP>(g + DP * DP + row * DP, r);
    st_vec<Real, DP>(g + 2 * DP * DP + row * DP, jreg);
  }
  if (bad && lane == 0) atomicOr(status, ST_NOT_PD);
}

// ---------------------------------------------------------------------------
// The same round with one CTA of CW_SCAN warps per block (p >= 16): the ten
// d x d products of the operator are split by output columns across the
// warps, the two Cholesky factorisations and the triangular solve run on
// warp 0. Same operator, same order of operations per output entry.
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
// Prefix scan of the covariance blocks by doubling. With homogeneous dynamics
// and R = r I every element with t >= 1 is the same, so every covariance
// block except the first (it holds t = 0) and a short last one has the same
// aggregate G; the inclusive prefixes are P_j = P_0 (x) G^j. Level k computes
// P_j = P_{j - 2^k} (x) G^(2^k) for 2^k <= j < min(2^(k+1), n_end) (CTA i:
// P[dst + i] = P[src + i] (x) Gk with src = 0, dst = 2^k) and, in CTA `cnt`,
// G^(2^(k+1)) = G^(2^k) (x) G^(2^k) when a later level needs it; a short last
// block is one more operator, P_{n-1} = P_{n-2} (x) G_last. Same depth as
// Hillis-Steele (log2 of the block count), one operator per prefix instead
// of one per block and level.
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __launch_bounds__(32 * CW_SCAN)
    k_cov_scan_double_mw(KP<Real> p, Real* __restrict__ P, const Real* __restrict__ Gk,
                         Real* __restrict__ Gk2, int src, int dst, int cnt, int32_t* __restrict__ status) {
  pdl_wait();
  pdl_trigger();
  constexpr long DD = (long)DP * DP;
  const int i = blockIdx.x;
  if (i < cnt)
    cov_combine_mw<Real, DP>(p, P + (long)(src + i) * 3 * DD, Gk, P + (long)(dst + i) * 3 * DD, status);
  else
    cov_combine_mw<Real, DP>(p, Gk, Gk, Gk2, status);
}

// ---------------------------------------------------------------------------
// In-block covariance filter from the prefix P^f_{s-1}, with the per-step tables,
// three warps per covariance block. Per step t, after the prediction P^p_t
// (warp 0): warp 0 factors P^p_t and warp 1 factors S_t = P^p_t + R; then
// warp 0 forms the backward elements of step t - 1 (G_{t-1}, chol Sigma_{t-1})
// and the running G product, warp 1 the gain tables of step t (W_t, K'_t, M_t
// and the running M product), warp 2 the update P^f_t = P^p_t - Y^T Y. The
// three chains share only read-only factors; P^f is double buffered so that
// the update of step t and the epilogue of step t - 1 run side by side.
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __launch_bounds__(96, 1) k_cov_apply(KP<Real> p, CovArgs<Real> a) {
  pdl_wait();
  pdl_trigger();
  refresh_delta(p);
  using Z = CovSizes<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC, LD = Lay<Real, DP>::LD;
  constexpr long DD = (long)DP * DP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  Real* sF = sm;
  Real* sFT = sF + MAT;
  Real* sQ = sFT + MAT;
  Real* sb = sQ + MAT;
  load_model_slots<Real, DP>(p, sF, sFT, sQ, sb);
  __syncthreads();
  const Real* sphi = sb + VEC;
  Real* SPb = sb + 2 * VEC;    // P^f, two buffers (step t and step t - 1)
  Real* SPP = SPb + 2 * MAT;   // P^p of the current step
  Real* SX = SPP + MAT;        // F P^f_{t-1}, then G_{t-1}
  Real* SL = SX + MAT;         // chol(P^p) (LS form), then Sigma, then chol(Sigma) (LS)
  Real* SLR = SL + MAT;        // chol(P^p) (right-aligned), then chol(Sigma) row-major
  Real* SY0 = SLR + MAT;       // warp 0 scratch
  Real* SG = SY0 + MAT;        // chol(S) (LS form)
  Real* SWm = SG + MAT;        // W_t (warp 1)
  Real* SA1 = SWm + MAT;       // warp 1 scratch
  Real* SY2 = SA1 + MAT;       // warp 2 scratch
  Real* SGh = SY2 + MAT;       // G_s ... G_{t-1} of this covariance block
  Real* SAH = SGh + MAT;       // M_t ... M_s of this covariance block
  Real* vdA = SAH + MAT;
  Real* vdB = vdA + VEC;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, k = blockIdx.x;
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  int bad = 0;
  if (warp == 0) {
    Real gi[DP];
#pragma unroll
    for (int j = 0; j < DP; ++j) gi[j] = (j == lane) ? (Real)1 : (Real)0;
    st_row<Real, DP>(SGh, row, gi, act);
    st_row<Real, DP>(SAH, row, gi, act);
  }
  auto store_row = [&](int tb, int t, const Real* S) {
    if (!act) return;
    Real r[DP];
    ld_row<Real, DP>(S, row, r);
    st_vec<Real, DP>(a.tab + ((long)tb * p.nT + t) * DD + row * DP, r);
  };
  // warp 0: P^p -> SPP and X = F P^f -> SX from P^f in SP
  auto predict = [&](const Real* SP) {
    Real pprow[DP];
    if (p.fdiag) {
      Real pr[DP], ph[DP], qr[DP];
      ld_row<Real, DP>(SP, row, pr);
      ld_vec<Real, DP>(sphi, ph);
      ld_row<Real, DP>(sQ, row, qr);
      const Real phi = sphi[row];
#pragma unroll
      for (int j = 0; j < DP; ++j) {
        pprow[j] = fma(pr[j], phi * ph[j], qr[j]);
        pr[j] *= phi;
      }
      __syncwarp();
      st_row<Real, DP>(SX, row, pr, act);
    } else {
      Real xr[DP];
      mm_row<Real, DP>(sF + row * LD, SP, xr);
      __syncwarp();
      st_row<Real, DP>(SX, row, xr, act);
      __syncwarp();
      mm_row<Real, DP>(SX + row * LD, sFT, pprow);
      Real qr[DP];
      ld_row<Real, DP>(sQ, row, qr);
#pragma unroll
      for (int j = 0; j < DP; ++j) pprow[j] += qr[j];
      symmetrise_store<Real, DP>(SY0, pprow, lane);
    }
    st_row<Real, DP>(SPP, row, pprow, act);
    __syncwarp();
  };
  // warp 0: chol(P^p) -> SL / SLR / vdA
  auto factor_P = [&]() {
    Real a_[DP];
    ld_row<Real, DP>(SPP, row, a_);
    chol_rot<Real, DP>(a_, SL, nullptr, SLR, vdA, nullptr, p.d, lane, &bad);
  };
  // warp 1: chol(S), S = P^p + R -> SG / vdB
  auto factor_S = [&]() {
    Real s_[DP];
    ld_row<Real, DP>(SPP, row, s_);
#pragma unroll
    for (int j = 0; j < DP; ++j) s_[j] += (j == lane && j < p.d) ? p.r : (Real)0;
    chol_rot<Real, DP>(s_, SG, nullptr, nullptr, vdB, nullptr, p.d, lane, &bad);
  };
  // warp 0, after the factor of P^p_{t+1} (SL / SLR / vdA), with P^f_t in SP and
  // X = F P^f_t in SX: G_t -> SX, chol(Sigma_t) -> SLR
  auto epilogue = [&](int t, const Real* SP) {
    {
      Real rr[DP];
      ld_col<Real, DP>(SX, row, rr);
      fsolve_rot<Real, DP, true>(SL, vdA, rr, SY0, lane);
    }
    __syncwarp();
    Real sig[DP];
    if constexpr (DP >= 16) {
      mm_tile_to_slot<Real, DP, true, true>(SY0, SY0, SP, SL, lane);
      __syncwarp();
      ld_row<Real, DP>(SL, row, sig);
    } else {
      ld_row<Real, DP>(SP, row, sig);
      mm_col<Real, DP, true, true>(SY0, row, SY0, sig);
    }
    {
      Real rr[DP];
      ld_col<Real, DP>(SY0, row, rr);
      bsolve_rot<Real, DP>(SLR, vdA, rr, SX, lane);
    }
    chol_rot<Real, DP>(sig, SL, SLR, nullptr, vdA, nullptr, p.d, lane, &bad);
    store_row(TG, t, SX);
    store_row(TLS, t, SLR);
  };
  // warp 1: K'_t = r S_t^{-1} = r W^T W with W = L_S^{-1} (columns of the identity
  // through the forward solve); M_t = (I - K_t) F = K'_t F, then SAH <- M_t SAH
  auto gain_tables = [&](int t) {
    {
      Real r[DP];
#pragma unroll
      for (int j = 0; j < DP; ++j) r[j] = (j == lane) ? (Real)1 : (Real)0;
      fsolve_rot<Real, DP, true>(SG, vdB, r, SWm, lane);
    }
    __syncwarp();
    double lg = (lane < p.d) ? -log((double)vdB[lane]) : 0.0;
    lg = warp_sum<double>(lg);
    if (lane == 0) a.ldt[t] = 2.0 * lg;
    Real mr[DP];
    mm_col<Real, DP>(SWm, row, SWm, mr);
#pragma unroll
    for (int j = 0; j < DP; ++j) mr[j] *= p.r;
    if (act) st_vec<Real, DP>(a.tab + ((long)TK * p.nT + t) * DD + row * DP, mr);
    if (p.fdiag) {
      Real ph[DP];
      ld_vec<Real, DP>(sphi, ph);
#pragma unroll
      for (int j = 0; j < DP; ++j) mr[j] *= ph[j];
    } else {
      st_row<Real, DP>(SA1, row, mr, act);
      __syncwarp();
      mm_row<Real, DP>(SA1 + row * LD, sF, mr);
      __syncwarp();
    }
    st_row<Real, DP>(SA1, row, mr, act);
    __syncwarp();
    Real ah[DP];
    mm_row<Real, DP>(SA1 + row * LD, SAH, ah);
    __syncwarp();
    st_row<Real, DP>(SAH, row, ah, act);
    __syncwarp();
  };
  // warp 0: SGh <- SGh G_t (G_t in SX)
  auto ghat = [&]() {
    Real gn[DP];
    mm_row<Real, DP>(SGh + row * LD, SX, gn);
    __syncwarp();
    st_row<Real, DP>(SGh, row, gn, act);
    __syncwarp();
  };
  // warp 2: Y = L_S^{-1} P^p (columns of SY2), P^f = P^p - Y^T Y -> SP
  auto update = [&](int t, Real* SP) {
    Real pprow[DP];
    ld_row<Real, DP>(SPP, row, pprow);
    {
      Real rr[DP];
#pragma unroll
      for (int j = 0; j < DP; ++j) rr[j] = pprow[j];
      fsolve_rot<Real, DP, true>(SG, vdB, rr, SY2, lane);
    }
    __syncwarp();
    if constexpr (DP >= 16) {
      st_row<Real, DP>(SP, row, pprow, act);
      __syncwarp();
      mm_tile_to_slot<Real, DP, true, true>(SY2, SY2, SP, SP, lane);
    } else {
      Real pf[DP];
#pragma unroll
      for (int j = 0; j < DP; ++j) pf[j] = pprow[j];
      mm_col<Real, DP, true, true>(SY2, row, SY2, pf);
      __syncwarp();
      st_row<Real, DP>(SP, row, pf, act);
    }
    __syncwarp();
    store_row(TPF, t, SP);
    __syncwarp();
  };

  // ---- block start: P^p_s
  if (warp == 0) {
    if (k == 0) {
      Real pp[DP];
      ld_vec<Real, DP>(p.P0 + row * DP, pp);
      st_row<Real, DP>(SPP, row, pp, act);
    } else {
      Real r[DP];
      ld_vec<Real, DP>(a.prefix + (long)(k - 1) * 3 * DP * DP + DP * DP + row * DP, r);
      st_row<Real, DP>(SPb + MAT, row, r, act);
      __syncwarp();
      predict(SPb + MAT);
    }
  }
  __syncthreads();
  int cur = 0;   // P^f_t -> SPb[cur], P^f_{t-1} in SPb[cur ^ 1]
  for (int t = s; t <= e; ++t) {
    Real* SPc = SPb + cur * MAT;
    Real* SPo = SPb + (cur ^ 1) * MAT;
    if (t > s) {
      if (warp == 0) predict(SPo);
      __syncthreads();
    }
    if (warp == 0 && t > s) factor_P();
    if (warp == 1) factor_S();
    __syncthreads();
    if (warp == 0) {
      if (t > s) {
        epilogue(t - 1, SPo);
        ghat();
      }
      store_row(TGP, t, SGh);
    } else if (warp == 1) {
      gain_tables(t);
    } else {
      update(t, SPc);
    }
    __syncthreads();
    cur ^= 1;
  }
  // ---- block end: P^f_e in SPb[cur ^ 1]
  if (warp == 0) {
    const Real* SPe = SPb + (cur ^ 1) * MAT;
    if (e < p.nT - 1) {
      predict(SPe);
      factor_P();
      epilogue(e, SPe);
    } else {
      Real pf[DP], z0[DP];
      ld_row<Real, DP>(SPe, row, pf);
      chol_rot<Real, DP>(pf, SL, SLR, nullptr, vdA, nullptr, p.d, lane, &bad);
      zero<Real, DP>(z0);
      st_row<Real, DP>(SX, row, z0, act);
      __syncwarp();
      store_row(TG, e, SX);
      store_row(TLS, e, SLR);
    }
    ghat();
    if (act) {
      Real r[DP];
      ld_row<Real, DP>(SGh, row, r);
      st_vec<Real, DP>(a.cblk + (long)k * DD + row * DP, r);
      ld_row<Real, DP>(SAH, row, r);
      st_vec<Real, DP>(a.cblk + ((long)p.nb + k) * DD + row * DP, r);
    }
  }
  if (bad && lane == 0) atomicOr(a.status, ST_NOT_PD);
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
