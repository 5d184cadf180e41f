// aux_cov2.cuh — the covariance pass of the table modes by doubling over the
// steps (covariance form, padded widths p <= 32).
//
// With homogeneous dynamics and R = r I every filtering element with t >= 1
// has the same matrix part E = (A, C, J) (Appendix A.2.1), and the element of
// t = 0 is the posterior of x_0 (A = 0, J = 0, C = P^f_0). The inclusive prefix
// of step t is P_t = e_0 (x) E^t: its C part is the filtering covariance P^f_t
// and its A and J parts vanish. Level k forms, for every t in
// [2^k, min(2^(k+1), T)), P_t = P_(t-2^k) (x) E^(2^k) — one operator per step
// that needs only the C part of its left operand — and, on one more CTA,
// E^(2^(k+1)) = E^(2^k) (x) E^(2^k) for the next level (each power with the
// Cholesky factor of its C part, formed by the squaring that produced it):
// ceil(log2 T) operators of depth and T - 1 prefix operators in all. Given every P^f_t the per-step
// tables depend on P^f_(t-1), P^f_t and the model only, so each step forms its
// own (k_c2_tables), and the products over the means partition run one chain
// per means block (k_c2_products). The tables are those of aux_cov.cuh:
//   tab[TK][t]  = K'_t = r S_t^{-1},  S_t = P^p_t + r I,   ldt[t] = log det S_t
//   tab[TG][t]  = G_t = P^f_t F^T (P^p_{t+1})^{-1}          (0 at t = T - 1)
//   tab[TLS][t] = chol(Sigma_t), Sigma_t = P^f_t - G_t P^p_{t+1} G_t^T
//                 (chol(P^f_{T-1}) at t = T - 1)
//   tab[TPF][t] = P^f_t
//   tab[TGP][t] = G_s ... G_{t-1} over the means block s..e of t (I at t = s)
//   btab[BGH][k] = G_s ... G_e,  btab[BAH][k] = M_e ... M_s (M_t = K'_t F),
//   ld[k] = sum of ldt over the means block.
#pragma once
#include "aux_cov.cuh"

namespace auxk {

template <typename Real> struct Cov2Args {
  Real* tab;         // [NTAB][T][DP][DP]
  Real* btab;        // [NBTAB][nb][DP][DP]
  double* ld;        // [nb]
  double* ldt;       // [T]
  Real* pw;          // [2][4 DP^2]: (A, C, J, chol(C) rows) of E^(2^k), double buffered over the levels
  int32_t* status;   // [1]: ST_NOT_PD when a factorisation failed
};

template <typename Real, int DP> struct Cov2Sizes {
  static constexpr int MAT = Lay<Real, DP>::MAT, VEC = Lay<Real, DP>::VEC;
  static constexpr size_t MODEL = (3 * MAT + 2 * VEC) * sizeof(Real);
  // init: model + 2 x (LS, Y, V) + 2 x (2 vectors)
  // init: model + 2 x (LS, right-aligned L rows, Y, V, r S^{-1} P rows) + 2 x 2 vectors
  static constexpr size_t INIT_SMEM = MODEL + (10 * MAT + 4 * VEC) * sizeof(Real);
  // products: running product, two staged tables, M row scratch, F slot
  static constexpr size_t PROD_SMEM = (5 * MAT + 2 * VEC) * sizeof(Real);
};

// ---------------------------------------------------------------------------
// The two elements of the pass: P^f_0 (posterior of x_0: S0 = P0 + R,
// C = P0 - P0 S0^{-1} P0) on warp 0, and E (conditional Kalman step from the
// identity element: S = Q + R, Y = L_S^{-1} Q, V = L_S^{-1} F, C = Q - Q S^{-1} Q,
// A = F - Q S^{-1} F, J = V^T V, and chol(C) for the first squaring) on warp 1. With R = r I, I - K = r S^{-1}, so the
// covariances are formed as C = r S^{-1} P = r L_S^{-T} Y (P = P0 or Q,
// symmetrised) and A = r L_S^{-T} V: no difference of two nearly equal matrices
// when r is small against P (the subtraction P - Y^T Y loses about
// log10(|P| / r) digits).
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __launch_bounds__(64, 1) k_c2_init(KP<Real> p, Cov2Args<Real> a) {
  pdl_wait();
  pdl_trigger();
  refresh_delta(p);
  using Z = Cov2Sizes<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC;
  constexpr long DD = (long)DP * DP;
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
  Real* LS = sb + 2 * VEC + warp * 5 * MAT;
  Real* LR = LS + MAT;       // right-aligned rows of L_S
  Real* SY = LR + MAT;
  Real* SV = SY + MAT;
  Real* SZ = SV + MAT;       // rows of P S^{-1}
  Real* vd = sb + 2 * VEC + 10 * MAT + warp * 2 * VEC;
  Real* vdummy = vd + VEC;
  int bad = 0;
  Real s_[DP];
  if (warp == 0) {
    ld_vec<Real, DP>(p.P0 + row * DP, s_);
  } else {
    ld_row<Real, DP>(sQ, row, s_);
  }
  Real cov[DP];
#pragma unroll
  for (int j = 0; j < DP; ++j) cov[j] = s_[j];
#pragma unroll
  for (int j = 0; j < DP; ++j) s_[j] += (j == lane && j < p.d) ? p.r : (Real)0;
  chol_la<Real, DP>(s_, LS, nullptr, LR, vd, nullptr, p.d, lane, &bad);
  Real r1[DP], r2[DP], rv[DP];
#pragma unroll
  for (int j = 0; j < DP; ++j) r1[j] = cov[j];   // column `row` of the symmetric P0 / Q
  ld_col<Real, DP>(sF, row, r2);
  zero<Real, DP>(rv);
  fsolve_multi<Real, DP, true>(LS, vd, r1, SY, r2, SV, rv, vdummy, lane);
  __syncwarp();
  {   // C = r L_S^{-T} Y: row `lane` of (L_S^{-T} Y)^T = P S^{-1}, then symmetrised
    Real yc[DP], cr[DP];
    ld_col<Real, DP>(SY, row, yc);
    bsolve_rot<Real, DP>(LR, vd, yc, SZ, lane);
    __syncwarp();
    ld_row<Real, DP>(SZ, row, cr);
    Real cc[DP];
    ld_col<Real, DP>(SZ, row, cc);
#pragma unroll
    for (int j = 0; j < DP; ++j) cov[j] = (Real)0.5 * p.r * (cr[j] + cc[j]);
  }
  if (warp == 0) {
    if (act) st_vec<Real, DP>(a.tab + ((long)TPF * p.nT + 0) * DD + row * DP, cov);
  } else {
    // A = (I - K) F = r S^{-1} F = r L_S^{-T} V (columns of V through the backward solve)
    Real an[DP], jn[DP], vc[DP];
    ld_col<Real, DP>(SV, row, vc);
    __syncwarp();
    bsolve_rot<Real, DP>(LR, vd, vc, SZ, lane);            // row `lane` of SZ = column `lane` of L_S^{-T} V
    __syncwarp();
    ld_col<Real, DP>(SZ, row, an);
#pragma unroll
    for (int j = 0; j < DP; ++j) an[j] *= p.r;
    mm_col<Real, DP>(SV, row, SV, jn);                      // J = V^T V
    if (act) {
      st_vec<Real, DP>(a.pw + row * DP, an);
      st_vec<Real, DP>(a.pw + DD + row * DP, cov);
      st_vec<Real, DP>(a.pw + 2 * DD + row * DP, jn);
    }
    // chol(C) rows, carried with the power (SY and SZ are free here)
    __syncwarp();
    chol_la<Real, DP>(cov, SY, SZ, nullptr, vdummy, nullptr, p.d, lane, &bad);
    Real ur[DP];
    ld_row<Real, DP>(SZ, row, ur);
    if (act) st_vec<Real, DP>(a.pw + 3 * DD + row * DP, ur);
  }
  if (bad && lane == 0) atomicOr(a.status, ST_NOT_PD);
}

// ---------------------------------------------------------------------------
// C part of P (x) right for a prefix P = (0, C_i, 0), one CTA of CW_SCAN warps:
// U = chol(C_i), N = I + U^T J_e U, B = U L_N^{-T}, P = A_e B, C = C_e + P P^T
// (the operator of Appendix A.2.1 with A_i = 0, J_i = 0, in its Cholesky form;
// same order of operations per entry as the first factorisation and products
// of cov2_power; factorisations on warp fw).
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__device__ void cov2_conly(const KP<Real>& p, const Real* __restrict__ Ci, const Real* __restrict__ right,
                           Real* __restrict__ outC, int32_t* __restrict__ status, int fw) {
  using Z = CovScanMW<Real, DP>;
  constexpr int MAT = Z::MAT, LD = Lay<Real, DP>::LD, NC = Z::NC;
  constexpr long DD = (long)DP * DP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  const int c0 = warp * NC;
  Real* SC = sm;
  Real* SU = SC + MAT;
  Real* S2 = SU + MAT;
  Real* S3 = S2 + MAT;
  Real* S4 = S3 + MAT;
  Real* SN = S4 + MAT;
  Real* SAe = SN + MAT;
  Real* SCe = SAe + MAT;
  Real* SJe = SCe + MAT;
  Real* vd1 = SJe + MAT;
  Real* vd2 = vd1 + Lay<Real, DP>::VEC;
  stage_mats<Real, DP>(SC, Ci, DD, 1);
  stage_mats<Real, DP>(SAe, right, DD, 3);
  cp_async_wait<0>();
  __syncthreads();
  int bad = 0;
  auto put = [&](Real* S, const Real (&v)[NC]) {
    if (act) stn<Real, NC>(S + row * LD + c0, v);
  };
  if (warp == fw) {   // U = chol(C_i): rows in SU
    Real a_[DP];
    ld_row<Real, DP>(SC, row, a_);
    chol_la<Real, DP>(a_, S2, SU, nullptr, vd1, nullptr, p.d, lane, &bad);
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
  if (warp == fw) {   // L_N = chol(N); B = U L_N^{-T} (rows in S2)
    Real a_[DP];
    ld_row<Real, DP>(SN, row, a_);
    chol_la<Real, DP>(a_, S4, nullptr, nullptr, vd2, nullptr, p.d, lane, &bad);
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
  __syncthreads();
  Real cn[NC];
  ldn<Real, NC>(SCe + row * LD + c0, cn);               // C = C_e + P P^T
  mm_col_c<Real, DP, NC, true>(S3, row, S3, c0, cn);
  if (act) stn<Real, NC>(outC + row * DP + c0, cn);
  if (bad && lane == 0 && warp == fw) atomicOr(status, ST_NOT_PD);
}

// ---------------------------------------------------------------------------
// The squaring E' = E (x) E of the doubling (the operator of Appendix A.2.1
// with both operands E = (A, C, J)), one CTA of CW_SCAN warps. Every power
// carries U = chol(C) (rows, lower triangular), so the operator starts at
// N = I + U^T J U:
//   L_N = chol(N), B = U L_N^{-T}, P = A B, X1 = J A, Z = B^T X1,
//   C' = C + P P^T,  J' = J + A^T X1 - Z^T Z (symmetrised),  A' = A A - P Z,
// and, when the next squaring needs it (fac), U' = chol(C') is factorised on
// warp fw while the other warps form A' and J': the factorisation that the
// next squaring would otherwise start with, taken off its critical path (the
// same routine on the same C', so the carried factor is the one it would
// compute). in, out: [4][DP][DP] (A, C, J, U).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bar_sync_others(int nthreads) {
  asm volatile("bar.sync 1, %0;\n" ::"r"(nthreads) : "memory");
}

template <typename Real, int DP>
__device__ void cov2_power(const KP<Real>& p, const Real* __restrict__ in, Real* __restrict__ out, bool fac,
                           int32_t* __restrict__ status, int fw) {
  using Z = CovScanMW<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC, LD = Lay<Real, DP>::LD, NC = Z::NC;
  constexpr long DD = (long)DP * DP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  const int c0 = warp * NC;
  Real* SA = sm;           // the staged element: A, C, J, U (consecutive slots)
  Real* SC = SA + MAT;
  Real* SJ = SC + MAT;
  Real* SU = SJ + MAT;     // U, then U' = chol(C') rows
  Real* SB = SU + MAT;     // B rows
  Real* SP = SB + MAT;     // J U, then P^T
  Real* SL = SP + MAT;     // chol(N) (LS form), then X1
  Real* SN = SL + MAT;     // N, then Z
  Real* SCn = SN + MAT;    // C' rows
  Real* SJn = SCn + MAT;   // J' before symmetrisation
  Real* LSc = SJn + MAT;   // chol(C') (LS form)
  Real* vdn = LSc + MAT;
  Real* vdc = vdn + VEC;
  stage_mats<Real, DP>(SA, in, DD, 4);
  cp_async_wait<0>();
  __syncthreads();
  int bad = 0;
  auto put = [&](Real* S, int cc, const Real (&v)[NC]) {
    if (act) stn<Real, NC>(S + row * LD + cc, v);
  };
  Real t1[NC];
  mm_row_c<Real, DP, NC>(SJ + row * LD, SU, c0, t1);   // J U
  put(SP, c0, t1);
  __syncthreads();
  mm_col_c<Real, DP, NC>(SU, row, SP, c0, t1);          // N = I + U^T J U
#pragma unroll
  for (int j = 0; j < NC; ++j) t1[j] += (c0 + j == lane) ? (Real)1 : (Real)0;
  put(SN, c0, t1);
  __syncthreads();
  if (warp == fw) {   // L_N = chol(N); B = U L_N^{-T}
    Real a[DP];
    ld_row<Real, DP>(SN, row, a);
    chol_la<Real, DP>(a, SL, nullptr, nullptr, vdn, nullptr, p.d, lane, &bad);
    Real r[DP];
    ld_row<Real, DP>(SU, row, r);
    fsolve_pf<Real, DP, false>(SL, vdn, r, SB, lane);
  }
  __syncthreads();
  mm_row_c<Real, DP, NC>(SA + row * LD, SB, c0, t1);   // P = A B, stored transposed
  if (act) {
#pragma unroll
    for (int j = 0; j < NC; ++j) SP[(c0 + j) * LD + row] = t1[j];
  }
  mm_row_c<Real, DP, NC>(SJ + row * LD, SA, c0, t1);   // X1 = J A
  put(SL, c0, t1);
  __syncthreads();
  Real cn[NC];
  ldn<Real, NC>(SC + row * LD + c0, cn);               // C' = C + P P^T
  mm_col_c<Real, DP, NC, true>(SP, row, SP, c0, cn);
  put(SCn, c0, cn);
  mm_col_c<Real, DP, NC>(SB, row, SL, c0, t1);          // Z = B^T X1
  put(SN, c0, t1);
  __syncthreads();
  if (warp == fw) {
    if (fac) {   // U' = chol(C')
      Real a[DP];
      ld_row<Real, DP>(SCn, row, a);
      chol_la<Real, DP>(a, LSc, SU, nullptr, vdc, nullptr, p.d, lane, &bad);
      Real r[DP];
      ld_row<Real, DP>(SU, row, r);
      if (act) st_vec<Real, DP>(out + 3 * DD + row * DP, r);
    }
  } else {
    // column block k of A', C', J' on warp k, block fw on the warp after it
    const int helper = (fw + 1) & (CW_SCAN - 1);
    for (int k = 0; k < CW_SCAN; ++k) {
      if (k == fw ? warp != helper : warp != k) continue;
      const int cc = k * NC;
      Real jn[NC], an[NC];
      ldn<Real, NC>(SJ + row * LD + cc, jn);            // J + A^T X1 - Z^T Z
      mm_col_c<Real, DP, NC, true>(SA, row, SL, cc, jn);
      mm_col_c<Real, DP, NC, true, true>(SN, row, SN, cc, jn);
      mm_row_c<Real, DP, NC>(SA + row * LD, SA, cc, an);   // A A - P Z
      mm_col_c<Real, DP, NC, true, true>(SP, row, SN, cc, an);
      put(SJn, cc, jn);
      ldn<Real, NC>(SCn + row * LD + cc, cn);
      if (act) {
        stn<Real, NC>(out + row * DP + cc, an);
        stn<Real, NC>(out + DD + row * DP + cc, cn);
      }
    }
    bar_sync_others(32 * (CW_SCAN - 1));
    for (int k = 0; k < CW_SCAN; ++k) {   // J' symmetrised
      if (k == fw ? warp != helper : warp != k) continue;
      const int cc = k * NC;
      Real jn[NC];
      ldn<Real, NC>(SJn + row * LD + cc, jn);
#pragma unroll
      for (int j = 0; j < NC; ++j) jn[j] = (Real)0.5 * (jn[j] + SJn[(cc + j) * LD + row]);
      if (act) stn<Real, NC>(out + 2 * DD + row * DP + cc, jn);
    }
  }
  if (bad && lane == 0 && warp == fw) atomicOr(status, ST_NOT_PD);
}

// Level k of the doubling. With sq, CTA 0 forms E^(2 pow2) into pout (the next
// level waits for it, so it is dispatched first), with its factor when the
// next level squares again (fac); CTA sq + i, i < cnt, forms P^f_(pow2 + i)
// from P^f_i and E^pow2 (pin). nsm: the device's SM count.
template <typename Real, int DP>
__global__ void __launch_bounds__(32 * CW_SCAN)
    k_c2_level(KP<Real> p, Cov2Args<Real> a, int pow2, int cnt, int sq, int fac, int nsm,
               const Real* __restrict__ pin, Real* __restrict__ pout) {
  pdl_wait();
  pdl_trigger();
  constexpr long DD = (long)DP * DP;
  const int fw = cov_fw(blockIdx.x, nsm);
  const int i = blockIdx.x - sq;
  Real* pf = a.tab + (long)TPF * p.nT * DD;
  if (i >= 0)
    cov2_conly<Real, DP>(p, pf + (long)i * DD, pin, pf + (long)(pow2 + i) * DD, a.status, fw);
  else
    cov2_power<Real, DP>(p, pin, pout, fac != 0, a.status, fw);
}

// ---------------------------------------------------------------------------
// Per-step tables, one CTA of two warps per step t.
//   warp 0 (gain tables): P^p_t = F P^f_(t-1) F^T + Q (P0 at t = 0),
//     L_S = chol(P^p_t + r I), ldt[t] = 2 sum log (L_S)_ii, W = L_S^{-1},
//     K'_t = r W^T W.
//   warp 1 (backward tables): X = F P^f_t, P^p_(t+1) = X F^T + Q,
//     L_P = chol(P^p_(t+1)), Y = L_P^{-1} X, Sigma_t = P^f_t - Y^T Y,
//     G_t^T = L_P^{-T} Y, chol(Sigma_t)  (t = T - 1: G = 0, chol(P^f_t)).
// Shared memory is laid out for the case at hand (Tab2Layout): with a
// diagonal F the F and F^T slots and the gain warp's prediction scratch are
// left out, Q is read from L2, the gain warp's W overwrites P^f_(t-1) and the
// backward warp reuses its slots as the steps free them (X -> Y -> G; the
// right-aligned factor rows -> chol(Sigma) rows), so that more steps' CTAs are
// resident at once (the kernel is latency-bound): 6 slots and 4 vectors with a
// diagonal F, eight CTAs per SM in FP32 at DP = 32 (as many as the registers
// allow), one wave for T = 1024 on 152 SMs.
// ---------------------------------------------------------------------------
template <typename Real, int DP> struct Tab2Layout {
  static constexpr int MAT = Lay<Real, DP>::MAT, VEC = Lay<Real, DP>::VEC;
  int sphi, sF, sFT, SPm, SP, LSg, SW, SXg, SX, LSb, LRb, vdg, vdb, vdb2, total;
  __host__ __device__ Tab2Layout(bool fdiag) {
    int o = 0;
    sphi = o; o += VEC;
    sF = sFT = SXg = -1;
    if (!fdiag) { sF = o; o += MAT; sFT = o; o += MAT; }
    SPm = o; o += MAT;
    SW = SPm;   // the gain warp's W = L_S^{-1} overwrites P^f_(t-1) once the prediction has read it
    SP = o; o += MAT;
    LSg = o; o += MAT;
    if (!fdiag) { SXg = o; o += MAT; }
    SX = o; o += MAT;
    LSb = o; o += MAT;
    LRb = o; o += MAT;
    vdg = o; o += VEC;
    vdb = o; o += VEC;
    vdb2 = o; o += VEC;
    total = o;
  }
  __host__ __device__ size_t bytes() const { return (size_t)total * sizeof(Real); }
};

template <typename Real, int DP>
__global__ void __launch_bounds__(64) k_c2_tables(KP<Real> p, Cov2Args<Real> a) {
  pdl_wait();
  pdl_trigger();
  refresh_delta(p);
  constexpr int LD = Lay<Real, DP>::LD;
  constexpr long DD = (long)DP * DP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const Tab2Layout<Real, DP> Lo(p.fdiag != 0);
  Real* sphi = sm + Lo.sphi;
  Real* sF = p.fdiag ? nullptr : sm + Lo.sF;
  Real* sFT = p.fdiag ? nullptr : sm + Lo.sFT;
  Real* SPm = sm + Lo.SPm;    // P^f_(t-1)
  Real* SP = sm + Lo.SP;      // P^f_t
  Real* LSg = sm + Lo.LSg;    // warp 0: chol(S) (LS form)
  Real* SW = sm + Lo.SW;      //         W = L_S^{-1}
  Real* SXg = p.fdiag ? nullptr : sm + Lo.SXg;   // F P^f_(t-1) (dense F)
  Real* SX = sm + Lo.SX;      // warp 1: prediction scratch, X = F P^f_t, then Y, then G
  Real* LSb = sm + Lo.LSb;    //         chol(P^p_(t+1)) (LS form), then chol(Sigma) (LS form)
  Real* LRb = sm + Lo.LRb;    //         chol(P^p_(t+1)) right-aligned rows, then chol(Sigma) rows
  Real* vdg = sm + Lo.vdg;
  Real* vdb = sm + Lo.vdb;
  Real* vdb2 = sm + Lo.vdb2;
  const int t = blockIdx.x;
  const Real* pf = a.tab + (long)TPF * p.nT * DD;
  if (t > 0) stage_mats<Real, DP>(SPm, pf + (long)(t - 1) * DD, DD, 1);
  stage_mats<Real, DP>(SP, pf + (long)t * DD, DD, 1);
  if (!p.fdiag) {
    for (int q = threadIdx.x; q < DP * DP; q += blockDim.x) {
      const int i = q / DP, j = q % DP;
      sF[i * LD + j] = p.F[q];
      sFT[j * LD + i] = p.F[q];
    }
  }
  if (threadIdx.x < DP) sphi[threadIdx.x] = p.F[threadIdx.x * DP + threadIdx.x];
  cp_async_wait<0>();
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  int bad = 0;
  // P^p of the step after the one whose P^f is in slot SPf (scratch slot SS, dense F)
  auto predict = [&](const Real* SPf, Real* SS, Real (&pp)[DP]) {
    if (p.fdiag) {
      Real pr[DP], ph[DP], qr[DP];
      ld_row<Real, DP>(SPf, row, pr);
      ld_vec<Real, DP>(sphi, ph);
      ld_vec<Real, DP>(p.Q + row * DP, qr);   // Q rows from L2
      const Real phi = sphi[row];
#pragma unroll
      for (int j = 0; j < DP; ++j) pp[j] = fma(pr[j], phi * ph[j], qr[j]);
    } else {
      Real xr[DP];
      mm_row<Real, DP>(sF + row * LD, SPf, xr);
      __syncwarp();
      st_row<Real, DP>(SS, row, xr, act);
      __syncwarp();
      mm_row<Real, DP>(SS + row * LD, sFT, pp);
      Real qr[DP];
      ld_vec<Real, DP>(p.Q + row * DP, qr);   // Q rows from L2
#pragma unroll
      for (int j = 0; j < DP; ++j) pp[j] += qr[j];
      symmetrise_store<Real, DP>(SS, pp, lane);
    }
  };
  if (warp == 0) {
    Real pp[DP];
    if (t == 0) ld_vec<Real, DP>(p.P0 + row * DP, pp);
    else predict(SPm, SXg, pp);
#pragma unroll
    for (int j = 0; j < DP; ++j) pp[j] += (j == lane && j < p.d) ? p.r : (Real)0;
    chol_la<Real, DP>(pp, LSg, nullptr, nullptr, vdg, nullptr, p.d, lane, &bad);
    double lg = (lane < p.d) ? -log((double)vdg[lane]) : 0.0;
    lg = warp_sum<double>(lg);
    if (lane == 0) a.ldt[t] = 2.0 * lg;
    Real r[DP];
#pragma unroll
    for (int j = 0; j < DP; ++j) r[j] = (j == lane) ? (Real)1 : (Real)0;
    fsolve_pf<Real, DP, true>(LSg, vdg, r, SW, lane);
    __syncwarp();
    Real kr[DP];
    mm_col<Real, DP>(SW, row, SW, kr);
#pragma unroll
    for (int j = 0; j < DP; ++j) kr[j] *= p.r;
    if (act) st_vec<Real, DP>(a.tab + ((long)TK * p.nT + t) * DD + row * DP, kr);
  } else {
    Real sig[DP];
    if (t < p.nT - 1) {
      Real pp[DP];
      predict(SP, SX, pp);   // SX: scratch until X is formed
      // X = F P^f_t
      Real xr[DP];
      if (p.fdiag) {
        ld_row<Real, DP>(SP, row, xr);
        const Real phi = sphi[row];
#pragma unroll
        for (int j = 0; j < DP; ++j) xr[j] *= phi;
      } else {
        mm_row<Real, DP>(sF + row * LD, SP, xr);
      }
      chol_la<Real, DP>(pp, LSb, nullptr, LRb, vdb, nullptr, p.d, lane, &bad);
      st_row<Real, DP>(SX, row, xr, act);
      __syncwarp();
      Real rr[DP];
      ld_col<Real, DP>(SX, row, rr);
      __syncwarp();
      fsolve_pf<Real, DP, true>(LSb, vdb, rr, SX, lane);   // Y = L_P^{-1} X (column `lane`), over X
      __syncwarp();
      ld_row<Real, DP>(SP, row, sig);
      mm_col<Real, DP, true, true>(SX, row, SX, sig);       // Sigma = P^f - Y^T Y
      ld_col<Real, DP>(SX, row, rr);
      __syncwarp();
      bsolve_rot<Real, DP>(LRb, vdb, rr, SX, lane);         // row `lane` of G = L_P^{-T} Y column, over Y
      __syncwarp();
      Real g[DP];
      ld_row<Real, DP>(SX, row, g);
      if (act) st_vec<Real, DP>(a.tab + ((long)TG * p.nT + t) * DD + row * DP, g);
    } else {
      Real z[DP];
      zero<Real, DP>(z);
      if (act) st_vec<Real, DP>(a.tab + ((long)TG * p.nT + t) * DD + row * DP, z);
      ld_row<Real, DP>(SP, row, sig);
    }
    chol_la<Real, DP>(sig, LSb, LRb, nullptr, vdb2, nullptr, p.d, lane, &bad);
    Real lr[DP];
    ld_row<Real, DP>(LRb, row, lr);
    if (act) st_vec<Real, DP>(a.tab + ((long)TLS * p.nT + t) * DD + row * DP, lr);
  }
  if (bad && lane == 0) atomicOr(a.status, ST_NOT_PD);
}

// ---------------------------------------------------------------------------
// Products over the means partition, two CTAs of CW_SCAN warps per means block
// k (steps s..e), products split by output columns across the warps, the next
// step's table staged while the current product runs:
//   CTA 2k:     TGP[t] = G_s ... G_(t-1) for t = s..e, BGH[k] = G_s ... G_e,
//               ld[k] = sum of ldt[t];
//   CTA 2k + 1: BAH[k] = M_e ... M_s, M_t = K'_t F.
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __launch_bounds__(32 * CW_SCAN) k_c2_products(KP<Real> p, Cov2Args<Real> a) {
  pdl_wait();
  pdl_trigger();
  using Z = Cov2Sizes<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC, LD = Lay<Real, DP>::LD, NC = DP / CW_SCAN;
  constexpr long DD = (long)DP * DP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  Real* SACC = sm;             // running product
  Real* STb = SACC + MAT;      // two staged tables
  Real* SM = STb + 2 * MAT;    // M_t = K'_t F (dense F)
  Real* sF = SM + MAT;
  Real* sphi = sF + MAT;
  const int k = blockIdx.x >> 1, which = blockIdx.x & 1;
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  const int c0 = warp * NC;
  const Real* src = a.tab + (long)(which == 0 ? TG : TK) * p.nT * DD;
  stage_mats<Real, DP>(STb, src + (long)s * DD, DD, 1);
  for (int q = threadIdx.x; q < DP * DP; q += blockDim.x) {
    const int i = q / DP, j = q % DP;
    SACC[i * LD + j] = (i == j) ? (Real)1 : (Real)0;
    sF[i * LD + j] = p.F[q];
  }
  if (threadIdx.x < DP) sphi[threadIdx.x] = p.F[threadIdx.x * DP + threadIdx.x];
  for (int t = s; t <= e; ++t) {
    Real* cur = STb + ((t - s) & 1) * MAT;
    if (t < e) stage_mats<Real, DP>(STb + ((t - s + 1) & 1) * MAT, src + (long)(t + 1) * DD, DD, 1);
    if (t < e) cp_async_wait<1>();
    else cp_async_wait<0>();
    __syncthreads();
    Real out[NC];
    if (which == 0) {
      if (act && warp == 0) {   // TGP[t] = running product before G_t
        Real r[DP];
        ld_row<Real, DP>(SACC, row, r);
        st_vec<Real, DP>(a.tab + ((long)TGP * p.nT + t) * DD + row * DP, r);
      }
      mm_row_c<Real, DP, NC>(SACC + row * LD, cur, c0, out);   // ACC G_t
    } else {
      if (p.fdiag) {   // M_t row = K'_t row scaled by diag F; ACC <- M_t ACC
        Real kr[DP], ph[DP], mr[DP];
        ld_row<Real, DP>(cur, row, kr);
        ld_vec<Real, DP>(sphi, ph);
#pragma unroll
        for (int j = 0; j < DP; ++j) mr[j] = kr[j] * ph[j];
#pragma unroll
        for (int j = 0; j < NC; ++j) out[j] = (Real)0;
        // out[j] = sum_q M[row][q] ACC[q][c0 + j]
#pragma unroll
        for (int q = 0; q < DP; ++q) {
          Real b[NC];
          ldn<Real, NC>(SACC + q * LD + c0, b);
          fma_row<Real, NC>(mr[q], b, out);
        }
      } else {
        Real mr[NC];
        mm_row_c<Real, DP, NC>(cur + row * LD, sF, c0, mr);   // M_t = K'_t F
        if (act) stn<Real, NC>(SM + row * LD + c0, mr);
        __syncthreads();
        mm_row_c<Real, DP, NC>(SM + row * LD, SACC, c0, out);  // M_t ACC
      }
    }
    __syncthreads();
    if (act) stn<Real, NC>(SACC + row * LD + c0, out);
    __syncthreads();
  }
  if (act && warp == 0) {
    Real r[DP];
    ld_row<Real, DP>(SACC, row, r);
    st_vec<Real, DP>(a.btab + ((long)(which == 0 ? BGH : BAH) * p.nb + k) * DD + row * DP, r);
  }
  if (which == 0 && warp == 1) {
    double acc = 0.0;
    for (int t = s + lane; t <= e; t += 32) acc += a.ldt[t];
    acc = warp_sum<double>(acc);
    if (lane == 0) a.ld[k] = acc;
  }
  (void)VEC;
}

}  // namespace auxk
