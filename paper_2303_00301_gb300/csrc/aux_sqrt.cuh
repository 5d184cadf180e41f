// aux_sqrt.cuh — square-root form of the per-chain parallel filter.
//
// Section 4.1 traces the single-precision divergence of the parallel filter
// to the covariance recursions and names the square-root form as the fix.
// Here every covariance-like block of an element is carried as a factor,
// C = U U^T and J = Z Z^T (Appendix A.2.1's elements (A, b, C, eta, J)), and a
// new covariance factor is formed by an orthogonal triangularisation
// tria([X1, X2]) = the lower-triangular L with L L^T = X1 X1^T + X2 X2^T
// (Householder reflections; no covariance is formed and then factorised):
//   element t >= 1  S = Q + R = Ls Ls^T, K = Q S^{-1}, K' = r S^{-1} = I - K,
//                   A = K' F, U = tria([K' chol Q, sqrt(r) K]) (Joseph form),
//                   Z = F^T Ls^{-T}, b = b_t + K (y_t - b_t), eta = F^T S^{-1} (y_t - b_t);
//   element t = 0   the same with P0 for Q and m0 for b_t, A = 0, Z = 0, eta = 0;
//   operator        W = U_i^T Z_j, Xi = chol(I + W W^T), Xi' = chol(I + W^T W)
//                   (both >= I: well conditioned), M^{-1} = I - U_i Xi^{-T} Xi^{-1} W Z_j^T,
//                   A = A_j M^{-1} A_i, b = A_j M^{-1} (b_i + U_i U_i^T eta_j) + b_j,
//                   U = tria([A_j U_i Xi^{-T}, U_j]),
//                   eta = (M^{-1} A_i)^T (eta_j - Z_j Z_j^T b_i) + eta_i,
//                   Z = tria([A_i^T Z_j Xi'^{-T}, Z_i]);
//   in-block filter the square-root Kalman step from (m^f_{t-1}, U^f_{t-1}):
//                   U^p = tria([F U^f, chol Q]), Ls = chol(U^p U^p^T + r I) (S >= r I),
//                   l_t = log N(y_t; m^p, Ls Ls^T), K = U^p U^p^T S^{-1},
//                   m^f = m^p + K (y_t - m^p), U^f = tria([K' U^p, sqrt(r) K]).
// The Cholesky factorisations left (of S >= r I and of I + W W^T >= I) are of
// matrices bounded away from singular; every covariance factor that can lose
// definiteness (C, J, P^p, P^f) comes out of tria.
// Padding: covariance factors keep zero rows and columns past d; the factors
// used only in solves (Ls, Xi, Xi') carry a unit diagonal there.
//
// Kernels (one warp per CTA: the square-root workspace is large):
//   k_sr_reduce      per (chain, block): the block's elements folded with the operator;
//   k_sr_scan_level  one Hillis-Steele round over the block aggregates;
//   k_sr_apply       per (chain, block): the square-root Kalman steps from the
//                    block's incoming prefix, with m^f, P^f, the likelihood terms
//                    and (APPLY_EPI) the backward elements (G_t, U_t) of the
//                    (G, U) scan, chol(Sigma_t) from tria in Joseph form.
// The aggregates use the covariance form's layout [A, U, Z, b, eta] (same size).
#pragma once
#include "aux_cov.cuh"

namespace auxk {

template <typename Real, int DP> struct SrSizes {
  static constexpr int MAT = Lay<Real, DP>::MAT, VEC = Lay<Real, DP>::VEC;
  static constexpr int ES = 3 * DP * DP + 2 * DP;
  static constexpr int VROW = 2 * VEC;   // one row of a tria input (2 DP, 16-byte aligned)
  // reduce / scan: model (F, chol Q), element constants (A, U, Z, K, F^T S^{-1}),
  // state (A, U, Z), 7 scratch slots; vectors: 2 inverse diagonals, 3 temporaries,
  // b, eta of the state and of the element, signs, tria row
  static constexpr size_t RED_SMEM = (17 * MAT + 10 * VEC + VROW) * sizeof(Real);
  // covariance apply of the table modes: 15 slots, 3 vectors
  static constexpr size_t COVAPP_SMEM = (15 * MAT + 2 * VEC + VROW) * sizeof(Real);
  // apply: F, chol Q, U^f, U^p, K, K', Ls (LS + LR), P^p, 3 scratch, G, G product;
  // vectors: inverse diagonal, m^f, m^p, innovation / noise, z, U_t, signs, tria row
  static constexpr size_t APP_SMEM = (14 * MAT + 7 * VEC + VROW) * sizeof(Real);
};

// ---------------------------------------------------------------------------
// tria of one warp: lane i holds row i of X = [X1, X2] (DP x 2 DP, rows >= DP
// zero) in x[]. Householder reflections from the right (X <- X H_0 ... H_{DP-1},
// H_j built from row j) make X lower triangular; the signs are then fixed so
// that the diagonal is non-negative. On exit x[0..DP) is row i of L
// (L L^T = X X^T) and x[DP..2DP) is zero. vrow: a shared row of 2 DP
// elements, vsg: a shared vector (both warp-private).
// ---------------------------------------------------------------------------
template <typename T, int DP>
__device__ __forceinline__ void tria_reg(T (&x)[2 * DP], T* vrow, T* vsg, int lane) {
  constexpr int K = 2 * DP;
#pragma unroll 1
  for (int j = 0; j < DP; ++j) {
    __syncwarp();
    if (lane == j) {
#pragma unroll
      for (int c = 0; c < K; ++c) vrow[c] = x[c];
    }
    __syncwarp();
    T part = (T)0;
    for (int c = j + 1 + lane; c < K; c += 32) part = fma(vrow[c], vrow[c], part);
    const T sigma = warp_sum<T>(part);
    const T alpha = vrow[j];
    T diag = alpha;
    if (sigma > (T)0) {   // warp-uniform
      const T nrm = sqrt(fma(alpha, alpha, sigma));
      const T beta = alpha > (T)0 ? -nrm : nrm;
      const T v0 = alpha - beta;
      const T scale = (T)2 / fma(v0, v0, sigma);
      T d0 = (T)0, d1 = (T)0;
#pragma unroll
      for (int c = 0; c < K; c += 2) {
        const T va = c > j ? vrow[c] : (c == j ? v0 : (T)0);
        const T vb = c + 1 > j ? vrow[c + 1] : (c + 1 == j ? v0 : (T)0);
        d0 = fma(x[c], va, d0);
        d1 = fma(x[c + 1], vb, d1);
      }
      const T f = -(d0 + d1) * scale;
      __syncwarp();   // the row is read again below, not kept in registers
#pragma unroll
      for (int c = 0; c < K; ++c) {
        const T vc = c > j ? vrow[c] : (c == j ? v0 : (T)0);
        x[c] = fma(f, vc, x[c]);
      }
      diag = beta;
    }
    if (lane == j) {
#pragma unroll
      for (int c = 0; c < K; ++c) {
        if (c > j) x[c] = (T)0;
        if (c == j) x[c] = diag;
      }
    }
  }
  __syncwarp();
  T dg = (T)0;
#pragma unroll
  for (int c = 0; c < DP; ++c)
    if (c == lane) dg = x[c];
  if (lane < DP) vsg[lane] = dg < (T)0 ? (T)-1 : (T)1;
  __syncwarp();
#pragma unroll
  for (int c = 0; c < DP; ++c) x[c] *= vsg[c];
  __syncwarp();
}

// the lane's row of [X1 row, X2 row] into x[]
template <typename T, int DP>
__device__ __forceinline__ void tria_row(const T (&a)[DP], const T (&b)[DP], T (&x)[2 * DP]) {
#pragma unroll
  for (int c = 0; c < DP; ++c) { x[c] = a[c]; x[DP + c] = b[c]; }
}

// rows of S^{-1} B (B symmetric, or any B: the result is (S^{-1} B)^T for a
// general B) through the factor of S: column `lane` of B forward, then backward.
// LS/LR/invd: the factor; Y: scratch slot; Out: result slot (row lane =
// (S^{-1} B[:, lane])^T). B is read through ld_col.
template <typename T, int DP>
__device__ __forceinline__ void solve_cols(const T* LS, const T* LR, const T* invd, const T* B, T* Y,
                                           T* Out, int lane) {
  const int row = lane < DP ? lane : 0;
  {
    T rr[DP];
    ld_col<T, DP>(B, row, rr);
    fsolve_rot<T, DP, true>(LS, invd, rr, Y, lane);
  }
  __syncwarp();
  {
    T rr[DP];
    ld_col<T, DP>(Y, row, rr);
    bsolve_rot<T, DP>(LR, invd, rr, Out, lane);
  }
  __syncwarp();
}

// the lane's row of a Cholesky factor (row-major, from chol_rot's LRow) with
// zero padding: rows >= d cleared (chol_rot puts a unit pivot there)
template <typename T, int DP>
__device__ __forceinline__ void zero_pad_row(T (&r)[DP], int d, int lane) {
  if (lane >= d) zero<T, DP>(r);
}

template <typename Real, int DP> struct SrWork {
  Real *T0, *T1, *T2, *T3, *T4, *T5, *T6;
  Real *vx, *vx2, *v1, *v2, *v3, *vsg, *vrow;
};

// ---------------------------------------------------------------------------
// (A_i, U_i, Z_i, b_i, eta_i) <- (A_i, U_i, Z_i, b_i, eta_i) (x) (A_j, U_j, Z_j, b_j, eta_j)
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__device__ void sr_combine(Real* SAi, Real* SUi, Real* SZi, Real* vbi, Real* vei, const Real* SAj,
                           const Real* SUj, const Real* SZj, const Real* vbj, const Real* vej,
                           const SrWork<Real, DP>& w, int d, int lane, int* bad) {
  constexpr int LD = Lay<Real, DP>::LD;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  __syncwarp();
  // W = U_i^T Z_j (T0), W^T (T1)
  Real wr[DP];
  mm_col<Real, DP>(SUi, row, SZj, wr);
  st_row<Real, DP>(w.T0, row, wr, act);
  st_col<Real, DP>(w.T1, row, wr, act);
  __syncwarp();
  // Xi = chol(I + W W^T): LS T2, LR T3, inverse diagonal vx
  {
    Real n[DP];
    mm_row<Real, DP>(w.T0 + row * LD, w.T1, n);
#pragma unroll
    for (int c = 0; c < DP; ++c) n[c] += (c == lane) ? (Real)1 : (Real)0;
    chol_rot<Real, DP>(n, w.T2, nullptr, w.T3, w.vx, nullptr, DP, lane, bad);
  }
  // Xi' = chol(I + W^T W): LS T4, inverse diagonal vx2
  {
    Real n[DP];
    mm_col<Real, DP>(w.T0, row, w.T0, n);
#pragma unroll
    for (int c = 0; c < DP; ++c) n[c] += (c == lane) ? (Real)1 : (Real)0;
    chol_rot<Real, DP>(n, w.T4, nullptr, nullptr, w.vx2, nullptr, DP, lane, bad);
  }
  // V1 = W Z_j^T (T5); Y^T = (N^{-1} V1)^T (T5, through T6)
  {
    Real v[DP];
    row_matT<Real, DP>(wr, SZj, v);
    __syncwarp();
    st_row<Real, DP>(w.T5, row, v, act);
    __syncwarp();
  }
  solve_cols<Real, DP>(w.T2, w.T3, w.vx, w.T5, w.T6, w.T5, lane);
  // M^{-1} = I - U_i Y (T6)
  Real ur[DP];
  ld_row<Real, DP>(SUi, row, ur);
  {
    Real mr[DP];
    row_matT<Real, DP>(ur, w.T5, mr);
#pragma unroll
    for (int c = 0; c < DP; ++c) mr[c] = ((c == lane) ? (Real)1 : (Real)0) - mr[c];
    __syncwarp();
    st_row<Real, DP>(w.T6, row, mr, act);
    __syncwarp();
  }
  // Q1 = M^{-1} A_i (T0); A = A_j Q1 (T5)
  {
    Real q[DP];
    mm_row<Real, DP>(w.T6 + row * LD, SAi, q);
    st_row<Real, DP>(w.T0, row, q, act);
    __syncwarp();
    mm_row<Real, DP>(SAj + row * LD, w.T0, q);
    st_row<Real, DP>(w.T5, row, q, act);
  }
  // b = A_j M^{-1} (b_i + U_i U_i^T eta_j) + b_j
  if (act) w.v1[lane] = dot_col_vec<Real, DP>(SUi, row, vej);
  __syncwarp();
  if (act) w.v2[lane] = vbi[lane] + dot_row_vec<Real, DP>(SUi + row * LD, w.v1);
  __syncwarp();
  if (act) w.v3[lane] = dot_row_vec<Real, DP>(w.T6 + row * LD, w.v2);
  __syncwarp();
  const Real bnew = act ? vbj[lane] + dot_row_vec<Real, DP>(SAj + row * LD, w.v3) : (Real)0;
  // eta = Q1^T (eta_j - Z_j Z_j^T b_i) + eta_i
  if (act) w.v1[lane] = dot_col_vec<Real, DP>(SZj, row, vbi);
  __syncwarp();
  if (act) w.v2[lane] = vej[lane] - dot_row_vec<Real, DP>(SZj + row * LD, w.v1);
  __syncwarp();
  const Real enew = act ? vei[lane] + dot_col_vec<Real, DP>(w.T0, row, w.v2) : (Real)0;
  // U = tria([A_j U_i Xi^{-T}, U_j]); S1 = Xi^{-1} U_i^T (T1)
  Real x[2 * DP];
  {
    fsolve_rot<Real, DP, true>(w.T2, w.vx, ur, w.T1, lane);
    __syncwarp();
    Real ar[DP], pr[DP], uj[DP];
    ld_row<Real, DP>(SAj, row, ar);
    row_matT<Real, DP>(ar, w.T1, pr);
    ld_row<Real, DP>(SUj, row, uj);
    tria_row<Real, DP>(pr, uj, x);
  }
  tria_reg<Real, DP>(x, w.vrow, w.vsg, lane);
  Real unew[DP];
#pragma unroll
  for (int c = 0; c < DP; ++c) unew[c] = x[c];
  // Z = tria([A_i^T Z_j Xi'^{-T}, Z_i]); S2 = Xi'^{-1} Z_j^T (T1)
  {
    Real zr[DP];
    ld_row<Real, DP>(SZj, row, zr);
    __syncwarp();
    fsolve_rot<Real, DP, true>(w.T4, w.vx2, zr, w.T1, lane);
    __syncwarp();
    Real ac[DP], pr[DP], zi[DP];
    ld_col<Real, DP>(SAi, row, ac);
    row_matT<Real, DP>(ac, w.T1, pr);
    ld_row<Real, DP>(SZi, row, zi);
    tria_row<Real, DP>(pr, zi, x);
  }
  tria_reg<Real, DP>(x, w.vrow, w.vsg, lane);
  // outputs
  Real ar[DP];
  ld_row<Real, DP>(w.T5, row, ar);
  __syncwarp();
  st_row<Real, DP>(SAi, row, ar, act);
  st_row<Real, DP>(SUi, row, unew, act);
  {
    Real zr[DP];
#pragma unroll
    for (int c = 0; c < DP; ++c) zr[c] = x[c];
    st_row<Real, DP>(SZi, row, zr, act);
  }
  if (act) { vbi[lane] = bnew; vei[lane] = enew; }
  __syncwarp();
}

// global aggregate <-> slots ([A, U, Z, b, eta], the covariance form's layout)
template <typename Real, int DP>
__device__ __forceinline__ void sr_load(const Real* g, Real* SA, Real* SU, Real* SZ, Real* vb, Real* ve,
                                        int lane) {
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  Real r[DP];
  ld_vec<Real, DP>(g + row * DP, r);
  st_row<Real, DP>(SA, row, r, act);
  ld_vec<Real, DP>(g + DP * DP + row * DP, r);
  st_row<Real, DP>(SU, row, r, act);
  ld_vec<Real, DP>(g + 2 * DP * DP + row * DP, r);
  st_row<Real, DP>(SZ, row, r, act);
  if (act) { vb[lane] = g[3 * DP * DP + lane]; ve[lane] = g[3 * DP * DP + DP + lane]; }
  __syncwarp();
}
template <typename Real, int DP>
__device__ __forceinline__ void sr_store(Real* g, const Real* SA, const Real* SU, const Real* SZ,
                                         const Real* vb, const Real* ve, int lane) {
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  __syncwarp();
  Real r[DP];
  ld_row<Real, DP>(SA, row, r);
  if (act) st_vec<Real, DP>(g + row * DP, r);
  ld_row<Real, DP>(SU, row, r);
  if (act) st_vec<Real, DP>(g + DP * DP + row * DP, r);
  ld_row<Real, DP>(SZ, row, r);
  if (act) st_vec<Real, DP>(g + 2 * DP * DP + row * DP, r);
  if (act) { g[3 * DP * DP + lane] = vb[lane]; g[3 * DP * DP + DP + lane] = ve[lane]; }
}

// ---------------------------------------------------------------------------
// Gain quantities of one conditioning on y ~ N(x, r I) with prior covariance
// factor rows (cov = the symmetric prior covariance in slot SP, its zero-padded
// factor rows `fac`): S = cov + r I = Ls Ls^T (LS/LR/invd), K = cov S^{-1} (SK),
// K' = r S^{-1} (SKp), and the posterior factor row tria([K' fac, sqrt(r) K])
// into x. Y: scratch slot.
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__device__ __forceinline__ void sr_condition(const KP<Real>& p, const Real* SP, const Real* SFac,
                                             Real* LS, Real* LR, Real* invd, Real* SK, Real* SKp, Real* Y,
                                             Real* vrow, Real* vsg, Real (&x)[2 * DP], int lane, int* bad) {
  constexpr int LD = Lay<Real, DP>::LD;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  {
    Real s[DP];
    ld_row<Real, DP>(SP, row, s);
#pragma unroll
    for (int c = 0; c < DP; ++c) s[c] += (c == lane) ? (lane < p.d ? p.r : (Real)1) : (Real)0;
    chol_rot<Real, DP>(s, LS, nullptr, LR, invd, nullptr, p.d, lane, bad);
  }
  solve_cols<Real, DP>(LS, LR, invd, SP, Y, SK, lane);   // (S^{-1} P)^T = P S^{-1}
  {
    // identity columns through the factor: S^{-1} (symmetric), times r
    Real e[DP];
#pragma unroll
    for (int c = 0; c < DP; ++c) e[c] = (c == lane) ? (Real)1 : (Real)0;
    fsolve_rot<Real, DP, true>(LS, invd, e, Y, lane);
    __syncwarp();
    ld_col<Real, DP>(Y, row, e);
    bsolve_rot<Real, DP>(LR, invd, e, SKp, lane);
    __syncwarp();
    Real k[DP];
    ld_row<Real, DP>(SKp, row, k);
#pragma unroll
    for (int c = 0; c < DP; ++c) k[c] = (lane < p.d && c < p.d) ? p.r * k[c] : (Real)0;
    __syncwarp();
    st_row<Real, DP>(SKp, row, k, act);
    __syncwarp();
  }
  Real a[DP], b[DP];
  mm_row<Real, DP>(SKp + row * LD, SFac, a);
  ld_row<Real, DP>(SK, row, b);
#pragma unroll
  for (int c = 0; c < DP; ++c) b[c] *= p.sqrt_r;
  tria_row<Real, DP>(a, b, x);
  tria_reg<Real, DP>(x, vrow, vsg, lane);
}

// ---------------------------------------------------------------------------
// Phase 1: the block's elements folded with the square-root operator.
// ---------------------------------------------------------------------------
template <typename Real, int DP, bool COV>
__device__ __forceinline__ void sr_reduce_body(KP<Real> p, const Real* __restrict__ yt, Real* __restrict__ agg,
                                               const int* __restrict__ kmap, Real* __restrict__ dst1,
                                               Real* __restrict__ dst2, int32_t* __restrict__ cstatus) {
  refresh_delta(p);
  using Z = SrSizes<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC, LD = Lay<Real, DP>::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  Real* SF = sm;
  Real* SCQ = SF + MAT;
  Real* SAe = SCQ + MAT;
  Real* SUe = SAe + MAT;
  Real* SZe = SUe + MAT;
  Real* SK = SZe + MAT;
  Real* SFS = SK + MAT;
  Real* SA = SFS + MAT;
  Real* SU = SA + MAT;
  Real* SZ = SU + MAT;
  SrWork<Real, DP> w;
  w.T0 = SZ + MAT; w.T1 = w.T0 + MAT; w.T2 = w.T1 + MAT; w.T3 = w.T2 + MAT;
  w.T4 = w.T3 + MAT; w.T5 = w.T4 + MAT; w.T6 = w.T5 + MAT;
  w.vx = w.T6 + MAT; w.vx2 = w.vx + VEC; w.v1 = w.vx2 + VEC; w.v2 = w.v1 + VEC; w.v3 = w.v2 + VEC;
  w.vsg = w.v3 + VEC;
  Real* vb = w.vsg + VEC;
  Real* ve = vb + VEC;
  Real* vbe = ve + VEC;
  Real* vee = vbe + VEC;
  w.vrow = vee + VEC;
  const int lane = threadIdx.x;
  // COV: matrix parts only (the covariance pass of the table modes), CTA b reduces
  // covariance block kmap[b] (or b) of the shared model; else block k of chain c
  const int c = COV ? 0 : blockIdx.x / p.nb;
  const int k = COV ? (kmap ? kmap[blockIdx.x] : blockIdx.x) : blockIdx.x % p.nb;
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  const Real* ytc = COV ? nullptr : yt + (long)c * p.nT * p.d;
  int bad = 0;
  Real r[DP], x[2 * DP];
  // model: F, chol Q (zero padded)
  ld_vec<Real, DP>(p.F + row * DP, r);
  st_row<Real, DP>(SF, row, r, act);
  ld_vec<Real, DP>(p.Q + row * DP, r);
  chol_rot<Real, DP>(r, w.T0, SCQ, nullptr, w.vx, nullptr, p.d, lane, &bad);
  __syncwarp();
  ld_row<Real, DP>(SCQ, row, r);
  zero_pad_row<Real, DP>(r, p.d, lane);
  __syncwarp();
  st_row<Real, DP>(SCQ, row, r, act);
  // element constants (t >= 1): condition the prior covariance Q on y
  ld_vec<Real, DP>(p.Q + row * DP, r);
  st_row<Real, DP>(w.T6, row, r, act);
  __syncwarp();
  sr_condition<Real, DP>(p, w.T6, SCQ, w.T0, w.T1, w.vx, SK, w.T2, w.T3, w.vrow, w.vsg, x, lane, &bad);
  {
    Real u[DP];
#pragma unroll
    for (int cc = 0; cc < DP; ++cc) u[cc] = x[cc];
    st_row<Real, DP>(SUe, row, u, act);
    mm_row<Real, DP>(w.T2 + row * LD, SF, u);     // A = K' F
    st_row<Real, DP>(SAe, row, u, act);
  }
  // Z = F^T Ls^{-T}: (Ls^{-1} F)^T; F^T S^{-1} = (S^{-1} F)^T
  {
    Real fc[DP];
    ld_col<Real, DP>(SF, row, fc);
    fsolve_rot<Real, DP, true>(w.T0, w.vx, fc, w.T4, lane);
    __syncwarp();
    ld_col<Real, DP>(w.T4, row, fc);
    st_row<Real, DP>(SZe, row, fc, act);
    __syncwarp();
  }
  solve_cols<Real, DP>(w.T0, w.T1, w.vx, SF, w.T4, SFS, lane);
  // the block's first element
  const Real bdyn = p.b[row];
  auto elem_vecs = [&](int t, Real* vbo, Real* veo) {   // b and eta of element t >= 1
    if (COV) {
      if (act) { vbo[lane] = (Real)0; veo[lane] = (Real)0; }
      __syncwarp();
      return;
    }
    const Real yi = lane < p.d ? ytc[(long)t * p.d + lane] : (Real)0;
    __syncwarp();
    if (act) w.v1[lane] = lane < p.d ? yi - bdyn : (Real)0;
    __syncwarp();
    if (act) {
      vbo[lane] = bdyn + dot_row_vec<Real, DP>(SK + row * LD, w.v1);
      veo[lane] = dot_row_vec<Real, DP>(SFS + row * LD, w.v1);
    }
    __syncwarp();
  };
  if (s == 0) {
    // t = 0: condition P0 on y_0; A = 0, Z = 0, eta = 0
    ld_vec<Real, DP>(p.P0 + row * DP, r);
    st_row<Real, DP>(w.T6, row, r, act);
    chol_rot<Real, DP>(r, w.T0, w.T5, nullptr, w.vx, nullptr, p.d, lane, &bad);
    __syncwarp();
    ld_row<Real, DP>(w.T5, row, r);
    zero_pad_row<Real, DP>(r, p.d, lane);
    __syncwarp();
    st_row<Real, DP>(w.T5, row, r, act);
    __syncwarp();
    sr_condition<Real, DP>(p, w.T6, w.T5, w.T0, w.T1, w.vx, w.T3, w.T2, w.T4, w.vrow, w.vsg, x, lane, &bad);
    Real u[DP];
#pragma unroll
    for (int cc = 0; cc < DP; ++cc) u[cc] = x[cc];
    st_row<Real, DP>(SU, row, u, act);
    zero<Real, DP>(u);
    st_row<Real, DP>(SA, row, u, act);
    st_row<Real, DP>(SZ, row, u, act);
    const Real m0 = p.m0[row];
    const Real yi = (!COV && lane < p.d) ? ytc[lane] : (Real)0;
    __syncwarp();
    if (act) w.v1[lane] = (!COV && lane < p.d) ? yi - m0 : (Real)0;
    __syncwarp();
    if (act) { vb[lane] = m0 + dot_row_vec<Real, DP>(w.T3 + row * LD, w.v1); ve[lane] = (Real)0; }
    __syncwarp();
  } else {
    Real u[DP];
    ld_row<Real, DP>(SAe, row, u);
    st_row<Real, DP>(SA, row, u, act);
    ld_row<Real, DP>(SUe, row, u);
    st_row<Real, DP>(SU, row, u, act);
    ld_row<Real, DP>(SZe, row, u);
    st_row<Real, DP>(SZ, row, u, act);
    elem_vecs(s, vb, ve);
  }
  for (int t = s + 1; t <= e; ++t) {
    elem_vecs(t, vbe, vee);
    sr_combine<Real, DP>(SA, SU, SZ, vb, ve, SAe, SUe, SZe, vbe, vee, w, p.d, lane, &bad);
  }
  if (COV) {   // (A, U, Z): the covariance form's (A, C, J) slots
    constexpr long DD = (long)DP * DP;
    Real* g = !kmap || blockIdx.x == 0 ? agg + (long)k * 3 * DD : (blockIdx.x == 1 ? dst1 : dst2);
    __syncwarp();
    Real q[DP];
    ld_row<Real, DP>(SA, row, q);
    if (act) st_vec<Real, DP>(g + row * DP, q);
    ld_row<Real, DP>(SU, row, q);
    if (act) st_vec<Real, DP>(g + DD + row * DP, q);
    ld_row<Real, DP>(SZ, row, q);
    if (act) st_vec<Real, DP>(g + 2 * DD + row * DP, q);
    if (bad && lane == 0) atomicOr(cstatus, ST_NOT_PD);
  } else {
    sr_store<Real, DP>(agg + (long)blockIdx.x * Z::ES, SA, SU, SZ, vb, ve, lane);
    if (bad && lane == 0) atomicOr(&p.status_iter[c], ST_NOT_PD);
  }
}

template <typename Real, int DP>
__global__ void __launch_bounds__(32, 1) k_sr_reduce(KP<Real> p, const Real* __restrict__ yt,
                                                     Real* __restrict__ agg) {
  sr_reduce_body<Real, DP, false>(p, yt, agg, nullptr, nullptr, nullptr, nullptr);
}

// ---------------------------------------------------------------------------
// Square-root covariance pass of the table modes (matrix parts only, layout
// (A, U, Z) in the covariance form's (A, C, J) slots): the distinct block
// aggregates (kmap), the prefixes by doubling, the in-block step with the
// per-step tables. Same tables as aux_cov.cuh's pass, from factors.
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __launch_bounds__(32, 1) k_srcov_reduce(KP<Real> p, Real* __restrict__ aggm,
                                                        int32_t* __restrict__ status, const int* __restrict__ kmap,
                                                        Real* __restrict__ dst1, Real* __restrict__ dst2) {
  sr_reduce_body<Real, DP, true>(p, nullptr, aggm, kmap, dst1, dst2, status);
}

// P[dst + i] = P[src + i] (x) Gk for CTA i < cnt; CTA cnt: Gk2 = Gk (x) Gk
template <typename Real, int DP>
__global__ void __launch_bounds__(32, 1) k_srcov_scan_double(KP<Real> p, Real* __restrict__ P,
                                                             const Real* __restrict__ Gk, Real* __restrict__ Gk2,
                                                             int src, int dst, int cnt, int32_t* __restrict__ status) {
  using Z = SrSizes<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC;
  constexpr long DD = (long)DP * DP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const int lane = threadIdx.x, i = blockIdx.x;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  Real* SA = sm;
  Real* SU = SA + MAT;
  Real* SZ = SU + MAT;
  Real* SAe = SZ + MAT;
  Real* SUe = SAe + MAT;
  Real* SZe = SUe + MAT;
  SrWork<Real, DP> w;
  w.T0 = SZe + MAT; w.T1 = w.T0 + MAT; w.T2 = w.T1 + MAT; w.T3 = w.T2 + MAT;
  w.T4 = w.T3 + MAT; w.T5 = w.T4 + MAT; w.T6 = w.T5 + MAT;
  w.vx = w.T6 + MAT; w.vx2 = w.vx + VEC; w.v1 = w.vx2 + VEC; w.v2 = w.v1 + VEC; w.v3 = w.v2 + VEC;
  w.vsg = w.v3 + VEC;
  Real* vb = w.vsg + VEC;
  Real* ve = vb + VEC;
  Real* vbe = ve + VEC;
  Real* vee = vbe + VEC;
  w.vrow = vee + VEC;
  const Real* L = i < cnt ? P + (long)(src + i) * 3 * DD : Gk;
  Real* out = i < cnt ? P + (long)(dst + i) * 3 * DD : Gk2;
  auto load3 = [&](const Real* g, Real* A, Real* U, Real* Zs) {
    Real q[DP];
    ld_vec<Real, DP>(g + row * DP, q);
    st_row<Real, DP>(A, row, q, act);
    ld_vec<Real, DP>(g + DD + row * DP, q);
    st_row<Real, DP>(U, row, q, act);
    ld_vec<Real, DP>(g + 2 * DD + row * DP, q);
    st_row<Real, DP>(Zs, row, q, act);
  };
  load3(L, SA, SU, SZ);
  load3(Gk, SAe, SUe, SZe);
  if (act) { vb[lane] = ve[lane] = vbe[lane] = vee[lane] = (Real)0; }
  __syncwarp();
  int bad = 0;
  sr_combine<Real, DP>(SA, SU, SZ, vb, ve, SAe, SUe, SZe, vbe, vee, w, p.d, lane, &bad);
  Real q[DP];
  ld_row<Real, DP>(SA, row, q);
  if (act) st_vec<Real, DP>(out + row * DP, q);
  ld_row<Real, DP>(SU, row, q);
  if (act) st_vec<Real, DP>(out + DD + row * DP, q);
  ld_row<Real, DP>(SZ, row, q);
  if (act) st_vec<Real, DP>(out + 2 * DD + row * DP, q);
  if (bad && lane == 0) atomicOr(status, ST_NOT_PD);
}

// ---------------------------------------------------------------------------
// Phase 2: out_k = in_{k-off} (x) in_k for k >= off, else in_k.
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __launch_bounds__(32, 1) k_sr_scan_level(KP<Real> p, const Real* __restrict__ in,
                                                         Real* __restrict__ out, int off) {
  using Z = SrSizes<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const int lane = threadIdx.x;
  const int c = blockIdx.x / p.nb, k = blockIdx.x % p.nb;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  const Real* g_in = in + (long)blockIdx.x * Z::ES;
  Real* g_out = out + (long)blockIdx.x * Z::ES;
  if (k < off) {
    for (int q = row; q < Z::ES / DP; q += DP) {
      if (!act) break;
      Real r[DP];
      ld_vec<Real, DP>(g_in + q * DP, r);
      st_vec<Real, DP>(g_out + q * DP, r);
    }
    return;
  }
  Real* SA = sm;
  Real* SU = SA + MAT;
  Real* SZ = SU + MAT;
  Real* SAe = SZ + MAT;
  Real* SUe = SAe + MAT;
  Real* SZe = SUe + MAT;
  SrWork<Real, DP> w;
  w.T0 = SZe + MAT; w.T1 = w.T0 + MAT; w.T2 = w.T1 + MAT; w.T3 = w.T2 + MAT;
  w.T4 = w.T3 + MAT; w.T5 = w.T4 + MAT; w.T6 = w.T5 + MAT;
  w.vx = w.T6 + MAT; w.vx2 = w.vx + VEC; w.v1 = w.vx2 + VEC; w.v2 = w.v1 + VEC; w.v3 = w.v2 + VEC;
  w.vsg = w.v3 + VEC;
  Real* vb = w.vsg + VEC;
  Real* ve = vb + VEC;
  Real* vbe = ve + VEC;
  Real* vee = vbe + VEC;
  w.vrow = vee + VEC;
  int bad = 0;
  sr_load<Real, DP>(in + (long)(blockIdx.x - off) * Z::ES, SA, SU, SZ, vb, ve, lane);
  sr_load<Real, DP>(g_in, SAe, SUe, SZe, vbe, vee, lane);
  sr_combine<Real, DP>(SA, SU, SZ, vb, ve, SAe, SUe, SZe, vbe, vee, w, p.d, lane, &bad);
  sr_store<Real, DP>(g_out, SA, SU, SZ, vb, ve, lane);
  if (bad && lane == 0) atomicOr(&p.status_iter[c], ST_NOT_PD);
}

// ---------------------------------------------------------------------------
// Phase 3: square-root Kalman steps over the block from its incoming prefix
// (the inclusive aggregate of block k - 1: b = m^f_{s-1}, U = U^f_{s-1}).
// Writes m^f (a.mf), P^f = U^f U^f^T (a.Pf) when given, and the likelihood
// terms (APPLY_LOGZ / APPLY_STORE_Q / APPLY_REV_DIFF as the covariance form).
// With APPLY_EPI also the backward elements of Eq. (A.14),
//   G_t = P^f_t F^T (P^p_{t+1})^{-1},  chol(Sigma_t) = tria([(I - G_t F) U^f_t, G_t chol Q])
//   (Joseph form of Sigma_t = P^f_t - G_t P^p_{t+1} G_t^T),
//   U_t = m^f_t - G_t m^p_{t+1} + chol(Sigma_t) eps_t   (G_{T-1} = 0, chol(Sigma_{T-1}) = U^f_{T-1}),
// and the block aggregates of the (G, U) scan: G_s ... G_e and
// sum_t (G_s ... G_{t-1}) U_t.
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __launch_bounds__(32, 1) k_sr_apply(KP<Real> p, ApplyArgs<Real> a) {
  refresh_delta(p);
  using Z = SrSizes<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC, LD = Lay<Real, DP>::LD;
  constexpr long DD = (long)DP * DP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  Real* SF = sm;
  Real* SCQ = SF + MAT;
  Real* SUf = SCQ + MAT;
  Real* SUp = SUf + MAT;
  Real* SK = SUp + MAT;
  Real* SKp = SK + MAT;
  Real* SLS = SKp + MAT;
  Real* SLR = SLS + MAT;
  Real* SP = SLR + MAT;     // P^p of the next conditioning
  Real* SY = SP + MAT;
  Real* SW = SY + MAT;
  Real* SB = SW + MAT;
  Real* SG = SB + MAT;
  Real* SGP = SG + MAT;     // G_s ... G_{t-1}
  Real* vx = SGP + MAT;
  Real* vm = vx + VEC;      // m^f
  Real* vmp = vm + VEC;     // m^p
  Real* ve = vmp + VEC;     // innovation, then the backward noise
  Real* vz = ve + VEC;
  Real* vu = vz + VEC;      // U_t
  Real* vsg = vu + VEC;
  Real* vrow = vsg + VEC;
  const int lane = threadIdx.x;
  const int c = blockIdx.x / p.nb, k = blockIdx.x % p.nb;
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  const bool epi = a.flags & APPLY_EPI;
  const Real* ytc = a.yt + (long)c * p.nT * p.d;
  int bad = 0;
  Real r[DP], x[2 * DP];
  ld_vec<Real, DP>(p.F + row * DP, r);
  st_row<Real, DP>(SF, row, r, act);
  ld_vec<Real, DP>(p.Q + row * DP, r);
  chol_rot<Real, DP>(r, SLS, SCQ, nullptr, vx, nullptr, p.d, lane, &bad);
  __syncwarp();
  ld_row<Real, DP>(SCQ, row, r);
  zero_pad_row<Real, DP>(r, p.d, lane);
  __syncwarp();
  st_row<Real, DP>(SCQ, row, r, act);
  // P^p = U^p U^p^T into SP
  auto form_pp = [&]() {
    Real u[DP], pr[DP];
    ld_row<Real, DP>(SUp, row, u);
    row_matT<Real, DP>(u, SUp, pr);
    st_row<Real, DP>(SP, row, pr, act);
    __syncwarp();
  };
  // prediction from (m^f, U^f): m^p = F m^f + b, U^p = tria([F U^f, chol Q])
  auto predict = [&]() {
    Real fu[DP], cq[DP];
    mm_row<Real, DP>(SF + row * LD, SUf, fu);
    ld_row<Real, DP>(SCQ, row, cq);
    tria_row<Real, DP>(fu, cq, x);
    const Real mpi = act ? dot_row_vec<Real, DP>(SF + row * LD, vm) + p.b[lane] : (Real)0;
    tria_reg<Real, DP>(x, vrow, vsg, lane);
    Real up[DP];
#pragma unroll
    for (int cc = 0; cc < DP; ++cc) up[cc] = x[cc];
    st_row<Real, DP>(SUp, row, up, act);
    if (act) vmp[lane] = mpi;
    __syncwarp();
    form_pp();
  };
  // the incoming filtering law, and the prediction of step s
  if (k > 0) {
    const Real* g = a.prefix + ((long)c * p.nb + (k - 1)) * Z::ES;
    ld_vec<Real, DP>(g + DP * DP + row * DP, r);
    st_row<Real, DP>(SUf, row, r, act);
    if (act) vm[lane] = g[3 * DP * DP + lane];
    __syncwarp();
    predict();
  } else {
    ld_vec<Real, DP>(p.P0 + row * DP, r);
    chol_rot<Real, DP>(r, SLS, SUp, nullptr, vx, nullptr, p.d, lane, &bad);
    __syncwarp();
    ld_row<Real, DP>(SUp, row, r);
    zero_pad_row<Real, DP>(r, p.d, lane);
    __syncwarp();
    st_row<Real, DP>(SUp, row, r, act);
    if (act) vmp[lane] = p.m0[lane];
    __syncwarp();
    form_pp();
  }
  if (epi) {
#pragma unroll
    for (int cc = 0; cc < DP; ++cc) r[cc] = (cc == lane) ? (Real)1 : (Real)0;
    st_row<Real, DP>(SGP, row, r, act);
  }
  Real ubar = (Real)0;
  double lz = 0.0;
  const double half_dlog2pi = 0.91893853320467274178032973640562 * p.d;
  for (int t = s; t <= e; ++t) {
    const long ct = (long)c * p.nT + t;
    // conditioning on y_t: Ls, K, K', U^f
    sr_condition<Real, DP>(p, SP, SUp, SLS, SLR, vx, SK, SKp, SY, vrow, vsg, x, lane, &bad);
    const Real yi = lane < p.d ? ytc[(long)t * p.d + lane] : (Real)0;
    const Real ei = lane < p.d ? yi - vmp[lane] : (Real)0;
    if (act) ve[lane] = ei;
    __syncwarp();
    {
      Real ev[DP];
      ld_vec<Real, DP>(ve, ev);
      fsolve_vec<Real, DP>(SLS, vx, ev, vz, lane);
    }
    __syncwarp();
    double qz = (lane < p.d) ? (double)vz[lane] * (double)vz[lane] : 0.0;
    double lg = (lane < p.d) ? -log((double)vx[lane]) : 0.0;
    qz = warp_sum<double>(qz);
    lg = warp_sum<double>(lg);
    const double q = qz, ld = 2.0 * lg;
    if (lane == 0) {
      if (a.flags & APPLY_STORE_Q) { a.fq[ct] = q; a.fld[ct] = ld; }
      if (a.flags & APPLY_REV_DIFF) lz += -0.5 * ((a.fld[ct] - ld) + (a.fq[ct] - q));
      if (a.flags & APPLY_LOGZ) lz += -(half_dlog2pi + 0.5 * (ld + q));
    }
    const Real mfi = act ? vmp[lane] + dot_row_vec<Real, DP>(SK + row * LD, ve) : (Real)0;
    {
      Real uf[DP];
#pragma unroll
      for (int cc = 0; cc < DP; ++cc) uf[cc] = x[cc];
      __syncwarp();
      st_row<Real, DP>(SUf, row, uf, act);
    }
    if (act) vm[lane] = mfi;
    __syncwarp();
    if (a.mf && lane < p.d) a.mf[ct * p.d + lane] = mfi;
    if (a.Pf) {
      Real pf[DP], uf[DP];
      ld_row<Real, DP>(SUf, row, uf);
      row_matT<Real, DP>(uf, SUf, pf);
      if (lane < p.d) {
#pragma unroll
        for (int jj = 0; jj < DP; ++jj)
          if (jj < p.d) a.Pf[(ct * p.d + lane) * p.d + jj] = pf[jj];
      }
    }
    const bool last = t == p.nT - 1;
    if (t < e || (epi && !last)) predict();   // (m^p, U^p, P^p) of step t + 1
    if (!epi) continue;
    // backward element of step t
    const Real en = (lane < p.d && !(a.flags & APPLY_SMOOTH))
                        ? (a.eps ? a.eps[ct * p.d + lane]
                                 : philox_normal<Real>(p.seed, (uint32_t)c, iter_of(p, a.iter), PURPOSE_BACKWARD,
                                                       (uint32_t)t, lane))
                        : (Real)0;
    __syncwarp();
    if (act) ve[lane] = en;
    __syncwarp();
    if (last) {
      Real g0[DP];
      zero<Real, DP>(g0);
      st_row<Real, DP>(SG, row, g0, act);
      Real uf[DP];
      ld_row<Real, DP>(SUf, row, uf);
#pragma unroll
      for (int cc = 0; cc < DP; ++cc) x[cc] = uf[cc];
      __syncwarp();
    } else {
      // G = P^f F^T (P^p)^{-1}: rows of (P^p^{-1} F P^f)^T through chol(P^p)
      {
        Real pf[DP], fp[DP], uf[DP];
        ld_row<Real, DP>(SUf, row, uf);
        row_matT<Real, DP>(uf, SUf, pf);
        st_row<Real, DP>(SW, row, pf, act);
        __syncwarp();
        mm_row<Real, DP>(SF + row * LD, SW, fp);
        st_row<Real, DP>(SB, row, fp, act);
        Real pp[DP];
        ld_row<Real, DP>(SP, row, pp);
        chol_rot<Real, DP>(pp, SLS, nullptr, SLR, vx, nullptr, p.d, lane, &bad);
      }
      solve_cols<Real, DP>(SLS, SLR, vx, SB, SY, SG, lane);
      // chol(Sigma) = tria([(I - G F) U^f, G chol Q])
      {
        Real gf[DP];
        mm_row<Real, DP>(SG + row * LD, SF, gf);
        __syncwarp();
        st_row<Real, DP>(SW, row, gf, act);
        __syncwarp();
      }
      {
        Real a1[DP], a2[DP];
        ld_row<Real, DP>(SUf, row, a1);
        mm_row<Real, DP, true, true>(SW + row * LD, SUf, a1);
        mm_row<Real, DP>(SG + row * LD, SCQ, a2);
        tria_row<Real, DP>(a1, a2, x);
      }
      tria_reg<Real, DP>(x, vrow, vsg, lane);
    }
    // U_t = m^f - G m^p_{t+1} + chol(Sigma) eps
    Real noise = (Real)0;
#pragma unroll
    for (int cc = 0; cc < DP; ++cc) noise = fma(x[cc], ve[cc], noise);
    const Real ui = mfi - (last ? (Real)0 : dot_row_vec<Real, DP>(SG + row * LD, vmp)) + noise;
    if (act) {
      Real gr[DP];
      ld_row<Real, DP>(SG, row, gr);
      st_vec<Real, DP>(a.G + ct * DD + row * DP, gr);
      a.U[ct * DP + lane] = ui;
      vu[lane] = ui;
    }
    __syncwarp();
    // block aggregates: ubar += (G_s ... G_{t-1}) U_t; G_s ... G_t
    ubar += dot_row_vec<Real, DP>(SGP + row * LD, vu);
    {
      Real gp[DP];
      if (last) zero<Real, DP>(gp);
      else mm_row<Real, DP>(SGP + row * LD, SG, gp);
      __syncwarp();
      st_row<Real, DP>(SGP, row, gp, act);
      __syncwarp();
    }
  }
  if (epi && act) {
    Real gp[DP];
    ld_row<Real, DP>(SGP, row, gp);
    st_vec<Real, DP>(a.gum + ((long)c * p.nb + k) * DD + row * DP, gp);
    a.guv[((long)c * p.nb + k) * DP + lane] = ubar;
  }
  if ((a.flags & (APPLY_LOGZ | APPLY_REV_DIFF)) && lane == 0) a.lz_part[(long)c * p.nb + k] = lz;
  if (bad && lane == 0) atomicOr(&p.status_iter[c], ST_NOT_PD);
}

// ---------------------------------------------------------------------------
// In-block square-root covariance filter of covariance block k (one warp) from
// the prefix factor U^f_{s-1}, writing the per-step tables of aux_cov.cuh:
//   TK[t] = K'_t = r S_t^{-1}, ldt[t] = log det S_t, TPF[t] = U^f_t U^f_t^T,
//   TG[t] = G_t, TLS[t] = chol(Sigma_t) = tria([(I - G_t F) U^f_t, G_t chol Q]),
//   TGP[t] = G_s ... G_{t-1}; and the block products G_s ... G_e and
//   M_e ... M_s (M_t = K'_t F) into cblk, as k_cov_apply does.
// Per step: the prediction U^p_t = tria([F U^f_{t-1}, chol Q]); the epilogue of
// step t - 1 (it needs P^p_t); the conditioning on y_t (U^f_t by tria in
// Joseph form); the running products.
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __launch_bounds__(32, 1) k_srcov_apply(KP<Real> p, CovArgs<Real> a) {
  refresh_delta(p);
  using Z = SrSizes<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC, LD = Lay<Real, DP>::LD;
  constexpr long DD = (long)DP * DP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  Real* SF = sm;
  Real* SCQ = SF + MAT;
  Real* SUf = SCQ + MAT;
  Real* SUp = SUf + MAT;
  Real* SK = SUp + MAT;
  Real* SKp = SK + MAT;
  Real* SLS = SKp + MAT;
  Real* SLR = SLS + MAT;
  Real* SP = SLR + MAT;
  Real* SY = SP + MAT;
  Real* SW = SY + MAT;
  Real* SB = SW + MAT;
  Real* SG = SB + MAT;
  Real* SGh = SG + MAT;
  Real* SAH = SGh + MAT;
  Real* vx = SAH + MAT;
  Real* vsg = vx + VEC;
  Real* vrow = vsg + VEC;
  const int lane = threadIdx.x, k = blockIdx.x;
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  int bad = 0;
  Real r[DP], x[2 * DP];
  ld_vec<Real, DP>(p.F + row * DP, r);
  st_row<Real, DP>(SF, row, r, act);
  ld_vec<Real, DP>(p.Q + row * DP, r);
  chol_rot<Real, DP>(r, SLS, SCQ, nullptr, vx, nullptr, p.d, lane, &bad);
  __syncwarp();
  ld_row<Real, DP>(SCQ, row, r);
  zero_pad_row<Real, DP>(r, p.d, lane);
  __syncwarp();
  st_row<Real, DP>(SCQ, row, r, act);
#pragma unroll
  for (int j = 0; j < DP; ++j) r[j] = (j == lane) ? (Real)1 : (Real)0;
  st_row<Real, DP>(SGh, row, r, act);
  st_row<Real, DP>(SAH, row, r, act);
  __syncwarp();
  auto store_row = [&](int tb, int t, const Real* S) {
    Real q[DP];
    ld_row<Real, DP>(S, row, q);
    if (act) st_vec<Real, DP>(a.tab + ((long)tb * p.nT + t) * DD + row * DP, q);
  };
  auto form_pp = [&]() {   // SP <- U^p U^p^T
    Real u[DP], pr[DP];
    ld_row<Real, DP>(SUp, row, u);
    row_matT<Real, DP>(u, SUp, pr);
    __syncwarp();
    st_row<Real, DP>(SP, row, pr, act);
    __syncwarp();
  };
  auto predict = [&]() {   // U^p = tria([F U^f, chol Q]), P^p
    Real fu[DP], cq[DP];
    mm_row<Real, DP>(SF + row * LD, SUf, fu);
    ld_row<Real, DP>(SCQ, row, cq);
    tria_row<Real, DP>(fu, cq, x);
    tria_reg<Real, DP>(x, vrow, vsg, lane);
    Real up[DP];
#pragma unroll
    for (int cc = 0; cc < DP; ++cc) up[cc] = x[cc];
    st_row<Real, DP>(SUp, row, up, act);
    __syncwarp();
    form_pp();
  };
  // with U^f_t in SUf and P^p_{t+1} in SP: G_t -> TG, chol(Sigma_t) -> TLS, SGh <- SGh G_t
  auto epilogue = [&](int t) {
    {
      Real pp[DP];
      ld_row<Real, DP>(SP, row, pp);
      chol_rot<Real, DP>(pp, SLS, nullptr, SLR, vx, nullptr, p.d, lane, &bad);
    }
    {
      Real pf[DP], fp[DP], uf[DP];
      ld_row<Real, DP>(SUf, row, uf);
      row_matT<Real, DP>(uf, SUf, pf);
      __syncwarp();
      st_row<Real, DP>(SW, row, pf, act);
      __syncwarp();
      mm_row<Real, DP>(SF + row * LD, SW, fp);
      st_row<Real, DP>(SB, row, fp, act);
      __syncwarp();
    }
    solve_cols<Real, DP>(SLS, SLR, vx, SB, SY, SG, lane);   // G = P^f F^T (P^p)^{-1}
    {
      Real gf[DP];
      mm_row<Real, DP>(SG + row * LD, SF, gf);
      __syncwarp();
      st_row<Real, DP>(SW, row, gf, act);
      __syncwarp();
    }
    {
      Real a1[DP], a2[DP];
      ld_row<Real, DP>(SUf, row, a1);
      mm_row<Real, DP, true, true>(SW + row * LD, SUf, a1);
      mm_row<Real, DP>(SG + row * LD, SCQ, a2);
      tria_row<Real, DP>(a1, a2, x);
    }
    tria_reg<Real, DP>(x, vrow, vsg, lane);
    {
      Real ls[DP];
#pragma unroll
      for (int cc = 0; cc < DP; ++cc) ls[cc] = x[cc];
      if (act) st_vec<Real, DP>(a.tab + ((long)TLS * p.nT + t) * DD + row * DP, ls);
    }
    store_row(TG, t, SG);
    Real gn[DP];
    mm_row<Real, DP>(SGh + row * LD, SG, gn);
    __syncwarp();
    st_row<Real, DP>(SGh, row, gn, act);
    __syncwarp();
  };
  // ---- block start: U^p_s
  if (k > 0) {
    ld_vec<Real, DP>(a.prefix + (long)(k - 1) * 3 * DD + DD + row * DP, r);
    st_row<Real, DP>(SUf, row, r, act);
    __syncwarp();
    predict();
  } else {
    ld_vec<Real, DP>(p.P0 + row * DP, r);
    chol_rot<Real, DP>(r, SLS, SUp, nullptr, vx, nullptr, p.d, lane, &bad);
    __syncwarp();
    ld_row<Real, DP>(SUp, row, r);
    zero_pad_row<Real, DP>(r, p.d, lane);
    __syncwarp();
    st_row<Real, DP>(SUp, row, r, act);
    __syncwarp();
    form_pp();
  }
  for (int t = s; t <= e; ++t) {
    if (t > s) {
      predict();          // U^p_t, P^p_t from U^f_{t-1}
      epilogue(t - 1);    // G_{t-1}, chol(Sigma_{t-1})
    }
    store_row(TGP, t, SGh);
    // conditioning on y_t
    sr_condition<Real, DP>(p, SP, SUp, SLS, SLR, vx, SK, SKp, SY, vrow, vsg, x, lane, &bad);
    double lg = (lane < p.d) ? -log((double)vx[lane]) : 0.0;
    lg = warp_sum<double>(lg);
    if (lane == 0) a.ldt[t] = 2.0 * lg;
    store_row(TK, t, SKp);
    {
      Real uf[DP], pf[DP];
#pragma unroll
      for (int cc = 0; cc < DP; ++cc) uf[cc] = x[cc];
      __syncwarp();
      st_row<Real, DP>(SUf, row, uf, act);
      __syncwarp();
      row_matT<Real, DP>(uf, SUf, pf);
      if (act) st_vec<Real, DP>(a.tab + ((long)TPF * p.nT + t) * DD + row * DP, pf);
    }
    // M_t = K'_t F, SAH <- M_t SAH
    {
      Real mr[DP], ah[DP];
      mm_row<Real, DP>(SKp + row * LD, SF, mr);
      __syncwarp();
      st_row<Real, DP>(SW, row, mr, act);
      __syncwarp();
      mm_row<Real, DP>(SW + row * LD, SAH, ah);
      __syncwarp();
      st_row<Real, DP>(SAH, row, ah, act);
      __syncwarp();
    }
  }
  // ---- block end
  if (e < p.nT - 1) {
    predict();
    epilogue(e);
  } else {
    Real z0[DP];
    zero<Real, DP>(z0);
    if (act) st_vec<Real, DP>(a.tab + ((long)TG * p.nT + e) * DD + row * DP, z0);
    store_row(TLS, e, SUf);
    __syncwarp();
    st_row<Real, DP>(SGh, row, z0, act);
    __syncwarp();
  }
  {
    Real q[DP];
    ld_row<Real, DP>(SGh, row, q);
    if (act) st_vec<Real, DP>(a.cblk + (long)k * DD + row * DP, q);
    ld_row<Real, DP>(SAH, row, q);
    if (act) st_vec<Real, DP>(a.cblk + ((long)p.nb + k) * DD + row * DP, q);
  }
  if (bad && lane == 0) atomicOr(a.status, ST_NOT_PD);
}

}  // namespace auxk
