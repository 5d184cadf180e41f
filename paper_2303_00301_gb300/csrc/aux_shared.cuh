// aux_shared.cuh — shared-covariance execution of the parallel filter.
//
// With the first-order proposal and Gaussian dynamics the covariance part of
// every filtering element depends only on (F, Q, P0, delta), never on the
// chain's data, so all chains of one model run the same covariance recursion.
// These kernels give one CTA the same scan block of CW chains: warp 0 (the
// leader) computes the matrix part once into CTA-shared slots and every warp
// computes its own chain's vector part (means, pseudo-observation residuals,
// likelihood terms, backward-sampler vectors) from them. Same phases, same
// arithmetic as the per-chain kernels; the matrix part of the scan aggregates
// and of the backward elements is stored once per block instead of per chain.
#pragma once
#include "aux_kernels.cuh"

namespace auxk {

template <typename Real, int DP> struct ShSizes {
  static constexpr int MAT = Lay<Real, DP>::MAT, VEC = Lay<Real, DP>::VEC;
  static constexpr int CW = 8;   // chains (warps) per CTA
  static constexpr size_t MODEL = (3 * MAT + 2 * VEC) * sizeof(Real);
  static constexpr size_t RED_SMEM = MODEL + (6 * MAT + 2 * VEC + CW * 4 * VEC) * sizeof(Real);
  static constexpr size_t SCAN_SMEM = (9 * MAT + VEC + CW * 8 * VEC) * sizeof(Real);
  static constexpr size_t APP_SMEM = MODEL + (7 * MAT + 3 * VEC + CW * 6 * VEC) * sizeof(Real);
};

// ---------------------------------------------------------------------------
// Phase 1 (shared covariance): the conditional Kalman recursion of
// k_filter_reduce, matrix part on the leader, vector part (b, eta) per chain.
// aggm: [nb][3 DP^2] (A, C, J), aggv: [C][nb][2 DP] (b, eta).
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __launch_bounds__(32 * ShSizes<Real, DP>::CW, 1)
    k_filter_reduce_sh(KP<Real> p, const Real* __restrict__ yt, Real* __restrict__ aggm,
                       Real* __restrict__ aggv) {
  using Z = ShSizes<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC, LD = Lay<Real, DP>::LD, CW = Z::CW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  Real* sF = sm;
  Real* sFT = sF + MAT;
  Real* sQ = sFT + MAT;
  Real* sb = sQ + MAT;
  load_model_slots<Real, DP>(p, sF, sFT, sQ, sb);
  __syncthreads();   // the model slots are written by all warps
  const Real* sphi = sb + VEC;
  Real* SA = sb + 2 * VEC;
  Real* SC = SA + MAT;
  Real* SX = SC + MAT;
  Real* SY = SX + MAT;
  Real* SW = SY + MAT;
  Real* SL = SW + MAT;
  Real* vdiag = SL + MAT;
  Real* vdummy = vdiag + VEC;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Real* vb = vdummy + VEC + warp * 4 * VEC;
  Real* veta = vb + VEC;
  Real* vr = veta + VEC;
  Real* vz = vr + VEC;
  const int k = blockIdx.x % p.nb, grp = blockIdx.x / p.nb;
  const int c = grp * CW + warp;
  const bool valid = c < p.C, leader = warp == 0;
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
  if (leader) {
    Real r[DP];
#pragma unroll
    for (int j = 0; j < DP; ++j) r[j] = (k > 0 && j == lane) ? (Real)1 : (Real)0;
    st_row<Real, DP>(SA, row, r, act);
    zero<Real, DP>(r);
    st_row<Real, DP>(SC, row, r, act);
  }
  if (act) { vb[lane] = (Real)0; veta[lane] = (Real)0; }
  __syncthreads();
  const Real* ytc = yt + (long)(valid ? c : 0) * p.nT * p.d;
  for (int t = s; t <= e; ++t) {
    if (leader) {
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
      // matrix updates (C, A in slots; J in registers) run after the barrier below
      // is passed, concurrently with the other warps' vector work: stash P^p in SC
      st_row<Real, DP>(SC, row, pprow, act);
    }
    Real mpi;
    if (t == 0) mpi = p.m0[row];
    else if (p.fdiag) mpi = sphi[row] * vb[row] + sb[row];
    else mpi = dot_row_vec<Real, DP>(sF + row * LD, vb) + sb[row];
    __syncthreads();
    if (valid) {
      const Real rres = (lane < p.d) ? ytc[(long)t * p.d + lane] - mpi : (Real)0;
      __syncwarp();
      if (act) vr[lane] = rres;
      __syncwarp();
      Real rr[DP];
      ld_vec<Real, DP>(vr, rr);
      fsolve_vec<Real, DP>(SL, vdiag, rr, vz, lane);
      __syncwarp();
      const Real bnew = mpi + dot_col_vec<Real, DP>(SY, row, vz);
      const Real etanew = veta[row] + dot_col_vec<Real, DP>(SW, row, vz);
      __syncwarp();
      if (act) { vb[lane] = bnew; veta[lane] = etanew; }
    }
    if (leader) {
      if constexpr (DP >= 16) {
        __syncwarp();
        mm_tile_to_slot<Real, DP, true, true>(SY, SY, SC, SC, lane);   // C = P^p - Y^T Y
        mm_tile_to_slot<Real, DP, true, true>(SY, SW, SX, SA, lane);   // A = F A - Y^T W
        mm_tile_regs<Real, DP, true, false>(SW, SW, jtile, lane);       // J += W^T W
      } else {
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
    }
    __syncthreads();
  }
  if (leader) {
    if constexpr (DP >= 16) {
      tile_store<Real, DP>(SY, jtile, lane);
      __syncwarp();
      ld_row<Real, DP>(SY, row, jreg);
    }
    if (grp == 0 && act) {
      Real* g = aggm + (long)k * 3 * DP * DP;
      Real r[DP];
      ld_row<Real, DP>(SA, row, r);
      st_vec<Real, DP>(g + row * DP, r);
      ld_row<Real, DP>(SC, row, r);
      st_vec<Real, DP>(g + DP * DP + row * DP, r);
      st_vec<Real, DP>(g + 2 * DP * DP + row * DP, jreg);
    }
    if (bad && lane == 0)
      for (int cc = grp * CW; cc < min(p.C, grp * CW + CW); ++cc) atomicOr(&p.status_iter[cc], ST_NOT_PD);
  }
  if (valid && act) {
    Real* v = aggv + ((long)c * p.nb + k) * 2 * DP;
    v[lane] = vb[lane];
    v[DP + lane] = veta[lane];
  }
}

// ---------------------------------------------------------------------------
// Phase 2 (shared covariance): one Hillis-Steele round; the leader runs the
// operator's matrix parts, every warp its chain's vector part.
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __launch_bounds__(32 * ShSizes<Real, DP>::CW, 1)
    k_filter_scan_level_sh(KP<Real> p, const Real* __restrict__ in_m, const Real* __restrict__ in_v,
                           Real* __restrict__ out_m, Real* __restrict__ out_v, int off) {
  using Z = ShSizes<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC, CW = Z::CW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x % p.nb, grp = blockIdx.x / p.nb;
  const int c = grp * CW + warp;
  const bool valid = c < p.C, leader = warp == 0;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  if (k < off) {
    if (leader && grp == 0 && act) {
      for (int q = row; q < 3 * DP; q += DP) {
        Real r[DP];
        ld_vec<Real, DP>(in_m + (long)k * 3 * DP * DP + q * DP, r);
        st_vec<Real, DP>(out_m + (long)k * 3 * DP * DP + q * DP, r);
      }
    }
    if (valid && act) {
      const long o = ((long)c * p.nb + k) * 2 * DP;
      out_v[o + lane] = in_v[o + lane];
      out_v[o + DP + lane] = in_v[o + DP + lane];
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
  Real* vb = vdiag + VEC + warp * 8 * VEC;
  Real* veta = vb + VEC;
  Real* vbe = veta + VEC;
  Real* vetae = vbe + VEC;
  Real* vt = vetae + VEC;
  int bad = 0;
  Real jreg[DP];
  if (leader) {
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
  if (valid && act) {
    const long oi = ((long)c * p.nb + (k - off)) * 2 * DP, oj = ((long)c * p.nb + k) * 2 * DP;
    vb[lane] = in_v[oi + lane];
    veta[lane] = in_v[oi + DP + lane];
    vbe[lane] = in_v[oj + lane];
    vetae[lane] = in_v[oj + DP + lane];
  }
  __syncthreads();
  if (leader) combine_matrix_1<Real, DP>(SC, SAe, SJe, SU, S2, S3, S4, vdiag, p.d, lane, &bad);
  __syncthreads();
  if (valid) combine_vectors<Real, DP>(SA, SAe, SJe, S2, S3, vb, veta, vbe, vetae, vt, lane);
  __syncthreads();
  if (leader) {
    combine_matrix_2<Real, DP>(SA, SC, jreg, SAe, SCe, SJe, SU, S2, S3, S4, lane);
    if (grp == 0 && act) {
      Real* g = out_m + (long)k * 3 * DP * DP;
      Real r[DP];
      ld_row<Real, DP>(SA, row, r);
      st_vec<Real, DP>(g + row * DP, r);
      ld_row<Real, DP>(SC, row, r);
      st_vec<Real, DP>(g + DP * DP + row * DP, r);
      st_vec<Real, DP>(g + 2 * DP * DP + row * DP, jreg);
    }
    if (bad && lane == 0)
      for (int cc = grp * CW; cc < min(p.C, grp * CW + CW); ++cc) atomicOr(&p.status_iter[cc], ST_NOT_PD);
  }
  if (valid && act) {
    const long o = ((long)c * p.nb + k) * 2 * DP;
    out_v[o + lane] = vb[lane];
    out_v[o + DP + lane] = veta[lane];
  }
}

// ---------------------------------------------------------------------------
// Phase 3 (shared covariance): the in-block Kalman filter; the leader runs the
// covariance recursion and the matrix part of the backward elements, every
// warp its chain's means, likelihood terms, U_t and backward aggregate.
// G_t and the block aggregates G_s ... G_e are stored once (chain stride 0).
// ---------------------------------------------------------------------------
template <typename Real> struct ApplyShArgs {
  const Real* yt;
  const Real* prem;     // final scan buffer, matrix part [nb][3 DP^2] (null if nb == 1)
  const Real* prev;     // final scan buffer, vector part [C][nb][2 DP]
  int flags;
  Real* G;              // [T][DP*DP]
  Real* U;              // [C][T][DP]
  Real* gum;            // [nb][DP*DP]
  Real* guv;            // [C][nb][DP]
  double* fq;
  double* fld;
  double* lz_part;
  Real* mf;
  Real* Pf;
  const Real* eps;
  uint64_t iter;
};

template <typename Real, int DP>
__global__ void __launch_bounds__(32 * ShSizes<Real, DP>::CW, 1)
    k_filter_apply_sh(KP<Real> p, ApplyShArgs<Real> a) {
  using Z = ShSizes<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC, LD = Lay<Real, DP>::LD, CW = Z::CW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  Real* sF = sm;
  Real* sFT = sF + MAT;
  Real* sQ = sFT + MAT;
  Real* sb = sQ + MAT;
  load_model_slots<Real, DP>(p, sF, sFT, sQ, sb);
  __syncthreads();   // the model slots are written by all warps
  const Real* sphi = sb + VEC;
  Real* SP = sb + 2 * VEC;
  Real* SX = SP + MAT;
  Real* SL = SX + MAT;
  Real* SLR = SL + MAT;
  Real* SY = SLR + MAT;
  Real* SG = SY + MAT;
  Real* SGh = SG + MAT;
  Real* vdA = SGh + MAT;
  Real* vdB = vdA + VEC;
  Real* vsc = vdB + VEC;       // [0]: log det of P^p + R
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Real* vm = vsc + VEC + warp * 6 * VEC;
  Real* vmp = vm + VEC;
  Real* vr = vmp + VEC;
  Real* vz = vr + VEC;
  Real* veps = vz + VEC;
  Real* vU = veps + VEC;
  const int k = blockIdx.x % p.nb, grp = blockIdx.x / p.nb;
  const int c = grp * CW + warp;
  const bool valid = c < p.C, leader = warp == 0;
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  const Real* ytc = a.yt + (long)(valid ? c : 0) * p.nT * p.d;
  const bool epi = a.flags & APPLY_EPI;
  int bad = 0;
  double lz_acc = 0.0;
  const double half_dlog2pi = 0.5 * p.d * 1.8378770664093454835606594728112;
  Real pprow[DP];
  Real uhat = 0;
  if (leader) {
    Real gi[DP];
#pragma unroll
    for (int j = 0; j < DP; ++j) gi[j] = (j == lane) ? (Real)1 : (Real)0;
    st_row<Real, DP>(SGh, row, gi, act);
  }

  auto all_mp = [&]() {        // m^p = F m^f + b for the warp's chain
    Real mpi;
    if (p.fdiag) mpi = sphi[row] * vm[row] + sb[row];
    else mpi = dot_row_vec<Real, DP>(sF + row * LD, vm) + sb[row];
    __syncwarp();
    if (act) vmp[lane] = mpi;
    __syncwarp();
  };
  auto leader_predict = [&]() {   // P^p (pprow) and X = F P^f (SX) from P^f (SP)
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
      __syncwarp();
      return;
    }
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
    symmetrise_store<Real, DP>(SY, pprow, lane);
  };
  auto leader_factor_S = [&]() {
    Real s_[DP];
#pragma unroll
    for (int j = 0; j < DP; ++j) s_[j] = pprow[j] + ((j == lane && j < p.d) ? p.r : (Real)0);
    chol_rot<Real, DP>(s_, SG, nullptr, nullptr, vdB, nullptr, p.d, lane, &bad);
  };
  auto leader_factor_2 = [&]() {
    Real a_[DP], s_[DP];
#pragma unroll
    for (int j = 0; j < DP; ++j) {
      a_[j] = pprow[j];
      s_[j] = pprow[j] + ((j == lane && j < p.d) ? p.r : (Real)0);
    }
    chol_rot2<Real, DP>(a_, SL, SLR, vdA, s_, SG, vdB, p.d, lane, &bad);
  };
  // after the factor of P^p_{t+1} (SL / SLR / vdA): G_t rows -> SX, rows of chol Sigma_t -> SLR
  auto leader_epilogue = [&](int t) {
    {
      Real rr[DP];
      ld_col<Real, DP>(SX, row, rr);
      fsolve_rot<Real, DP, true>(SL, vdA, rr, SY, lane);
    }
    __syncwarp();
    Real sig[DP];
    if constexpr (DP >= 16) {
      mm_tile_to_slot<Real, DP, true, true>(SY, SY, SP, SL, lane);
      __syncwarp();
      ld_row<Real, DP>(SL, row, sig);
    } else {
      ld_row<Real, DP>(SP, row, sig);
      mm_col<Real, DP, true, true>(SY, row, SY, sig);
    }
    {
      Real rr[DP];
      ld_col<Real, DP>(SY, row, rr);
      bsolve_rot<Real, DP>(SLR, vdA, rr, SX, lane);
    }
    chol_rot<Real, DP>(sig, SL, SLR, nullptr, vdA, nullptr, p.d, lane, &bad);
    if (grp == 0 && act) {
      Real gr[DP];
      ld_row<Real, DP>(SX, row, gr);
      st_vec<Real, DP>(a.G + (long)t * DP * DP + row * DP, gr);
    }
  };
  auto all_U = [&](int t) {      // U_t = m^f_t - G_t m^p_{t+1} + chol(Sigma_t) eps_t
    if (!valid) return;
    Real ei = 0;
    if (lane < p.d)
      ei = a.eps ? a.eps[((long)c * p.nT + t) * p.d + lane]
                 : philox_normal<Real>(p.seed, (uint32_t)c, a.iter, PURPOSE_BACKWARD, (uint32_t)t, lane);
    __syncwarp();
    if (act) veps[lane] = ei;
    __syncwarp();
    const Real ui = vm[row] - dot_row_vec<Real, DP>(SX + row * LD, vmp) +
                    dot_row_vec<Real, DP>(SLR + row * LD, veps);
    if (act) {
      a.U[((long)c * p.nT + t) * DP + lane] = ui;
      vU[lane] = ui;
    }
    __syncwarp();
    uhat += dot_row_vec<Real, DP>(SGh + row * LD, vU);
  };
  auto leader_ghat = [&]() {     // G^ <- G^ G_t
    Real gn[DP];
    mm_row<Real, DP>(SGh + row * LD, SX, gn);
    __syncwarp();
    st_row<Real, DP>(SGh, row, gn, act);
    __syncwarp();
  };
  auto leader_update = [&]() {   // Y_s = L_S^{-1} P^p (columns of SY), P^f -> SP, log det
    {
      Real rr[DP];
#pragma unroll
      for (int j = 0; j < DP; ++j) rr[j] = pprow[j];
      fsolve_rot<Real, DP, true>(SG, vdB, rr, SY, lane);
    }
    __syncwarp();
    if constexpr (DP >= 16) {
      st_row<Real, DP>(SP, row, pprow, act);
      __syncwarp();
      mm_tile_to_slot<Real, DP, true, true>(SY, SY, SP, SP, lane);
    } else {
      Real pf[DP];
#pragma unroll
      for (int j = 0; j < DP; ++j) pf[j] = pprow[j];
      mm_col<Real, DP, true, true>(SY, row, SY, pf);
      __syncwarp();
      st_row<Real, DP>(SP, row, pf, act);
    }
    Real lg = (lane < p.d) ? -log(vdB[lane]) : (Real)0;
    lg = warp_sum<Real>(lg);
    if (lane == 0) vsc[0] = (Real)2 * lg;
    __syncwarp();
  };
  auto all_update = [&](int t) {  // m^f, likelihood terms for the warp's chain
    if (!valid) return;
    const Real rres = (lane < p.d) ? ytc[(long)t * p.d + lane] - vmp[lane] : (Real)0;
    __syncwarp();
    if (act) vr[lane] = rres;
    __syncwarp();
    Real rr[DP];
    ld_vec<Real, DP>(vr, rr);
    fsolve_vec<Real, DP>(SG, vdB, rr, vz, lane);
    __syncwarp();
    const Real mfi = vmp[row] + dot_col_vec<Real, DP>(SY, row, vz);
    Real zz[DP];
    ld_vec<Real, DP>(vz, zz);
    const Real qz = dot_rr<Real, DP>(zz, zz);
    __syncwarp();
    if (act) vm[lane] = mfi;
    __syncwarp();
    const double q = (double)qz, ld = (double)vsc[0];
    const long ct = (long)c * p.nT + t;
    if (lane == 0) {
      if (a.flags & APPLY_STORE_Q) { a.fq[ct] = q; a.fld[ct] = ld; }
      if (a.flags & APPLY_REV_DIFF) lz_acc += -0.5 * ((a.fld[ct] - ld) + (a.fq[ct] - q));
      if (a.flags & APPLY_LOGZ) lz_acc += -(half_dlog2pi + 0.5 * (ld + q));
    }
    if (a.mf && lane < p.d) a.mf[ct * p.d + lane] = mfi;
    if (a.Pf && lane < p.d) {
      for (int j = 0; j < p.d; ++j) a.Pf[(ct * p.d + lane) * p.d + j] = SP[lane * LD + j];
    }
  };

  // ---- block start
  if (k == 0) {
    if (leader) ld_vec<Real, DP>(p.P0 + row * DP, pprow);
    if (act) vmp[lane] = p.m0[lane];
    __syncwarp();
  } else {
    if (leader) {
      Real r[DP];
      ld_vec<Real, DP>(a.prem + (long)(k - 1) * 3 * DP * DP + DP * DP + row * DP, r);
      st_row<Real, DP>(SP, row, r, act);
      __syncwarp();
      leader_predict();
    }
    if (valid && act) vm[lane] = a.prev[((long)c * p.nb + (k - 1)) * 2 * DP + lane];
    __syncwarp();
    all_mp();
  }
  if (leader) { leader_factor_S(); leader_update(); }
  __syncthreads();
  all_update(s);
  __syncthreads();
  for (int t = s + 1; t <= e; ++t) {
    all_mp();
    if (leader) {
      leader_predict();
      if (epi) { leader_factor_2(); leader_epilogue(t - 1); }
      else leader_factor_S();
    }
    __syncthreads();
    if (epi) {
      all_U(t - 1);
      __syncthreads();
      if (leader) leader_ghat();
    }
    if (leader) leader_update();
    __syncthreads();
    all_update(t);
    __syncthreads();
  }
  if (epi) {
    if (e < p.nT - 1) {
      all_mp();
      if (leader) {
        leader_predict();
        Real a_[DP];
#pragma unroll
        for (int j = 0; j < DP; ++j) a_[j] = pprow[j];
        chol_rot<Real, DP>(a_, SL, nullptr, SLR, vdA, nullptr, p.d, lane, &bad);
        leader_epilogue(e);
      }
    } else if (leader) {
      Real pf[DP], z0[DP];
      ld_row<Real, DP>(SP, row, pf);
      chol_rot<Real, DP>(pf, SL, SLR, nullptr, vdA, nullptr, p.d, lane, &bad);
      zero<Real, DP>(z0);
      st_row<Real, DP>(SX, row, z0, act);
      if (grp == 0 && act) st_vec<Real, DP>(a.G + (long)e * DP * DP + row * DP, z0);
    }
    __syncthreads();
    all_U(e);
    __syncthreads();
    if (leader) {
      leader_ghat();
      if (grp == 0 && act) {
        Real gr[DP];
        ld_row<Real, DP>(SGh, row, gr);
        st_vec<Real, DP>(a.gum + (long)k * DP * DP + row * DP, gr);
      }
    }
    if (valid && act) a.guv[((long)c * p.nb + k) * DP + lane] = uhat;
  }
  if ((a.flags & (APPLY_REV_DIFF | APPLY_LOGZ)) && valid && lane == 0)
    a.lz_part[(long)c * p.nb + k] = lz_acc;
  if (leader && bad && lane == 0)
    for (int cc = grp * CW; cc < min(p.C, grp * CW + CW); ++cc) atomicOr(&p.status_iter[cc], ST_NOT_PD);
}

}  // namespace auxk
