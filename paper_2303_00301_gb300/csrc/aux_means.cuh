// aux_means.cuh — the per-chain half of the parallel filter and of the
// backward sampler when the covariance tables of aux_cov.cuh are available:
// every step is a few DP x DP matrix-vector products with matrices shared by
// all chains.
//
// Filtering means (Kalman filter algorithm, Appendix A.1, with H = I, R = r I):
//   m^p_0 = m0,  m^p_t = F m^f_{t-1} + b,  e_t = ytilde_t - m^p_t,
//   m^f_t = ytilde_t - K'_t e_t  (K'_t = r S_t^{-1} = I - K_t),
//   log-likelihood term  -(d/2) log 2 pi - (1/2) (log det S_t + e_t^T K'_t e_t / r).
// The recursion is affine in m^f_{s-1} with linear part AH_k over a block, so
// the blocked scan keeps the structure of the full filter (Appendix A.2.1):
//   k_mf_reduce    each block from m^f_{s-1} = 0 (block 0 from m0): block-end z_k;
//   k_mean_cross   per chain, m^f_{e_k} = AH_k m^f_{e_{k-1}} + z_k over the blocks;
//   k_mf_apply     each block again from its true start, with the likelihood
//                  terms and the backward elements of Eq. (A.14),
//                  U_t = m^f_t - G_t m^p_{t+1} + chol(Sigma_t) eps_t, and the block
//                  aggregate sum_t (G_s ... G_{t-1}) U_t of the (G, U) scan;
//   k_mean_cross   (backward) per chain, x*_{s_k} = GH_k x*_{e_k + 1} + Ubar_k;
//   k_mb_apply     x*_t = G_t x*_{t+1} + U_t inside each block (Proposition A.1),
//                  with the MH terms at x* and ytilde*.
// One CTA runs MEAN_CHAINS chains of the same block (lane = row, MEAN_CPW
// chains per warp), so the tables of step t are staged once per CTA in shared
// memory, with asynchronous copies one step ahead, and each table row is read
// from shared memory once per warp for all of its chains.
#pragma once
#include "aux_cov.cuh"

namespace auxk {

template <typename Real> struct MeanArgs {
  const Real* tab;            // [NTAB][T][DP][DP]
  const Real* btab;           // [NBTAB][nb][DP][DP]
  const double* ld;           // [nb]
  const int32_t* cov_status;  // [1]
  // k_mf_reduce
  const Real* x;              // state [C][T][d]: linearise first (A1, A2); null: read yt
  Real* u;                    // [C][T][d] (written when x != null)
  Real* v;                    // [C][T][d] (written when x != null)
  Real* yt;                   // [C][T][d] pseudo-observations
  Real* z;                    // [C][nb][DP] block-end means from a zero start
  uint64_t iter;
  // k_mf_apply
  int flags;                  // APPLY_EPI | APPLY_STORE_Q | APPLY_REV_DIFF | APPLY_LOGZ
  const Real* mstart;         // [C][nb][DP] m^f_{s_k - 1} (k >= 1)
  Real* U;                    // [C][T][DP]
  Real* guv;                  // [C][nb][DP]
  double* fqb;                // [C][nb] sum of |w_t|^2 over the block
  double* lz_part;            // [C][nb]
  Real* mf;                   // optional [C][T][d]
  Real* Pf;                   // optional [C][T][d][d]
  const Real* eps;            // optional [C][T][d] backward noise (else Philox)
  int32_t* status;            // optional sticky per-chain status
};

constexpr int MEAN_CHAINS = 8;   // chains per CTA (all of the same scan block)
constexpr int MEAN_CPW = 1;      // chains per warp in the reduce / apply kernels

// Staging buffers: the tables of step t + PREF are copied while step t
// computes (PREF steps of latency cover an L2 or, right after an L2 flush, an
// HBM read); step t reads buffer t % NBUF and the buffer refilled at step t
// was last read at step t - 2, which every warp has finished once it passed
// the barrier of step t - 1, so one barrier per step suffices.
constexpr int PREF = 2;
constexpr int NBUF = PREF + 2;

template <typename Real, int DP> struct MeanSizes {
  static constexpr int MAT = Lay<Real, DP>::MAT, VEC = Lay<Real, DP>::VEC;
  // NBUF staging buffers of NT tables, R_y^{-1}, three vector slots per warp
  static constexpr size_t smem(int nt) {
    return (size_t)(NBUF * nt * MAT + MAT + MEAN_CHAINS * 3 * VEC) * sizeof(Real);
  }
  static constexpr size_t RED = smem(1), APP = smem(4), BWD = smem(1);
  static constexpr size_t CROSS = (size_t)((NBUF + 1) * MAT + 3 * VEC) * sizeof(Real);   // one warp
};

// lane value -> vector slot (all lanes of the warp call it)
template <typename Real, int DP>
__device__ __forceinline__ void put_vec(Real* vs, Real val, int lane) {
  __syncwarp();
  if (lane < DP) vs[lane] = val;
  __syncwarp();
}

// the lane's row constants of the dynamics: F_ii, b_i
template <typename Real> struct RowDyn {
  Real phi, b;
};
template <typename Real, int DP>
__device__ __forceinline__ RowDyn<Real> row_dyn(const KP<Real>& p, int row) {
  return RowDyn<Real>{p.F[row * DP + row], p.b[row]};
}

// m^p = F m + b for the lane's row, m given per lane (slot vs used for dense F)
template <typename Real, int DP>
__device__ __forceinline__ Real predict_mean(const KP<Real>& p, const RowDyn<Real>& rd, Real m,
                                             Real* vs, int lane, int row) {
  if (p.fdiag) return fma(rd.phi, m, rd.b);
  put_vec<Real, DP>(vs, m, lane);
  Real f[DP];
  ld_vec<Real, DP>(p.F + row * DP, f);
  return dot_rv<Real, DP>(f, vs) + rd.b;
}

// R_y^{-1} rows into a padded slot (linear-Gaussian emission)
template <typename Real, int DP>
__device__ __forceinline__ void load_ryinv(const KP<Real>& p, Real* sRy) {
  constexpr int LD = Lay<Real, DP>::LD;
  for (int q = threadIdx.x; q < DP * DP; q += blockDim.x) sRy[(q / DP) * LD + q % DP] = p.Ryinv[q];
}

// ---------------------------------------------------------------------------
// Block-local filtering means from a zero start (block 0: from m0), optionally
// fused with the linearisation (A1) and the auxiliary draw (A2).
// Grid: nb * ceil(C / MEAN_CHAINS) CTAs of MEAN_CHAINS / CPW warps; CTA (g, k)
// runs chains g * MEAN_CHAINS + warp * CPW + j, j < CPW, of block k. A warp
// loads each table row once per step and applies it to its CPW chains.
// ---------------------------------------------------------------------------
template <typename Real, int DP, int CPW>
__global__ void __launch_bounds__(32 * MEAN_CHAINS / CPW) k_mf_reduce(KP<Real> p, MeanArgs<Real> a) {
  pdl_wait();
  pdl_trigger();
  refresh_delta(p);
  using Z = MeanSizes<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC, LD = Lay<Real, DP>::LD;
  constexpr long DD = (long)DP * DP;
  constexpr int NT = 1;   // K'
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* buf = reinterpret_cast<Real*>(smem_raw);
  Real* sRy = buf + NBUF * NT * MAT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Real* vbase = sRy + MAT + warp * 3 * CPW * VEC;   // per chain j: vr, vw, vq
  const int k = blockIdx.x % p.nb, cbase = (blockIdx.x / p.nb) * MEAN_CHAINS + warp * CPW;
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  const RowDyn<Real> rd = row_dyn<Real, DP>(p, row);
  const long tstride = (long)p.nT * DD;
  if (a.x && p.emis == AUX_EMIS_LINEAR_GAUSSIAN) load_ryinv<Real, DP>(p, sRy);
  auto stage = [&](int t) {   // the tables of step t, or an empty copy group past the block
    if (t <= e) stage_mats<Real, DP>(buf + ((t - s) % NBUF) * NT * MAT, a.tab + (long)TK * tstride + t * DD, tstride, NT);
    else cp_async_commit();
  };
  for (int q = 0; q < PREF; ++q) stage(s + q);
  bool valid[CPW];
  int cidx[CPW];
#pragma unroll
  for (int j = 0; j < CPW; ++j) { cidx[j] = cbase + j; valid[j] = cidx[j] < p.C; }
  const bool any = valid[0];
  // the lane's inputs of step t, fetched two steps ahead: x_t and y_t, or ytilde_t
  auto fetch = [&](int t, int j, Real& xv, Real& yv) {
    xv = 0; yv = 0;
    if (!valid[j] || lane >= p.d) return;
    const long ct = (long)cidx[j] * p.nT + t;
    if (a.x) {
      xv = a.x[ct * p.d + lane];
      yv = p.y[(p.y_per_chain ? ct : (long)t) * p.d + lane];
    } else {
      yv = a.yt[ct * p.d + lane];
    }
  };
  Real x1[CPW], y1[CPW], x2[CPW], y2[CPW], m[CPW];
#pragma unroll
  for (int j = 0; j < CPW; ++j) {
    fetch(s, j, x1[j], y1[j]);
    if (s + 1 <= e) fetch(s + 1, j, x2[j], y2[j]);
    m[j] = 0;
  }
  for (int t = s; t <= e; ++t) {
    const int cur = (t - s) % NBUF;
    Real xi[CPW], yv[CPW];
#pragma unroll
    for (int j = 0; j < CPW; ++j) {
      xi[j] = x1[j]; yv[j] = y1[j];
      x1[j] = x2[j]; y1[j] = y2[j];
      if (t + 2 <= e) fetch(t + 2, j, x2[j], y2[j]);
    }
    stage(t + PREF);
    cp_async_wait<PREF>();
    __syncthreads();
    if (any) {
      const Real* sK = buf + cur * NT * MAT;
      Real yti[CPW], mp[CPW];
#pragma unroll
      for (int j = 0; j < CPW; ++j) {
        Real* vq = vbase + (3 * j + 2) * VEC;
        const long ct = (long)cidx[j] * p.nT + t;
        yti[j] = 0;
        if (a.x) {
          const bool obs = !p.mask || p.mask[t];
          Real vi = 0;
          if (p.emis == AUX_EMIS_LINEAR_GAUSSIAN) {
            put_vec<Real, DP>(vq, (lane < p.d) ? yv[j] - xi[j] : (Real)0, lane);
            vi = dot_row_vec<Real, DP>(sRy + row * LD, vq);
          } else if (lane < p.d) {
            vi = (Real)-0.5 + (Real)0.5 * yv[j] * yv[j] * exp(-xi[j]);
          }
          if (!obs) vi = 0;
          if (lane < p.d && valid[j]) {
            const Real ep = philox_normal<Real>(p.seed, (uint32_t)cidx[j], iter_of(p, a.iter), PURPOSE_AUX, (uint32_t)t, lane);
            const Real ui = xi[j] + p.sqrt_r * ep;
            yti[j] = ui + p.r * vi;
            a.u[ct * p.d + lane] = ui;
            a.v[ct * p.d + lane] = vi;
            a.yt[ct * p.d + lane] = yti[j];
          }
        } else {
          yti[j] = yv[j];
        }
        mp[j] = (t == 0) ? p.m0[row] : predict_mean<Real, DP>(p, rd, m[j], vq, lane, row);
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < CPW; ++j)
        if (act) vbase[3 * j * VEC + lane] = yti[j] - mp[j];
      __syncwarp();
      Real kr[DP];
      ld_vec<Real, DP>(sK + row * LD, kr);
#pragma unroll
      for (int j = 0; j < CPW; ++j) m[j] = yti[j] - dot_rv<Real, DP>(kr, vbase + 3 * j * VEC);
    }
  }
#pragma unroll
  for (int j = 0; j < CPW; ++j) {
    if (valid[j] && act) a.z[((long)cidx[j] * p.nb + k) * DP + lane] = m[j];
    if (valid[j] && a.x && k == 0 && lane == 0) p.status_iter[cidx[j]] = *a.cov_status;
  }
}

// ---------------------------------------------------------------------------
// Composition of the block aggregates, one warp per chain.
//   forward  (mats = AH): out[c][k] = m^f_{e_{k-1}}, k = 1 .. nb-1, from
//            m^f_{e_0} = in[c][0] and m^f_{e_k} = AH_k m^f_{e_{k-1}} + in[c][k];
//   backward (mats = GH): out[c][k] = x*_{e_k + 1}, k = nb-1 .. 0, from
//            out[c][nb-1] = 0 and x*_{e_{k-1} + 1} = GH_k out[c][k] + in[c][k].
// Grid: C CTAs of one warp. The recursion is one dependent matrix-vector
// product per block; a CTA per chain keeps each step's copy, barrier and
// product on its own SM (eight chains per CTA put eight chains' steps
// behind one barrier on four SMs).
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __launch_bounds__(32)
    k_mean_cross(KP<Real> p, const Real* __restrict__ mats, const Real* __restrict__ in,
                 Real* __restrict__ out, int backward) {
  pdl_wait();
  pdl_trigger();
  using Z = MeanSizes<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC, LD = Lay<Real, DP>::LD;
  constexpr long DD = (long)DP * DP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* buf = reinterpret_cast<Real*>(smem_raw);
  const int lane = threadIdx.x;
  Real* vq = buf + (NBUF + 1) * MAT;
  const int c = blockIdx.x;
  const bool valid = c < p.C;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  const long cb = (long)(valid ? c : 0) * p.nb;
  // matrices used, in order: forward AH_1 .. AH_{nb-2}; backward GH_{nb-1} .. GH_1
  const int n = backward ? p.nb - 1 : max(0, p.nb - 2);
  auto kk_of = [&](int j) { return backward ? p.nb - 1 - j : 1 + j; };
  Real m = 0;
  if (backward) {
    if (valid && act) out[(cb + p.nb - 1) * DP + lane] = (Real)0;
  } else {
    m = in[cb * DP + row];
    if (valid && act && p.nb > 1) out[(cb + 1) * DP + lane] = m;
  }
  auto stage = [&](int j) {
    if (j < n) stage_mats<Real, DP>(buf + (j % NBUF) * MAT, mats + kk_of(j) * DD, DD, 1);
    else cp_async_commit();
  };
  for (int q = 0; q < PREF; ++q) stage(q);
  Real in1 = (n > 0) ? in[(cb + kk_of(0)) * DP + row] : (Real)0;
  Real in2 = (n > 1) ? in[(cb + kk_of(1)) * DP + row] : (Real)0;
  for (int j = 0; j < n; ++j) {
    const int cur = j % NBUF, kk = kk_of(j);
    const Real inc = in1;
    in1 = in2;
    if (j + 2 < n) in2 = in[(cb + kk_of(j + 2)) * DP + row];
    stage(j + PREF);
    cp_async_wait<PREF>();
    __syncthreads();
    if (valid) {
      put_vec<Real, DP>(vq, m, lane);
      m = dot_row_vec<Real, DP>(buf + cur * MAT + row * LD, vq) + inc;
      if (act) out[(cb + (backward ? kk - 1 : kk + 1)) * DP + lane] = m;
    }
  }
}

// ---------------------------------------------------------------------------
// The same compositions in two levels. Either direction is an affine
// recursion over the blocks, y_j = M_j y_(j-1) + c_j, j = 1 .. n:
//   forward  M_j = AH_j, c_j = in[j], y_0 = in[0], out[j + 1] = y_j (n = nb - 2);
//   backward M_j = GH_(nb-j), c_j = in[nb-j], y_0 = 0, out[nb-1-j] = y_j (n = nb - 1).
// The maps are cut into groups of XGS consecutive j; with the prefix products
// within each group PP_j = M_j M_(j-1) ... M_(first of the group) (chain
// independent: k_cov_xprod, once per covariance pass), every chain forms
//   v_j = M_j v_(j-1) + c_j from v = 0 at each group's start (the groups side by side),
//   Y_(g+1) = PP_(end of g) Y_g + v_(end of g) from Y_0 = y_0 (one warp, serial over the groups),
//   y_j = PP_j Y_(g(j)) + v_j (every j side by side),
// the same values as the one-by-one recursion with XGS + (number of groups) + 1
// dependent matrix-vector products instead of n. One CTA per chain, one warp per group.
// ---------------------------------------------------------------------------
constexpr int XGS = 8;        // maps per group
constexpr int XG_MAX = 16;    // groups per CTA (one warp each): n <= 128

template <typename Real, int DP>
__device__ __forceinline__ int xmap_index(int j, int nb, int backward) {   // block of M_j and c_j
  return backward ? nb - j : j;
}

// PP_j for both directions: CTA (dir, g) walks group g of direction dir (4 warps, products split by columns)
template <typename Real, int DP>
__global__ void __launch_bounds__(32 * CW_SCAN) k_cov_xprod(KP<Real> p, Real* __restrict__ btab) {
  pdl_wait();
  pdl_trigger();
  constexpr int MAT = Lay<Real, DP>::MAT, LD = Lay<Real, DP>::LD, NC = DP / CW_SCAN;
  constexpr long DD = (long)DP * DP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* SACC = reinterpret_cast<Real*>(smem_raw);
  Real* SM = SACC + MAT;
  const int dir = blockIdx.x & 1, g = blockIdx.x >> 1;
  const int nb = p.nb, n = dir ? nb - 1 : nb - 2;
  const int j0 = g * XGS + 1, j1 = min(n, (g + 1) * XGS);
  if (j0 > j1) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  const int c0 = warp * NC;
  const Real* mats = btab + (long)(dir ? BGH : BAH) * nb * DD;
  Real* pp = btab + (long)(dir ? XPG : XPA) * nb * DD;
  for (int q = threadIdx.x; q < DP * DP; q += blockDim.x)
    SACC[(q / DP) * LD + q % DP] = (q / DP == q % DP) ? (Real)1 : (Real)0;
  for (int j = j0; j <= j1; ++j) {
    __syncthreads();
    stage_mats<Real, DP>(SM, mats + (long)xmap_index<Real, DP>(j, nb, dir) * DD, DD, 1);
    cp_async_wait<0>();
    __syncthreads();
    Real out[NC];
    mm_row_c<Real, DP, NC>(SM + row * LD, SACC, c0, out);   // M_j ACC
    __syncthreads();
    if (act) {
      stn<Real, NC>(SACC + row * LD + c0, out);
      stn<Real, NC>(pp + (long)j * DD + row * DP + c0, out);
    }
  }
}

template <typename Real, int DP> struct Cross2Sizes {
  // the group-start maps PP_(h XGS), h = 1 .. XG_MAX - 1, staged at the start; then the vector slots
  static constexpr size_t SMEM = (size_t)(XG_MAX - 1) * Lay<Real, DP>::MAT * sizeof(Real) +
                                 (size_t)(3 * XG_MAX + 1) * Lay<Real, DP>::VEC * sizeof(Real);
  static constexpr size_t XPROD_SMEM = (size_t)2 * Lay<Real, DP>::MAT * sizeof(Real);
};

// Every matrix this kernel reads is known before the chain's vectors are: the
// serial phase 2 reads its G - 1 group-start maps from shared memory, copied
// (cp.async) by the whole CTA while phase 1 runs; phase 1 keeps the next two
// maps' rows in flight and loads its XGS right-hand sides up front; phase 3
// loads the next map's row before the current product.
template <typename Real, int DP>
__global__ void __launch_bounds__(32 * XG_MAX)
    k_mean_cross2(KP<Real> p, const Real* __restrict__ btab, const Real* __restrict__ in,
                  Real* __restrict__ out, int backward) {
  pdl_wait();
  pdl_trigger();
  constexpr int VEC = Lay<Real, DP>::VEC, MAT = Lay<Real, DP>::MAT, LD = Lay<Real, DP>::LD;
  constexpr long DD = (long)DP * DP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sPP = reinterpret_cast<Real*>(smem_raw);   // [XG_MAX - 1] staged group-start maps
  Real* sv = sPP + (XG_MAX - 1) * MAT;             // [XG_MAX] per-warp broadcast slots
  Real* sY = sv + XG_MAX * VEC;                    // [XG_MAX + 1] group starts Y_g
  Real* sV = sY + (XG_MAX + 1) * VEC;              // [XG_MAX] group-end local values
  const int c = blockIdx.x;
  const int g = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  const int nb = p.nb, n = backward ? nb - 1 : nb - 2;
  const int G = (n + XGS - 1) / XGS;
  const long cb = (long)c * nb;
  const Real* mats = btab + (long)(backward ? BGH : BAH) * nb * DD;
  const Real* pp = btab + (long)(backward ? XPG : XPA) * nb * DD;
  if (G > 1) stage_mats<Real, DP>(sPP, pp + (long)XGS * DD, (long)XGS * DD, G - 1);
  const Real y0 = backward ? (Real)0 : in[cb * DP + row];
  if (g == 0 && act) {
    if (backward) out[(cb + nb - 1) * DP + lane] = (Real)0;
    else if (nb > 1) out[(cb + 1) * DP + lane] = y0;
  }
  auto oidx = [&](int j) { return backward ? nb - 1 - j : j + 1; };
  auto mrow = [&](int j) { return mats + (long)xmap_index<Real, DP>(j, nb, backward) * DD + row * DP; };
  Real* vq = sv + g * VEC;
  // phase 1: local values from zero at the group start
  Real v[XGS];
  const int j0 = g * XGS + 1;
  if (g < G) {
    Real cjv[XGS];
#pragma unroll
    for (int s = 0; s < XGS; ++s)
      cjv[s] = (j0 + s <= n) ? in[(cb + xmap_index<Real, DP>(j0 + s, nb, backward)) * DP + row] : (Real)0;
    Real cur = (Real)0;
    Real mr[DP], m1[DP], m2[DP];
    if (j0 <= n) ld_vec<Real, DP>(mrow(j0), m1);
    if (j0 + 1 <= n) ld_vec<Real, DP>(mrow(j0 + 1), m2);
#pragma unroll
    for (int s = 0; s < XGS; ++s) {
      const int j = j0 + s;
      v[s] = cur;
      if (j <= n) {
#pragma unroll
        for (int q = 0; q < DP; ++q) { mr[q] = m1[q]; m1[q] = m2[q]; }
        if (j + 2 <= n && s + 2 < XGS) ld_vec<Real, DP>(mrow(j + 2), m2);
        put_vec<Real, DP>(vq, cur, lane);
        cur = dot_rv<Real, DP>(mr, vq) + cjv[s];
        v[s] = cur;
      }
    }
    if (act) sV[g * VEC + lane] = cur;
  }
  cp_async_wait<0>();
  __syncthreads();
  // phase 2: the group starts, one warp, maps from shared memory
  if (g == 0) {
    Real Y = y0;
    if (act) sY[lane] = Y;
    for (int h = 0; h + 1 < G; ++h) {
      Real pr[DP];
      ld_vec<Real, DP>(sPP + h * MAT + row * LD, pr);
      put_vec<Real, DP>(vq, Y, lane);
      Y = dot_rv<Real, DP>(pr, vq) + sV[h * VEC + row];
      if (act) sY[(h + 1) * VEC + lane] = Y;
    }
  }
  __syncthreads();
  // phase 3: every map's value from its group start
  if (g < G) {
    Real pr[DP], pn[DP];
    if (j0 <= n) ld_vec<Real, DP>(pp + (long)j0 * DD + row * DP, pn);
#pragma unroll
    for (int s = 0; s < XGS; ++s) {
      const int j = j0 + s;
      if (j <= n) {
#pragma unroll
        for (int q = 0; q < DP; ++q) pr[q] = pn[q];
        if (j + 1 <= n && s + 1 < XGS) ld_vec<Real, DP>(pp + (long)(j + 1) * DD + row * DP, pn);
        const Real yj = dot_rv<Real, DP>(pr, sY + g * VEC) + v[s];
        if (act) out[(cb + oidx(j)) * DP + lane] = yj;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Filtering means from the true block start, likelihood terms and
// (APPLY_EPI) the backward elements with the block aggregate. Same grid and
// chain layout as k_mf_reduce.
// ---------------------------------------------------------------------------
template <typename Real, int DP, int CPW>
__global__ void __launch_bounds__(32 * MEAN_CHAINS / CPW) k_mf_apply(KP<Real> p, MeanArgs<Real> a) {
  pdl_wait();
  pdl_trigger();
  refresh_delta(p);
  using Z = MeanSizes<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC, LD = Lay<Real, DP>::LD;
  constexpr long DD = (long)DP * DP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const bool epi = a.flags & APPLY_EPI;
  const int NT = epi ? 4 : 1;   // K' (, G, chol(Sigma), G_s .. G_{t-1})
  Real* buf = reinterpret_cast<Real*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Real* vbase = buf + NBUF * 4 * MAT + MAT + warp * 3 * CPW * VEC;   // per chain j: vr, vw, vq
  const int k = blockIdx.x % p.nb, cbase = (blockIdx.x / p.nb) * MEAN_CHAINS + warp * CPW;
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  const RowDyn<Real> rd = row_dyn<Real, DP>(p, row);
  const long tstride = (long)p.nT * DD;
  const Real* PF = a.tab + (long)TPF * tstride;
  auto stage = [&](int t) {   // the tables of step t, or an empty copy group past the block
    if (t <= e) stage_mats<Real, DP>(buf + ((t - s) % NBUF) * 4 * MAT, a.tab + (long)TK * tstride + t * DD, tstride, NT);
    else cp_async_commit();
  };
  for (int q = 0; q < PREF; ++q) stage(s + q);
  bool valid[CPW];
  int cidx[CPW];
#pragma unroll
  for (int j = 0; j < CPW; ++j) { cidx[j] = cbase + j; valid[j] = cidx[j] < p.C; }
  const bool any = valid[0];
  Real mp[CPW], ubar[CPW];
  TermSum<Real> qacc[CPW];
#pragma unroll
  for (int j = 0; j < CPW; ++j) {
    ubar[j] = 0; mp[j] = 0;
    if (valid[j]) {
      if (k == 0) mp[j] = p.m0[row];
      else mp[j] = predict_mean<Real, DP>(p, rd, a.mstart[((long)cidx[j] * p.nb + k) * DP + row],
                                          vbase + (3 * j + 2) * VEC, lane, row);
    }
  }
  // the lane's ytilde_t and (given) eps_t, fetched two steps ahead
  auto fetch = [&](int t, int j, Real& yv, Real& ev) {
    yv = 0; ev = 0;
    if (!valid[j] || lane >= p.d) return;
    const long ct = (long)cidx[j] * p.nT + t;
    yv = a.yt[ct * p.d + lane];
    if (epi && a.eps) ev = a.eps[ct * p.d + lane];
  };
  Real y1[CPW], e1[CPW], y2[CPW], e2[CPW];
#pragma unroll
  for (int j = 0; j < CPW; ++j) {
    fetch(s, j, y1[j], e1[j]);
    if (s + 1 <= e) fetch(s + 1, j, y2[j], e2[j]);
  }
  for (int t = s; t <= e; ++t) {
    const int cur = (t - s) % NBUF;
    Real yti[CPW], eg[CPW];
#pragma unroll
    for (int j = 0; j < CPW; ++j) {
      yti[j] = y1[j]; eg[j] = e1[j];
      y1[j] = y2[j]; e1[j] = e2[j];
      if (t + 2 <= e) fetch(t + 2, j, y2[j], e2[j]);
    }
    stage(t + PREF);
    cp_async_wait<PREF>();
    __syncthreads();
    if (any) {
      const Real* sK = buf + cur * 4 * MAT;
      Real ej[CPW];
      __syncwarp();
#pragma unroll
      for (int j = 0; j < CPW; ++j) {
        ej[j] = act ? yti[j] - mp[j] : (Real)0;
        if (act) vbase[3 * j * VEC + lane] = ej[j];
      }
      __syncwarp();
      Real kr[DP];
      ld_vec<Real, DP>(sK + row * LD, kr);
      Real m[CPW], mpn[CPW];
#pragma unroll
      for (int j = 0; j < CPW; ++j) {
        const Real kv = dot_rv<Real, DP>(kr, vbase + 3 * j * VEC);
        qacc[j].add_prod(ej[j], kv);   // e^T K' e, summed over the lanes at the end
        m[j] = yti[j] - kv;
        const long ct = (long)cidx[j] * p.nT + t;
        if (valid[j] && a.mf && lane < p.d) a.mf[ct * p.d + lane] = m[j];
        if (valid[j] && a.Pf && lane < p.d)
          for (int jj = 0; jj < p.d; ++jj) a.Pf[(ct * p.d + lane) * p.d + jj] = PF[t * DD + lane * DP + jj];
        mpn[j] = (t < p.nT - 1) ? predict_mean<Real, DP>(p, rd, m[j], vbase + (3 * j + 2) * VEC, lane, row)
                                : (Real)0;
      }
      if (epi) {
        const Real* sG = sK + MAT;
        const Real* sLS = sG + MAT;
        const Real* sGP = sLS + MAT;
        Real ei[CPW];
#pragma unroll
        for (int j = 0; j < CPW; ++j) {
          ei[j] = 0;
          if (lane < p.d && valid[j] && !(a.flags & APPLY_SMOOTH))
            ei[j] = a.eps ? eg[j]
                          : philox_normal<Real>(p.seed, (uint32_t)cidx[j], iter_of(p, a.iter), PURPOSE_BACKWARD, (uint32_t)t, lane);
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < CPW; ++j)
          if (act) { vbase[3 * j * VEC + lane] = mpn[j]; vbase[(3 * j + 1) * VEC + lane] = ei[j]; }
        __syncwarp();
        Real gr[DP], lr[DP];
        ld_vec<Real, DP>(sG + row * LD, gr);
        ld_vec<Real, DP>(sLS + row * LD, lr);
        Real ui[CPW];
#pragma unroll
        for (int j = 0; j < CPW; ++j) {
          ui[j] = m[j] - dot_rv<Real, DP>(gr, vbase + 3 * j * VEC) + dot_rv<Real, DP>(lr, vbase + (3 * j + 1) * VEC);
          if (valid[j] && act) a.U[((long)cidx[j] * p.nT + t) * DP + lane] = ui[j];
        }
#pragma unroll
        for (int j = 0; j < CPW; ++j)
          if (act) vbase[(3 * j + 2) * VEC + lane] = ui[j];
        __syncwarp();
        ld_vec<Real, DP>(sGP + row * LD, gr);
#pragma unroll
        for (int j = 0; j < CPW; ++j) ubar[j] += dot_rv<Real, DP>(gr, vbase + (3 * j + 2) * VEC);
      }
#pragma unroll
      for (int j = 0; j < CPW; ++j) mp[j] = mpn[j];
    }
  }
#pragma unroll
  for (int j = 0; j < CPW; ++j) {
    if (!valid[j]) continue;
    const double q = warp_sum<double>(qacc[j].value()) / (double)p.r;
    const int c = cidx[j];
    if (lane == 0) {
      const long ck = (long)c * p.nb + k;
      if (a.flags & APPLY_STORE_Q) a.fqb[ck] = q;
      if (a.flags & APPLY_REV_DIFF) a.lz_part[ck] = -0.5 * (a.fqb[ck] - q);
      if (a.flags & APPLY_LOGZ) {
        const double half_dlog2pi = 0.5 * p.d * 1.8378770664093454835606594728112;
        a.lz_part[ck] = -((double)(e - s + 1) * half_dlog2pi + 0.5 * (a.ld[k] + q));
      }
      if (a.status && k == 0 && *a.cov_status) atomicOr(&a.status[c], *a.cov_status);
    }
    if (epi && act) a.guv[((long)c * p.nb + k) * DP + lane] = ubar[j];
  }
}

// ---------------------------------------------------------------------------
// Backward sampling inside each block from x*_{e+1} (k_mean_cross, backward):
// x*_t = G_t x*_{t+1} + U_t (G_{T-1} = 0), with the MH terms when b.mh.
// Same grid and chain layout as k_mf_reduce.
// ---------------------------------------------------------------------------
template <typename Real, int DP, int CPW>
__global__ void __launch_bounds__(32 * MEAN_CHAINS / CPW)
    k_mb_apply(KP<Real> p, BackArgs<Real> b, const Real* __restrict__ xnext) {
  pdl_wait();
  pdl_trigger();
  refresh_delta(p);
  using Z = MeanSizes<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC, LD = Lay<Real, DP>::LD;
  constexpr long DD = (long)DP * DP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* buf = reinterpret_cast<Real*>(smem_raw);
  Real* sRy = buf + NBUF * MAT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Real* vbase = sRy + MAT + warp * 3 * CPW * VEC;   // per chain j: vx, vxs
  const int k = blockIdx.x % p.nb, cbase = (blockIdx.x / p.nb) * MEAN_CHAINS + warp * CPW;
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  if (b.mh && p.emis == AUX_EMIS_LINEAR_GAUSSIAN) load_ryinv<Real, DP>(p, sRy);
  auto stage = [&](int t) {   // G_t, or an empty copy group before the block
    if (t >= s) stage_mats<Real, DP>(buf + ((e - t) % NBUF) * MAT, b.G + t * DD, DD, 1);
    else cp_async_commit();
  };
  for (int q = 0; q < PREF; ++q) stage(e - q);
  bool valid[CPW];
  long cb[CPW];
  Real xi[CPW], u1[CPW], u2[CPW];
  MhIn<Real> q1[CPW], q2[CPW];
  TermSum<Real> acc[CPW];
#pragma unroll
  for (int j = 0; j < CPW; ++j) {
    const int c = cbase + j;
    valid[j] = c < p.C;
    cb[j] = (long)(valid[j] ? c : 0) * p.nT;
    xi[j] = valid[j] ? xnext[((long)c * p.nb + k) * DP + row] : (Real)0;
    // the lane's U_t and MH inputs, fetched two steps ahead
    u1[j] = b.U[(cb[j] + e) * DP + row];
    q1[j] = b.mh ? mh_load<Real>(p, b, cb[j] + e, e, lane) : MhIn<Real>{};
    u2[j] = (e - 1 >= s) ? b.U[(cb[j] + e - 1) * DP + row] : (Real)0;
    q2[j] = (b.mh && e - 1 >= s) ? mh_load<Real>(p, b, cb[j] + e - 1, e - 1, lane) : MhIn<Real>{};
  }
  const bool any = valid[0];
  for (int t = e; t >= s; --t) {
    const int cur = (e - t) % NBUF;
    Real uc[CPW];
    MhIn<Real> qc[CPW];
#pragma unroll
    for (int j = 0; j < CPW; ++j) {
      uc[j] = u1[j]; qc[j] = q1[j];
      u1[j] = u2[j]; q1[j] = q2[j];
      if (t - 2 >= s) {
        u2[j] = b.U[(cb[j] + t - 2) * DP + row];
        if (b.mh) q2[j] = mh_load<Real>(p, b, cb[j] + t - 2, t - 2, lane);
      }
    }
    stage(t - PREF);
    cp_async_wait<PREF>();
    __syncthreads();
    if (any) {
      __syncwarp();
#pragma unroll
      for (int j = 0; j < CPW; ++j)
        if (act) vbase[3 * j * VEC + lane] = xi[j];
      __syncwarp();
      Real gr[DP];
      ld_vec<Real, DP>(buf + cur * MAT + row * LD, gr);
#pragma unroll
      for (int j = 0; j < CPW; ++j) {
        xi[j] = dot_rv<Real, DP>(gr, vbase + 3 * j * VEC) + uc[j];
        const long ct = cb[j] + t;
        if (valid[j] && lane < p.d) b.xs[ct * p.d + lane] = xi[j];
        if (b.mh && valid[j])
          mh_step_terms<Real, DP>(p, b, ct, t, xi[j], qc[j], sRy, vbase + (3 * j + 1) * VEC, lane, row, acc[j]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < CPW; ++j) {
    if (valid[j] && b.mh) {
      const double r = warp_sum<double>(acc[j].value());
      if (lane == 0) b.mh_part[(long)(cbase + j) * p.nb + k] = r;
    }
  }
}

}  // namespace auxk
