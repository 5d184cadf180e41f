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
  double qacc[CPW];
#pragma unroll
  for (int j = 0; j < CPW; ++j) {
    ubar[j] = 0; qacc[j] = 0.0; mp[j] = 0;
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
        qacc[j] += (double)ej[j] * (double)kv;   // e^T K' e, summed over the lanes at the end
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
    const double q = warp_sum<double>(qacc[j]) / (double)p.r;
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
  double acc[CPW];
#pragma unroll
  for (int j = 0; j < CPW; ++j) {
    const int c = cbase + j;
    valid[j] = c < p.C;
    cb[j] = (long)(valid[j] ? c : 0) * p.nT;
    xi[j] = valid[j] ? xnext[((long)c * p.nb + k) * DP + row] : (Real)0;
    acc[j] = 0.0;
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
          acc[j] += mh_step_terms<Real, DP>(p, b, ct, t, xi[j], qc[j], sRy, vbase + (3 * j + 1) * VEC, lane, row);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < CPW; ++j) {
    if (valid[j] && b.mh) {
      const double r = warp_sum<double>(acc[j]);
      if (lane == 0) b.mh_part[(long)(cbase + j) * p.nb + k] = r;
    }
  }
}

}  // namespace auxk
