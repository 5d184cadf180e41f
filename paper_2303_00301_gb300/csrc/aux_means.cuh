// aux_means.cuh — the per-chain half of the parallel filter when the
// covariance tables of aux_cov.cuh are available: every step is a handful of
// DP x DP matrix-vector products with matrices shared by all chains.
//
// Filtering means (Kalman filter algorithm, Appendix A.1, with H = I, R = r I):
//   m^p_0 = m0,  m^p_t = F m^f_{t-1} + b,
//   w_t = W_t (ytilde_t - m^p_t),  m^f_t = ytilde_t - r W_t^T w_t,
//   log-likelihood term  -(d/2) log 2 pi - (1/2) (log det S_t + |w_t|^2).
// The recursion is affine in m^f_{s-1} with linear part AH_k over a block, so
// the blocked scan keeps the structure of the full filter: k_mf_reduce runs each
// block from m^f_{s-1} = 0 (block 0 from m0) and keeps the block-end mean z_k;
// k_mf_apply composes the aggregates of the earlier blocks (m^f_{e_k} =
// AH_k m^f_{e_{k-1}} + z_k) and re-runs its block from the true start, with
// the backward elements of Eq. (A.14): U_t = m^f_t - G_t m^p_{t+1} +
// chol(Sigma_t) eps_t and the block aggregate sum_t (G_s ... G_{t-1}) U_t that
// the (G, U) suffix scan of Proposition A.1 (k_sample_backward) consumes.
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
  Real* U;                    // [C][T][DP]
  Real* guv;                  // [C][nb][DP]
  double* fqb;                // [C][nb] sum of |w_t|^2 over the block
  double* lz_part;            // [C][nb]
  Real* mf;                   // optional [C][T][d]
  Real* Pf;                   // optional [C][T][d][d]
  const Real* eps;            // optional [C][T][d] backward noise (else Philox)
  int32_t* status;            // optional sticky per-chain status
};

constexpr int MEAN_WPC = 8;   // warps (chain-blocks) per CTA

// sum_j grow[j] v[j]: grow a 16-byte aligned global row (read-only path),
// v a shared vector slot (broadcast reads)
template <typename Real, int DP>
__device__ __forceinline__ Real gdot(const Real* __restrict__ grow, const Real* v) {
  using V = typename Vec16<Real>::V;
  constexpr int N = Vec16<Real>::N;
  Real acc[4] = {(Real)0, (Real)0, (Real)0, (Real)0};
#pragma unroll
  for (int q = 0; q < DP / N; ++q) {
    Real ga[N], vb[N];
    unpack<Real>(__ldg(reinterpret_cast<const V*>(grow) + q), ga);
    unpack<Real>(reinterpret_cast<const V*>(v)[q], vb);
#pragma unroll
    for (int j = 0; j < N; ++j) acc[(q * N + j) & 3] = fma(ga[j], vb[j], acc[(q * N + j) & 3]);
  }
  return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

// lane value -> vector slot (all lanes of the warp call it)
template <typename Real, int DP>
__device__ __forceinline__ void put_vec(Real* vs, Real val, int lane) {
  __syncwarp();
  if (lane < DP) vs[lane] = val;
  __syncwarp();
}

// m^p = F m + b for the lane's row, m given per lane (slot vs used for dense F)
template <typename Real, int DP>
__device__ __forceinline__ Real predict_mean(const KP<Real>& p, Real m, Real* vs, int lane, int row) {
  if (p.fdiag) return fma(p.F[row * DP + row], m, p.b[row]);
  put_vec<Real, DP>(vs, m, lane);
  return gdot<Real, DP>(p.F + row * DP, vs) + p.b[row];
}

// ---------------------------------------------------------------------------
// Block-local filtering means from a zero start (block 0: from m0), optionally
// fused with the linearisation (A1) and the auxiliary draw (A2).
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __launch_bounds__(32 * MEAN_WPC) k_mf_reduce(KP<Real> p, MeanArgs<Real> a) {
  constexpr int VEC = Lay<Real, DP>::VEC;
  constexpr long DD = (long)DP * DP;
  __shared__ __align__(16) Real vsm[MEAN_WPC * 3 * VEC];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = blockIdx.x * MEAN_WPC + warp;
  if (item >= p.C * p.nb) return;
  const int k = item / p.C, c = item % p.C;
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  Real* vr = vsm + warp * 3 * VEC;
  Real* vw = vr + VEC;
  Real* vq = vw + VEC;
  const Real* W = a.tab + (long)TW * p.nT * DD;
  const Real* WT = a.tab + (long)TWT * p.nT * DD;
  Real m = 0;
  for (int t = s; t <= e; ++t) {
    const long ct = (long)c * p.nT + t;
    Real yti = 0;
    if (a.x) {
      const Real* yr = p.y + (p.y_per_chain ? ct : (long)t) * p.d;
      const bool obs = !p.mask || p.mask[t];
      const Real xi = (lane < p.d) ? a.x[ct * p.d + lane] : (Real)0;
      Real vi = 0;
      if (p.emis == AUX_EMIS_LINEAR_GAUSSIAN) {
        put_vec<Real, DP>(vq, (lane < p.d) ? yr[lane] - xi : (Real)0, lane);
        vi = gdot<Real, DP>(p.Ryinv + row * DP, vq);
      } else if (lane < p.d) {
        vi = (Real)-0.5 + (Real)0.5 * yr[lane] * yr[lane] * exp(-xi);
      }
      if (!obs) vi = 0;
      if (lane < p.d) {
        const Real ep = philox_normal<Real>(p.seed, (uint32_t)c, a.iter, PURPOSE_AUX, (uint32_t)t, lane);
        const Real ui = xi + p.sqrt_r * ep;
        yti = ui + p.r * vi;
        a.u[ct * p.d + lane] = ui;
        a.v[ct * p.d + lane] = vi;
        a.yt[ct * p.d + lane] = yti;
      }
    } else if (lane < p.d) {
      yti = a.yt[ct * p.d + lane];
    }
    const Real mp = (t == 0) ? p.m0[row] : predict_mean<Real, DP>(p, m, vq, lane, row);
    put_vec<Real, DP>(vr, act ? yti - mp : (Real)0, lane);
    const Real wi = gdot<Real, DP>(W + t * DD + row * DP, vr);
    put_vec<Real, DP>(vw, wi, lane);
    m = yti - p.r * gdot<Real, DP>(WT + t * DD + row * DP, vw);
  }
  if (act) a.z[((long)c * p.nb + k) * DP + lane] = m;
  if (a.x && k == 0 && lane == 0) p.status_iter[c] = *a.cov_status;
}

// ---------------------------------------------------------------------------
// Filtering means from the true block start, likelihood terms, and (APPLY_EPI)
// the backward elements U_t with the block aggregate of the (G, U) scan.
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __launch_bounds__(32 * MEAN_WPC) k_mf_apply(KP<Real> p, MeanArgs<Real> a) {
  constexpr int VEC = Lay<Real, DP>::VEC;
  constexpr long DD = (long)DP * DP;
  __shared__ __align__(16) Real vsm[MEAN_WPC * 3 * VEC];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = blockIdx.x * MEAN_WPC + warp;
  if (item >= p.C * p.nb) return;
  const int k = item / p.C, c = item % p.C;
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  Real* vr = vsm + warp * 3 * VEC;
  Real* vw = vr + VEC;
  Real* vq = vw + VEC;
  const Real* W = a.tab + (long)TW * p.nT * DD;
  const Real* WT = a.tab + (long)TWT * p.nT * DD;
  const Real* G = a.tab + (long)TG * p.nT * DD;
  const Real* LS = a.tab + (long)TLS * p.nT * DD;
  const Real* GP = a.tab + (long)TGP * p.nT * DD;
  const Real* PF = a.tab + (long)TPF * p.nT * DD;
  const Real* AH = a.btab + (long)BAH * p.nb * DD;
  const bool epi = a.flags & APPLY_EPI;
  // m^f_{s-1}: compose the aggregates of blocks 0 .. k-1
  Real m = 0;
  if (k > 0) {
    m = a.z[((long)c * p.nb) * DP + row];
    for (int kk = 1; kk < k; ++kk) {
      put_vec<Real, DP>(vq, m, lane);
      m = gdot<Real, DP>(AH + kk * DD + row * DP, vq) + a.z[((long)c * p.nb + kk) * DP + row];
    }
  }
  Real mp = (k == 0) ? p.m0[row] : predict_mean<Real, DP>(p, m, vq, lane, row);
  double qacc = 0.0;
  Real ubar = 0;
  for (int t = s; t <= e; ++t) {
    const long ct = (long)c * p.nT + t;
    const Real yti = (lane < p.d) ? a.yt[ct * p.d + lane] : (Real)0;
    put_vec<Real, DP>(vr, act ? yti - mp : (Real)0, lane);
    const Real wi = gdot<Real, DP>(W + t * DD + row * DP, vr);
    if (act) qacc += (double)wi * (double)wi;
    put_vec<Real, DP>(vw, wi, lane);
    m = yti - p.r * gdot<Real, DP>(WT + t * DD + row * DP, vw);
    if (a.mf && lane < p.d) a.mf[ct * p.d + lane] = m;
    if (a.Pf && lane < p.d)
      for (int j = 0; j < p.d; ++j) a.Pf[(ct * p.d + lane) * p.d + j] = PF[t * DD + lane * DP + j];
    const Real mpn = (t < p.nT - 1) ? predict_mean<Real, DP>(p, m, vq, lane, row) : (Real)0;
    if (epi) {
      Real ei = 0;
      if (lane < p.d)
        ei = a.eps ? a.eps[ct * p.d + lane]
                   : philox_normal<Real>(p.seed, (uint32_t)c, a.iter, PURPOSE_BACKWARD, (uint32_t)t, lane);
      __syncwarp();
      if (act) { vr[lane] = mpn; vw[lane] = ei; }
      __syncwarp();
      const Real ui = m - gdot<Real, DP>(G + t * DD + row * DP, vr) +
                      gdot<Real, DP>(LS + t * DD + row * DP, vw);
      if (act) a.U[ct * DP + lane] = ui;
      put_vec<Real, DP>(vq, ui, lane);
      ubar += gdot<Real, DP>(GP + t * DD + row * DP, vq);
    }
    mp = mpn;
  }
  const double q = warp_sum<double>(qacc);
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
  if (epi && act) a.guv[((long)c * p.nb + k) * DP + lane] = ubar;
}

}  // namespace auxk
