// aux_batch.cu — many independent models (instances of uneven T and d_x,
// one or more chains each) advanced by one persistent launch per MCMC
// iteration (Algorithm 2 for every chain of every model).
//
// Each model is an aux_model handle in a table mode (FP32, first-order
// proposal, scan sampler, homogeneous dynamics with diagonal F, no delta
// adaptation). Its per-step tables K'_t = r S_t^{-1}, G_t and chol(Sigma_t)
// are copied once (cached) or after every covariance pass (shared) into the
// batch layout below, and the batch forms its own block tables for a block
// length of its choosing (the autotuner's): within means block k = [s, e]
//   GP_t = G_s ... G_{t-1}   (GP_s = I), the prefix products of the (G, U) scan,
//   GH_k = G_s ... G_e,      AH_k = M_e ... M_s with M_t = K'_t F,
// the linear parts of the block compositions of Appendix A.2.2 and A.2.1.
//
// One MCMC iteration of chain c is a list of warp items, by pass:
//   FR  block k: linearise at x (A1), u and ytilde (A2, Eq. (2.7)); filtering
//                means from a zero start (block 0: from m0) -> z_k
//   FX  chain:   m^f_{e_k} = AH_k m^f_{e_{k-1}} + z_k over the blocks
//   FA  block k: filtering means from the true start, the likelihood quadratic
//                forms, U_t = m^f_t - G_t m^p_{t+1} + chol(Sigma_t) eps_t
//                (Eq. (A.14)) and the block aggregate sum_t GP_t U_t
//   BX  chain:   x*_{e_k + 1} from the later blocks' aggregates (Prop. A.1)
//   BR  block k: x*_t = G_t x*_{t+1} + U_t down the block with the MH terms and
//                ytilde*_t = u_t + r v*_t, then the reverse filter of the block
//                from a zero start -> z_k
//   RX  chain:   as FX for the reverse pass
//   RA  block k: the reverse filter from the true start: log Z(x) - log Z(x*)
//   MH  chain:   log alpha and the MH test of Algorithm 2
//   CM  block k: x <- x* on acceptance
// The list holds the passes in this order, so every item's inputs are written
// by items earlier in the list. Warps of a persistent grid take items from an
// atomic counter; before it starts, an item waits until every item of the
// previous pass of its chain has signalled completion (per-(chain, pass)
// counters: release by a fence and an atomic add, acquire loads by every lane
// of the waiting warp). An item waits only on items taken before it, whose
// warps are running, so the list always drains. Every wait is bounded (time and
// iterations): a wait that runs out raises the batch's abort word, after which
// the remaining items are skipped; the host reads it as AUX_E_TIMEOUT. The
// last warp to leave resets the counters for the next launch.
//
// Batch layout of a DP x DP matrix (DP = 8, 16, 32, 64): the 16-byte quad q of
// row i (elements 4q .. 4q + 3) is quad number q * DP + i, so that when lane i
// reads quad q of its row, the warp reads consecutive 16-byte words. A lane
// owns rows lane and lane + 32 (DP = 64).
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "aux_cov.cuh"   // the table slots (TK, TG, TLS)

namespace auxk {
namespace batch {

constexpr int FR = 0, FX = 1, FA = 2, BX = 3, BR = 4, RX = 5, RA = 6, MH = 7, CM = 8, NPASS = 9;
constexpr unsigned FULL = 0xffffffffu;
constexpr long long kWaitNs = 2000000000LL;   // a wait gives up after 2 s ...
constexpr int kWaitIters = 1 << 24;           // ... or this many polls
constexpr int kMaxDP = 64;

// one chain of one model
struct Job {
  int d, DP, T, L, nb, emis, y_per_chain, c;
  uint64_t seed;
  float r, sqrt_r;
  const float* y;          // [T][d] (or the chain's [T][d] when per chain)
  const uint8_t* mask;     // [T] or null
  const float *m0, *F, *b, *Ryinv;   // the model's padded constants
  const int32_t* cov_status;
  const float *K, *G, *LS, *GP;      // [T][DP * DP], batch layout
  const float *AH, *GH;              // [nb][DP * DP], batch layout
  float* x;                          // [T][d]
  float *u, *v, *yt, *yts, *xs;      // [T][d]
  float* U;                          // [T][DP]
  float *z, *ms, *gu, *xn;           // [nb][DP]
  double *fq, *lz, *mh;              // [nb]
  int32_t *status_iter, *status, *accept;   // the chain's words
  double* la;
};

struct Args {
  const Job* jobs;
  const int2* items;       // (job, pass << 16 | block)
  int n_items;
  unsigned* cnt;           // [jobs][NPASS]
  int n_jobs;
  unsigned* head;          // next item
  unsigned* exited;        // warps that left
  unsigned total_warps;
  int* abort;              // nonzero: a wait ran out; the rest of the launch is skipped
  const uint64_t* iter;    // the MCMC iteration (device)
  uint32_t* acc_count;     // [jobs] or null
  double* log_alpha;       // [jobs] or null
};

__device__ __forceinline__ long long globaltimer() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

// every lane waits (acquire) until *ctr >= need; false when the batch aborted
__device__ bool wait_count(const unsigned* ctr, unsigned need, int* abort, int lane) {
  long long t0 = 0;
  if (lane == 0) t0 = globaltimer();
  unsigned ns = 32;
  for (int it = 0;; ++it) {
    const unsigned v = ld_acquire(ctr);
    if (__all_sync(FULL, v >= need)) return true;
    if (__any_sync(FULL, ld_volatile(abort) != 0)) return false;
    int out = 0;
    if (lane == 0) out = (it >= kWaitIters) || (globaltimer() - t0 > kWaitNs);
    if (__shfl_sync(FULL, out, 0)) {
      if (lane == 0) atomicExch(abort, 1);
      return false;
    }
    __nanosleep(ns);
    if (ns < 1024) ns *= 2;
  }
}

template <int DP> struct RPL { static constexpr int R = DP > 32 ? 2 : 1; };

// y[r] = sum_j M[i][j] v[j] for the lane's rows i = lane + 32 r (zero for i >= DP).
// M in the batch layout (read-only), v a warp slot; the even and odd j go to two
// accumulators, the order of the narrow kernels' dot products.
template <int DP>
__device__ __forceinline__ void bmv(const float* __restrict__ M, const float* v, int lane,
                                    float (&y)[RPL<DP>::R]) {
  constexpr int R = RPL<DP>::R;
  const float4* M4 = reinterpret_cast<const float4*>(M);
  const float4* v4 = reinterpret_cast<const float4*>(v);
  float a0[R], a1[R];
#pragma unroll
  for (int r = 0; r < R; ++r) { a0[r] = 0.f; a1[r] = 0.f; }
  const bool act0 = lane < DP;
#pragma unroll 8
  for (int q = 0; q < DP / 4; ++q) {
    const float4 x = v4[q];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = lane + 32 * r;
      if (r == 0 && !act0) continue;
      const float4 m = __ldg(M4 + q * DP + i);
      fma_pair(a0[r], a1[r], m.x, m.y, x.x, x.y);
      fma_pair(a0[r], a1[r], m.z, m.w, x.z, x.w);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) y[r] = (r == 0 && !act0) ? 0.f : a0[r] + a1[r];
}

// the same for a row-major DP x DP matrix (R_y^{-1} of the model)
template <int DP>
__device__ __forceinline__ void rmv(const float* __restrict__ M, const float* v, int lane,
                                    float (&y)[RPL<DP>::R]) {
  constexpr int R = RPL<DP>::R;
  const float4* v4 = reinterpret_cast<const float4*>(v);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = lane + 32 * r;
    float a0 = 0.f, a1 = 0.f;
    if (i < DP) {
      const float4* M4 = reinterpret_cast<const float4*>(M + (long)i * DP);
#pragma unroll 8
      for (int q = 0; q < DP / 4; ++q) {
        const float4 x = v4[q], m = __ldg(M4 + q);
        fma_pair(a0, a1, m.x, m.y, x.x, x.y);
        fma_pair(a0, a1, m.z, m.w, x.z, x.w);
      }
    }
    y[r] = a0 + a1;
  }
}

// the lane's rows into a warp slot (all lanes call it)
template <int DP>
__device__ __forceinline__ void bput(float* slot, const float (&val)[RPL<DP>::R], int lane) {
  __syncwarp();
#pragma unroll
  for (int r = 0; r < RPL<DP>::R; ++r)
    if (lane + 32 * r < DP) slot[lane + 32 * r] = val[r];
  __syncwarp();
}

__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }

// filtering means of block [s, e] from the zero start (block 0: from m0), on
// ytilde given (yin) or formed from x (lin); the block end into z_k
template <int DP>
__device__ void reduce_block(const Job& J, int k, uint64_t iter, bool lin, const float* yin, float* vs,
                             int lane) {
  constexpr int R = RPL<DP>::R;
  const int s = k * J.L, e = min(J.T, s + J.L) - 1, d = J.d;
  float m[R], phi[R], bb[R], m0v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = lane + 32 * r;
    m[r] = 0.f;
    phi[r] = i < DP ? J.F[i * DP + i] : 0.f;
    bb[r] = i < DP ? J.b[i] : 0.f;
    m0v[r] = i < DP ? J.m0[i] : 0.f;
  }
  if (lin && k == 0 && lane == 0) *J.status_iter = *J.cov_status;
  for (int t = s; t <= e; ++t) {
    float yti[R];
    if (lin) {
      float xi[R], yv[R], vi[R];
      const bool obs = !J.mask || J.mask[t];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = lane + 32 * r;
        xi[r] = i < d ? J.x[(long)t * d + i] : 0.f;
        yv[r] = i < d ? J.y[(long)t * d + i] : 0.f;
        vi[r] = 0.f;
      }
      if (J.emis == AUX_EMIS_LINEAR_GAUSSIAN) {
        float dv[R];
#pragma unroll
        for (int r = 0; r < R; ++r) dv[r] = yv[r] - xi[r];
        bput<DP>(vs + 2 * kMaxDP, dv, lane);
        rmv<DP>(J.Ryinv, vs + 2 * kMaxDP, lane, vi);
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) vi[r] = -0.5f + 0.5f * yv[r] * yv[r] * expf(-xi[r]);
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = lane + 32 * r;
        yti[r] = 0.f;
        if (!obs) vi[r] = 0.f;
        if (i < d) {
          const float ep = philox_normal<float>(J.seed, (uint32_t)J.c, iter, PURPOSE_AUX, (uint32_t)t, i);
          const float ui = xi[r] + J.sqrt_r * ep;
          yti[r] = ui + J.r * vi[r];
          J.u[(long)t * d + i] = ui;
          J.v[(long)t * d + i] = vi[r];
          J.yt[(long)t * d + i] = yti[r];
        }
      }
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = lane + 32 * r;
        yti[r] = i < d ? yin[(long)t * d + i] : 0.f;
      }
    }
    float ev[R], kv[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float mp = (t == 0) ? m0v[r] : fmaf(phi[r], m[r], bb[r]);
      ev[r] = lane + 32 * r < DP ? yti[r] - mp : 0.f;
    }
    bput<DP>(vs, ev, lane);
    bmv<DP>(J.K + (long)t * DP * DP, vs, lane, kv);
#pragma unroll
    for (int r = 0; r < R; ++r) m[r] = yti[r] - kv[r];
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (lane + 32 * r < DP) J.z[(long)k * DP + lane + 32 * r] = m[r];
}

// composition over the blocks: forward y_{k} = AH_k y_{k-1} + z_k into ms[k + 1];
// backward y = GH_k y + gu_k into xn[k - 1] (xn[nb - 1] = 0)
template <int DP>
__device__ void cross(const Job& J, bool backward, float* vs, int lane) {
  constexpr int R = RPL<DP>::R;
  const int nb = J.nb;
  float y[R], in[R], nx[R];
  if (backward) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      y[r] = 0.f;
      if (lane + 32 * r < DP) J.xn[(long)(nb - 1) * DP + lane + 32 * r] = 0.f;
    }
    for (int kk = nb - 1; kk >= 1; --kk) {
      bput<DP>(vs, y, lane);
#pragma unroll
      for (int r = 0; r < R; ++r) in[r] = lane + 32 * r < DP ? ldcg(J.gu + (long)kk * DP + lane + 32 * r) : 0.f;
      bmv<DP>(J.GH + (long)kk * DP * DP, vs, lane, nx);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        y[r] = nx[r] + in[r];
        if (lane + 32 * r < DP) J.xn[(long)(kk - 1) * DP + lane + 32 * r] = y[r];
      }
    }
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      y[r] = lane + 32 * r < DP ? ldcg(J.z + lane + 32 * r) : 0.f;
      if (lane + 32 * r < DP && nb > 1) J.ms[(long)DP + lane + 32 * r] = y[r];
    }
    for (int kk = 1; kk <= nb - 2; ++kk) {
      bput<DP>(vs, y, lane);
#pragma unroll
      for (int r = 0; r < R; ++r) in[r] = lane + 32 * r < DP ? ldcg(J.z + (long)kk * DP + lane + 32 * r) : 0.f;
      bmv<DP>(J.AH + (long)kk * DP * DP, vs, lane, nx);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        y[r] = nx[r] + in[r];
        if (lane + 32 * r < DP) J.ms[(long)(kk + 1) * DP + lane + 32 * r] = y[r];
      }
    }
  }
}

// filtering means from the block's true start on ytilde (forward: with the
// backward elements and their block aggregate; reverse: the likelihood difference)
template <int DP>
__device__ void apply_block(const Job& J, int k, uint64_t iter, bool epi, const float* yin, float* vs, int lane) {
  constexpr int R = RPL<DP>::R;
  const int s = k * J.L, e = min(J.T, s + J.L) - 1, d = J.d;
  const long DD = (long)DP * DP;
  float phi[R], bb[R], mp[R], ubar[R];
  TermSum<float> qacc;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = lane + 32 * r;
    phi[r] = i < DP ? J.F[i * DP + i] : 0.f;
    bb[r] = i < DP ? J.b[i] : 0.f;
    ubar[r] = 0.f;
    mp[r] = 0.f;
    if (i < DP) mp[r] = (k == 0) ? J.m0[i] : fmaf(phi[r], ldcg(J.ms + (long)k * DP + i), bb[r]);
  }
  for (int t = s; t <= e; ++t) {
    float yti[R], ev[R], kv[R], m[R], mpn[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = lane + 32 * r;
      yti[r] = i < d ? ldcg(yin + (long)t * d + i) : 0.f;
      ev[r] = i < DP ? yti[r] - mp[r] : 0.f;
    }
    bput<DP>(vs, ev, lane);
    bmv<DP>(J.K + t * DD, vs, lane, kv);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      qacc.add_prod(ev[r], kv[r]);
      m[r] = yti[r] - kv[r];
      mpn[r] = (t < J.T - 1) ? fmaf(phi[r], m[r], bb[r]) : 0.f;
    }
    if (epi) {
      float ei[R], g1[R], g2[R], ui[R], gp[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = lane + 32 * r;
        ei[r] = i < d ? philox_normal<float>(J.seed, (uint32_t)J.c, iter, PURPOSE_BACKWARD, (uint32_t)t, i) : 0.f;
      }
      __syncwarp();
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (lane + 32 * r < DP) { vs[lane + 32 * r] = mpn[r]; vs[kMaxDP + lane + 32 * r] = ei[r]; }
      __syncwarp();
      bmv<DP>(J.G + t * DD, vs, lane, g1);
      bmv<DP>(J.LS + t * DD, vs + kMaxDP, lane, g2);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        ui[r] = m[r] - g1[r] + g2[r];
        if (lane + 32 * r < DP) J.U[(long)t * DP + lane + 32 * r] = ui[r];
      }
      bput<DP>(vs + 2 * kMaxDP, ui, lane);
      bmv<DP>(J.GP + t * DD, vs + 2 * kMaxDP, lane, gp);
#pragma unroll
      for (int r = 0; r < R; ++r) ubar[r] += gp[r];
    }
#pragma unroll
    for (int r = 0; r < R; ++r) mp[r] = mpn[r];
  }
  const double q = warp_sum<double>(qacc.value()) / (double)J.r;
  if (lane == 0) {
    if (epi) J.fq[k] = q;
    else J.lz[k] = -0.5 * (ldcg(J.fq + k) - q);
  }
  if (epi) {
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (lane + 32 * r < DP) J.gu[(long)k * DP + lane + 32 * r] = ubar[r];
  }
}

// backward sampling down block k with the MH terms, then the block's reverse
// filter from a zero start on ytilde*
template <int DP>
__device__ void back_block(const Job& J, int k, uint64_t iter, float* vs, int lane) {
  constexpr int R = RPL<DP>::R;
  const int s = k * J.L, e = min(J.T, s + J.L) - 1, d = J.d;
  const long DD = (long)DP * DP;
  float xi[R];
#pragma unroll
  for (int r = 0; r < R; ++r) xi[r] = lane + 32 * r < DP ? ldcg(J.xn + (long)k * DP + lane + 32 * r) : 0.f;
  TermSum<float> acc;
  for (int t = e; t >= s; --t) {
    float gx[R];
    bput<DP>(vs, xi, lane);
    bmv<DP>(J.G + t * DD, vs, lane, gx);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = lane + 32 * r;
      xi[r] = gx[r] + (i < DP ? ldcg(J.U + (long)t * DP + i) : 0.f);
    }
    const bool obs = !J.mask || J.mask[t];
    float vsi[R], yi[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = lane + 32 * r;
      yi[r] = i < d ? J.y[(long)t * d + i] : 0.f;
      vsi[r] = 0.f;
      if (i < d) J.xs[(long)t * d + i] = xi[r];
    }
    if (J.emis == AUX_EMIS_LINEAR_GAUSSIAN) {
      float dv[R];
#pragma unroll
      for (int r = 0; r < R; ++r) dv[r] = lane + 32 * r < d ? yi[r] - xi[r] : 0.f;
      bput<DP>(vs + kMaxDP, dv, lane);
      rmv<DP>(J.Ryinv, vs + kMaxDP, lane, vsi);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = lane + 32 * r;
      if (i >= d) continue;
      const long idx = (long)t * d + i;
      const float xo = J.x[idx], ui = ldcg(J.u + idx), vi = ldcg(J.v + idx), y = yi[r];
      float gdiff = 0.f, vs_i = vsi[r];
      if (obs) {
        if (J.emis == AUX_EMIS_SV) {
          vs_i = -0.5f + 0.5f * y * y * expf(-xi[r]);
          gdiff = -0.5f * (xi[r] - xo) - 0.5f * y * y * (expf(-xi[r]) - expf(-xo));
        } else {
          gdiff = -0.5f * (y - xi[r]) * vs_i + 0.5f * (y - xo) * vi;
        }
      } else {
        vs_i = 0.f;
      }
      const float fwd = vi * (ui - xi[r]) + 0.5f * J.r * vi * vi;
      const float rev = vs_i * (ui - xo) + 0.5f * J.r * vs_i * vs_i;
      acc.add(gdiff);
      acc.add(fwd);
      acc.add(-rev);
      J.yts[idx] = ui + J.r * vs_i;
    }
  }
  const double sum = warp_sum<double>(acc.value());
  if (lane == 0) J.mh[k] = sum;
  // the same lanes read back their own ytilde*_t
  reduce_block<DP>(J, k, iter, false, J.yts, vs, lane);
}

__device__ void mh_test(const Job& J, const Args& a, int jid, uint64_t iter, int lane) {
  double s = 0.0;
  for (int k = lane; k < J.nb; k += 32) s += ldcg(J.mh + k) + ldcg(J.lz + k);
  s = warp_sum<double>(s);
  if (lane == 0) {
    const double la = s;
    int st = *(volatile int32_t*)J.status_iter;
    if (!isfinite(la)) st |= ST_NONFINITE;
    const uint4 r = philox_word(J.seed, (uint32_t)J.c, iter, PURPOSE_MH, 0, 0);
    const double lu = log(u01<double>(r.x));
    const int acc = (st == 0) && (lu < la);
    *J.accept = acc;
    *J.status |= st;
    *J.la = la;
    if (a.log_alpha) a.log_alpha[jid] = la;
    if (a.acc_count && acc) a.acc_count[jid] += 1;
  }
}

__device__ void commit_block(const Job& J, int k, int lane) {
  if (!*(volatile int32_t*)J.accept) return;
  const int s = k * J.L, e = min(J.T, s + J.L) - 1;
  const long n0 = (long)s * J.d, n1 = (long)(e + 1) * J.d;
  for (long q = n0 + lane; q < n1; q += 32) J.x[q] = ldcg(J.xs + q);
}

template <int DP>
__device__ void run_item(const Job& J, const Args& a, int jid, int pass, int k, uint64_t iter, float* vs,
                         int lane) {
  switch (pass) {
    case FR: reduce_block<DP>(J, k, iter, true, nullptr, vs, lane); break;
    case FX: cross<DP>(J, false, vs, lane); break;
    case FA: apply_block<DP>(J, k, iter, true, J.yt, vs, lane); break;
    case BX: cross<DP>(J, true, vs, lane); break;
    case BR: back_block<DP>(J, k, iter, vs, lane); break;
    case RX: cross<DP>(J, false, vs, lane); break;
    case RA: apply_block<DP>(J, k, iter, false, J.yts, vs, lane); break;
    case MH: mh_test(J, a, jid, iter, lane); break;
    case CM: commit_block(J, k, lane); break;
    default: break;
  }
}

// the persistent launch: WPC warps per CTA, each taking items until the list is empty
template <int WPC>
__global__ void __launch_bounds__(32 * WPC) k_batch_step(Args a) {
  __shared__ __align__(16) float vslot[WPC][3 * kMaxDP];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* vs = vslot[warp];
  const uint64_t iter = *a.iter;
  for (;;) {
    unsigned idx = 0;
    if (lane == 0) idx = atomicAdd(a.head, 1u);
    idx = __shfl_sync(FULL, idx, 0);
    if (idx >= (unsigned)a.n_items) break;
    const int2 item = a.items[idx];
    const int jid = item.x, pass = item.y >> 16, k = item.y & 0xffff;
    const Job& J = a.jobs[jid];
    bool go;
    if (pass > 0) {
      const unsigned need = (pass & 1) ? (unsigned)J.nb : 1u;   // odd passes follow a block pass
      go = wait_count(a.cnt + (long)jid * NPASS + pass - 1, need, a.abort, lane);
    } else {
      go = !__any_sync(FULL, ld_volatile(a.abort) != 0);
    }
    if (!go) continue;
    switch (J.DP) {
      case 4: run_item<4>(J, a, jid, pass, k, iter, vs, lane); break;
      case 8: run_item<8>(J, a, jid, pass, k, iter, vs, lane); break;
      case 16: run_item<16>(J, a, jid, pass, k, iter, vs, lane); break;
      case 32: run_item<32>(J, a, jid, pass, k, iter, vs, lane); break;
      default: run_item<64>(J, a, jid, pass, k, iter, vs, lane); break;
    }
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicAdd(a.cnt + (long)jid * NPASS + pass, 1u);
  }
  // the last warp out resets the list for the next launch
  unsigned last = 0;
  __syncwarp();
  if (lane == 0) {
    __threadfence();
    last = atomicAdd(a.exited, 1u) == a.total_warps - 1;
  }
  last = __shfl_sync(FULL, last, 0);
  if (last) {
    __threadfence();
    for (long q = lane; q < (long)a.n_jobs * NPASS; q += 32) a.cnt[q] = 0u;
    if (lane == 0) { *a.head = 0u; *a.exited = 0u; }
    __threadfence();
  }
}

static __global__ void k_batch_iter_next(uint64_t* it) { *it += 1; }

// per-step tables of one model into the batch layout: K' (symmetric), G and
// chol(Sigma) (stored as matrices by the narrow kernels, transposed by the wide ones)
struct CopyDesc {
  const float* src;     // the model's [NTAB][T][DP * DP] tables
  float *K, *G, *LS;    // batch layout [T][DP * DP]
  int T, DP, transposed;
  long first;           // first element of this model in the launch's flat index
};

static __global__ void k_batch_copy(const CopyDesc* __restrict__ ds, int n, long total) {
  for (long g = (long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long)gridDim.x * blockDim.x) {
    int lo = 0, hi = n - 1;   // the model of element g
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (ds[mid].first <= g) lo = mid; else hi = mid - 1;
    }
    const CopyDesc& c = ds[lo];
    const long DD = (long)c.DP * c.DP, e = g - c.first;
    const int slot = (int)(e / ((long)c.T * DD));
    const long te = e % ((long)c.T * DD);
    const int t = (int)(te / DD), w = (int)(te % DD);
    // w indexes the destination: quad q of row i, element j = 4q + (w & 3)
    const int quad = w >> 2, i = quad % c.DP, j = (quad / c.DP) * 4 + (w & 3);
    const int which = slot == 0 ? TK : (slot == 1 ? TG : TLS);
    const float* src = c.src + ((long)which * c.T + t) * DD;
    const float val = (c.transposed && which != TK) ? src[(long)j * c.DP + i] : src[(long)i * c.DP + j];
    float* dst = slot == 0 ? c.K : (slot == 1 ? c.G : c.LS);
    dst[t * DD + w] = val;
  }
}

// block tables of one (model, block): GP_t, GH_k, AH_k in the batch layout.
// One CTA of kMaxDP threads (thread = row; rows >= DP idle), the running
// products and the step's matrix in shared memory.
struct BlockDesc {
  const float *K, *G, *F;   // batch layout tables, the model's padded F
  float *GP, *AH, *GH;
  int T, DP, L, nb;
  int first;                // first CTA of this model
};
constexpr int BLK_LD = kMaxDP + 1;
constexpr size_t BLK_SMEM = 3 * (size_t)kMaxDP * BLK_LD * sizeof(float);

template <int DP>
__device__ void block_tables(const BlockDesc& b, int k, float* sm) {
  float* sGP = sm;                       // G_s ... G_{t-1}
  float* sAH = sm + kMaxDP * BLK_LD;     // M_{t-1} ... M_s
  float* sM = sm + 2 * kMaxDP * BLK_LD;  // the step's G_t, then K'_t F
  const long DD = (long)DP * DP;
  const int i = threadIdx.x;
  const bool act = i < DP;
  const int s = k * b.L, e = min(b.T, s + b.L) - 1;
  auto bl = [](int ii, int jj) { return (((jj >> 2) * DP + ii) << 2) + (jj & 3); };
  if (act)
    for (int j = 0; j < DP; ++j) { sGP[i * BLK_LD + j] = (i == j) ? 1.f : 0.f; sAH[i * BLK_LD + j] = sGP[i * BLK_LD + j]; }
  float nw[DP];
  for (int t = s; t <= e; ++t) {
    __syncthreads();
    if (act)
      for (int j = 0; j < DP; ++j) {
        b.GP[t * DD + bl(i, j)] = sGP[i * BLK_LD + j];   // GP_t: the product before G_t
        sM[i * BLK_LD + j] = b.G[t * DD + bl(i, j)];
      }
    __syncthreads();
    // GP <- GP G_t (row i)
#pragma unroll
    for (int j = 0; j < DP; ++j) nw[j] = 0.f;
    if (act)
      for (int q = 0; q < DP; ++q) {
        const float g = sGP[i * BLK_LD + q];
#pragma unroll
        for (int j = 0; j < DP; ++j) nw[j] = fmaf(g, sM[q * BLK_LD + j], nw[j]);
      }
    __syncthreads();
    if (act)
      for (int j = 0; j < DP; ++j) {
        sGP[i * BLK_LD + j] = nw[j];
        sM[i * BLK_LD + j] = b.K[t * DD + bl(i, j)] * b.F[j * DP + j];   // row i of K'_t F
      }
    __syncthreads();
    // AH <- (K'_t F) AH (row i)
#pragma unroll
    for (int j = 0; j < DP; ++j) nw[j] = 0.f;
    if (act)
      for (int q = 0; q < DP; ++q) {
        const float kq = sM[i * BLK_LD + q];
#pragma unroll
        for (int j = 0; j < DP; ++j) nw[j] = fmaf(kq, sAH[q * BLK_LD + j], nw[j]);
      }
    __syncthreads();
    if (act)
      for (int j = 0; j < DP; ++j) sAH[i * BLK_LD + j] = nw[j];
  }
  __syncthreads();
  if (act)
    for (int j = 0; j < DP; ++j) {
      b.GH[k * DD + bl(i, j)] = sGP[i * BLK_LD + j];
      b.AH[k * DD + bl(i, j)] = sAH[i * BLK_LD + j];
    }
}

static __global__ void __launch_bounds__(kMaxDP) k_batch_blocks(const BlockDesc* __restrict__ ds, int n) {
  extern __shared__ __align__(16) float bsm[];
  int lo = 0, hi = n - 1;   // the model of this CTA
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ds[mid].first <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const BlockDesc& b = ds[lo];
  const int k = blockIdx.x - b.first;
  switch (b.DP) {
    case 4: block_tables<4>(b, k, bsm); break;
    case 8: block_tables<8>(b, k, bsm); break;
    case 16: block_tables<16>(b, k, bsm); break;
    case 32: block_tables<32>(b, k, bsm); break;
    default: block_tables<64>(b, k, bsm); break;
  }
}

}  // namespace batch
}  // namespace auxk

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
using auxk::batch::Job;
using auxk::batch::CopyDesc;
using auxk::batch::BlockDesc;
using auxk::batch::NPASS;

namespace {

constexpr int kStreams = 16;            // branches of the shared mode's covariance passes
constexpr double kLFactors[3] = {0.5, 1.0, 2.0};   // block length candidates, x sqrt(T)

int batch_L(int T, double f) { return std::max(2, std::min(T, (int)std::lround(f * std::sqrt((double)T)))); }

int dp_class(int DP) { return DP <= 8 ? 0 : (DP == 16 ? 1 : (DP == 32 ? 2 : 3)); }

}  // namespace

struct aux_batch {
  int device = 0, n_sm = 0;
  std::vector<aux_model*> models;
  std::vector<float*> x;
  std::vector<int> L, nb, job0;          // per model: block length, blocks, first job
  int n_jobs = 0;
  int shared = 0;                        // rerun every model's covariance pass each step
  // launch shape (aux_batch_set_config / the tuner)
  int wpc = 8, cps = 0, order = 0;
  double lf[4] = {1.0, 1.0, 1.0, 1.0};   // block length factor per width class (DP 4-8, 16, 32, 64)
  // device memory
  std::vector<void*> allocs;
  std::vector<float*> K, G, LS, GP, AH, GH;   // per model
  Job* d_jobs = nullptr;
  int2* d_items = nullptr;
  int n_items = 0, cap_items = 0;
  unsigned* d_cnt = nullptr;             // [jobs][NPASS], then head, exited
  int* d_abort = nullptr;
  uint64_t* d_iter = nullptr;
  CopyDesc* d_copy = nullptr;
  long copy_total = 0;
  BlockDesc* d_blocks = nullptr;
  int n_block_ctas = 0;
  std::vector<float*> zb;                // per job block vectors [4][nb_max][DP] and sums [3][nb_max]
  std::vector<double*> sb;
  std::vector<cudaStream_t> streams;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
};

namespace {

int balloc(aux_batch* b, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(p, bytes) != cudaSuccess) { *p = nullptr; return AUX_E_OOM; }
  b->allocs.push_back(*p);
  return AUX_OK;
}

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? AUX_OK : AUX_E_CUDA; }

// the largest number of blocks any block-length candidate gives a model
int nb_max(int T) {
  int m = 1;
  for (double f : kLFactors) m = std::max(m, (T + batch_L(T, f) - 1) / batch_L(T, f));
  return m;
}

// jobs and work list for the current block lengths (host copies uploaded to the device)
int build_lists(aux_batch* b, cudaStream_t st) {
  const int nm = (int)b->models.size();
  std::vector<Job> jobs;
  jobs.reserve(b->n_jobs);
  for (int i = 0; i < nm; ++i) {
    aux_model* m = b->models[i];
    b->L[i] = batch_L(m->T, b->lf[dp_class(m->DP)]);
    b->nb[i] = (m->T + b->L[i] - 1) / b->L[i];
    const int DP = m->DP, T = m->T, d = m->d, nbm = nb_max(T);
    for (int c = 0; c < m->C; ++c) {
      Job j{};
      j.d = d; j.DP = DP; j.T = T; j.L = b->L[i]; j.nb = b->nb[i]; j.emis = m->emis;
      j.y_per_chain = m->y_per_chain; j.c = c; j.seed = m->seed;
      j.r = (float)(0.5 * m->delta);
      j.sqrt_r = (float)std::sqrt(0.5 * m->delta);
      j.y = (const float*)m->y + (m->y_per_chain ? (long)c * T * d : 0);
      j.mask = m->mask;
      j.m0 = (const float*)m->m0; j.F = (const float*)m->F; j.b = (const float*)m->b;
      j.Ryinv = (const float*)m->Ryinv;
      j.cov_status = m->cov_status;
      j.K = b->K[i]; j.G = b->G[i]; j.LS = b->LS[i]; j.GP = b->GP[i]; j.AH = b->AH[i]; j.GH = b->GH[i];
      const long pc = (long)c * T * d;
      j.x = b->x[i] + pc;
      j.u = (float*)m->u + pc; j.v = (float*)m->v + pc; j.yt = (float*)m->yt + pc;
      j.yts = (float*)m->yts + pc; j.xs = (float*)m->xs + pc;
      j.U = (float*)m->U + (long)c * T * DP;
      float* zb = b->zb[b->job0[i] + c];
      j.z = zb; j.ms = zb + (long)nbm * DP; j.gu = zb + 2L * nbm * DP; j.xn = zb + 3L * nbm * DP;
      double* sb = b->sb[b->job0[i] + c];
      j.fq = sb; j.lz = sb + nbm; j.mh = sb + 2 * nbm;
      j.status_iter = m->status_iter + c; j.status = m->status + c; j.accept = m->accept + c;
      j.la = m->la_all + c;
      jobs.push_back(j);
    }
  }
  // items pass by pass; within a pass the jobs by T (descending: order 0, ascending: order 1)
  std::vector<int> perm(b->n_jobs);
  for (int j = 0; j < b->n_jobs; ++j) perm[j] = j;
  std::stable_sort(perm.begin(), perm.end(), [&](int p, int q) {
    return b->order == 0 ? jobs[p].T > jobs[q].T : jobs[p].T < jobs[q].T;
  });
  std::vector<int2> items;
  for (int pass = 0; pass < NPASS; ++pass)
    for (int j : perm) {
      const int n = (pass & 1) ? 1 : jobs[j].nb;
      for (int k = 0; k < n; ++k) items.push_back(make_int2(j, (pass << 16) | k));
    }
  b->n_items = (int)items.size();
  if (b->n_items > b->cap_items) return AUX_E_INVALID_ARG;
  cudaError_t e = cudaMemcpyAsync(b->d_jobs, jobs.data(), jobs.size() * sizeof(Job), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, st);
  // block tables of every (model, block)
  std::vector<BlockDesc> bd(nm);
  int first = 0;
  for (int i = 0; i < nm; ++i) {
    aux_model* m = b->models[i];
    bd[i] = BlockDesc{b->K[i], b->G[i], (const float*)m->F, b->GP[i], b->AH[i], b->GH[i],
                      m->T, m->DP, b->L[i], b->nb[i], first};
    first += b->nb[i];
  }
  b->n_block_ctas = first;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_blocks, bd.data(), bd.size() * sizeof(BlockDesc), cudaMemcpyHostToDevice, st);
  // host vectors must outlive the copies
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_rc(e);
}

void launch_blocks(aux_batch* b, cudaStream_t st) {
  auxk::batch::k_batch_blocks<<<b->n_block_ctas, auxk::batch::kMaxDP, auxk::batch::BLK_SMEM, st>>>(
      b->d_blocks, (int)b->models.size());
}

void launch_copy(aux_batch* b, cudaStream_t st) {
  const long n = b->copy_total;
  const int grid = (int)std::min<long>((n + 255) / 256, (long)b->n_sm * 16);
  auxk::batch::k_batch_copy<<<grid, 256, 0, st>>>(b->d_copy, (int)b->models.size(), n);
}

template <int WPC>
int launch_step_wpc(aux_batch* b, uint32_t* acc, double* la, cudaStream_t st) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, auxk::batch::k_batch_step<WPC>, 32 * WPC, 0) != cudaSuccess ||
      occ < 1)
    return AUX_E_CUDA;
  const int cps = b->cps > 0 ? std::min(b->cps, occ) : occ;
  const int grid = std::max(1, std::min(b->n_sm * cps, (b->n_items + WPC - 1) / WPC));
  auxk::batch::Args a{};
  a.jobs = b->d_jobs; a.items = b->d_items; a.n_items = b->n_items;
  a.cnt = b->d_cnt; a.n_jobs = b->n_jobs;
  a.head = b->d_cnt + (long)b->n_jobs * NPASS; a.exited = a.head + 1;
  a.total_warps = (unsigned)(grid * WPC);
  a.abort = b->d_abort; a.iter = b->d_iter; a.acc_count = acc; a.log_alpha = la;
  auxk::batch::k_batch_step<WPC><<<grid, 32 * WPC, 0, st>>>(a);
  return cuda_rc(cudaGetLastError());
}

int launch_step(aux_batch* b, uint32_t* acc, double* la, cudaStream_t st) {
  switch (b->wpc) {
    case 4: return launch_step_wpc<4>(b, acc, la, st);
    case 16: return launch_step_wpc<16>(b, acc, la, st);
    default: return launch_step_wpc<8>(b, acc, la, st);
  }
}

// every model's covariance pass, side by side on the batch's streams
int refresh_tables(aux_batch* b, cudaStream_t st) {
  int rc = cuda_rc(cudaEventRecord(b->fork, st));
  for (int s = 0; s < kStreams && !rc; ++s) rc = cuda_rc(cudaStreamWaitEvent(b->streams[s], b->fork, 0));
  for (size_t i = 0; i < b->models.size() && !rc; ++i) {
    aux_model* m = b->models[i];
    rc = m->ops->tables(m, 1, b->streams[i % kStreams]);
  }
  for (int s = 0; s < kStreams && !rc; ++s) {
    rc = cuda_rc(cudaEventRecord(b->join[s], b->streams[s]));
    if (!rc) rc = cuda_rc(cudaStreamWaitEvent(st, b->join[s], 0));
  }
  return rc;
}

}  // namespace

extern "C" {

int aux_batch_create(aux_model* const* models, void* const* x, int32_t n_models, uint64_t iteration,
                     void* stream, aux_batch** out) {
  if (!models || !x || !out || n_models < 1) return AUX_E_INVALID_ARG;
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  for (int i = 0; i < n_models; ++i) {
    aux_model* m = models[i];
    if (!m || !x[i]) return AUX_E_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (models[j] == m) return AUX_E_INVALID_ARG;
    if (m->fact || m->dtype != AUX_F32 || m->mode == AUX_MODE_PER_CHAIN || m->order != AUX_PROPOSAL_FIRST_ORDER ||
        m->sampler != AUX_SAMPLER_SCAN || m->tv || !m->fdiag || m->adapt ||
        (m->DP != 4 && m->DP != 8 && m->DP != 16 && m->DP != 32 && m->DP != 64) ||
        (m->emis != AUX_EMIS_SV && m->emis != AUX_EMIS_LINEAR_GAUSSIAN) || !m->ops->tables)
      return AUX_E_UNSUPPORTED;
  }
  aux_batch* b = new (std::nothrow) aux_batch();
  if (!b) return AUX_E_OOM;
  int rc = AUX_OK;
  cudaGetDevice(&b->device);
  if (cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) rc = AUX_E_CUDA;
  b->models.assign(models, models + n_models);
  for (int i = 0; i < n_models; ++i) b->x.push_back((float*)x[i]);
  b->L.assign(n_models, 0);
  b->nb.assign(n_models, 0);
  int cap = 0;
  std::vector<CopyDesc> cd;
  long total = 0;
  for (int i = 0; i < n_models && !rc; ++i) {
    aux_model* m = models[i];
    b->job0.push_back(b->n_jobs);
    b->n_jobs += m->C;
    const long DD = (long)m->DP * m->DP, T = m->T;
    const int nbm = nb_max(m->T);
    cap += m->C * (5 * nbm + 4);
    float* t = nullptr;
    rc = balloc(b, (void**)&t, (size_t)(4 * T + 2 * nbm) * DD * sizeof(float));
    if (rc) break;
    b->K.push_back(t); b->G.push_back(t + T * DD); b->LS.push_back(t + 2 * T * DD); b->GP.push_back(t + 3 * T * DD);
    b->AH.push_back(t + 4 * T * DD); b->GH.push_back(t + (4 * T + nbm) * DD);
    for (int c = 0; c < m->C && !rc; ++c) {
      float* z = nullptr;
      double* s = nullptr;
      rc = balloc(b, (void**)&z, (size_t)4 * nbm * m->DP * sizeof(float));
      if (!rc) rc = balloc(b, (void**)&s, (size_t)3 * nbm * sizeof(double));
      b->zb.push_back(z);
      b->sb.push_back(s);
    }
    cd.push_back(CopyDesc{(const float*)m->tab, b->K[i], b->G[i], b->LS[i], m->T, m->DP, m->DP > 32 ? 1 : 0, total});
    total += 3 * T * DD;
  }
  b->copy_total = total;
  b->cap_items = cap;
  if (!rc) rc = balloc(b, (void**)&b->d_jobs, (size_t)b->n_jobs * sizeof(Job));
  if (!rc) rc = balloc(b, (void**)&b->d_items, (size_t)cap * sizeof(int2));
  if (!rc) rc = balloc(b, (void**)&b->d_cnt, ((size_t)b->n_jobs * NPASS + 2) * sizeof(unsigned));
  if (!rc) rc = balloc(b, (void**)&b->d_abort, sizeof(int));
  if (!rc) rc = balloc(b, (void**)&b->d_iter, sizeof(uint64_t));
  if (!rc) rc = balloc(b, (void**)&b->d_copy, cd.size() * sizeof(CopyDesc));
  if (!rc) rc = balloc(b, (void**)&b->d_blocks, (size_t)n_models * sizeof(BlockDesc));
  if (!rc) rc = cuda_rc(cudaMemsetAsync(b->d_cnt, 0, ((size_t)b->n_jobs * NPASS + 2) * sizeof(unsigned), st));
  if (!rc) rc = cuda_rc(cudaMemsetAsync(b->d_abort, 0, sizeof(int), st));
  if (!rc) rc = cuda_rc(cudaMemcpyAsync(b->d_iter, &iteration, sizeof(uint64_t), cudaMemcpyHostToDevice, st));
  if (!rc) rc = cuda_rc(cudaMemcpyAsync(b->d_copy, cd.data(), cd.size() * sizeof(CopyDesc), cudaMemcpyHostToDevice, st));
  if (!rc) rc = cuda_rc(cudaFuncSetAttribute(auxk::batch::k_batch_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)auxk::batch::BLK_SMEM));
  for (int s = 0; s < kStreams && !rc; ++s) {
    cudaStream_t q = nullptr;
    rc = cuda_rc(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
    if (!rc) b->streams.push_back(q);
    cudaEvent_t ev = nullptr;
    if (!rc) rc = cuda_rc(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    if (!rc) b->join.push_back(ev);
  }
  if (!rc) rc = cuda_rc(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  // every model's tables (cached: computed once, kept while valid), then the batch's copies
  for (int i = 0; i < n_models && !rc; ++i) rc = models[i]->ops->tables(models[i], 0, st);
  if (!rc) rc = build_lists(b, st);
  if (!rc) { launch_copy(b, st); launch_blocks(b, st); rc = cuda_rc(cudaGetLastError()); }
  if (!rc) rc = cuda_rc(cudaStreamSynchronize(st));
  if (rc) { aux_batch_free(b); return rc; }
  *out = b;
  return AUX_OK;
}

void aux_batch_free(aux_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  for (void* p : b->allocs) cudaFree(p);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

int aux_batch_set_mode(aux_batch* b, int32_t mode) {
  if (!b || (mode != AUX_MODE_SHARED_COV && mode != AUX_MODE_CACHED_COV)) return AUX_E_INVALID_ARG;
  b->shared = mode == AUX_MODE_SHARED_COV;
  return AUX_OK;
}

int aux_batch_step(aux_batch* b, int32_t n_iters, uint32_t* accept_count, double* log_alpha, void* stream) {
  if (!b || n_iters < 0) return AUX_E_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = AUX_OK;
  for (int it = 0; it < n_iters && !rc; ++it) {
    if (b->shared) {
      rc = refresh_tables(b, st);
      if (!rc) { launch_copy(b, st); launch_blocks(b, st); }
    }
    if (!rc) rc = launch_step(b, accept_count, log_alpha, st);
    if (!rc) {
      auxk::batch::k_batch_iter_next<<<1, 1, 0, st>>>(b->d_iter);
      rc = cuda_rc(cudaGetLastError());
    }
  }
  return rc;
}

int aux_batch_set_config(aux_batch* b, int32_t warps_per_cta, int32_t ctas_per_sm, int32_t order,
                         const double* block_factor, void* stream) {
  if (!b || (warps_per_cta != 4 && warps_per_cta != 8 && warps_per_cta != 16) || ctas_per_sm < 0 ||
      (order != 0 && order != 1))
    return AUX_E_INVALID_ARG;
  if (block_factor)
    for (int c = 0; c < 4; ++c)
      if (!(block_factor[c] > 0.0) || block_factor[c] > 64.0) return AUX_E_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  b->wpc = warps_per_cta;
  b->cps = ctas_per_sm;
  b->order = order;
  if (block_factor)
    for (int c = 0; c < 4; ++c) b->lf[c] = block_factor[c];
  // snap the factors to the candidates the buffers are sized for
  for (int c = 0; c < 4; ++c) {
    double best = kLFactors[0];
    for (double f : kLFactors)
      if (std::fabs(std::log(f / b->lf[c])) < std::fabs(std::log(best / b->lf[c]))) best = f;
    b->lf[c] = best;
  }
  int rc = build_lists(b, st);
  if (!rc) { launch_blocks(b, st); rc = cuda_rc(cudaGetLastError()); }
  return rc;
}

int aux_batch_get_config(aux_batch* b, int32_t* warps_per_cta, int32_t* ctas_per_sm, int32_t* order,
                         double* block_factor, int32_t* block_len) {
  if (!b) return AUX_E_INVALID_ARG;
  if (warps_per_cta) *warps_per_cta = b->wpc;
  if (ctas_per_sm) *ctas_per_sm = b->cps;
  if (order) *order = b->order;
  if (block_factor)
    for (int c = 0; c < 4; ++c) block_factor[c] = b->lf[c];
  if (block_len)
    for (size_t i = 0; i < b->models.size(); ++i) block_len[i] = b->L[i];
  return AUX_OK;
}

int aux_batch_set_iteration(aux_batch* b, uint64_t iteration, void* stream) {
  if (!b) return AUX_E_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(b->d_iter, &iteration, sizeof(uint64_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_rc(e);
}

int aux_batch_get_iteration(aux_batch* b, uint64_t* iteration) {
  if (!b || !iteration) return AUX_E_INVALID_ARG;
  return cuda_rc(cudaMemcpy(iteration, b->d_iter, sizeof(uint64_t), cudaMemcpyDeviceToHost));
}

int aux_batch_get_status(aux_batch* b, int32_t* aborted) {
  if (!b) return AUX_E_INVALID_ARG;
  int ab = 0;
  if (cudaMemcpy(&ab, b->d_abort, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return AUX_E_CUDA;
  if (aborted) *aborted = ab;
  if (ab) return AUX_E_TIMEOUT;
  for (aux_model* m : b->models) {
    std::vector<int32_t> st(m->C);
    if (cudaMemcpy(st.data(), m->status, st.size() * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
      return AUX_E_CUDA;
    for (int32_t s : st)
      if (s & auxk::ST_NOT_PD) return AUX_E_NOT_PD;
    for (int32_t s : st)
      if (s) return AUX_E_NONFINITE;
  }
  return AUX_OK;
}

// Autotuner: times the persistent step over launch shapes and block lengths by
// coordinate descent (warps per CTA, CTAs per SM, item order, then the block
// length factor of each width class) and keeps the fastest. The chains' states
// and the iteration counter are restored afterwards; accept counts are not touched.
int aux_batch_tune(aux_batch* b, int32_t reps, void* stream, double* best_ms) {
  if (!b || reps < 1) return AUX_E_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return AUX_E_UNSUPPORTED;
  const int nm = (int)b->models.size();
  std::vector<size_t> xbytes(nm);
  size_t tot = 0;
  for (int i = 0; i < nm; ++i) {
    xbytes[i] = (size_t)b->models[i]->C * b->models[i]->T * b->models[i]->d * sizeof(float);
    tot += xbytes[i];
  }
  char* save = nullptr;
  if (cudaMalloc(&save, tot) != cudaSuccess) return AUX_E_OOM;
  uint64_t it0 = 0;
  int rc = aux_batch_get_iteration(b, &it0);
  size_t off = 0;
  for (int i = 0; i < nm && !rc; ++i) {
    rc = cuda_rc(cudaMemcpyAsync(save + off, b->x[i], xbytes[i], cudaMemcpyDeviceToDevice, st));
    off += xbytes[i];
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!rc) rc = cuda_rc(cudaEventCreate(&e0));
  if (!rc) rc = cuda_rc(cudaEventCreate(&e1));
  auto time_cfg = [&](double* ms) -> int {
    int r = aux_batch_step(b, 1, nullptr, nullptr, st);   // warm-up
    if (!r) r = cuda_rc(cudaEventRecord(e0, st));
    if (!r) r = aux_batch_step(b, reps, nullptr, nullptr, st);
    if (!r) r = cuda_rc(cudaEventRecord(e1, st));
    if (!r) r = cuda_rc(cudaEventSynchronize(e1));
    float f = 0.f;
    if (!r) r = cuda_rc(cudaEventElapsedTime(&f, e0, e1));
    *ms = (double)f / reps;
    return r;
  };
  struct Cfg { int wpc, cps, order; double lf[4]; };
  Cfg best{b->wpc, b->cps, b->order, {b->lf[0], b->lf[1], b->lf[2], b->lf[3]}};
  double best_t = 1e30;
  auto apply = [&](const Cfg& c) { return aux_batch_set_config(b, c.wpc, c.cps, c.order, c.lf, st); };
  auto trial = [&](const Cfg& c) -> int {
    int r = apply(c);
    double ms = 0.0;
    if (!r) r = time_cfg(&ms);
    if (!r && ms < best_t) { best_t = ms; best = c; }
    return r;
  };
  bool present[4] = {false, false, false, false};
  for (aux_model* m : b->models) present[dp_class(m->DP)] = true;
  if (!rc) rc = trial(best);
  for (int w : {4, 8, 16}) { Cfg c = best; c.wpc = w; if (!rc && w != best.wpc) rc = trial(c); }
  for (int cps : {1, 2}) { Cfg c = best; c.cps = cps; if (!rc && cps != best.cps) rc = trial(c); }
  { Cfg c = best; c.order = 1 - best.order; if (!rc) rc = trial(c); }
  for (int cls = 0; cls < 4; ++cls) {
    if (!present[cls]) continue;
    for (double f : kLFactors) { Cfg c = best; c.lf[cls] = f; if (!rc && f != best.lf[cls]) rc = trial(c); }
  }
  if (!rc) rc = apply(best);
  // restore the chains and the iteration
  off = 0;
  for (int i = 0; i < nm && !rc; ++i) {
    rc = cuda_rc(cudaMemcpyAsync(b->x[i], save + off, xbytes[i], cudaMemcpyDeviceToDevice, st));
    off += xbytes[i];
  }
  if (!rc) rc = aux_batch_set_iteration(b, it0, st);
  cudaStreamSynchronize(st);
  cudaFree(save);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (best_ms) *best_ms = best_t;
  return rc;
}

}  // extern "C"
