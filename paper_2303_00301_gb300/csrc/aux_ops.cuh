// aux_ops.cuh — host-side launch sequences for one precision and padded dimension.
#pragma once
#include <algorithm>
#include <cmath>
#include <vector>

#include "aux_bridge.cuh"
#include "aux_cov2.cuh"
#include "aux_grad.cuh"
#include "aux_means.cuh"
#include "aux_sqrt.cuh"

namespace auxk {
namespace {

__global__ void k_sum_parts(const double* __restrict__ part, int nb, double* __restrict__ out) {
  const int c = blockIdx.x;
  __shared__ double red[32];
  double s = 0.0;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) s += part[(long)c * nb + k];
  s = warp_sum<double>(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
    out[c] = t;
  }
}

inline int cuda_ok(cudaError_t e) { return e == cudaSuccess ? AUX_OK : AUX_E_CUDA; }

}  // namespace

template <typename Real>
KP<Real> make_kp(const aux_model* m) {
  KP<Real> p;
  p.C = m->C; p.nT = m->T; p.d = m->d; p.DP = m->DP; p.L = m->L; p.nb = m->nb;
  p.r = (Real)(0.5 * m->delta);
  p.sqrt_r = (Real)std::sqrt(0.5 * m->delta);
  p.emis = m->emis; p.y_per_chain = m->y_per_chain; p.seed = m->seed;
  p.fdiag = m->fdiag;
  p.F = (const Real*)m->F; p.Q = (const Real*)m->Q; p.P0 = (const Real*)m->P0;
  p.m0 = (const Real*)m->m0; p.b = (const Real*)m->b; p.Ryinv = (const Real*)m->Ryinv;
  p.y = (const Real*)m->y; p.mask = m->mask;
  p.status_iter = m->status_iter;
  p.order = m->order;
  p.rho = nullptr;
  p.delta_dev = m->adapt ? m->delta_dev : nullptr;
  p.iter_dev = nullptr;   // set by the MCMC step only (aux_set_device_iteration)
  p.tv = m->tv;
  p.Ftv = (const Real*)m->Ftv; p.FTtv = (const Real*)m->FTtv; p.Qtv = (const Real*)m->Qtv;
  p.btv = (const Real*)m->btv;
  return p;
}

// Launch with programmatic stream serialisation when the stream is not being
// captured: the kernel may then be scheduled while its predecessor in the
// stream runs, and waits for it in pdl_wait(). Under stream capture the launch
// is an ordinary one (measured: inside a CUDA graph the programmatic edges
// made the step slower, 0.569 -> 0.590 ms, while eager steps gained 5 %).
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = cs == cudaStreamCaptureStatusNone ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

template <typename Real, int DP>
struct Ops {
  using Z = Sizes<Real, DP>;

  static constexpr size_t kMaxSmemPerCta = 227 * 1024;   // opt-in dynamic shared memory of one CTA
  static int prepare() {
    cudaError_t e = cudaSuccess;
    e = cudaFuncSetAttribute(k_filter_reduce<Real, DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Z::RED_SMEM);
    if (e != cudaSuccess) return AUX_E_CUDA;
    e = cudaFuncSetAttribute(k_filter_scan_level<Real, DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Z::SCAN_SMEM);
    if (e != cudaSuccess) return AUX_E_CUDA;
    e = cudaFuncSetAttribute(k_filter_apply<Real, DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Z::APP_SMEM);
    if (e != cudaSuccess) return AUX_E_CUDA;
    e = cudaFuncSetAttribute(k_sample_backward<Real, DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Z::BWD_SMEM);
    if (e != cudaSuccess) return AUX_E_CUDA;
    // the gradient's smoother kernels need more than a CTA's 227 KB of shared
    // memory in FP64 at DP = 32; aux_loglik_grad refuses that case
    if constexpr (GradSizes<Real, DP>::RED_SMEM <= kMaxSmemPerCta && GradSizes<Real, DP>::APP_SMEM <= kMaxSmemPerCta) {
      e = cudaFuncSetAttribute(k_smooth_reduce<Real, DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GradSizes<Real, DP>::RED_SMEM);
      if (e != cudaSuccess) return AUX_E_CUDA;
      e = cudaFuncSetAttribute(k_smooth_apply<Real, DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GradSizes<Real, DP>::APP_SMEM);
      if (e != cudaSuccess) return AUX_E_CUDA;
    }
    e = cudaFuncSetAttribute(k_grad_final<Real, DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    if (e != cudaSuccess) return AUX_E_CUDA;
    e = cudaFuncSetAttribute(k_cov_gp_fix<Real, DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CovSizes<Real, DP>::FIX_SMEM);
    if (e != cudaSuccess) return AUX_E_CUDA;
    e = cudaFuncSetAttribute(k_c2_init<Real, DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cov2Sizes<Real, DP>::INIT_SMEM);
    if (e != cudaSuccess) return AUX_E_CUDA;
    e = cudaFuncSetAttribute(k_c2_level<Real, DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CovScanMW<Real, DP>::SMEM);
    if (e != cudaSuccess) return AUX_E_CUDA;
    e = cudaFuncSetAttribute(k_c2_tables<Real, DP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Tab2Layout<Real, DP>(false).bytes());
    if (e != cudaSuccess) return AUX_E_CUDA;
    e = cudaFuncSetAttribute(k_c2_products<Real, DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cov2Sizes<Real, DP>::PROD_SMEM);
    if (e != cudaSuccess) return AUX_E_CUDA;
    e = cudaFuncSetAttribute(k_mf_reduce<Real, DP, MEAN_CPW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MeanSizes<Real, DP>::RED);
    if (e != cudaSuccess) return AUX_E_CUDA;
    e = cudaFuncSetAttribute(k_mf_apply<Real, DP, MEAN_CPW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MeanSizes<Real, DP>::APP);
    if (e != cudaSuccess) return AUX_E_CUDA;
    e = cudaFuncSetAttribute(k_mb_apply<Real, DP, MEAN_CPW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MeanSizes<Real, DP>::BWD);
    if (e != cudaSuccess) return AUX_E_CUDA;
    e = cudaFuncSetAttribute(k_mean_cross<Real, DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MeanSizes<Real, DP>::CROSS);
    if (e != cudaSuccess) return AUX_E_CUDA;
    e = cudaFuncSetAttribute(k_mean_cross2<Real, DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cross2Sizes<Real, DP>::SMEM);
    if (e != cudaSuccess) return AUX_E_CUDA;
    e = cudaFuncSetAttribute(k_cov_xprod<Real, DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cross2Sizes<Real, DP>::XPROD_SMEM);
    if (e != cudaSuccess) return AUX_E_CUDA;
    e = cudaFuncSetAttribute(k_br_node<Real, DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BrSizes<Real, DP>::NODE_SMEM);
    if (e != cudaSuccess) return AUX_E_CUDA;
    e = cudaFuncSetAttribute(k_sr_reduce<Real, DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SrSizes<Real, DP>::RED_SMEM);
    if (e != cudaSuccess) return AUX_E_CUDA;
    e = cudaFuncSetAttribute(k_sr_scan_level<Real, DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SrSizes<Real, DP>::RED_SMEM);
    if (e != cudaSuccess) return AUX_E_CUDA;
    e = cudaFuncSetAttribute(k_sr_apply<Real, DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SrSizes<Real, DP>::APP_SMEM);
    if (e != cudaSuccess) return AUX_E_CUDA;
    e = cudaFuncSetAttribute(k_srcov_reduce<Real, DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SrSizes<Real, DP>::RED_SMEM);
    if (e != cudaSuccess) return AUX_E_CUDA;
    e = cudaFuncSetAttribute(k_srcov_scan_double<Real, DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SrSizes<Real, DP>::RED_SMEM);
    if (e != cudaSuccess) return AUX_E_CUDA;
    e = cudaFuncSetAttribute(k_srcov_apply<Real, DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SrSizes<Real, DP>::COVAPP_SMEM);
    return cuda_ok(e);
  }

  static int items(const aux_model* m) { return m->C * m->nb; }

  // MH test per chain, then x <- x* for the accepted chains
  static void mh_commit(aux_model* m, const KP<Real>& p, Real* x, uint64_t iter, uint32_t* acc,
                        double* log_alpha, cudaStream_t st) {
    ProfScope ps(m, PK_MH, st, 2 + (m->adapt ? 1 : 0) + (m->dev_iter ? 1 : 0));
    launch_pdl(k_mh<Real>, m->C, 128, 0, st, p, (const double*)m->mh_part, (const double*)m->lz_part, iter,
               acc, log_alpha, m->status, m->accept, m->la_all);
    const long n = (long)m->C * m->T * m->d;
    const int grid = (int)std::min<long>((n + 255) / 256, (long)m->n_sm * 8);
    launch_pdl(k_commit<Real>, grid, 256, 0, st, p, x, (const Real*)m->xs, (const int32_t*)m->accept);
    if (m->adapt)
      launch_pdl(k_adapt_delta, 1, 256, 0, st, (const double*)m->la_all, m->C, m->delta_dev, m->adapt_count,
                 m->adapt_target, m->adapt_gain);
    if (m->dev_iter) launch_pdl(k_iter_next, 1, 1, 0, st, m->iter_dev);
  }


  // parallel filter on yt: phase 1, Hillis-Steele rounds, phase 3
  // block aggregates and their scan: the inclusive block prefixes (marginals)
  static const Real* filter_prefix(aux_model* m, const KP<Real>& p, const Real* yt, cudaStream_t st) {
    const int n = items(m);
    Real* b0 = (Real*)m->agg0;
    Real* b1 = (Real*)m->agg1;
    { ProfScope ps(m, PK_REDUCE, st);
    k_filter_reduce<Real, DP><<<(n + Z::RED_WPC - 1) / Z::RED_WPC, 32 * Z::RED_WPC, Z::RED_SMEM, st>>>(
        p, yt, b0); }
    for (int off = 1; off < m->nb; off *= 2) {
      { ProfScope ps(m, PK_SCAN, st);
      k_filter_scan_level<Real, DP><<<(n + Z::SCAN_WPC - 1) / Z::SCAN_WPC, 32 * Z::SCAN_WPC, Z::SCAN_SMEM, st>>>(p, b0, b1, off); }
      Real* tmp = b0; b0 = b1; b1 = tmp;
    }
    return (m->nb > 1) ? b0 : nullptr;
  }

  // in-block filtering from the block prefixes over the blocks of a.rg
  static void filter_apply(aux_model* m, const KP<Real>& p, ApplyArgs<Real> a, cudaStream_t st) {
    const int n = m->C * (a.rg.k_cnt ? a.rg.k_cnt : m->nb);
    ProfScope ps(m, PK_APPLY, st);
    k_filter_apply<Real, DP><<<(n + Z::APP_WPC - 1) / Z::APP_WPC, 32 * Z::APP_WPC, Z::APP_SMEM, st>>>(p, a);
  }

  static void filter(aux_model* m, const KP<Real>& p, const Real* yt, ApplyArgs<Real> a,
                     cudaStream_t st) {
    a.prefix = filter_prefix(m, p, yt, st);
    a.yt = yt;
    filter_apply(m, p, a, st);
  }

  // square-root form of the per-chain filter (aux_sqrt.cuh): the same three phases
  static void sr_filter(aux_model* m, const KP<Real>& p, const Real* yt, ApplyArgs<Real> a,
                        cudaStream_t st) {
    using SZ = SrSizes<Real, DP>;
    const int n = items(m);
    Real* b0 = (Real*)m->agg0;
    Real* b1 = (Real*)m->agg1;
    { ProfScope ps(m, PK_REDUCE, st);
      k_sr_reduce<Real, DP><<<n, 32, SZ::RED_SMEM, st>>>(p, yt, b0); }
    for (int off = 1; off < m->nb; off *= 2) {
      { ProfScope ps(m, PK_SCAN, st);
        k_sr_scan_level<Real, DP><<<n, 32, SZ::RED_SMEM, st>>>(p, b0, b1, off); }
      Real* tmp = b0; b0 = b1; b1 = tmp;
    }
    a.yt = yt;
    a.prefix = (m->nb > 1) ? b0 : nullptr;
    ProfScope ps(m, PK_APPLY, st);
    k_sr_apply<Real, DP><<<n, 32, SZ::APP_SMEM, st>>>(p, a);
  }

  static ApplyArgs<Real> apply_args(aux_model* m, int flags, uint64_t iter) {
    ApplyArgs<Real> a{};
    a.flags = flags;
    a.G = (Real*)m->G; a.U = (Real*)m->U; a.gum = (Real*)m->gum; a.guv = (Real*)m->guv;
    a.fq = m->fq; a.fld = m->fld; a.lz_part = m->lz_part;
    a.mf = nullptr; a.Pf = nullptr; a.eps = nullptr;
    a.iter = iter;
    return a;
  }

  static void backward(aux_model* m, const KP<Real>& p, BackArgs<Real> b, cudaStream_t st) {
    const int n = items(m);
    ProfScope ps(m, PK_BACKWARD, st);
    k_sample_backward<Real, DP><<<(n + Z::BWD_WPC - 1) / Z::BWD_WPC, 32 * Z::BWD_WPC, Z::BWD_SMEM, st>>>(p, b);
  }

  // ---- covariance tables shared by all chains (AUX_MODE_SHARED_COV, AUX_MODE_CACHED_COV)
  using CZ = CovSizes<Real, DP>;
  static constexpr long DD = (long)DP * DP;

  // the two-level cross-block composition (k_mean_cross2) covers up to XG_MAX
  // groups of XGS maps; the backward direction has nb - 1 maps
  static bool cross2_ok(const aux_model* m) { return m->nb - 1 <= XG_MAX * XGS; }
  static int cross2_groups(const aux_model* m) { return std::max(1, (m->nb - 1 + XGS - 1) / XGS); }
  static void cross2_products(aux_model* m, const KP<Real>& p, cudaStream_t st) {
    if (!cross2_ok(m) || m->nb < 2) return;
    launch_pdl(k_cov_xprod<Real, DP>, 2 * cross2_groups(m), 32 * CW_SCAN, Cross2Sizes<Real, DP>::XPROD_SMEM, st,
               p, (Real*)m->btab);
  }

  // Covariance form: prefixes by doubling over the steps, then every step's
  // tables and the products of the means partition (aux_cov2.cuh).
  static void cov2_pass(aux_model* m, const KP<Real>& p, cudaStream_t st) {
    Cov2Args<Real> a{};
    a.tab = (Real*)m->tab; a.btab = (Real*)m->btab; a.ld = m->cov_ld; a.ldt = m->cov_ldt;
    a.pw = (Real*)m->cagg0;
    a.status = m->cov_status;
    using C2 = Cov2Sizes<Real, DP>;
    {
      ProfScope ps(m, PK_COV_REDUCE, st);
      cudaMemsetAsync(m->cov_status, 0, sizeof(int32_t), st);
      launch_pdl(k_c2_init<Real, DP>, 1, 64, C2::INIT_SMEM, st, p, a);
    }
    int lvl = 0;
    for (int pow2 = 1; pow2 < m->T; pow2 *= 2, ++lvl) {
      ProfScope ps(m, PK_COV_SCAN, st);
      const int cnt = std::min(pow2, m->T - pow2);
      const int sq = 2 * pow2 < m->T ? 1 : 0;
      const int fac = 4 * pow2 < m->T ? 1 : 0;   // the next level squares E^(2 pow2) again
      const Real* pin = a.pw + (lvl & 1) * 4 * DD;
      Real* pout = a.pw + ((lvl + 1) & 1) * 4 * DD;
      launch_pdl(k_c2_level<Real, DP>, cnt + sq, 32 * CW_SCAN, CovScanMW<Real, DP>::SMEM, st, p, a, pow2, cnt,
                 sq, fac, m->n_sm, pin, pout);
    }
    {
      ProfScope ps(m, PK_COV_APPLY, st);
      launch_pdl(k_c2_tables<Real, DP>, m->T, 64, Tab2Layout<Real, DP>(m->fdiag != 0).bytes(), st, p, a);
    }
    {
      ProfScope ps(m, PK_COV_PRODUCTS, st, (cross2_ok(m) && m->nb >= 2) ? 2 : 1);
      launch_pdl(k_c2_products<Real, DP>, 2 * m->nb, 32 * CW_SCAN, C2::PROD_SMEM, st, p, a);
      cross2_products(m, p, st);
    }
  }

  static void cov_pass(aux_model* m, const KP<Real>& p, cudaStream_t st) {
    m->br_valid = 0;
    if (!m->sqrt_form) {
      cov2_pass(m, p, st);
      return;
    }
    KP<Real> pc = p;   // the covariance scan runs on its own partition (block length Lc)
    pc.L = m->Lc;
    pc.nb = m->nbc;
    Real* b0 = (Real*)m->cagg0;
    Real* b1 = (Real*)m->cagg1;
    const int nbc = m->nbc;
    // square-root form (aux_sqrt.cuh): distinct block aggregates and doubling
    // on (A, U, Z) factors, for every padded width
    using SZ = SrSizes<Real, DP>;
    const bool rag = nbc >= 3 && (m->T % m->Lc) != 0;
    Real* Q0 = b1;
    Real* Q1 = b1 + 3 * DD;
    Real* tail = b1 + 6 * DD;
    {
      ProfScope ps(m, PK_COV_REDUCE, st);
      cudaMemsetAsync(m->cov_status, 0, sizeof(int32_t), st);
      k_srcov_reduce<Real, DP><<<nbc == 1 ? 1 : (rag ? 3 : 2), 32, SZ::RED_SMEM, st>>>(
          pc, b0, m->cov_status, (const int*)m->cov_kmap, Q0, tail);
    }
    const int n_end = rag ? nbc - 1 : nbc;
    Real *gk = Q0, *gk2 = Q1;
    for (int pow2 = 1; pow2 < n_end; pow2 *= 2) {
      ProfScope ps(m, PK_COV_SCAN, st);
      const int cnt = std::min(pow2, n_end - pow2);
      const int next = 2 * pow2 < n_end ? 1 : 0;
      k_srcov_scan_double<Real, DP><<<cnt + next, 32, SZ::RED_SMEM, st>>>(pc, b0, (const Real*)gk, gk2, 0, pow2,
                                                                          cnt, m->cov_status);
      Real* tmp = gk; gk = gk2; gk2 = tmp;
    }
    if (rag) {
      ProfScope ps(m, PK_COV_SCAN, st);
      k_srcov_scan_double<Real, DP><<<1, 32, SZ::RED_SMEM, st>>>(pc, b0, (const Real*)tail, (Real*)nullptr,
                                                                nbc - 2, nbc - 1, 1, m->cov_status);
    }
    CovArgs<Real> a{};
    a.prefix = (m->nbc > 1) ? b0 : nullptr;
    a.tab = (Real*)m->tab; a.btab = (Real*)m->btab; a.ld = m->cov_ld; a.ldt = m->cov_ldt;
    a.status = m->cov_status;
    a.cblk = b1;   // the scan buffer not holding the prefix
    a.R = m->L / m->Lc;
    {
      ProfScope ps(m, PK_COV_APPLY, st);
      k_srcov_apply<Real, DP><<<m->nbc, 32, SrSizes<Real, DP>::COVAPP_SMEM, st>>>(pc, a);
    }
    {
      ProfScope ps(m, PK_COV_PRODUCTS, st, (cross2_ok(m) && m->nb >= 2) ? 3 : 2);
      launch_pdl(k_cov_products<Real, DP>, m->nb, 32, CZ::PROD_SMEM, st, p, a, m->nbc);
      launch_pdl(k_cov_gp_fix<Real, DP>, (m->T + CZ::FIX_WPC - 1) / CZ::FIX_WPC, 32 * CZ::FIX_WPC, CZ::FIX_SMEM,
                 st, p, a, m->Lc, m->nbc);
      cross2_products(m, p, st);
    }
  }

  // the tables for this call: recomputed (shared mode) or reused while valid (cached mode)
  static void ensure_cov(aux_model* m, const KP<Real>& p, cudaStream_t st) {
    if (m->mode == AUX_MODE_CACHED_COV && m->cov_valid) return;
    cov_pass(m, p, st);
    m->cov_valid = 1;
  }

  static MeanArgs<Real> mean_args(aux_model* m) {
    MeanArgs<Real> a{};
    a.tab = (const Real*)m->tab; a.btab = (const Real*)m->btab; a.ld = m->cov_ld;
    a.cov_status = m->cov_status; a.z = (Real*)m->zb;
    a.U = (Real*)m->U; a.guv = (Real*)m->guv; a.fqb = m->fq; a.lz_part = m->lz_part;
    return a;
  }

  using MZ = MeanSizes<Real, DP>;
  static int mean_grid(const aux_model* m) { return m->nb * ((m->C + MEAN_CHAINS - 1) / MEAN_CHAINS); }
  static constexpr int MEAN_THREADS = 32 * MEAN_CHAINS / MEAN_CPW;

  // block-local pass, composition over the blocks, in-block pass from the true starts
  static void means_filter(aux_model* m, const KP<Real>& p, MeanArgs<Real> a, cudaStream_t st) {
    const int grid = mean_grid(m);
    { ProfScope ps(m, PK_REDUCE, st);
      launch_pdl(k_mf_reduce<Real, DP, MEAN_CPW>, grid, MEAN_THREADS, MZ::RED, st, p, a); }
    a.x = nullptr;
    { ProfScope ps(m, PK_SCAN, st);
      if (cross2_ok(m))
        launch_pdl(k_mean_cross2<Real, DP>, m->C, 32 * cross2_groups(m), Cross2Sizes<Real, DP>::SMEM, st,
                   p, (const Real*)m->btab, (const Real*)a.z, (Real*)m->ms, 0);
      else
        launch_pdl(k_mean_cross<Real, DP>, m->C, 32, MZ::CROSS, st,
                   p, (const Real*)m->btab + (long)BAH * m->nb * DD, a.z, (Real*)m->ms, 0); }
    a.mstart = (const Real*)m->ms;
    { ProfScope ps(m, PK_APPLY, st);
      launch_pdl(k_mf_apply<Real, DP, MEAN_CPW>, grid, MEAN_THREADS, MZ::APP, st, p, a); }
  }

  static BackArgs<Real> back_args_tab(aux_model* m) {
    BackArgs<Real> b{};
    b.G = (const Real*)m->tab + (long)TG * m->T * DD;
    b.U = (const Real*)m->U;
    b.gum = (const Real*)m->btab + (long)BGH * m->nb * DD;
    b.guv = (const Real*)m->guv;
    b.g_cs = 0; b.gm_cs = 0;
    return b;
  }

  // (G, U) suffix scan on the tables: composition over the blocks, then in-block
  static void backward_tab(aux_model* m, const KP<Real>& p, BackArgs<Real> b, cudaStream_t st) {
    ProfScope ps(m, PK_BACKWARD, st, 2);
    Real* xnext = (Real*)m->zb;
    if (cross2_ok(m))
      launch_pdl(k_mean_cross2<Real, DP>, m->C, 32 * cross2_groups(m), Cross2Sizes<Real, DP>::SMEM, st,
                 p, (const Real*)m->btab, b.guv, xnext, 1);
    else
      launch_pdl(k_mean_cross<Real, DP>, m->C, 32, MZ::CROSS, st, p, b.gum, b.guv, xnext, 1);
    launch_pdl(k_mb_apply<Real, DP, MEAN_CPW>, mean_grid(m), MEAN_THREADS, MZ::BWD, st, p, b,
               (const Real*)xnext);
  }

  // ---- divide-and-conquer (bridging) sampler (aux_bridge.cuh)
  using BZ = BrSizes<Real, DP>;

  // the levels j >= 1 of the dyadic tree over n = T - 1 intervals
  static std::vector<BrLevel> br_levels(const aux_model* m) {
    std::vector<BrLevel> lv;
    int prev_cnt = m->T - 1, prev_off = 0, off = 0;
    for (int j = 1; prev_cnt > 1; ++j) {
      const int cnt = (prev_cnt + 1) / 2;
      lv.push_back(BrLevel{j, off, cnt, prev_off, prev_cnt});
      prev_off = off;
      off += cnt;
      prev_cnt = cnt;
    }
    return lv;
  }

  // shared (table modes): leaves from the tables; per chain: leaves from the filter's G and Sigma
  static BrTree<Real> br_tree(aux_model* m, bool shared) {
    BrTree<Real> tr{};
    const long NN = std::max(m->br_NN, 1);
    Real* base = (Real*)(shared ? m->br_tree : m->br_ctree);
    const long cs = shared ? 0 : NN * DD;
    if (shared) {
      tr.G0 = (const Real*)m->tab + (long)TG * m->T * DD; tr.g0_cs = 0;
      tr.L0 = (const Real*)m->br_L0; tr.l0_cs = 0;
      tr.status = m->cov_status; tr.per_chain_status = 0;
    } else {
      tr.G0 = (const Real*)m->G; tr.g0_cs = (long)m->T * DD;
      tr.L0 = (const Real*)m->Sig; tr.l0_cs = (long)m->T * DD;
      tr.status = m->status_iter; tr.per_chain_status = 1;
    }
    const long nch = shared ? 1 : m->C;
    tr.E = base;
    tr.L = base + nch * NN * DD;
    tr.B = base + 2 * nch * NN * DD;
    tr.nn_cs = cs;
    return tr;
  }

  static void br_build(aux_model* m, const KP<Real>& p, const BrTree<Real>& tr, bool shared, cudaStream_t st) {
    const int n = m->T - 1;
    const std::vector<BrLevel> lv = br_levels(m);
    if (shared && n >= 1) {
      ProfScope ps(m, PK_BR_TREE, st);
      k_br_leaf<Real, DP><<<(n + 7) / 8, 256, 0, st>>>((const Real*)m->tab + (long)TLS * m->T * DD,
                                                       (Real*)m->br_L0, n);
    }
    const int nch = shared ? 1 : m->C;
    for (const BrLevel& l : lv) {
      ProfScope ps(m, PK_BR_TREE, st);
      k_br_node<Real, DP><<<nch * l.cnt, 32, BZ::NODE_SMEM, st>>>(p, tr, l);
    }
  }

  // the table modes' tree follows the covariance tables
  static void br_ensure_shared(aux_model* m, const KP<Real>& p, cudaStream_t st) {
    if (m->br_valid) return;
    br_build(m, p, br_tree(m, true), true, st);
    m->br_valid = 1;
  }

  // node offsets up the tree, the two ends, the split points down the tree:
  // one cluster per chain (k_b_sample)
  static void br_sample(aux_model* m, const KP<Real>& p, const BrTree<Real>& tr, BrMeans<Real> mv,
                        cudaStream_t st) {
    const std::vector<BrLevel> lv = br_levels(m);
    mv.gN = (Real*)m->br_g;
    mv.NN = std::max(m->br_NN, 1);
    BrLevels L{};
    L.n = (int)lv.size();
    for (int i = 0; i < L.n && i < BR_MAX_LEVELS; ++i) L.l[i] = lv[i];
    const int rj = lv.empty() ? 0 : lv.back().j, ro = lv.empty() ? 0 : lv.back().off;
    ProfScope ps(m, PK_BRIDGE, st);
    k_b_sample<Real, DP><<<m->C * BR_CLUSTER, 32 * BR_WARPS, BZ::SAMPLE_SMEM, st>>>(p, tr, mv, L, rj, ro);
  }

  static void br_mh_terms(aux_model* m, const KP<Real>& p, const BackArgs<Real>& b, cudaStream_t st) {
    ProfScope ps(m, PK_BRIDGE, st);
    const long items = (long)m->C * m->nb;
    const size_t sm = (size_t)(Lay<Real, DP>::MAT + BZ::WPC * BZ::VEC) * sizeof(Real);
    k_b_mh<Real, DP><<<(int)((items + BZ::WPC - 1) / BZ::WPC), 32 * BZ::WPC, sm, st>>>(p, b);
  }

  static BrMeans<Real> br_means_tab(aux_model* m, Real* xs, const Real* eps, uint64_t iter) {
    BrMeans<Real> mv{};
    mv.U = (const Real*)m->U;
    mv.PT = (const Real*)m->tab + (long)TPF * m->T * DD + (long)(m->T - 1) * DD;
    mv.pt_cs = 0;
    mv.xs = xs; mv.eps = eps; mv.iter = iter;
    return mv;
  }

  static BrMeans<Real> br_means_chain(aux_model* m, Real* xs, const Real* eps, uint64_t iter) {
    BrMeans<Real> mv{};
    mv.U = (const Real*)m->U;
    mv.PT = (const Real*)m->Sig + (long)(m->T - 1) * DD;
    mv.pt_cs = (long)m->T * DD;
    mv.xs = xs; mv.eps = eps; mv.iter = iter;
    return mv;
  }

  static int kalman_step_means(aux_model* m, void* xv, int n_iters, uint64_t iter0, uint32_t* acc,
                               double* log_alpha, cudaStream_t st) {
    KP<Real> p = make_kp<Real>(m);
    if (m->dev_iter) p.iter_dev = m->iter_dev;
    Real* x = (Real*)xv;
    for (int it = 0; it < n_iters; ++it) {
      const uint64_t iter = iter0 + (uint64_t)it;
      // an adapted delta changes the covariances every iteration
      if (m->adapt) cov_pass(m, p, st);
      else if (it == 0) ensure_cov(m, p, st);
      const bool br = m->sampler == AUX_SAMPLER_BRIDGING;
      if (br) br_ensure_shared(m, p, st);
      MeanArgs<Real> a = mean_args(m);
      a.x = x; a.u = (Real*)m->u; a.v = (Real*)m->v; a.yt = (Real*)m->yt; a.iter = iter;
      a.flags = APPLY_EPI | APPLY_STORE_Q | (br ? APPLY_SMOOTH : 0);
      means_filter(m, p, a, st);
      BackArgs<Real> b = back_args_tab(m);
      b.xs = (Real*)m->xs; b.mh = 1; b.x = x; b.u = (const Real*)m->u; b.v = (const Real*)m->v;
      b.yts = (Real*)m->yts; b.mh_part = m->mh_part;
      if (br) {
        br_sample(m, p, br_tree(m, true), br_means_tab(m, (Real*)m->xs, nullptr, iter), st);
        br_mh_terms(m, p, b, st);
      } else {
        backward_tab(m, p, b, st);
      }
      MeanArgs<Real> r = mean_args(m);
      r.yt = (Real*)m->yts; r.flags = APPLY_REV_DIFF;
      means_filter(m, p, r, st);
      mh_commit(m, p, x, iter, acc, log_alpha, st);
    }
    return cuda_ok(cudaGetLastError());
  }

  static int kalman_step(aux_model* m, void* xv, int n_iters, uint64_t iter0, uint32_t* acc,
                         double* log_alpha, cudaStream_t st) {
    if (m->sqrt_form && m->mode == AUX_MODE_PER_CHAIN && (m->order != 1 || m->sampler != AUX_SAMPLER_SCAN))
      return AUX_E_UNSUPPORTED;
    if (m->mode != AUX_MODE_PER_CHAIN) {
      // the tables assume R = (delta/2) I; the second-order variances depend on the chain's state
      if (m->order != 1) return AUX_E_UNSUPPORTED;
      return kalman_step_means(m, xv, n_iters, iter0, acc, log_alpha, st);
    }
    KP<Real> p = make_kp<Real>(m);
    if (m->dev_iter) p.iter_dev = m->iter_dev;
    const bool second = m->order == 2;
    KP<Real> pf = p, pr = p;   // forward and reverse filters: the pseudo-observation variances
    if (second) { pf.rho = (const Real*)m->rho; pr.rho = (const Real*)m->rhos; }
    Real* x = (Real*)xv;
    const long n = (long)m->C * m->T * m->d;
    const int lin_grid = (int)std::min<long>((n + 255) / 256, (long)m->n_sm * 16);
    for (int it = 0; it < n_iters; ++it) {
      const uint64_t iter = iter0 + (uint64_t)it;
      { ProfScope ps(m, PK_LINEARISE, st);
      k_linearise<Real><<<lin_grid, 256, 0, st>>>(p, x, (Real*)m->u, (Real*)m->v, (Real*)m->yt,
                                                  (Real*)m->rho, iter); }
      const bool br = m->sampler == AUX_SAMPLER_BRIDGING;
      ApplyArgs<Real> fa = apply_args(m, APPLY_EPI | APPLY_STORE_Q | (br ? APPLY_SMOOTH : 0), iter);
      fa.Sig = (Real*)m->Sig;
      if (m->sqrt_form) sr_filter(m, pf, (const Real*)m->yt, fa, st);
      else filter(m, pf, (const Real*)m->yt, fa, st);
      BackArgs<Real> b{};
      b.G = (const Real*)m->G; b.U = (const Real*)m->U; b.gum = (const Real*)m->gum;
      b.guv = (const Real*)m->guv; b.g_cs = (long)m->T * DP * DP; b.gm_cs = (long)m->nb * DP * DP;
      b.xs = (Real*)m->xs; b.mh = 1; b.x = x; b.u = (const Real*)m->u; b.v = (const Real*)m->v;
      b.yts = (Real*)m->yts; b.mh_part = m->mh_part;
      b.yt = (const Real*)m->yt; b.rho = (const Real*)m->rho; b.rhos = (Real*)m->rhos;
      if (br) {
        const BrTree<Real> tr = br_tree(m, false);
        br_build(m, pf, tr, false, st);
        br_sample(m, p, tr, br_means_chain(m, (Real*)m->xs, nullptr, iter), st);
        br_mh_terms(m, p, b, st);
      } else {
        backward(m, p, b, st);
      }
      if (m->sqrt_form) sr_filter(m, pr, (const Real*)m->yts, apply_args(m, APPLY_REV_DIFF, iter), st);
      else filter(m, pr, (const Real*)m->yts, apply_args(m, APPLY_REV_DIFF, iter), st);
      mh_commit(m, p, x, iter, acc, log_alpha, st);
    }
    return cuda_ok(cudaGetLastError());
  }

  static int loglik(aux_model* m, const void* yt, double* logZ, void* mf, void* Pf, cudaStream_t st) {
    const KP<Real> p = make_kp<Real>(m);
    if (m->mode != AUX_MODE_PER_CHAIN) {
      ensure_cov(m, p, st);
      MeanArgs<Real> a = mean_args(m);
      a.yt = (Real*)yt; a.flags = APPLY_LOGZ; a.mf = (Real*)mf; a.Pf = (Real*)Pf; a.status = m->status;
      means_filter(m, p, a, st);
      { ProfScope ps(m, PK_SUM, st); k_sum_parts<<<m->C, 128, 0, st>>>(m->lz_part, m->nb, logZ); }
      return cuda_ok(cudaGetLastError());
    }
    ApplyArgs<Real> a = apply_args(m, APPLY_LOGZ, 0);
    a.mf = (Real*)mf;
    a.Pf = (Real*)Pf;
    if (m->sqrt_form) sr_filter(m, p, (const Real*)yt, a, st);
    else filter(m, p, (const Real*)yt, a, st);
    { ProfScope ps(m, PK_SUM, st);
    k_sum_parts<<<m->C, 128, 0, st>>>(m->lz_part, m->nb, logZ); }
    return cuda_ok(cudaGetLastError());
  }

  static int sample_path(aux_model* m, const void* yt, const void* eps, uint64_t iter, void* xs,
                         double* logZ, cudaStream_t st) {
    if (m->sqrt_form && m->mode == AUX_MODE_PER_CHAIN && m->sampler != AUX_SAMPLER_SCAN)
      return AUX_E_UNSUPPORTED;
    const KP<Real> p = make_kp<Real>(m);
    if (m->mode != AUX_MODE_PER_CHAIN) {
      ensure_cov(m, p, st);
      const bool br = m->sampler == AUX_SAMPLER_BRIDGING;
      if (br) br_ensure_shared(m, p, st);
      MeanArgs<Real> a = mean_args(m);
      a.yt = (Real*)yt; a.flags = APPLY_EPI | APPLY_LOGZ | (br ? APPLY_SMOOTH : 0);
      a.eps = (const Real*)eps; a.iter = iter;
      a.status = m->status;
      means_filter(m, p, a, st);
      if (br) {
        br_sample(m, p, br_tree(m, true), br_means_tab(m, (Real*)xs, (const Real*)eps, iter), st);
      } else {
        BackArgs<Real> b = back_args_tab(m);
        b.xs = (Real*)xs; b.mh = 0;
        backward_tab(m, p, b, st);
      }
      if (logZ) { ProfScope ps(m, PK_SUM, st); k_sum_parts<<<m->C, 128, 0, st>>>(m->lz_part, m->nb, logZ); }
      return cuda_ok(cudaGetLastError());
    }
    const bool br = m->sampler == AUX_SAMPLER_BRIDGING;
    ApplyArgs<Real> a = apply_args(m, APPLY_EPI | APPLY_LOGZ | (br ? APPLY_SMOOTH : 0), iter);
    a.eps = (const Real*)eps;
    a.Sig = (Real*)m->Sig;
    if (m->sqrt_form) sr_filter(m, p, (const Real*)yt, a, st);
    else filter(m, p, (const Real*)yt, a, st);
    if (br) {
      const BrTree<Real> tr = br_tree(m, false);
      br_build(m, p, tr, false, st);
      br_sample(m, p, tr, br_means_chain(m, (Real*)xs, (const Real*)eps, iter), st);
      if (logZ) { ProfScope ps(m, PK_SUM, st); k_sum_parts<<<m->C, 128, 0, st>>>(m->lz_part, m->nb, logZ); }
      return cuda_ok(cudaGetLastError());
    }
    BackArgs<Real> b{};
    b.G = (const Real*)m->G; b.U = (const Real*)m->U; b.gum = (const Real*)m->gum;
    b.guv = (const Real*)m->guv; b.g_cs = (long)m->T * DP * DP; b.gm_cs = (long)m->nb * DP * DP;
    b.xs = (Real*)xs; b.mh = 0;
    backward(m, p, b, st);
    if (logZ) { ProfScope ps(m, PK_SUM, st); k_sum_parts<<<m->C, 128, 0, st>>>(m->lz_part, m->nb, logZ); }
    return cuda_ok(cudaGetLastError());
  }

  // gradient of log Z w.r.t. (mu, phi, L, delta): forward filter storing the
  // noise-free backward elements and Sigma_t, smoother aggregates, smoother
  // sweep with the score statistics, FP64 reduction per chain
  static int loglik_grad(aux_model* m, const void* yt, double* logZ, double* g_mu, double* g_phi,
                         double* g_L, double* g_delta, cudaStream_t st) {
    using GZ = GradSizes<Real, DP>;
    KP<Real> p = make_kp<Real>(m);
    p.delta_dev = nullptr;   // the gradient is taken at the description's delta (a theta component)
    ApplyArgs<Real> a = apply_args(m, APPLY_EPI | APPLY_LOGZ | APPLY_SMOOTH, 0);
    a.Sig = (Real*)m->Sig;
    a.yt = (const Real*)yt;
    a.prefix = filter_prefix(m, p, (const Real*)yt, st);
    SmoothArgs<Real> sa{};
    sa.yt = (const Real*)yt; sa.sgu = (Real*)m->sgu; sa.gpart = (Real*)m->gpart;
    sa.opart = m->opart; sa.s0 = (Real*)m->s0;
    auto smooth = [&](bool reduce, const BlockRange& rg) {
      const int n = m->C * (rg.k_cnt ? rg.k_cnt : m->nb);
      sa.rg = rg;
      ProfScope ps(m, PK_SMOOTH, st);
      if (reduce)
        k_smooth_reduce<Real, DP><<<(n + GZ::WPC - 1) / GZ::WPC, 32 * GZ::WPC, GZ::RED_SMEM, st>>>(p, sa);
      else
        k_smooth_apply<Real, DP><<<(n + GZ::WPC - 1) / GZ::WPC, 32 * GZ::WPC, GZ::APP_SMEM, st>>>(p, sa);
    };
    if (!m->grad_kc) {   // G_t, Sigma_t, U_t of every step stored
      filter_apply(m, p, a, st);
      sa.G = (const Real*)m->G; sa.U = (const Real*)m->U; sa.Sig = (const Real*)m->Sig;
      smooth(true, BlockRange{});
      smooth(false, BlockRange{});
    } else {
      // recompute-not-store: chunks of grad_kc blocks; the in-block filter runs
      // once for the smoother's block aggregates and again for its sweep, each
      // time into the chunk's scratch (the aggregates of all blocks are small)
      const long cs = (long)m->grad_kc * m->L, nst = (long)m->C * cs;
      a.G = (Real*)m->gscr;
      a.Sig = a.G + nst * DD;
      a.U = a.Sig + nst * DD;
      sa.G = a.G; sa.Sig = a.Sig; sa.U = a.U;
      for (int pass = 0; pass < 2; ++pass)
        for (int k0 = 0; k0 < m->nb; k0 += m->grad_kc) {
          BlockRange rg;
          rg.k_lo = k0;
          rg.k_cnt = std::min(m->grad_kc, m->nb - k0);
          rg.t_lo = (long)k0 * m->L;
          rg.cs = cs;
          a.rg = rg;
          filter_apply(m, p, a, st);
          smooth(pass == 0, rg);
        }
    }
    if (logZ) { ProfScope ps(m, PK_SUM, st); k_sum_parts<<<m->C, 128, 0, st>>>(m->lz_part, m->nb, logZ); }
    GradOut go{g_mu, g_phi, g_L, g_delta};
    const size_t fsm = (size_t)(5 * m->d * m->d + 2 * m->d + 32) * sizeof(double);
    {
      ProfScope ps(m, PK_GRAD, st);
      k_grad_final<Real, DP><<<m->C, 256, fsm, st>>>(p, (const Real*)m->gpart, m->opart,
                                                     (const Real*)m->s0, m->gconst, m->delta, go);
    }
    return cuda_ok(cudaGetLastError());
  }

  static int tables(aux_model* m, int force, cudaStream_t st) {
    if (m->mode == AUX_MODE_PER_CHAIN) return AUX_E_UNSUPPORTED;
    const KP<Real> p = make_kp<Real>(m);
    if (force || !m->cov_valid) { cov_pass(m, p, st); m->cov_valid = 1; }
    return cuda_ok(cudaGetLastError());
  }

  static const AuxOps* table() {
    static const AuxOps t = {&prepare, &kalman_step, &loglik, &sample_path, &loglik_grad, &tables};
    return &t;
  }
};

}  // namespace auxk
