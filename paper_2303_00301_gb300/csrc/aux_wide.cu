// Host-side launch sequences of the table modes for padded dimensions 64 and
// 128 (aux_wide.cuh), single precision. The per-chain element scan, the
// second-order proposal, the square-root form, the bridging sampler and the
// gradient are not offered at these widths (AUX_E_UNSUPPORTED).
#include "aux_ops.cuh"
#include "aux_wide.cuh"

namespace auxk {

// MX: the mixed-precision form (AUX_MIXED): the covariance pass's products on
// the tensor cores in split TF32 with FP32 accumulation, the factorisations of
// C_i and N = I + U^T J_e U in the doubling in FP64; the means are unchanged.
template <typename Real, int DP, bool MX>
struct WOps {
  using Z = WSz<Real, DP>;
  static constexpr long DD = Z::DD;

  static int prepare() {
    cudaError_t e = cudaSuccess;
#define AUX_W_ATTR(K, S)                                                             \
    if ((e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(S))) != cudaSuccess) \
      return AUX_E_CUDA;
    AUX_W_ATTR((k_w_elem<Real, DP, MX>), Z::SMEM)
    AUX_W_ATTR((k_w_double<Real, DP, MX>), MX ? Z::SMEM_MX : Z::SMEM)
    AUX_W_ATTR((k_w_epi<Real, DP, MX>), Z::SMEM)
    AUX_W_ATTR((k_w_prod<Real, DP, MX>), Z::SMEM)
    AUX_W_ATTR((k_wmf_reduce<Real, DP>), Z::MSMEM)
    AUX_W_ATTR((k_wmf_apply<Real, DP>), Z::MSMEM)
    AUX_W_ATTR((k_wmb_apply<Real, DP>), Z::MSMEM)
    AUX_W_ATTR((k_wmean_cross<Real, DP>), Z::XSMEM)
#undef AUX_W_ATTR
    return AUX_OK;
  }

  static WCovArgs<Real> cov_args(aux_model* m) {
    WCovArgs<Real> a{};
    a.tab = (Real*)m->tab; a.btab = (Real*)m->btab; a.ldt = m->cov_ldt; a.ld = m->cov_ld;
    a.status = m->cov_status; a.gk = (Real*)m->cagg0; a.scr = (Real*)m->cagg1;
    return a;
  }

  // the two distinct elements, the prefixes by doubling, the per-step tables, the block products
  static void cov_pass(aux_model* m, const KP<Real>& p, cudaStream_t st) {
    WCovArgs<Real> a = cov_args(m);
    {
      ProfScope ps(m, PK_COV_REDUCE, st);
      cudaMemsetAsync(m->cov_status, 0, sizeof(int32_t), st);
      k_w_elem<Real, DP, MX><<<1, WT, Z::SMEM, st>>>(p, a);
    }
    Real* gk = a.gk;
    Real* gk2 = a.gk + 3 * DD;
    for (int pow2 = 1; pow2 < m->T; pow2 *= 2) {
      ProfScope ps(m, PK_COV_SCAN, st);
      const int cnt = std::min(pow2, m->T - pow2);
      const int sq = 2 * pow2 < m->T ? 1 : 0;
      k_w_double<Real, DP, MX><<<std::min(cnt + sq, W_SLOTS_PER_SM * m->n_sm), WT, MX ? Z::SMEM_MX : Z::SMEM, st>>>(
          p, a, pow2, cnt, sq, gk, gk2);
      std::swap(gk, gk2);
    }
    {
      ProfScope ps(m, PK_COV_APPLY, st);
      k_w_epi<Real, DP, MX><<<std::min(m->T + 1, W_SLOTS_PER_SM * m->n_sm), WT, Z::SMEM, st>>>(p, a);
    }
    {
      ProfScope ps(m, PK_COV_PRODUCTS, st);
      k_w_prod<Real, DP, MX><<<std::min(m->nb, W_SLOTS_PER_SM * m->n_sm), WT, Z::SMEM, st>>>(p, a);
    }
  }

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

  // row groups of a means CTA: as many as the chains need (one chain per instance uses one)
  static int mean_threads(const aux_model* m) {
    const int groups = (m->C + WCPT<DP> - 1) / WCPT<DP>;
    return DP * std::min(Z::NRG, groups);
  }
  static int mean_grid(const aux_model* m) {
    const int cpc = mean_threads(m) / DP * WCPT<DP>;
    return m->nb * ((m->C + cpc - 1) / cpc);
  }

  static void means_filter(aux_model* m, const KP<Real>& p, MeanArgs<Real> a, cudaStream_t st) {
    const int grid = mean_grid(m);
    { ProfScope ps(m, PK_REDUCE, st);
      k_wmf_reduce<Real, DP><<<grid, mean_threads(m), Z::MSMEM, st>>>(p, a); }
    a.x = nullptr;
    { ProfScope ps(m, PK_SCAN, st);
      k_wmean_cross<Real, DP><<<m->C, DP, Z::XSMEM, st>>>(p, (const Real*)m->btab, a.z, (Real*)m->ms, 0); }
    a.mstart = (const Real*)m->ms;
    { ProfScope ps(m, PK_APPLY, st);
      k_wmf_apply<Real, DP><<<grid, mean_threads(m), Z::MSMEM, st>>>(p, a); }
  }

  static BackArgs<Real> back_args(aux_model* m) {
    BackArgs<Real> b{};
    b.G = (const Real*)m->tab + (long)TG * m->T * DD;   // G^T per step
    b.U = (const Real*)m->U;
    b.gum = (const Real*)m->btab + (long)m->nb * DD;   // (G_s ... G_e)^T per block
    b.guv = (const Real*)m->guv;
    return b;
  }

  static void backward(aux_model* m, const KP<Real>& p, BackArgs<Real> b, cudaStream_t st) {
    ProfScope ps(m, PK_BACKWARD, st, 2);
    Real* xnext = (Real*)m->zb;
    k_wmean_cross<Real, DP><<<m->C, DP, Z::XSMEM, st>>>(p, b.gum, b.guv, xnext, 1);
    k_wmb_apply<Real, DP><<<mean_grid(m), mean_threads(m), Z::MSMEM, st>>>(p, b, (const Real*)xnext);
  }

  static void mh_commit(aux_model* m, const KP<Real>& p, Real* x, uint64_t iter, uint32_t* acc,
                        double* log_alpha, cudaStream_t st) {
    ProfScope ps(m, PK_MH, st, 2 + (m->adapt ? 1 : 0) + (m->dev_iter ? 1 : 0));
    k_mh<Real><<<m->C, 128, 0, st>>>(p, (const double*)m->mh_part, (const double*)m->lz_part, iter, acc,
                                     log_alpha, m->status, m->accept, m->la_all);
    const long n = (long)m->C * m->T * m->d;
    const int grid = (int)std::min<long>((n + 255) / 256, (long)m->n_sm * 8);
    k_commit<Real><<<grid, 256, 0, st>>>(p, x, (const Real*)m->xs, (const int32_t*)m->accept);
    if (m->adapt)
      k_adapt_delta<<<1, 256, 0, st>>>((const double*)m->la_all, m->C, m->delta_dev, m->adapt_count,
                                       m->adapt_target, m->adapt_gain);
    if (m->dev_iter) k_iter_next<<<1, 1, 0, st>>>(m->iter_dev);
  }

  static bool supported(const aux_model* m) {
    return m->mode != AUX_MODE_PER_CHAIN && m->sampler == AUX_SAMPLER_SCAN && !m->sqrt_form;
  }

  static int kalman_step(aux_model* m, void* xv, int n_iters, uint64_t iter0, uint32_t* acc,
                         double* log_alpha, cudaStream_t st) {
    if (!supported(m) || m->order != 1) return AUX_E_UNSUPPORTED;
    KP<Real> p = make_kp<Real>(m);
    if (m->dev_iter) p.iter_dev = m->iter_dev;
    Real* x = (Real*)xv;
    for (int it = 0; it < n_iters; ++it) {
      const uint64_t iter = iter0 + (uint64_t)it;
      if (m->adapt) cov_pass(m, p, st);
      else if (it == 0) ensure_cov(m, p, st);
      MeanArgs<Real> a = mean_args(m);
      a.x = x; a.u = (Real*)m->u; a.v = (Real*)m->v; a.yt = (Real*)m->yt; a.iter = iter;
      a.flags = APPLY_EPI | APPLY_STORE_Q;
      means_filter(m, p, a, st);
      BackArgs<Real> b = back_args(m);
      b.xs = (Real*)m->xs; b.mh = 1; b.x = x; b.u = (const Real*)m->u; b.v = (const Real*)m->v;
      b.yts = (Real*)m->yts; b.mh_part = m->mh_part;
      backward(m, p, b, st);
      MeanArgs<Real> r = mean_args(m);
      r.yt = (Real*)m->yts; r.flags = APPLY_REV_DIFF;
      means_filter(m, p, r, st);
      mh_commit(m, p, x, iter, acc, log_alpha, st);
    }
    return cuda_ok(cudaGetLastError());
  }

  static int loglik(aux_model* m, const void* yt, double* logZ, void* mf, void* Pf, cudaStream_t st) {
    if (!supported(m)) return AUX_E_UNSUPPORTED;
    const KP<Real> p = make_kp<Real>(m);
    ensure_cov(m, p, st);
    MeanArgs<Real> a = mean_args(m);
    a.yt = (Real*)yt; a.flags = APPLY_LOGZ; a.mf = (Real*)mf; a.Pf = (Real*)Pf; a.status = m->status;
    means_filter(m, p, a, st);
    { ProfScope ps(m, PK_SUM, st); k_sum_parts<<<m->C, 128, 0, st>>>(m->lz_part, m->nb, logZ); }
    return cuda_ok(cudaGetLastError());
  }

  static int sample_path(aux_model* m, const void* yt, const void* eps, uint64_t iter, void* xs,
                         double* logZ, cudaStream_t st) {
    if (!supported(m)) return AUX_E_UNSUPPORTED;
    const KP<Real> p = make_kp<Real>(m);
    ensure_cov(m, p, st);
    MeanArgs<Real> a = mean_args(m);
    a.yt = (Real*)yt; a.flags = APPLY_EPI | APPLY_LOGZ;
    a.eps = (const Real*)eps; a.iter = iter; a.status = m->status;
    means_filter(m, p, a, st);
    BackArgs<Real> b = back_args(m);
    b.xs = (Real*)xs; b.mh = 0;
    backward(m, p, b, st);
    if (logZ) { ProfScope ps(m, PK_SUM, st); k_sum_parts<<<m->C, 128, 0, st>>>(m->lz_part, m->nb, logZ); }
    return cuda_ok(cudaGetLastError());
  }

  static int loglik_grad(aux_model*, const void*, double*, double*, double*, double*, double*, cudaStream_t) {
    return AUX_E_UNSUPPORTED;
  }

  static int tables(aux_model* m, int force, cudaStream_t st) {
    if (!supported(m)) return AUX_E_UNSUPPORTED;
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

size_t aux_wide_scratch_elems(int DP, int n_sm) {
  return (size_t)auxk::W_SLOTS_PER_SM * n_sm * auxk::W_SCR * DP * DP;
}

const AuxOps* aux_ops_f32_wide(int DP) {
  switch (DP) {
    case 64: return auxk::WOps<float, 64, false>::table();
    case 128: return auxk::WOps<float, 128, false>::table();
    default: return nullptr;
  }
}

const AuxOps* aux_ops_mixed_wide(int DP) {
  switch (DP) {
    case 64: return auxk::WOps<float, 64, true>::table();
    case 128: return auxk::WOps<float, 128, true>::table();
    default: return nullptr;
  }
}
