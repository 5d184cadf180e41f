// aux_internal.h — the model handle and the per-precision operation table.
#pragma once
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "aux_kalman.h"

struct AuxOps;

// The device words of the adapted delta read by the kernels: delta, r = delta
// / 2 and sqrt(r) in FP64, then (r, sqrt r) rounded to FP32 in the fourth word
// (the layout that k_adapt_delta writes on the device).
inline void delta_words(double delta, double w[4]) {
  const double r = 0.5 * delta, sr = std::sqrt(r);
  w[0] = delta;
  w[1] = r;
  w[2] = sr;
  const float f[2] = {(float)r, (float)sr};
  std::memcpy(&w[3], f, sizeof(f));
}

struct aux_model {
  int dtype = 0, d = 0, DP = 0, T = 0, C = 0, emis = 0, y_per_chain = 0;
  int L = 0, nb = 0;
  int fdiag = 0;             // F has no off-diagonal entries
  int tv = 0;                // time-varying dynamics (AUX_DYN_TIME_VARYING)
  void *Ftv = nullptr, *FTtv = nullptr, *Qtv = nullptr, *btv = nullptr;   // [T-1] slot-layout stacks
  int mode = AUX_MODE_PER_CHAIN;
  int order = AUX_PROPOSAL_FIRST_ORDER;
  int diag_hess = 0;         // the emission's Hessian is diagonal (SV, or R_y diagonal)
  double delta = 0.0;
  uint64_t seed = 0;
  size_t esz = 0;            // bytes per compute-type element
  cudaStream_t stream = nullptr;
  int device = 0;
  int n_sm = 0;               // multiprocessors of the device (grid caps, scratch slots)
  // model on the device, compute type, padded to DP
  void *F = nullptr, *Q = nullptr, *P0 = nullptr, *m0 = nullptr, *b = nullptr, *Ryinv = nullptr;
  void *y = nullptr;
  uint8_t *mask = nullptr;
  // workspace
  void *u = nullptr, *v = nullptr, *yt = nullptr, *xs = nullptr, *yts = nullptr;
  void *agg0 = nullptr, *agg1 = nullptr;
  void *G = nullptr, *U = nullptr, *gum = nullptr, *guv = nullptr;
  double *fq = nullptr, *fld = nullptr, *mh_part = nullptr, *lz_part = nullptr;
  int32_t *status_iter = nullptr, *status = nullptr;
  int32_t *accept = nullptr;  // [C] this step's MH decisions
  void *rho = nullptr, *rhos = nullptr;   // second order: [C][T][d] forward / reverse variances
  double *la_all = nullptr;  // [C] this step's log alpha
  // on-device delta adaptation (aux_set_delta_adaptation)
  int adapt = 0;
  double adapt_target = 0.5, adapt_gain = 1.0;
  double *delta_dev = nullptr;   // [4] words: delta, r, sqrt r (FP64), (r, sqrt r) in FP32 (delta_words)
  int32_t *adapt_count = nullptr;
  // device-resident MCMC iteration (aux_set_device_iteration): replayable steps
  int dev_iter = 0;
  uint64_t *iter_dev = nullptr;
  // factorised-prior path (aux_fact.cu): Student-t emission, diagonal F, Q, P0
  int fact = 0;
  double nu = 0.0;
  void *fmodel = nullptr;    // [5][d]: diag F, b, diag Q, diag P0, m0
  void *flam = nullptr;      // [d][d] inverse scale matrix
  void *ftab = nullptr;      // [4][T][d]: K', G, sqrt(Sigma), block prefix of G
  void *fbt = nullptr;       // [2][nb][d]: block products of K' f and of G
  double *fldb = nullptr;    // [nb][d] sum of log S_t over the block
  void *fz = nullptr, *fms = nullptr, *fub = nullptr;   // [C][nb][d]
  double *ffq = nullptr, *flz = nullptr;                 // [C][nb][d]
  double *fgam = nullptr, *fmh = nullptr;                // [C][T]
  // gradient (aux_loglik_grad): theta constants and lazily allocated smoother buffers
  int grad_ok = 0;           // the model has the SV parameterisation
  // gradient memory (aux_set_grad_memory): 0 stores G_t, Sigma_t, U_t for all
  // steps; otherwise their store is capped and the filter is recomputed per
  // chunk of grad_kc scan blocks (gscr: the chunk's scratch)
  size_t grad_mem = 0;
  int grad_kc = 0;
  void *gscr = nullptr;
  size_t gscr_bytes = 0;
  double *gconst = nullptr;  // mu, phi, L, Q, Q^{-1}, P0^{-1} (FP64, unpadded)
  void *Sig = nullptr, *sgu = nullptr, *gpart = nullptr, *s0 = nullptr;
  double *opart = nullptr;
  // covariance tables of the table modes (aux_cov.cuh), allocated on the first switch
  void *tab = nullptr, *btab = nullptr, *zb = nullptr, *ms = nullptr;
  void *cagg0 = nullptr, *cagg1 = nullptr;   // covariance scan buffers [nbc][3 DP^2] (cagg0: >= 8 DP^2)
  double *cov_ld = nullptr, *cov_ldt = nullptr;
  int32_t *cov_status = nullptr;
  int *cov_kmap = nullptr;   // [3] blocks 0, 1, nbc - 1: the distinct covariance block aggregates
  int Lc = 0, nbc = 0;       // block length and block count of the covariance scan
  int cov_valid = 0;         // the tables match the current model
  // divide-and-conquer sampler (aux_set_sampler, aux_bridge.cuh)
  int sampler = AUX_SAMPLER_SCAN;
  int br_NN = 0;             // internal nodes of the tree over T - 1 intervals
  void *br_L0 = nullptr;     // [T-1][DP^2] leaf covariances (table modes)
  void *br_tree = nullptr;   // shared tree: E, L [NN][DP^2], bridges [NN][3][DP^2]
  void *br_ctree = nullptr;  // per-chain trees: the same per chain
  void *br_g = nullptr;      // [C][NN][DP] node offsets g
  int br_valid = 0;          // the shared tree matches the covariance tables
  // square-root form of the per-chain filter (aux_set_filter_form, aux_sqrt.cuh)
  int sqrt_form = 0;
  const AuxOps *ops = nullptr;
  std::vector<void *> allocs;
  // optional per-launch CUDA-event timing (aux_set_profiling)
  struct Rec { int kind, n; cudaEvent_t a, b; };
  bool profiling = false;
  std::vector<Rec> recs;      // recorded this window
  std::vector<Rec> pool;      // free event pairs
};

// kernel kinds reported by aux_read_profile (order of AUX_PROFILE_* in the header)
enum { PK_LINEARISE = 0, PK_TEMPLATE, PK_REDUCE, PK_SCAN, PK_APPLY, PK_BACKWARD, PK_MH, PK_SUM,
       PK_SMOOTH, PK_GRAD, PK_COV_REDUCE, PK_COV_SCAN, PK_COV_APPLY, PK_COV_PRODUCTS, PK_BR_TREE,
       PK_BRIDGE, PK_COUNT };

// bracket a launch with events on its stream when profiling is on
struct ProfScope {
  aux_model *m;
  cudaStream_t st;
  aux_model::Rec r;
  bool on;
  // `launches`: the kernels the scope launches (counted by aux_read_profile)
  ProfScope(aux_model *m_, int kind, cudaStream_t st_, int launches = 1)
      : m(m_), st(st_), on(m_->profiling) {
    if (!on) return;
    if (!m->pool.empty()) { r = m->pool.back(); m->pool.pop_back(); }
    else { cudaEventCreate(&r.a); cudaEventCreate(&r.b); }
    r.kind = kind;
    r.n = launches;
    cudaEventRecord(r.a, st);
  }
  ~ProfScope() {
    if (!on) return;
    cudaEventRecord(r.b, st);
    m->recs.push_back(r);
  }
};

struct AuxOps {
  int (*prepare)();
  int (*kalman_step)(aux_model *, void *x, int n_iters, uint64_t iter0, uint32_t *acc,
                     double *log_alpha, cudaStream_t);
  int (*loglik)(aux_model *, const void *yt, double *logZ, void *mf, void *Pf, cudaStream_t);
  int (*sample_path)(aux_model *, const void *yt, const void *eps, uint64_t iter, void *xs,
                     double *logZ, cudaStream_t);
  int (*loglik_grad)(aux_model *, const void *yt, double *logZ, double *g_mu, double *g_phi,
                     double *g_L, double *g_delta, cudaStream_t);
  // the covariance tables of a table mode: recomputed when `force` or not valid
  int (*tables)(aux_model *, int force, cudaStream_t);
};

int aux_fact_prepare(aux_model *m);
int aux_fact_kalman_step(aux_model *m, void *x, int n_iters, uint64_t iter0, uint32_t *acc,
                         double *log_alpha, cudaStream_t st);
int aux_fact_loglik(aux_model *m, const void *yt, double *logZ, void *mf, cudaStream_t st);
int aux_fact_sample_path(aux_model *m, const void *yt, const void *eps, uint64_t iter, void *xs,
                         double *logZ, cudaStream_t st);

const AuxOps *aux_ops_f32(int DP);
const AuxOps *aux_ops_f64(int DP);
const AuxOps *aux_ops_f32_wide(int DP);   // padded dimensions 64 and 128 (aux_wide.cu)
const AuxOps *aux_ops_mixed_wide(int DP); // the same, mixed precision (AUX_MIXED)
size_t aux_wide_scratch_elems(int DP, int n_sm);   // per-CTA scratch of the wide covariance pass

// element counts of the per-block buffers for a padded dimension DP
inline size_t aux_es(int DP) { return 3u * DP * DP + 2u * DP; }
