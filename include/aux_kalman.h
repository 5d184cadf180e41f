/*
 * aux_kalman.h — C ABI of the GB300 auxiliary Kalman sampler.
 *
 * The library implements the first-order auxiliary Kalman sampler for
 * state-space models with Gaussian dynamics (Corenflos & Sarkka,
 * arXiv:2303.00301, Section 2.2, Eqs. (2.5)-(2.7) and Algorithm 2):
 *
 *   target   pi(x) ∝ N(x_0; m0, P0) prod_{t>=1} N(x_t; F x_{t-1} + b, Q)
 *                     prod_t h(y_t | x_t),         t = 0 .. T-1
 *   one step u_t = x_t + sqrt(delta/2) eps_t,  v_t = grad_{x_t} log h(y_t | x_t),
 *            ytilde_t = u_t + (delta/2) v_t,
 *            x* ~ smoothing law of the LGSSM (F, b, Q; H = I, R = (delta/2) I)
 *                 given ytilde, sampled by a parallel-in-time Kalman filter
 *                 (Appendix A.2.1) and a parallel backward-sampling scan
 *                 (Proposition A.1, parallel RTS sampler of Appendix A.2.2),
 *            accept x* with the Metropolis-Hastings ratio of Algorithm 2.
 *
 * Emission models: linear-Gaussian log h = log N(y; x, R_y) (Appendix A,
 * Eq. (A.1)) and multivariate stochastic volatility
 * log h = sum_i log N(y_i; 0, exp(x_i)) (Section 4.1). Sigma_t = I.
 *
 * Conventions for every entry point:
 *  - T is the number of states (array length); arrays are row-major and
 *    chain-major: paths [C][T][d], matrices [..][d][d].
 *  - "device" pointers are caller-owned CUDA device memory; "host" pointers
 *    are read during the call only. The model handle owns its workspace.
 *  - Compute type: AUX_F32 -> float, AUX_F64 -> double. Device path buffers
 *    (x, ytilde, mf, Pf, eps, xstar) are in the compute type; log-likelihoods
 *    and log acceptance ratios are always double.
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls only enqueue work; results are valid after the stream completes.
 *  - Return value: AUX_OK or an AUX_E_* code. Argument errors are detected on
 *    the host before anything is enqueued. Numerical failures on the device
 *    (a non-positive Cholesky pivot, a non-finite ratio) never trap: they are
 *    latched into per-chain status words read by aux_get_status, and the
 *    affected chain's proposal is rejected.
 *  - Random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed by the seed
 *    given to aux_init_model, counter (word, t | purpose << 24,
 *    iteration & 0xffffffff, chain); each 32-bit word r gives
 *    u = ((r >> 9) + 0.5) 2^-23 and Box-Muller pairs give normals. A step's
 *    draws depend only on (seed, chain, iteration), so runs are resumable.
 */
#ifndef AUX_KALMAN_H
#define AUX_KALMAN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AUX_ABI_VERSION 3

/* status codes */
#define AUX_OK             0
#define AUX_E_INVALID_ARG  1  /* bad pointer, size, enum or version */
#define AUX_E_NOT_PD       2  /* P0, Q or R_y not positive definite; or a device Cholesky pivot <= 0 */
#define AUX_E_NONFINITE    3  /* NaN/Inf in an input or in a device log-ratio */
#define AUX_E_CUDA         4  /* a CUDA runtime call failed */
#define AUX_E_TIMEOUT      5  /* reserved: a bounded device wait gave up */
#define AUX_E_OOM          6  /* workspace allocation failed */
#define AUX_E_UNSUPPORTED  7  /* valid but not built (e.g. d_x > 128) */
#define AUX_E_TOO_LARGE    8  /* the problem does not fit the fixed scratch of aux_loglik_noalloc */

/* compute types */
#define AUX_F32 0
#define AUX_F64 1
/* Mixed precision (33 <= d_x <= 128, the table modes; see "Wide state
 * dimensions"): buffers, tables and per-chain means in FP32 as AUX_F32; the
 * covariance pass's dense products on the tensor cores with TF32 operands and
 * FP32 accumulation, each product split into three TF32 products
 * (a_hi b_hi + a_hi b_lo + a_lo b_hi, x_hi = tf32(x), x_lo = tf32(x - x_hi));
 * the factorisations in the element operator's (I + C_i J_j) solve, chol(C_i)
 * and chol(N), N = I + U^T J_j U, and the inverse of chol(N), in FP64; log
 * determinants and likelihood sums in FP64 as in every dtype. The device
 * buffers passed to the entry points are float. Other sizes, the per-chain
 * mode, the factorised prior and aux_loglik_noalloc return AUX_E_UNSUPPORTED
 * (aux_loglik_noalloc: AUX_E_INVALID_ARG). */
#define AUX_MIXED 2

/* execution modes (aux_set_mode) */
#define AUX_MODE_PER_CHAIN  0  /* every chain runs its own covariance recursion (default) */
#define AUX_MODE_SHARED_COV 1  /* one covariance pass per call, shared by all chains */
#define AUX_MODE_CACHED_COV 2  /* one covariance pass per model, reused until the model changes */

/* dynamics kinds (aux_model_desc.dyn_kind) */
#define AUX_DYN_HOMOGENEOUS  0  /* one (F, b, Q) for every transition (default) */
#define AUX_DYN_TIME_VARYING 1  /* (F_t, b_t, Q_t) per transition into x_{t+1}, t = 0 .. T-2 */

/* emission models */
#define AUX_EMIS_LINEAR_GAUSSIAN 0
#define AUX_EMIS_SV              1
#define AUX_EMIS_STUDENT_T       2  /* multivariate t, scale R_y, nu degrees of freedom (Section 4.2) */

/* Model description (Section 2.2, Eq. (2.5); SV model of Section 4.1).
 * All arrays are HOST pointers to double, copied by aux_init_model. */
typedef struct {
  int32_t abi_version;   /* AUX_ABI_VERSION */
  int32_t dtype;         /* AUX_F32 | AUX_F64 | AUX_MIXED */
  int32_t d_x;           /* state dimension: 1..128 (AUX_F32; 33..128 in the table
                            modes only, see "Wide state dimensions"), 1..32 (AUX_F64);
                            1..1024 with AUX_EMIS_STUDENT_T (factorised prior, see below) */
  int32_t T;             /* number of states, T >= 1 */
  int32_t n_chains;      /* C >= 1 */
  int32_t emis_kind;     /* AUX_EMIS_* */
  int32_t y_per_chain;   /* 0: y is [T][d] shared by all chains; 1: y is [C][T][d] */
  int32_t block_len;     /* time steps per scan block; 0 = library default */
  const double *m0;      /* [d]    mean of p_0 */
  const double *P0;      /* [d*d]  covariance of p_0 (symmetric positive definite) */
  const double *F;       /* [d*d]  transition matrix */
  const double *b;       /* [d]    transition offset */
  const double *Q;       /* [d*d]  transition covariance (SPD) */
  const double *y;       /* observations, see y_per_chain */
  const uint8_t *obs_mask; /* [T] or NULL: log h_t == 0 where obs_mask[t] == 0 */
  const double *R_y;     /* [d*d] emission covariance (linear-Gaussian) or scale matrix
                            (Student-t), else NULL */
  double delta;          /* step size delta > 0; auxiliary covariance (delta/2) I */
  double nu;             /* Student-t degrees of freedom (> 0), ignored otherwise */
  int32_t dyn_kind;      /* AUX_DYN_HOMOGENEOUS | AUX_DYN_TIME_VARYING (see below) */
} aux_model_desc;

/* Time-varying dynamics (Algorithm 2 with local F_t, b_t, Q_t; the model of
 * Appendix A with time-indexed transitions). With AUX_DYN_TIME_VARYING, F, b and
 * Q point to T - 1 stacked transitions, F [T-1][d][d], b [T-1][d], Q [T-1][d][d]
 * (each Q_t SPD): x_{t+1} = F_t x_t + b_t + N(0, Q_t). The per-chain path runs
 * them (both proposals, the scan sampler, the covariance form, d_x <= 32); the
 * table modes, the square-root form, the bridging sampler, the gradient and the
 * SV parameterisation calls assume one transition and return AUX_E_UNSUPPORTED
 * (aux_set_mode with a table mode included); so do AUX_MIXED and the factorised
 * prior. aux_set_model_params keeps the handle's dyn_kind. */

/* Factorised prior (Section 4.2). With AUX_EMIS_STUDENT_T,
 *   log h(y_t | x_t) = log t_nu(y_t; x_t, R_y),
 * which does not factorise over the coordinates, and F, Q, P0 must be diagonal
 * (else AUX_E_UNSUPPORTED). The auxiliary LGSSM then splits into d_x
 * independent scalar LGSSMs and the library runs them as such (one thread per
 * chain, scan block and coordinate), with the first-order proposal; the
 * execution mode is not used (the scalar covariance tables are kept until the
 * model changes, or recomputed every iteration while delta adapts).
 * aux_loglik takes mf (not Pf); aux_loglik_grad, aux_set_model_params and the
 * second-order proposal return AUX_E_UNSUPPORTED for such a handle. */

/* Wide state dimensions (33 <= d_x <= 128, AUX_F32; padded to 64 or 128).
 * These run the table modes only (aux_set_mode with AUX_MODE_SHARED_COV or
 * AUX_MODE_CACHED_COV before the first step): the covariance pass forms the
 * filtering covariances of every step by doubling over the steps (the prefix
 * of step t is the first element composed with t copies of the shared
 * element, Appendix A.2.1), then the per-step gains, backward gains and
 * chol(Sigma_t) independently per step, with CTA-wide dense routines; the
 * per-chain means follow the same recursions as for narrow d. In
 * AUX_MODE_PER_CHAIN aux_kalman_step, aux_loglik and aux_sample_path return
 * AUX_E_UNSUPPORTED; so do aux_loglik_grad, the second-order proposal, the
 * square-root form and the bridging sampler (their setters return it). The
 * first switch to a table mode also allocates 2 * (SM count) * 8 DP^2 elements of
 * scratch for the covariance pass. */

typedef struct aux_model aux_model;   /* opaque handle */

/* Create a model handle: validates the description (P0, Q, R_y must be SPD,
 * all values finite), copies the model to the device of the current CUDA
 * context, and allocates the workspace for n_chains chains of length T.
 * seed keys the Philox streams. On success *out owns device memory until
 * aux_free_model. Errors: INVALID_ARG, NOT_PD, NONFINITE, UNSUPPORTED, OOM, CUDA. */
int aux_init_model(const aux_model_desc *desc, uint64_t seed, void *stream, aux_model **out);

/* n_iters auxiliary Kalman MH steps (Algorithm 2 with Gaussian dynamics)
 * on all chains, iterations iter0 .. iter0 + n_iters - 1.
 *   x            device [C][T][d], compute type: chain states, updated in place.
 *   accept_count device [C] uint32 or NULL: incremented by each acceptance.
 *   log_alpha    device [C] double or NULL: log MH ratio of the last step.
 * The MH test accepts iff log U < log alpha, U the (chain, iteration) uniform.
 * Errors: INVALID_ARG, CUDA. Device failures: see aux_get_status. */
int aux_kalman_step(aux_model *m, void *x, int32_t n_iters, uint64_t iter0,
                    uint32_t *accept_count, double *log_alpha, void *stream);

/* Log marginal likelihood of the auxiliary LGSSM for given pseudo-observations
 * (the likelihood of the Kalman filter algorithm, Appendix A.1, with predictive terms
 * N(ytilde_t; m^p_t, P^p_t + R), computed by the parallel filter of Appendix A.2.1).
 *   ytilde device [C][T][d] compute type.
 *   logZ   device [C] double (required).
 *   mf     device [C][T][d] or NULL: filtering means m^f_t.
 *   Pf     device [C][T][d][d] or NULL: filtering covariances P^f_t. */
int aux_loglik(aux_model *m, const void *ytilde, double *logZ, void *mf, void *Pf, void *stream);

/* One draw from the smoothing law of the auxiliary LGSSM given ytilde
 * (parallel filter + backward (G, U) scan, Proposition A.1).
 *   ytilde device [C][T][d]; eps device [C][T][d] standard normals used as the
 *   backward noise of U_t (or NULL: the Philox backward stream of
 *   (chain, iteration)); xstar device [C][T][d] output; logZ device [C] or NULL. */
int aux_sample_path(aux_model *m, const void *ytilde, const void *eps, uint64_t iteration,
                    void *xstar, double *logZ, void *stream);

/* Gradient of log Z (as computed by aux_loglik) with respect to
 * theta = (mu, phi, chol Sigma, delta) of the multivariate stochastic-volatility
 * parameterisation (Section 4.1): F = diag(phi), b = (I - F) mu, Q = L L^T with
 * L = chol Sigma lower triangular, p_0 the stationary law (m0 = mu,
 * P0_ij = Q_ij / (1 - phi_i phi_j)), R = (delta/2) I; ytilde is held fixed. The
 * paper differentiates by automatic differentiation; here the gradient is
 * Fisher's identity, the expected complete-data score under the smoothing law,
 * with the smoother computed by the parallel backward scan of Appendix A.2.2.
 *   ytilde      device [C][T][d] compute type.
 *   logZ        device [C] double or NULL.
 *   g_mu        device [C][d] double;  g_Phi device [C][d] double (d/d phi_i);
 *   g_cholSigma device [C][d][d] double (lower triangle; upper entries 0);
 *   g_delta     device [C] double.
 * Errors: INVALID_ARG; UNSUPPORTED unless F is diagonal with |phi_i| < 1,
 * m0 = (I - F)^{-1} b and P0 is the stationary covariance, and for AUX_F64
 * with d_x > 16 (the smoother's per-block staging would exceed a CTA's shared
 * memory); OOM on the first call (it allocates C*T*d^2 elements for the
 * backward covariances). */
int aux_loglik_grad(aux_model *m, const void *ytilde, double *logZ, double *g_mu, double *g_Phi,
                    double *g_cholSigma, double *g_delta, void *stream);
/* (ytilde may be NULL: the pseudo-observations of the last aux_kalman_step's
 * proposal, ytilde_t = u_t + (delta/2) v_t at the state before that step, kept in
 * the handle's workspace.) */

/* Cap on the device memory aux_loglik_grad may use for the backward elements
 * (G_t, U_t) and covariances Sigma_t that its smoother reads, C*T*(2 p^2 + p)
 * elements when all are stored (p = d_x rounded up to 4, 8, 16 or 32).
 * max_bytes = 0 (the default): store them all. Otherwise, when that store
 * would exceed max_bytes, the gradient recomputes instead of storing: the
 * in-block filter (Appendix A.2.1, from the stored block prefixes of the
 * scan) runs over chunks of scan blocks into a scratch of at most max_bytes
 * (at least one block of every chain), once for the smoother's block
 * aggregates and once for its backward sweep, so the filter's in-block pass
 * runs twice. The result is the same as with the full store (the same
 * arithmetic per block). Errors: INVALID_ARG; UNSUPPORTED where
 * aux_loglik_grad is. */
int aux_set_grad_memory(aux_model *m, uint64_t max_bytes);

/* The SV parameterisation theta = (mu, phi, L = chol Sigma) behind the C ABI
 * (Section 4.1): F = diag(phi), b = (1 - phi) mu, Q = L L^T, p_0 the stationary
 * law (m0 = mu, P0_ij = Q_ij / (1 - phi_i phi_j)). The handle keeps theta on the
 * device beside the constants aux_loglik_grad needs (Q^{-1}, P0^{-1}); one warp
 * rebuilds the padded model and those constants from theta, in FP64.
 *
 * aux_set_sv_theta: host theta (mu [d], phi [d] with |phi_i| < 1, L [d][d] lower
 * triangular with positive diagonal; its upper part is ignored) and delta > 0;
 * synchronises the handle's stream, writes the model (y, R_y and the mask are
 * kept) and marks cached tables stale. Errors: INVALID_ARG, NONFINITE, NOT_PD
 * (a diagonal entry of L <= 0), UNSUPPORTED (factorised prior, d_x > 32), CUDA.
 *
 * aux_sv_theta_step: the gradient-based theta-update inside the Gibbs sweep.
 * The paper updates its static parameters inside the sampler (Section 4.3)
 * without stating a rule; this one is a projected gradient-ascent step on the
 * mean over chains of log p(ytilde_c | theta):
 *   mu <- mu + lr mean_c g_mu[c],  phi <- clip(phi + lr mean_c g_phi[c], -0.999, 0.999),
 *   L  <- tril(L + lr mean_c g_L[c]),  diag(L) <- max(diag(L), 1e-6),
 * then the model is rebuilt from theta; delta is left to the sampler. The
 * gradients are device arrays laid out as aux_loglik_grad writes them
 * ([C][d], [C][d], [C][d][d]). Everything stays on the device (no host
 * synchronisation), so a sweep aux_kalman_step -> aux_loglik_grad(ytilde = NULL)
 * -> aux_sv_theta_step can be captured in a CUDA graph once aux_loglik_grad's
 * first call has allocated its buffers. Requires the SV parameterisation
 * (set by aux_init_model / aux_set_model_params / aux_set_sv_theta).
 * Errors: INVALID_ARG, UNSUPPORTED (no SV parameterisation, factorised prior,
 * d_x > 32, or AUX_MODE_CACHED_COV, whose kept tables would go stale), CUDA.
 *
 * aux_get_sv_theta: the current theta (host arrays mu [d], phi [d], L [d][d];
 * synchronises). Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
int aux_set_sv_theta(aux_model *m, const double *mu, const double *phi, const double *L, double delta);
int aux_sv_theta_step(aux_model *m, const double *g_mu, const double *g_phi, const double *g_L, double lr,
                      void *stream);
int aux_get_sv_theta(aux_model *m, double *mu, double *phi, double *L);

/* Choose how the filter and the backward sampler are executed. All modes
 * compute the same quantities (the same x*, log Z and log alpha up to
 * floating-point rounding). With the first-order proposal of Section 2.2 and
 * Gaussian dynamics the pseudo-observation noise is R = (delta/2) I, so the
 * covariance part of every filtering element (Appendix A.2.1) and of every
 * backward element (Eq. (A.14)) depends only on (m0, P0, F, Q, delta): it is
 * the same for every chain and every iteration.
 *   AUX_MODE_PER_CHAIN   every chain runs the full element recursion
 *                        (covariances included) in every pass.
 *   AUX_MODE_SHARED_COV  each call runs the covariance half of the blocked
 *                        scan once (the gains, G_t, chol(Sigma_t) and block
 *                        aggregates, as tables of T*6*d^2 elements owned by
 *                        the handle); each chain then runs only matrix-vector
 *                        recursions on its means.
 *   AUX_MODE_CACHED_COV  as SHARED_COV, but the tables are kept and reused by
 *                        later calls until aux_set_model_params or aux_set_mode
 *                        invalidates them.
 * The first switch to a table mode allocates the tables (may return OOM).
 * A factorisation failure in the covariance pass is reported for every chain
 * (status words; the MH step rejects). aux_loglik_grad always runs per chain.
 * Errors: INVALID_ARG, OOM. */
int aux_set_mode(aux_model *m, int32_t mode);

/* Proposals (aux_set_proposal) */
#define AUX_PROPOSAL_FIRST_ORDER  1  /* Eq. (2.7): R = (delta/2) I (default) */
#define AUX_PROPOSAL_SECOND_ORDER 2  /* Eqs. (2.8)-(2.9): Hessian of log h in the pseudo-observations */

/* Choose the auxiliary proposal of aux_kalman_step (Section 2.2).
 * AUX_PROPOSAL_FIRST_ORDER linearises gamma_t = log h(y_t | x_t) to first
 * order: pseudo-observations ytilde_t = u_t + (delta/2) v_t with covariance
 * R = (delta/2) I (Eq. (2.7)). AUX_PROPOSAL_SECOND_ORDER adds the Hessian
 * Lambda_t of gamma_t at x_t (Eq. (2.8)) and samples from the LGSSM with
 * observations omega_t = Omega_t ((2/delta) u_t + v_t - Lambda_t x_t) and
 * covariance Omega_t = ((2/delta) I - Lambda_t)^{-1} (Eq. (2.9), Sigma_t = I);
 * the MH ratio then keeps the Omega-dependent proposal terms. The library
 * supports diagonal Hessians (the SV emission, or a linear-Gaussian emission
 * with diagonal R_y; with a Gaussian emission the second-order proposal is
 * exact and every step is accepted). The second-order proposal runs in
 * AUX_MODE_PER_CHAIN only: its covariances depend on the chain's state, so
 * aux_kalman_step returns AUX_E_UNSUPPORTED in a table mode. The first switch
 * to the second order allocates 2*C*T*d elements (may return OOM).
 * aux_loglik, aux_sample_path and aux_loglik_grad are unaffected (they take
 * pseudo-observations with R = (delta/2) I).
 * Errors: INVALID_ARG (unknown order), UNSUPPORTED (non-diagonal Hessian), OOM. */
int aux_set_proposal(aux_model *m, int32_t order);

/* Filter forms (aux_set_filter_form) */
#define AUX_FILTER_COVARIANCE  0  /* elements (A, b, C, eta, J), Appendix A.2.1 (default) */
#define AUX_FILTER_SQUARE_ROOT 1  /* the same elements with C and J as triangular factors */

/* Choose the arithmetic form of the per-chain parallel filter of aux_loglik.
 * Section 4.1 reports that the parallel filter diverged in single precision
 * and names the square-root form as the remedy (the paper ran in double
 * precision instead). AUX_FILTER_SQUARE_ROOT carries every element's C and J
 * as factors U U^T and Z Z^T, forms each new covariance factor by an
 * orthogonal (Householder) triangularisation of [X1, X2] (the factor of
 * X1 X1^T + X2 X2^T) instead of adding and subtracting covariances, and runs
 * the in-block filter as the square-root Kalman step (Joseph form). Its
 * results equal the covariance form's up to rounding; it costs several times
 * more. With it the in-block filter also forms the backward elements of the
 * (G, U) scan, chol(Sigma_t) by triangularisation in Joseph form, so that
 * aux_kalman_step and aux_sample_path run on the square-root filter too.
 * In the table modes (AUX_MODE_SHARED_COV, AUX_MODE_CACHED_COV) the form
 * applies to the covariance pass: the shared block aggregates, their prefixes
 * and the in-block Riccati steps that write the per-step tables run on
 * factors, so that the tables (gains, filtering covariances, backward gains
 * and chol(Sigma_t)) are accurate in single precision; the per-chain means
 * passes are linear in the means and unchanged. Scope: in AUX_MODE_PER_CHAIN,
 * first-order proposal and AUX_SAMPLER_SCAN (other combinations return
 * AUX_E_UNSUPPORTED from the calls that need them); in a table mode, every
 * sampler. Not available for the factorised-prior model (UNSUPPORTED).
 * Errors: INVALID_ARG, UNSUPPORTED. */
int aux_set_filter_form(aux_model *m, int32_t form);

/* Pathwise samplers (aux_set_sampler) */
#define AUX_SAMPLER_SCAN     0  /* (G, U) suffix scan, Eqs. (A.14)-(A.15), Proposition A.1 (default) */
#define AUX_SAMPLER_BRIDGING 1  /* divide-and-conquer bridging sampler, Section 2.4.2, Appendix A.2.3 */

/* Choose how aux_kalman_step and aux_sample_path draw the path from the
 * smoothing law of the auxiliary LGSSM once the filter has run. Both samplers
 * draw from the same law in O(log T) depth; they map the noise differently,
 * so the same (seed, chain, iteration) gives different paths.
 * AUX_SAMPLER_SCAN composes the backward conditionals (G_t, U_t) with a
 * suffix scan. AUX_SAMPLER_BRIDGING builds the dyadic tree of the backward
 * conditionals p(x_k | x_m, y) = N(E x_m + g, L) over the intervals
 * [a 2^j, (a+1) 2^j] (clipped to T - 1), with the bridge
 * p(x_l | x_k, x_m, y) = N(G x_k + Gamma x_m + w, V) at each split point
 * l = (2a+1) 2^(j-1), then draws x_{T-1} from the last filtering law, x_0 given
 * x_{T-1}, and the split points level by level from the root down; state t
 * takes the t-th normal of the backward stream (or row t of a given eps)
 * whatever its level. In the table modes the tree's matrices are built once
 * per covariance pass and shared by all chains; in AUX_MODE_PER_CHAIN every
 * chain has its own tree (both proposals). Not available for the
 * factorised-prior model (UNSUPPORTED). The switch allocates the tree for the
 * current mode, and aux_set_mode for a later mode (may return OOM): per
 * chain about 5 C (T-1) DP^2 elements, shared 6 (T-1) DP^2.
 * Errors: INVALID_ARG, UNSUPPORTED, OOM. */
int aux_set_sampler(aux_model *m, int32_t sampler);

/* On-line adaptation of delta to a target acceptance rate, on the device.
 * The paper tunes delta to a target acceptance but states no rule (Section 4);
 * this one is a Robbins-Monro recursion on log delta shared by the handle's
 * chains: after the MH test of iteration k = 1, 2, ... of aux_kalman_step,
 *   log delta <- log delta + gain k^{-0.6} (a_k - target),
 * a_k = mean over chains of min(1, exp(log alpha)) (0 for a non-finite log
 * alpha), log delta clamped to [-40, 40]. Every later step (and aux_loglik,
 * aux_sample_path) uses the adapted delta; the update stays on the device
 * (no host synchronisation). In the table modes the covariance pass then
 * runs every iteration. Enabling starts from the handle's current delta and
 * k = 0; disabling freezes delta at its adapted value (synchronises).
 * aux_loglik_grad uses the handle's host delta (a theta component), i.e. the
 * description's value or the value frozen at the last disable.
 * enable: 0 or 1; target in (0, 1); gain > 0.
 * Errors: INVALID_ARG, OOM, CUDA. */
int aux_set_delta_adaptation(aux_model *m, int32_t enable, double target, double gain);

/* Keep the MCMC iteration index on the device, so that a sequence of
 * aux_kalman_step calls can be captured once in a CUDA graph and replayed:
 * while enabled, iteration k of a call draws its Philox streams with the
 * device counter's value (instead of iter0 + k) and the call's last launch of
 * each iteration adds 1 to it. Enabling sets the counter to `start`
 * (synchronises). Replays of a captured call are then the same steps as the
 * eager calls with iter0 = start, start + n_iters, ... aux_sample_path keeps
 * its explicit iteration. Errors: INVALID_ARG, OOM, CUDA. */
int aux_set_device_iteration(aux_model *m, int32_t enable, uint64_t start);

/* The device counter's current value (synchronises). Errors: INVALID_ARG (not
 * enabled yet), CUDA. */
int aux_get_device_iteration(aux_model *m, uint64_t *iteration);

/* The handle's current delta (the adapted value while adaptation is on;
 * synchronises the handle's last stream then). Errors: INVALID_ARG, CUDA. */
int aux_get_delta(aux_model *m, double *delta);

/* Replace the model of an existing handle (same dtype, d_x, T, n_chains,
 * emis_kind, y_per_chain): validates as aux_init_model, then overwrites the
 * device copies of m0, P0, F, b, Q, y, R_y and delta. Synchronises the handle's
 * last stream first. Used for parameter updates between sampler sweeps. */
int aux_set_model_params(aux_model *m, const aux_model_desc *desc);

/* Copy the latched per-chain device status words to host memory
 * (synchronises the handle's last stream) and clear them.
 *   per_chain_status host [C] int32 or NULL. Returns AUX_OK if every chain is
 *   clean, else the first non-zero code. */
int aux_get_status(aux_model *m, int32_t *per_chain_status);

/* Kernel kinds reported by aux_read_profile. */
#define AUX_PROFILE_LINEARISE 0  /* v, u, ytilde at the current state (Eq. (2.7)) */
#define AUX_PROFILE_TEMPLATE  1  /* reserved (no kernel of this kind is launched) */
#define AUX_PROFILE_REDUCE    2  /* block aggregates of the filtering elements (Appendix A.2.1) */
#define AUX_PROFILE_SCAN      3  /* one Hillis-Steele round over block aggregates (Appendix A.2.1) */
#define AUX_PROFILE_APPLY     4  /* in-block filtering from the block prefix + (G_t, U_t) (Eq. (A.14)) */
#define AUX_PROFILE_BACKWARD  5  /* backward (G, U) scan, x*, and MH partial sums (Proposition A.1) */
#define AUX_PROFILE_MH        6  /* log alpha, MH test and state update (Algorithm 2) */
#define AUX_PROFILE_SUM       7  /* log Z reduction */
#define AUX_PROFILE_SMOOTH    8  /* smoother aggregates and sweep with score statistics (gradient) */
#define AUX_PROFILE_GRAD      9  /* FP64 gradient assembly per chain */
#define AUX_PROFILE_COV_REDUCE   10 /* covariance pass (table modes): block aggregates */
#define AUX_PROFILE_COV_SCAN     11 /* covariance pass: one Hillis-Steele round */
#define AUX_PROFILE_COV_APPLY    12 /* covariance pass: in-block filter and per-step tables */
#define AUX_PROFILE_COV_PRODUCTS 13 /* covariance pass: block products of the means partition */
#define AUX_PROFILE_BRIDGE_TREE  14 /* bridging sampler: leaf covariances and tree matrices, all levels */
#define AUX_PROFILE_BRIDGE       15 /* bridging sampler: node offsets, the two ends, split points, MH terms */
#define AUX_PROFILE_KINDS        16

/* Turn per-launch timing on or off for this handle: while on, every kernel
 * launch is bracketed by two CUDA events recorded on its own stream. */
int aux_set_profiling(aux_model *m, int32_t enable);

/* Accumulated device time (ms, from the event pairs) and launch count per
 * kernel kind since the last read; waits for the recorded events and resets
 * the window. ms_per_kind, launches_per_kind: host arrays of n_kinds entries. */
int aux_read_profile(aux_model *m, double *ms_per_kind, int32_t *launches_per_kind, int32_t n_kinds);

/* aux_loglik without any device allocation. The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc, such as code that
 * runs inside a host callback, under an allocator it must not bypass, or in a
 * process whose device-memory budget is fixed before it starts, and that
 * therefore cannot create a model handle.
 * It computes the same log marginal likelihood as aux_loglik, logZ[c] for each
 * chain's pseudo-observations, from the host model description alone (only
 * dtype, d_x, T, n_chains, block_len, m0, P0, F, b, Q, delta and dyn_kind are read;
 * time-varying dynamics return AUX_E_UNSUPPORTED).
 *   desc   host model description (see aux_model_desc).
 *   ytilde device [C][T][d] compute type (caller-owned input).
 *   logZ   device [C] double (caller-owned output).
 * All scratch lives in one device array of AUX_NOALLOC_SCRATCH_BYTES that is
 * part of the library: every GPU that loads the library holds it until the
 * process exits. Problems needing more scratch return AUX_E_TOO_LARGE; the
 * scratch needed is about 2 * C * ceil(T / block_len) * (3 p^2 + 2 p) elements,
 * p = d_x rounded up to 4, 8, 16 or 32.
 * The call is synchronous: it waits for the work already queued on stream,
 * uploads the model from a host stack buffer, runs the pass, waits for it and
 * reads back the status words and logZ. It returns AUX_E_NOT_PD when a device
 * factorisation failed and AUX_E_NONFINITE when a status word or some logZ[c]
 * is not finite (logZ then holds what the pass produced). Because it
 * synchronises and reads host memory it cannot be captured: while stream is
 * capturing it returns AUX_E_UNSUPPORTED and enqueues nothing.
 * The first call on a device does a one-time set-up for that device (it looks
 * up the array's device address and sets kernel attributes), under a lock, so
 * first calls from several host threads are safe. Every call shares the
 * array, which keeps the last call's contents: calls whose work overlaps on
 * the GPU (other streams or host threads) race, so serialise them. */
#define AUX_NOALLOC_SCRATCH_BYTES (32u << 20)
int aux_loglik_noalloc(const aux_model_desc *desc, const void *ytilde, double *logZ, void *stream);

/* ------------------------------------------------------------------------
 * Batched instances: many independent models (uneven T and d_x, one or more
 * chains each) advanced by ONE persistent launch per MCMC iteration.
 * Section 2.4 (parallel-in-time sampling of long series) applied across
 * instances: every chain of every model runs the MH step of Algorithm 2 with
 * the table-mode means path (filtering means, (G, U) backward sampling of
 * Appendix A.2.2 / Proposition A.1, MH test), as a list of warp items that a
 * persistent grid drains; items wait for their inputs through per-chain
 * completion counters with bounded waits (no kernel boundary between the
 * passes, no per-instance launches).
 *
 * A batch refers to caller-owned model handles and state buffers; they must
 * outlive it. Each handle must be FP32, in AUX_MODE_SHARED_COV or
 * AUX_MODE_CACHED_COV, first-order proposal, scan sampler, homogeneous
 * dynamics with a diagonal F, no delta adaptation, padded width 4 .. 64
 * (d_x <= 64), SV or linear-Gaussian emission; each handle at most once.
 * Otherwise AUX_E_UNSUPPORTED / AUX_E_INVALID_ARG. Chain c of model i draws the
 * same Philox streams as aux_kalman_step on that handle at the same
 * iteration. Errors: AUX_E_OOM, AUX_E_CUDA; a device wait that runs out
 * (2 s) aborts the rest of that launch and is reported by
 * aux_batch_get_status as AUX_E_TIMEOUT. */
typedef struct aux_batch aux_batch;

/* Create a batch over models[0 .. n_models) with state buffers x[i] (device,
 * [C_i][T_i][d_i] FP32, updated in place by every step). Computes each
 * model's covariance tables if they are not valid, copies them into the
 * batch's layout and forms the block tables (device memory owned by the
 * batch: 4 T + 2 ceil(T / L) matrices of p^2 words per model, p the padded
 * width). iteration: the MCMC iteration of the first step (kept on the
 * device, incremented by every step). Synchronises stream. */
int aux_batch_create(aux_model *const *models, void *const *x, int32_t n_models, uint64_t iteration,
                     void *stream, aux_batch **out);

/* AUX_MODE_CACHED_COV (default): the tables are kept; AUX_MODE_SHARED_COV:
 * every step first reruns every model's covariance pass (side by side on 16
 * internal streams, joined back into stream) and re-copies the tables. */
int aux_batch_set_mode(aux_batch *b, int32_t mode);

/* n_iters MCMC iterations of every chain of every model, stream-ordered and
 * asynchronous, capturable in a CUDA graph (the iteration is read from device
 * memory). accept_count: device [total chains] uint32 incremented on
 * acceptance, or NULL; log_alpha: device [total chains] double, or NULL;
 * chains are numbered model by model. Per-chain status words go to each
 * model's handle (aux_get_status). */
int aux_batch_step(aux_batch *b, int32_t n_iters, uint32_t *accept_count, double *log_alpha, void *stream);

/* Launch shape: warps per CTA (4, 8 or 16), CTAs per SM (0: as many as fit),
 * item order within a pass (0: longest series first, 1: shortest first) and
 * the block length factor of each width class (padded width <= 8, 16, 32,
 * 64): L = round(f sqrt(T)), f snapped to {0.5, 1, 2}; NULL keeps them.
 * Rebuilds the work list and block tables (synchronises stream). */
int aux_batch_set_config(aux_batch *b, int32_t warps_per_cta, int32_t ctas_per_sm, int32_t order,
                         const double *block_factor, void *stream);
/* The current shape; block_factor: [4] or NULL; block_len: [n_models] or NULL. */
int aux_batch_get_config(aux_batch *b, int32_t *warps_per_cta, int32_t *ctas_per_sm, int32_t *order,
                         double *block_factor, int32_t *block_len);

/* The autotuner: times `reps` steps (after one warm-up step) of each candidate
 * launch shape by coordinate descent (warps per CTA, CTAs per SM, item order,
 * then the block length factor of each width class present) and keeps the
 * fastest; best_ms (host, or NULL) receives its time per step. The states
 * x[i] and the iteration counter are restored afterwards (it allocates one
 * temporary copy of the states); accept counts are untouched. Synchronous;
 * AUX_E_UNSUPPORTED under stream capture. */
int aux_batch_tune(aux_batch *b, int32_t reps, void *stream, double *best_ms);

/* The device iteration counter (set: synchronises stream). */
int aux_batch_set_iteration(aux_batch *b, uint64_t iteration, void *stream);
int aux_batch_get_iteration(aux_batch *b, uint64_t *iteration);

/* Synchronous check: AUX_E_TIMEOUT if a device wait ran out (aborted, when
 * not NULL, receives 1), else AUX_E_NOT_PD / AUX_E_NONFINITE if some chain's
 * status word is set, else AUX_OK. */
int aux_batch_get_status(aux_batch *b, int32_t *aborted);

/* Release the batch (synchronises the device); the models are untouched. */
void aux_batch_free(aux_batch *b);

/* Release the handle and its device memory (synchronises). NULL is a no-op. */
void aux_free_model(aux_model *m);

/* Static string for a status code. */
const char *aux_status_string(int code);

#ifdef __cplusplus
}
#endif
#endif /* AUX_KALMAN_H */
