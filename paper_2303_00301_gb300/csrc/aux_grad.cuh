// aux_grad.cuh — gradient of the auxiliary LGSSM log-likelihood with respect to
// theta = (mu, phi, L, delta) of the multivariate SV model (Section 4.1:
// F = diag(phi), b = (I - F) mu, Q = L L^T, stationary p_0, R = (delta/2) I),
// pseudo-observations ytilde held fixed.
//
// The paper differentiates with automatic differentiation; here the gradient
// is Fisher's identity, grad log p(y | theta) = E[grad log p(x, y | theta) | y],
// evaluated with the smoothed moments of the auxiliary LGSSM. The smoother is
// the parallel backward scan of Appendix A.2.2 run on the noise-free backward
// elements (G_t, u_t = m^f_t - G_t m^p_{t+1}, Sigma_t) with the operator
// (G_i, u_i, S_i) o (G_j, u_j, S_j) = (G_i G_j, G_i u_j + u_i, G_i S_j G_i^T + S_i)
// (the smoothed covariance obeys P^s_t = G_t P^s_{t+1} G_t^T + Sigma_t):
//   k_smooth_reduce  block aggregates of (G, u, Sigma) — one warp per (chain, block)
//   k_smooth_apply   per block, the state at the block's end from the later
//                    aggregates, then the backward sweep m^s_t, P^s_t and the
//                    lag-one cross-covariance C_{t+1} = P^s_{t+1} G_t^T, with the
//                    per-block sums of the complete-data score statistics
//   k_grad_final     per chain (FP64): sums over blocks and the gradient.
#pragma once
#include "aux_kernels.cuh"

namespace auxk {

template <typename Real> struct SmoothArgs {
  const Real* G;      // [C][T][DP*DP]
  const Real* U;      // [C][T][DP] (noise-free)
  const Real* Sig;    // [C][T][DP*DP]
  const Real* yt;     // [C][T][d]
  Real* sgu;          // [C][nb][SGS]: G^ rows, S^ rows, u^
  Real* gpart;        // [C][nb][SGS]: M rows, D rows, sum of e-bar
  double* opart;      // [C][nb]: sum |ytilde - m^s|^2 + tr P^s
  Real* s0;           // [C][DP*DP + DP]: S0 rows, a_0
  BlockRange rg;      // blocks to run; indexing of G, U, Sig (G, U, Sig hold the range only)
};

template <typename Real, int DP> struct GradSizes {
  static constexpr int MAT = Lay<Real, DP>::MAT, VEC = Lay<Real, DP>::VEC;
  static constexpr int SGS = 2 * DP * DP + DP;
  static constexpr int WPC = 8;
  static constexpr int RED_WARP_ELEMS = 5 * MAT + VEC;
  static constexpr size_t RED_SMEM = (size_t)WPC * RED_WARP_ELEMS * sizeof(Real);
  static constexpr int APP_WARP_ELEMS = 4 * MAT + 4 * VEC;
  static constexpr size_t APP_SMEM = (size_t)(2 * VEC + WPC * APP_WARP_ELEMS) * sizeof(Real);
};

template <typename Real, int DP>
__global__ void __launch_bounds__(32 * GradSizes<Real, DP>::WPC)
    k_smooth_reduce(KP<Real> p, SmoothArgs<Real> a) {
  using Z = GradSizes<Real, DP>;
  constexpr int MAT = Z::MAT, LD = Lay<Real, DP>::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = blockIdx.x * Z::WPC + warp;
  if (item >= p.C * a.rg.count(p.nb)) return;
  int c, k;
  a.rg.item(item, p.nb, c, k);
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  Real* SGh = sm + warp * Z::RED_WARP_ELEMS;
  Real* SGhT = SGh + MAT;
  Real* SGt = SGhT + MAT;
  Real* SSt = SGt + MAT;
  Real* SW = SSt + MAT;
  Real* vu = SW + MAT;
  Real gi[DP], sigh[DP];
#pragma unroll
  for (int j = 0; j < DP; ++j) { gi[j] = (j == lane) ? (Real)1 : (Real)0; sigh[j] = (Real)0; }
  st_row<Real, DP>(SGh, row, gi, act);
  st_row<Real, DP>(SGhT, row, gi, act);
  Real uh = 0;
  for (int t = s; t <= e; ++t) {
    const long ct = a.rg.ct(c, t, p.nT);
    Real r[DP];
    __syncwarp();
    ld_vec<Real, DP>(a.G + ct * DP * DP + row * DP, r);
    st_row<Real, DP>(SGt, row, r, act);
    ld_vec<Real, DP>(a.Sig + ct * DP * DP + row * DP, r);
    st_row<Real, DP>(SSt, row, r, act);
    if (act) vu[lane] = a.U[ct * DP + lane];
    __syncwarp();
    {
      Real w[DP];
      mm_row<Real, DP>(SGh + row * LD, SSt, w);      // (G^ Sigma_t) row
      st_row<Real, DP>(SW, row, w, act);
    }
    __syncwarp();
    mm_row<Real, DP, true>(SW + row * LD, SGhT, sigh);   // S^ += G^ Sigma_t G^T
    uh += dot_row_vec<Real, DP>(SGh + row * LD, vu);     // u^ += G^ u_t
    Real gn[DP];
    mm_row<Real, DP>(SGh + row * LD, SGt, gn);           // G^ <- G^ G_t
    __syncwarp();
    st_row<Real, DP>(SGh, row, gn, act);
    st_col<Real, DP>(SGhT, row, gn, act);
  }
  __syncwarp();
  Real* out = a.sgu + ((long)c * p.nb + k) * Z::SGS;
  if (act) {
    Real r[DP];
    ld_row<Real, DP>(SGh, row, r);
    st_vec<Real, DP>(out + row * DP, r);
    st_vec<Real, DP>(out + DP * DP + row * DP, sigh);
    out[2 * DP * DP + lane] = uh;
  }
}

template <typename Real, int DP>
__global__ void __launch_bounds__(32 * GradSizes<Real, DP>::WPC)
    k_smooth_apply(KP<Real> p, SmoothArgs<Real> a) {
  using Z = GradSizes<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC, LD = Lay<Real, DP>::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  Real* sphi = sm;            // diag F
  Real* smu = sm + VEC;       // mu = m0
  if (threadIdx.x < DP) {
    sphi[threadIdx.x] = p.F[threadIdx.x * DP + threadIdx.x];
    smu[threadIdx.x] = p.m0[threadIdx.x];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = blockIdx.x * Z::WPC + warp;
  if (item >= p.C * a.rg.count(p.nb)) return;
  int c, k;
  a.rg.item(item, p.nb, c, k);
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  Real* SP = sm + 2 * VEC + warp * Z::APP_WARP_ELEMS;
  Real* SGt = SP + MAT;
  Real* SGtT = SGt + MAT;
  Real* SCr = SGtT + MAT;
  Real* vm = SCr + MAT;
  Real* va = vm + VEC;
  Real* ve = va + VEC;
  Real* vu = ve + VEC;
  const Real phi_i = sphi[row], mu_i = smu[row];
  // smoothed (m, P) at the first state of the next block
  if (k < p.nb - 1) {
    const Real* gl = a.sgu + ((long)c * p.nb + p.nb - 1) * Z::SGS;
    Real r[DP];
    ld_vec<Real, DP>(gl + DP * DP + row * DP, r);
    st_row<Real, DP>(SP, row, r, act);
    if (act) vm[lane] = gl[2 * DP * DP + lane];
    for (int kk = p.nb - 2; kk > k; --kk) {
      const Real* gk = a.sgu + ((long)c * p.nb + kk) * Z::SGS;
      __syncwarp();
      ld_vec<Real, DP>(gk + row * DP, r);
      st_row<Real, DP>(SGt, row, r, act);
      __syncwarp();
      const Real mi = dot_row_vec<Real, DP>(SGt + row * LD, vm) + gk[2 * DP * DP + row];
      Real v[DP];
      mm_row<Real, DP>(SGt + row * LD, SP, v);        // V = G^ P (row)
      st_col<Real, DP>(SGtT, row, v, act);             // SGtT = V^T
      __syncwarp();
      Real pn[DP];
      ld_vec<Real, DP>(gk + DP * DP + row * DP, pn);
      mm_row<Real, DP, true>(SGt + row * LD, SGtT, pn);  // G^ P G^T + S^
      __syncwarp();
      st_row<Real, DP>(SP, row, pn, act);
      if (act) vm[lane] = mi;
    }
  }
  Real Mr[DP], Dr[DP];
  zero<Real, DP>(Mr);
  zero<Real, DP>(Dr);
  Real esum = 0;
  double O = 0.0;
  Real ph[DP];
  ld_vec<Real, DP>(sphi, ph);
  for (int t = e; t >= s; --t) {
    const long ct = a.rg.ct(c, t, p.nT);        // G, U, Sigma
    const long cy = (long)c * p.nT + t;          // ytilde
    __syncwarp();
    if (t == p.nT - 1) {
      Real r[DP];
      ld_vec<Real, DP>(a.Sig + ct * DP * DP + row * DP, r);
      st_row<Real, DP>(SP, row, r, act);
      if (act) vm[lane] = a.U[ct * DP + lane];
    } else {
      Real g[DP];
      ld_vec<Real, DP>(a.G + ct * DP * DP + row * DP, g);
      st_row<Real, DP>(SGt, row, g, act);
      st_col<Real, DP>(SGtT, row, g, act);
      if (act) vu[lane] = a.U[ct * DP + lane];
      __syncwarp();
      Real cr[DP];
      mm_row<Real, DP>(SP + row * LD, SGtT, cr);        // C_{t+1} = P_{t+1} G_t^T
      st_row<Real, DP>(SCr, row, cr, act);
      __syncwarp();
      Real pn[DP];
      ld_vec<Real, DP>(a.Sig + ct * DP * DP + row * DP, pn);
      mm_row<Real, DP, true>(SGt + row * LD, SCr, pn);  // P_t = G_t C_{t+1} + Sigma_t
      const Real mt = dot_row_vec<Real, DP>(SGt + row * LD, vm) + vu[row];
      const Real at1 = vm[row] - mu_i, at = mt - mu_i;
      const Real eb = at1 - phi_i * at;
      if (act) { ve[lane] = eb; va[lane] = at; }
      __syncwarp();
      Real ev[DP], av[DP], pold[DP], ccol[DP];
      ld_vec<Real, DP>(ve, ev);
      ld_vec<Real, DP>(va, av);
      ld_row<Real, DP>(SP, row, pold);
      ld_col<Real, DP>(SCr, row, ccol);
#pragma unroll
      for (int j = 0; j < DP; ++j) {
        Mr[j] += eb * ev[j] + pold[j] - cr[j] * ph[j] - phi_i * ccol[j] + phi_i * pn[j] * ph[j];
        Dr[j] += eb * av[j] + cr[j] - phi_i * pn[j];
      }
      esum += eb;
      __syncwarp();
      st_row<Real, DP>(SP, row, pn, act);
      if (act) vm[lane] = mt;
    }
    __syncwarp();
    if (lane < p.d) {
      const Real r = a.yt[cy * p.d + lane] - vm[lane];
      O += (double)r * (double)r + (double)SP[lane * LD + lane];
    }
  }
  __syncwarp();
  if (k == 0) {
    const Real a0 = vm[row] - mu_i;
    if (act) va[lane] = a0;
    __syncwarp();
    Real av[DP], pr[DP];
    ld_vec<Real, DP>(va, av);
    ld_row<Real, DP>(SP, row, pr);
#pragma unroll
    for (int j = 0; j < DP; ++j) pr[j] += a0 * av[j];
    Real* s0 = a.s0 + (long)c * (DP * DP + DP);
    if (act) {
      st_vec<Real, DP>(s0 + row * DP, pr);
      s0[DP * DP + lane] = a0;
    }
  }
  const long ck = (long)c * p.nb + k;
  Real* gp = a.gpart + ck * Z::SGS;
  if (act) {
    st_vec<Real, DP>(gp + row * DP, Mr);
    st_vec<Real, DP>(gp + DP * DP + row * DP, Dr);
    gp[2 * DP * DP + lane] = esum;
  }
  O = warp_sum<double>(O);
  if (lane == 0) a.opart[ck] = O;
}

// FP64 constants of theta, unpadded: mu[d], phi[d], L[d*d], Q[d*d], Q^{-1}[d*d], P0^{-1}[d*d]
struct GradOut {
  double* g_mu;     // [C][d]
  double* g_phi;    // [C][d]
  double* g_L;      // [C][d][d]
  double* g_delta;  // [C]
};

template <typename Real, int DP>
__global__ void __launch_bounds__(256)
    k_grad_final(KP<Real> p, const Real* __restrict__ gpart, const double* __restrict__ opart,
                 const Real* __restrict__ s0, const double* __restrict__ gc, double delta,
                 GradOut out) {
  const int c = blockIdx.x, d = p.d, nb = p.nb;
  constexpr int SGS = GradSizes<Real, DP>::SGS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* M = reinterpret_cast<double*>(smem_raw);
  double* D = M + d * d;
  double* S0 = D + d * d;
  double* A = S0 + d * d;          // scratch
  double* B = A + d * d;           // scratch
  double* es = B + d * d;
  double* a0 = es + d;
  double* red = a0 + d;            // 32
  const double* mu = gc;
  const double* phi = mu + d;
  const double* L = phi + d;
  const double* Q = L + d * d;
  const double* Qi = Q + d * d;
  const double* P0i = Qi + d * d;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int q = tid; q < d * d; q += nt) {
    const int i = q / d, j = q % d;
    double m = 0.0, dd = 0.0;
    for (int k = 0; k < nb; ++k) {
      const Real* gp = gpart + ((long)c * nb + k) * SGS;
      m += (double)gp[i * DP + j];
      dd += (double)gp[DP * DP + i * DP + j];
    }
    M[q] = m;
    D[q] = dd;
    S0[q] = (double)s0[(long)c * (DP * DP + DP) + i * DP + j];
  }
  for (int i = tid; i < d; i += nt) {
    double e = 0.0;
    for (int k = 0; k < nb; ++k) e += (double)gpart[((long)c * nb + k) * SGS + 2 * DP * DP + i];
    es[i] = e;
    a0[i] = (double)s0[(long)c * (DP * DP + DP) + DP * DP + i];
  }
  double o = 0.0;
  for (int k = tid; k < nb; k += nt) o += opart[(long)c * nb + k];
  o = warp_sum<double>(o);
  if ((tid & 31) == 0) red[tid >> 5] = o;
  __syncthreads();
  // A = P0^{-1} S0
  for (int q = tid; q < d * d; q += nt) {
    const int i = q / d, j = q % d;
    double acc = 0.0;
    for (int k = 0; k < d; ++k) acc += P0i[i * d + k] * S0[k * d + j];
    A[q] = acc;
  }
  __syncthreads();
  // B = Gamma = (A P0^{-1} - P0^{-1}) / 2
  for (int q = tid; q < d * d; q += nt) {
    const int i = q / d, j = q % d;
    double acc = 0.0;
    for (int k = 0; k < d; ++k) acc += A[i * d + k] * P0i[k * d + j];
    B[q] = 0.5 * (acc - P0i[q]);
  }
  __syncthreads();
  // g_mu, g_phi
  for (int i = tid; i < d; i += nt) {
    double qe = 0.0, pa = 0.0, qd = 0.0, gp = 0.0;
    for (int k = 0; k < d; ++k) {
      qe += Qi[i * d + k] * es[k];
      pa += P0i[i * d + k] * a0[k];
      qd += Qi[i * d + k] * D[k * d + i];
      const double w = 1.0 - phi[i] * phi[k];
      gp += B[i * d + k] * Q[i * d + k] * phi[k] / (w * w);
    }
    out.g_mu[(long)c * d + i] = (1.0 - phi[i]) * qe + pa;
    out.g_phi[(long)c * d + i] = qd + 2.0 * gp;
  }
  // A = Q^{-1} M
  for (int q = tid; q < d * d; q += nt) {
    const int i = q / d, j = q % d;
    double acc = 0.0;
    for (int k = 0; k < d; ++k) acc += Qi[i * d + k] * M[k * d + j];
    A[q] = acc;
  }
  __syncthreads();
  // S0 <- G_Q = -(T-1)/2 Q^{-1} + (A Q^{-1}) / 2 + Gamma / W  (S0 is no longer needed)
  for (int q = tid; q < d * d; q += nt) {
    const int i = q / d, j = q % d;
    double acc = 0.0;
    for (int k = 0; k < d; ++k) acc += A[i * d + k] * Qi[k * d + j];
    S0[q] = -0.5 * (p.nT - 1) * Qi[q] + 0.5 * acc + B[q] / (1.0 - phi[i] * phi[j]);
  }
  __syncthreads();
  // g_L = tril(2 G_Q L)
  for (int q = tid; q < d * d; q += nt) {
    const int i = q / d, j = q % d;
    double acc = 0.0;
    if (j <= i)
      for (int k = j; k < d; ++k) acc += S0[i * d + k] * L[k * d + j];
    out.g_L[(long)c * d * d + q] = (j <= i) ? 2.0 * acc : 0.0;
  }
  if (tid == 0) {
    double ot = 0.0;
    for (int w = 0; w < (nt + 31) / 32; ++w) ot += red[w];
    out.g_delta[c] = -(double)p.nT * d / (2.0 * delta) + ot / (delta * delta);
  }
}

}  // namespace auxk
