// aux_wide.cuh — the table modes (a covariance pass shared by all chains, then
// per-chain means) for padded dimensions 64 and 128.
//
// The narrow kernels give each row of a DP x DP matrix to one lane of a warp,
// which holds for DP <= 32 only. Here every dense step is a CTA-level routine
// of WT threads on matrices in global memory (L2-resident working sets):
//   w_gemm    C = alpha op(A) op(B) + beta C0, k-chunks staged in shared memory,
//             (DP/16)^2 outputs per thread;
//   w_chol    right-looking Cholesky in shared memory, blocks of 8 columns
//             (three barriers per block);
//   w_trinv   the inverse of the triangular factor, blocked by 32 (diagonal
//             blocks on separate warps, then each panel as one product pair).
// Covariance pass (homogeneous dynamics, R = r I, Appendix A.2.1 elements):
//   k_w_elem    the two distinct elements: t = 0, (0, C_0, 0), and every t >= 1,
//               (A, C, J), with S = Q + R:  A = r S^{-1} F, C = Q - Q S^{-1} Q,
//               J = F^T S^{-1} F; the prefix of t = 0 is its own C_0;
//   k_w_double  prefixes by doubling at step granularity: the prefix of t has
//               A = 0 and J = 0 (the first element has both zero), so
//               P_t = P_{t - 2^k} (x) E^(2^k) needs the C part only,
//               C = C_e + A_e B B^T A_e^T with B = U chol(N)^{-T}, U = chol(C_i),
//               N = I + U^T J_e U (SPD, eigenvalues >= 1); one CTA also squares
//               E^(2^k) with the full operator for the next level;
//   k_w_epi     per step, from P^f_{t-1} and P^f_t (embarrassingly parallel):
//               P^p_t, S_t, K'_t = r S_t^{-1}, log det S_t, and the backward
//               quantities of step t - 1, G = P^f F^T (P^p)^{-1} and
//               chol(Sigma), Sigma = P^f - G P^p G^T = P^f - W W^T with
//               W = (chol(P^p)^{-1} F P^f)^T;
//   k_w_prod    per means block, M_e ... M_s (M_t = K'_t F), G_s ... G_e and the
//               sum of log det S_t.
// Tables read by the means kernels with one row index per thread are stored
// transposed (G^T, chol(Sigma)^T, the block products), so that a warp reads
// consecutive entries; K' and P^f are symmetric.
// Means (one CTA per block and group of chains, thread = (row, chain slot)):
//   k_wmf_reduce, k_wmean_cross, k_wmf_apply, k_wmb_apply: the recursions of
//   aux_means.cuh (filtering means, cross-block composition, likelihood
//   terms, backward elements U_t and the block aggregate of the (G, U) scan,
//   backward sampling with the MH terms); the block aggregate
//   sum_t (G_s ... G_{t-1}) U_t is formed by Horner's rule backwards over the
//   block instead of from a table of prefix products.
#pragma once
#include "aux_means.cuh"

namespace auxk {

constexpr int WT = 256;          // threads of every wide kernel
constexpr int W_SLOTS_PER_SM = 2;  // CTAs with their own scratch: 2 per SM of the device
constexpr int W_SCR = 8;         // scratch matrices per slot
// chains per thread in the means kernels (8 chains per CTA at DP = 128, 16 at 64)
template <int DP> constexpr int WCPT = 4;

// k-chunk and shared-memory layout of the tensor-core product (w_gemm_tc, below)
constexpr int TCK = 32;   // k per staged chunk
template <int DP> struct TcSz {
  static constexpr int LK = TCK + 4;     // row stride of a chunk stored k-contiguous
  static constexpr int LM = DP + 8;      // row stride of a chunk stored m/n-contiguous
  static constexpr int CH = (DP * LK > TCK * LM ? DP * LK : TCK * LM);   // floats per operand chunk
  static constexpr size_t SMEM = 2 * (size_t)CH * sizeof(float);
  static constexpr int MT = DP / 64, NT = DP / 16;   // m16 and n8 tiles per warp
};

template <typename Real, int DP> struct WSz {
  static constexpr int LDS = DP + 1;                 // shared row stride (odd: column access is conflict-free)
  static constexpr int KC = 32;                      // k-chunk of w_gemm
  static constexpr int R = DP / 16;                  // outputs per thread and dimension in w_gemm
  static constexpr int NRG = WT / DP;                // row groups of the means kernels
  static constexpr int CPC = NRG * WCPT<DP>;            // chains per CTA of the means kernels
  static constexpr long DD = (long)DP * DP;
  static constexpr size_t FULL = (size_t)DP * LDS;   // one padded matrix
  // one padded matrix (factor, inverted in place) or the two k-chunks of w_gemm; the
  // pivots (FP64) and a column (two CTAs per SM at DP = 128)
  static constexpr size_t GEMM = 2 * (size_t)KC * LDS;
  // bytes of the working area: the factor slot, or the staged chunks of w_gemm / w_gemm_tc
  static constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
  static constexpr size_t WORK = cmax(cmax(FULL * sizeof(Real), GEMM * sizeof(Real)), TcSz<DP>::SMEM);
  static constexpr size_t SMEM = WORK + (2 * DP + 8) * sizeof(double);
  // the mixed-precision doubling: the working area holds one FP64 slot (the
  // factorisations of C_i and N); then the pivots and an FP64 column
  static constexpr size_t WORK_MX = cmax(FULL * sizeof(double), TcSz<DP>::SMEM);
  static constexpr size_t SMEM_MX = WORK_MX + (2 * DP + 8) * sizeof(double) + DP * sizeof(double);
  // matrix staging buffers of the means kernels (one copy in flight while one is read)
  static constexpr int NBUF = 2;
  // means: NBUF matrix staging buffers, three vector slots per chain, per-chain FP64 sums
  static constexpr int WPG = DP / 32;   // warps per row group
  static constexpr size_t MSMEM = (size_t)(NBUF * DD + 3 * CPC * DP) * sizeof(Real) + (size_t)CPC * WPG * sizeof(double);
  // composition over the blocks: the staging buffers, two vector slots
  static constexpr size_t XSMEM = (size_t)(NBUF * DD + 2 * DP) * sizeof(Real);
};

// ---------------------------------------------------------------------------
// CTA-level dense routines. Matrices are DP x DP, row-major, in global memory;
// every routine starts and ends with a CTA barrier, so that its outputs are
// visible to the whole CTA when it returns.
// ---------------------------------------------------------------------------
// C = alpha op(A) op(B) + beta C0 (+ I when addI), op = transpose for TA / TB.
// bscale: the rows of op(B) scaled by bscale[k] (a diagonal left factor of B).
// C may alias A, B or C0: every read of A and B precedes every store.
template <typename Real, int DP>
__device__ void w_gemm(const Real* A, bool ta, const Real* B, bool tb, Real* C, const Real* C0, Real alpha,
                       Real beta, Real* sm, const Real* bscale = nullptr, bool addI = false) {
  using Z = WSz<Real, DP>;
  constexpr int KC = Z::KC, LDS = Z::LDS, R = Z::R;
  Real* As = sm;              // As[kk][i] = op(A)[i][k0 + kk]
  Real* Bs = sm + KC * LDS;   // Bs[kk][j] = op(B)[k0 + kk][j]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  Real acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = (Real)0;
  for (int k0 = 0; k0 < DP; k0 += KC) {
    __syncthreads();
    for (int q = tid; q < DP * KC; q += WT) {
      if (!ta) {
        const int i = q / KC, kk = q % KC;
        As[kk * LDS + i] = A[(long)i * DP + k0 + kk];
      } else {
        const int kk = q / DP, i = q % DP;
        As[kk * LDS + i] = A[(long)(k0 + kk) * DP + i];
      }
      int kb, j;
      Real bv;
      if (!tb) {
        kb = q / DP; j = q % DP;
        bv = B[(long)(k0 + kb) * DP + j];
      } else {
        j = q / KC; kb = q % KC;
        bv = B[(long)j * DP + k0 + kb];
      }
      if (bscale) bv *= bscale[k0 + kb];
      Bs[kb * LDS + j] = bv;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KC; ++kk) {
      Real a[R], b[R];
#pragma unroll
      for (int i = 0; i < R; ++i) a[i] = As[kk * LDS + ty + 16 * i];
#pragma unroll
      for (int j = 0; j < R; ++j) b[j] = Bs[kk * LDS + tx + 16 * j];
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
  }
  __syncthreads();   // every read of A and B is done (C may alias them)
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int r = ty + 16 * i, c = tx + 16 * j;
      Real v = alpha * acc[i][j];
      if (beta != (Real)0) v = fma(beta, C0[(long)r * DP + c], v);
      if (addI && r == c) v += (Real)1;
      C[(long)r * DP + c] = v;
    }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// The same product on the tensor cores (mixed precision, AUX_MIXED):
// mma.sync m16n8k8 with TF32 operands and FP32 accumulation, each product
// split into three TF32 products, a_hi b_hi + a_hi b_lo + a_lo b_hi with
// x_hi = tf32(x) and x_lo = tf32(x - x_hi), so that the result keeps about
// single-precision accuracy. The 8 warps tile the DP x DP output 4 x 2
// (warp tile DP/4 x DP/2); k-chunks of TCK columns of op(A) and rows of op(B)
// are staged by cp.async in the layout that makes the fragment loads
// conflict-free: rows of length TCK (+4) when op(A) (op(B)) is read along k
// in memory, rows of length DP (+8) otherwise. Same contract as w_gemm.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t tf32_of(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_of(x);
  lo = tf32_of(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// stage chunk k0 of op(X) (X row-major DP x DP): k-contiguous rows (kmajor: element
// (m, kk) at m * LK + kk, read from X[m][k0 + kk]) or m-contiguous rows (element
// (kk, m) at kk * LM + m, read from X[k0 + kk][m])
template <int DP>
__device__ __forceinline__ void tc_stage(float* dst, const float* X, int k0, bool kmajor) {
  using Z = TcSz<DP>;
  if (kmajor) {
    constexpr int CPR = TCK / 4;
    for (int q = threadIdx.x; q < DP * CPR; q += WT) {
      const int m = q / CPR, c = q % CPR;
      cp_async16(dst + m * Z::LK + c * 4, X + (long)m * DP + k0 + c * 4);
    }
  } else {
    constexpr int CPR = DP / 4;
    for (int q = threadIdx.x; q < TCK * CPR; q += WT) {
      const int kk = q / CPR, c = q % CPR;
      cp_async16(dst + kk * Z::LM + c * 4, X + (long)(k0 + kk) * DP + c * 4);
    }
  }
  cp_async_commit();
}

template <int DP>
__device__ void w_gemm_tc(const float* A, bool ta, const float* B, bool tb, float* C, const float* C0, float alpha,
                          float beta, float* sm, const float* bscale = nullptr, bool addI = false) {
  using Z = TcSz<DP>;
  constexpr int MT = Z::MT, NT = Z::NT, LK = Z::LK, LM = Z::LM;
  float* As = sm;
  float* Bs = sm + Z::CH;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int m0 = (warp >> 1) * (DP / 4), n0 = (warp & 1) * (DP / 2);
  // op(A)[i][k] = A[i][k] (k-contiguous) or A[k][i]; op(B)[k][j] = B[k][j] (j-contiguous) or B[j][k]
  const bool akm = !ta, bkm = tb;
  float acc[MT][NT][4];
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  for (int k0 = 0; k0 < DP; k0 += TCK) {
    __syncthreads();   // the previous chunk is consumed
    tc_stage<DP>(As, A, k0, akm);
    tc_stage<DP>(Bs, B, k0, bkm);
    cp_async_wait<0>();
    __syncthreads();
#pragma unroll 1
    for (int ks = 0; ks < TCK; ks += 8) {
      uint32_t ah[MT][4], al[MT][4];
#pragma unroll
      for (int i = 0; i < MT; ++i) {
        const int r0 = m0 + i * 16 + g;
        float av[4];
        if (akm) {
          av[0] = As[r0 * LK + ks + t];
          av[1] = As[(r0 + 8) * LK + ks + t];
          av[2] = As[r0 * LK + ks + t + 4];
          av[3] = As[(r0 + 8) * LK + ks + t + 4];
        } else {
          av[0] = As[(ks + t) * LM + r0];
          av[1] = As[(ks + t) * LM + r0 + 8];
          av[2] = As[(ks + t + 4) * LM + r0];
          av[3] = As[(ks + t + 4) * LM + r0 + 8];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) tf32_split(av[q], ah[i][q], al[i][q]);
      }
      float s0 = 1.f, s1 = 1.f;
      if (bscale) {
        s0 = bscale[k0 + ks + t];
        s1 = bscale[k0 + ks + t + 4];
      }
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const int c = n0 + j * 8 + g;
        float b0, b1;
        if (bkm) {
          b0 = Bs[c * LK + ks + t];
          b1 = Bs[c * LK + ks + t + 4];
        } else {
          b0 = Bs[(ks + t) * LM + c];
          b1 = Bs[(ks + t + 4) * LM + c];
        }
        b0 *= s0;
        b1 *= s1;
        uint32_t bh0, bl0, bh1, bl1;
        tf32_split(b0, bh0, bl0);
        tf32_split(b1, bh1, bl1);
#pragma unroll
        for (int i = 0; i < MT; ++i) {
          mma_tf32(acc[i][j], al[i], bh0, bh1);
          mma_tf32(acc[i][j], ah[i], bl0, bl1);
          mma_tf32(acc[i][j], ah[i], bh0, bh1);
        }
      }
    }
  }
  __syncthreads();   // every read of A and B is done (C may alias them)
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = m0 + i * 16 + g + 8 * h, c = n0 + j * 8 + 2 * t;
        float v0 = alpha * acc[i][j][2 * h], v1 = alpha * acc[i][j][2 * h + 1];
        if (beta != 0.f) {
          v0 = fmaf(beta, C0[(long)r * DP + c], v0);
          v1 = fmaf(beta, C0[(long)r * DP + c + 1], v1);
        }
        if (addI) {
          if (r == c) v0 += 1.f;
          if (r == c + 1) v1 += 1.f;
        }
        *reinterpret_cast<float2*>(C + (long)r * DP + c) = make_float2(v0, v1);
      }
  __syncthreads();
}

// out = alpha * X (+ beta * Y) elementwise, optionally transposed X (out must not alias X then)
template <typename Real, int DP>
__device__ void w_axpby(const Real* X, bool tx, Real alpha, const Real* Y, Real beta, Real* out) {
  __syncthreads();
  for (int q = threadIdx.x; q < DP * DP; q += WT) {
    const int i = q / DP, j = q % DP;
    Real v = alpha * (tx ? X[(long)j * DP + i] : X[q]);
    if (Y) v = fma(beta, Y[q], v);
    out[q] = v;
  }
  __syncthreads();
}

// symmetric part (X + X^T) / 2 into out (out must not alias X)
template <typename Real, int DP>
__device__ void w_sym(const Real* X, Real* out) {
  __syncthreads();
  for (int q = threadIdx.x; q < DP * DP; q += WT) {
    const int i = q / DP, j = q % DP;
    out[q] = (Real)0.5 * (X[q] + X[(long)j * DP + i]);
  }
  __syncthreads();
}

// Lower Cholesky factor of the symmetric (A + addiag I) into the shared slot S
// (row-major, stride LDS, zero above the diagonal). Rows and columns >= d are
// the identity (the padding). A pivot below d that is not positive and finite
// sets *bad and is replaced by 1. Returns sum_{k<d} log L_kk in thread 0 (the
// only thread that uses it; warp 0 sums the FP64 logarithms, a few per lane).
// piv: DP + 8 doubles of shared scratch. The FP64 work per call is DP square
// roots and DP logarithms in all: on this GPU FP64 runs at a small fraction of
// the FP32 rate, so every thread doing its own would dominate the routine.
// Elimination without square roots (S_ik becomes L_ik sqrt(p_k), p_k the
// pivots), right-looking in blocks of 8 columns with three CTA barriers per
// block instead of one per column:
//   (a) the block's 8 x 8 diagonal part, lanes 0..7 of warp 0 (lane = row,
//       column entries by shuffles), its pivots and their reciprocals;
//   (b) the panel below it, one thread per row, row-local:
//       S_i,k+c -= sum_{c'<c} (S_i,k+c' / p_k+c') S_k+c,k+c';
//   (c) the rank-8 update of the trailing rows,
//       S_ij -= sum_c (S_i,k+c / p_k+c) S_j,k+c  (k + 8 <= j <= i < d),
//       each thread some columns of one row, the 8 multipliers of its row in
//       registers.
template <typename Real, int DP, typename SlotT = Real>
__device__ double w_chol(const Real* A, Real addiag, int d, SlotT* S, double* piv, int* bad) {
  using Z = WSz<Real, DP>;
  constexpr int LDS = Z::LDS, P = WT / DP, NK = 8;
  static_assert(WT % DP == 0, "every thread keeps one column in the scaling pass");
  static_assert(DP % NK == 0 && WT >= DP, "blocks of 8 columns, one thread per panel row");
  __syncthreads();
  for (int q = threadIdx.x; q < DP * DP; q += WT) {
    const int i = q / DP, j = q % DP;
    SlotT v;
    if (i >= d || j >= d) v = (i == j) ? (SlotT)1 : (SlotT)0;
    else v = (SlotT)A[q] + (i == j ? (SlotT)addiag : (SlotT)0);
    S[i * LDS + j] = v;
  }
  double* rinv = piv + DP;   // the current block's pivot reciprocals
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = threadIdx.x % DP, part = threadIdx.x / DP;
  for (int k = 0; k < d; k += NK) {
    __syncthreads();
    if (warp == 0) {   // (a)
      const int r = lane < NK ? lane : 0;
      SlotT w[NK];
#pragma unroll
      for (int c = 0; c < NK; ++c) w[c] = (c <= r) ? S[(k + r) * LDS + k + c] : (SlotT)0;
#pragma unroll
      for (int c = 0; c < NK; ++c) {
        SlotT pc = __shfl_sync(FULL_MASK, w[c], c);
        const bool ok = pc > (SlotT)0 && pc < (SlotT)INFINITY;
        if (!ok) pc = (SlotT)1;
        const SlotT ic = (SlotT)1 / pc;
        if (lane == 0) {
          piv[k + c] = (double)pc;
          rinv[c] = (double)ic;
          if (!ok && k + c < d) *bad = 1;
        }
        const SlotT l = w[c] * ic;
#pragma unroll
        for (int c2 = c + 1; c2 < NK; ++c2) {
          const SlotT wc = __shfl_sync(FULL_MASK, w[c], c2);   // S_k+c2,k+c
          if (lane > c && c2 <= r) w[c2] = fma(-l, wc, w[c2]);
        }
        if (lane == c) w[c] = pc;
      }
      if (lane < NK) {
#pragma unroll
        for (int c = 0; c < NK; ++c)
          if (c <= lane) S[(k + lane) * LDS + k + c] = w[c];
      }
    }
    __syncthreads();
    {   // (b)
      const int ip = k + NK + (int)threadIdx.x;
      if (ip < d) {
        SlotT* Si = S + ip * LDS + k;
        SlotT x[NK];
#pragma unroll
        for (int c = 0; c < NK; ++c) x[c] = Si[c];
#pragma unroll
        for (int c = 0; c < NK; ++c) {
          const SlotT l = x[c] * (SlotT)rinv[c];
#pragma unroll
          for (int c2 = c + 1; c2 < NK; ++c2) x[c2] = fma(-l, S[(k + c2) * LDS + k + c], x[c2]);
        }
#pragma unroll
        for (int c = 0; c < NK; ++c) Si[c] = x[c];
      }
    }
    __syncthreads();
    if (i >= k + NK && i < d) {   // (c)
      SlotT li[NK];
      SlotT* Srow = S + i * LDS;
#pragma unroll
      for (int c = 0; c < NK; ++c) li[c] = Srow[k + c] * (SlotT)rinv[c];
      for (int j = k + NK + part; j <= i; j += P) {
        const SlotT* Sj = S + j * LDS + k;
        SlotT acc = Srow[j];
#pragma unroll
        for (int c = 0; c < NK; ++c) acc = fma(-li[c], Sj[c], acc);
        Srow[j] = acc;
      }
    }
  }
  __syncthreads();
  // scale: L_ik = S_ik / sqrt(p_k) (i > k), L_kk = sqrt(p_k); zero above the diagonal.
  // Thread t only touches column t mod DP: one square root per thread.
  {
    const int c = threadIdx.x % DP;
    const SlotT sp = c < d ? (SlotT)sqrt(piv[c]) : (SlotT)1;
    const SlotT isp = (SlotT)1 / sp;
    for (int r = threadIdx.x / DP; r < DP; r += P) {
      if (c >= d) { S[r * LDS + c] = (r == c) ? (SlotT)1 : (SlotT)0; continue; }
      SlotT v = (SlotT)0;
      if (r == c) v = sp;
      else if (r > c) v = (sizeof(SlotT) == 4) ? S[r * LDS + c] / sp : S[r * LDS + c] * isp;
      S[r * LDS + c] = v;
    }
  }
  __syncthreads();
  double ld = 0.0;
  if (threadIdx.x < 32) {
    for (int k = threadIdx.x; k < d; k += 32) ld += 0.5 * log(piv[k]);
    ld = warp_sum<double>(ld);
  }
  return ld;
}

// One block column of the blocked inverse (w_trinv): rows r0 .. DP - 1 of block
// column jb (the panel P, still holding L) become -X P D, where X (rows and
// columns >= r0) and D (the diagonal block of jb) are already inverted. Thread
// (row, column group) keeps NC of the row's 32 outputs in registers; every
// read of a stage precedes its stores (a CTA barrier between them). The sums
// run over k up to the last row of the warp: X is zero above its diagonal.
template <typename Real, int DP, int TPR>
__device__ __forceinline__ void w_trinv_panel(Real* S, int jb) {
  constexpr int LDS = WSz<float, DP>::LDS, NC = 32 / TPR;
  const int r0 = 32 * (jb + 1), c0 = 32 * jb;
  const int rr = threadIdx.x / TPR, cg = threadIdx.x % TPR;
  const int r = r0 + rr;
  const bool act = r < DP;
  const int rlast = min(DP - 1, r0 + (int)((threadIdx.x | 31) / TPR));   // last row of this warp
  Real q[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) q[c] = (Real)0;
  if (act) {   // Q = X P
    const Real* Sr = S + r * LDS;
    for (int k = r0; k <= rlast; ++k) {
      const Real x = Sr[k];
      const Real* Lk = S + k * LDS + c0 + cg;
#pragma unroll
      for (int c = 0; c < NC; ++c) q[c] = fma(x, Lk[c * TPR], q[c]);
    }
  }
  __syncthreads();
  if (act) {
#pragma unroll
    for (int c = 0; c < NC; ++c) S[r * LDS + c0 + cg + c * TPR] = q[c];
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < NC; ++c) q[c] = (Real)0;
  if (act) {   // -Q D
    const Real* Qr = S + r * LDS + c0;
    const Real* D = S + c0 * LDS + c0 + cg;
#pragma unroll 4
    for (int k = 0; k < 32; ++k) {
      const Real x = Qr[k];
#pragma unroll
      for (int c = 0; c < NC; ++c) q[c] = fma(x, D[k * LDS + c * TPR], q[c]);
    }
  }
  __syncthreads();
  if (act) {
#pragma unroll
    for (int c = 0; c < NC; ++c) S[r * LDS + c0 + cg + c * TPR] = -q[c];
  }
}

// L^{-1} in place of the lower-triangular L in the shared slot S (zero above
// the diagonal), blocked by 32:
// (1) the diagonal blocks inverted side by side, warp w on block w, lane = row,
//     by columns from the last: with the block's trailing columns inverted,
//     (L^{-1})_jj = 1 / L_jj, (L^{-1})_ij = -(1 / L_jj) sum_{k=j+1..i} (L^{-1})_ik L_kj (i > j),
//     one warp barrier per column;
// (2) the block columns from the second last to the first: from X L = I, the
//     blocks below the diagonal are X_(i,jb) = -(sum_{k=jb+1..i} X_(i,k) L_(k,jb)) X_(jb,jb)
//     (w_trinv_panel), a few CTA barriers per block column.
// col: DP elements of shared scratch (the old column j, 32 per diagonal block).
template <typename Real, int DP>
__device__ void w_trinv(Real* S, Real* col) {
  constexpr int LDS = WSz<float, DP>::LDS, NB = DP / 32;
  static_assert(DP % 32 == 0 && WT >= 32 * NB && WT % 32 == 0, "one warp per diagonal block");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (warp < NB) {
    Real* B = S + (32 * warp) * LDS + 32 * warp;
    Real* cw = col + 32 * warp;
    Real* Bi = B + lane * LDS;
    for (int j = 31; j >= 0; --j) {
      __syncwarp();
      cw[lane] = Bi[j];
      __syncwarp();
      const Real ajj = (Real)1 / cw[j];
      if (lane > j) {
        Real a0 = (Real)0, a1 = (Real)0;
        int k = j + 1;
        for (; k + 1 <= lane; k += 2) {
          a0 = fma(Bi[k], cw[k], a0);
          a1 = fma(Bi[k + 1], cw[k + 1], a1);
        }
        if (k <= lane) a0 = fma(Bi[k], cw[k], a0);
        Bi[j] = -ajj * (a0 + a1);
      }
      if (lane == j) Bi[j] = ajj;
    }
  }
  for (int jb = NB - 2; jb >= 0; --jb) {
    __syncthreads();
    const int R = DP - 32 * (jb + 1);   // panel rows: 32, 64 or 96
    if (R <= WT / 8) w_trinv_panel<Real, DP, 8>(S, jb);
    else if (R <= WT / 4) w_trinv_panel<Real, DP, 4>(S, jb);
    else w_trinv_panel<Real, DP, 2>(S, jb);
  }
  __syncthreads();
}

// shared slot (stride LDS) -> global, optionally transposed
template <typename Real, int DP, typename SlotT = Real>
__device__ void w_store(const SlotT* S, Real* g, bool transpose) {
  constexpr int LDS = WSz<Real, DP>::LDS;
  __syncthreads();
  for (int q = threadIdx.x; q < DP * DP; q += WT) {
    const int i = q / DP, j = q % DP;
    g[q] = (Real)(transpose ? S[j * LDS + i] : S[i * LDS + j]);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Covariance pass
// ---------------------------------------------------------------------------
// the product of the covariance pass: CUDA-core FP32 (w_gemm) or, in the
// mixed-precision form, split-TF32 tensor cores (w_gemm_tc)
template <typename Real, int DP, bool MX>
__device__ __forceinline__ void w_mm(const Real* A, bool ta, const Real* B, bool tb, Real* C, const Real* C0,
                                     Real alpha, Real beta, Real* sm, const Real* bscale = nullptr,
                                     bool addI = false) {
  if constexpr (MX) w_gemm_tc<DP>(A, ta, B, tb, C, C0, alpha, beta, sm, bscale, addI);
  else w_gemm<Real, DP>(A, ta, B, tb, C, C0, alpha, beta, sm, bscale, addI);
}

template <typename Real> struct WCovArgs {
  Real* tab;          // [NTAB][T][DP][DP]: TK, TG^T, TLS^T, (unused), TPF
  Real* btab;         // [2][nb][DP][DP]: (M_e ... M_s)^T, (G_s ... G_e)^T per means block
  double* ldt;        // [T] log det S_t
  double* ld;         // [nb] per means block
  int32_t* status;    // [1] ST_NOT_PD
  Real* gk;           // [2][3][DP][DP] E^(2^k) (A, C, J), double-buffered
  Real* scr;          // [W_SLOTS_PER_SM * SMs][W_SCR][DP][DP]
};

template <typename Real, int DP>
__device__ __forceinline__ Real* w_slot(const WCovArgs<Real>& a, int s, int i) {
  return a.scr + ((long)s * W_SCR + i) * WSz<Real, DP>::DD;
}

// the distinct elements: prefix 0 = C_0 into TPF[0]; E = (A, C, J) into gk[0]
template <typename Real, int DP, bool MX>
__global__ void __launch_bounds__(WT, 2) k_w_elem(KP<Real> p, WCovArgs<Real> a) {
  refresh_delta(p);
  using Z = WSz<Real, DP>;
  constexpr long DD = Z::DD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* S0 = reinterpret_cast<Real*>(smem_raw);
  double* piv = reinterpret_cast<double*>(smem_raw + Z::WORK);
  Real* S1 = reinterpret_cast<Real*>(piv + DP + 8);   // a column
  Real* s0 = w_slot<Real, DP>(a, 0, 0);
  Real* s1 = w_slot<Real, DP>(a, 0, 1);
  Real* s2 = w_slot<Real, DP>(a, 0, 2);
  int bad = 0;
  const long tstride = (long)p.nT * DD;
  // t = 0: C_0 = P0 - P0 S0^{-1} P0 = r S0^{-1} P0 = r L^{-T} Y, Y = L^{-1} P0, L = chol(P0 + R)
  // (with R = r I, I - K = r S^{-1}: no difference of nearly equal matrices for small r)
  w_chol<Real, DP>(p.P0, p.r, p.d, S0, piv, &bad);
  w_trinv<Real, DP>(S0, S1);
  w_store<Real, DP>(S0, s0, false);
  w_mm<Real, DP, MX>(s0, false, p.P0, false, s1, nullptr, (Real)1, (Real)0, S0);
  w_mm<Real, DP, MX>(s0, true, s1, false, s2, nullptr, p.r, (Real)0, S0);
  w_sym<Real, DP>(s2, a.tab + (long)TPF * tstride);
  // t >= 1: S = Q + R = L L^T, Y = L^{-1} Q, W = L^{-1} F; C = r L^{-T} Y (symmetrised)
  Real* EA = a.gk;
  Real* EC = EA + DD;
  Real* EJ = EC + DD;
  w_chol<Real, DP>(p.Q, p.r, p.d, S0, piv, &bad);
  w_trinv<Real, DP>(S0, S1);
  w_store<Real, DP>(S0, s0, false);
  w_mm<Real, DP, MX>(s0, false, p.Q, false, s1, nullptr, (Real)1, (Real)0, S0);
  w_mm<Real, DP, MX>(s0, true, s1, false, s2, nullptr, p.r, (Real)0, S0);
  w_sym<Real, DP>(s2, EC);                                                            // C = r S^{-1} Q
  w_mm<Real, DP, MX>(s0, false, p.F, false, s2, nullptr, (Real)1, (Real)0, S0);  // W = L^{-1} F
  w_mm<Real, DP, MX>(s2, true, s2, false, EJ, nullptr, (Real)1, (Real)0, S0);    // J = W^T W
  w_mm<Real, DP, MX>(s0, true, s2, false, EA, nullptr, p.r, (Real)0, S0);        // A = r L^{-T} W
  if (bad && threadIdx.x == 0) atomicOr(a.status, ST_NOT_PD);
}

// C part of (0, C_i, 0) (x) (A_e, C_e, J_e) into out; with full (A_i, J_i also given,
// Ao / Jo not null) the whole operator. Scratch: slot s.
template <typename Real, int DP, bool MX>
__device__ void w_combine(const KP<Real>& p, const WCovArgs<Real>& a, int s, const Real* Ai, const Real* Ci,
                          const Real* Ji, const Real* Ae, const Real* Ce, const Real* Je, Real* Ao, Real* Co,
                          Real* Jo, Real* S0, Real* S1, double* piv, int* bad) {
  Real* U = w_slot<Real, DP>(a, s, 0);
  Real* X = w_slot<Real, DP>(a, s, 1);
  Real* N = w_slot<Real, DP>(a, s, 2);
  Real* B = w_slot<Real, DP>(a, s, 3);
  Real* Pm = w_slot<Real, DP>(a, s, 4);
  // the factorisations of C_i and of N = I + U^T J_e U, and the inverse of chol(N):
  // in FP64 in the mixed-precision form (the slot S0 then holds doubles)
  if constexpr (MX) {
    double* D0 = reinterpret_cast<double*>(S0);
    w_chol<Real, DP, double>(Ci, (Real)0, p.d, D0, piv, bad);            // U = chol(C_i)
    w_store<Real, DP, double>(D0, U, false);
  } else {
    w_chol<Real, DP>(Ci, (Real)0, p.d, S0, piv, bad);                    // U = chol(C_i)
    w_store<Real, DP>(S0, U, false);
  }
  w_mm<Real, DP, MX>(Je, false, U, false, X, nullptr, (Real)1, (Real)0, S0);         // J_e U
  w_mm<Real, DP, MX>(U, true, X, false, N, nullptr, (Real)1, (Real)0, S0, nullptr, true);   // N = I + U^T J_e U
  if constexpr (MX) {
    double* D0 = reinterpret_cast<double*>(S0);
    double* D1 = reinterpret_cast<double*>(S1);
    w_chol<Real, DP, double>(N, (Real)0, p.d, D0, piv, bad);
    w_trinv<double, DP>(D0, D1);
    w_store<Real, DP, double>(D0, N, false);                             // chol(N)^{-1}
  } else {
    w_chol<Real, DP>(N, (Real)0, p.d, S0, piv, bad);
    w_trinv<Real, DP>(S0, S1);
    w_store<Real, DP>(S0, N, false);                                      // chol(N)^{-1}
  }
  w_mm<Real, DP, MX>(U, false, N, true, B, nullptr, (Real)1, (Real)0, S0);           // B = U chol(N)^{-T}
  w_mm<Real, DP, MX>(Ae, false, B, false, Pm, nullptr, (Real)1, (Real)0, S0);        // P = A_e B
  if (Ao) {
    Real* X1 = w_slot<Real, DP>(a, s, 5);
    Real* Zm = w_slot<Real, DP>(a, s, 6);
    Real* Jt = w_slot<Real, DP>(a, s, 7);
    w_mm<Real, DP, MX>(Je, false, Ai, false, X1, nullptr, (Real)1, (Real)0, S0);     // X1 = J_e A_i
    w_mm<Real, DP, MX>(B, true, X1, false, Zm, nullptr, (Real)1, (Real)0, S0);       // Z = B^T X1
    w_mm<Real, DP, MX>(Ai, true, X1, false, Jt, Ji, (Real)1, (Real)1, S0);          // J_i + A_i^T X1
    w_mm<Real, DP, MX>(Zm, true, Zm, false, Jt, Jt, (Real)-1, (Real)1, S0);         // - Z^T Z
    w_sym<Real, DP>(Jt, Jo);
    w_mm<Real, DP, MX>(Ae, false, Ai, false, Ao, nullptr, (Real)1, (Real)0, S0);     // A_e A_i
    w_mm<Real, DP, MX>(Pm, false, Zm, false, Ao, Ao, (Real)-1, (Real)1, S0);        // - P Z
  }
  w_mm<Real, DP, MX>(Pm, false, Pm, true, Co, Ce, (Real)1, (Real)1, S0);            // C = C_e + P P^T
}

// one doubling level: prefixes TPF[pow2 + i] = TPF[i] (x) E^(pow2), i < cnt; item cnt
// (when sq): E^(2 pow2) = E^(pow2) (x) E^(pow2) into gk2
template <typename Real, int DP, bool MX>
__global__ void __launch_bounds__(WT, MX ? 1 : 2) k_w_double(KP<Real> p, WCovArgs<Real> a, int pow2, int cnt, int sq,
                                                  const Real* __restrict__ gk, Real* __restrict__ gk2) {
  using Z = WSz<Real, DP>;
  constexpr long DD = Z::DD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* S0 = reinterpret_cast<Real*>(smem_raw);
  double* piv = reinterpret_cast<double*>(smem_raw + (MX ? Z::WORK_MX : Z::WORK));
  Real* S1 = reinterpret_cast<Real*>(piv + DP + 8);   // a column
  int bad = 0;
  Real* PF = a.tab + (long)TPF * p.nT * DD;
  const int n = cnt + (sq ? 1 : 0);
  // the squaring first: it alone is on the path to the next level
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const int item = sq ? (it == 0 ? cnt : it - 1) : it;
    if (item == cnt)
      w_combine<Real, DP, MX>(p, a, blockIdx.x, gk, gk + DD, gk + 2 * DD, gk, gk + DD, gk + 2 * DD, gk2, gk2 + DD,
                          gk2 + 2 * DD, S0, S1, piv, &bad);
    else
      w_combine<Real, DP, MX>(p, a, blockIdx.x, nullptr, PF + (long)item * DD, nullptr, gk, gk + DD, gk + 2 * DD,
                          nullptr, PF + (long)(pow2 + item) * DD, nullptr, S0, S1, piv, &bad);
  }
  if (bad && threadIdx.x == 0) atomicOr(a.status, ST_NOT_PD);
}

// per step t = 0 .. T (item T: the last step's backward quantities only)
template <typename Real, int DP, bool MX>
__global__ void __launch_bounds__(WT, 2) k_w_epi(KP<Real> p, WCovArgs<Real> a) {
  refresh_delta(p);
  using Z = WSz<Real, DP>;
  constexpr long DD = Z::DD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* S0 = reinterpret_cast<Real*>(smem_raw);
  double* piv = reinterpret_cast<double*>(smem_raw + Z::WORK);
  Real* S1 = reinterpret_cast<Real*>(piv + DP + 8);   // a column
  const long ts = (long)p.nT * DD;
  Real* TKt = a.tab + (long)TK * ts;
  Real* TGt = a.tab + (long)TG * ts;
  Real* TLt = a.tab + (long)TLS * ts;
  const Real* PF = a.tab + (long)TPF * ts;
  const int s = blockIdx.x;
  Real* Pp = w_slot<Real, DP>(a, s, 0);
  Real* Li = w_slot<Real, DP>(a, s, 1);
  Real* X = w_slot<Real, DP>(a, s, 2);
  Real* Y = w_slot<Real, DP>(a, s, 3);
  Real* Sg = w_slot<Real, DP>(a, s, 4);
  int bad = 0;
  for (int t = blockIdx.x; t <= p.nT; t += gridDim.x) {
    if (t < p.nT) {
      // P^p_t
      if (t == 0) {
        w_axpby<Real, DP>(p.P0, false, (Real)1, nullptr, (Real)0, Pp);
      } else if (p.fdiag) {
        __syncthreads();
        const Real* Pf = PF + (long)(t - 1) * DD;
        for (int q = threadIdx.x; q < DP * DP; q += WT) {
          const int i = q / DP, j = q % DP;
          Pp[q] = fma(p.F[i * DP + i] * p.F[j * DP + j], Pf[q], p.Q[q]);
        }
        __syncthreads();
      } else {
        w_mm<Real, DP, MX>(p.F, false, PF + (long)(t - 1) * DD, false, X, nullptr, (Real)1, (Real)0, S0);
        w_mm<Real, DP, MX>(X, false, p.F, true, Pp, p.Q, (Real)1, (Real)1, S0);
      }
      // S_t = P^p_t + R: K'_t = r L^{-T} L^{-1}, log det S_t
      const double ld = w_chol<Real, DP>(Pp, p.r, p.d, S0, piv, &bad);
      if (threadIdx.x == 0) a.ldt[t] = 2.0 * ld;
      w_trinv<Real, DP>(S0, S1);
      w_store<Real, DP>(S0, Li, false);
      w_mm<Real, DP, MX>(Li, true, Li, false, TKt + (long)t * DD, nullptr, p.r, (Real)0, S0);
    }
    if (t >= 1) {
      // backward quantities of step t - 1
      const Real* Pf = PF + (long)(t - 1) * DD;
      if (t < p.nT) {
        w_chol<Real, DP>(Pp, (Real)0, p.d, S0, piv, &bad);
        w_trinv<Real, DP>(S0, S1);
        w_store<Real, DP>(S0, Li, false);                         // chol(P^p_t)^{-1}
        if (p.fdiag) {
          __syncthreads();
          for (int q = threadIdx.x; q < DP * DP; q += WT) X[q] = p.F[(q / DP) * DP + q / DP] * Pf[q];
          __syncthreads();
        } else {
          w_mm<Real, DP, MX>(p.F, false, Pf, false, X, nullptr, (Real)1, (Real)0, S0);   // F P^f
        }
        w_mm<Real, DP, MX>(Li, false, X, false, Y, nullptr, (Real)1, (Real)0, S0);       // Y = W^T
        w_mm<Real, DP, MX>(Li, true, Y, false, TGt + (long)(t - 1) * DD, nullptr, (Real)1, (Real)0, S0);   // G^T
        w_mm<Real, DP, MX>(Y, true, Y, false, Sg, Pf, (Real)-1, (Real)1, S0);            // Sigma
        w_chol<Real, DP>(Sg, (Real)0, p.d, S0, piv, &bad);
      } else {
        w_axpby<Real, DP>(Pf, false, (Real)0, nullptr, (Real)0, TGt + (long)(t - 1) * DD);   // G_{T-1} = 0
        w_chol<Real, DP>(Pf, (Real)0, p.d, S0, piv, &bad);
      }
      w_store<Real, DP>(S0, TLt + (long)(t - 1) * DD, true);      // chol(Sigma)^T
    }
  }
  if (bad && threadIdx.x == 0) atomicOr(a.status, ST_NOT_PD);
}

// per means block k: (M_e ... M_s)^T, (G_s ... G_e)^T, sum of log det S_t
template <typename Real, int DP, bool MX>
__global__ void __launch_bounds__(WT, 2) k_w_prod(KP<Real> p, WCovArgs<Real> a) {
  using Z = WSz<Real, DP>;
  constexpr long DD = Z::DD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* S0 = reinterpret_cast<Real*>(smem_raw);
  const long ts = (long)p.nT * DD;
  const Real* TKt = a.tab + (long)TK * ts;
  const Real* TGt = a.tab + (long)TG * ts;
  for (int k = blockIdx.x; k < p.nb; k += gridDim.x) {
    const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
    Real* AH = w_slot<Real, DP>(a, blockIdx.x, 0);
    Real* GH = w_slot<Real, DP>(a, blockIdx.x, 1);
    Real* X = w_slot<Real, DP>(a, blockIdx.x, 2);
    Real* Fd = w_slot<Real, DP>(a, blockIdx.x, 3);   // diag(F) when F is diagonal
    __syncthreads();
    for (int q = threadIdx.x; q < DP * DP; q += WT) {
      const Real id = (q / DP == q % DP) ? (Real)1 : (Real)0;
      AH[q] = id;
      GH[q] = id;
    }
    if (threadIdx.x < DP) Fd[threadIdx.x] = p.F[threadIdx.x * DP + threadIdx.x];
    __syncthreads();
    for (int t = s; t <= e; ++t) {
      if (p.fdiag) {
        w_mm<Real, DP, MX>(TKt + (long)t * DD, false, AH, false, AH, nullptr, (Real)1, (Real)0, S0, Fd);
      } else {
        w_mm<Real, DP, MX>(p.F, false, AH, false, X, nullptr, (Real)1, (Real)0, S0);
        w_mm<Real, DP, MX>(TKt + (long)t * DD, false, X, false, AH, nullptr, (Real)1, (Real)0, S0);
      }
      w_mm<Real, DP, MX>(GH, false, TGt + (long)t * DD, true, GH, nullptr, (Real)1, (Real)0, S0);
    }
    w_axpby<Real, DP>(AH, true, (Real)1, nullptr, (Real)0, a.btab + (long)k * DD);
    w_axpby<Real, DP>(GH, true, (Real)1, nullptr, (Real)0, a.btab + ((long)p.nb + k) * DD);
    if (threadIdx.x == 0) {
      double sl = 0.0;
      for (int t = s; t <= e; ++t) sl += a.ldt[t];
      a.ld[k] = sl;
    }
  }
}

// ---------------------------------------------------------------------------
// Means. CTA (k, grp): block k, chains grp * cpc + g * WCPT<DP> + j (thread row
// r = tid % DP, row group g = tid / DP, j < WCPT<DP>; cpc = WCPT<DP> * blockDim.x / DP,
// the CTA has as many row groups as its chains need, at most WT / DP). vs: three vector slots
// per chain slot, [3][CPC][DP].
// ---------------------------------------------------------------------------
// out[j] = sum_k Mt[k][r] v[slot(j)][k] (Mt: the transposed matrix, in shared or
// global memory, so that the threads of a warp read consecutive entries)
template <typename Real, int DP>
__device__ __forceinline__ void w_matvec(const Real* Mt, const Real* v, int g, int r, Real (&out)[WCPT<DP>]) {
  using V = typename Vec16<Real>::V;
  constexpr int N = Vec16<Real>::N;   // k per 16-byte word of a chain vector
#pragma unroll
  for (int j = 0; j < WCPT<DP>; ++j) out[j] = (Real)0;
#pragma unroll 4
  for (int k = 0; k < DP; k += N) {
    Real m[N];
#pragma unroll
    for (int q = 0; q < N; ++q) m[q] = Mt[(k + q) * DP + r];
#pragma unroll
    for (int j = 0; j < WCPT<DP>; ++j) {
      Real vv[N];
      unpack<Real>(*reinterpret_cast<const V*>(v + (g * WCPT<DP> + j) * DP + k), vv);
#pragma unroll
      for (int q = 0; q < N; ++q) out[j] = fma(m[q], vv[q], out[j]);
    }
  }
}

// A sequence of DP x DP matrices read in a fixed order, src(0), src(1), ...
// (src(j) null past the end), staged into NB shared buffers with NB - 1 copies
// in flight. get(src) waits for matrix i, then (after a CTA barrier, so that
// every thread sees the whole copy and is done with matrix i - 1, whose
// buffer is refilled next) issues the copy of matrix i + NB - 1 and returns
// matrix i's buffer.
template <typename Real, int DP>
struct WStream {
  static constexpr int NB = WSz<Real, DP>::NBUF;
  Real* buf;
  int i;
  __device__ __forceinline__ void fetch(int j, const Real* src) {
    constexpr int N = Vec16<Real>::N, NV = DP * DP / N;
    Real* dst = buf + (long)(j % NB) * DP * DP;
    if (src)
      for (int q = threadIdx.x; q < NV; q += blockDim.x) cp_async16(dst + q * N, src + q * N);
    cp_async_commit();
  }
  template <typename F>
  __device__ __forceinline__ void begin(Real* b, F&& src) {
    buf = b;
    i = 0;
    for (int j = 0; j < NB - 1; ++j) fetch(j, src(j));
  }
  template <typename F>
  __device__ __forceinline__ const Real* get(F&& src) {
    cp_async_wait<NB - 2>();
    __syncthreads();
    const Real* cur = buf + (long)(i % NB) * DP * DP;
    fetch(i + NB - 1, src(i + NB - 1));
    ++i;
    return cur;
  }
};

// m^p = F m + b for the thread's row (dense F: m in the vector slot vm)
template <typename Real, int DP>
__device__ __forceinline__ void w_predict(const KP<Real>& p, const Real (&m)[WCPT<DP>], Real* vm, int g, int r,
                                          Real (&mp)[WCPT<DP>]) {
  if (p.fdiag) {
    const Real phi = p.F[r * DP + r], bb = p.b[r];
#pragma unroll
    for (int j = 0; j < WCPT<DP>; ++j) mp[j] = fma(phi, m[j], bb);
    return;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < WCPT<DP>; ++j) vm[(g * WCPT<DP> + j) * DP + r] = m[j];
  __syncthreads();
#pragma unroll
  for (int j = 0; j < WCPT<DP>; ++j) {
    Real s = p.b[r];
    for (int k = 0; k < DP; ++k) s = fma(p.F[r * DP + k], vm[(g * WCPT<DP> + j) * DP + k], s);
    mp[j] = s;
  }
}

// block-local filtering means from a zero start (block 0: from m0), with the
// linearisation and the auxiliary draw when a.x is given
template <typename Real, int DP>
__global__ void __launch_bounds__(WT) k_wmf_reduce(KP<Real> p, MeanArgs<Real> a) {
  refresh_delta(p);
  using Z = WSz<Real, DP>;
  constexpr int CPC = Z::CPC;   // shared-memory layout (the largest CTA)
  const int cpc = (int)(blockDim.x / DP) * WCPT<DP>;   // chains of this CTA
  constexpr long DD = Z::DD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sbuf = reinterpret_cast<Real*>(smem_raw);
  Real* v0 = sbuf + Z::NBUF * DD;
  Real* v1 = v0 + CPC * DP;
  Real* v2 = v1 + CPC * DP;
  const int k = blockIdx.x % p.nb, grp = blockIdx.x / p.nb;
  const int r = threadIdx.x % DP, g = threadIdx.x / DP;
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  const Real* TKt = a.tab + (long)TK * p.nT * DD;
  auto src = [&](int j) -> const Real* { return s + j <= e ? TKt + (long)(s + j) * DD : nullptr; };
  WStream<Real, DP> mq;
  mq.begin(sbuf, src);
  int cidx[WCPT<DP>];
  bool valid[WCPT<DP>];
#pragma unroll
  for (int j = 0; j < WCPT<DP>; ++j) {
    cidx[j] = grp * cpc + g * WCPT<DP> + j;
    valid[j] = cidx[j] < p.C;
  }
  const bool lg = a.x && p.emis == AUX_EMIS_LINEAR_GAUSSIAN;
  Real m[WCPT<DP>];
#pragma unroll
  for (int j = 0; j < WCPT<DP>; ++j) m[j] = (Real)0;
  // the thread's inputs of step t (x_t and y_t, or ytilde_t), fetched one step ahead
  auto fetch_in = [&](int t, Real (&xa)[WCPT<DP>], Real (&ya)[WCPT<DP>]) {
#pragma unroll
    for (int j = 0; j < WCPT<DP>; ++j) {
      xa[j] = ya[j] = (Real)0;
      if (t <= e && valid[j] && r < p.d) {
        const long ct = (long)cidx[j] * p.nT + t;
        if (a.x) {
          xa[j] = a.x[ct * p.d + r];
          ya[j] = p.y[(p.y_per_chain ? ct : (long)t) * p.d + r];
        } else {
          ya[j] = a.yt[ct * p.d + r];
        }
      }
    }
  };
  Real xnx[WCPT<DP>], ynx[WCPT<DP>];
  fetch_in(s, xnx, ynx);
  for (int t = s; t <= e; ++t) {
    Real yti[WCPT<DP>], xi[WCPT<DP>], yv[WCPT<DP>];
#pragma unroll
    for (int j = 0; j < WCPT<DP>; ++j) {
      xi[j] = xnx[j];
      yv[j] = a.x ? ynx[j] : (Real)0;
      yti[j] = a.x ? (Real)0 : ynx[j];
    }
    fetch_in(t + 1, xnx, ynx);
    if (a.x) {
      Real vi[WCPT<DP>];
      if (lg) {   // v = R_y^{-1} (y - x)
        __syncthreads();
#pragma unroll
        for (int j = 0; j < WCPT<DP>; ++j) v1[(g * WCPT<DP> + j) * DP + r] = (r < p.d) ? yv[j] - xi[j] : (Real)0;
        __syncthreads();
        w_matvec<Real, DP>(p.Ryinv, v1, g, r, vi);
      }
      const bool obs = !p.mask || p.mask[t];
#pragma unroll
      for (int j = 0; j < WCPT<DP>; ++j) {
        if (!lg) vi[j] = (r < p.d) ? (Real)-0.5 + (Real)0.5 * yv[j] * yv[j] * exp(-xi[j]) : (Real)0;
        if (!obs) vi[j] = (Real)0;
        if (valid[j] && r < p.d) {
          const long ct = (long)cidx[j] * p.nT + t;
          const Real ep = philox_normal<Real>(p.seed, (uint32_t)cidx[j], iter_of(p, a.iter), PURPOSE_AUX,
                                              (uint32_t)t, r);
          const Real ui = xi[j] + p.sqrt_r * ep;
          yti[j] = ui + p.r * vi[j];
          a.u[ct * p.d + r] = ui;
          a.v[ct * p.d + r] = vi[j];
          a.yt[ct * p.d + r] = yti[j];
        }
      }
    }
    Real mp[WCPT<DP>];
    if (t == 0) {
#pragma unroll
      for (int j = 0; j < WCPT<DP>; ++j) mp[j] = p.m0[r];
    } else {
      w_predict<Real, DP>(p, m, v2, g, r, mp);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < WCPT<DP>; ++j) v0[(g * WCPT<DP> + j) * DP + r] = (r < p.d) ? yti[j] - mp[j] : (Real)0;
    const Real* sK = mq.get(src);
    Real kv[WCPT<DP>];
    w_matvec<Real, DP>(sK, v0, g, r, kv);
#pragma unroll
    for (int j = 0; j < WCPT<DP>; ++j) m[j] = (r < p.d) ? yti[j] - kv[j] : (Real)0;
  }
#pragma unroll
  for (int j = 0; j < WCPT<DP>; ++j) {
    if (valid[j]) a.z[((long)cidx[j] * p.nb + k) * DP + r] = m[j];
    if (valid[j] && a.x && k == 0 && r == 0) p.status_iter[cidx[j]] = *a.cov_status;
  }
}

// composition over the blocks, one CTA of DP threads per chain (the recursions of k_mean_cross);
// matsT: the transposed block products
template <typename Real, int DP>
__global__ void __launch_bounds__(DP) k_wmean_cross(KP<Real> p, const Real* __restrict__ matsT,
                                                    const Real* __restrict__ in, Real* __restrict__ out,
                                                    int backward) {
  constexpr long DD = WSz<Real, DP>::DD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sbuf = reinterpret_cast<Real*>(smem_raw);
  Real* vb = sbuf + WSz<Real, DP>::NBUF * DD;   // two vector slots
  const int c = blockIdx.x, r = threadIdx.x;
  const long cb = (long)c * p.nb;
  const int n = backward ? p.nb - 1 : max(0, p.nb - 2);
  auto kk_of = [&](int j) { return backward ? p.nb - 1 - j : 1 + j; };
  auto src = [&](int j) -> const Real* { return j < n ? matsT + (long)kk_of(j) * DD : nullptr; };
  WStream<Real, DP> mq;
  mq.begin(sbuf, src);
  Real m = (Real)0;
  if (backward) {
    out[(cb + p.nb - 1) * DP + r] = (Real)0;
  } else {
    m = in[cb * DP + r];
    if (p.nb > 1) out[(cb + 1) * DP + r] = m;
  }
  for (int j = 0; j < n; ++j) {
    const int kk = kk_of(j);
    Real* v = vb + (j & 1) * DP;
    v[r] = m;
    const Real* M = mq.get(src);
    Real sacc = in[(cb + kk) * DP + r];
#pragma unroll 16
    for (int q = 0; q < DP; ++q) sacc = fma(M[q * DP + r], v[q], sacc);
    m = sacc;
    out[(cb + (backward ? kk - 1 : kk + 1)) * DP + r] = m;
  }
}

// sum over the rows of a chain slot (FP64): each warp of the row group stores its
// partial in red[slot][warp]; after a barrier w_rowsum_get adds them in warp order,
// so the result does not depend on the warps' timing
template <typename Real, int DP>
__device__ __forceinline__ void w_rowsum(double* red, int slot, double v) {
  v = warp_sum<double>(v);
  if ((threadIdx.x & 31) == 0) red[slot * (DP / 32) + (threadIdx.x % DP) / 32] = v;
}
template <int DP>
__device__ __forceinline__ double w_rowsum_get(const double* red, int slot) {
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < DP / 32; ++w) s += red[slot * (DP / 32) + w];
  return s;
}

// filtering means from the true block start, likelihood terms, and (APPLY_EPI) the
// backward elements U_t with the block aggregate of the (G, U) scan
template <typename Real, int DP>
__global__ void __launch_bounds__(WT) k_wmf_apply(KP<Real> p, MeanArgs<Real> a) {
  refresh_delta(p);
  using Z = WSz<Real, DP>;
  constexpr int CPC = Z::CPC;   // shared-memory layout (the largest CTA)
  const int cpc = (int)(blockDim.x / DP) * WCPT<DP>;   // chains of this CTA
  constexpr long DD = Z::DD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sbuf = reinterpret_cast<Real*>(smem_raw);
  Real* v0 = sbuf + Z::NBUF * DD;
  Real* v1 = v0 + CPC * DP;
  Real* v2 = v1 + CPC * DP;
  double* red = reinterpret_cast<double*>(v2 + CPC * DP);
  const int k = blockIdx.x % p.nb, grp = blockIdx.x / p.nb;
  const int r = threadIdx.x % DP, g = threadIdx.x / DP;
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  const long ts = (long)p.nT * DD;
  const Real* TKt = a.tab + (long)TK * ts;
  const Real* TGt = a.tab + (long)TG * ts;
  const Real* TLt = a.tab + (long)TLS * ts;
  const Real* PF = a.tab + (long)TPF * ts;
  const bool epi = a.flags & APPLY_EPI;
  // matrices in the order of use: per step K' (, G, chol(Sigma)^T); then G_{e-1} .. G_s
  const int n = e - s + 1, per = epi ? 3 : 1, nfwd = n * per, ntot = nfwd + (epi ? n - 1 : 0);
  auto src = [&](int i) -> const Real* {
    if (i >= ntot) return nullptr;
    if (i >= nfwd) return TGt + (long)(e - 1 - (i - nfwd)) * DD;
    const long t = s + i / per;
    const int w = i % per;
    return (w == 0 ? TKt : (w == 1 ? TGt : TLt)) + t * DD;
  };
  WStream<Real, DP> mq;
  mq.begin(sbuf, src);
  int cidx[WCPT<DP>];
  bool valid[WCPT<DP>];
  Real mp[WCPT<DP>];
  double qacc[WCPT<DP>];
#pragma unroll
  for (int j = 0; j < WCPT<DP>; ++j) {
    cidx[j] = grp * cpc + g * WCPT<DP> + j;
    valid[j] = cidx[j] < p.C;
    qacc[j] = 0.0;
  }
  if (k == 0) {
#pragma unroll
    for (int j = 0; j < WCPT<DP>; ++j) mp[j] = p.m0[r];
  } else {
    Real ms[WCPT<DP>];
#pragma unroll
    for (int j = 0; j < WCPT<DP>; ++j) ms[j] = valid[j] ? a.mstart[((long)cidx[j] * p.nb + k) * DP + r] : (Real)0;
    w_predict<Real, DP>(p, ms, v2, g, r, mp);
  }
  // the thread's ytilde_t and (given) eps_t, fetched one step ahead
  auto fetch_in = [&](int t, Real (&ya)[WCPT<DP>], Real (&ea)[WCPT<DP>]) {
#pragma unroll
    for (int j = 0; j < WCPT<DP>; ++j) {
      const bool ok = t <= e && valid[j] && r < p.d;
      const long idx = ((long)cidx[j] * p.nT + t) * p.d + r;
      ya[j] = ok ? a.yt[idx] : (Real)0;
      ea[j] = (ok && epi && a.eps) ? a.eps[idx] : (Real)0;
    }
  };
  Real ynx[WCPT<DP>], enx[WCPT<DP>];
  fetch_in(s, ynx, enx);
  for (int t = s; t <= e; ++t) {
    Real yti[WCPT<DP>], egv[WCPT<DP>];
#pragma unroll
    for (int j = 0; j < WCPT<DP>; ++j) { yti[j] = ynx[j]; egv[j] = enx[j]; }
    fetch_in(t + 1, ynx, enx);
    Real ej[WCPT<DP>];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < WCPT<DP>; ++j) {
      ej[j] = (r < p.d) ? yti[j] - mp[j] : (Real)0;
      v0[(g * WCPT<DP> + j) * DP + r] = ej[j];
    }
    Real kv[WCPT<DP>], m[WCPT<DP>];
    w_matvec<Real, DP>(mq.get(src), v0, g, r, kv);
#pragma unroll
    for (int j = 0; j < WCPT<DP>; ++j) {
      qacc[j] += (double)ej[j] * (double)kv[j];
      m[j] = (r < p.d) ? yti[j] - kv[j] : (Real)0;
      const long ct = (long)cidx[j] * p.nT + t;
      if (valid[j] && a.mf && r < p.d) a.mf[ct * p.d + r] = m[j];
      if (valid[j] && a.Pf && r < p.d)
        for (int jj = 0; jj < p.d; ++jj) a.Pf[(ct * p.d + r) * p.d + jj] = PF[t * DD + (long)r * DP + jj];
    }
    Real mpn[WCPT<DP>];
    if (t < p.nT - 1) w_predict<Real, DP>(p, m, v2, g, r, mpn);
    else {
#pragma unroll
      for (int j = 0; j < WCPT<DP>; ++j) mpn[j] = (Real)0;
    }
    if (epi) {
      // U_t = m^f_t - G_t m^p_{t+1} + chol(Sigma_t) eps_t
      __syncthreads();
#pragma unroll
      for (int j = 0; j < WCPT<DP>; ++j) {
        Real ei = (Real)0;
        if (r < p.d && valid[j] && !(a.flags & APPLY_SMOOTH))
          ei = a.eps ? egv[j]
                     : philox_normal<Real>(p.seed, (uint32_t)cidx[j], iter_of(p, a.iter), PURPOSE_BACKWARD,
                                           (uint32_t)t, r);
        v1[(g * WCPT<DP> + j) * DP + r] = mpn[j];
        v2[(g * WCPT<DP> + j) * DP + r] = ei;
      }
      Real gm[WCPT<DP>], ln[WCPT<DP>];
      w_matvec<Real, DP>(mq.get(src), v1, g, r, gm);
      w_matvec<Real, DP>(mq.get(src), v2, g, r, ln);
#pragma unroll
      for (int j = 0; j < WCPT<DP>; ++j)
        if (valid[j]) a.U[((long)cidx[j] * p.nT + t) * DP + r] = m[j] - gm[j] + ln[j];
    }
#pragma unroll
    for (int j = 0; j < WCPT<DP>; ++j) mp[j] = mpn[j];
  }
  if (epi) {
    // block aggregate sum_t (G_s ... G_{t-1}) U_t by Horner's rule from the block end
    Real ub[WCPT<DP>];
#pragma unroll
    for (int j = 0; j < WCPT<DP>; ++j) ub[j] = valid[j] ? a.U[((long)cidx[j] * p.nT + e) * DP + r] : (Real)0;
    Real un[WCPT<DP>];
#pragma unroll
    for (int j = 0; j < WCPT<DP>; ++j)
      un[j] = (valid[j] && e - 1 >= s) ? a.U[((long)cidx[j] * p.nT + e - 1) * DP + r] : (Real)0;
    for (int t = e - 1; t >= s; --t) {
      Real uc[WCPT<DP>];
#pragma unroll
      for (int j = 0; j < WCPT<DP>; ++j) {
        uc[j] = un[j];
        un[j] = (valid[j] && t - 1 >= s) ? a.U[((long)cidx[j] * p.nT + t - 1) * DP + r] : (Real)0;
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < WCPT<DP>; ++j) v1[(g * WCPT<DP> + j) * DP + r] = ub[j];
      Real gu[WCPT<DP>];
      w_matvec<Real, DP>(mq.get(src), v1, g, r, gu);
#pragma unroll
      for (int j = 0; j < WCPT<DP>; ++j) ub[j] = gu[j] + uc[j];
    }
#pragma unroll
    for (int j = 0; j < WCPT<DP>; ++j)
      if (valid[j]) a.guv[((long)cidx[j] * p.nb + k) * DP + r] = ub[j];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < WCPT<DP>; ++j) w_rowsum<Real, DP>(red, g * WCPT<DP> + j, qacc[j]);
  __syncthreads();
  if (r == 0) {
#pragma unroll
    for (int j = 0; j < WCPT<DP>; ++j) {
      if (!valid[j]) continue;
      const double q = w_rowsum_get<DP>(red, g * WCPT<DP> + j) / (double)p.r;
      const int c = cidx[j];
      const long ck = (long)c * p.nb + k;
      if (a.flags & APPLY_STORE_Q) a.fqb[ck] = q;
      if (a.flags & APPLY_REV_DIFF) a.lz_part[ck] = -0.5 * (a.fqb[ck] - q);
      if (a.flags & APPLY_LOGZ) {
        const double half_dlog2pi = 0.5 * p.d * 1.8378770664093454835606594728112;
        a.lz_part[ck] = -((double)(e - s + 1) * half_dlog2pi + 0.5 * (a.ld[k] + q));
      }
      if (a.status && k == 0 && *a.cov_status) atomicOr(&a.status[c], *a.cov_status);
    }
  }
}

// backward sampling inside each block from x*_{e+1}: x*_t = G_t x*_{t+1} + U_t, with the MH
// terms of mh_step_terms (first-order proposal) when b.mh
template <typename Real, int DP>
__global__ void __launch_bounds__(WT) k_wmb_apply(KP<Real> p, BackArgs<Real> b, const Real* __restrict__ xnext) {
  refresh_delta(p);
  using Z = WSz<Real, DP>;
  constexpr int CPC = Z::CPC;   // shared-memory layout (the largest CTA)
  const int cpc = (int)(blockDim.x / DP) * WCPT<DP>;   // chains of this CTA
  constexpr long DD = Z::DD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sbuf = reinterpret_cast<Real*>(smem_raw);
  Real* v0 = sbuf + Z::NBUF * DD;
  Real* v1 = v0 + CPC * DP;
  double* red = reinterpret_cast<double*>(v1 + 2 * CPC * DP);
  const int k = blockIdx.x % p.nb, grp = blockIdx.x / p.nb;
  const int r = threadIdx.x % DP, g = threadIdx.x / DP;
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  auto src = [&](int j) -> const Real* { return e - j >= s ? b.G + (long)(e - j) * DD : nullptr; };
  WStream<Real, DP> mq;
  mq.begin(sbuf, src);
  const bool lg = b.mh && p.emis == AUX_EMIS_LINEAR_GAUSSIAN;
  int cidx[WCPT<DP>];
  bool valid[WCPT<DP>];
  Real xi[WCPT<DP>];
  double acc[WCPT<DP>];
#pragma unroll
  for (int j = 0; j < WCPT<DP>; ++j) {
    cidx[j] = grp * cpc + g * WCPT<DP> + j;
    valid[j] = cidx[j] < p.C;
    xi[j] = valid[j] ? xnext[((long)cidx[j] * p.nb + k) * DP + r] : (Real)0;
    acc[j] = 0.0;
  }
  // the thread's U_t and MH inputs (x_t, u_t, v_t, y_t) of step t, fetched one step ahead
  constexpr int CPT = WCPT<DP>;
  auto fetch_in = [&](int t, Real (&ua)[CPT], Real (&xa)[CPT], Real (&uia)[CPT], Real (&va)[CPT],
                      Real (&ya)[CPT]) {
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      ua[j] = xa[j] = uia[j] = va[j] = ya[j] = (Real)0;
      if (t < s || !valid[j]) continue;
      const long ct = (long)cidx[j] * p.nT + t;
      ua[j] = b.U[ct * DP + r];
      if (b.mh && r < p.d) {
        const long idx = ct * p.d + r;
        xa[j] = b.x[idx]; uia[j] = b.u[idx]; va[j] = b.v[idx];
        ya[j] = p.y[(p.y_per_chain ? ct : (long)t) * p.d + r];
      }
    }
  };
  Real un[CPT], xon[CPT], uin[CPT], vin[CPT], yin[CPT];
  fetch_in(e, un, xon, uin, vin, yin);
  for (int t = e; t >= s; --t) {
    Real uc[CPT], xoc[CPT], uic[CPT], vic[CPT], yic[CPT];
#pragma unroll
    for (int j = 0; j < CPT; ++j) { uc[j] = un[j]; xoc[j] = xon[j]; uic[j] = uin[j]; vic[j] = vin[j]; yic[j] = yin[j]; }
    fetch_in(t - 1, un, xon, uin, vin, yin);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < WCPT<DP>; ++j) v0[(g * WCPT<DP> + j) * DP + r] = xi[j];
    Real gx[WCPT<DP>];
    w_matvec<Real, DP>(mq.get(src), v0, g, r, gx);
#pragma unroll
    for (int j = 0; j < WCPT<DP>; ++j) {
      xi[j] = gx[j] + uc[j];
      if (valid[j] && r < p.d) b.xs[((long)cidx[j] * p.nT + t) * p.d + r] = xi[j];
    }
    if (!b.mh) continue;
    Real vsi[WCPT<DP>];
    if (lg) {
      __syncthreads();
#pragma unroll
      for (int j = 0; j < WCPT<DP>; ++j) v1[(g * WCPT<DP> + j) * DP + r] = (r < p.d) ? yic[j] - xi[j] : (Real)0;
      __syncthreads();
      w_matvec<Real, DP>(p.Ryinv, v1, g, r, vsi);
    }
    const bool obs = !p.mask || p.mask[t];
#pragma unroll
    for (int j = 0; j < WCPT<DP>; ++j) {
      if (!valid[j] || r >= p.d) continue;
      const long ct = (long)cidx[j] * p.nT + t, idx = ct * p.d + r;
      const Real xo = xoc[j], ui = uic[j], vi = vic[j], yi = yic[j];
      const Real xs = xi[j];
      Real vs = lg ? vsi[j] : (Real)0, gdiff = (Real)0;
      if (obs) {
        if (p.emis == AUX_EMIS_SV) {
          vs = (Real)-0.5 + (Real)0.5 * yi * yi * exp(-xs);
          gdiff = (Real)-0.5 * (xs - xo) - (Real)0.5 * yi * yi * (exp(-xs) - exp(-xo));
        } else {
          gdiff = (Real)-0.5 * (yi - xs) * vs + (Real)0.5 * (yi - xo) * vi;
        }
      } else {
        vs = (Real)0;
      }
      const Real fwd = vi * (ui - xs) + (Real)0.5 * p.r * vi * vi;
      const Real rev = vs * (ui - xo) + (Real)0.5 * p.r * vs * vs;
      acc[j] += (double)gdiff + (double)fwd - (double)rev;
      b.yts[idx] = ui + p.r * vs;
    }
  }
  if (!b.mh) return;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < WCPT<DP>; ++j) w_rowsum<Real, DP>(red, g * WCPT<DP> + j, acc[j]);
  __syncthreads();
  if (r == 0) {
#pragma unroll
    for (int j = 0; j < WCPT<DP>; ++j)
      if (valid[j]) b.mh_part[(long)cidx[j] * p.nb + k] = w_rowsum_get<DP>(red, g * WCPT<DP> + j);
  }
}

}  // namespace auxk
