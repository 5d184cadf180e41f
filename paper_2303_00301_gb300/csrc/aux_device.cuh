// aux_device.cuh — device building blocks of the auxiliary Kalman sampler.
//
// * Philox4x32-10 (Salmon et al., SC'11) and Box-Muller normals, with the
//   counter layout documented in include/aux_kalman.h.
// * Warp-level dense linear algebra on DP x DP matrices (DP <= 32, padded
//   dimension). Lane i owns row i: a matrix operand is either a register
//   row (T r[DP]) or a shared-memory "slot" (row stride LD = DP + 16 bytes
//   worth of elements, so that a lane loading its own row with 16-byte
//   vectors is bank-conflict free, a broadcast row read is one wavefront and
//   a column read across lanes hits consecutive banks).
//   Products take the other operand's rows (broadcast) or columns from
//   shared memory; Cholesky factors are stored transposed (LT = L^T, upper),
//   so that a column of L is a contiguous row of the slot.
// Padding convention: entries of padded rows/columns (index >= d) are zero
// in every covariance-like matrix; the Cholesky routine uses a unit pivot
// there, so factors and solves keep the padding exact.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace auxk {

constexpr unsigned FULL_MASK = 0xffffffffu;

// ---------------------------------------------------------------- launch order
// Programmatic dependent launch (sm_90 and later). A kernel launched with the
// programmatic-serialization attribute may be scheduled before its
// predecessor in the stream has finished: pdl_wait() blocks until the
// predecessor grid has completed and its memory writes are visible (it returns
// at once for a kernel launched without the attribute), and pdl_trigger()
// lets the successor be scheduled. Kernels on the table-mode step call both
// first thing, so their reads always follow the predecessor's writes.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// ---------------------------------------------------------------- Philox
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

enum Purpose : uint32_t { PURPOSE_AUX = 0, PURPOSE_BACKWARD = 1, PURPOSE_MH = 2 };

__device__ __forceinline__ uint4 philox_word(uint64_t seed, uint32_t chain, uint64_t iter,
                                             uint32_t purpose, uint32_t t, uint32_t word) {
  const uint4 ctr = make_uint4(word, (t & 0xFFFFFFu) | (purpose << 24), (uint32_t)iter, chain);
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  return philox4x32_10(ctr, key);
}

template <typename T> __device__ __forceinline__ T u01(uint32_t r) {
  // ((r >> 9) + 0.5) * 2^-23: exact in binary32 and binary64, inside (0, 1)
  return ((T)(r >> 9) + (T)0.5) * (T)(1.0 / 8388608.0);
}

__device__ __forceinline__ void sincospi_t(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_t(double x, double* s, double* c) { sincospi(x, s, c); }

// standard normal number i of the (seed, chain, iter, purpose, t) stream
template <typename T>
__device__ __forceinline__ T philox_normal(uint64_t seed, uint32_t chain, uint64_t iter,
                                           uint32_t purpose, uint32_t t, int i) {
  const uint4 r = philox_word(seed, chain, iter, purpose, t, (uint32_t)(i >> 2));
  const uint32_t ra = (i & 2) ? r.z : r.x;
  const uint32_t rb = (i & 2) ? r.w : r.y;
  const T rad = sqrt((T)-2 * log(u01<T>(ra)));
  T s, c;
  sincospi_t((T)2 * u01<T>(rb), &s, &c);
  return rad * ((i & 1) ? s : c);
}

// ---------------------------------------------------------------- layout
template <typename T> struct Vec16;
template <> struct Vec16<float> { using V = float4; static constexpr int N = 4; };
template <> struct Vec16<double> { using V = double2; static constexpr int N = 2; };

template <typename T, int DP> struct Lay {
  static constexpr int N = Vec16<T>::N;
  static constexpr int LD = DP + N;          // row stride in elements (16 B pad)
  static constexpr int MAT = DP * LD;         // elements of one matrix slot
  static constexpr int VEC = (DP + N - 1) / N * N;  // elements of one vector slot
  static_assert(DP % N == 0, "DP must be a multiple of the 16-byte vector width");
};

template <typename T> __device__ __forceinline__ void unpack(const typename Vec16<T>::V& v, T* o);
template <> __device__ __forceinline__ void unpack<float>(const float4& v, float* o) {
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
template <> __device__ __forceinline__ void unpack<double>(const double2& v, double* o) {
  o[0] = v.x; o[1] = v.y;
}
template <typename T> __device__ __forceinline__ typename Vec16<T>::V pack(const T* o);
template <> __device__ __forceinline__ float4 pack<float>(const float* o) {
  return make_float4(o[0], o[1], o[2], o[3]);
}
template <> __device__ __forceinline__ double2 pack<double>(const double* o) {
  return make_double2(o[0], o[1]);
}

// contiguous DP elements (16-byte aligned) -> registers
template <typename T, int DP>
__device__ __forceinline__ void ld_vec(const T* p, T (&r)[DP]) {
  using V = typename Vec16<T>::V;
  constexpr int N = Vec16<T>::N;
  const V* q = reinterpret_cast<const V*>(p);
#pragma unroll
  for (int k = 0; k < DP / N; ++k) unpack<T>(q[k], &r[k * N]);
}
template <typename T, int DP>
__device__ __forceinline__ void st_vec(T* p, const T (&r)[DP]) {
  using V = typename Vec16<T>::V;
  constexpr int N = Vec16<T>::N;
  V* q = reinterpret_cast<V*>(p);
#pragma unroll
  for (int k = 0; k < DP / N; ++k) q[k] = pack<T>(&r[k * N]);
}

// row `row` of a slot
template <typename T, int DP>
__device__ __forceinline__ void ld_row(const T* S, int row, T (&r)[DP]) {
  ld_vec<T, DP>(S + row * Lay<T, DP>::LD, r);
}
template <typename T, int DP>
__device__ __forceinline__ void st_row(T* S, int row, const T (&r)[DP], bool active) {
  if (active) st_vec<T, DP>(S + row * Lay<T, DP>::LD, r);
}
// store a register row as column `col` of a slot: S[k][col] = r[k]
template <typename T, int DP>
__device__ __forceinline__ void st_col(T* S, int col, const T (&r)[DP], bool active) {
  if (active) {
#pragma unroll
    for (int k = 0; k < DP; ++k) S[k * Lay<T, DP>::LD + col] = r[k];
  }
}
// column `col` of a slot: r[k] = S[k][col]
template <typename T, int DP>
__device__ __forceinline__ void ld_col(const T* S, int col, T (&r)[DP]) {
#pragma unroll
  for (int k = 0; k < DP; ++k) r[k] = S[k * Lay<T, DP>::LD + col];
}

template <typename T, int DP>
__device__ __forceinline__ void zero(T (&r)[DP]) {
#pragma unroll
  for (int k = 0; k < DP; ++k) r[k] = (T)0;
}

// ---------------------------------------------------------------------------
// Fused multiply-adds over a register row, out[j] = fma(s, b[j], out[j]).
// In single precision adjacent pairs go through one packed instruction
// (fma.rn.f32x2: two independent fused multiply-adds, each rounded once, so
// every element's value and order of accumulation are those of fmaf).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void fma_pair(float& c0, float& c1, float a0, float a1, float b0, float b1) {
  unsigned long long ra, rb, rc;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a0), "f"(a1));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b0), "f"(b1));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rc) : "f"(c0), "f"(c1));
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(rc) : "l"(ra), "l"(rb));
  asm("mov.b64 {%0, %1}, %2;" : "=f"(c0), "=f"(c1) : "l"(rc));
}
__device__ __forceinline__ void fma_pair(double& c0, double& c1, double a0, double a1, double b0,
                                         double b1) {
  c0 = fma(a0, b0, c0);
  c1 = fma(a1, b1, c1);
}

template <typename T, int N>
__device__ __forceinline__ void fma_row(T s, const T (&b)[N], T (&out)[N]) {
  if constexpr (N % 2 == 0) {
#pragma unroll
    for (int j = 0; j < N; j += 2) fma_pair(out[j], out[j + 1], s, s, b[j], b[j + 1]);
  } else {
#pragma unroll
    for (int j = 0; j < N; ++j) out[j] = fma(s, b[j], out[j]);
  }
}

// out[j] (+)= sum_k a[k] * B[k][j]         (a: register row, B: slot, broadcast rows)
template <typename T, int DP, bool ACC = false, bool NEG = false>
__device__ __forceinline__ void row_mat(const T (&a)[DP], const T* B, T (&out)[DP]) {
  if (!ACC) zero<T, DP>(out);
  constexpr int N = Vec16<T>::N;
#pragma unroll
  for (int k = 0; k < DP; ++k) {
    const T ak = NEG ? -a[k] : a[k];
    T b[DP];
    ld_row<T, DP>(B, k, b);
    fma_row<T, DP>(ak, b, out);
  }
  (void)N;
}

// out[j] = sum_k a[k] * B[j][k]            (dot with every row of B)
template <typename T, int DP>
__device__ __forceinline__ void row_matT(const T (&a)[DP], const T* B, T (&out)[DP]) {
#pragma unroll
  for (int j = 0; j < DP; ++j) {
    T b[DP];
    ld_row<T, DP>(B, j, b);
    T acc0 = 0, acc1 = 0;
#pragma unroll
    for (int k = 0; k < DP; k += 2) {
      acc0 = fma(a[k], b[k], acc0);
      if (k + 1 < DP) acc1 = fma(a[k + 1], b[k + 1], acc1);
    }
    out[j] = acc0 + acc1;
  }
}

// dot of a register row with a vector slot (broadcast)
template <typename T, int DP>
__device__ __forceinline__ T dot_rv(const T (&a)[DP], const T* v) {
  T b[DP];
  ld_vec<T, DP>(v, b);
  T acc0 = 0, acc1 = 0;
#pragma unroll
  for (int k = 0; k < DP; k += 2) {
    if (k + 1 < DP) fma_pair(acc0, acc1, a[k], a[k + 1], b[k], b[k + 1]);
    else acc0 = fma(a[k], b[k], acc0);
  }
  return acc0 + acc1;
}

template <typename T, int DP>
__device__ __forceinline__ T dot_rr(const T (&a)[DP], const T (&b)[DP]) {
  T acc0 = 0, acc1 = 0;
#pragma unroll
  for (int k = 0; k < DP; k += 2) {
    if (k + 1 < DP) fma_pair(acc0, acc1, a[k], a[k + 1], b[k], b[k + 1]);
    else acc0 = fma(a[k], b[k], acc0);
  }
  return acc0 + acc1;
}

// Cholesky of the symmetric matrix whose row `lane` is a[] (all lanes of the
// warp call it; lanes >= DP pass anything). Writes LT = L^T (upper) to the
// slot LT and 1/L_kk to inv_diag[k]. Indices k >= d get a unit pivot. A
// non-positive or non-finite pivot at k < d sets *bad and is replaced by 1.
// Contains the __syncwarp() needed before reading LT.
template <typename T, int DP>
__device__ __forceinline__ void chol_rows(T (&a)[DP], T* LT, T* inv_diag, int d, int lane,
                                          int* bad) {
  constexpr int LD = Lay<T, DP>::LD;
  __syncwarp();
#pragma unroll
  for (int k = 0; k < DP; ++k) {
    T akk = __shfl_sync(FULL_MASK, a[k], k);
    T piv = (T)1;
    if (k < d) {
      if (!(akk > (T)0) || !(akk < (T)INFINITY)) { *bad = 1; akk = (T)1; }
      piv = sqrt(akk);
    }
    const T inv = (T)1 / piv;
    T l = (lane == k) ? piv : ((lane > k) ? a[k] * inv : (T)0);
    if (lane < DP) LT[k * LD + lane] = l;
    if (lane == 0) inv_diag[k] = inv;
    __syncwarp();
    if (k + 1 < DP) {
      T lk[DP];
      ld_row<T, DP>(LT, k, lk);
      const T nl = -l;
#pragma unroll
      for (int j = k + 1; j < DP; ++j) a[j] = fma(nl, lk[j], a[j]);
    }
  }
  __syncwarp();
}

// Per-lane forward substitution: y = L^{-1} rhs with L given as LT = L^T.
template <typename T, int DP>
__device__ __forceinline__ void fwd_subst(const T* LT, const T* inv_diag, T (&rhs)[DP],
                                          T (&y)[DP]) {
  T id[DP];
  ld_vec<T, DP>(inv_diag, id);
#pragma unroll
  for (int k = 0; k < DP; ++k) {
    y[k] = rhs[k] * id[k];
    if (k + 1 < DP) {
      T lk[DP];
      ld_row<T, DP>(LT, k, lk);  // lk[j] = L[j][k]
      const T ny = -y[k];
#pragma unroll
      for (int j = k + 1; j < DP; ++j) rhs[j] = fma(ny, lk[j], rhs[j]);
    }
  }
}

// Per-lane backward substitution: y = L^{-T} rhs with L given as LT = L^T.
template <typename T, int DP>
__device__ __forceinline__ void bwd_subst(const T* LT, const T* inv_diag, const T (&rhs)[DP],
                                          T (&y)[DP]) {
  T id[DP];
  ld_vec<T, DP>(inv_diag, id);
#pragma unroll
  for (int k = DP - 1; k >= 0; --k) {
    T lk[DP];
    ld_row<T, DP>(LT, k, lk);  // lk[j] = L^T[k][j] = L[j][k]
    T acc = rhs[k];
#pragma unroll
    for (int j = k + 1; j < DP; ++j) acc = fma(-lk[j], y[j], acc);
    y[k] = acc * id[k];
  }
}

// ---------------------------------------------------------------------------
// Rolled primitives. Only the inner index j (a register-array index) is
// unrolled; the k loops run as real loops so that the code of a p = 32 kernel
// stays inside the instruction cache. The left operand of a product is read
// from shared memory (a contiguous row, or a column of a slot).
// ---------------------------------------------------------------------------

// out[j] (+/-)= sum_k arow[k] * B[k][j]       (arow: 16-byte aligned shared row)
template <typename T, int DP, bool ACC = false, bool NEG = false>
__device__ __forceinline__ void mm_row(const T* arow, const T* B, T (&out)[DP]) {
  using V = typename Vec16<T>::V;
  constexpr int N = Vec16<T>::N, LD = Lay<T, DP>::LD;
  if (!ACC) zero<T, DP>(out);
#pragma unroll 1
  for (int k0 = 0; k0 < DP; k0 += N) {
    T a[N];
    unpack<T>(*reinterpret_cast<const V*>(arow + k0), a);
#pragma unroll
    for (int kk = 0; kk < N; ++kk) {
      const T ak = NEG ? -a[kk] : a[kk];
      T b[DP];
      ld_vec<T, DP>(B + (k0 + kk) * LD, b);
      fma_row<T, DP>(ak, b, out);
    }
  }
}

// out[j] (+/-)= sum_k A[k][col] * B[k][j]     (left operand: column `col` of slot A)
template <typename T, int DP, bool ACC = false, bool NEG = false>
__device__ __forceinline__ void mm_col(const T* A, int col, const T* B, T (&out)[DP]) {
  constexpr int N = Vec16<T>::N, LD = Lay<T, DP>::LD;
  if (!ACC) zero<T, DP>(out);
#pragma unroll 1
  for (int k0 = 0; k0 < DP; k0 += N) {
#pragma unroll
    for (int kk = 0; kk < N; ++kk) {
      const T a = A[(k0 + kk) * LD + col];
      const T ak = NEG ? -a : a;
      T b[DP];
      ld_vec<T, DP>(B + (k0 + kk) * LD, b);
      fma_row<T, DP>(ak, b, out);
    }
  }
}

// sum_k arow[k] v[k] and sum_k A[k][col] v[k] (v: shared vector, broadcast)
template <typename T, int DP>
__device__ __forceinline__ T dot_row_vec(const T* arow, const T* v) {
  T a[DP], b[DP];
  ld_vec<T, DP>(arow, a);
  ld_vec<T, DP>(v, b);
  return dot_rr<T, DP>(a, b);
}
template <typename T, int DP>
__device__ __forceinline__ T dot_col_vec(const T* A, int col, const T* v) {
  T a[DP], b[DP];
  ld_col<T, DP>(A, col, a);
  ld_vec<T, DP>(v, b);
  return dot_rr<T, DP>(a, b);
}

// Cholesky in "rotating" form. Lane i passes row i of the SPD matrix in a[]
// (consumed). Before step k, a[j] holds the updated entry (i, k + j), so the
// pivot column is always a[0] and the update shifts the row down by one:
// a[j] <- a[j+1] - l_ik L[k+1+j][k]. Outputs:
//   LS   (required, also the working slot): LS[k][m] = L[k+m][k] (row k of L^T
//        starting at the diagonal), used by fsolve_rot;
//   LRow (optional): L row-major;  LR (optional): LR[i][m] = L[i][i-(DP-1)+m]
//        (row i right-aligned, zeros on the left), used by bsolve_rot;
//   inv_diag[k] = 1 / L[k][k];  returns sum_k L[lane][k] eps[k] when eps != null.
// Indices k >= d get a unit pivot; a non-positive or non-finite pivot below d
// sets *bad and is replaced by 1.
template <typename T, int DP>
__device__ T chol_rot(T (&a)[DP], T* LS, T* LRow, T* LR, T* inv_diag, const T* eps, int d,
                      int lane, int* bad) {
  constexpr int LD = Lay<T, DP>::LD;
  const bool act = lane < DP;
  T acc = 0;
  __syncwarp();
  if (LR && act) {
    T z[DP];
    zero<T, DP>(z);
    st_vec<T, DP>(LR + lane * LD, z);
  }
  if (LRow && act) {
    T z[DP];
    zero<T, DP>(z);
    st_vec<T, DP>(LRow + lane * LD, z);
  }
  __syncwarp();
#pragma unroll 1
  for (int k = 0; k < DP; ++k) {
    T akk = __shfl_sync(FULL_MASK, a[0], k);
    T piv = (T)1;
    if (k < d) {
      if (!(akk > (T)0) || !(akk < (T)INFINITY)) { *bad = 1; akk = (T)1; }
      piv = sqrt(akk);
    }
    const T inv = (T)1 / piv;
    const T l = (lane == k) ? piv : ((lane > k) ? a[0] * inv : (T)0);
    if (act && lane >= k) {
      LS[k * LD + (lane - k)] = l;
      if (LRow) LRow[lane * LD + k] = l;
      if (LR) LR[lane * LD + (DP - 1) - (lane - k)] = l;
    }
    if (lane == 0) inv_diag[k] = inv;
    if (eps) acc = fma(l, eps[k], acc);
    __syncwarp();
    T lk[DP];
    ld_vec<T, DP>(LS + k * LD, lk);
    const T nl = -l;
#pragma unroll
    for (int j = 0; j < DP - 1; ++j) a[j] = fma(nl, lk[j + 1], a[j + 1]);
    a[DP - 1] = (T)0;
  }
  __syncwarp();
  return acc;
}

// chol_rot without the rotation: lane i keeps row i in place (before step k,
// a[j] for j >= k holds the updated entry (i, j); step k applies
// a[j] <- a[j] - l_ik L[j][k]), fully unrolled, with the pivot's square root
// and reciprocal taken speculatively and replaced by a select when the pivot
// fails or k >= d. Same inputs, outputs and padding rules as chol_rot, and the
// same values. Faster on the per-chain element kernels; the square-root and
// bridging kernels keep chol_rot (their larger bodies lose more to the
// unrolled code than they gain).
template <typename T, int DP>
__device__ T chol_ur(T (&a)[DP], T* LS, T* LRow, T* LR, T* inv_diag, const T* eps, int d,
                      int lane, int* bad) {
  constexpr int LD = Lay<T, DP>::LD;
  const bool act = lane < DP;
  T acc = 0;
  __syncwarp();
  if (LR && act) {
    T z[DP];
    zero<T, DP>(z);
    st_vec<T, DP>(LR + lane * LD, z);
  }
  if (LRow && act) {
    T z[DP];
    zero<T, DP>(z);
    st_vec<T, DP>(LRow + lane * LD, z);
  }
  __syncwarp();
  // lane i keeps row i unshifted (entry j in a[j]); column k's factor entries
  // reach the lanes through the LS row just stored, one broadcast read per
  // update; the pivot's square root and reciprocal are taken speculatively and
  // a failed pivot (or a padding column) is replaced by a select afterwards,
  // off the pivot-to-pivot critical path
#pragma unroll
  for (int k = 0; k < DP; ++k) {
    const T akk = __shfl_sync(FULL_MASK, a[k], k);
    const T piv0 = sqrt(akk);
    const T inv0 = (T)1 / piv0;
    const bool ok = akk > (T)0 && akk < (T)INFINITY;
    if (k < d && !ok) *bad = 1;
    const bool good = k < d && ok;
    const T piv = good ? piv0 : (T)1;
    const T inv = good ? inv0 : (T)1;
    const T l = (lane == k) ? piv : ((lane > k) ? a[k] * inv : (T)0);
    if (act && lane >= k) {
      LS[k * LD + (lane - k)] = l;
      if (LRow) LRow[lane * LD + k] = l;
      if (LR) LR[lane * LD + (DP - 1) - (lane - k)] = l;
    }
    if (lane == 0) inv_diag[k] = inv;
    if (eps) acc = fma(l, eps[k], acc);
    __syncwarp();
    const T nl = -l;
#pragma unroll
    for (int j = k + 1; j < DP; ++j) a[j] = fma(nl, LS[k * LD + (j - k)], a[j]);
  }
  zero<T, DP>(a);   // the row is consumed
  __syncwarp();
  return acc;
}

__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }

// chol_rot with a one-column lookahead and a reciprocal square root: the
// pivot of column k + 1 is updated and broadcast (two shuffles) before the
// rest of column k's rank-1 update, whose shared-memory row load and fused
// multiply-adds then hide the broadcast's latency, and the pivot's
// reciprocal square root comes from one rsqrt (the diagonal of the factor is
// the pivot times it). Same inputs, outputs and padding rules as chol_rot.
template <typename T, int DP>
__device__ T chol_la(T (&a)[DP], T* LS, T* LRow, T* LR, T* inv_diag, const T* eps, int d, int lane,
                     int* bad) {
  constexpr int LD = Lay<T, DP>::LD;
  const bool act = lane < DP;
  T acc = 0;
  __syncwarp();
  if (act) {
    T z[DP];
    zero<T, DP>(z);
    if (LR) st_vec<T, DP>(LR + lane * LD, z);
    if (LRow) st_vec<T, DP>(LRow + lane * LD, z);
  }
  // pivot of column 0
  T pk = __shfl_sync(FULL_MASK, a[0], 0);
  T piv = (T)1, inv = (T)1;
  if (0 < d) {
    if (!(pk > (T)0) || !(pk < (T)INFINITY)) { *bad = 1; pk = (T)1; }
    inv = rsqrt_t(pk);
    piv = pk * inv;
  }
#pragma unroll 1
  for (int k = 0; k < DP; ++k) {
    const T l = (lane == k) ? piv : ((lane > k) ? a[0] * inv : (T)0);
    if (act && lane >= k) {
      LS[k * LD + (lane - k)] = l;
      if (LRow) LRow[lane * LD + k] = l;
      if (LR) LR[lane * LD + (DP - 1) - (lane - k)] = l;
    }
    if (lane == 0) inv_diag[k] = inv;
    if (eps) acc = fma(l, eps[k], acc);
    // lookahead: entry (i, k + 1) and the pivot of column k + 1
    const T lk1 = __shfl_sync(FULL_MASK, l, (k + 1) & 31);
    const T a1 = fma(-l, lk1, a[1]);
    T pn = __shfl_sync(FULL_MASK, a1, (k + 1) & 31);
    __syncwarp();
    T lk[DP];
    ld_vec<T, DP>(LS + k * LD, lk);
#pragma unroll
    for (int j = 1; j < DP - 1; ++j) a[j] = fma(-l, lk[j + 1], a[j + 1]);
    a[0] = a1;
    a[DP - 1] = (T)0;
    piv = (T)1;
    inv = (T)1;
    if (k + 1 < d) {
      if (!(pn > (T)0) || !(pn < (T)INFINITY)) { *bad = 1; pn = (T)1; }
      inv = rsqrt_t(pn);
      piv = pn * inv;
    }
  }
  __syncwarp();
  return acc;
}

// Forward solve L y = r as fsolve_rot, with the factor's next row loaded while
// the current one is applied (two register buffers, two steps per trip).
template <typename T, int DP, bool AS_COLUMN>
__device__ __forceinline__ void fsolve_pf(const T* LS, const T* inv_diag, T (&r)[DP], T* Y, int lane) {
  constexpr int LD = Lay<T, DP>::LD;
  static_assert(DP % 2 == 0, "two steps per trip");
  const bool act = lane < DP;
  T l0[DP], l1[DP];
  ld_vec<T, DP>(LS, l0);
#pragma unroll 1
  for (int k = 0; k < DP; k += 2) {
    ld_vec<T, DP>(LS + (k + 1) * LD, l1);
    const T y0 = r[0] * inv_diag[k];
    if (act) {
      if (AS_COLUMN) Y[k * LD + lane] = y0;
      else Y[lane * LD + k] = y0;
    }
#pragma unroll
    for (int j = 0; j < DP - 1; ++j) r[j] = fma(-y0, l0[j + 1], r[j + 1]);
    r[DP - 1] = (T)0;
    if (k + 2 < DP) ld_vec<T, DP>(LS + (k + 2) * LD, l0);
    const T y1 = r[0] * inv_diag[k + 1];
    if (act) {
      if (AS_COLUMN) Y[(k + 1) * LD + lane] = y1;
      else Y[lane * LD + k + 1] = y1;
    }
#pragma unroll
    for (int j = 0; j < DP - 1; ++j) r[j] = fma(-y1, l1[j + 1], r[j + 1]);
    r[DP - 1] = (T)0;
  }
}

// Two independent factorizations interleaved (ILP); outputs as in chol_rot.
template <typename T, int DP>
__device__ void chol_rot2(T (&a)[DP], T* LS, T* LR, T* invd, T (&b)[DP], T* LS2, T* invd2,
                          int d, int lane, int* bad) {
  constexpr int LD = Lay<T, DP>::LD;
  const bool act = lane < DP;
  __syncwarp();
  if (LR && act) {
    T z[DP];
    zero<T, DP>(z);
    st_vec<T, DP>(LR + lane * LD, z);
  }
  __syncwarp();
#pragma unroll 1
  for (int k = 0; k < DP; ++k) {
    T akk = __shfl_sync(FULL_MASK, a[0], k);
    T bkk = __shfl_sync(FULL_MASK, b[0], k);
    T pa = (T)1, pb = (T)1;
    if (k < d) {
      if (!(akk > (T)0) || !(akk < (T)INFINITY)) { *bad = 1; akk = (T)1; }
      if (!(bkk > (T)0) || !(bkk < (T)INFINITY)) { *bad = 1; bkk = (T)1; }
      pa = sqrt(akk);
      pb = sqrt(bkk);
    }
    const T ia = (T)1 / pa, ib = (T)1 / pb;
    const T la = (lane == k) ? pa : ((lane > k) ? a[0] * ia : (T)0);
    const T lb = (lane == k) ? pb : ((lane > k) ? b[0] * ib : (T)0);
    if (act && lane >= k) {
      LS[k * LD + (lane - k)] = la;
      LS2[k * LD + (lane - k)] = lb;
      if (LR) LR[lane * LD + (DP - 1) - (lane - k)] = la;
    }
    if (lane == 0) { invd[k] = ia; invd2[k] = ib; }
    __syncwarp();
    T ka[DP], kb[DP];
    ld_vec<T, DP>(LS + k * LD, ka);
    ld_vec<T, DP>(LS2 + k * LD, kb);
    const T na = -la, nb = -lb;
#pragma unroll
    for (int j = 0; j < DP - 1; ++j) {
      a[j] = fma(na, ka[j + 1], a[j + 1]);
      b[j] = fma(nb, kb[j + 1], b[j + 1]);
    }
    a[DP - 1] = (T)0;
    b[DP - 1] = (T)0;
  }
  __syncwarp();
}

// Forward solve L y = r for the lane's own r (consumed), rotating form.
// y is written to slot Y as column `lane` (Y[k][lane]) or as row `lane` (Y[lane][k]).
template <typename T, int DP, bool AS_COLUMN>
__device__ __forceinline__ void fsolve_rot(const T* LS, const T* inv_diag, T (&r)[DP], T* Y,
                                           int lane) {
  constexpr int LD = Lay<T, DP>::LD;
  const bool act = lane < DP;
#pragma unroll 1
  for (int k = 0; k < DP; ++k) {
    const T yk = r[0] * inv_diag[k];
    if (act) {
      if (AS_COLUMN) Y[k * LD + lane] = yk;
      else Y[lane * LD + k] = yk;
    }
    T lk[DP];
    ld_vec<T, DP>(LS + k * LD, lk);
    const T ny = -yk;
#pragma unroll
    for (int j = 0; j < DP - 1; ++j) r[j] = fma(ny, lk[j + 1], r[j + 1]);
    r[DP - 1] = (T)0;
  }
}

// Forward solves with one factor and several right-hand sides in one pass (one
// row of LS feeds every system): r1 and r2 are per lane (results written as
// columns `lane` of Y1 and Y2), rv is the same in every lane (result to yv).
template <typename T, int DP, bool TWO>
__device__ __forceinline__ void fsolve_multi(const T* LS, const T* inv_diag, T (&r1)[DP], T* Y1,
                                             T (&r2)[DP], T* Y2, T (&rv)[DP], T* yv, int lane) {
  constexpr int LD = Lay<T, DP>::LD;
  const bool act = lane < DP;
#pragma unroll 1
  for (int k = 0; k < DP; ++k) {
    const T id = inv_diag[k];
    const T y1 = r1[0] * id;
    const T y2 = TWO ? r2[0] * id : (T)0;
    const T yvk = rv[0] * id;
    if (act) {
      Y1[k * LD + lane] = y1;
      if (TWO) Y2[k * LD + lane] = y2;
    }
    if (lane == 0) yv[k] = yvk;
    T lk[DP];
    ld_vec<T, DP>(LS + k * LD, lk);
#pragma unroll
    for (int j = 0; j < DP - 1; ++j) {
      r1[j] = fma(-y1, lk[j + 1], r1[j + 1]);
      if (TWO) r2[j] = fma(-y2, lk[j + 1], r2[j + 1]);
      rv[j] = fma(-yvk, lk[j + 1], rv[j + 1]);
    }
    r1[DP - 1] = (T)0;
    if (TWO) r2[DP - 1] = (T)0;
    rv[DP - 1] = (T)0;
  }
}

// Forward solve L y = r with the same r in every lane; y goes to the vector slot yv.
template <typename T, int DP>
__device__ __forceinline__ void fsolve_vec(const T* LS, const T* inv_diag, T (&r)[DP], T* yv,
                                           int lane) {
  constexpr int LD = Lay<T, DP>::LD;
#pragma unroll 1
  for (int k = 0; k < DP; ++k) {
    const T yk = r[0] * inv_diag[k];
    if (lane == 0) yv[k] = yk;
    T lk[DP];
    ld_vec<T, DP>(LS + k * LD, lk);
    const T ny = -yk;
#pragma unroll
    for (int j = 0; j < DP - 1; ++j) r[j] = fma(ny, lk[j + 1], r[j + 1]);
    r[DP - 1] = (T)0;
  }
}

// Backward solve L^T y = r for the lane's own r (consumed), rotating from the
// right with the right-aligned rows LR; y is written as row `lane` of slot Y.
template <typename T, int DP>
__device__ __forceinline__ void bsolve_rot(const T* LR, const T* inv_diag, T (&r)[DP], T* Y,
                                           int lane) {
  constexpr int LD = Lay<T, DP>::LD;
  const bool act = lane < DP;
#pragma unroll 1
  for (int k = DP - 1; k >= 0; --k) {
    const T yk = r[DP - 1] * inv_diag[k];
    if (act) Y[lane * LD + k] = yk;
    T lr[DP];
    ld_vec<T, DP>(LR + k * LD, lr);
    const T ny = -yk;
#pragma unroll
    for (int m = DP - 1; m >= 1; --m) r[m] = fma(ny, lr[m - 1], r[m - 1]);
    r[0] = (T)0;
  }
}

// ---------------------------------------------------------------------------
// Register-tiled product for p in {16, 32}: lane (r, q) = (lane / 4, lane % 4)
// owns the output tile rows TR r .. TR r + TR - 1, columns TC q .. TC q + TC - 1
// (TR = p / 8, TC = p / 4; a 4 x 8 tile at p = 32), so each k needs TR + TC
// operand values per lane instead of p + 1.
//   Out = Init (+/-) A^T B   when A_COLS (left operand: columns of slot A)
//   Out = Init (+/-) A B     otherwise (left operand: rows of slot A)
// Init may be null (zero) or equal to Out. The caller orders the slot accesses
// (a __syncwarp() before the call if Out/Init were just written by other
// lanes, and after it before other lanes read Out).
// ---------------------------------------------------------------------------
template <typename T, int DP> struct Tile {
  static constexpr int TR = DP / 8, TC = DP / 4;
};

// N contiguous elements at an address aligned to N * sizeof(T) (N * sizeof(T) <= 16 or a
// multiple of 16): one or more vector loads/stores
template <typename T, int N>
__device__ __forceinline__ void ldn(const T* p, T (&r)[N]) {
  if constexpr (N * sizeof(T) % 16 == 0) {
    using V = typename Vec16<T>::V;
    constexpr int M = Vec16<T>::N;
#pragma unroll
    for (int q = 0; q < N / M; ++q) unpack<T>(reinterpret_cast<const V*>(p)[q], &r[q * M]);
  } else if constexpr (N == 2 && sizeof(T) == 4) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    r[0] = v.x; r[1] = v.y;
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) r[i] = p[i];
  }
}
template <typename T, int N>
__device__ __forceinline__ void stn(T* p, const T (&r)[N]) {
  if constexpr (N * sizeof(T) % 16 == 0) {
    using V = typename Vec16<T>::V;
    constexpr int M = Vec16<T>::N;
#pragma unroll
    for (int q = 0; q < N / M; ++q) reinterpret_cast<V*>(p)[q] = pack<T>(&r[q * M]);
  } else if constexpr (N == 2 && sizeof(T) == 4) {
    *reinterpret_cast<float2*>(p) = make_float2(r[0], r[1]);
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) p[i] = r[i];
  }
}

template <typename T, int DP, bool A_COLS, bool NEG>
__device__ __forceinline__ void mm_tile_regs(const T* A, const T* B, T (&acc)[Tile<T, DP>::TR][Tile<T, DP>::TC],
                                             int lane) {
  constexpr int TR = Tile<T, DP>::TR, TC = Tile<T, DP>::TC, LD = Lay<T, DP>::LD;
  static_assert(DP == 16 || DP == 32, "tiled product needs p = 16 or 32");
  const int r0 = (lane >> 2) * TR, c0 = (lane & 3) * TC;
#pragma unroll 1
  for (int k0 = 0; k0 < DP; k0 += 4) {
    T a[4][TR];
    if (A_COLS) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) ldn<T, TR>(A + (k0 + kk) * LD + r0, a[kk]);
    } else {
#pragma unroll
      for (int i = 0; i < TR; ++i) {
        T r4[4];
        ldn<T, 4>(A + (r0 + i) * LD + k0, r4);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) a[kk][i] = r4[kk];
      }
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      T b[TC];
      ldn<T, TC>(B + (k0 + kk) * LD + c0, b);
#pragma unroll
      for (int i = 0; i < TR; ++i) {
        const T ai = NEG ? -a[kk][i] : a[kk][i];
        fma_row<T, TC>(ai, b, acc[i]);
      }
    }
  }
}

template <typename T, int DP>
__device__ __forceinline__ void tile_load(const T* S, T (&acc)[Tile<T, DP>::TR][Tile<T, DP>::TC], int lane) {
  constexpr int TR = Tile<T, DP>::TR, TC = Tile<T, DP>::TC, LD = Lay<T, DP>::LD;
  const int r0 = (lane >> 2) * TR, c0 = (lane & 3) * TC;
#pragma unroll
  for (int i = 0; i < TR; ++i) {
    if (S) ldn<T, TC>(S + (r0 + i) * LD + c0, acc[i]);
    else
#pragma unroll
      for (int j = 0; j < TC; ++j) acc[i][j] = (T)0;
  }
}

template <typename T, int DP>
__device__ __forceinline__ void tile_store(T* S, const T (&acc)[Tile<T, DP>::TR][Tile<T, DP>::TC], int lane) {
  constexpr int TR = Tile<T, DP>::TR, TC = Tile<T, DP>::TC, LD = Lay<T, DP>::LD;
  const int r0 = (lane >> 2) * TR, c0 = (lane & 3) * TC;
#pragma unroll
  for (int i = 0; i < TR; ++i) stn<T, TC>(S + (r0 + i) * LD + c0, acc[i]);
}

template <typename T, int DP, bool A_COLS, bool NEG>
__device__ __forceinline__ void mm_tile_to_slot(const T* A, const T* B, const T* Init, T* Out, int lane) {
  T acc[Tile<T, DP>::TR][Tile<T, DP>::TC];
  tile_load<T, DP>(Init, acc, lane);
  mm_tile_regs<T, DP, A_COLS, NEG>(A, B, acc, lane);
  __syncwarp();
  tile_store<T, DP>(Out, acc, lane);
}

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Per-lane running sums of the per-step log-likelihood and MH terms. FP64
// arithmetic runs at a small fraction of the FP32 rate on this GPU, and a few
// FP64 operations per step on every warp of the step loops cost more than the
// loops' FP32 work, so in single precision the sum is carried as an
// unevaluated pair of floats hi + lo: each addend enters through Knuth's
// two-sum (the rounding error of hi + x, exact) and a product x y through its
// exact split x y = p + fma(x, y, -p), which keeps about 48 significant bits
// over a block of steps; the pair is converted to FP64 once per block. The
// intrinsics keep the compiler from contracting the error terms. In double
// precision the sum is a plain double.
// ---------------------------------------------------------------------------
template <typename Real> struct TermSum;
template <> struct TermSum<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ void add_prod(double x, double y) { v += x * y; }
  __device__ __forceinline__ void add_f64(double x) { v += x; }
  __device__ __forceinline__ double value() const { return v; }
};
template <> struct TermSum<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp)));
    hi = s;
  }
  __device__ __forceinline__ void add_prod(float x, float y) {
    const float p = __fmul_rn(x, y);
    add(p);
    lo = __fadd_rn(lo, __fmaf_rn(x, y, -p));
  }
  // an FP64 addend (rare paths): its float head and the float of the remainder
  __device__ __forceinline__ void add_f64(double x) {
    const float h = (float)x;
    add(h);
    lo = __fadd_rn(lo, (float)(x - (double)h));
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// ---------------------------------------------------------------------------
// Column-sliced products for several warps sharing one d x d product: the
// lane's row, output columns c0 .. c0 + NC - 1 (c0 a multiple of NC, NC * size
// a multiple of 16 bytes).
//   mm_row_c:  out[j] (+/-)= sum_k arow[k] B[k][c0 + j]     (arow: shared row)
//   mm_col_c:  out[j] (+/-)= sum_k A[k][col] B[k][c0 + j]   (column col of slot A)
// ---------------------------------------------------------------------------
template <typename T, int DP, int NC, bool ACC = false, bool NEG = false>
__device__ __forceinline__ void mm_row_c(const T* arow, const T* B, int c0, T (&out)[NC]) {
  constexpr int LD = Lay<T, DP>::LD;
  if (!ACC) {
#pragma unroll
    for (int j = 0; j < NC; ++j) out[j] = (T)0;
  }
#pragma unroll 4
  for (int k = 0; k < DP; ++k) {
    const T ak = NEG ? -arow[k] : arow[k];
    T b[NC];
    ldn<T, NC>(B + k * LD + c0, b);
    fma_row<T, NC>(ak, b, out);
  }
}

template <typename T, int DP, int NC, bool ACC = false, bool NEG = false>
__device__ __forceinline__ void mm_col_c(const T* A, int col, const T* B, int c0, T (&out)[NC]) {
  constexpr int LD = Lay<T, DP>::LD;
  if (!ACC) {
#pragma unroll
    for (int j = 0; j < NC; ++j) out[j] = (T)0;
  }
#pragma unroll 4
  for (int k = 0; k < DP; ++k) {
    const T ak = NEG ? -A[k * LD + col] : A[k * LD + col];
    T b[NC];
    ldn<T, NC>(B + k * LD + c0, b);
    fma_row<T, NC>(ak, b, out);
  }
}

// ---------------------------------------------------------------------------
// Asynchronous global -> shared copies (16 bytes per instruction, L1 bypassed)
// used to stage the next step's tables while the current step computes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Copy ntab row-major DP x DP matrices, src0 + j * stride (j < ntab), into
// consecutive padded slots at dst (all threads of the CTA take part), then
// close the copy group.
template <typename T, int DP>
__device__ __forceinline__ void stage_mats(T* dst, const T* src0, long stride, int ntab) {
  constexpr int N = Vec16<T>::N, CPR = DP / N, LD = Lay<T, DP>::LD, MAT = Lay<T, DP>::MAT;
  constexpr int PER = DP * CPR;
  for (int q = threadIdx.x; q < ntab * PER; q += blockDim.x) {
    const int j = q / PER, rem = q - j * PER, r = rem / CPR, cc = rem - r * CPR;
    cp_async16(dst + j * MAT + r * LD + cc * N, src0 + j * stride + r * DP + cc * N);
  }
  cp_async_commit();
}

}  // namespace auxk
