// aux_noalloc.cu — aux_loglik_noalloc: the log-likelihood pass without any
// device allocation, for callers that cannot call cudaMalloc (code running
// under an allocator it must not bypass, inside a host callback, or in a
// process whose device-memory budget is fixed up front).
//
// Its scratch (padded model, block aggregates, partial sums,
// status words) lives in one file-scope device array of AUX_NOALLOC_SCRATCH_BYTES.
// The array is part of the library's module: every GPU that loads the library
// holds it until the process exits. All calls share it, so calls whose work
// overlaps on the GPU (different streams, or several host threads) race and
// must be serialised by the caller. The per-device set-up (the array's device
// address, kernel attributes) is guarded by a lock, so first calls from several
// host threads do not race on it. Each call is synchronous: it returns after
// its pass has finished and its status words have been read back.
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>

#include "aux_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[AUX_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {};     // device address of the array, per device
// set-up done per device (address known) and per (device, dtype, DP) (kernels
// configured); written under g_setup_lock, read lock-free once set
std::atomic<bool> g_ready[kMaxDevices];
std::atomic<bool> g_ready_ops[kMaxDevices][2][33];
std::mutex g_setup_lock;

// One-time set-up for the current device `dev` and the kernels of (dtype, DP).
int setup_device(int dev, int dtype, int DP, const AuxOps* ops) {
  if (g_ready[dev].load(std::memory_order_acquire) &&
      g_ready_ops[dev][dtype][DP].load(std::memory_order_acquire))
    return AUX_OK;
  std::lock_guard<std::mutex> lock(g_setup_lock);
  if (!g_ready[dev].load(std::memory_order_relaxed)) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return AUX_E_CUDA;
    g_scratch_ptr[dev] = p;
    g_ready[dev].store(true, std::memory_order_release);
  }
  if (!g_ready_ops[dev][dtype][DP].load(std::memory_order_relaxed)) {
    if (ops->prepare() != AUX_OK) return AUX_E_CUDA;
    g_ready_ops[dev][dtype][DP].store(true, std::memory_order_release);
  }
  return AUX_OK;
}

// After the pass: the OR of the status words [2][C] (per-iteration and latched)
// and the finiteness of logZ[C], read back in chunks through host stack buffers
// (waits for the stream). A failed factorisation gives AUX_E_NOT_PD, a
// non-finite status bit or log-likelihood AUX_E_NONFINITE.
int read_status(const unsigned char* st_iter, const unsigned char* st, const double* logZ, int C,
                cudaStream_t s) {
  constexpr int CH = 512;
  int32_t h[2][CH];
  double z[CH];
  int32_t any = 0;
  bool finite_z = true;
  for (int c0 = 0; c0 < C; c0 += CH) {
    const int n = C - c0 < CH ? C - c0 : CH;
    const size_t off = (size_t)c0 * sizeof(int32_t);
    if (cudaMemcpyAsync(h[0], st_iter + off, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(h[1], st + off, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(z, logZ + c0, n * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return AUX_E_CUDA;
    for (int i = 0; i < n; ++i) {
      any |= h[0][i] | h[1][i];
      if (!std::isfinite(z[i])) finite_z = false;
    }
  }
  if (any & 1) return AUX_E_NOT_PD;
  if ((any & 2) || !finite_z) return AUX_E_NONFINITE;
  return AUX_OK;
}

int pick_dp_noalloc(int d) {
  if (d <= 4) return 4;
  if (d <= 8) return 8;
  if (d <= 16) return 16;
  if (d <= 32) return 32;
  return 0;
}

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

// byte offsets of the scratch regions for one problem size
struct Layout {
  size_t F, Q, P0, m0, b, Ryinv, agg0, agg1, lz, st_iter, st, total;
};

Layout layout(int DP, int C, int nb, size_t esz) {
  Layout L{};
  size_t o = 0;
  const size_t mat = align256((size_t)DP * DP * esz), vec = align256((size_t)DP * esz);
  L.F = o; o += mat;
  L.Q = o; o += mat;
  L.P0 = o; o += mat;
  L.m0 = o; o += vec;
  L.b = o; o += vec;
  L.Ryinv = o; o += mat;
  L.agg0 = o; o += align256((size_t)C * nb * aux_es(DP) * esz);
  L.agg1 = o; o += align256((size_t)C * nb * aux_es(DP) * esz);
  L.lz = o; o += align256((size_t)C * nb * sizeof(double));
  L.st_iter = o; o += align256((size_t)C * sizeof(int32_t));
  L.st = o; o += align256((size_t)C * sizeof(int32_t));
  L.total = o;
  return L;
}

bool finite(const double* a, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

// SPD check of a small symmetric matrix without heap memory (d <= 32)
bool spd(const double* A, int d) {
  double L[32 * 32];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < i; ++j) {
      const double a = A[i * d + j], b = A[j * d + i];
      if (std::fabs(a - b) > 1e-12 * (std::fabs(a) + std::fabs(b) + 1e-300)) return false;
    }
  for (int j = 0; j < d; ++j) {
    double s = A[j * d + j];
    for (int k = 0; k < j; ++k) s -= L[j * 32 + k] * L[j * 32 + k];
    if (!(s > 0.0)) return false;
    const double ljj = std::sqrt(s);
    L[j * 32 + j] = ljj;
    for (int i = j + 1; i < d; ++i) {
      double t = A[i * d + j];
      for (int k = 0; k < j; ++k) t -= L[i * 32 + k] * L[j * 32 + k];
      L[i * 32 + j] = t / ljj;
    }
  }
  return true;
}

// pad a d x d (or d) host array into a DP x DP (or DP) staging block of the compute type
template <typename Real>
void stage(const double* src, int d, int DP, bool matrix, Real* dst) {
  const int n = matrix ? DP * DP : DP;
  for (int i = 0; i < n; ++i) dst[i] = (Real)0;
  if (!src) return;
  if (matrix) {
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) dst[i * DP + j] = (Real)src[i * d + j];
  } else {
    for (int i = 0; i < d; ++i) dst[i] = (Real)src[i];
  }
}

template <typename Real>
int upload_model(const aux_model_desc* desc, int DP, unsigned char* base, const Layout& L,
                 cudaStream_t st) {
  // one staging block on the host stack: F, Q, P0 (DP x DP) and m0, b (DP)
  Real buf[3 * 32 * 32 + 2 * 32];
  Real* F = buf;
  Real* Q = F + DP * DP;
  Real* P0 = Q + DP * DP;
  Real* m0 = P0 + DP * DP;
  Real* b = m0 + DP;
  stage<Real>(desc->F, desc->d_x, DP, true, F);
  stage<Real>(desc->Q, desc->d_x, DP, true, Q);
  stage<Real>(desc->P0, desc->d_x, DP, true, P0);
  stage<Real>(desc->m0, desc->d_x, DP, false, m0);
  stage<Real>(desc->b, desc->d_x, DP, false, b);
  const size_t mb = (size_t)DP * DP * sizeof(Real), vb = (size_t)DP * sizeof(Real);
  cudaError_t e = cudaMemcpyAsync(base + L.F, F, mb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + L.Q, Q, mb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + L.P0, P0, mb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + L.m0, m0, vb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + L.b, b, vb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + L.Ryinv, 0, mb, st);
  // the host staging block lives on this stack frame: wait for the copies
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? AUX_OK : AUX_E_CUDA;
}

}  // namespace

extern "C" int aux_loglik_noalloc(const aux_model_desc* desc, const void* ytilde, double* logZ,
                                  void* stream) {
  if (!desc || !ytilde || !logZ) return AUX_E_INVALID_ARG;
  if (desc->abi_version != AUX_ABI_VERSION) return AUX_E_INVALID_ARG;
  if (desc->dtype != AUX_F32 && desc->dtype != AUX_F64) return AUX_E_INVALID_ARG;
  if (desc->dyn_kind != AUX_DYN_HOMOGENEOUS) return AUX_E_UNSUPPORTED;   // one transition (F, b, Q)
  const int d = desc->d_x, T = desc->T, C = desc->n_chains;
  if (d < 1 || T < 1 || C < 1 || desc->block_len < 0) return AUX_E_INVALID_ARG;
  if (!desc->m0 || !desc->P0 || !desc->F || !desc->b || !desc->Q) return AUX_E_INVALID_ARG;
  if (!(desc->delta > 0.0) || !std::isfinite(desc->delta)) return AUX_E_INVALID_ARG;
  const int DP = pick_dp_noalloc(d);
  if (DP == 0 || (desc->dtype == AUX_F64 && DP > 16)) return AUX_E_UNSUPPORTED;
  const size_t dd = (size_t)d * d;
  if (!finite(desc->m0, d) || !finite(desc->P0, dd) || !finite(desc->F, dd) ||
      !finite(desc->b, d) || !finite(desc->Q, dd))
    return AUX_E_NONFINITE;
  if (!spd(desc->P0, d) || !spd(desc->Q, d)) return AUX_E_NOT_PD;

  int L_blk = desc->block_len;
  if (L_blk == 0) L_blk = (int)std::ceil(std::sqrt((double)T));
  if (L_blk < 1) L_blk = 1;
  if (L_blk > T) L_blk = T;
  const int nb = (T + L_blk - 1) / L_blk;
  const size_t esz = desc->dtype == AUX_F32 ? sizeof(float) : sizeof(double);
  const Layout lay = layout(DP, C, nb, esz);
  if (lay.total > (size_t)AUX_NOALLOC_SCRATCH_BYTES) return AUX_E_TOO_LARGE;

  cudaStream_t st = (cudaStream_t)stream;
  // The call synchronises its stream and reads host stack memory: it cannot be
  // part of a captured graph. Refuse before anything is enqueued.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
    return AUX_E_UNSUPPORTED;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return AUX_E_CUDA;
  const AuxOps* ops = desc->dtype == AUX_F32 ? aux_ops_f32(DP) : aux_ops_f64(DP);
  if (!ops) return AUX_E_UNSUPPORTED;
  // set-up, once per device (this device is current): the array's device address
  // and the kernels' attributes
  if (setup_device(dev, desc->dtype, DP, ops) != AUX_OK) return AUX_E_CUDA;

  unsigned char* base = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  int rc = desc->dtype == AUX_F32 ? upload_model<float>(desc, DP, base, lay, st)
                                  : upload_model<double>(desc, DP, base, lay, st);
  if (rc) return rc;
  // status words must start at zero; everything else is fully written by the pass
  if (cudaMemsetAsync(base + lay.st_iter, 0, 2 * align256((size_t)C * sizeof(int32_t)), st) != cudaSuccess)
    return AUX_E_CUDA;

  // a handle on the stack whose buffers all point into the scratch array
  aux_model m;
  m.dtype = desc->dtype; m.d = d; m.DP = DP; m.T = T; m.C = C;
  m.emis = desc->emis_kind; m.y_per_chain = 0;
  m.L = L_blk; m.nb = nb; m.delta = desc->delta; m.seed = 0; m.esz = esz;
  m.stream = st; m.device = dev; m.ops = ops;
  if (cudaDeviceGetAttribute(&m.n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return AUX_E_CUDA;
  m.fdiag = 1;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      if (i != j && desc->F[i * d + j] != 0.0) m.fdiag = 0;
  m.F = base + lay.F; m.Q = base + lay.Q; m.P0 = base + lay.P0;
  m.m0 = base + lay.m0; m.b = base + lay.b; m.Ryinv = base + lay.Ryinv;
  m.agg0 = base + lay.agg0; m.agg1 = base + lay.agg1;
  m.lz_part = reinterpret_cast<double*>(base + lay.lz);
  m.status_iter = reinterpret_cast<int32_t*>(base + lay.st_iter);
  m.status = reinterpret_cast<int32_t*>(base + lay.st);
  rc = ops->loglik(&m, ytilde, logZ, nullptr, nullptr, st);
  if (rc) return rc;
  // wait for the pass and report a failed factorisation or a non-finite value
  return read_status(base + lay.st_iter, base + lay.st, logZ, C, st);
}
