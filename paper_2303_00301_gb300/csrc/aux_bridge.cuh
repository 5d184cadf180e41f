// aux_bridge.cuh — the divide-and-conquer (bridging) pathwise sampler,
// Section 2.4.2 and Appendix A.2.3: an alternative to the (G, U) suffix scan
// of Proposition A.1 with the same O(log T) depth.
//
// The backward conditionals p(x_t | x_{t+1}, y) = N(E x_{t+1} + g, L) with
// (E, g, L) = (G_t, m^f_t - G_t m^p_{t+1}, Sigma_t) are the leaves of the
// dyadic tree over the n = T - 1 unit intervals: node a of level j covers
// [a 2^j, min((a+1) 2^j, n)] and joins children 2a and 2a+1 of level j - 1
//   E = E_l E_r,  g = E_l g_r + g_l,  L = E_l L_r E_l^T + L_l,
// and, at its split point l = (2a+1) 2^(j-1), the bridge
//   G = L_r E_l^T L^{-1},  Gamma = E_r - G E,  V = L_r - G L G^T,
//   p(x_l | x_k, x_m, y) = N(G x_k + Gamma x_m + g_r - G g, V).
// A node without a right child (ragged n) is its left child.
//
// The matrices depend only on the covariances: in the table modes (first
// order, R = (delta/2) I) one tree serves every chain and is built once per
// covariance pass; in the per-chain mode every chain has its own. The
// vectors g and the draws are per chain:
//   k_br_leaf   leaf covariances Sigma_t = LS_t LS_t^T from the Cholesky table;
//   k_br_node   one warp per node (and chain): E, L and the bridge (G, Gamma,
//               chol V), level by level from the leaves up;
//   k_b_sample  one cluster of 8 CTAs per chain, tree levels separated by
//               cluster barriers: g of every node, leaves up; the two ends,
//               x_{T-1} = m^f + chol(P^f) eps_{T-1} and
//               x_0 = E x_{T-1} + g + chol(L) eps_0 with the root's (E, g, L);
//               the split points x_l from x_k and x_m, root down;
//   k_b_mh      one warp per (chain, block): the MH terms at x* (as in the
//               scan sampler's last kernel).
// State t draws eps_t of the backward stream (or row t of the given eps), at
// whichever level it is sampled.
#pragma once
#include "aux_kernels.cuh"

namespace auxk {

// tree of one chain; the chain strides are 0 when the tree is shared
template <typename Real> struct BrTree {
  const Real* G0; long g0_cs;   // leaf E = G_t at G0 + c g0_cs + t DD
  const Real* L0; long l0_cs;   // leaf L = Sigma_t at L0 + c l0_cs + t DD
  Real* E;                      // internal nodes: E at E + c nn_cs + i DD
  Real* L;                      // L at L + c nn_cs + i DD
  Real* B;                      // bridges at B + 3 c nn_cs + 3 i DD: G, Gamma, chol V (row-major, lower)
  long nn_cs;                   // NN DD, or 0
  int32_t* status;              // ST_NOT_PD: status[0] (shared tree) or status[c]
  int per_chain_status;
};

// per-chain vectors and outputs
template <typename Real> struct BrMeans {
  const Real* U;                // [C][T][DP] leaf g_t (noise-free U_t; U_{T-1} = m^f_{T-1})
  Real* gN;                     // [C][NN][DP] g of the internal nodes
  const Real* PT; long pt_cs;   // P^f_{T-1} (row-major) at PT + c pt_cs
  Real* xs;                     // [C][T][d] the draw
  const Real* eps;              // [C][T][d] or null: Philox backward stream
  uint64_t iter;
  int NN;
};

// one level of the tree (levels j >= 1; level 0 is the leaves)
struct BrLevel {
  int j, off, cnt;    // level, index of its first node among the internal nodes, node count
  int coff, ccnt;     // the same for its children (coff unused when j == 1)
};

template <typename Real, int DP> struct BrSizes {
  static constexpr int MAT = Lay<Real, DP>::MAT, VEC = Lay<Real, DP>::VEC;
  static constexpr size_t NODE_SMEM = (8 * MAT + 2 * VEC) * sizeof(Real);
  static constexpr int WPC = 8;   // warps per CTA of the MH-terms kernel
  // k_b_sample: 8 warps x 3 vectors, the ends' Cholesky slot and 3 vectors
  static constexpr size_t SAMPLE_SMEM = (8 * 3 * VEC + MAT + 3 * VEC) * sizeof(Real);
};

// E and L of node idx of level j (j == 0: a leaf) of chain c
template <typename Real, int DP>
__device__ __forceinline__ const Real* node_E(const BrTree<Real>& tr, int j, int off, int idx, int c) {
  constexpr long DD = (long)DP * DP;
  return j == 0 ? tr.G0 + c * tr.g0_cs + idx * DD : tr.E + c * tr.nn_cs + (off + idx) * DD;
}
template <typename Real, int DP>
__device__ __forceinline__ const Real* node_L(const BrTree<Real>& tr, int j, int off, int idx, int c) {
  constexpr long DD = (long)DP * DP;
  return j == 0 ? tr.L0 + c * tr.l0_cs + idx * DD : tr.L + c * tr.nn_cs + (off + idx) * DD;
}
// g of node idx of level j of chain c
template <typename Real, int DP>
__device__ __forceinline__ const Real* node_g(const BrMeans<Real>& mv, int nT, int j, int off, int idx,
                                              int c) {
  return j == 0 ? mv.U + ((long)c * nT + idx) * DP : mv.gN + ((long)c * mv.NN + off + idx) * DP;
}

// ---------------------------------------------------------------------------
// Leaf covariances of the table modes: L0[t] = LS_t LS_t^T, t < n (one warp per t).
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __launch_bounds__(256) k_br_leaf(const Real* __restrict__ LS, Real* __restrict__ L0,
                                                 int n) {
  constexpr long DD = (long)DP * DP;
  const int lane = threadIdx.x & 31;
  const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (t >= n || lane >= DP) return;
  const Real* S = LS + t * DD;
  Real ri[DP], out[DP];
  ld_vec<Real, DP>(S + lane * DP, ri);
#pragma unroll 4
  for (int j = 0; j < DP; ++j) {
    Real rj[DP];
    ld_vec<Real, DP>(S + j * DP, rj);
    out[j] = dot_rr<Real, DP>(ri, rj);
  }
  st_vec<Real, DP>(L0 + t * DD + lane * DP, out);
}

// ---------------------------------------------------------------------------
// One node of level lv.j for chain blockIdx.x / cnt (one warp per CTA).
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __launch_bounds__(32, 1) k_br_node(KP<Real> p, BrTree<Real> tr, BrLevel lv) {
  refresh_delta(p);
  using Z = BrSizes<Real, DP>;
  constexpr int MAT = Z::MAT, LD = Lay<Real, DP>::LD;
  constexpr long DD = (long)DP * DP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  Real* SEL = sm;             // E_l, later the right-aligned rows of chol(L)
  Real* SELT = SEL + MAT;     // E_l^T, later G
  Real* SER = SELT + MAT;     // E_r
  Real* SLRc = SER + MAT;     // L_r
  Real* ST1 = SLRc + MAT;     // T1 = E_l L_r
  Real* SE = ST1 + MAT;       // E
  Real* SY = SE + MAT;        // scratch
  Real* SLS = SY + MAT;       // Cholesky working slot
  Real* invd = SLS + MAT;
  const int lane = threadIdx.x;
  const int c = blockIdx.x / lv.cnt, a = blockIdx.x % lv.cnt;
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  const int jc = lv.j - 1;
  const bool two = 2 * a + 1 < lv.ccnt;
  Real* Eo = tr.E + c * tr.nn_cs + (long)(lv.off + a) * DD;
  Real* Lo = tr.L + c * tr.nn_cs + (long)(lv.off + a) * DD;
  const Real* EL = node_E<Real, DP>(tr, jc, lv.coff, 2 * a, c);
  const Real* LL = node_L<Real, DP>(tr, jc, lv.coff, 2 * a, c);
  Real el[DP], r[DP];
  ld_vec<Real, DP>(EL + row * DP, el);
  if (!two) {   // the node is its left child
    ld_vec<Real, DP>(LL + row * DP, r);
    if (act) { st_vec<Real, DP>(Eo + row * DP, el); st_vec<Real, DP>(Lo + row * DP, r); }
    return;
  }
  const Real* ER = node_E<Real, DP>(tr, jc, lv.coff, 2 * a + 1, c);
  const Real* LR = node_L<Real, DP>(tr, jc, lv.coff, 2 * a + 1, c);
  st_row<Real, DP>(SEL, row, el, act);
  st_col<Real, DP>(SELT, row, el, act);
  ld_vec<Real, DP>(ER + row * DP, r);
  st_row<Real, DP>(SER, row, r, act);
  ld_vec<Real, DP>(LR + row * DP, r);
  st_row<Real, DP>(SLRc, row, r, act);
  __syncwarp();
  Real t1[DP], er[DP];
  mm_row<Real, DP>(SEL + row * LD, SLRc, t1);   // T1 = E_l L_r
  mm_row<Real, DP>(SEL + row * LD, SER, er);    // E = E_l E_r
  st_row<Real, DP>(ST1, row, t1, act);
  st_row<Real, DP>(SE, row, er, act);
  __syncwarp();
  Real lr[DP];
  ld_vec<Real, DP>(LL + row * DP, lr);
  mm_row<Real, DP, true>(ST1 + row * LD, SELT, lr);   // L = T1 E_l^T + L_l
  symmetrise_store<Real, DP>(SY, lr, lane);
  if (act) { st_vec<Real, DP>(Eo + row * DP, er); st_vec<Real, DP>(Lo + row * DP, lr); }
  int bad = 0;
  // G = T1^T L^{-1}: G^T = L^{-1} T1 by a forward and a backward solve per column of T1
  chol_rot<Real, DP>(lr, SLS, nullptr, SEL, invd, nullptr, p.d, lane, &bad);
  {
    Real rr[DP];
    ld_col<Real, DP>(ST1, row, rr);
    fsolve_rot<Real, DP, true>(SLS, invd, rr, SY, lane);
  }
  __syncwarp();
  {
    Real rr[DP];
    ld_col<Real, DP>(SY, row, rr);
    bsolve_rot<Real, DP>(SEL, invd, rr, SELT, lane);   // SELT <- G (rows)
  }
  __syncwarp();
  Real* Bo = tr.B + 3 * c * tr.nn_cs + 3 * (long)(lv.off + a) * DD;
  Real gr[DP];
  ld_row<Real, DP>(SELT, row, gr);
  if (act) st_vec<Real, DP>(Bo + row * DP, gr);
  Real gm[DP];
  ld_row<Real, DP>(SER, row, gm);
  mm_row<Real, DP, true, true>(SELT + row * LD, SE, gm);   // Gamma = E_r - G E
  if (act) st_vec<Real, DP>(Bo + DD + row * DP, gm);
  // V = L_r - G L G^T = L_r - G T1 (L G^T = T1)
  Real vr[DP];
  ld_row<Real, DP>(SLRc, row, vr);
  mm_row<Real, DP, true, true>(SELT + row * LD, ST1, vr);
  symmetrise_store<Real, DP>(SY, vr, lane);
  chol_rot<Real, DP>(vr, SLS, SY, nullptr, invd, nullptr, p.d, lane, &bad);
  __syncwarp();
  ld_row<Real, DP>(SY, row, vr);
  if (act) st_vec<Real, DP>(Bo + 2 * DD + row * DP, vr);
  if (bad && lane == 0) atomicOr(tr.status + (tr.per_chain_status ? c : 0), ST_NOT_PD);
}

// the backward-stream normal of state t for the lane (0 past d)
template <typename Real>
__device__ __forceinline__ Real br_eps(const KP<Real>& p, const BrMeans<Real>& mv, int c, int t, int lane) {
  if (lane >= p.d) return (Real)0;
  return mv.eps ? mv.eps[((long)c * p.nT + t) * p.d + lane]
                : philox_normal<Real>(p.seed, (uint32_t)c, iter_of(p, mv.iter), PURPOSE_BACKWARD, (uint32_t)t, lane);
}

// g of node a of level lv.j for chain c: g = E_l g_r + g_l (one warp; vg: warp-private vector)
template <typename Real, int DP>
__device__ __forceinline__ void br_up_node(const KP<Real>& p, const BrTree<Real>& tr, const BrMeans<Real>& mv,
                                           const BrLevel& lv, int c, int a, Real* vg, int lane) {
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  const int jc = lv.j - 1;
  const bool two = 2 * a + 1 < lv.ccnt;
  // every global load of the node first, so that their latencies overlap
  Real e[DP];
  if (two) ld_vec<Real, DP>(node_E<Real, DP>(tr, jc, lv.coff, 2 * a, c) + row * DP, e);
  const Real gl = node_g<Real, DP>(mv, p.nT, jc, lv.coff, 2 * a, c)[row];
  const Real grv = two ? node_g<Real, DP>(mv, p.nT, jc, lv.coff, 2 * a + 1, c)[row] : (Real)0;
  Real out = gl;
  if (two) {
    __syncwarp();
    if (act) vg[lane] = grv;
    __syncwarp();
    out = dot_rv<Real, DP>(e, vg) + gl;
  }
  if (act) mv.gN[((long)c * mv.NN + lv.off + a) * DP + lane] = out;
}

// the two ends of chain c's path (one warp): x_{T-1} | y, then x_0 | x_{T-1}, y.
// root: level and index of the root among the internal nodes (n >= 2), or the leaf 0 (n == 1).
template <typename Real, int DP>
__device__ __forceinline__ void br_root(const KP<Real>& p, const BrTree<Real>& tr, const BrMeans<Real>& mv,
                                        int root_j, int root_off, int c, Real* SLS, Real* invd, Real* ve,
                                        Real* vx, int lane) {
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  const int n = p.nT - 1;
  int bad = 0;
  const Real e_n = br_eps<Real>(p, mv, c, n, lane);
  if (act) ve[lane] = e_n;
  __syncwarp();
  Real a[DP];
  ld_vec<Real, DP>(mv.PT + c * mv.pt_cs + row * DP, a);
  const Real le = chol_rot<Real, DP>(a, SLS, nullptr, nullptr, invd, ve, p.d, lane, &bad);
  const Real xn = mv.U[((long)c * p.nT + n) * DP + row] + le;
  if (lane < p.d) mv.xs[((long)c * p.nT + n) * p.d + lane] = xn;
  if (n >= 1) {
    const Real e0 = br_eps<Real>(p, mv, c, 0, lane);
    __syncwarp();
    if (act) { ve[lane] = e0; vx[lane] = xn; }
    __syncwarp();
    ld_vec<Real, DP>(node_L<Real, DP>(tr, root_j, root_off, 0, c) + row * DP, a);
    const Real l0 = chol_rot<Real, DP>(a, SLS, nullptr, nullptr, invd, ve, p.d, lane, &bad);
    Real er[DP];
    ld_vec<Real, DP>(node_E<Real, DP>(tr, root_j, root_off, 0, c) + row * DP, er);
    const Real x0 = dot_rv<Real, DP>(er, vx) + node_g<Real, DP>(mv, p.nT, root_j, root_off, 0, c)[row] + l0;
    if (lane < p.d) mv.xs[(long)c * p.nT * p.d + lane] = x0;
  }
  if (bad && lane == 0) atomicOr(&p.status_iter[c], ST_NOT_PD);
}

// split point of node a of level lv.j for chain c (one warp):
// x_l = G (x_k - g) + Gamma x_m + g_r + chol(V) eps_l
template <typename Real, int DP>
__device__ __forceinline__ void br_down_node(const KP<Real>& p, const BrTree<Real>& tr, const BrMeans<Real>& mv,
                                             const BrLevel& lv, int c, int a, Real* v1, Real* v2, Real* v3,
                                             int lane) {
  constexpr long DD = (long)DP * DP;
  if (2 * a + 1 >= lv.ccnt) return;   // no split point (warp-uniform)
  const int n = p.nT - 1;
  const int k = a << lv.j, l = (2 * a + 1) << (lv.j - 1), m = min((a + 1) << lv.j, n);
  const bool act = lane < DP;
  const int row = act ? lane : 0;
  const long cx = (long)c * p.nT * p.d;
  // every global load of the node first, so that their latencies overlap
  const Real* Bn = tr.B + 3 * c * tr.nn_cs + 3 * (long)(lv.off + a) * DD;
  Real rg[DP], rm[DP], rv[DP];
  ld_vec<Real, DP>(Bn + row * DP, rg);
  ld_vec<Real, DP>(Bn + DD + row * DP, rm);
  ld_vec<Real, DP>(Bn + 2 * DD + row * DP, rv);
  const Real g = node_g<Real, DP>(mv, p.nT, lv.j, lv.off, a, c)[row];
  const Real gr = node_g<Real, DP>(mv, p.nT, lv.j - 1, lv.coff, 2 * a + 1, c)[row];
  const Real xk = lane < p.d ? mv.xs[cx + (long)k * p.d + lane] : (Real)0;
  const Real xm = lane < p.d ? mv.xs[cx + (long)m * p.d + lane] : (Real)0;
  const Real el = br_eps<Real>(p, mv, c, l, lane);
  __syncwarp();
  if (act) { v1[lane] = xk - g; v2[lane] = xm; v3[lane] = el; }
  __syncwarp();
  Real x = dot_rv<Real, DP>(rg, v1) + gr;
  x += dot_rv<Real, DP>(rm, v2);
  x += dot_rv<Real, DP>(rv, v3);
  if (lane < p.d) mv.xs[cx + (long)l * p.d + lane] = x;
}

// all levels of the tree, in kernel parameters
constexpr int BR_MAX_LEVELS = 30;
struct BrLevels {
  BrLevel l[BR_MAX_LEVELS];
  int n;
};

// one cluster of BR_CLUSTER CTAs per chain; a cluster barrier (hardware,
// release / acquire at cluster scope, so the global writes of one level are
// visible to the next level's readers) separates the tree levels
constexpr int BR_CLUSTER = 8, BR_WARPS = 8;
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// ---------------------------------------------------------------------------
// The draw of one chain per cluster: node offsets g up the tree (level by
// level), the two ends (CTA 0, warp 0), the split points down the tree. The
// warps of the cluster share the nodes of a level; every thread reaches every
// barrier.
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __cluster_dims__(BR_CLUSTER, 1, 1) __launch_bounds__(32 * BR_WARPS)
    k_b_sample(KP<Real> p, BrTree<Real> tr, BrMeans<Real> mv, BrLevels lv, int root_j, int root_off) {
  using Z = BrSizes<Real, DP>;
  constexpr int MAT = Z::MAT, VEC = Z::VEC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Real* v1 = sm + warp * 3 * VEC;
  Real* v2 = v1 + VEC;
  Real* v3 = v2 + VEC;
  Real* SLS = sm + BR_WARPS * 3 * VEC;     // the ends: Cholesky slot and vectors
  Real* invd = SLS + MAT;
  Real* ve = invd + VEC;
  Real* vx = ve + VEC;
  const int c = blockIdx.x / BR_CLUSTER, rank = blockIdx.x % BR_CLUSTER;
  const int gw = rank * BR_WARPS + warp, nw = BR_CLUSTER * BR_WARPS;
  for (int j = 0; j < lv.n; ++j) {
    const BrLevel L = lv.l[j];
    for (int a = gw; a < L.cnt; a += nw) br_up_node<Real, DP>(p, tr, mv, L, c, a, v1, lane);
    cluster_barrier();
  }
  if (rank == 0 && warp == 0) br_root<Real, DP>(p, tr, mv, root_j, root_off, c, SLS, invd, ve, vx, lane);
  cluster_barrier();
  for (int j = lv.n - 1; j >= 0; --j) {
    const BrLevel L = lv.l[j];
    for (int a = gw; a < L.cnt; a += nw) br_down_node<Real, DP>(p, tr, mv, L, c, a, v1, v2, v3, lane);
    cluster_barrier();
  }
}

// ---------------------------------------------------------------------------
// MH terms at the drawn x* (one warp per (chain, block)), as the scan sampler's
// last kernel computes them: per-block sums into b.mh_part, ytilde* into b.yts.
// ---------------------------------------------------------------------------
template <typename Real, int DP>
__global__ void __launch_bounds__(32 * BrSizes<Real, DP>::WPC) k_b_mh(KP<Real> p, BackArgs<Real> b) {
  using Z = BrSizes<Real, DP>;
  constexpr int MAT = Lay<Real, DP>::MAT, VEC = Z::VEC, LD = Lay<Real, DP>::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  refresh_delta(p);
  Real* sRy = reinterpret_cast<Real*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Real* vxs = sRy + MAT + warp * VEC;
  if (p.emis == AUX_EMIS_LINEAR_GAUSSIAN)
    for (int q = threadIdx.x; q < DP * DP; q += blockDim.x) sRy[(q / DP) * LD + q % DP] = p.Ryinv[q];
  __syncthreads();
  const long item = (long)blockIdx.x * Z::WPC + warp;
  if (item >= (long)p.C * p.nb) return;
  const int c = (int)(item / p.nb), k = (int)(item % p.nb);
  const int s = k * p.L, e = min(p.nT, s + p.L) - 1;
  const int row = lane < DP ? lane : 0;
  TermSum<Real> acc;
  for (int t = s; t <= e; ++t) {
    const long ct = (long)c * p.nT + t;
    const Real xi = lane < p.d ? b.xs[ct * p.d + lane] : (Real)0;
    mh_step_terms<Real, DP>(p, b, ct, t, xi, mh_load<Real>(p, b, ct, t, lane), sRy, vxs, lane, row, acc);
  }
  const double sum = warp_sum<double>(acc.value());
  if (lane == 0) b.mh_part[(long)c * p.nb + k] = sum;
}

}  // namespace auxk
