// Multigrid V-cycle used as the preconditioner of the pressure-increment CG
// (Eq. 12).  The linear solver is not fixed by the paper (Sec. 2.2); the
// hierarchy (mg.cpp) is the geometric one of the nested Kuhn meshes.
//
// One V-cycle, z = B r (damped Jacobi, nu sweeps down and nu up on the
// composite level and G0, nu_coarse below; exact dense solve on the coarsest
// level; restriction = transpose of prolongation), is a symmetric positive
// definite operator, as CG requires.
//
//   composite level : sweeps with the chunked Poisson stencil and the
//                     interface sums; hanging nodes re-expanded after each
//                     sweep;
//   large levels    : 7-point operator in neighbour-list form, one thread per
//                     node, one launch per step over all problems;
//   small levels    : one CTA per problem runs the rest of the cycle (every
//                     level with at most MG_SMALL_NODES nodes, and the dense
//                     coarsest solve) with block barriers between steps.
#include <algorithm>

#include "async.cuh"
#include "fe.hpp"
#include "mgdev.hpp"

namespace ibg {

IBG_KCOUNT_DEFINE
unsigned long long mg_kcount() {
  unsigned long long v = 0;
  cudaMemcpyFromSymbol(&v, g_kcount, sizeof(v));
  return v;
}

namespace {

__device__ __forceinline__ bool keep_slot(uint16_t m, uint16_t dmask) {
  return (m & D_VALID) && !(m & (D_HANG | dmask));
}

// First two Jacobi steps from zero in one pass: x1 = w D^-1 b is pointwise, so
// x2 = x1 + w D^-1 (b - A x1) takes the neighbours' x1 from their b and D^-1.
template <typename T>
__device__ __forceinline__ T level_jac2(const MGLevelDev<T>& L, T omega, int64_t j) {
  const T x1 = omega * L.dinv[j] * L.b[j];
  T ax = L.diag[j] * x1;
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    const int nb = L.nbr[6 * j + d];
    if (nb >= 0) ax += L.offd[6 * j + d] * (omega * L.dinv[nb] * L.b[nb]);
  }
  return x1 + omega * L.dinv[j] * (L.b[j] - ax);
}

template <typename T>
__device__ __forceinline__ T level_ax(const MGLevelDev<T>& L, const T* __restrict__ x, int64_t j) {
  T v = L.diag[j] * x[j];
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    const int nb = L.nbr[6 * j + d];
    if (nb >= 0) v += L.offd[6 * j + d] * x[nb];
  }
  return v;
}

// ---------------------------------------------------------------- composite level
// The pointwise composite kernels move 16-byte vectors of W = 16 / sizeof(T)
// consecutive slots; a vector without a valid slot (brick padding) is skipped,
// and padding slots inside a vector are written with their value, zero.
template <typename T> struct V16;
template <> struct V16<float> { using v = float4; using m = uint2; static constexpr int W = 4; };
template <> struct V16<double> { using v = double2; using m = uint32_t; static constexpr int W = 2; };

// z = w D^-1 r on kept slots (w = omega with multigrid, 1 for the Jacobi
// preconditioner), 0 elsewhere
template <typename T>
__global__ void __launch_bounds__(512) k_mg_c_jac0(DevGrid g, const T* __restrict__ r, T* __restrict__ z,
                                                   const T* __restrict__ dinv, uint16_t dmask,
                                                   const uint8_t* __restrict__ on, T omega, const KState* ks) {
  KCOUNT();
  using V = typename V16<T>::v;
  using MT = typename V16<T>::m;
  constexpr int W = V16<T>::W;
  const int b0 = g.scbrick[blockIdx.x], b1 = g.scbrick[blockIdx.x + 1];
  const int inst = g.binst[b0];
  if (ks[inst].done) return;
  const T w = on[inst] ? omega : T(1);
  const int64_t s1 = (int64_t)b1 * DBV;
#pragma unroll 2
  for (int64_t s = (int64_t)b0 * DBV + threadIdx.x * W; s < s1; s += (int64_t)blockDim.x * W) {
    const MT mv = *reinterpret_cast<const MT*>(g.meta + s);
    const uint16_t* mm = reinterpret_cast<const uint16_t*>(&mv);
    uint16_t mor = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) mor |= mm[j];
    if (!(mor & D_VALID)) continue;
    const V rv = *reinterpret_cast<const V*>(r + s), dv = *reinterpret_cast<const V*>(dinv + s);
    const T* re = reinterpret_cast<const T*>(&rv);
    const T* de = reinterpret_cast<const T*>(&dv);
    V zv;
    T* ze = reinterpret_cast<T*>(&zv);
#pragma unroll
    for (int j = 0; j < W; ++j) ze[j] = keep_slot(mm[j], dmask) ? T(w * de[j] * re[j]) : T(0);
    *reinterpret_cast<V*>(z + s) = zv;
  }
}

// zout = zin + omega D^-1 (r - A zin) on kept slots
template <typename T>
__global__ void __launch_bounds__(512) k_mg_c_smooth(DevGrid g, const T* __restrict__ zin, T* __restrict__ zout,
                                                     const T* __restrict__ r, const T* __restrict__ q,
                                                     const T* __restrict__ dinv, uint16_t dmask,
                                                     const uint8_t* __restrict__ on, T omega, const KState* ks) {
  KCOUNT();
  using V = typename V16<T>::v;
  using MT = typename V16<T>::m;
  constexpr int W = V16<T>::W;
  const int b0 = g.scbrick[blockIdx.x], b1 = g.scbrick[blockIdx.x + 1];
  const int inst = g.binst[b0];
  if (ks[inst].done || !on[inst]) return;
  const int64_t s1 = (int64_t)b1 * DBV;
#pragma unroll 2
  for (int64_t s = (int64_t)b0 * DBV + threadIdx.x * W; s < s1; s += (int64_t)blockDim.x * W) {
    const MT mv = *reinterpret_cast<const MT*>(g.meta + s);
    const uint16_t* mm = reinterpret_cast<const uint16_t*>(&mv);
    uint16_t mor = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) mor |= mm[j];
    if (!(mor & D_VALID)) continue;
    const V zv = *reinterpret_cast<const V*>(zin + s), rv = *reinterpret_cast<const V*>(r + s);
    const V qv = *reinterpret_cast<const V*>(q + s), dv = *reinterpret_cast<const V*>(dinv + s);
    const T* ze = reinterpret_cast<const T*>(&zv);
    const T* re = reinterpret_cast<const T*>(&rv);
    const T* qe = reinterpret_cast<const T*>(&qv);
    const T* de = reinterpret_cast<const T*>(&dv);
    V ov;
    T* oe = reinterpret_cast<T*>(&ov);
#pragma unroll
    for (int j = 0; j < W; ++j) oe[j] = keep_slot(mm[j], dmask) ? T(ze[j] + omega * de[j] * (re[j] - qe[j])) : T(0);
    *reinterpret_cast<V*>(zout + s) = ov;
  }
}

// Composite <-> G0 transfers.  The weights are those of P1 interpolation on
// the G0 Kuhn tetrahedron holding a composite node (multiples of 2^-l, exact
// in floating point), computed per node from lattice positions instead of
// read from stored CSR rows: the transfers stream the composite vectors once
// and read only the small G0 vectors and lattice map besides.

// zout = zin + P0 x0 on kept slots, in two passes.  Pass 1 gathers, for
// every brick, the G0 values of its footprint (the G0 nodes its slots
// interpolate from: 8^3 own positions at level 0, T^3 nodes at level l >= 1)
// into a flat array, one thread per entry.  Pass 2 streams the composite
// slots and reads the footprint values (cached per brick).  Vertices in the
// order of the reference CSR rows (v0 .. v3 of the tetrahedron, zero weights
// and Dirichlet G0 nodes skipped), so the sums are those of the stored form,
// bit for bit.
template <typename T>
__global__ void k_mg_fp_gather(MGLevelDev<T> L0, const uint8_t* __restrict__ on, const KState* ks) {
  KCOUNT();
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= L0.nfp) return;
  const int32_t id = L0.fnode[f];
  L0.fp[f] = id >= 0 ? L0.xa[id] : T(0);
}

// Pass 2: a CTA per chunk of up to 8 bricks; thread t takes node t of every
// brick of the chunk, so that the bricks' constants come from shared memory
// and all of a thread's loads of one pass are in flight together.  The
// set-up data is read before the wait for the previous kernel (programmatic
// dependent launch), so the first wave's reads overlap that kernel's tail.
template <typename T>
__global__ void __launch_bounds__(512, 3) k_mg_c_prolong(DevGrid g, MGLevelDev<T> L0, const T* __restrict__ zin,
                                                      T* __restrict__ zout, uint16_t dmask,
                                                      const uint8_t* __restrict__ on, const KState* ks) {
  constexpr int CH = 8;
  __shared__ int sl[CH], sq[CH][3], sc0[CH][3];
  __shared__ int64_t sfb[CH];
  // set-up data (the chunk, its instance, the metadata and the bricks'
  // lattice constants) before the wait for the previous kernel; then this
  // thread's values and the solver flags, all in flight together
  const int b0 = g.scbrick[blockIdx.x], b1 = g.scbrick[blockIdx.x + 1];
  const int inst = g.binst[b0];
  const int nb = min(b1 - b0, CH);
  const int t = threadIdx.x;
  uint16_t m[CH];
  T z[CH];
#pragma unroll
  for (int i = 0; i < CH; ++i) m[i] = i < nb ? g.meta[(int64_t)(b0 + i) * DBV + t] : uint16_t(0);
  if (t < nb) {
    const int b = b0 + t, l = g.blev[b], sc = 1 << l;
    sl[t] = l;
    sfb[t] = L0.fbase[b];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int nla = L0.lat_n[3 * inst + a];
      sq[t][a] = L0.bco[3 * b + a] * DBS;                                  // brick origin, level lattice
      sc0[t][a] = l ? min(L0.bco[3 * b + a] * DBS / sc, nla - 2) : 0;     // the footprint's first G0 node
    }
  }
  KCOUNT();
#pragma unroll
  for (int i = 0; i < CH; ++i) z[i] = i < nb ? zin[(int64_t)(b0 + i) * DBV + t] : T(0);
  const bool skip = ks[inst].done || !on[inst];
  __syncthreads();
  if (skip) return;
  const int nl[3] = {L0.lat_n[3 * inst], L0.lat_n[3 * inst + 1], L0.lat_n[3 * inst + 2]};
  const int lt[3] = {t & 7, (t >> 3) & 7, t >> 6};
  // every brick's value first, the stores after: no store stands between
  // two bricks' footprint loads, so all of them are in flight together
  T out[CH];
#pragma unroll
  for (int i = 0; i < CH; ++i) {
    out[i] = T(0);
    if (i >= nb || !keep_slot(m[i], dmask)) continue;
    const T* fp = L0.fp + sfb[i];
    const int l = sl[i];
    if (l == 0) {   // a G0 node itself: weight 1 on its own footprint entry
      out[i] = z[i] + T(1) * fp[t];
      continue;
    }
    const int sc = 1 << l, nt = (6 + sc) / sc + 1;
    int c[3], f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int p = sq[i][a] + lt[a];
      c[a] = min(p >> l, nl[a] - 2);   // the last cell holds the far lattice plane
      f[a] = p - (c[a] << l);
      c[a] -= sc0[i][a];
    }
    // axes by decreasing offset, ties in axis order: a stable three-element
    // sort (swaps on strict inequality only)
    int a0 = 0, a1 = 1, a2 = 2, f0 = f[0], f1 = f[1], f2 = f[2];
    if (f1 > f0) { int x = a0; a0 = a1; a1 = x; x = f0; f0 = f1; f1 = x; }
    if (f2 > f1) { int x = a1; a1 = a2; a2 = x; x = f1; f1 = f2; f2 = x; }
    if (f1 > f0) { int x = a0; a0 = a1; a1 = x; x = f0; f0 = f1; f1 = x; }
    const int vb[4] = {0, 1 << a0, (1 << a0) | (1 << a1), 7};
    const int wn[4] = {sc - f0, f0 - f1, f1 - f2, f2};
    const T inv = T(1) / T(sc);   // a power of two: exact
    T v = z[i];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (wn[k] == 0) continue;
      const int e = ((c[2] + ((vb[k] >> 2) & 1)) * nt + (c[1] + ((vb[k] >> 1) & 1))) * nt + (c[0] + (vb[k] & 1));
      v += (T(wn[k]) * inv) * fp[e];   // a Dirichlet G0 node's entry is zero
    }
    out[i] = v;
  }
#pragma unroll
  for (int i = 0; i < CH; ++i)   // brick padding stays zero: no store
    if (i < nb && (m[i] & D_VALID)) zout[(int64_t)(b0 + i) * DBV + t] = out[i];
}

// b0 = R0 (r - A z), R0 = P0^T over owner slots, in two passes.
// Pass 1, one CTA per composite brick of level l >= 1: the brick's residual
// values (owner copies that are neither hanging nor Dirichlet) in shared
// memory, then l restrictions by one level each down to the G0 nodes of the
// brick's footprint.  The nested Kuhn meshes make P0 the product of one-level
// interpolations, each of which takes a coarse node with weight 1 and the
// midpoint of each of the seven Kuhn edge directions (+-x, +-y, +-z, +-(1,1,0),
// +-(0,1,1), +-(1,0,1), +-(1,1,1)) with weight 1/2; its transpose gathers, for
// a coarse node at fine position 2t, the value there plus half of its 14
// Kuhn neighbours.  An array of w nodes per axis becomes one of w / 2 + 1
// (8 -> 5 -> 3 -> 2), each sum in a fixed order.
constexpr int R0_GROUP = 128;                    // threads per brick of the restriction
constexpr int R0_BRICKS = 4;                     // bricks per CTA
constexpr int R0_THREADS = R0_GROUP * R0_BRICKS;
__device__ __forceinline__ void kuhn_dir(int k, int& dx, int& dy, int& dz) {
  // k = 0..13: +-x, +-y, +-z, +-(1,1,0), +-(0,1,1), +-(1,0,1), +-(1,1,1)
  const int sg = (k & 1) ? -1 : 1, a = k >> 1;
  dx = sg * (a == 0 || a == 3 || a == 5 || a == 6);
  dy = sg * (a == 1 || a == 3 || a == 4 || a == 6);
  dz = sg * (a == 2 || a == 4 || a == 5 || a == 6);
}

// One level of the restriction for the 128 threads of a brick group (lt =
// the thread's index in the group).
template <typename T>
__device__ __forceinline__ void restrict_one_level(const T* in, int w, T* out, int wo, int lt) {
  for (int j = lt; j < wo * wo * wo; j += R0_GROUP) {
    const int tx = j % wo, ty = (j / wo) % wo, tz = j / (wo * wo);
    const int cx = 2 * tx, cy = 2 * ty, cz = 2 * tz;
    auto at = [&](int x, int y, int z) -> T {
      return (x >= 0 && x < w && y >= 0 && y < w && z >= 0 && z < w) ? in[(z * w + y) * w + x] : T(0);
    };
    T acc = at(cx, cy, cz);
    T half = T(0);
#pragma unroll
    for (int k = 0; k < 14; ++k) {
      int dx, dy, dz;
      kuhn_dir(k, dx, dy, dz);
      half += at(cx + dx, cy + dy, cz + dz);
    }
    out[j] = acc + T(0.5) * half;
  }
}

// Barrier of the 128 threads (4 warps) of brick group grp (named barrier grp + 1).
__device__ __forceinline__ void group_sync(int grp) {
  asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(R0_GROUP) : "memory");
}

// Four fine bricks per CTA of 512 threads, one group of 128 threads (four
// slots per thread) per brick with its own named barrier, so that a CTA has
// four bricks' loads in flight after two dependent rounds (the brick index,
// then its residual values, metadata, level and instance together; the
// instance's solver flags decide only whether the sums are written).
template <typename T>
__global__ void __launch_bounds__(R0_THREADS) k_mg_r0_part(DevGrid g, MGLevelDev<T> L0, const T* __restrict__ r,
                                                           const T* __restrict__ q, uint16_t dmask,
                                                           const uint8_t* __restrict__ on, const KState* ks) {
  KCOUNT();
  __shared__ T bufa[R0_BRICKS][DBV];
  __shared__ T bufb[R0_BRICKS][125];
  const int grp = threadIdx.x / R0_GROUP, lt = threadIdx.x % R0_GROUP;
  const int fi = blockIdx.x * R0_BRICKS + grp;
  if (fi >= L0.nfb) return;   // the whole group: its barrier is its own
  const int b = L0.fbr[fi];
  T v[DBV / R0_GROUP];
  uint16_t mm[DBV / R0_GROUP];
#pragma unroll
  for (int k = 0; k < DBV / R0_GROUP; ++k) {
    const int64_t s = (int64_t)b * DBV + lt + k * R0_GROUP;
    mm[k] = g.meta[s];
    v[k] = T(r[s] - q[s]);
  }
  const int inst = g.binst[b];
  int l = g.blev[b];
  const int pb = L0.pbase[b];
  if (ks[inst].done || !on[inst]) return;
#pragma unroll
  for (int k = 0; k < DBV / R0_GROUP; ++k) {
    const uint16_t m = mm[k];
    bufa[grp][lt + k * R0_GROUP] = ((m & D_VALID) && !(m & (D_HANG | D_DUP | dmask))) ? v[k] : T(0);
  }
  group_sync(grp);
  int w = DBS;
  T* in = bufa[grp];
  T* out = bufb[grp];
  while (l > 1) {   // down to level 1 inside shared memory, alternating buffers
    const int wo = w / 2 + 1;
    restrict_one_level(in, w, out, wo, lt);
    group_sync(grp);
    T* tmp = in; in = out; out = tmp;
    w = wo;
    --l;
  }
  // the last level straight into the partial sums of the brick's G0 nodes
  restrict_one_level(in, w, L0.part + pb, w / 2 + 1, lt);
}

// Pass 2, one thread per G0 node: the level-0 owner copy at its position
// (weight 1) plus the partial sums of the finer bricks around it, in brick order.
template <typename T>
__global__ void k_mg_r0_sum(MGLevelDev<T> L0, const T* __restrict__ r, const T* __restrict__ q,
                            const uint8_t* __restrict__ on, const KState* ks) {
  KCOUNT();
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= L0.n) return;
  const int inst = L0.inst[j];
  if (ks[inst].done || !on[inst]) return;
  const int32_t sl = L0.r0slot[j];
  T v = sl >= 0 ? T(r[sl] - q[sl]) : T(0);
  for (int e = L0.r0ptr[j]; e < L0.r0ptr[j + 1]; ++e) v += L0.part[L0.r0idx[e]];
  L0.b[j] = v;
}

// ---------------------------------------------------------------- large levels
// node j of level k takes part when its problem is not done and runs level k
// grid-wide (small[i] > k)
template <typename T>
__device__ __forceinline__ bool level_node_on(const MGLevelDev<T>& L, int64_t j, int k, const uint8_t* on,
                                              const int32_t* small, const KState* ks) {
  const int i = L.inst[j];
  return on[i] && small[i] > k && !ks[i].done;
}

template <typename T>
__global__ void k_mg_l_jac0(MGLevelDev<T> L, int k, T omega, const uint8_t* on, const int32_t* small,
                            const KState* ks) {
  KCOUNT();
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= L.n || !level_node_on(L, j, k, on, small, ks)) return;
  L.xa[j] = omega * L.dinv[j] * L.b[j];
}

template <typename T>
__global__ void k_mg_l_jac2(MGLevelDev<T> L, int k, T omega, const uint8_t* on, const int32_t* small,
                            const KState* ks) {
  KCOUNT();
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= L.n || !level_node_on(L, j, k, on, small, ks)) return;
  L.xb[j] = level_jac2(L, omega, j);
}

template <typename T>
__global__ void k_mg_l_sweep(MGLevelDev<T> L, int k, const T* __restrict__ xin, T* __restrict__ xout, T omega,
                             const uint8_t* on, const int32_t* small, const KState* ks) {
  KCOUNT();
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= L.n || !level_node_on(L, j, k, on, small, ks)) return;
  xout[j] = xin[j] + omega * L.dinv[j] * (L.b[j] - level_ax(L, xin, j));
}

template <typename T>
__global__ void k_mg_l_resid(MGLevelDev<T> L, int k, const T* __restrict__ x, const uint8_t* on,
                             const int32_t* small, const KState* ks) {
  KCOUNT();
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= L.n || !level_node_on(L, j, k, on, small, ks)) return;
  L.res[j] = L.b[j] - level_ax(L, x, j);
}

// b of level k+1 = R res of level k (rows of problems with small > k)
template <typename T>
__global__ void k_mg_l_restrict(MGLevelDev<T> Lc, const T* __restrict__ res, int k, const uint8_t* on,
                                const int32_t* small, const KState* ks) {
  KCOUNT();
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= Lc.n || !level_node_on(Lc, j, k, on, small, ks)) return;
  T v = T(0);
  for (int e = Lc.rptr[j]; e < Lc.rptr[j + 1]; ++e) v += Lc.rw[e] * res[Lc.rcol[e]];
  Lc.b[j] = v;
}

// xout = xin + P x(k+1) on level k
template <typename T>
__global__ void k_mg_l_prolong(MGLevelDev<T> L, MGLevelDev<T> Lc, int k, const T* __restrict__ xin,
                               T* __restrict__ xout, const uint8_t* on, const int32_t* small, const KState* ks) {
  KCOUNT();
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= L.n || !level_node_on(L, j, k, on, small, ks)) return;
  T v = xin[j];
  for (int e = Lc.pptr[j]; e < Lc.pptr[j + 1]; ++e) v += Lc.pw[e] * Lc.xa[Lc.pcol[e]];
  xout[j] = v;
}

// ---------------------------------------------------------------- small levels
template <typename T>
struct SmallArgs {
  const MGLevelDev<T>* lev;
  const uint8_t* on;
  const int32_t* small;
  const int32_t* coarsest;
  const int64_t* cinv_off;
  const T* cinv;
  T omega;
  int nu;
};

constexpr int SMALL_THREADS = 1024;

// The small levels and the coarsest solve of problem i, by the whole CTA
// (block barriers between steps); each node's value is computed by one
// thread, in an order that does not depend on the CTA's size.
template <typename T>
__device__ void small_cycle(const SmallArgs<T>& a, int i, const KState* ks) {
  if (!a.on[i] || ks[i].done) return;
  const int k0 = a.small[i], K = a.coarsest[i];
  const int t = threadIdx.x, nt = blockDim.x;
  // down: pre-smoothing, residual, restriction
  for (int k = k0; k < K; ++k) {
    const MGLevelDev<T>& L = a.lev[k];
    const int j0 = L.noff[i], j1 = L.noff[i + 1];
    T* cur = L.xa;
    T* oth = L.xb;
    int s0 = 1;
    if (a.nu >= 2) {   // the first two steps in one pass, result in xb
      for (int j = j0 + t; j < j1; j += nt) L.xb[j] = level_jac2(L, a.omega, j);
      cur = L.xb;
      oth = L.xa;
      s0 = 2;
    } else {
      for (int j = j0 + t; j < j1; j += nt) L.xa[j] = a.omega * L.dinv[j] * L.b[j];
    }
    __syncthreads();
    for (int s = s0; s < a.nu; ++s) {
      for (int j = j0 + t; j < j1; j += nt) oth[j] = cur[j] + a.omega * L.dinv[j] * (L.b[j] - level_ax(L, cur, j));
      __syncthreads();
      T* tmp = cur; cur = oth; oth = tmp;
    }
    for (int j = j0 + t; j < j1; j += nt) L.res[j] = L.b[j] - level_ax(L, cur, j);
    __syncthreads();
    const MGLevelDev<T>& C = a.lev[k + 1];
    for (int j = C.noff[i] + t; j < C.noff[i + 1]; j += nt) {
      T v = T(0);
      for (int e = C.rptr[j]; e < C.rptr[j + 1]; ++e) v += C.rw[e] * L.res[C.rcol[e]];
      C.b[j] = v;
    }
    __syncthreads();
  }
  // coarsest: x = A^-1 b with the (symmetrised) dense inverse, read by columns
  {
    const MGLevelDev<T>& L = a.lev[K];
    const int j0 = L.noff[i], n = L.noff[i + 1] - j0;
    const T* Ai = a.cinv + a.cinv_off[i];
    for (int r = t; r < n; r += nt) {
      T v = T(0);
      for (int c = 0; c < n; ++c) v += Ai[(int64_t)c * n + r] * L.b[j0 + c];
      L.xa[j0 + r] = v;
    }
    __syncthreads();
  }
  // up: prolongation, post-smoothing; each level's result ends in xa
  for (int k = K - 1; k >= k0; --k) {
    const MGLevelDev<T>& L = a.lev[k];
    const MGLevelDev<T>& C = a.lev[k + 1];
    const int j0 = L.noff[i], j1 = L.noff[i + 1];
    T* cur = (a.nu % 2 == 1) ? L.xa : L.xb;          // pre-smoothed iterate
    T* y = (a.nu % 2 == 0) ? L.xa : L.xb;
    for (int j = j0 + t; j < j1; j += nt) {
      T v = cur[j];
      for (int e = C.pptr[j]; e < C.pptr[j + 1]; ++e) v += C.pw[e] * C.xa[C.pcol[e]];
      y[j] = v;
    }
    __syncthreads();
    T* o = (y == L.xa) ? L.xb : L.xa;
    for (int s = 0; s < a.nu; ++s) {
      for (int j = j0 + t; j < j1; j += nt) o[j] = y[j] + a.omega * L.dinv[j] * (L.b[j] - level_ax(L, y, j));
      __syncthreads();
      T* tmp = y; y = o; o = tmp;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(SMALL_THREADS) k_mg_small(SmallArgs<T> a, const KState* ks) {
  KCOUNT();
  small_cycle(a, blockIdx.x, ks);
}

// ---------------------------------------------------------------- persistent coarse levels
// Launch choice IB_TUNE_MG_PERSIST = 2: the part of the V-cycle below the
// composite grid in one cooperative launch instead of about 25 small ones:
// the grid-wide levels down (pre-smoothing, residual, restriction), every
// problem's small levels and coarsest solve (CTA i takes problem i, as
// k_mg_small does), and the grid-wide levels up (prolongation,
// post-smoothing), with a grid barrier wherever the separate launches had a
// kernel boundary.  Every node's arithmetic is that of the separate kernels in
// the same order, so the result is bitwise the same.  All CTAs are resident
// (cooperative launch); each barrier wait is bounded in wall-clock time, and
// on expiry the CTA records ASYNC_TIMEOUT for every problem and returns.
constexpr int LV_THREADS = 512;

template <typename T>
struct LevelsArgs {
  SmallArgs<T> sa;       // levels (device copy), flags, coarsest inverses, omega, nu_coarse
  int nu;                // sweeps on G0 (level 0 of the list)
  int max_big;           // levels run grid-wide
  int ninst;
  unsigned* bar;         // [2]: arrivals, generation (zero at the start of a step)
  int32_t* aerr;         // [ninst] error words of the step
};

// Barrier over all CTAs of a cooperative launch: arrivals on bar[0], release
// by the generation word bar[1]; the last CTA to arrive resets the count and
// advances the generation.  Returns false (after recording the timeout) when
// the wait ran out.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int ninst, int32_t* aerr) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* gen = bar + 1;
    const unsigned g0 = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*gen == g0) {
        if (global_ns() - t0 > ASYNC_WAIT_NS) {
          for (int i = 0; i < ninst; ++i) atomicMax(aerr + i, ASYNC_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <typename T>
__global__ void __launch_bounds__(LV_THREADS) k_mg_levels(LevelsArgs<T> a, const KState* ks) {
  KCOUNT();
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x, nth = int64_t(gridDim.x) * blockDim.x;
  const SmallArgs<T>& S = a.sa;
  const T w = S.omega;
  // levels down: pre-smoothing, residual, restriction
  for (int k = 0; k < a.max_big; ++k) {
    const MGLevelDev<T>& L = S.lev[k];
    const int nuk = k == 0 ? a.nu : S.nu;
    T* x = L.xa;
    T* y = L.xb;
    int s0 = 1;
    if (nuk >= 2) {   // the first two steps in one pass, result in xb
      for (int64_t j = tid; j < L.n; j += nth)
        if (level_node_on(L, j, k, S.on, S.small, ks)) L.xb[j] = level_jac2(L, w, j);
      x = L.xb;
      y = L.xa;
      s0 = 2;
    } else {
      for (int64_t j = tid; j < L.n; j += nth)
        if (level_node_on(L, j, k, S.on, S.small, ks)) L.xa[j] = w * L.dinv[j] * L.b[j];
    }
    if (!grid_barrier(a.bar, a.ninst, a.aerr)) return;
    for (int s = s0; s < nuk; ++s) {
      for (int64_t j = tid; j < L.n; j += nth)
        if (level_node_on(L, j, k, S.on, S.small, ks)) y[j] = x[j] + w * L.dinv[j] * (L.b[j] - level_ax(L, x, j));
      if (!grid_barrier(a.bar, a.ninst, a.aerr)) return;
      T* tmp = x; x = y; y = tmp;
    }
    for (int64_t j = tid; j < L.n; j += nth)
      if (level_node_on(L, j, k, S.on, S.small, ks)) L.res[j] = L.b[j] - level_ax(L, x, j);
    if (!grid_barrier(a.bar, a.ninst, a.aerr)) return;
    const MGLevelDev<T>& C = S.lev[k + 1];
    for (int64_t j = tid; j < C.n; j += nth) {
      if (!level_node_on(C, j, k, S.on, S.small, ks)) continue;
      T v = T(0);
      for (int e = C.rptr[j]; e < C.rptr[j + 1]; ++e) v += C.rw[e] * L.res[C.rcol[e]];
      C.b[j] = v;
    }
    if (!grid_barrier(a.bar, a.ninst, a.aerr)) return;
  }
  // small levels and the coarsest solve, a CTA per problem
  for (int i = blockIdx.x; i < a.ninst; i += gridDim.x) small_cycle(S, i, ks);
  if (!grid_barrier(a.bar, a.ninst, a.aerr)) return;
  // levels up: prolongation, post-smoothing; each level's result ends in xa
  for (int k = a.max_big - 1; k >= 0; --k) {
    const MGLevelDev<T>& L = S.lev[k];
    const MGLevelDev<T>& C = S.lev[k + 1];
    const int nuk = k == 0 ? a.nu : S.nu;
    T* c = (nuk % 2 == 1) ? L.xa : L.xb;
    T* y = (nuk % 2 == 0) ? L.xa : L.xb;
    for (int64_t j = tid; j < L.n; j += nth) {
      if (!level_node_on(L, j, k, S.on, S.small, ks)) continue;
      T v = c[j];
      for (int e = C.pptr[j]; e < C.pptr[j + 1]; ++e) v += C.pw[e] * C.xa[C.pcol[e]];
      y[j] = v;
    }
    if (!grid_barrier(a.bar, a.ninst, a.aerr)) return;
    T* o = (y == L.xa) ? L.xb : L.xa;
    for (int s = 0; s < nuk; ++s) {
      for (int64_t j = tid; j < L.n; j += nth)
        if (level_node_on(L, j, k, S.on, S.small, ks)) o[j] = y[j] + w * L.dinv[j] * (L.b[j] - level_ax(L, y, j));
      if (k > 0 || s + 1 < nuk)
        if (!grid_barrier(a.bar, a.ninst, a.aerr)) return;
      T* tmp = y; y = o; o = tmp;
    }
  }
}

inline unsigned nblk256(int64_t n) { return unsigned((n + 255) / 256); }

}  // namespace

template <typename T>
void mg_vcycle(const DevGrid& g, const MGDev<T>& mg, const T* r, T* z, T* zs, T* q, const T* dinv, uint16_t dmask,
               const KState* ks, cudaStream_t st, Prof* prof, int pcls) {
  const int nu = mg.nu;
  const T w = mg.omega;
  KState* ksm = const_cast<KState*>(ks);
  Prof* pr = prof && prof->on ? prof : nullptr;
  auto timed = [&](int c, auto&& f) {
    if (pr) pr->begin(pcls + c, st);
    f();
    if (pr) pr->end(st);
  };
  // q = A x, then its interface sums into both stored copies
  auto apply = [&](const T* x) {
    timed(0, [&] { fe_poisson_apply<T>(g, x, q, dmask, ksm, mg.on, st); });
    fe_sync<T>(g, 1, q, dmask, st);
  };
  auto smooth = [&](const T* zin, T* zout) {
    timed(1, [&] {
      IBG_LAUNCH(k_mg_c_smooth<T>, g.nschunks, DBV, 0, st, g, zin, zout, r, q, dinv, dmask, mg.on, w, ks);
    });
  };
  // composite pre-smoothing
  timed(2, [&] { IBG_LAUNCH(k_mg_c_jac0<T>, g.nschunks, DBV, 0, st, g, r, z, dinv, dmask, mg.on, w, ks); });
  fe_expand2<T>(g, 1, z, (T*)nullptr, st);
  if (!mg.any) return;
  T* cur = z;
  T* oth = zs;
  for (int s = 1; s < nu; ++s) {
    apply(cur);
    smooth(cur, oth);
    fe_expand2<T>(g, 1, oth, (T*)nullptr, st);
    T* tmp = cur; cur = oth; oth = tmp;
  }
  apply(cur);
  if (pr) pr->begin(pcls + 2, st);
  if (mg.lev[0].nfb > 0)
    IBG_LAUNCH(k_mg_r0_part<T>, (mg.lev[0].nfb + R0_BRICKS - 1) / R0_BRICKS, R0_THREADS, 0, st, g, mg.lev[0], r,
               (const T*)q, dmask, mg.on, ks);
  IBG_LAUNCH(k_mg_r0_sum<T>, nblk256(mg.lev[0].n), 256, 0, st, mg.lev[0], r, (const T*)q, mg.on, ks);
  SmallArgs<T> sa{mg.dlev, mg.on, mg.small, mg.coarsest, mg.cinv_off, mg.cinv, w, mg.nu_coarse};
  if (mg.lv_ctas > 0 && mg.bar) {
    // levels down, small levels, levels up: one cooperative launch
    LevelsArgs<T> la{sa, nu, mg.max_big, mg.ninst, mg.bar, g.aerr};
    launch_cooperative(k_mg_levels<T>, mg.lv_ctas, LV_THREADS, 0, st, la, ks);
  } else {
  // large levels, down
  for (int k = 0; k < mg.max_big; ++k) {
    const MGLevelDev<T>& L = mg.lev[k];
    const unsigned nb = nblk256(L.n);
    const int nuk = k == 0 ? nu : mg.nu_coarse;
    T* a = L.xa;
    T* b = L.xb;
    int s0 = 1;
    if (nuk >= 2) {   // the first two steps in one pass, result in xb
      IBG_LAUNCH(k_mg_l_jac2<T>, nb, 256, 0, st, L, k, w, mg.on, mg.small, ks);
      a = L.xb;
      b = L.xa;
      s0 = 2;
    } else {
      IBG_LAUNCH(k_mg_l_jac0<T>, nb, 256, 0, st, L, k, w, mg.on, mg.small, ks);
    }
    for (int s = s0; s < nuk; ++s) {
      IBG_LAUNCH(k_mg_l_sweep<T>, nb, 256, 0, st, L, k, (const T*)a, b, w, mg.on, mg.small, ks);
      T* tmp = a; a = b; b = tmp;
    }
    IBG_LAUNCH(k_mg_l_resid<T>, nb, 256, 0, st, L, k, (const T*)a, mg.on, mg.small, ks);
    IBG_LAUNCH(k_mg_l_restrict<T>, nblk256(mg.lev[k + 1].n), 256, 0, st, mg.lev[k + 1], (const T*)L.res, k, mg.on,
               mg.small, ks);
  }
  // small levels and the coarsest solve, one CTA per problem
  IBG_LAUNCH(k_mg_small<T>, mg.ninst, SMALL_THREADS, 0, st, sa, ks);
  // large levels, up
  for (int k = mg.max_big - 1; k >= 0; --k) {
    const MGLevelDev<T>& L = mg.lev[k];
    const unsigned nb = nblk256(L.n);
    const int nuk = k == 0 ? nu : mg.nu_coarse;
    T* c = (nuk % 2 == 1) ? L.xa : L.xb;
    T* y = (nuk % 2 == 0) ? L.xa : L.xb;
    IBG_LAUNCH(k_mg_l_prolong<T>, nb, 256, 0, st, L, mg.lev[k + 1], k, (const T*)c, y, mg.on, mg.small, ks);
    T* o = (y == L.xa) ? L.xb : L.xa;
    for (int s = 0; s < nuk; ++s) {
      IBG_LAUNCH(k_mg_l_sweep<T>, nb, 256, 0, st, L, k, (const T*)y, o, w, mg.on, mg.small, ks);
      T* tmp = y; y = o; o = tmp;
    }
  }
  }
  // composite: prolongation and post-smoothing, ending in z
  T* y = (nu % 2 == 0) ? z : zs;
  if (mg.lev[0].nfp > 0)
    IBG_LAUNCH(k_mg_fp_gather<T>, nblk256(mg.lev[0].nfp), 256, 0, st, mg.lev[0], mg.on, ks);
  IBG_LAUNCH(k_mg_c_prolong<T>, g.nschunks, DBV, 0, st, g, mg.lev[0], (const T*)cur, y, dmask, mg.on, ks);
  if (pr) pr->end(st);
  fe_expand2<T>(g, 1, y, (T*)nullptr, st);
  T* o = (y == z) ? zs : z;
  for (int s = 0; s < nu; ++s) {
    apply(y);
    smooth(y, o);
    fe_expand2<T>(g, 1, o, (T*)nullptr, st);
    T* tmp = y; y = o; o = tmp;
  }
}

template <typename T>
int mg_levels_ctas() {
  int dev = 0, nsm = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mg_levels<T>, LV_THREADS, 0) != cudaSuccess)
    return 0;
  return nsm * std::min(per, 2);
}
template int mg_levels_ctas<float>();
template int mg_levels_ctas<double>();

template void mg_vcycle<float>(const DevGrid&, const MGDev<float>&, const float*, float*, float*, float*,
                               const float*, uint16_t, const KState*, cudaStream_t, Prof*, int);
template void mg_vcycle<double>(const DevGrid&, const MGDev<double>&, const double*, double*, double*, double*,
                                const double*, uint16_t, const KState*, cudaStream_t, Prof*, int);

}  // namespace ibg
