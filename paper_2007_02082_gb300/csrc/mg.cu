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

// zout = zin + P0 x0 on kept slots
template <typename T>
__global__ void __launch_bounds__(512) k_mg_c_prolong(DevGrid g, MGLevelDev<T> L0, const T* __restrict__ zin,
                                                      T* __restrict__ zout, uint16_t dmask,
                                                      const uint8_t* __restrict__ on, const KState* ks) {
  KCOUNT();
  const int b0 = g.scbrick[blockIdx.x], b1 = g.scbrick[blockIdx.x + 1];
  const int inst = g.binst[b0];
  if (ks[inst].done || !on[inst]) return;
  for (int64_t s = (int64_t)b0 * DBV + threadIdx.x; s < (int64_t)b1 * DBV; s += blockDim.x) {
    const uint16_t m = g.meta[s];
    if (!(m & D_VALID)) continue;   // brick padding stays zero
    if (!keep_slot(m, dmask)) { zout[s] = T(0); continue; }
    T v = zin[s];
    for (int e = L0.pptr[s]; e < L0.pptr[s + 1]; ++e) v += L0.pw[e] * L0.xa[L0.pcol[e]];
    zout[s] = v;
  }
}

// b0 = R0 (r - A z): G0 rows gather owner slots of the composite level
template <typename T>
__global__ void k_mg_restrict0(DevGrid g, MGLevelDev<T> L0, const T* __restrict__ r, const T* __restrict__ q,
                               const uint8_t* __restrict__ on, const KState* ks) {
  KCOUNT();
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= L0.n) return;
  const int inst = L0.inst[j];
  if (ks[inst].done || !on[inst]) return;
  T v = T(0);
  for (int e = L0.rptr[j]; e < L0.rptr[j + 1]; ++e) {
    const int64_t s = L0.rcol[e];
    v += L0.rw[e] * (r[s] - q[s]);
  }
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

template <typename T>
__global__ void __launch_bounds__(SMALL_THREADS) k_mg_small(SmallArgs<T> a, const KState* ks) {
  KCOUNT();
  const int i = blockIdx.x;
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
  IBG_LAUNCH(k_mg_restrict0<T>, nblk256(mg.lev[0].n), 256, 0, st, g, mg.lev[0], r, q, mg.on, ks);
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
  SmallArgs<T> sa{mg.dlev, mg.on, mg.small, mg.coarsest, mg.cinv_off, mg.cinv, w, mg.nu_coarse};
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
  // composite: prolongation and post-smoothing, ending in z
  T* y = (nu % 2 == 0) ? z : zs;
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

template void mg_vcycle<float>(const DevGrid&, const MGDev<float>&, const float*, float*, float*, float*,
                               const float*, uint16_t, const KState*, cudaStream_t, Prof*, int);
template void mg_vcycle<double>(const DevGrid&, const MGDev<double>&, const double*, double*, double*, double*,
                                const double*, uint16_t, const KState*, cudaStream_t, Prof*, int);

}  // namespace ibg
