// Krylov solvers of the IPCS step.  The linear solvers are not stated in the
// paper (Sec. 2.2); these are the build's choice: Jacobi-preconditioned CG for
// the symmetric Poisson (Eq. 12) and mass systems, right-preconditioned
// BiCGStab for the nonsymmetric Oseen system (Eq. 9).
//
// CG iteration (3 or 4 kernels):
//   k_apply (fe.cu): p_new = z + beta p_old on the brick tile, q = A p_new
//                    (local per level), fused p.q -> alpha;
//   k_sync (fe.cu):  interface sum of q into both stored copies (refined
//                    grids only; one thread per interface node);
//   k_cg_update:     x += alpha p, r -= alpha q, z = D^-1 r, FP64 r.z and r.r
//                    -> beta, convergence, loop condition;
//   k_expand:        hanging z = mean of parents (refined grids only).
// Summing the interface copies in their own small kernel keeps the streaming
// updates free of the chain of dependent index loads an interface sum needs
// (measured: the in-line sums stalled 43 % of the warps of the refined
// 64x64x256 tube for most of each update).
// The search direction ping-pongs between two buffers, so a loop body holds two
// iterations.  All inner products accumulate in FP64 in a fixed order.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ff.cuh"
#include "krylov.hpp"

namespace ibg {

IBG_KCOUNT_DEFINE
unsigned long long krylov_kcount() {
  unsigned long long v = 0;
  cudaMemcpyFromSymbol(&v, g_kcount, sizeof(v));
  return v;
}

// Component c of a slot is an unknown (dof: owner copies only; keep: every
// stored copy) unless it is hanging, Dirichlet by the solve's mask, or, in a
// velocity solve, a tangential component held by the port condition.
__device__ __forceinline__ bool kdof(uint16_t m, uint16_t dmask, int c = 0) {
  return (m & D_VALID) && !(m & (D_HANG | D_DUP | dmask)) && !tan_dir(m, dmask, c);
}
__device__ __forceinline__ bool kkeep(uint16_t m, uint16_t dmask, int c = 0) {
  return (m & D_VALID) && !(m & (D_HANG | dmask)) && !tan_dir(m, dmask, c);
}

// block-wide OR of a per-thread flag, result valid in every thread
__device__ __forceinline__ bool block_any(bool v) { return __syncthreads_or(v ? 1 : 0) != 0; }

__global__ void k_init_states(KState* ks, int nc, double tol2, int max_iter) {
  KCOUNT();
  const int c = threadIdx.x + blockIdx.x * blockDim.x;
  if (c >= nc) return;
  KState k;
  memset(&k, 0, sizeof(k));
  k.tol2 = tol2;
  k.max_iter = max_iter;
  ks[c] = k;
}

// record a finished solve of every instance (rec[i * 4], os[i]); with os set
// (inner solve of a defect-correction loop) iterations accumulate and a
// breakdown is passed to the outer loop, which decides (the field solves
// stop; the force solve goes on while its passes still make progress) and
// records the status
__global__ void k_collect(const KState* ks, int nc, int ninst, SolveRec* rec, OState* os) {
  KCOUNT();
  const int i = threadIdx.x + blockIdx.x * blockDim.x;
  if (i >= ninst) return;
  SolveRec& R = rec[i * 4];
  double rel = 0.0;
  int st = R.status;
  for (int c = 0; c < nc; ++c) {
    const KState& k = ks[i * nc + c];
    R.iters[c] += k.iter;
    st = max(st, k.status);
    if (k.bb > 0) rel = fmax(rel, sqrt(fmax(k.rr, 0.0) / k.bb));
  }
  if (os) {
    if (st == 5) os[i].inner_status = 5;
  } else {
    R.status = st;
    R.relres = rel;
    R.outer = 1;
  }
}

__global__ void k_init_outer(OState* os, int ninst, int nc, double tol2, int max_outer) {
  KCOUNT();
  const int i = threadIdx.x + blockIdx.x * blockDim.x;
  if (i >= ninst) return;
  OState o;
  memset(&o, 0, sizeof(o));
  o.tol2 = tol2;
  o.max_iter = max_outer;
  o.nc = nc;
  os[i] = o;
}

__global__ void k_collect_outer(const OState* os, int ninst, SolveRec* rec) {
  KCOUNT();
  const int i = threadIdx.x + blockIdx.x * blockDim.x;
  if (i >= ninst) return;
  SolveRec& R = rec[i * 4];
  R.outer = os[i].iter;
  R.relres = sqrt(fmax(os[i].rel2, 0.0));
  R.status = max(R.status, os[i].status);
}

// Coupled components (one system in NC unknowns per node, the momentum
// operator of the symmetric viscous form): each component's partial sums
// become the sums over the components, so the NC states take the same
// scalars and converge together, which is BiCGStab on the whole vector.
template <int NC, int NQ>
__device__ __forceinline__ void couple_sums(double* o) {
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double t = 0.0;
#pragma unroll
    for (int c = 0; c < NC; ++c) t += o[NQ * c + q];
#pragma unroll
    for (int c = 0; c < NC; ++c) o[NQ * c + q] = t;
  }
}

// ---------------------------------------------------------------- CG
template <typename T, int NC>
__global__ void __launch_bounds__(512) k_cg_start(DevGrid g, const T* __restrict__ b, const T* __restrict__ y,
                                                  T* __restrict__ r, T* __restrict__ z, T* __restrict__ p,
                                                  const T* __restrict__ dinv, uint16_t dmask, KState* ks,
                                                  double* partials, unsigned* counter, Cond cond,
                                                  const OState* skip_os) {
  KCOUNT();
  const int64_t s = (int64_t)blockIdx.x * DBV + threadIdx.x;
  const uint16_t m = g.meta[s];
  T tv[3 * NC];
  for (int c = 0; c < NC; ++c) {
    const bool dof = kdof(m, dmask, c), keep = kkeep(m, dmask, c);
    const int64_t i = c * g.nslots + s;
    T rv = keep ? (y ? T(b[i] - y[i]) : b[i]) : T(0);
    T zv = rv * dinv[s];
    r[i] = rv;
    z[i] = zv;
    p[i] = zv;
    tv[3 * c] = dof ? rv * zv : T(0);
    tv[3 * c + 1] = dof ? rv * rv : T(0);
    tv[3 * c + 2] = dof ? b[i] * b[i] : T(0);
  }
  double* out = partials + (int64_t)gridDim.x * 3 * NC;
  if (!grid_sum_last<T, 3 * NC>(tv, partials, counter, g.bseg, g.ninst, out)) return;
  bool any = false;
  for (int i = threadIdx.x; i < g.ninst; i += blockDim.x) {
    const bool skip = skip_os && skip_os[i].done;
    for (int c = 0; c < NC; ++c) {
      KState& k = ks[i * NC + c];
      const double* t = out + (int64_t)i * 3 * NC + 3 * c;
      k.rz = t[0];
      k.rr = t[1];
      // reference norm max(||b||, ||r0||): covers a zero right-hand side with a
      // nonzero Dirichlet lifting as well as warm starts
      k.bb = fmax(t[2], k.rr);
      k.iter = 0;
      k.status = 0;
      k.alpha = 0.0;
      k.beta = 0.0;
      k.af = k.bf = 0.f;
      k.done = (skip || k.rr <= k.tol2 * k.bb) ? 1 : 0;
      if (!skip && !isfinite(k.rr)) { k.done = 1; k.status = 5; }
      any = any || !k.done;
    }
  }
  any = block_any(any);
  if (threadIdx.x == 0) set_cond(cond, any);
}

// Streaming form of k_cg_update: each thread handles W = 16 / sizeof(T)
// consecutive slots with 16-byte loads and stores (q interface-summed).
template <int W>
__device__ __forceinline__ uint16_t vec_or_n(const uint16_t* mm) {
  uint16_t o = 0;
#pragma unroll
  for (int j = 0; j < W; ++j) o |= mm[j];
  return o;
}

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; using mt = uint2; static constexpr int W = 4; };
template <> struct Vec16<double> { using type = double2; using mt = uint32_t; static constexpr int W = 2; };

template <typename T, int NC>
__global__ void __launch_bounds__(512) k_cg_update_vec(DevGrid g, T* __restrict__ x, T* __restrict__ r,
                                                       T* __restrict__ z, const T* __restrict__ p,
                                                       const T* __restrict__ q, const T* __restrict__ dinv,
                                                       uint16_t dmask, KState* ks, double* partials,
                                                       unsigned* counter, Cond cond) {
  KCOUNT();
  using V = typename Vec16<T>::type;
  using MT = typename Vec16<T>::mt;
  constexpr int W = Vec16<T>::W;
  const int b0 = g.scbrick[blockIdx.x], b1 = g.scbrick[blockIdx.x + 1];
  const KState* ki = ks + g.binst[b0] * NC;
  bool act[NC];
  T alc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    act[c] = !ki[c].done;
    alc[c] = k_alpha<T>(ki[c]);
  }
  T tv[2 * NC];
#pragma unroll
  for (int c = 0; c < 2 * NC; ++c) tv[c] = T(0);
  const int64_t s1 = (int64_t)b1 * DBV;
#pragma unroll 2
  for (int64_t s = (int64_t)b0 * DBV + threadIdx.x * W; s < s1; s += (int64_t)blockDim.x * W) {
    const MT mv = *reinterpret_cast<const MT*>(g.meta + s);
    const uint16_t* mm = reinterpret_cast<const uint16_t*>(&mv);
    if (!(vec_or_n<W>(mm) & D_VALID)) continue;   // brick padding: always zero, never read or written
    const V dv = *reinterpret_cast<const V*>(dinv + s);
    const T* de = reinterpret_cast<const T*>(&dv);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (!act[c]) continue;
      const T a = alc[c];
      const int64_t i = (int64_t)c * g.nslots + s;
      const T* qc = q + (int64_t)c * g.nslots;
      V xv = *reinterpret_cast<const V*>(x + i);
      V rv = *reinterpret_cast<const V*>(r + i);
      const V pv = *reinterpret_cast<const V*>(p + i);
      const V qv = *reinterpret_cast<const V*>(q + i);
      T* xe = reinterpret_cast<T*>(&xv);
      T* re = reinterpret_cast<T*>(&rv);
      const T* pe = reinterpret_cast<const T*>(&pv);
      const T* qe = reinterpret_cast<const T*>(&qv);
      V zv;
      T* ze = reinterpret_cast<T*>(&zv);
#pragma unroll
      for (int j = 0; j < W; ++j) {
        const uint16_t m = mm[j];
        const T qq = qe[j];
        if (m & D_VALID) xe[j] += a * pe[j];
        const T rn = kkeep(m, dmask, c) ? T(re[j] - a * qq) : T(0);
        re[j] = rn;
        ze[j] = rn * de[j];
        if (kdof(m, dmask, c)) {
          tv[2 * c] += rn * ze[j];
          tv[2 * c + 1] += rn * rn;
        }
      }
      *reinterpret_cast<V*>(x + i) = xv;
      *reinterpret_cast<V*>(r + i) = rv;
      *reinterpret_cast<V*>(z + i) = zv;
    }
  }
  double* out = partials + (int64_t)gridDim.x * 2 * NC;
  if (!grid_sum_last<T, 2 * NC>(tv, partials, counter, g.scseg, g.ninst, out)) return;
  bool any = false;
  for (int i = threadIdx.x; i < g.ninst; i += blockDim.x)
    for (int c = 0; c < NC; ++c) {
      KState& kk = ks[i * NC + c];
      if (kk.done) continue;
      kk.iter++;
      kk.rr = out[(int64_t)i * 2 * NC + 2 * c + 1];
      const double rzn = out[(int64_t)i * 2 * NC + 2 * c];
      if (!isfinite(kk.rr) || !isfinite(rzn)) { kk.done = 1; kk.status = 5; continue; }
      if (kk.rr <= kk.tol2 * kk.bb) { kk.done = 1; continue; }
      if (kk.iter >= kk.max_iter) { kk.done = 1; kk.status = 4; continue; }
      kk.beta = rzn / kk.rz;
      kk.bf = float(kk.beta);
      kk.rz = rzn;
      any = true;
    }
  any = block_any(any);
  if (threadIdx.x == 0) set_cond(cond, any);
}

// ---------------------------------------------------------------- CG with a multigrid preconditioner
// The preconditioner is applied between the update and the next direction, so
// r.z and beta move into k_cg_rz after the V-cycle.

// r = b - A x on kept slots; ||r||^2, ||b||^2 -> rr, bb, done
template <typename T>
__global__ void __launch_bounds__(512) k_cg_start_r(DevGrid g, const T* __restrict__ b, const T* __restrict__ y,
                                                    T* __restrict__ r, uint16_t dmask, KState* ks,
                                                    double* partials, unsigned* counter, const OState* skip_os) {
  KCOUNT();
  const int64_t s = (int64_t)blockIdx.x * DBV + threadIdx.x;
  const uint16_t m = g.meta[s];
  const bool dof = kdof(m, dmask), keep = kkeep(m, dmask);
  const T rv = keep ? (y ? T(b[s] - y[s]) : b[s]) : T(0);
  r[s] = rv;
  T tv[2] = {dof ? rv * rv : T(0), dof ? b[s] * b[s] : T(0)};
  double* out = partials + (int64_t)gridDim.x * 2;
  if (!grid_sum_last<T, 2>(tv, partials, counter, g.bseg, g.ninst, out)) return;
  for (int i = threadIdx.x; i < g.ninst; i += blockDim.x) {
    const bool skip = skip_os && skip_os[i].done;
    KState& k = ks[i];
    k.rr = out[(int64_t)i * 2];
    k.bb = fmax(out[(int64_t)i * 2 + 1], k.rr);
    k.rz = 0.0;
    k.iter = 0;
    k.status = 0;
    k.alpha = 0.0;
    k.beta = 0.0;
    k.af = k.bf = 0.f;
    k.done = (skip || k.rr <= k.tol2 * k.bb) ? 1 : 0;
    if (!skip && !isfinite(k.rr)) { k.done = 1; k.status = 5; }
  }
}

// k_cg_update_vec without the preconditioner: x += alpha p, r -= alpha q
// (q interface-summed), ||r||^2 -> convergence and iteration cap
template <typename T>
__global__ void __launch_bounds__(512) k_cg_update_r(DevGrid g, T* __restrict__ x, T* __restrict__ r,
                                                     const T* __restrict__ p, const T* __restrict__ q,
                                                     uint16_t dmask, KState* ks, double* partials,
                                                     unsigned* counter) {
  KCOUNT();
  using V = typename Vec16<T>::type;
  using MT = typename Vec16<T>::mt;
  constexpr int W = Vec16<T>::W;
  const int b0 = g.scbrick[blockIdx.x], b1 = g.scbrick[blockIdx.x + 1];
  const KState& k = ks[g.binst[b0]];
  T tv[1] = {T(0)};
  if (!k.done) {
    const T a = k_alpha<T>(k);
    const int64_t s1 = (int64_t)b1 * DBV;
  #pragma unroll 2
  for (int64_t s = (int64_t)b0 * DBV + threadIdx.x * W; s < s1; s += (int64_t)blockDim.x * W) {
      const MT mv = *reinterpret_cast<const MT*>(g.meta + s);
      const uint16_t* mm = reinterpret_cast<const uint16_t*>(&mv);
      if (!(vec_or_n<W>(mm) & D_VALID)) continue;   // brick padding: always zero, never read or written
      V xv = *reinterpret_cast<const V*>(x + s);
      V rv = *reinterpret_cast<const V*>(r + s);
      V pv = *reinterpret_cast<const V*>(p + s);
      V qv = *reinterpret_cast<const V*>(q + s);
      T* xe = reinterpret_cast<T*>(&xv);
      T* re = reinterpret_cast<T*>(&rv);
      T* pe = reinterpret_cast<T*>(&pv);
      T* qe = reinterpret_cast<T*>(&qv);
#pragma unroll
      for (int j = 0; j < W; ++j) {
        const uint16_t m = mm[j];
        const T qq = qe[j];
        if (m & D_VALID) xe[j] += a * pe[j];
        const T rn = kkeep(m, dmask) ? T(re[j] - a * qq) : T(0);
        re[j] = rn;
        if (kdof(m, dmask)) tv[0] += rn * rn;
      }
      *reinterpret_cast<V*>(x + s) = xv;
      *reinterpret_cast<V*>(r + s) = rv;
    }
  }
  double* out = partials + (int64_t)gridDim.x;
  if (!grid_sum_last<T, 1>(tv, partials, counter, g.scseg, g.ninst, out)) return;
  for (int i = threadIdx.x; i < g.ninst; i += blockDim.x) {
    KState& kk = ks[i];
    if (kk.done) continue;
    kk.iter++;
    kk.rr = out[i];
    if (!isfinite(kk.rr)) { kk.done = 1; kk.status = 5; continue; }
    if (kk.rr <= kk.tol2 * kk.bb) { kk.done = 1; continue; }
    if (kk.iter >= kk.max_iter) { kk.done = 1; kk.status = 4; continue; }
  }
}

// r.z over DOF slots -> beta (0 on the first pass), rz; loop condition
template <typename T>
__global__ void __launch_bounds__(512) k_cg_rz(DevGrid g, const T* __restrict__ r, const T* __restrict__ z,
                                               uint16_t dmask, KState* ks, double* partials, unsigned* counter,
                                               Cond cond, int first) {
  KCOUNT();
  const int b0 = g.scbrick[blockIdx.x], b1 = g.scbrick[blockIdx.x + 1];
  const KState& k = ks[g.binst[b0]];
  T tv[1] = {T(0)};
  if (!k.done)
    for (int64_t s = (int64_t)b0 * DBV + threadIdx.x; s < (int64_t)b1 * DBV; s += blockDim.x)
      if (kdof(g.meta[s], dmask)) tv[0] += r[s] * z[s];
  double* out = partials + (int64_t)gridDim.x;
  if (!grid_sum_last<T, 1>(tv, partials, counter, g.scseg, g.ninst, out)) return;
  bool any = false;
  for (int i = threadIdx.x; i < g.ninst; i += blockDim.x) {
    KState& kk = ks[i];
    if (kk.done) continue;
    const double rzn = out[i];
    if (!isfinite(rzn) || !(rzn > 0.0)) { kk.done = 1; kk.status = 5; continue; }
    kk.beta = first ? 0.0 : rzn / kk.rz;
    kk.bf = float(kk.beta);
    kk.rz = rzn;
    any = true;
  }
  any = block_any(any);
  if (threadIdx.x == 0) set_cond(cond, any);
}

// ---------------------------------------------------------------- BiCGStab
template <typename T, int NC>
__global__ void __launch_bounds__(512) k_bcg_start(DevGrid g, const T* __restrict__ b, const T* __restrict__ y,
                                                   T* __restrict__ r, T* __restrict__ rh, T* __restrict__ p,
                                                   T* __restrict__ v, uint16_t dmask, KState* ks,
                                                   double* partials, unsigned* counter, Cond cond,
                                                   const OState* skip_os, int coupled) {
  KCOUNT();
  const int64_t s = (int64_t)blockIdx.x * DBV + threadIdx.x;
  const uint16_t m = g.meta[s];
  T tw[2 * NC];
  for (int c = 0; c < NC; ++c) {
    const bool dof = kdof(m, dmask, c), keep = kkeep(m, dmask, c);
    const int64_t i = c * g.nslots + s;
    T rv = keep ? (y ? T(b[i] - y[i]) : b[i]) : T(0);
    r[i] = rv;
    rh[i] = rv;
    p[i] = T(0);
    v[i] = T(0);
    tw[2 * c] = dof ? rv * rv : T(0);
    tw[2 * c + 1] = dof ? b[i] * b[i] : T(0);
  }
  double* out = partials + (int64_t)gridDim.x * 2 * NC;
  if (!grid_sum_last<T, 2 * NC>(tw, partials, counter, g.bseg, g.ninst, out)) return;
  bool any = false;
  for (int i = threadIdx.x; i < g.ninst; i += blockDim.x) {
    const bool skip = skip_os && skip_os[i].done;
    if (coupled) couple_sums<NC, 2>(out + (int64_t)i * 2 * NC);
    for (int c = 0; c < NC; ++c) {
      KState& k = ks[i * NC + c];
      k.rr = out[(int64_t)i * 2 * NC + 2 * c];
      k.bb = fmax(out[(int64_t)i * 2 * NC + 2 * c + 1], k.rr);
      k.rho = k.rr;
      k.alpha = 1.0;
      k.omega = 1.0;
      k.beta = 0.0;
      k.af = 1.f;
      k.of = 1.f;
      k.bf = 0.f;
      k.iter = 0;
      k.status = 0;
      k.done = (skip || k.rr <= k.tol2 * k.bb) ? 1 : 0;
      if (!skip && !isfinite(k.rr)) { k.done = 1; k.status = 5; }
      any = any || !k.done;
    }
  }
  any = block_any(any);
  if (threadIdx.x == 0) set_cond(cond, any);
}

// ---------------------------------------------------------------- BiCGStab, streaming form
// Chunked, 16-byte vector forms of the BiCGStab updates.  The operator outputs
// v = A ph and t = A sh are interface-summed (fe_apply) before they are read.

// p = r + beta (p - omega v), ph = D^-1 p  (kept slots; 0 elsewhere)
template <typename T, int NC>
__global__ void __launch_bounds__(512) k_bcgv_p(DevGrid g, const T* __restrict__ r, T* __restrict__ p,
                                                const T* __restrict__ v, T* __restrict__ ph,
                                                const T* __restrict__ dinv, uint16_t dmask, const KState* ks) {
  KCOUNT();
  using V = typename Vec16<T>::type;
  using MT = typename Vec16<T>::mt;
  constexpr int W = Vec16<T>::W;
  const int b0 = g.scbrick[blockIdx.x], b1 = g.scbrick[blockIdx.x + 1];
  const KState* ki = ks + g.binst[b0] * NC;
  bool act[NC];
  T bec[NC], omc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    act[c] = !ki[c].done;
    bec[c] = k_beta<T>(ki[c]);
    omc[c] = k_omega<T>(ki[c]);
  }
  const int64_t s1 = (int64_t)b1 * DBV;
#pragma unroll 2
  for (int64_t s = (int64_t)b0 * DBV + threadIdx.x * W; s < s1; s += (int64_t)blockDim.x * W) {
    const MT mv = *reinterpret_cast<const MT*>(g.meta + s);
    const uint16_t* mm = reinterpret_cast<const uint16_t*>(&mv);
    if (!(vec_or_n<W>(mm) & D_VALID)) continue;   // brick padding: always zero, never read or written
    const V dv = *reinterpret_cast<const V*>(dinv + s);
    const T* de = reinterpret_cast<const T*>(&dv);
    for (int c = 0; c < NC; ++c) {
      if (!act[c]) continue;
      const T be = bec[c], om = omc[c];
      const int64_t i = (int64_t)c * g.nslots + s;
      const V rv = *reinterpret_cast<const V*>(r + i);
      const V vv = *reinterpret_cast<const V*>(v + i);
      V pv = *reinterpret_cast<const V*>(p + i);
      V hv;
      const T* re = reinterpret_cast<const T*>(&rv);
      const T* ve = reinterpret_cast<const T*>(&vv);
      T* pe = reinterpret_cast<T*>(&pv);
      T* he = reinterpret_cast<T*>(&hv);
#pragma unroll
      for (int j = 0; j < W; ++j) {
        const uint16_t m = mm[j];
        const T vs = ve[j];
        const T pn = kkeep(m, dmask, c) ? T(re[j] + be * (pe[j] - om * vs)) : T(0);
        pe[j] = pn;
        he[j] = pn * de[j];
      }
      *reinterpret_cast<V*>(p + i) = pv;
      *reinterpret_cast<V*>(ph + i) = hv;
    }
  }
}

// mode 0: alpha = rho / (rh, v);  mode 1: omega = (t, s) / (t, t)
template <typename T, int NC>
__global__ void __launch_bounds__(512) k_bcgv_dot(DevGrid g, const T* __restrict__ a1, const T* __restrict__ b1v,
                                                  uint16_t dmask, int mode, KState* ks, double* partials,
                                                  unsigned* counter, int coupled) {
  KCOUNT();
  using V = typename Vec16<T>::type;
  using MT = typename Vec16<T>::mt;
  constexpr int W = Vec16<T>::W;
  const int b0 = g.scbrick[blockIdx.x], b1 = g.scbrick[blockIdx.x + 1];
  const KState* ki = ks + g.binst[b0] * NC;
  bool act[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) act[c] = !ki[c].done;
  T tw[2 * NC];
#pragma unroll
  for (int c = 0; c < 2 * NC; ++c) tw[c] = T(0);
  // b1v is the operator output (v or t); a1 is rh (mode 0) or s (mode 1)
  const int64_t s1 = (int64_t)b1 * DBV;
#pragma unroll 2
  for (int64_t s = (int64_t)b0 * DBV + threadIdx.x * W; s < s1; s += (int64_t)blockDim.x * W) {
    const MT mv = *reinterpret_cast<const MT*>(g.meta + s);
    const uint16_t* mm = reinterpret_cast<const uint16_t*>(&mv);
    if (!(vec_or_n<W>(mm) & D_VALID)) continue;   // brick padding: always zero, never read or written
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (!act[c]) continue;
      const int64_t i = (int64_t)c * g.nslots + s;
      const V av = *reinterpret_cast<const V*>(a1 + i);
      const V bv = *reinterpret_cast<const V*>(b1v + i);
      const T* ae = reinterpret_cast<const T*>(&av);
      const T* be = reinterpret_cast<const T*>(&bv);
#pragma unroll
      for (int j = 0; j < W; ++j) {
        const uint16_t m = mm[j];
        if (!kdof(m, dmask, c)) continue;
        const T q = be[j];
        tw[2 * c] += ae[j] * q;
        if (mode == 1) tw[2 * c + 1] += q * q;
      }
    }
  }
  double* out = partials + (int64_t)gridDim.x * 2 * NC;
  if (!grid_sum_last<T, 2 * NC>(tw, partials, counter, g.scseg, g.ninst, out)) return;
  for (int i = threadIdx.x; i < g.ninst; i += blockDim.x) {
    if (coupled) couple_sums<NC, 2>(out + (int64_t)i * 2 * NC);
    for (int c = 0; c < NC; ++c) {
      KState& k = ks[i * NC + c];
      if (k.done) continue;
      const double t0 = out[(int64_t)i * 2 * NC + 2 * c], t1 = out[(int64_t)i * 2 * NC + 2 * c + 1];
      if (mode == 0) {
        k.rv = t0;
        if (k.rv == 0.0 || !isfinite(k.rv)) { k.done = 1; k.status = 5; k.alpha = 0.0; k.af = 0.f; continue; }
        k.alpha = k.rho / k.rv;
        k.af = float(k.alpha);
      } else {
        k.ts = t0;
        k.tt = t1;
        k.omega = (k.tt > 0.0) ? k.ts / k.tt : 0.0;
        k.of = float(k.omega);
      }
    }
  }
}

// s = r - alpha v, sh = D^-1 s
template <typename T, int NC>
__global__ void __launch_bounds__(512) k_bcgv_s(DevGrid g, const T* __restrict__ r, const T* __restrict__ v,
                                                T* __restrict__ sv, T* __restrict__ sh, const T* __restrict__ dinv,
                                                uint16_t dmask, const KState* ks) {
  KCOUNT();
  using V = typename Vec16<T>::type;
  using MT = typename Vec16<T>::mt;
  constexpr int W = Vec16<T>::W;
  const int b0 = g.scbrick[blockIdx.x], b1 = g.scbrick[blockIdx.x + 1];
  const KState* ki = ks + g.binst[b0] * NC;
  bool act[NC];
  T alc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    act[c] = !ki[c].done;
    alc[c] = k_alpha<T>(ki[c]);
  }
  const int64_t s1 = (int64_t)b1 * DBV;
#pragma unroll 2
  for (int64_t s = (int64_t)b0 * DBV + threadIdx.x * W; s < s1; s += (int64_t)blockDim.x * W) {
    const MT mv = *reinterpret_cast<const MT*>(g.meta + s);
    const uint16_t* mm = reinterpret_cast<const uint16_t*>(&mv);
    if (!(vec_or_n<W>(mm) & D_VALID)) continue;   // brick padding: always zero, never read or written
    const V dv = *reinterpret_cast<const V*>(dinv + s);
    const T* de = reinterpret_cast<const T*>(&dv);
    for (int c = 0; c < NC; ++c) {
      if (!act[c]) continue;
      const T al = alc[c];
      const int64_t i = (int64_t)c * g.nslots + s;
      const V rv = *reinterpret_cast<const V*>(r + i);
      const V vv = *reinterpret_cast<const V*>(v + i);
      V so, ho;
      const T* re = reinterpret_cast<const T*>(&rv);
      const T* ve = reinterpret_cast<const T*>(&vv);
      T* se = reinterpret_cast<T*>(&so);
      T* he = reinterpret_cast<T*>(&ho);
#pragma unroll
      for (int j = 0; j < W; ++j) {
        const uint16_t m = mm[j];
        const T vs = ve[j];
        const T sn = kkeep(m, dmask, c) ? T(re[j] - al * vs) : T(0);
        se[j] = sn;
        he[j] = sn * de[j];
      }
      *reinterpret_cast<V*>(sv + i) = so;
      *reinterpret_cast<V*>(sh + i) = ho;
    }
  }
}

// x += alpha ph + omega sh, r = s - omega t; ||r||^2, (rh, r) -> beta, rho
template <typename T, int NC>
__global__ void __launch_bounds__(512) k_bcgv_xr(DevGrid g, T* __restrict__ x, T* __restrict__ r,
                                                 const T* __restrict__ rh, const T* __restrict__ ph,
                                                 const T* __restrict__ sh, const T* __restrict__ sv,
                                                 const T* __restrict__ tv, uint16_t dmask, KState* ks,
                                                 double* partials, unsigned* counter, Cond cond, int coupled) {
  KCOUNT();
  using V = typename Vec16<T>::type;
  using MT = typename Vec16<T>::mt;
  constexpr int W = Vec16<T>::W;
  const int b0 = g.scbrick[blockIdx.x], b1 = g.scbrick[blockIdx.x + 1];
  const KState* ki = ks + g.binst[b0] * NC;
  bool act[NC];
  T alc[NC], omc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    act[c] = !ki[c].done;
    alc[c] = k_alpha<T>(ki[c]);
    omc[c] = k_omega<T>(ki[c]);
  }
  T tw[2 * NC];
#pragma unroll
  for (int c = 0; c < 2 * NC; ++c) tw[c] = T(0);
  const int64_t s1 = (int64_t)b1 * DBV;
#pragma unroll 2
  for (int64_t s = (int64_t)b0 * DBV + threadIdx.x * W; s < s1; s += (int64_t)blockDim.x * W) {
    const MT mv = *reinterpret_cast<const MT*>(g.meta + s);
    const uint16_t* mm = reinterpret_cast<const uint16_t*>(&mv);
    if (!(vec_or_n<W>(mm) & D_VALID)) continue;   // brick padding: always zero, never read or written
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (!act[c]) continue;
      const T al = alc[c], om = omc[c];
      const int64_t i = (int64_t)c * g.nslots + s;
      V xv = *reinterpret_cast<const V*>(x + i);
      const V pv = *reinterpret_cast<const V*>(ph + i);
      const V hv = *reinterpret_cast<const V*>(sh + i);
      const V sv_ = *reinterpret_cast<const V*>(sv + i);
      const V tv_ = *reinterpret_cast<const V*>(tv + i);
      const V qv = *reinterpret_cast<const V*>(rh + i);
      V ro;
      T* xe = reinterpret_cast<T*>(&xv);
      const T* pe = reinterpret_cast<const T*>(&pv);
      const T* he = reinterpret_cast<const T*>(&hv);
      const T* se = reinterpret_cast<const T*>(&sv_);
      const T* te = reinterpret_cast<const T*>(&tv_);
      const T* qe = reinterpret_cast<const T*>(&qv);
      T* oe = reinterpret_cast<T*>(&ro);
#pragma unroll
      for (int j = 0; j < W; ++j) {
        const uint16_t m = mm[j];
        if (m & D_VALID) xe[j] += al * pe[j] + om * he[j];
        const T ts = te[j];
        const T rn = kkeep(m, dmask, c) ? T(se[j] - om * ts) : T(0);
        oe[j] = rn;
        if (kdof(m, dmask, c)) {
          tw[2 * c] += rn * rn;
          tw[2 * c + 1] += qe[j] * rn;
        }
      }
      *reinterpret_cast<V*>(x + i) = xv;
      *reinterpret_cast<V*>(r + i) = ro;
    }
  }
  double* out = partials + (int64_t)gridDim.x * 2 * NC;
  if (!grid_sum_last<T, 2 * NC>(tw, partials, counter, g.scseg, g.ninst, out)) return;
  bool any = false;
  for (int i = threadIdx.x; i < g.ninst; i += blockDim.x) {
    if (coupled) couple_sums<NC, 2>(out + (int64_t)i * 2 * NC);
    for (int c = 0; c < NC; ++c) {
      KState& k = ks[i * NC + c];
      if (k.done) continue;
      k.iter++;
      k.rr = out[(int64_t)i * 2 * NC + 2 * c];
      const double rhon = out[(int64_t)i * 2 * NC + 2 * c + 1];
      if (!isfinite(k.rr)) { k.done = 1; k.status = 5; continue; }
      if (k.rr <= k.tol2 * k.bb) { k.done = 1; continue; }
      if (k.iter >= k.max_iter) { k.done = 1; k.status = 4; continue; }
      if (k.omega == 0.0 || rhon == 0.0 || !isfinite(rhon)) { k.done = 1; k.status = 5; continue; }
      k.beta = (rhon / k.rho) * (k.alpha / k.omega);
      k.bf = float(k.beta);
      k.rho = rhon;
      any = true;
    }
  }
  any = block_any(any);
  if (threadIdx.x == 0) set_cond(cond, any);
}

// ---------------------------------------------------------------- FP64 outer loop
// r = b - y on DOF rows, formed exactly from the FP64 values as a pair of FP32
// numbers (ff_diff; r64 holds the pairs, hi and lo, in place of FP64 values),
// the inner initial guess zeroed (e32); ||r||^2 and, on the first pass,
// ||b||^2 for the reference norm, each thread keeping a scaled FP32 sum of
// squares (scale, sum: no FP64 instruction per element, no underflow for
// entries above 2^-126) that it hands to the FP64 grid sum as scale^2 sum;
// per component the power of two that brings ||r|| into [0.5, 1) (sexp), by
// which k_scale_residual divides r when it rounds it to FP32 as the inner
// right-hand side, so that the FP32 iterations never see values whose
// squares leave the FP32 range (a problem in SI units has velocity
// residuals near 1e-20).  Sets the outer loop condition and the condition of
// the inner-solve branch.  One CTA per chunk of bricks.
__device__ __forceinline__ void sumsq_add(float& scale, float& sum, float x) {
  const float a = fabsf(x);
  if (a == 0.f) return;
  if (a > scale) {
    const float q = scale / a;
    sum = 1.f + sum * (q * q);
    scale = a;
  } else {
    const float q = a / scale;
    sum += q * q;
  }
}
__device__ __forceinline__ double sumsq_value(float scale, float sum) {
  const double s = f2d(scale);
  return f2d(sum) * (s * s);
}

template <int NC>
__global__ void __launch_bounds__(512) k_residual_outer(DevGrid g, const double* __restrict__ b,
                                                        const double* __restrict__ y, double* __restrict__ r64,
                                                        float* __restrict__ e32, uint16_t dmask, OState* os,
                                                        double* partials, unsigned* counter, Cond cloop,
                                                        Cond cbranch) {
  KCOUNT();
  const int b0 = g.scbrick[blockIdx.x], b1 = g.scbrick[blockIdx.x + 1];
  const OState& oi = os[g.binst[b0]];
  const bool first = oi.iter == 0;
  float rs[NC], rq[NC], bs[NC], bq[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) rs[c] = rq[c] = bs[c] = bq[c] = 0.f;
  // pairs of slots: 16-byte FP64 loads, 16-byte pair and 8-byte FP32 stores
  const int64_t s1 = (int64_t)b1 * DBV;
  if (!oi.done) {
#pragma unroll 2
    for (int64_t s = (int64_t)b0 * DBV + threadIdx.x * 2; s < s1; s += (int64_t)blockDim.x * 2) {
      const uint32_t mv = *reinterpret_cast<const uint32_t*>(g.meta + s);
      const uint16_t mm[2] = {uint16_t(mv & 0xFFFFu), uint16_t(mv >> 16)};
      if (!((mm[0] | mm[1]) & D_VALID)) continue;   // brick padding: r and e32 stay zero there
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int64_t i = c * g.nslots + s;
        const double2 bv = *reinterpret_cast<const double2*>(b + i);
        const double2 yv = *reinterpret_cast<const double2*>(y + i);
        const double be[2] = {bv.x, bv.y}, ye[2] = {yv.x, yv.y};
        ff rv[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const ff fb = dsplit(be[j]);
          rv[j] = kkeep(mm[j], dmask, c) ? ff_diff(fb, dsplit(ye[j])) : ff{0.f, 0.f};
          if (kdof(mm[j], dmask, c)) {
            sumsq_add(rs[c], rq[c], rv[j].h);
            if (first) sumsq_add(bs[c], bq[c], fb.h);
          }
        }
        *reinterpret_cast<float4*>(r64 + i) = make_float4(rv[0].h, rv[0].l, rv[1].h, rv[1].l);
        *reinterpret_cast<float2*>(e32 + i) = make_float2(0.f, 0.f);
      }
    }
  }
  double w[2 * NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    w[2 * c] = sumsq_value(rs[c], rq[c]);
    w[2 * c + 1] = sumsq_value(bs[c], bq[c]);
  }
  double* out = partials + (int64_t)gridDim.x * 2 * NC;
  if (!grid_sum_last<double, 2 * NC>(w, partials, counter, g.scseg, g.ninst, out)) return;
  bool any = false;
  for (int i = threadIdx.x; i < g.ninst; i += blockDim.x) {
    OState& o = os[i];
    if (o.done) continue;
    double rel2 = 0.0;
    bool finite = true;
    for (int c = 0; c < NC; ++c) {
      const double rr = out[(int64_t)i * 2 * NC + 2 * c], bb = out[(int64_t)i * 2 * NC + 2 * c + 1];
      if (o.iter == 0) o.ref[c] = fmax(bb, rr);
      if (!isfinite(rr)) finite = false;
      if (o.ref[c] > 0.0) rel2 = fmax(rel2, rr / o.ref[c]);
      int ex = 0;
      if (rr > 0.0 && isfinite(rr)) frexp(sqrt(rr), &ex);
      o.sexp[c] = ex;
    }
    o.rel2 = rel2;
    // converged; or stagnated at the attainable FP64 accuracy (the residual
    // fell by less than 4x in the last pass while within 1e3 of the tolerance)
    const bool stagnated = o.iter > 0 && rel2 > 0.0625 * o.prev2 && rel2 <= 1e6 * o.tol2;
    if (!finite || o.inner_status == 5) { o.done = 1; o.status = 5; }
    else if (rel2 <= o.tol2 || stagnated) o.done = 1;
    else if (o.iter >= o.max_iter) { o.done = 1; o.status = 4; }
    o.prev2 = rel2;
    if (!o.done) { o.iter++; any = true; }
  }
  any = block_any(any);
  if (threadIdx.x == 0) {
    set_cond(cloop, any);
    set_cond(cbranch, any);
  }
}

// r32 = r * 2^-sexp, rounded to FP32: the scaled inner right-hand side (only
// instances whose outer loop is still running); r comes as the pair (hi, lo)
// that k_residual_outer stored in place of an FP64 value
__global__ void k_scale_residual(DevGrid g, const double* __restrict__ r64, float* __restrict__ r32, int nc,
                                 const OState* os) {
  KCOUNT();
  const OState& o = os[g.binst[blockIdx.x]];
  if (o.done) return;
  const int64_t s = (int64_t)blockIdx.x * DBV + threadIdx.x;
  const float2* rp = reinterpret_cast<const float2*>(r64);
  for (int c = 0; c < nc; ++c) {
    const float2 p = rp[c * g.nslots + s];
    // a power of two applied in at most two exact steps (the scale may leave
    // the normal FP32 range; the scaled values do not)
    const int e = -o.sexp[c];
    const int e1 = e > 126 ? 126 : (e < -126 ? -126 : e);
    const int e2 = max(-126, min(126, e - e1));
    const float v = __fadd_rn(p.x, p.y);
    r32[c * g.nslots + s] = __fmul_rn(__fmul_rn(v, __int_as_float((127 + e1) << 23)), __int_as_float((127 + e2) << 23));
  }
}

// x += e * 2^sexp (the inner solution of the scaled right-hand side), only
// for instances whose outer loop is still running
// (e exactly in FP64 from its bits, the power of two on the exponent field:
// one FP64 instruction per element, the addition)
__global__ void k_add_f2d_active(DevGrid g, const float* __restrict__ e, double* __restrict__ x, int nc,
                                 const OState* os) {
  KCOUNT();
  const OState& o = os[g.binst[blockIdx.x]];
  if (o.done) return;
  const int64_t s = (int64_t)blockIdx.x * DBV + threadIdx.x;
  for (int c = 0; c < nc; ++c) x[c * g.nslots + s] += scale2(f2d(e[c * g.nslots + s]), o.sexp[c]);
}

// ---------------------------------------------------------------- drivers
template <typename T>
struct Work {
  T *r, *z, *pa, *pb, *q;            // CG
  T *rh, *p, *v, *sv, *tv, *ph, *sh; // BiCGStab (r shared)
};

template <typename T>
static Work<T> carve(T* w, int64_t L) {
  Work<T> k;
  k.r = w;
  k.z = w + L;
  k.pa = w + 2 * L;
  k.pb = w + 3 * L;
  k.q = w + 4 * L;
  k.rh = w + L;
  k.p = w + 2 * L;
  k.v = w + 3 * L;
  k.sv = w + 4 * L;
  k.tv = w + 5 * L;
  k.ph = w + 6 * L;
  k.sh = w + 7 * L;
  return k;
}

static inline void pbegin(Prof* p, int c, cudaStream_t s) { if (p && p->on) p->begin(c, s); }
static inline void pend(Prof* p, cudaStream_t s) { if (p && p->on) p->end(s); }

// one CG solve of A x = b in precision T (x: initial guess in, solution out)
template <typename T, int NC>
static cudaError_t cg_enqueue(const SolveArgs& a, const OpDesc<T>& A, const T* b, T* x, T* work, cudaStream_t st,
                              CaptureCtx* cc, double rtol, const OState* skip_os, bool x_zero) {
  const DevGrid& g = *a.g;
  const int64_t L = int64_t(NC) * g.nslots;
  Work<T> w = carve(work, L);
  RedBuf rb = a.rb;
  IBG_LAUNCH(k_init_states, (g.ninst * NC + 127) / 128, 128, 0, st, a.ks, g.ninst * NC, rtol * rtol, a.max_iter);
  Cond cond;
  const bool cap = cc && cc->capturing;
  if (cap) {
    cudaError_t e = cond_handle(st, 0, &cond);
    if (e != cudaSuccess) return e;
  }
  if (!x_zero) fe_apply<T>(g, A, NC, x, w.q, st);
  IBG_LAUNCH((k_cg_start<T, NC>), g.nbricks, DBV, 0, st, g, b, x_zero ? (const T*)nullptr : (const T*)w.q, w.r,
             w.z, w.pa, A.dinv, A.dmask, a.ks, rb.partials, rb.counter, cond, skip_os);
  fe_expand2<T>(g, NC, w.z, w.pa, st);
  auto iter = [&](cudaStream_t s, const Cond& c, T* pold, T* pnew) {
    pbegin(a.prof, a.pbase + 0, s);
    fe_apply_cg<T>(g, A, NC, w.z, pold, pnew, w.q, a.ks, rb, s);
    pend(a.prof, s);
    fe_sync<T>(g, NC, w.q, A.dmask, s);
    pbegin(a.prof, a.pbase + 1, s);
    IBG_LAUNCH((k_cg_update_vec<T, NC>), g.nschunks, DBV, 0, s, g, x, w.r, w.z, pnew, w.q, A.dinv, A.dmask, a.ks,
               rb.partials, rb.counter, c);
    pend(a.prof, s);
    fe_expand2<T>(g, NC, w.z, (T*)nullptr, s);
  };
  return run_loop(cc, st, cond, a.ks, a.ks_host, g.ninst * NC, a.max_iter, 2, 16, [&](cudaStream_t s, const Cond& c) {
    iter(s, c, w.pa, w.pb);
    iter(s, c, w.pb, w.pa);
  });
}

template <typename T>
static const MGDev<T>* mg_of(const SolveArgs& a) {
  if constexpr (sizeof(T) == 4) return a.mg32; else return a.mg64;
}

// CG with the multigrid V-cycle as preconditioner (Poisson, one component)
template <typename T>
static cudaError_t cg_mg_enqueue(const SolveArgs& a, const OpDesc<T>& A, const MGDev<T>& mg, const T* b, T* x,
                                 T* work, cudaStream_t st, CaptureCtx* cc, double rtol, const OState* skip_os,
                                 bool x_zero) {
  const DevGrid& g = *a.g;
  const int64_t L = g.nslots;
  Work<T> w = carve(work, L);
  T* zs = work + 5 * L;
  RedBuf rb = a.rb;
  IBG_LAUNCH(k_init_states, (g.ninst + 127) / 128, 128, 0, st, a.ks, g.ninst, rtol * rtol, a.max_iter);
  Cond cond;
  if (cc && cc->capturing) {
    cudaError_t e = cond_handle(st, 0, &cond);
    if (e != cudaSuccess) return e;
  }
  if (!x_zero) fe_apply<T>(g, A, 1, x, w.q, st);
  IBG_LAUNCH(k_cg_start_r<T>, g.nbricks, DBV, 0, st, g, b, x_zero ? (const T*)nullptr : (const T*)w.q, w.r, A.dmask,
             a.ks, rb.partials, rb.counter, skip_os);
  mg_vcycle<T>(g, mg, w.r, w.z, zs, w.q, A.dinv, A.dmask, a.ks, st, a.prof, 9);
  IBG_LAUNCH(k_cg_rz<T>, g.nschunks, DBV, 0, st, g, w.r, w.z, A.dmask, a.ks, rb.partials, rb.counter, cond, 1);
  auto iter = [&](cudaStream_t s, const Cond& c, T* pold, T* pnew) {
    pbegin(a.prof, a.pbase + 0, s);
    fe_apply_cg<T>(g, A, 1, w.z, pold, pnew, w.q, a.ks, rb, s);
    pend(a.prof, s);
    fe_sync<T>(g, 1, w.q, A.dmask, s);
    pbegin(a.prof, a.pbase + 1, s);
    IBG_LAUNCH(k_cg_update_r<T>, g.nschunks, DBV, 0, s, g, x, w.r, pnew, w.q, A.dmask, a.ks, rb.partials,
               rb.counter);
    pend(a.prof, s);
    mg_vcycle<T>(g, mg, w.r, w.z, zs, w.q, A.dinv, A.dmask, a.ks, s, a.prof, 9);
    IBG_LAUNCH(k_cg_rz<T>, g.nschunks, DBV, 0, s, g, w.r, w.z, A.dmask, a.ks, rb.partials, rb.counter, c, 0);
  };
  return run_loop(cc, st, cond, a.ks, a.ks_host, g.ninst, a.max_iter, 1, 4, [&](cudaStream_t s, const Cond& c) {
    iter(s, c, w.pa, w.pb);
    iter(s, c, w.pb, w.pa);
  });
}

template <typename T, int NC>
static cudaError_t bcg_enqueue(const SolveArgs& a, const OpDesc<T>& A, const T* b, T* x, T* work, cudaStream_t st,
                               CaptureCtx* cc, double rtol, const OState* skip_os, bool x_zero) {
  const DevGrid& g = *a.g;
  const int64_t L = int64_t(NC) * g.nslots;
  Work<T> w = carve(work, L);
  RedBuf rb = a.rb;
  IBG_LAUNCH(k_init_states, (g.ninst * NC + 127) / 128, 128, 0, st, a.ks, g.ninst * NC, rtol * rtol, a.max_iter);
  Cond cond;
  if (cc && cc->capturing) {
    cudaError_t e = cond_handle(st, 0, &cond);
    if (e != cudaSuccess) return e;
  }
  if (!x_zero) fe_apply<T>(g, A, NC, x, w.tv, st);
  const int cpl = a.coupled ? 1 : 0;
  IBG_LAUNCH((k_bcg_start<T, NC>), g.nbricks, DBV, 0, st, g, b, x_zero ? (const T*)nullptr : (const T*)w.tv, w.r,
             w.rh, w.p, w.v, A.dmask, a.ks, rb.partials, rb.counter, cond, skip_os, cpl);
  // v and t hold the interface-summed operator outputs (the start kernel set v = 0)
  return run_loop(cc, st, cond, a.ks, a.ks_host, g.ninst * NC, a.max_iter, 1, 8, [&](cudaStream_t s, const Cond& c) {
    pbegin(a.prof, a.pbase + 2, s);
    IBG_LAUNCH((k_bcgv_p<T, NC>), g.nschunks, DBV, 0, s, g, w.r, w.p, w.v, w.ph, A.dinv, A.dmask, a.ks);
    pend(a.prof, s);
    fe_expand2<T>(g, NC, w.ph, (T*)nullptr, s);
    pbegin(a.prof, a.pbase + 0, s);
    fe_apply_local<T>(g, A, NC, w.ph, w.v, s);
    pend(a.prof, s);
    fe_sync<T>(g, NC, w.v, A.dmask, s);
    IBG_LAUNCH((k_bcgv_dot<T, NC>), g.nschunks, DBV, 0, s, g, w.rh, w.v, A.dmask, 0, a.ks, rb.partials, rb.counter,
               cpl);
    IBG_LAUNCH((k_bcgv_s<T, NC>), g.nschunks, DBV, 0, s, g, w.r, w.v, w.sv, w.sh, A.dinv, A.dmask, a.ks);
    fe_expand2<T>(g, NC, w.sh, (T*)nullptr, s);
    pbegin(a.prof, a.pbase + 0, s);
    fe_apply_local<T>(g, A, NC, w.sh, w.tv, s);
    pend(a.prof, s);
    fe_sync<T>(g, NC, w.tv, A.dmask, s);
    IBG_LAUNCH((k_bcgv_dot<T, NC>), g.nschunks, DBV, 0, s, g, w.sv, w.tv, A.dmask, 1, a.ks, rb.partials,
               rb.counter, cpl);
    pbegin(a.prof, a.pbase + 1, s);
    IBG_LAUNCH((k_bcgv_xr<T, NC>), g.nschunks, DBV, 0, s, g, x, w.r, w.rh, w.ph, w.sh, w.sv, w.tv, A.dmask, a.ks,
               rb.partials, rb.counter, c, cpl);
    pend(a.prof, s);
  });
}

// x_zero: the initial guess is zero (the mixed path's corrections), so its
// operator product is not formed and the residual starts as b
template <typename T>
static cudaError_t inner_enqueue(const SolveArgs& a, const OpDesc<T>& A, const T* b, T* x, T* work, cudaStream_t st,
                                 CaptureCtx* cc, double rtol, const OState* skip_os, bool x_zero) {
  if (a.bicg) return a.nc == 1 ? bcg_enqueue<T, 1>(a, A, b, x, work, st, cc, rtol, skip_os, x_zero)
                               : bcg_enqueue<T, 3>(a, A, b, x, work, st, cc, rtol, skip_os, x_zero);
  if (a.nc == 1 && a.op == OP_POISSON) {
    const MGDev<T>* mg = mg_of<T>(a);
    if (mg && mg->any) return cg_mg_enqueue<T>(a, A, *mg, b, x, work, st, cc, rtol, skip_os, x_zero);
  }
  return a.nc == 1 ? cg_enqueue<T, 1>(a, A, b, x, work, st, cc, rtol, skip_os, x_zero)
                   : cg_enqueue<T, 3>(a, A, b, x, work, st, cc, rtol, skip_os, x_zero);
}

cudaError_t solve_enqueue(const SolveArgs& a, cudaStream_t st, CaptureCtx* cc) {
  const DevGrid& g = *a.g;
  OpDesc<double> A64{a.op, a.coef64, a.dmask, a.dinv64, a.prof, a.pbase};
  const int ib = (g.ninst + 127) / 128;
  if (!a.mixed) {
    cudaError_t e = inner_enqueue<double>(a, A64, a.b, a.x, a.w64, st, cc, a.rtol, nullptr, false);
    if (e != cudaSuccess) return e;
    IBG_LAUNCH(k_collect, ib, 128, 0, st, a.ks, a.nc, g.ninst, a.rec, (OState*)nullptr);
    return cudaSuccess;
  }
  OpDesc<float> A32{a.op, a.coef32, a.dmask, a.dinv32, a.prof, a.pbase};
  IBG_LAUNCH(k_init_outer, ib, 128, 0, st, a.os, g.ninst, a.nc, a.rtol * a.rtol, a.max_outer);
  const bool cap = cc && cc->capturing;
  auto residual = [&](cudaStream_t s, const Cond& cl, const Cond& cb) {
    fe_apply_resid(g, A64, a.nc, a.x, a.y64, a.coeflo32 ? a.coef32 : nullptr, a.coeflo32, s);
    if (a.nc == 1)
      IBG_LAUNCH(k_residual_outer<1>, g.nschunks, DBV, 0, s, g, a.b, a.y64, a.r64, a.e32, a.dmask, a.os, a.rb.partials,
                 a.rb.counter, cl, cb);
    else
      IBG_LAUNCH(k_residual_outer<3>, g.nschunks, DBV, 0, s, g, a.b, a.y64, a.r64, a.e32, a.dmask, a.os, a.rb.partials,
                 a.rb.counter, cl, cb);
  };
  auto correction = [&](cudaStream_t s) {
    IBG_LAUNCH(k_scale_residual, g.nbricks, DBV, 0, s, g, (const double*)a.r64, a.r32, a.nc, (const OState*)a.os);
    // the correction starts from zero (k_residual_outer cleared e32)
    cudaError_t e = inner_enqueue<float>(a, A32, a.r32, a.e32, a.w32, s, cc, a.rtol_inner, a.os, true);
    IBG_LAUNCH(k_collect, ib, 128, 0, s, a.ks, a.nc, g.ninst, a.rec, a.os);
    IBG_LAUNCH(k_add_f2d_active, g.nbricks, DBV, 0, s, g, a.e32, a.x, a.nc, (const OState*)a.os);
    // the FP32 correction carries hanging values rounded in FP32: restore the
    // constraint (hanging = mean of parents) in FP64
    fe_expand<double>(g, a.nc, a.x, s);
    return e;
  };
  cudaError_t err = cudaSuccess;
  if (cap) {
    Cond cl;
    if ((err = cond_handle(st, 1, &cl)) != cudaSuccess) return err;
    err = cond_node(*cc, st, cl, cudaGraphCondTypeWhile, [&](cudaStream_t s) {
      Cond cb;
      cudaError_t e = cond_handle(s, 0, &cb);
      if (e != cudaSuccess) { err = e; return; }
      residual(s, cl, cb);
      e = cond_node(*cc, s, cb, cudaGraphCondTypeIf, [&](cudaStream_t s2) {
        cudaError_t e2 = correction(s2);
        if (e2 != cudaSuccess) err = e2;
      });
      if (e != cudaSuccess) err = e;
    });
    if (err != cudaSuccess) return err;
  } else {
    const Cond none;
    for (int it = 0; it <= a.max_outer + 1; ++it) {
      residual(st, none, none);
      cudaMemcpyAsync(a.os_host, a.os, g.ninst * sizeof(OState), cudaMemcpyDeviceToHost, st);
      if ((err = cudaStreamSynchronize(st)) != cudaSuccess) return err;
      bool all = true;
      for (int i = 0; i < g.ninst; ++i) all = all && a.os_host[i].done;
      if (all) break;
      if ((err = correction(st)) != cudaSuccess) return err;
    }
  }
  IBG_LAUNCH(k_collect_outer, ib, 128, 0, st, a.os, g.ninst, a.rec);
  return cudaSuccess;
}

__global__ void k_rec_clear(SolveRec* rec, int n) {
  KCOUNT();
  const int i = threadIdx.x + blockIdx.x * blockDim.x;
  if (i < n) {
    SolveRec r;
    memset(&r, 0, sizeof(r));
    rec[i] = r;
  }
}

void rec_clear(SolveRec* rec, int n, cudaStream_t st) { IBG_LAUNCH(k_rec_clear, (n + 127) / 128, 128, 0, st, rec, n); }

}  // namespace ibg
