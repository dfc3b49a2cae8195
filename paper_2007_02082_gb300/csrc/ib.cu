// BCE-IB kernels (Sec. 2.3): the 4-point delta kernel of Eq. 18, interpolation
// B_F = U_B - h^3 D^T u~ (Eq. 23), the force matrix of Eq. 22 and its PCG solve,
// and spreading f = sum_i F_i D_ij dS_i (Eq. 19) fused with u = u~ + dt f/rho
// (Eq. 14).  With area elements on the columns (dS_k in A_F[i,k]) A_F = S diag(dS)
// with S symmetric; the solver works with G = dS * F, so F = G / dS.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ib.hpp"
#include "krylov.hpp"

namespace ibg {

IBG_KCOUNT_DEFINE
unsigned long long ib_kcount() {
  unsigned long long v = 0;
  cudaMemcpyFromSymbol(&v, g_kcount, sizeof(v));
  return v;
}

// Eq. 18
__device__ __forceinline__ double delta4(double r) {
  r = fabs(r);
  if (r <= 1.0) return (3.0 - 2.0 * r + sqrt(1.0 + 4.0 * r - 4.0 * r * r)) * 0.125;
  if (r <= 2.0) return (5.0 - 2.0 * r - sqrt(-7.0 + 12.0 * r - 4.0 * r * r)) * 0.125;
  return 0.0;
}

__global__ void k_ib_weights(int64_t M, const double* __restrict__ X, const int32_t* __restrict__ org,
                             const int32_t* __restrict__ slot, const int32_t* __restrict__ pinst,
                             const double* __restrict__ iorigin, const double* __restrict__ ihf,
                             double* __restrict__ W) {
  KCOUNT();
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= M * 64) return;
  const int64_t i = e >> 6;
  const int a = int(e & 63);
  if (slot[e] < 0) { W[e] = 0.0; return; }
  const double* o = iorigin + 3 * pinst[i];
  const double* h = ihf + 3 * pinst[i];
  const double x = o[0] + double(org[3 * i] + (a & 3)) * h[0];
  const double y = o[1] + double(org[3 * i + 1] + ((a >> 2) & 3)) * h[1];
  const double z = o[2] + double(org[3 * i + 2] + (a >> 4)) * h[2];
  W[e] = delta4((x - X[3 * i]) / h[0]) * delta4((y - X[3 * i + 1]) / h[1]) * delta4((z - X[3 * i + 2]) / h[2]);
}

// one warp per row: S[i,k] = scale * sum over free common support nodes of w_ia w_kb
__global__ void k_af_values(int64_t M, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const int32_t* __restrict__ org, const uint64_t* __restrict__ fb,
                            const double* __restrict__ W, const double* __restrict__ pscale,
                            double* __restrict__ val, double* __restrict__ dinv, float* __restrict__ val32,
                            float* __restrict__ dinv32) {
  KCOUNT();
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= M) return;
  for (int e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) {
    const int k = col[e];
    const int dx = org[3 * k] - org[3 * i], dy = org[3 * k + 1] - org[3 * i + 1], dz = org[3 * k + 2] - org[3 * i + 2];
    double acc = 0.0;
    for (int a = 0; a < 64; ++a) {
      if (!(fb[i] >> a & 1)) continue;
      const int bx = (a & 3) - dx, by = ((a >> 2) & 3) - dy, bz = (a >> 4) - dz;
      if (bx < 0 || by < 0 || bz < 0 || bx > 3 || by > 3 || bz > 3) continue;
      const int bb = (bz * 4 + by) * 4 + bx;
      acc += W[i * 64 + a] * W[(int64_t)k * 64 + bb];
    }
    const double scale = pscale[i];
    val[e] = scale * acc;
    if (val32) val32[e] = float(scale * acc);
    if (k == i) {
      dinv[i] = acc > 0.0 ? 1.0 / (scale * acc) : 0.0;
      if (dinv32) dinv32[i] = float(dinv[i]);
    }
  }
}

// one warp per point: B_F = U_B - sum_a w_ia u(slot_ia), fixed lane order
__global__ void k_ib_gather(int64_t M, const int32_t* __restrict__ slot, const double* __restrict__ W,
                            const double* __restrict__ u, int64_t nslots, const double* __restrict__ UB,
                            double* __restrict__ BF) {
  KCOUNT();
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= M) return;
  double acc[3] = {0, 0, 0};
  for (int a = lane; a < 64; a += 32) {
    const int32_t s = slot[i * 64 + a];
    if (s < 0) continue;
    const double w = W[i * 64 + a];
    for (int c = 0; c < 3; ++c) acc[c] += w * u[c * nslots + s];
  }
  for (int c = 0; c < 3; ++c)
    for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_down_sync(0xffffffffu, acc[c], o);
  if (lane == 0)
    for (int c = 0; c < 3; ++c) BF[3 * i + c] = UB[3 * i + c] - acc[c];
}

// ---------------------------------------------------------------- PCG on S (3 rhs, [M][3])
constexpr int IBB = 256;   // threads per block; 8 rows per block in the SpMV

__device__ __forceinline__ void spmv_row(int64_t i, int lane, const int32_t* __restrict__ rowptr,
                                         const int32_t* __restrict__ col, const double* __restrict__ val,
                                         const double* __restrict__ x, double (&acc)[3]) {
  acc[0] = acc[1] = acc[2] = 0.0;
  for (int e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) {
    const double v = val[e];
    const int k = col[e];
    for (int c = 0; c < 3; ++c) acc[c] += v * x[3 * k + c];
  }
  for (int c = 0; c < 3; ++c)
    for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_down_sync(0xffffffffu, acc[c], o);
}

// q = S p; p.q -> alpha (mode 1) | y = S x (mode 0).  Warp per row, 8 rows per block.
__global__ void __launch_bounds__(IBB) k_af_apply(IBDev ib, const double* __restrict__ p, double* __restrict__ q,
                                                  int mode, KState* ks, double* partials, unsigned* counter) {
  KCOUNT();
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  double acc[3] = {0, 0, 0};
  if (i < ib.M) spmv_row(i, lane, ib.rowptr, ib.col, ib.val, p, acc);
  double v[3] = {0, 0, 0};
  if (i < ib.M && lane == 0)
    for (int c = 0; c < 3; ++c) {
      q[3 * i + c] = acc[c];
      v[c] = p[3 * i + c] * acc[c];
    }
  if (mode == 0) return;
  double* out = partials + (int64_t)gridDim.x * 3;
  if (!grid_sum_last<double, 3>(v, partials, counter, ib.seg_w, ib.ninst, out)) return;
  for (int n = threadIdx.x; n < ib.ninst; n += blockDim.x)
    for (int c = 0; c < 3; ++c) {
      KState& k = ks[n * 3 + c];
      if (k.done) continue;
      const double pq = out[n * 3 + c];
      k.pq = pq;
      if (!(pq > 0.0) || !isfinite(pq)) { k.done = 1; k.status = 5; k.alpha = 0.0; continue; }
      k.alpha = k.rz / pq;
    }
}

// CG iteration form of the SpMV: p_new = z + beta p_old (read on the fly for
// every column, written for the row), q = S p_new, p_new.q -> alpha.  Eight
// lanes per row (A_F has a few dozen entries per row).
constexpr int AFL = 8;
static_assert(IBB / AFL == 32, "seg_g holds 32-row block ranges");
template <typename T>
__global__ void __launch_bounds__(IBB) k_af_apply_p(IBDev ib, const T* __restrict__ val, const T* __restrict__ z,
                                                    const T* __restrict__ pold, T* __restrict__ pnew,
                                                    T* __restrict__ q, KState* ks, double* partials,
                                                    unsigned* counter) {
  KCOUNT();
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / AFL;
  const int lane = threadIdx.x % AFL;
  T v[3] = {0, 0, 0};
  if (i < ib.M) {
    const KState* ki = ks + ib.pinst[i] * 3;
    const T b0 = k_beta<T>(ki[0]), b1 = k_beta<T>(ki[1]), b2 = k_beta<T>(ki[2]);
    T acc[3] = {0, 0, 0};
    for (int e = ib.rowptr[i] + lane; e < ib.rowptr[i + 1]; e += AFL) {
      const T w = val[e];
      const int64_t k = ib.col[e];
      acc[0] += w * (z[3 * k] + b0 * pold[3 * k]);
      acc[1] += w * (z[3 * k + 1] + b1 * pold[3 * k + 1]);
      acc[2] += w * (z[3 * k + 2] + b2 * pold[3 * k + 2]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
      for (int o = AFL / 2; o > 0; o >>= 1) acc[c] += __shfl_down_sync(0xffffffffu, acc[c], o, AFL);
    if (lane == 0) {
      const T bc[3] = {b0, b1, b2};
      for (int c = 0; c < 3; ++c) {
        const T pv = z[3 * i + c] + bc[c] * pold[3 * i + c];
        pnew[3 * i + c] = pv;
        q[3 * i + c] = acc[c];
        v[c] = pv * acc[c];
      }
    }
  }
  double* out = partials + (int64_t)gridDim.x * 3;
  if (!grid_sum_last<T, 3>(v, partials, counter, ib.seg_g, ib.ninst, out)) return;
  for (int n = threadIdx.x; n < ib.ninst; n += blockDim.x)
    for (int c = 0; c < 3; ++c) {
      KState& k = ks[n * 3 + c];
      if (k.done) continue;
      const double pq = out[n * 3 + c];
      k.pq = pq;
      if (!(pq > 0.0) || !isfinite(pq)) { k.done = 1; k.status = 5; k.alpha = 0.0; k.af = 0.f; continue; }
      k.alpha = k.rz / pq;
      k.af = float(k.alpha);
    }
}

// r = b - y (y may be null: zero initial guess), z = D^-1 r, p = 0; skip_os:
// instances whose FP64 outer loop is done take no inner iterations
template <typename T>
__global__ void __launch_bounds__(IBB) k_af_start(IBDev ib, const T* __restrict__ dinv, const T* __restrict__ b,
                                                  const T* __restrict__ y, T* __restrict__ r, T* __restrict__ z,
                                                  T* __restrict__ p, KState* ks, double* partials,
                                                  unsigned* counter, Cond cond, const OState* skip_os) {
  KCOUNT();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  T v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (i < ib.M)
    for (int c = 0; c < 3; ++c) {
      const T rv = y ? T(b[3 * i + c] - y[3 * i + c]) : b[3 * i + c];
      const T zv = rv * dinv[i];
      r[3 * i + c] = rv;
      z[3 * i + c] = zv;
      p[3 * i + c] = T(0);
      v[3 * c] = rv * zv;
      v[3 * c + 1] = rv * rv;
      v[3 * c + 2] = b[3 * i + c] * b[3 * i + c];
    }
  double* out = partials + (int64_t)gridDim.x * 9;
  if (!grid_sum_last<T, 9>(v, partials, counter, ib.seg_t, ib.ninst, out)) return;
  bool any = false;
  for (int n = threadIdx.x; n < ib.ninst; n += blockDim.x)
    for (int c = 0; c < 3; ++c) {
      KState& k = ks[n * 3 + c];
      const double* t = out + n * 9 + 3 * c;
      const bool skip = skip_os && skip_os[n].done;
      k.rz = t[0];
      k.rr = t[1];
      k.bb = fmax(t[2], k.rr);
      k.beta = 0.0;
      k.bf = 0.f;
      k.iter = 0;
      k.status = 0;
      k.done = (skip || k.rr <= k.tol2 * k.bb) ? 1 : 0;
      if (!skip && !isfinite(k.rr)) { k.done = 1; k.status = 5; }
      any = any || !k.done;
    }
  any = __syncthreads_or(any ? 1 : 0) != 0;
  if (threadIdx.x == 0) set_cond(cond, any);
}

template <typename T>
__global__ void __launch_bounds__(IBB) k_af_update(IBDev ib, const T* __restrict__ dinv, T* __restrict__ x,
                                                   T* __restrict__ r, T* __restrict__ z, const T* __restrict__ p,
                                                   const T* __restrict__ q, KState* ks, double* partials,
                                                   unsigned* counter, Cond cond) {
  KCOUNT();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  T v[6] = {0, 0, 0, 0, 0, 0};
  if (i < ib.M) {
    const KState* ki = ks + ib.pinst[i] * 3;
    for (int c = 0; c < 3; ++c) {
      if (ki[c].done) continue;
      const T a = k_alpha<T>(ki[c]);
      x[3 * i + c] += a * p[3 * i + c];
      const T rv = r[3 * i + c] - a * q[3 * i + c];
      const T zv = rv * dinv[i];
      r[3 * i + c] = rv;
      z[3 * i + c] = zv;
      v[2 * c] = rv * zv;
      v[2 * c + 1] = rv * rv;
    }
  }
  double* out = partials + (int64_t)gridDim.x * 6;
  if (!grid_sum_last<T, 6>(v, partials, counter, ib.seg_t, ib.ninst, out)) return;
  bool any = false;
  for (int n = threadIdx.x; n < ib.ninst; n += blockDim.x)
    for (int c = 0; c < 3; ++c) {
      KState& k = ks[n * 3 + c];
      if (k.done) continue;
      k.iter++;
      k.rr = out[n * 6 + 2 * c + 1];
      const double rzn = out[n * 6 + 2 * c];
      if (!isfinite(k.rr)) { k.done = 1; k.status = 5; continue; }
      if (k.rr <= k.tol2 * k.bb) { k.done = 1; continue; }
      if (k.iter >= k.max_iter) { k.done = 1; k.status = 4; continue; }
      k.beta = rzn / k.rz;
      k.bf = float(k.beta);
      k.rz = rzn;
      any = true;
    }
  any = __syncthreads_or(any ? 1 : 0) != 0;
  if (threadIdx.x == 0) set_cond(cond, any);
}

// one thread per free support node: u += coef * sum_e W[ent] G[point(ent)]
__global__ void k_ib_spread(int64_t n, const int32_t* __restrict__ n_dev, const int32_t* __restrict__ sp_slot,
                            const int32_t* __restrict__ sp_off, const int32_t* __restrict__ sp_ent,
                            const double* __restrict__ W, const double* __restrict__ G,
                            const int32_t* __restrict__ binst, const double* __restrict__ icoef,
                            double* __restrict__ u, int64_t nslots) {
  KCOUNT();
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= (n_dev ? int64_t(*n_dev) : n)) return;
  double acc[3] = {0, 0, 0};
  for (int e = sp_off[j]; e < sp_off[j + 1]; ++e) {
    const int32_t ent = sp_ent[e];
    const double w = W[ent];
    const int64_t i = ent >> 6;
    for (int c = 0; c < 3; ++c) acc[c] += w * G[3 * i + c];
  }
  const int32_t s = sp_slot[j];
  const double coef = icoef[binst[s >> 9]];
  for (int c = 0; c < 3; ++c) u[c * nslots + s] += coef * acc[c];
}

// ---------------------------------------------------------------- host wrappers
void ib_weights(const IBDev& ib, cudaStream_t st) {
  if (ib.M == 0) return;
  const int64_t n = ib.M * 64;
  IBG_LAUNCH(k_ib_weights, int((n + 255) / 256), 256, 0, st, ib.M, ib.X, ib.org, ib.slot, ib.pinst, ib.iorigin,
             ib.ihf, ib.W);
}

void ib_assemble(const IBDev& ib, cudaStream_t st) {
  if (ib.M == 0) return;
  const int64_t th = ib.M * 32;
  IBG_LAUNCH(k_af_values, int((th + 255) / 256), 256, 0, st, ib.M, ib.rowptr, ib.col, ib.org, ib.freeb, ib.W,
             ib.pscale, ib.val, ib.dinv, ib.val32, ib.dinv32);
}

void ib_gather(const IBDev& ib, const double* u, int64_t nslots, const double* UB, double* BF, cudaStream_t st) {
  if (ib.M == 0) return;
  const int64_t th = ib.M * 32;
  IBG_LAUNCH(k_ib_gather, int((th + 255) / 256), 256, 0, st, ib.M, ib.slot, ib.W, u, nslots, UB, BF);
}

cudaError_t ib_solve(const IBDev& ib, const double* BF, double* G, double* work, KState* ks, KState* ks_host,
                     RedBuf rb, double rtol, int max_iter, SolveRec* rec, cudaStream_t st, CaptureCtx* cc) {
  if (ib.M == 0) return cudaSuccess;
  const int64_t L = 3 * ib.M;
  double *r = work, *z = work + L, *p = work + 2 * L, *q = work + 3 * L;
  IBG_LAUNCH(k_init_states, (ib.ninst * 3 + 127) / 128, 128, 0, st, ks, ib.ninst * 3, rtol * rtol, max_iter);
  Cond cond;
  if (cc && cc->capturing) {
    cudaError_t e = cond_handle(st, 0, &cond);
    if (e != cudaSuccess) return e;
  }
  const int gw = int((ib.M * 32 + IBB - 1) / IBB);   // warp-per-row grids
  const int gt = int((ib.M + IBB - 1) / IBB);        // thread-per-row grids
  IBG_LAUNCH(k_af_apply, gw, IBB, 0, st, ib, G, q, 0, ks, rb.partials, rb.counter);
  IBG_LAUNCH((k_af_start<double>), gt, IBB, 0, st, ib, ib.dinv, BF, (const double*)q, r, z, p, ks, rb.partials,
             rb.counter, cond, (const OState*)nullptr);
  // k_af_start left p = z and beta = 0; the direction ping-pongs between p and
  // p2, two iterations per loop body
  double* p2 = work + 4 * L;
  const int g8 = int((ib.M * AFL + IBB - 1) / IBB);
  auto iter = [&](cudaStream_t s, const Cond& c, const double* pold, double* pnew) {
    IBG_LAUNCH((k_af_apply_p<double>), g8, IBB, 0, s, ib, (const double*)ib.val, (const double*)z, pold, pnew, q,
               ks, rb.partials, rb.counter);
    IBG_LAUNCH((k_af_update<double>), gt, IBB, 0, s, ib, ib.dinv, G, r, z, (const double*)pnew, (const double*)q,
               ks, rb.partials, rb.counter, c);
  };
  cudaError_t e = run_loop(cc, st, cond, ks, ks_host, ib.ninst * 3, max_iter, 4, 32,
                           [&](cudaStream_t s, const Cond& c) {
    iter(s, c, p, p2);
    iter(s, c, p2, p);
  });
  if (e != cudaSuccess) return e;
  IBG_LAUNCH(k_collect, (ib.ninst + 127) / 128, 128, 0, st, ks, 3, ib.ninst, rec, (OState*)nullptr);
  return cudaSuccess;
}

// ---------------------------------------------------------------- mixed precision
// FP64 outer loop of the mixed force solve: r = B_F - S G on every row, FP64
// norms per instance and component, r rounded to FP32 as the inner right-hand
// side with a zero inner guess; the loop and branch conditions as for the
// field solves (converged, stagnated near the FP64 floor, or out of passes).
__global__ void __launch_bounds__(IBB) k_af_resid_outer(IBDev ib, const double* __restrict__ b,
                                                        const double* __restrict__ y, float* __restrict__ r32,
                                                        float* __restrict__ e32, OState* os, double* partials,
                                                        unsigned* counter, Cond cloop, Cond cbranch) {
  KCOUNT();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double w[6] = {0, 0, 0, 0, 0, 0};
  if (i < ib.M) {
    const OState& oi = os[ib.pinst[i]];
    for (int c = 0; c < 3; ++c) {
      const double rv = b[3 * i + c] - y[3 * i + c];
      r32[3 * i + c] = float(rv);
      e32[3 * i + c] = 0.f;
      w[2 * c] = rv * rv;
      w[2 * c + 1] = oi.iter == 0 ? b[3 * i + c] * b[3 * i + c] : 0.0;
    }
  }
  double* out = partials + (int64_t)gridDim.x * 6;
  if (!grid_sum_last<double, 6>(w, partials, counter, ib.seg_t, ib.ninst, out)) return;
  bool any = false;
  for (int n = threadIdx.x; n < ib.ninst; n += blockDim.x) {
    OState& o = os[n];
    if (o.done) continue;
    double rel2 = 0.0;
    bool finite = true;
    for (int c = 0; c < 3; ++c) {
      const double rr = out[n * 6 + 2 * c], bb = out[n * 6 + 2 * c + 1];
      if (o.iter == 0) o.ref[c] = fmax(bb, rr);
      if (!isfinite(rr)) finite = false;
      if (o.ref[c] > 0.0) rel2 = fmax(rel2, rr / o.ref[c]);
    }
    o.rel2 = rel2;
    const bool stagnated = o.iter > 0 && rel2 > 0.0625 * o.prev2 && rel2 <= 1e6 * o.tol2;
    // An FP32 inner breakdown (A_F can be too ill-conditioned for FP32 when
    // the points are denser than the grid, Sec. 2.5) ends that pass with the
    // correction it has built; the FP64 loop goes on while every such pass
    // still reduces the residual by 4x.
    const bool inner_stuck = o.inner_status == 5 && !(rel2 < 0.0625 * o.prev2);
    if (!finite || (inner_stuck && !(rel2 <= o.tol2))) { o.done = 1; o.status = 5; }
    else if (rel2 <= o.tol2 || stagnated) o.done = 1;
    else if (o.iter >= o.max_iter) { o.done = 1; o.status = 4; }
    o.prev2 = rel2;
    o.inner_status = 0;
    if (!o.done) { o.iter++; any = true; }
  }
  any = __syncthreads_or(any ? 1 : 0) != 0;
  if (threadIdx.x == 0) {
    set_cond(cloop, any);
    set_cond(cbranch, any);
  }
}

// G += e for the instances whose outer loop is still running
__global__ void k_af_add(IBDev ib, const float* __restrict__ e, double* __restrict__ G, const OState* os) {
  KCOUNT();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= ib.M || os[ib.pinst[i]].done) return;
  for (int c = 0; c < 3; ++c) G[3 * i + c] += double(e[3 * i + c]);
}

cudaError_t ib_solve_mixed(const IBDev& ib, const double* BF, double* G, double* y64, float* w32, KState* ks,
                           KState* ks_host, OState* os, OState* os_host, RedBuf rb, double rtol, double rtol_inner,
                           int max_iter, int max_outer, SolveRec* rec, cudaStream_t st, CaptureCtx* cc) {
  if (ib.M == 0) return cudaSuccess;
  const int64_t L = 3 * ib.M;
  float *r32 = w32, *e32 = w32 + L, *r = w32 + 2 * L, *z = w32 + 3 * L, *pa = w32 + 4 * L, *pb = w32 + 5 * L,
        *q = w32 + 6 * L;
  const int gw = int((ib.M * 32 + IBB - 1) / IBB);
  const int gt = int((ib.M + IBB - 1) / IBB);
  const int g8 = int((ib.M * AFL + IBB - 1) / IBB);
  const int gi = (ib.ninst + 127) / 128;
  IBG_LAUNCH(k_init_outer, gi, 128, 0, st, os, ib.ninst, 3, rtol * rtol, max_outer);
  auto residual = [&](cudaStream_t s, const Cond& cl, const Cond& cb) {
    IBG_LAUNCH(k_af_apply, gw, IBB, 0, s, ib, (const double*)G, y64, 0, ks, rb.partials, rb.counter);
    IBG_LAUNCH(k_af_resid_outer, gt, IBB, 0, s, ib, BF, (const double*)y64, r32, e32, os, rb.partials, rb.counter,
               cl, cb);
  };
  cudaError_t err = cudaSuccess;
  auto correction = [&](cudaStream_t s) {
    IBG_LAUNCH(k_init_states, (ib.ninst * 3 + 127) / 128, 128, 0, s, ks, ib.ninst * 3, rtol_inner * rtol_inner,
               max_iter);
    Cond ci;
    if (cc && cc->capturing) {
      cudaError_t e = cond_handle(s, 0, &ci);
      if (e != cudaSuccess) return e;
    }
    IBG_LAUNCH((k_af_start<float>), gt, IBB, 0, s, ib, (const float*)ib.dinv32, (const float*)r32,
               (const float*)nullptr, r, z, pa, ks, rb.partials, rb.counter, ci, (const OState*)os);
    auto iter = [&](cudaStream_t s2, const Cond& c2, const float* pold, float* pnew) {
      IBG_LAUNCH((k_af_apply_p<float>), g8, IBB, 0, s2, ib, (const float*)ib.val32, (const float*)z, pold, pnew, q,
                 ks, rb.partials, rb.counter);
      IBG_LAUNCH((k_af_update<float>), gt, IBB, 0, s2, ib, (const float*)ib.dinv32, e32, r, z, (const float*)pnew,
                 (const float*)q, ks, rb.partials, rb.counter, c2);
    };
    cudaError_t e = run_loop(cc, s, ci, ks, ks_host, ib.ninst * 3, max_iter, 4, 32, [&](cudaStream_t s2, const Cond& c2) {
      iter(s2, c2, pa, pb);
      iter(s2, c2, pb, pa);
    });
    if (e != cudaSuccess) return e;
    IBG_LAUNCH(k_collect, gi, 128, 0, s, (const KState*)ks, 3, ib.ninst, rec, os);
    IBG_LAUNCH(k_af_add, gt, IBB, 0, s, ib, (const float*)e32, G, (const OState*)os);
    return cudaSuccess;
  };
  if (cc && cc->capturing) {
    Cond cl;
    if ((err = cond_handle(st, 1, &cl)) != cudaSuccess) return err;
    cudaError_t e = cond_node(*cc, st, cl, cudaGraphCondTypeWhile, [&](cudaStream_t s) {
      Cond cb;
      cudaError_t e1 = cond_handle(s, 0, &cb);
      if (e1 != cudaSuccess) { err = e1; return; }
      residual(s, cl, cb);
      e1 = cond_node(*cc, s, cb, cudaGraphCondTypeIf, [&](cudaStream_t s2) {
        cudaError_t e2 = correction(s2);
        if (e2 != cudaSuccess) err = e2;
      });
      if (e1 != cudaSuccess) err = e1;
    });
    if (e != cudaSuccess) return e;
    if (err != cudaSuccess) return err;
  } else {
    const Cond none;
    for (int it = 0; it <= max_outer + 1; ++it) {
      residual(st, none, none);
      cudaMemcpyAsync(os_host, os, ib.ninst * sizeof(OState), cudaMemcpyDeviceToHost, st);
      if ((err = cudaStreamSynchronize(st)) != cudaSuccess) return err;
      bool all = true;
      for (int i = 0; i < ib.ninst; ++i) all = all && os_host[i].done;
      if (all) break;
      if ((err = correction(st)) != cudaSuccess) return err;
    }
  }
  IBG_LAUNCH(k_collect_outer, gi, 128, 0, st, (const OState*)os, ib.ninst, rec);
  return cudaSuccess;
}

// Condition of the FP64 fallback: some instance's mixed force solve failed;
// the records of those instances are cleared for the fallback's own status.
__global__ void k_af_failed(const OState* os, int ninst, SolveRec* rec, Cond cond) {
  KCOUNT();
  bool any = false;
  for (int i = threadIdx.x; i < ninst; i += blockDim.x)
    if (os[i].status != 0) {
      any = true;
      rec[i * 4].status = 0;
    }
  any = __syncthreads_or(any ? 1 : 0) != 0;
  if (threadIdx.x == 0) set_cond(cond, any);
}

cudaError_t ib_fp64_fallback(const IBDev& ib, const double* BF, double* G, double* work, KState* ks,
                             KState* ks_host, const OState* os, OState* os_host, RedBuf rb, double rtol, int max_iter,
                             SolveRec* rec, cudaStream_t st, CaptureCtx* cc) {
  if (ib.M == 0) return cudaSuccess;
  if (cc && cc->capturing) {
    Cond cf;
    cudaError_t e = cond_handle(st, 0, &cf);
    if (e != cudaSuccess) return e;
    IBG_LAUNCH(k_af_failed, 1, 128, 0, st, os, ib.ninst, rec, cf);
    cudaError_t err = cudaSuccess;
    e = cond_node(*cc, st, cf, cudaGraphCondTypeIf, [&](cudaStream_t s) {
      err = ib_solve(ib, BF, G, work, ks, ks_host, rb, rtol, max_iter, rec, s, cc);
    });
    return e != cudaSuccess ? e : err;
  }
  cudaMemcpyAsync(os_host, os, ib.ninst * sizeof(OState), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  bool any = false;
  for (int i = 0; i < ib.ninst; ++i) any = any || os_host[i].status != 0;
  if (!any) return cudaSuccess;
  IBG_LAUNCH(k_af_failed, 1, 128, 0, st, os, ib.ninst, rec, Cond());
  return ib_solve(ib, BF, G, work, ks, ks_host, rb, rtol, max_iter, rec, st, cc);
}

void ib_spread(const IBDev& ib, const double* G, double* u, int64_t nslots, cudaStream_t st) {
  const int64_t n = ib.n_sp_dev ? ib.sp_cap : ib.n_sp;
  if (n == 0) return;
  IBG_LAUNCH(k_ib_spread, int((n + 255) / 256), 256, 0, st, ib.n_sp, ib.n_sp_dev, ib.sp_slot, ib.sp_off, ib.sp_ent,
             ib.W, G, ib.binst, ib.icoef, u, nslots);
}

}  // namespace ibg
