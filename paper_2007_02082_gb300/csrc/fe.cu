// Matrix-free P1 operators on the brick-stored composite grid, and the Krylov
// solvers of the IPCS step (Sec. 2.2, Eq. 9 and Eq. 12; velocity correction).
//
// Every operator is applied per level on the level's own node lattice: one CTA
// per 8x8x8-node brick stages the brick plus a one-node halo in shared memory
// and every thread produces one node's row.  The constrained (hanging-node)
// operator P^T (sum_l A_l) P is completed by fe_sync (sum of the two stored
// copies of an interface node plus half of each hanging child) and fe_expand
// (hanging value = mean of parents).  Inner products run in FP64 with a fixed
// reduction order (block partials, then one block sums them in block order), so
// results are bitwise reproducible.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "async.cuh"
#include "ff.cuh"
#include "fe.hpp"
#include "kuhn_weights.hpp"

namespace ibg {

IBG_KCOUNT_DEFINE
unsigned long long fe_kcount() {
  unsigned long long v = 0;
  cudaMemcpyFromSymbol(&v, g_kcount, sizeof(v));
  return v;
}

std::atomic<long long> g_launches{0};

// ---------------------------------------------------------------- tables
__constant__ int8_t c_sten[15][3];
__constant__ int16_t c_toff[15];               // tile offset of each stencil slot
__constant__ int8_t c_slot_of_rel[27];

static const int8_t h_sten[15][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                                     {0, 0, 1},  {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {0, 1, 1},
                                     {0, -1, -1}, {1, 0, 1}, {-1, 0, -1}, {1, 1, 1},  {-1, -1, -1}};

cudaError_t fe_init_tables() {
  int8_t slot_of_rel[27];
  std::memset(slot_of_rel, -1, sizeof(slot_of_rel));
  int16_t toff[15];
  for (int k = 0; k < 15; ++k) {
    slot_of_rel[(h_sten[k][2] + 1) * 9 + (h_sten[k][1] + 1) * 3 + (h_sten[k][0] + 1)] = int8_t(k);
    toff[k] = int16_t((h_sten[k][2] * TILE + h_sten[k][1]) * TILE + h_sten[k][0]);
  }
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_sten, h_sten, sizeof(h_sten))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_toff, toff, sizeof(toff))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_slot_of_rel, slot_of_rel, sizeof(slot_of_rel))) != cudaSuccess) return e;
  return cudaSuccess;
}

// ---------------------------------------------------------------- helpers
// Gradient couplings of a node (kuhn_weights.hpp); k and a are compile-time
// after unrolling, so each is a short sum of mask bits.
__device__ __forceinline__ void grad_weights(int mask, int (&gw)[15][3]) {
#pragma unroll
  for (int k = 0; k < 15; ++k)
#pragma unroll
    for (int a = 0; a < 3; ++a) gw[k][a] = grad_weight(mask, k, a);
}

// Warp-uniform dispatch on the incident-cell mask.  Where every lane's eight
// incident cells are active (the bulk of a grid) the body runs with the mask as
// a compile-time constant: every closed-form weight folds to a constant, zero
// couplings drop out, and no integer weight is converted at run time (a
// conversion to FP64 costs as much as an FP64 FMA).  Elsewhere the body runs
// with the runtime mask.  Every lane of the warp must call it.
struct FullMask {
  __host__ __device__ constexpr operator int() const { return 0xFF; }
};
template <typename Body>
__device__ __forceinline__ void with_mask(int mask, Body&& body) {
  if (__all_sync(0xffffffffu, mask == 0xFF)) body(FullMask{});
  else body(mask);
}
// A small integer weight (|w| < 2^20) as T.  For FP64 the IEEE-754 bits are
// built with 32-bit integer operations (sign, the exponent from the leading
// bit, the mantissa below it in the high word, a zero low word): exact, and it
// keeps the conversion off the FP64 pipe, which issues at a small fraction of
// the FP32 and integer rates on this GPU.
template <typename T>
__device__ __forceinline__ T wconv(int w) {
  if constexpr (sizeof(T) == 8) {
    const unsigned a = unsigned(w < 0 ? -w : w);
    const int e = 31 - __clz(a);   // a in [2^e, 2^(e+1)) for a > 0
    const unsigned hi = (unsigned(1023 + e) << 20) | ((a << ((20 - e) & 31)) & 0xFFFFFu) | (w < 0 ? 0x80000000u : 0u);
    return __hiloint2double(a ? int(hi) : 0, 0);
  } else {
    return T(w);
  }
}

// true when the mask argument of a with_mask body is the compile-time constant
template <typename MK>
__device__ __forceinline__ constexpr bool const_mask() {
  return !std::is_same_v<std::decay_t<MK>, int>;
}

// Symmetric viscous form: out_i += dt nu sum_k sum_j F_ij w(mask, k, i, j)
// x_j(neighbour k), the transpose-gradient couplings (grad u^T, grad v) per
// Kuhn tetrahedron (kuhn_weights.hpp), F_ij = (V/6)/(h_i h_j) from the
// stencil factors.  xk(k, v) loads the three components at neighbour k.
template <typename T, typename MK, typename XK>
__device__ __forceinline__ void add_transpose(MK mk, const T* F, T dtnu, XK&& xk, T (&out)[3]) {
  T acc[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) acc[i][j] = T(0);
#pragma unroll
  for (int k = 0; k < 15; ++k) {
    T v[3];
    xk(k, v);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int w = trans_weight(mk, k, i, j);
        if (!const_mask<MK>() || w != 0) acc[i][j] += wconv<T>(w) * v[j];
      }
  }
  const T fij[3][3] = {{F[0], F[8], F[10]}, {F[8], F[1], F[9]}, {F[10], F[9], F[2]}};
#pragma unroll
  for (int i = 0; i < 3; ++i) out[i] += dtnu * (fij[i][0] * acc[i][0] + fij[i][1] * acc[i][1] + fij[i][2] * acc[i][2]);
}

__device__ __forceinline__ void spacing(const DevGrid& g, int b, double (&h)[3]) {
  const int inst = g.binst[b], lev = g.blev[b];
  const double* p = g.hl + (inst * 4 + lev) * 3;
  h[0] = p[0];
  h[1] = p[1];
  h[2] = p[2];
}
__device__ __forceinline__ bool is_dof(uint16_t m, uint16_t dmask) {
  return (m & D_VALID) && !(m & (D_HANG | D_DUP | dmask));
}

enum Post : int { POST_NONE = 0, POST_CG_ALPHA = 1 };

// Interface sum of an operator output: both stored copies get the sum of their
// level parts plus half of each hanging child's; rows with a dmask bit are zeroed.
// The indices are loaded once and every component's values together, so one
// entry costs three dependent loads (indices, values and children's slots,
// children's values) whatever NC is.
template <typename T, int NC>
__global__ void k_sync(DevGrid g, T* __restrict__ y, uint16_t dmask) {
  KCOUNT();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.n_if) return;
  const int32_t sc = g.if_c[e], sf = g.if_f[e];
  const int32_t k0 = g.if_off[e], k1 = g.if_off[e + 1];
  const uint16_t mc = g.meta[sc];
  const bool zero = (mc & dmask) != 0;
  T tot[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) tot[c] = y[c * g.nslots + sc] + y[c * g.nslots + sf];
  for (int k = k0; k < k1; ++k) {
    const int32_t kid = g.if_kid[k];
#pragma unroll
    for (int c = 0; c < NC; ++c) tot[c] += T(0.5) * y[c * g.nslots + kid];
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const T v = (zero || (NC == 3 && tan_dir(mc, dmask, c))) ? T(0) : tot[c];
    y[c * g.nslots + sc] = v;
    y[c * g.nslots + sf] = v;
  }
}

template <typename T, int NC>
__global__ void k_expand(DevGrid g, T* __restrict__ x, T* __restrict__ x2) {
  KCOUNT();
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= g.n_hang) return;
  const int32_t s = g.hg[h], p1 = g.hp1[h], p2 = g.hp2[h];
  for (int c = 0; c < NC; ++c) {
    T* xc = x + c * g.nslots;
    xc[s] = T(0.5) * (xc[p1] + xc[p2]);
    if (x2) {
      T* x2c = x2 + c * g.nslots;
      x2c[s] = T(0.5) * (x2c[p1] + x2c[p2]);
    }
  }
}

// ---------------------------------------------------------------- Jacobi
template <typename T, int OP>
__global__ void __launch_bounds__(512) k_diag(DevGrid g, const T* __restrict__ coef, T* __restrict__ diag) {
  KCOUNT();
  const int64_t s = (int64_t)blockIdx.x * DBV + threadIdx.x;
  const uint16_t m = g.meta[s];
  // FP32 momentum coefficients are stored compactly (valid slots only)
  constexpr bool compact = OP != OP_POISSON && OP != OP_MASS && sizeof(T) == 4;
  const int64_t ci = compact ? compact_index(g, blockIdx.x, threadIdx.x, (m & D_VALID) != 0) : s;
  T d = T(0);
  if (m & D_VALID) {
    const T* F = stencil_factors<T>(g, blockIdx.x);
    const int mask = m & 0xFF;
    if (OP == OP_POISSON)
      d = T(stiff_edge_count(mask, 0, 1) + stiff_edge_count(mask, 0, -1)) * F[0] +
          T(stiff_edge_count(mask, 1, 1) + stiff_edge_count(mask, 1, -1)) * F[1] +
          T(stiff_edge_count(mask, 2, 1) + stiff_edge_count(mask, 2, -1)) * F[2];
    else if (OP == OP_MASS) d = T(mass_weight(mask, 0)) * F[3];
    else d = coef[ci];
  }
  diag[s] = d;
}

template <typename T>
__global__ void __launch_bounds__(512) k_dinv(DevGrid g, const T* __restrict__ diag, T* __restrict__ dinv,
                                              uint16_t dmask) {
  KCOUNT();
  const int64_t s = (int64_t)blockIdx.x * DBV + threadIdx.x;
  const uint16_t m = g.meta[s];
  const bool keep = (m & D_VALID) && !(m & (D_HANG | dmask));
  dinv[s] = (keep && diag[s] != T(0)) ? T(1) / diag[s] : T(0);
}

// ---------------------------------------------------------------- tet-loop kernels (FP64)
// out_c = (M u_c) - dt (G_c p), both from the mask tables:
//   M u_c = V/120 sum_k massw[k] u_c(k),  (G_c p) = (V/24)/h_c sum_k gradw[k][c] p(k)
__global__ void __launch_bounds__(512) k_rhs_mass_grad(DevGrid g, const double* __restrict__ u,
                                                       const double* __restrict__ p, double* __restrict__ out) {
  KCOUNT();
  __shared__ double tile[4 * TILE3];
  const int b = blockIdx.x;
  load_tile<double>(tile, u, g.nslots, 3, g.bnbr + 27 * b);
  load_tile<double>(tile + 3 * TILE3, p, g.nslots, 1, g.bnbr + 27 * b);
  __syncthreads();
  const int t = threadIdx.x;
  const int64_t s = (int64_t)b * DBV + t;
  const uint16_t m = g.meta[s];
  const bool valid = (m & D_VALID) != 0;
  double o[3] = {0, 0, 0};
  with_mask(valid ? (m & 0xFF) : 0, [&](auto mk) {
    if (!valid) return;
    const int ti = tile_index(t & 7, (t >> 3) & 7, t >> 6);
    const double* F = stencil_factors<double>(g, b);
    const double dt = g.pdt[g.binst[b]];
    double gp[3] = {0, 0, 0};
#pragma unroll
    for (int k = 0; k < 15; ++k) {
      const int j = ti + c_toff[k];
      const int mw = mass_weight(mk, k);
      const double pk = tile[3 * TILE3 + j];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (!const_mask<decltype(mk)>() || mw != 0) o[a] += wconv<double>(mw) * tile[a * TILE3 + j];
        const int gw = grad_weight(mk, k, a);
        if (!const_mask<decltype(mk)>() || gw != 0) gp[a] += wconv<double>(gw) * pk;
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) o[a] = F[3] * o[a] - dt * F[4 + a] * gp[a];
  });
  for (int a = 0; a < 3; ++a) out[a * g.nslots + s] = o[a];
}

// out = -(1/dt) (div u, q) = -(1/dt) sum_c (V/24)/h_c sum_k gradw[k][c] u_c(k)
__global__ void __launch_bounds__(512) k_rhs_div(DevGrid g, const double* __restrict__ u, double* __restrict__ out) {
  KCOUNT();
  __shared__ double tile[3 * TILE3];
  const int b = blockIdx.x;
  load_tile<double>(tile, u, g.nslots, 3, g.bnbr + 27 * b);
  __syncthreads();
  const int t = threadIdx.x;
  const int64_t s = (int64_t)b * DBV + t;
  const uint16_t m = g.meta[s];
  const bool valid = (m & D_VALID) != 0;
  double o = 0.0;
  with_mask(valid ? (m & 0xFF) : 0, [&](auto mk) {
    if (!valid) return;
    const int ti = tile_index(t & 7, (t >> 3) & 7, t >> 6);
    const double* F = stencil_factors<double>(g, b);
    double d[3] = {0, 0, 0};
#pragma unroll
    for (int k = 0; k < 15; ++k) {
      const int j = ti + c_toff[k];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int gw = grad_weight(mk, k, a);
        if (!const_mask<decltype(mk)>() || gw != 0) d[a] += wconv<double>(gw) * tile[a * TILE3 + j];
      }
    }
    o = F[4] * d[0] + F[5] * d[1] + F[6] * d[2];
  });
  out[s] = -o / g.pdt[g.binst[b]];
}

// ---------------------------------------------------------------- FP64-accurate sums in FP32 pairs
// The mixed path's right-hand sides (Eq. 9, Eq. 12, the velocity correction)
// and the operator products of its FP64 outer residuals, with FP64 inputs and
// outputs and the stencil sums carried in double-FP32 (ff.cuh): every node
// value is split once into a pair when its tile is loaded, integer weights
// multiply exactly, and each partial sum keeps its rounding errors, so a sum
// is accurate to about 2^-44 of the sum of its terms' magnitudes.  Where the
// weights sum to zero (gradient, divergence, stiffness) the sums run over
// differences to the node's own value, formed exactly (ff_diff), so the result
// keeps that accuracy relative to itself rather than to the node values.
// The FP64 path keeps the FP64 kernels above.

// tile of ncomp FP64 components as FP32 pairs; missing neighbours read as zero
__device__ __forceinline__ void load_tile_ff(ff* tile, const double* __restrict__ x, int64_t cs, int ncomp,
                                             const int32_t* __restrict__ nb27) {
  for (int t = threadIdx.x; t < TILE3; t += blockDim.x) {
    const int hx = t % TILE, hy = (t / TILE) % TILE, hz = t / (TILE * TILE);
    const int lx = hx - 1, ly = hy - 1, lz = hz - 1;
    const int ox = lx < 0 ? -1 : (lx > 7 ? 1 : 0), oy = ly < 0 ? -1 : (ly > 7 ? 1 : 0);
    const int oz = lz < 0 ? -1 : (lz > 7 ? 1 : 0);
    const int nb = nb27[(oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)];
    const int64_t s = (int64_t)nb * DBV + (((lz & 7) * DBS + (ly & 7)) * DBS + (lx & 7));
    for (int c = 0; c < ncomp; ++c) tile[c * TILE3 + t] = nb >= 0 ? dsplit(x[c * cs + s]) : ff{0.f, 0.f};
  }
}

// per-CTA constants as pairs: F[3] (V/120) and dt F[4 + a] ((V/24)/h_a dt)
__device__ __forceinline__ void ff_brick_factors(const DevGrid& g, int b, ff* sf) {
  if (threadIdx.x < 4) {
    const double* F = stencil_factors<double>(g, b);
    const double dt = g.pdt[g.binst[b]];
    sf[threadIdx.x] = dsplit(threadIdx.x == 0 ? F[3] : dt * F[3 + threadIdx.x]);
  }
}

// out_c = M u_c - dt G_c p (k_rhs_mass_grad's operation)
__global__ void __launch_bounds__(512) k_rhs_mass_grad_ff(DevGrid g, const double* __restrict__ u,
                                                          const double* __restrict__ p, double* __restrict__ out) {
  KCOUNT();
  __shared__ ff tile[4 * TILE3];
  __shared__ ff sf[4];
  const int b = blockIdx.x;
  load_tile_ff(tile, u, g.nslots, 3, g.bnbr + 27 * b);
  load_tile_ff(tile + 3 * TILE3, p, g.nslots, 1, g.bnbr + 27 * b);
  ff_brick_factors(g, b, sf);
  __syncthreads();
  const int t = threadIdx.x;
  const int64_t s = (int64_t)b * DBV + t;
  const uint16_t m = g.meta[s];
  const bool valid = (m & D_VALID) != 0;
  double o[3] = {0, 0, 0};
  with_mask(valid ? (m & 0xFF) : 0, [&](auto mk) {
    if (!valid) return;
    const int ti = tile_index(t & 7, (t >> 3) & 7, t >> 6);
    ff ms[3], gp[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) ms[a] = gp[a] = ff{0.f, 0.f};
    const ff p0 = tile[3 * TILE3 + ti];
#pragma unroll
    for (int k = 0; k < 15; ++k) {
      const int j = ti + c_toff[k];
      const int mw = mass_weight(mk, k);
      if (!const_mask<decltype(mk)>() || mw != 0)
#pragma unroll
        for (int a = 0; a < 3; ++a) ff_madd_int(ms[a], wf(mw), tile[a * TILE3 + j]);
      if (k == 0) continue;   // the gradient weights sum to zero: differences to p at the node
      const ff dp = ff_diff(tile[3 * TILE3 + j], p0);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int gw = grad_weight(mk, k, a);
        if (!const_mask<decltype(mk)>() || gw != 0) ff_madd_int(gp[a], wf(gw), dp);
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) o[a] = ff2d(ff_add(ff_mul(ms[a], sf[0]), ff_neg(ff_mul(gp[a], sf[1 + a]))));
  });
  for (int a = 0; a < 3; ++a) out[a * g.nslots + s] = o[a];
}

// out = -(1/dt) (div u, q) (k_rhs_div's operation)
__global__ void __launch_bounds__(512, 3) k_rhs_div_ff(DevGrid g, const double* __restrict__ u,
                                                    double* __restrict__ out) {
  KCOUNT();
  __shared__ ff tile[3 * TILE3];
  __shared__ ff sf[4];
  const int b = blockIdx.x;
  load_tile_ff(tile, u, g.nslots, 3, g.bnbr + 27 * b);
  if (threadIdx.x < 3) {
    // (V/24)/h_a / dt as a pair
    const double* F = stencil_factors<double>(g, b);
    sf[threadIdx.x] = dsplit(F[4 + threadIdx.x] / g.pdt[g.binst[b]]);
  }
  __syncthreads();
  const int t = threadIdx.x;
  const int64_t s = (int64_t)b * DBV + t;
  const uint16_t m = g.meta[s];
  const bool valid = (m & D_VALID) != 0;
  double o = 0.0;
  with_mask(valid ? (m & 0xFF) : 0, [&](auto mk) {
    if (!valid) return;
    const int ti = tile_index(t & 7, (t >> 3) & 7, t >> 6);
    ff d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = ff{0.f, 0.f};
#pragma unroll
    for (int k = 1; k < 15; ++k) {   // zero-sum weights: differences to the node's own value
      const int j = ti + c_toff[k];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int gw = grad_weight(mk, k, a);
        if (!const_mask<decltype(mk)>() || gw != 0)
          ff_madd_int(d[a], wf(gw), ff_diff(tile[a * TILE3 + j], tile[a * TILE3 + ti]));
      }
    }
    o = -ff2d(ff_add(ff_add(ff_mul(d[0], sf[0]), ff_mul(d[1], sf[1])), ff_mul(d[2], sf[2])));
  });
  out[s] = o;
}

// Residual operator products of the mixed path, one CTA per brick:
//   OP_MASS:    y_c = M x_c (3 components)
//   OP_COEF:    y_c = sum_k coef_k x_c(k), the coefficients as compact FP32 pairs
//               (k_mom_coef_ff; momentum, gradient form)
//   OP_POISSON: y = K x (7-point)
// Rows with the dmask flag give zero; brick padding is not written.
template <int OP>
__global__ void __launch_bounds__(512) k_apply_ff(DevGrid g, const double* __restrict__ x, double* __restrict__ y,
                                                  const float* __restrict__ chi, const float* __restrict__ clo,
                                                  uint16_t dmask) {
  KCOUNT();
  constexpr int NC = OP == OP_POISSON ? 1 : 3;
  __shared__ ff tile[NC * TILE3];
  __shared__ ff sf[4];
  const int b = blockIdx.x;
  load_tile_ff(tile, x, g.nslots, NC, g.bnbr + 27 * b);
  if (threadIdx.x < 4) {
    const double* F = stencil_factors<double>(g, b);
    sf[threadIdx.x] = dsplit(OP == OP_POISSON ? F[threadIdx.x] : F[3]);
  }
  __syncthreads();
  const int t = threadIdx.x;
  const int64_t s = (int64_t)b * DBV + t;
  const uint16_t m = g.meta[s];
  const bool act = (m & D_VALID) && !(m & dmask);
  double o[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) o[c] = 0.0;
  const int ti = tile_index(t & 7, (t >> 3) & 7, t >> 6);
  if constexpr (OP == OP_COEF) {
    const int64_t ci = compact_index(g, b, t, (m & D_VALID) != 0);
    if (act) {
      ff acc[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[c] = ff{0.f, 0.f};
#pragma unroll
      for (int k = 0; k < 15; ++k) {
        const ff ck{chi[(int64_t)k * g.ncomp + ci], clo[(int64_t)k * g.ncomp + ci]};
#pragma unroll
        for (int c = 0; c < 3; ++c) ff_madd(acc[c], ck, tile[c * TILE3 + ti + c_toff[k]]);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) o[c] = ff2d(acc[c]);
    }
  } else {
    with_mask(act ? (m & 0xFF) : 0, [&](auto mk) {
      if (!act) return;
      if constexpr (OP == OP_MASS) {
        ff acc[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[c] = ff{0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 15; ++k) {
          const int mw = mass_weight(mk, k);
          if (!const_mask<decltype(mk)>() || mw != 0)
#pragma unroll
            for (int c = 0; c < 3; ++c) ff_madd_int(acc[c], wf(mw), tile[c * TILE3 + ti + c_toff[k]]);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) o[c] = ff2d(ff_mul(acc[c], sf[0]));
      } else {
        // sum over the axes of (V/6)/h_a^2 (w_a+ (x - x_a+) + w_a- (x - x_a-))
        const ff x0 = tile[ti];
        ff tot{0.f, 0.f};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const int st = a == 0 ? 1 : a == 1 ? TILE : TILE * TILE;
          ff acc{0.f, 0.f};
          ff_madd_int(acc, wf(stiff_edge_count(mk, a, 1)), ff_diff(x0, tile[ti + st]));
          ff_madd_int(acc, wf(stiff_edge_count(mk, a, -1)), ff_diff(x0, tile[ti - st]));
          tot = ff_add(tot, ff_mul(acc, sf[a]));
        }
        o[0] = ff2d(tot);
      }
    });
  }
  if (m & D_VALID)
#pragma unroll
    for (int c = 0; c < NC; ++c) y[(int64_t)c * g.nslots + s] = o[c];
}

// Stencil slot of a neighbour offset (compile-time after unrolling).
__host__ __device__ constexpr int slot_of_rel(int rx, int ry, int rz) {
  return (rx == 0 && ry == 0 && rz == 0) ? 0
       : (rx == 1 && ry == 0 && rz == 0) ? 1 : (rx == -1 && ry == 0 && rz == 0) ? 2
       : (rx == 0 && ry == 1 && rz == 0) ? 3 : (rx == 0 && ry == -1 && rz == 0) ? 4
       : (rx == 0 && ry == 0 && rz == 1) ? 5 : (rx == 0 && ry == 0 && rz == -1) ? 6
       : (rx == 1 && ry == 1 && rz == 0) ? 7 : (rx == -1 && ry == -1 && rz == 0) ? 8
       : (rx == 0 && ry == 1 && rz == 1) ? 9 : (rx == 0 && ry == -1 && rz == -1) ? 10
       : (rx == 1 && ry == 0 && rz == 1) ? 11 : (rx == -1 && ry == 0 && rz == -1) ? 12
       : (rx == 1 && ry == 1 && rz == 1) ? 13 : (rx == -1 && ry == -1 && rz == -1) ? 14 : -1;
}

// dt C(u^n) row entries of a node: (u_h . grad phi_b, phi_a) on every
// tetrahedron holding the node, C_nb = sum_T (|T|/20) (S_T + u_n) . grad phi_b
// (S_T = sum of u over the tetrahedron's vertices), accumulated tetrahedron by
// tetrahedron with every index known at compile time.  tile: 3 components of
// u on the brick's 10^3 tile; wv = dt |T| / 20 = dt V / 120; ih = 1 / h.
template <typename CT, typename MK>
__device__ __forceinline__ void conv_coef(MK mask, const CT* tile, int ti, CT wv, CT ihx, CT ihy, CT ihz,
                                          CT (&cc)[15]) {
#pragma unroll
  for (int k = 0; k < 15; ++k) cc[k] = CT(0);
  const CT ih[3] = {ihx, ihy, ihz};
  const CT un[3] = {tile[ti], tile[TILE3 + ti], tile[2 * TILE3 + ti]};
  constexpr int KP[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (!((mask >> c) & 1)) continue;
    const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
    const int qb = (1 - dx) | ((1 - dy) << 1) | ((1 - dz) << 2);
#pragma unroll
    for (int p = 0; p < 6; ++p) {
      const int a1 = KP[p][0], a2 = KP[p][1], a3 = KP[p][2];
      const int vb[4] = {0, 1 << a1, (1 << a1) | (1 << a2), 7};
      if (qb != vb[0] && qb != vb[1] && qb != vb[2] && qb != vb[3]) continue;
      int off[4], sl[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int rx = dx - 1 + (vb[k] & 1), ry = dy - 1 + ((vb[k] >> 1) & 1), rz = dz - 1 + ((vb[k] >> 2) & 1);
        off[k] = (rz * TILE + ry) * TILE + rx;
        sl[k] = slot_of_rel(rx, ry, rz);
      }
      CT w[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const CT* ta = tile + a * TILE3 + ti;
        w[a] = wv * (ta[off[0]] + ta[off[1]] + ta[off[2]] + ta[off[3]] + un[a]);
      }
      // grad phi_0 = -e_a1/h, grad phi_1 = e_a1/h - e_a2/h, grad phi_2 = e_a2/h - e_a3/h, grad phi_3 = e_a3/h
      const CT g1 = w[a1] * ih[a1], g2 = w[a2] * ih[a2], g3 = w[a3] * ih[a3];
      cc[sl[0]] -= g1;
      cc[sl[1]] += g1 - g2;
      cc[sl[2]] += g2 - g3;
      cc[sl[3]] += g3;
    }
  }
}

// coef[k] = (M + dt C(u) + dt nu K) row entries (Eq. 9 operator), k over the
// 15 slots.  Mass and stiffness come from the mask tables, the convection
// entries from conv_coef.
template <typename CT>
__global__ void __launch_bounds__(512) k_mom_coef(DevGrid g, const double* __restrict__ u, double* __restrict__ coef,
                                                  float* __restrict__ coef32) {
  KCOUNT();
  __shared__ CT tile[3 * TILE3];
  const int b = blockIdx.x;
  {
    const int32_t* nb27 = g.bnbr + 27 * b;
    for (int t = threadIdx.x; t < TILE3; t += blockDim.x) {
      const int hx = t % TILE, hy = (t / TILE) % TILE, hz = t / (TILE * TILE);
      const int lx = hx - 1, ly = hy - 1, lz = hz - 1;
      const int ox = lx < 0 ? -1 : (lx > 7 ? 1 : 0), oy = ly < 0 ? -1 : (ly > 7 ? 1 : 0);
      const int oz = lz < 0 ? -1 : (lz > 7 ? 1 : 0);
      const int nb = nb27[(oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)];
      const int64_t sl = (int64_t)nb * DBV + (((lz & 7) * DBS + (ly & 7)) * DBS + (lx & 7));
      for (int c = 0; c < 3; ++c) tile[c * TILE3 + t] = nb >= 0 ? CT(u[c * g.nslots + sl]) : CT(0);
    }
  }
  __syncthreads();
  const int t = threadIdx.x;
  const int64_t s = (int64_t)b * DBV + t;
  const uint16_t m = g.meta[s];
  double cf[15];
#pragma unroll
  for (int k = 0; k < 15; ++k) cf[k] = 0.0;
  const bool valid = (m & D_VALID) != 0;
  with_mask(valid ? (m & 0xFF) : 0, [&](auto mask) {
    if (!valid) return;
    const int ti = tile_index(t & 7, (t >> 3) & 7, t >> 6);
    const double* F = stencil_factors<double>(g, b);
    const int inst = g.binst[b];
    const double dt = g.pdt[inst], nu = g.pnu[inst];
    double h[3];
    spacing(g, b, h);
    const double dnu = dt * nu;
    // M + dt nu K from the incident-cell mask (exact integer weights)
#pragma unroll
    for (int k = 0; k < 15; ++k) cf[k] = wconv<double>(mass_weight(mask, k)) * F[3];
    double diagK = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double kp = dnu * wconv<double>(stiff_edge_count(mask, a, 1)) * F[a];
      const double km = dnu * wconv<double>(stiff_edge_count(mask, a, -1)) * F[a];
      cf[1 + 2 * a] -= kp;
      cf[2 + 2 * a] -= km;
      diagK += kp + km;
    }
    cf[0] += diagK;
    // dt C(u^n), accumulated in CT (FP32 on the mixed path, FP64 on the FP64 path)
    CT cc[15];
    conv_coef<CT>(mask, tile, ti, CT(dt * F[3]), CT(1.0 / h[0]), CT(1.0 / h[1]), CT(1.0 / h[2]), cc);
#pragma unroll
    for (int k = 0; k < 15; ++k) cf[k] += double(cc[k]);
  });
  // FP32 copy in the compact layout (valid slots only) read by k_apply15_mom32
  const int64_t ci = coef32 ? compact_index(g, b, t, (m & D_VALID) != 0) : 0;
#pragma unroll
  for (int k = 0; k < 15; ++k) {
    coef[(int64_t)k * g.nslots + s] = cf[k];
    if (coef32 && (m & D_VALID)) coef32[(int64_t)k * g.ncomp + ci] = float(cf[k]);
  }
}

// The mixed path's momentum coefficients (gradient viscous form): the mass and
// stiffness parts as FP32 pairs from the FP64 stencil factors, the convection
// part in FP32 (conv_coef<float>, as k_mom_coef<float>), each sum kept as a
// pair and stored as two compact planes: hi (coef32, rounded to nearest: the
// FP32 operator of the inner iterations) and lo (coeflo), hi + lo within
// about 2^-44 of the coefficient, for the outer residual (k_apply_ff<OP_COEF>).
// Per-brick constants come from one thread; no FP64 arithmetic per node.
__global__ void __launch_bounds__(512) k_mom_coef_ff(DevGrid g, const double* __restrict__ u,
                                                     float* __restrict__ coef32, float* __restrict__ coeflo) {
  KCOUNT();
  __shared__ float tile[3 * TILE3];
  __shared__ ff sm3, sk[3];
  __shared__ float swv, sih[3];
  const int b = blockIdx.x;
  {
    const int32_t* nb27 = g.bnbr + 27 * b;
    for (int t = threadIdx.x; t < TILE3; t += blockDim.x) {
      const int hx = t % TILE, hy = (t / TILE) % TILE, hz = t / (TILE * TILE);
      const int lx = hx - 1, ly = hy - 1, lz = hz - 1;
      const int ox = lx < 0 ? -1 : (lx > 7 ? 1 : 0), oy = ly < 0 ? -1 : (ly > 7 ? 1 : 0);
      const int oz = lz < 0 ? -1 : (lz > 7 ? 1 : 0);
      const int nb = nb27[(oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)];
      const int64_t sl = (int64_t)nb * DBV + (((lz & 7) * DBS + (ly & 7)) * DBS + (lx & 7));
      for (int c = 0; c < 3; ++c) {
        float v = 0.f;
        if (nb >= 0) {
          const ff x = dsplit(u[c * g.nslots + sl]);
          v = __fadd_rn(x.h, x.l);   // u rounded to FP32
        }
        tile[c * TILE3 + t] = v;
      }
    }
  }
  if (threadIdx.x == 0) {
    const double* F = stencil_factors<double>(g, b);
    const int inst = g.binst[b];
    const double dt = g.pdt[inst], dnu = dt * g.pnu[inst];
    double h[3];
    spacing(g, b, h);
    sm3 = dsplit(F[3]);
    for (int a = 0; a < 3; ++a) {
      sk[a] = dsplit(dnu * F[a]);
      sih[a] = float(1.0 / h[a]);
    }
    swv = float(dt * F[3]);
  }
  __syncthreads();
  const int t = threadIdx.x;
  const int64_t s = (int64_t)b * DBV + t;
  const uint16_t m = g.meta[s];
  const bool valid = (m & D_VALID) != 0;
  ff cf[15];
#pragma unroll
  for (int k = 0; k < 15; ++k) cf[k] = ff{0.f, 0.f};
  with_mask(valid ? (m & 0xFF) : 0, [&](auto mask) {
    if (!valid) return;
    const int ti = tile_index(t & 7, (t >> 3) & 7, t >> 6);
    // M + dt nu K: integer weights times the factors, as pairs
#pragma unroll
    for (int k = 0; k < 15; ++k) cf[k] = ff_mul(ff{wf(mass_weight(mask, k)), 0.f}, sm3);
    ff diagK{0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const ff kp = ff_mul(ff{wf(stiff_edge_count(mask, a, 1)), 0.f}, sk[a]);
      const ff km = ff_mul(ff{wf(stiff_edge_count(mask, a, -1)), 0.f}, sk[a]);
      cf[1 + 2 * a] = ff_add(cf[1 + 2 * a], ff_neg(kp));
      cf[2 + 2 * a] = ff_add(cf[2 + 2 * a], ff_neg(km));
      diagK = ff_add(diagK, ff_add(kp, km));
    }
    cf[0] = ff_add(cf[0], diagK);
    float cc[15];
    conv_coef<float>(mask, tile, ti, swv, sih[0], sih[1], sih[2], cc);
#pragma unroll
    for (int k = 0; k < 15; ++k) cf[k] = ff_add(cf[k], ff{cc[k], 0.f});
  });
  const int64_t ci = compact_index(g, b, t, valid);
  if (valid)
#pragma unroll
    for (int k = 0; k < 15; ++k) {
      const float hi = __fadd_rn(cf[k].h, cf[k].l);
      coef32[(int64_t)k * g.ncomp + ci] = hi;
      coeflo[(int64_t)k * g.ncomp + ci] = __fadd_rn(__fsub_rn(cf[k].h, hi), cf[k].l);
    }
}

// ---------------------------------------------------------------- elementwise
__global__ void k_cast_d2f(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  KCOUNT();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = float(a[i]);
}
__global__ void k_add_f2d(int64_t n, const float* __restrict__ a, double* __restrict__ b) {
  KCOUNT();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] += double(a[i]);
}
__global__ void k_add_d(int64_t n, const double* __restrict__ a, double* __restrict__ b) {
  KCOUNT();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] += a[i];
}
__global__ void k_copy_d(int64_t n, const double* __restrict__ a, double* __restrict__ b) {
  KCOUNT();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}
template <typename T>
__global__ void k_zero(int64_t n, T* __restrict__ a) {
  KCOUNT();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = T(0);
}

template <typename T>
__global__ void k_gather_canon(int64_t N, const int32_t* __restrict__ cs, int nc, int64_t nslots,
                               const T* __restrict__ x, T* __restrict__ out) {
  KCOUNT();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    for (int c = 0; c < nc; ++c) out[i * nc + c] = x[c * nslots + cs[i]];
}
__global__ void k_scatter_canon(int64_t N, const int32_t* __restrict__ cs, int nc, int64_t nslots,
                                const double* __restrict__ in, double* __restrict__ x) {
  KCOUNT();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    for (int c = 0; c < nc; ++c) x[c * nslots + cs[i]] = in[i * nc + c];
}
__global__ void k_copy_to_fine(DevGrid g, int nc, double* __restrict__ x) {
  KCOUNT();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.n_if) return;
  for (int c = 0; c < nc; ++c) x[c * g.nslots + g.if_f[e]] = x[c * g.nslots + g.if_c[e]];
}

// port waveform a0 + sum_k a_k cos(k w t) + b_k sin(k w t), w = 2 pi / period
__device__ __forceinline__ double port_wave(const PortDev& P, double t) {
  const double w = 2.0 * 3.14159265358979323846 / P.period;
  double v = P.a0;
  for (int k = 0; k < P.nh; ++k) v += P.a[k] * cos((k + 1) * w * t) + P.b[k] * sin((k + 1) * w * t);
  return v;
}

__global__ void k_set_inlet(int64_t n, const int32_t* __restrict__ slot, const int32_t* __restrict__ port,
                            const double* __restrict__ shape, const PortDev* __restrict__ ports,
                            const double* __restrict__ tp, int64_t nslots, double* __restrict__ u) {
  KCOUNT();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const PortDev& P = ports[port[i]];
    u[P.axis * nslots + slot[i]] = port_wave(P, tp[P.inst]) * shape[i];
  }
}
// Phi = p_in(t^{n+1}) - p^n on every stored copy of a pressure-inlet node
__global__ void k_set_pinlet(int64_t n, const int32_t* __restrict__ slot, const int32_t* __restrict__ port,
                             const PortDev* __restrict__ ports, const double* __restrict__ tp,
                             const double* __restrict__ p, double* __restrict__ phi) {
  KCOUNT();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const PortDev& P = ports[port[i]];
    const int32_t s = slot[i];
    phi[s] = port_wave(P, tp[P.inst]) - p[s];
  }
}
// per instance: t_next = t_commit + dt, or (commit) t_commit = t_next where ok[i]
__global__ void k_time(double* tc, double* tn, const double* dt, int n, int commit, const int32_t* ok) {
  KCOUNT();
  const int i = threadIdx.x + blockIdx.x * blockDim.x;
  if (i >= n) return;
  if (commit) {
    if (!ok || ok[i]) tc[i] = tn[i];
  } else {
    tn[i] = tc[i] + dt[i];
  }
}

// ---------------------------------------------------------------- profiling
void Prof::begin(int c, cudaStream_t st) {
  if (!on) return;
  if (2 * (used + 1) > int(ev.size())) {
    for (int k = 0; k < 64; ++k) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      ev.push_back(e);
    }
  }
  cls.push_back(c);
  cudaEventRecord(ev[2 * used], st);
}
void Prof::end(cudaStream_t st) {
  if (!on) return;
  cudaEventRecord(ev[2 * used + 1], st);
  used++;
}
void Prof::collect() {
  for (int i = 0; i < used; ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]) == cudaSuccess) {
      ms[cls[i]] += t;
      n[cls[i]] += 1;
    }
  }
  used = 0;
  cls.clear();
}
void Prof::release() {
  for (auto e : ev) cudaEventDestroy(e);
  ev.clear();
  cls.clear();
  used = 0;
}

// ---------------------------------------------------------------- host wrappers
static inline int nblk(int64_t n, int bs = 256) {
  int64_t b = (n + bs - 1) / bs;
  return int(std::min<int64_t>(std::max<int64_t>(b, 1), 152 * 16));
}

// CG iteration kernel for the Poisson operator (the hot loop of the step):
// one CTA per chunk of bricks; for each brick p_new = z + beta p_old is formed
// for the brick's own nodes (one coalesced load per array and thread) and for
// the six face halos (threads 0..383, one face node each; index math done once
// per thread), q = K p_new by the 7-point stencil (interior nodes: the brick
// level's constant coefficients; boundary nodes: the incident-cell mask
// table), and p.q is accumulated per thread across the chunk.
//
// With CG = false the kernel is a plain local apply q = K z (no direction
// update, no reduction) over the chunks of problems that are not done and,
// when `on` is given, use multigrid.
template <typename T, bool CG>
__global__ void __launch_bounds__(512) k_poisson_cg(DevGrid g, const T* __restrict__ z, const T* __restrict__ pold,
                                                    T* __restrict__ pnew, T* __restrict__ q, uint16_t dmask,
                                                    KState* __restrict__ ks, double* __restrict__ partials,
                                                    unsigned* __restrict__ counter, const uint8_t* __restrict__ on) {
  KCOUNT();
  __shared__ T tile[TILE3];
  const int b0 = g.cbrick[blockIdx.x], b1 = g.cbrick[blockIdx.x + 1];
  const int inst = g.binst[b0];
  const bool done = ks ? ks[inst].done != 0 : false;   // plain applies may pass no solver state
  T acc = T(0);
  if (!CG && (done || (on && !on[inst]))) return;
  if (!done) {
    const T beta = CG ? k_beta<T>(ks[inst]) : T(0);
    const int t = threadIdx.x;
    const int lx = t & 7, ly = (t >> 3) & 7, lz = t >> 6;
    const int ti = tile_index(lx, ly, lz);
    // face halo element of this thread (t < 384)
    int fnb = 13, fli = 0, fti = 0;
    if (t < 384) {
      const int f = t >> 6, u = t & 7, v = (t >> 3) & 7;
      int hx, hy, hz, ox = 0, oy = 0, oz = 0, gx, gy, gz;
      if (f < 2) { hx = f ? 8 : -1; hy = u; hz = v; ox = f ? 1 : -1; gx = f ? 0 : 7; gy = u; gz = v; }
      else if (f < 4) { hx = u; hy = (f & 1) ? 8 : -1; hz = v; oy = (f & 1) ? 1 : -1; gx = u; gy = (f & 1) ? 0 : 7; gz = v; }
      else { hx = u; hy = v; hz = (f & 1) ? 8 : -1; oz = (f & 1) ? 1 : -1; gx = u; gy = v; gz = (f & 1) ? 0 : 7; }
      fnb = (oz + 1) * 9 + (oy + 1) * 3 + (ox + 1);
      fli = (gz * DBS + gy) * DBS + gx;
      fti = tile_index(hx, hy, hz);
    }
    // software pipeline: the next brick's value, halo value and metadata are
    // loaded into registers while the current brick is computed
    auto own = [&](int bb) -> T {
      const int64_t s = (int64_t)bb * DBV + t;
      return CG ? T(z[s] + beta * pold[s]) : z[s];
    };
    auto halo = [&](int bb) -> T {
      if (t >= 384) return T(0);
      const int nb = g.bnbr[27 * bb + fnb];
      const int64_t fs = (int64_t)nb * DBV + fli;
      return nb >= 0 ? (CG ? T(z[fs] + beta * pold[fs]) : z[fs]) : T(0);
    };
    T pn = own(b0), hn = halo(b0);
    uint16_t mn = g.meta[(int64_t)b0 * DBV + t];
    for (int bb = b0; bb < b1; ++bb) {
      const int64_t s = (int64_t)bb * DBV + t;
      const T pv = pn;
      const uint16_t m = mn;
      tile[ti] = pv;
      if (t < 384) tile[fti] = hn;
      __syncthreads();
      if (bb + 1 < b1) {
        pn = own(bb + 1);
        hn = halo(bb + 1);
        mn = g.meta[s + DBV];
      }
      T out = T(0);
      const bool valid = (m & D_VALID) != 0;
      with_mask(valid ? (m & 0xFF) : 0, [&](auto mk) {
        if (!valid) return;
        const T* F = stencil_factors<T>(g, bb);
        const T xm = tile[ti - 1], xp = tile[ti + 1], ym = tile[ti - TILE], yp = tile[ti + TILE];
        const T zm = tile[ti - TILE * TILE], zp = tile[ti + TILE * TILE];
        // Kuhn tetrahedra holding each axis edge (kuhn_weights.hpp): the P1
        // stiffness is -(V/6)/h_a^2 times this count, the diagonal their sum
        const int wxp = stiff_edge_count(mk, 0, 1), wxm = stiff_edge_count(mk, 0, -1);
        const int wyp = stiff_edge_count(mk, 1, 1), wym = stiff_edge_count(mk, 1, -1);
        const int wzp = stiff_edge_count(mk, 2, 1), wzm = stiff_edge_count(mk, 2, -1);
        const T fx = F[0], fy = F[1], fz = F[2];
        out = fx * (wconv<T>(wxp) * (pv - xp) + wconv<T>(wxm) * (pv - xm)) +
              fy * (wconv<T>(wyp) * (pv - yp) + wconv<T>(wym) * (pv - ym)) +
              fz * (wconv<T>(wzp) * (pv - zp) + wconv<T>(wzm) * (pv - zm));
      });
      if (m & dmask) out = T(0);
      if (m & D_VALID) {   // brick padding stays zero: no store
        q[s] = out;
        if (CG) pnew[s] = pv;
      }
      if (CG) acc += pv * out;
      __syncthreads();
    }
  }
  if (!CG) return;
  T v[1] = {acc};
  double* out = partials + (int64_t)gridDim.x;
  if (!grid_sum_last<T, 1>(v, partials, counter, g.cseg, g.ninst, out)) return;
  for (int i = threadIdx.x; i < g.ninst; i += blockDim.x) {
    KState& kk = ks[i];
    if (kk.done) continue;
    const double pq = out[i];
    kk.pq = pq;
    if (!(pq > 0.0) || !isfinite(pq)) { kk.done = 1; kk.status = 5; kk.alpha = 0.0; kk.af = 0.f; continue; }
    kk.alpha = kk.rz / pq;
    kk.af = float(kk.alpha);
  }
}

// ---------------------------------------------------------------- staged Poisson stencil
// The FP32 7-point Poisson kernels of the mixed path (the CG iteration form and
// the plain apply of the V-cycle).  One CTA of 128 threads walks a chunk of
// bricks through a ring of stages in shared memory (p7_stages), stages - 1
// bricks ahead of the one it computes.  Per brick a stage receives
//   * the brick's own values of each input vector and its metadata: bulk
//     copies of contiguous 2 KB / 1 KB runs (cp.async.bulk, the TMA unit's
//     untiled form) completing on the stage's mbarrier;
//   * the six face halos of each input vector by asynchronous copies
//     (cp.async, zero-filled where there is no neighbour): 16-byte pieces of
//     the y and z faces, single values of the x faces; each thread waits for
//     its own copy groups.  (Face boxes of a tensor map were measured slower:
//     their 16-32 byte rows bound the copies by the TMA unit's request rate.)
// No register holds a value in transit.  Each thread computes four
// consecutive nodes of an x row straight from the stage with 16-byte shared
// loads, and stores them as one 16-byte vector; one CTA barrier per brick.
// The single-node form of this kernel was bound by instruction issue, not by
// memory.  Where every node of a warp has all eight incident cells active the
// stiffness edge counts are the constant 6; elsewhere they come from a table
// of the 256 incident-cell masks in shared memory.  The arithmetic is that of
// k_poisson_cg, in the same order.
// ring depth: the apply (3.5 KB per brick from memory) keeps 4 bricks ahead,
// eight CTAs per SM; the CG form (6.5 KB per brick, twice the stage) 3 ahead,
// six CTAs per SM
template <int NV>
__host__ __device__ constexpr int p7_stages() { return NV == 2 ? 4 : 5; }
constexpr int P7_THREADS = 128;
constexpr int P7_CHUNK = 8;    // bricks per chunk at most (the chunk table's)
template <int NV>   // input vectors: 2 (z and p_old) for the CG form, 1 for the apply
struct P7Stage {
  // per vector 896 floats: the brick's own 512 values, then the face halos,
  // face f (-x, +x, -y, +y, -z, +z) at 512 + 64 f, its element (u, v) at 8 v + u
  static constexpr int VEC = 896;
  static constexpr int META = NV * VEC * 4;       // 512 x uint16
  static constexpr int BYTES = META + 1024;
};

__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool fill) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(fill ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool fill) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(fill ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// The face copies of one thread: copy A (every thread) is a 16-byte piece of a
// y or z face (threads 0..63) or an -x face value (64..127); copy B (threads
// 0..63) a +x face value.  fa/fb: face, ha/hb: node index in the neighbour
// brick, da/db: float offset in the vector block.
struct P7Copies {
  int fa, ha, da, hb, db;
};
__device__ __forceinline__ P7Copies p7_copies(int t) {
  P7Copies c;
  if (t < 64) {
    const int f = 2 + (t >> 4), q = t & 15, v = q >> 1, u0 = (q & 1) * 4;
    const int far = (f & 1) ? 0 : 7;           // the neighbour's plane next to this brick
    c.fa = f;
    c.ha = f < 4 ? (v * DBS + far) * DBS + u0 : (far * DBS + v) * DBS + u0;
    c.da = DBV + 64 * f + 8 * v + u0;
    const int e = t, u = e & 7, w = e >> 3;    // +x face element (u, w): x = 0 of the neighbour
    c.hb = (w * DBS + u) * DBS;
    c.db = DBV + 64 + 8 * w + u;
  } else {
    const int e = t - 64, u = e & 7, w = e >> 3;   // -x face element: x = 7 of the neighbour
    c.fa = 0;
    c.ha = (w * DBS + u) * DBS + 7;
    c.da = DBV + 8 * w + u;
    c.hb = c.db = 0;
  }
  return c;
}

// Fill one stage with brick i of the chunk (every thread calls it): warp 0
// issues the bulk copies, every thread its face copies.  nbf[6 i + f] is the
// neighbour brick across face f.
template <int NV>
__device__ __forceinline__ void p7_issue(const DevGrid& g, unsigned char* stage, uint64_t* bar, int b,
                                         const int* nbf, int i, const float* v0, const float* v1,
                                         const P7Copies& c) {
  const int t = threadIdx.x;
  float* sv = reinterpret_cast<float*>(stage);
  if (t < 32) {
    if (t == 0) mbar_arrive_expect_tx(bar, uint32_t(NV * 2048 + 1024));
    __syncwarp();
    if (t < NV) bulk_g2s(sv + t * P7Stage<NV>::VEC, (t ? v1 : v0) + (int64_t)b * DBV, 2048u, bar);
    else if (t == NV) bulk_g2s(stage + P7Stage<NV>::META, g.meta + (int64_t)b * DBV, 1024u, bar);
  }
  const int na = nbf[6 * i + c.fa];
  const int64_t sa = na >= 0 ? (int64_t)na * DBV + c.ha : 0;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const float* src = (v ? v1 : v0);
    float* dst = sv + v * P7Stage<NV>::VEC;
    if (t < 64) {
      cp_async16(dst + c.da, src + sa, na >= 0);
      const int nb = nbf[6 * i + 1];
      cp_async4(dst + c.db, src + (nb >= 0 ? (int64_t)nb * DBV + c.hb : 0), nb >= 0);
    } else {
      cp_async4(dst + c.da, src + sa, na >= 0);
    }
  }
  cp_async_commit();
}

template <bool CG>
__global__ void __launch_bounds__(P7_THREADS, 8)
    k_poisson7_staged(DevGrid g, const float* __restrict__ z, const float* __restrict__ pold,
                      float* __restrict__ pnew, float* __restrict__ q, uint16_t dmask, KState* __restrict__ ks,
                      double* __restrict__ partials, unsigned* __restrict__ counter, const uint8_t* __restrict__ on) {
  KCOUNT();
  constexpr int NV = CG ? 2 : 1;
  constexpr int VEC = P7Stage<NV>::VEC;
  using S = P7Stage<NV>;
  constexpr int P7_STAGES = p7_stages<NV>();
  extern __shared__ unsigned char p7_dyn[];
  __shared__ __align__(8) uint64_t full[P7_STAGES];
  __shared__ int nbf[6 * P7_CHUNK];
  __shared__ float fac[3 * P7_CHUNK];   // stencil factors (V/6)/h_a^2 of each brick
  __shared__ uint32_t ecnt[256];        // per mask: edge counts, 4 bits each, (+x, -x, +y, -y, +z, -z)
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p7_dyn) + 127) & ~uintptr_t(127));
  const int b0 = g.cbrick[blockIdx.x], b1 = g.cbrick[blockIdx.x + 1];
  const int inst = g.binst[b0];
  const bool done = ks ? ks[inst].done != 0 : false;
  float acc = 0.f;
  if (!CG && (done || (on && !on[inst]))) return;
  if (!done) {
    const float beta = CG ? k_beta<float>(ks[inst]) : 0.f;
    const int t = threadIdx.x;
    const int n = b1 - b0;
    if (t < 6 * n) {
      // face f: -x, +x, -y, +y, -z, +z -> entry of the 27-entry neighbour table
      const int f = t % 6;
      nbf[t] = g.bnbr[27 * (b0 + t / 6) + (f == 0 ? 12 : f == 1 ? 14 : f == 2 ? 10 : f == 3 ? 16 : f == 4 ? 4 : 22)];
    } else if (t >= 64 && t < 64 + 3 * n) {
      const int j = t - 64;
      fac[j] = stencil_factors<float>(g, b0 + j / 3)[j % 3];
    }
    for (int mk = t; mk < 256; mk += P7_THREADS) {
      uint32_t w = 0;
#pragma unroll
      for (int e = 0; e < 6; ++e) w |= uint32_t(stiff_edge_count(mk, e >> 1, (e & 1) ? -1 : 1)) << (4 * e);
      ecnt[mk] = w;
    }
    if (t == 0)
      for (int k = 0; k < P7_STAGES; ++k) mbar_init(&full[k]);
    __syncthreads();
    const P7Copies cc = p7_copies(t);
    // this thread's four nodes: x = 4 seg .. 4 seg + 3 of row (ly, lz); offsets
    // in a vector block of the node, of the rows and planes next to it and of
    // the x neighbours of its first and last node
    const int seg = t & 1, ly = (t >> 1) & 7, lz = t >> 4;
    const int o = (lz * 8 + ly) * 8 + 4 * seg;
    const int oym = ly > 0 ? o - 8 : DBV + 128 + 8 * lz + 4 * seg, oyp = ly < 7 ? o + 8 : DBV + 192 + 8 * lz + 4 * seg;
    const int ozm = lz > 0 ? o - 64 : DBV + 256 + 8 * ly + 4 * seg, ozp = lz < 7 ? o + 64 : DBV + 320 + 8 * ly + 4 * seg;
    const int oxl = seg ? o - 1 : DBV + 8 * lz + ly, oxr = seg ? DBV + 64 + 8 * lz + ly : o + 4;
    for (int k = 0; k < P7_STAGES - 1; ++k) {
      if (k < n) p7_issue<NV>(g, sm + k * S::BYTES, &full[k], b0 + k, nbf, k, z, pold, cc);
      else cp_async_commit();
    }
    for (int i = 0; i < n; ++i) {
      const int k = i % P7_STAGES;
      cp_async_wait<P7_STAGES - 2>();   // this thread's face copies of brick i
      if (t == 0) mbar_wait_or_flag(&full[k], uint32_t(i / P7_STAGES) & 1u, g.aerr + inst);
      __syncthreads();   // stage k complete and visible; every thread is past brick i - 1
      {
        const int ir = i + P7_STAGES - 1, kr = ir % P7_STAGES;   // the stage of brick i - 1
        if (ir < n) p7_issue<NV>(g, sm + kr * S::BYTES, &full[kr], b0 + ir, nbf, ir, z, pold, cc);
        else cp_async_commit();
      }
      const unsigned char* st = sm + k * S::BYTES;
      const float* vb = reinterpret_cast<const float*>(st);
      // p (= z + beta p_old for the CG form): four nodes, or one value
      auto p4 = [&](int off) -> float4 {
        float4 a = *reinterpret_cast<const float4*>(vb + off);
        if constexpr (CG) {
          const float4 b = *reinterpret_cast<const float4*>(vb + off + VEC);
          a = make_float4(float(a.x + beta * b.x), float(a.y + beta * b.y), float(a.z + beta * b.z),
                          float(a.w + beta * b.w));
        }
        return a;
      };
      auto p1 = [&](int off) -> float {
        if constexpr (CG) return float(vb[off] + beta * vb[off + VEC]);
        else return vb[off];
      };
      const float4 pc = p4(o), ym = p4(oym), yp = p4(oyp), zm = p4(ozm), zp = p4(ozp);
      const float xl = p1(oxl), xr = p1(oxr);
      const uint2 mm = *reinterpret_cast<const uint2*>(st + S::META + 2 * o);
      const uint16_t m[4] = {uint16_t(mm.x & 0xFFFFu), uint16_t(mm.x >> 16), uint16_t(mm.y & 0xFFFFu),
                             uint16_t(mm.y >> 16)};
      const float fx = fac[3 * i], fy = fac[3 * i + 1], fz = fac[3 * i + 2];
      const float pv[4] = {pc.x, pc.y, pc.z, pc.w};
      const float xv[6] = {xl, pc.x, pc.y, pc.z, pc.w, xr};
      const float ymv[4] = {ym.x, ym.y, ym.z, ym.w}, ypv[4] = {yp.x, yp.y, yp.z, yp.w};
      const float zmv[4] = {zm.x, zm.y, zm.z, zm.w}, zpv[4] = {zp.x, zp.y, zp.z, zp.w};
      float out[4];
      const bool full4 = ((m[0] & m[1] & m[2] & m[3] & (D_VALID | 0xFF)) == (D_VALID | 0xFF));
      if (__all_sync(0xffffffffu, full4)) {
        // every node of the warp: all eight incident cells active, edge counts 6
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float w = 6.f;
          out[j] = fx * (w * (pv[j] - xv[j + 2]) + w * (pv[j] - xv[j])) + fy * (w * (pv[j] - ypv[j]) + w * (pv[j] - ymv[j])) +
                   fz * (w * (pv[j] - zpv[j]) + w * (pv[j] - zmv[j]));
        }
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          out[j] = 0.f;
          if (m[j] & D_VALID) {
            const uint32_t w = ecnt[m[j] & 0xFF];
            const float wxp = float(w & 15u), wxm = float((w >> 4) & 15u), wyp = float((w >> 8) & 15u);
            const float wym = float((w >> 12) & 15u), wzp = float((w >> 16) & 15u), wzm = float((w >> 20) & 15u);
            out[j] = fx * (wxp * (pv[j] - xv[j + 2]) + wxm * (pv[j] - xv[j])) +
                     fy * (wyp * (pv[j] - ypv[j]) + wym * (pv[j] - ymv[j])) +
                     fz * (wzp * (pv[j] - zpv[j]) + wzm * (pv[j] - zmv[j]));
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (m[j] & dmask) out[j] = 0.f;
      // brick padding: the inputs are zero there, so are p and the output
      const int64_t s = (int64_t)(b0 + i) * DBV + o;
      *reinterpret_cast<float4*>(q + s) = make_float4(out[0], out[1], out[2], out[3]);
      if constexpr (CG) {
        *reinterpret_cast<float4*>(pnew + s) = pc;
#pragma unroll
        for (int j = 0; j < 4; ++j) acc += pv[j] * out[j];
      }
    }
  }
  if (!CG) return;
  float v[1] = {acc};
  double* out = partials + (int64_t)gridDim.x;
  if (!grid_sum_last<float, 1>(v, partials, counter, g.cseg, g.ninst, out)) return;
  for (int i = threadIdx.x; i < g.ninst; i += blockDim.x) {
    KState& kk = ks[i];
    if (kk.done) continue;
    const double pq = out[i];
    kk.pq = pq;
    if (!(pq > 0.0) || !isfinite(pq)) { kk.done = 1; kk.status = 5; kk.alpha = 0.0; kk.af = 0.f; continue; }
    kk.alpha = kk.rz / pq;
    kk.af = float(kk.alpha);
  }
}

template <int NV>
static constexpr size_t p7_smem() { return size_t(p7_stages<NV>()) * P7Stage<NV>::BYTES + 128; }

// ---------------------------------------------------------------- persistent Poisson stencil
// A launch choice (IB_TUNE_POISSON_KERNEL = 3): the staged kernel above made
// persistent.  A whole number of CTAs per SM (DevGrid::p7_ctas), each walking
// the chunks c, c + p7_ctas, ... brick by brick through one ring of
// shared-memory stages that runs on across chunk boundaries, so that no CTA
// start, table set-up or ring fill sits between chunks.  The per-brick schedule
// (brick, face neighbours, instance, chunk, stencil factors: P7Hdr, written by
// the host once per grid) is read by 16-byte asynchronous copies
// 2 (stages - 1) bricks ahead into a ring of headers.  Per brick the copies,
// the four-nodes-per-thread arithmetic and the CG form's per-chunk p.q partial
// are those of k_poisson7_staged, so both give the same bits.  Measured on the
// two-level aorta (59 M valid slots) it is slower than one CTA per chunk (the
// static schedule leaves SMs idle while the slowest CTAs finish; the hardware
// scheduler balances per chunk), so the default stays k_poisson7_staged.
// ring depth (stages) of the persistent form
template <int NV>
__host__ __device__ constexpr int p7p_stages() { return 4; }
constexpr int P7_HRING = 16;      // header ring: headers run 2 (stages - 1) bricks ahead
constexpr int P7_MAXINST = 256;   // instances whose flags a CTA keeps in shared memory
static_assert(P7_HRING >= 2 * (p7p_stages<1>() - 1) + 2 && P7_HRING >= 2 * (p7p_stages<2>() - 1) + 2,
              "header ring too short for its look-ahead");
// Fill one data stage with brick h.b (every thread calls it; no commit here):
// warp 0 issues the bulk copies, every thread its face copies.
template <int NV>
__device__ __forceinline__ void p7p_issue(const DevGrid& g, unsigned char* stage, uint64_t* bar, const P7Hdr& h,
                                         const float* v0, const float* v1, const P7Copies& c) {
  const int t = threadIdx.x;
  float* sv = reinterpret_cast<float*>(stage);
  if (t < 32) {
    if (t == 0) mbar_arrive_expect_tx(bar, uint32_t(NV * 2048 + 1024));
    __syncwarp();
    if (t < NV) bulk_g2s(sv + t * P7Stage<NV>::VEC, (t ? v1 : v0) + (int64_t)h.b * DBV, 2048u, bar);
    else if (t == NV) bulk_g2s(stage + P7Stage<NV>::META, g.meta + (int64_t)h.b * DBV, 1024u, bar);
  }
  const int na = h.nb[c.fa], nb = h.nb[1];
  const int64_t sa = na >= 0 ? (int64_t)na * DBV + c.ha : 0;
  const int64_t sb = nb >= 0 ? (int64_t)nb * DBV + c.hb : 0;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const float* src = (v ? v1 : v0);
    float* dst = sv + v * P7Stage<NV>::VEC;
    if (t < 64) {
      cp_async16(dst + c.da, src + sa, na >= 0);
      cp_async4(dst + c.db, src + sb, nb >= 0);
    } else {
      cp_async4(dst + c.da, src + sa, na >= 0);
    }
  }
}

template <bool CG>
__global__ void __launch_bounds__(P7_THREADS, 6)
    k_poisson7_persist(DevGrid g, const float* __restrict__ z, const float* __restrict__ pold,
                      float* __restrict__ pnew, float* __restrict__ q, uint16_t dmask, KState* __restrict__ ks,
                      double* __restrict__ partials, unsigned* __restrict__ counter, const uint8_t* __restrict__ on) {
  constexpr int NV = CG ? 2 : 1;
  constexpr int VEC = P7Stage<NV>::VEC;
  using S = P7Stage<NV>;
  constexpr int ST = p7p_stages<NV>();
  extern __shared__ unsigned char p7p_dyn[];
  __shared__ __align__(8) uint64_t full[ST];
  __shared__ __align__(16) P7Hdr hdr[P7_HRING];
  __shared__ uint32_t ecnt[256];        // per mask: edge counts, 4 bits each, (+x, -x, +y, -y, +z, -z)
  __shared__ float bet[P7_MAXINST];     // beta of each instance (CG form)
  __shared__ uint8_t act[P7_MAXINST];   // instance still iterating (and selected by `on`)
  __shared__ float sred[32];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p7p_dyn) + 127) & ~uintptr_t(127));
  const int t = threadIdx.x;
  const int j0 = g.p7_off[blockIdx.x], n = g.p7_off[blockIdx.x + 1] - j0;
  const int4* hsrc = g.p7_hdr + 4 * (int64_t)j0;
  // until KCOUNT only data written at set-up: the mask table, the barriers,
  // the headers of the first ST - 1 bricks
  for (int mk = t; mk < 256; mk += P7_THREADS) {
    uint32_t w = 0;
#pragma unroll
    for (int e = 0; e < 6; ++e) w |= uint32_t(stiff_edge_count(mk, e >> 1, (e & 1) ? -1 : 1)) << (4 * e);
    ecnt[mk] = w;
  }
  if (t == 0)
    for (int k = 0; k < ST; ++k) mbar_init(&full[k]);
  if (t < 4 * (ST - 1) && (t >> 2) < n)
    cp_async16(reinterpret_cast<int4*>(&hdr[t >> 2]) + (t & 3), hsrc + t, true);
  cp_async_commit();
  KCOUNT();
  for (int i = t; i < g.ninst; i += P7_THREADS) {
    const bool live = !(ks && ks[i].done) && (CG || !on || on[i]);
    act[i] = live ? 1 : 0;
    if constexpr (CG) bet[i] = k_beta<float>(ks[i]);
  }
  cp_async_wait<0>();
  __syncthreads();
  const P7Copies cc = p7_copies(t);
  // this thread's four nodes: x = 4 seg .. 4 seg + 3 of row (ly, lz); offsets
  // in a vector block of the node, of the rows and planes next to it and of
  // the x neighbours of its first and last node
  const int seg = t & 1, ly = (t >> 1) & 7, lz = t >> 4;
  const int o = (lz * 8 + ly) * 8 + 4 * seg;
  const int oym = ly > 0 ? o - 8 : DBV + 128 + 8 * lz + 4 * seg, oyp = ly < 7 ? o + 8 : DBV + 192 + 8 * lz + 4 * seg;
  const int ozm = lz > 0 ? o - 64 : DBV + 256 + 8 * ly + 4 * seg, ozp = lz < 7 ? o + 64 : DBV + 320 + 8 * ly + 4 * seg;
  const int oxl = seg ? o - 1 : DBV + 8 * lz + ly, oxr = seg ? DBV + 64 + 8 * lz + ly : o + 4;
  // data of brick j into stage j % ST (a plain arrival where its
  // instance is idle), and the header of brick j + ST - 1; one copy
  // group per call, so that the group of brick i is complete ST - 1
  // calls later
  auto issue = [&](int j) {
    if (j < n) {
      const P7Hdr& h = hdr[j % P7_HRING];
      const int k = j % ST;
      if (act[h.inst]) p7p_issue<NV>(g, sm + k * S::BYTES, &full[k], h, z, pold, cc);
      else if (t == 0) mbar_arrive(&full[k]);
      const int jh = j + ST - 1;
      if (t < 4 && jh < n)
        cp_async16(reinterpret_cast<int4*>(&hdr[jh % P7_HRING]) + t, hsrc + 4 * (int64_t)jh + t, true);
    }
    cp_async_commit();
  };
  for (int k = 0; k < ST - 1; ++k) issue(k);
  float acc = 0.f;
  for (int i = 0; i < n; ++i) {
    const int k = i % ST;
    const P7Hdr& h = hdr[i % P7_HRING];   // visible since the barrier of brick i - ST + 1
    const int inst = h.inst;
    const bool live = act[inst] != 0;
    cp_async_wait<ST - 2>();   // this thread's face copies of brick i, the header of i + ST - 1
    if (t == 0) mbar_wait_or_flag(&full[k], uint32_t(i / ST) & 1u, g.aerr + inst);
    __syncthreads();   // stage k complete and visible; every thread is past brick i - 1
    issue(i + ST - 1);
    if (live) {
      const float beta = CG ? bet[inst] : 0.f;
      const unsigned char* st = sm + k * S::BYTES;
      const float* vb = reinterpret_cast<const float*>(st);
      // p (= z + beta p_old for the CG form): four nodes, or one value
      auto p4 = [&](int off) -> float4 {
        float4 a = *reinterpret_cast<const float4*>(vb + off);
        if constexpr (CG) {
          const float4 b = *reinterpret_cast<const float4*>(vb + off + VEC);
          a = make_float4(float(a.x + beta * b.x), float(a.y + beta * b.y), float(a.z + beta * b.z),
                          float(a.w + beta * b.w));
        }
        return a;
      };
      auto p1 = [&](int off) -> float {
        if constexpr (CG) return float(vb[off] + beta * vb[off + VEC]);
        else return vb[off];
      };
      const float4 pc = p4(o), ym = p4(oym), yp = p4(oyp), zm = p4(ozm), zp = p4(ozp);
      const float xl = p1(oxl), xr = p1(oxr);
      const uint2 mm = *reinterpret_cast<const uint2*>(st + S::META + 2 * o);
      const uint16_t m[4] = {uint16_t(mm.x & 0xFFFFu), uint16_t(mm.x >> 16), uint16_t(mm.y & 0xFFFFu),
                             uint16_t(mm.y >> 16)};
      const float fx = h.fac[0], fy = h.fac[1], fz = h.fac[2];
      const float pv[4] = {pc.x, pc.y, pc.z, pc.w};
      const float xv[6] = {xl, pc.x, pc.y, pc.z, pc.w, xr};
      const float ymv[4] = {ym.x, ym.y, ym.z, ym.w}, ypv[4] = {yp.x, yp.y, yp.z, yp.w};
      const float zmv[4] = {zm.x, zm.y, zm.z, zm.w}, zpv[4] = {zp.x, zp.y, zp.z, zp.w};
      float out[4];
      const bool full4 = ((m[0] & m[1] & m[2] & m[3] & (D_VALID | 0xFF)) == (D_VALID | 0xFF));
      if (__all_sync(0xffffffffu, full4)) {
        // every node of the warp: all eight incident cells active, edge counts 6
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float w = 6.f;
          out[j] = fx * (w * (pv[j] - xv[j + 2]) + w * (pv[j] - xv[j])) + fy * (w * (pv[j] - ypv[j]) + w * (pv[j] - ymv[j])) +
                   fz * (w * (pv[j] - zpv[j]) + w * (pv[j] - zmv[j]));
        }
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          out[j] = 0.f;
          if (m[j] & D_VALID) {
            const uint32_t w = ecnt[m[j] & 0xFF];
            const float wxp = float(w & 15u), wxm = float((w >> 4) & 15u), wyp = float((w >> 8) & 15u);
            const float wym = float((w >> 12) & 15u), wzp = float((w >> 16) & 15u), wzm = float((w >> 20) & 15u);
            out[j] = fx * (wxp * (pv[j] - xv[j + 2]) + wxm * (pv[j] - xv[j])) +
                     fy * (wyp * (pv[j] - ypv[j]) + wym * (pv[j] - ymv[j])) +
                     fz * (wzp * (pv[j] - zpv[j]) + wzm * (pv[j] - zmv[j]));
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (m[j] & dmask) out[j] = 0.f;
      // brick padding: the inputs are zero there, so are p and the output
      const int64_t s = (int64_t)h.b * DBV + o;
      *reinterpret_cast<float4*>(q + s) = make_float4(out[0], out[1], out[2], out[3]);
      if constexpr (CG) {
        *reinterpret_cast<float4*>(pnew + s) = pc;
#pragma unroll
        for (int j = 0; j < 4; ++j) acc += pv[j] * out[j];
      }
    }
    if constexpr (CG) {
      if (h.last) {   // the chunk's p.q partial (zero for an idle instance)
        float v[1] = {acc};
        block_sum<float, 1>(v, sred);
        if (t == 0) partials[h.chunk] = double(v[0]);
        acc = 0.f;
      }
    }
  }
  if constexpr (CG) {
    double* out = partials + (int64_t)g.nchunks;
    if (!segment_sums_last<1>(partials, counter, g.cseg, g.ninst, out)) return;
    for (int i = threadIdx.x; i < g.ninst; i += blockDim.x) {
      KState& kk = ks[i];
      if (kk.done) continue;
      const double pq = out[i];
      kk.pq = pq;
      if (!(pq > 0.0) || !isfinite(pq)) { kk.done = 1; kk.status = 5; kk.alpha = 0.0; kk.af = 0.f; continue; }
      kk.alpha = kk.rz / pq;
      kk.af = float(kk.alpha);
    }
  }
}

template <int NV>
static constexpr size_t p7p_smem() { return size_t(p7p_stages<NV>()) * P7Stage<NV>::BYTES + 128; }

// CTAs per SM of the persistent Poisson kernels (the smaller of the two forms'
// occupancies), for the schedule the host writes per grid.
int fe_p7_ctas_per_sm() {
  int a = 0, b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_poisson7_persist<true>, P7_THREADS, p7p_smem<2>()) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_poisson7_persist<false>, P7_THREADS, p7p_smem<1>()) !=
          cudaSuccess)
    return 0;
  return std::min(a, b);
}

// The staged kernels serve FP32 vectors on 16-byte boundaries (every vector of
// the library; the bulk and 16-byte copies need it) over the chunks of at most
// P7_CHUNK bricks (the persistent one also needs its schedule and at most
// P7_MAXINST instances); returns false (nothing launched) otherwise.
template <typename T, bool CG>
static bool launch_p7(const DevGrid& g, const T* z, const T* pold, T* pnew, T* q, uint16_t dmask, KState* ks,
                      double* partials, unsigned* counter, const uint8_t* on, cudaStream_t st) {
  if constexpr (sizeof(T) != 4) {
    return false;
  } else {
    auto a16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    if (g.poisson_kernel == 2) return false;
    if (!a16(z) || !a16(q) || (CG && (!a16(pold) || !a16(pnew)))) return false;
    if (g.poisson_kernel == 3 && g.p7_ctas > 0 && g.ninst <= P7_MAXINST) {
      IBG_LAUNCH((k_poisson7_persist<CG>), g.p7_ctas, P7_THREADS, p7p_smem<CG ? 2 : 1>(), st, g, z, pold, pnew, q,
                 dmask, ks, partials, counter, on);
      return true;
    }
    IBG_LAUNCH((k_poisson7_staged<CG>), g.nchunks, P7_THREADS, p7_smem<CG ? 2 : 1>(), st, g, z, pold, pnew, q, dmask,
               ks, partials, counter, on);
    return true;
  }
}

// Halo element t (t < HALO15) of a brick for the 15-point Kuhn stencil: the six
// faces (384 nodes), the six edges reached by the offsets +-(1,1,0),
// +-(0,1,1), +-(1,0,1) (48 nodes) and the corners +-(1,1,1).  Gives the
// neighbour-brick index (0..26), the local index in that brick and the tile index.
constexpr int HALO15 = 434;
__device__ __forceinline__ void halo15(int t, int& nbk, int& li, int& ti) {
  int hx, hy, hz, ox = 0, oy = 0, oz = 0, gx, gy, gz;
  if (t < 384) {
    const int f = t >> 6, u = t & 7, v = (t >> 3) & 7;
    if (f < 2) { hx = f ? 8 : -1; hy = u; hz = v; ox = f ? 1 : -1; gx = f ? 0 : 7; gy = u; gz = v; }
    else if (f < 4) { hx = u; hy = (f & 1) ? 8 : -1; hz = v; oy = (f & 1) ? 1 : -1; gx = u; gy = (f & 1) ? 0 : 7; gz = v; }
    else { hx = u; hy = v; hz = (f & 1) ? 8 : -1; oz = (f & 1) ? 1 : -1; gx = u; gy = v; gz = (f & 1) ? 0 : 7; }
  } else if (t < 432) {
    const int e = (t - 384) >> 3, u = (t - 384) & 7;
    const int sg = (e & 1) ? -1 : 1, hi = (e & 1) ? -1 : 8, lo = (e & 1) ? 7 : 0;
    if (e < 2) { hx = hi; hy = hi; hz = u; ox = sg; oy = sg; gx = lo; gy = lo; gz = u; }        // +-(1,1,0)
    else if (e < 4) { hx = u; hy = hi; hz = hi; oy = sg; oz = sg; gx = u; gy = lo; gz = lo; }   // +-(0,1,1)
    else { hx = hi; hy = u; hz = hi; ox = sg; oz = sg; gx = lo; gy = u; gz = lo; }              // +-(1,0,1)
  } else {
    const int sg = t == 432 ? 1 : -1, hi = t == 432 ? 8 : -1, lo = t == 432 ? 0 : 7;
    hx = hy = hz = hi;
    ox = oy = oz = sg;
    gx = gy = gz = lo;
  }
  nbk = (oz + 1) * 9 + (oy + 1) * 3 + (ox + 1);
  li = (gz * DBS + gy) * DBS + gx;
  ti = tile_index(hx, hy, hz);
}

// 15-point operators (consistent mass from the incident-cell mask, or the
// per-slot momentum coefficients), NC components, one CTA per chunk of bricks
// (PB = false) or per brick (PB = true: more CTAs in flight for the streaming
// coefficient reads of a plain apply).
// FUSEP: p_new = z + beta p_old while staging the tile (written for the
// brick's nodes), y = A p_new, and per-component p.y -> alpha (POST_CG_ALPHA).
// One CTA per chunk, the FP32 mass operator fits 40 registers (a 16-byte
// spill) when asked for 3 CTAs of 512 threads per SM (57-71 and 2 CTAs
// otherwise); every other instance keeps the compiler's own choice (a minimum
// of 0).  The chunk's neighbour tables sit in shared memory, so a halo load
// waits on no neighbour-table load.
template <typename T, int OP, int NC, bool FUSEP, bool PB, bool SYM = false>
__global__ void __launch_bounds__(512, (sizeof(T) == 4 && OP == OP_MASS && !PB) ? 3 : 0)
    k_apply15(DevGrid g, const T* __restrict__ x, T* __restrict__ y,
                                                 const T* __restrict__ coef, uint16_t dmask, int post,
                                                 KState* __restrict__ ks, double* __restrict__ partials,
                                                 unsigned* __restrict__ counter, const T* __restrict__ zf,
                                                 T* __restrict__ pnew) {
  // FP32 with 3 components: one float4 per tile node (one 16-byte shared load
  // per stencil neighbour); otherwise one plane per component
  constexpr bool V4 = sizeof(T) == 4 && NC == 3;
  constexpr int NBR = PB ? 1 : 8;   // bricks per CTA at most (the chunk table's)
  __shared__ __align__(16) T tile[V4 ? 4 * TILE3 : NC * TILE3];
  __shared__ int snb[NBR * 27];     // the chunk's neighbour tables
  float4* tile4 = reinterpret_cast<float4*>(tile);
  auto tval = [&](int c, int j) -> T {
    if constexpr (V4) return reinterpret_cast<const T*>(tile4 + j)[c];
    else return tile[c * TILE3 + j];
  };
  // set-up data before the wait for the previous kernel: the chunk, its
  // instance and its bricks' neighbour tables (so that no halo load waits on
  // a neighbour-table load)
  const int b0 = PB ? int(blockIdx.x) : g.cbrick[blockIdx.x];
  const int b1 = PB ? b0 + 1 : g.cbrick[blockIdx.x + 1];
  const int inst = g.binst[b0];
  for (int e = threadIdx.x; e < (b1 - b0) * 27; e += blockDim.x) snb[e] = g.bnbr[27 * b0 + e];
  KCOUNT();
  bool skip = false;
  T beta[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) beta[c] = T(0);
  if (FUSEP) {
    skip = true;
    for (int c = 0; c < NC; ++c) {
      skip = skip && ks[inst * NC + c].done;
      beta[c] = k_beta<T>(ks[inst * NC + c]);
    }
  }
  T acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = T(0);
  if (!skip) {
    const int t = threadIdx.x;
    const int lx = t & 7, ly = (t >> 3) & 7, lz = t >> 6;
    const int ti = tile_index(lx, ly, lz);
    int hnb = 13, hli = 0, hti = 0;
    if (t < HALO15) halo15(t, hnb, hli, hti);
    // software pipeline over the chunk: the next brick's values, halo values
    // and metadata are loaded into registers while the current one is computed
    T vo[NC], vh[NC];
    auto fetch = [&](int bb) {
      const int64_t s = (int64_t)bb * DBV + t;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int64_t i = (int64_t)c * g.nslots + s;
        vo[c] = FUSEP ? T(zf[i] + beta[c] * x[i]) : x[i];
      }
      if (t < HALO15) {
        const int nb = snb[27 * (bb - b0) + hnb];
        const int64_t hs = (int64_t)nb * DBV + hli;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int64_t i = (int64_t)c * g.nslots + hs;
          vh[c] = nb >= 0 ? (FUSEP ? T(zf[i] + beta[c] * x[i]) : x[i]) : T(0);
        }
      }
    };
    __syncthreads();   // snb complete
    fetch(b0);
    uint16_t mn = g.meta[(int64_t)b0 * DBV + t];
    for (int bb = b0; bb < b1; ++bb) {
      const int64_t s = (int64_t)bb * DBV + t;
      if constexpr (V4) {
        tile4[ti] = make_float4(vo[0], vo[1], vo[2], 0.f);
        if (t < HALO15) tile4[hti] = make_float4(vh[0], vh[1], vh[2], 0.f);
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          tile[c * TILE3 + ti] = vo[c];
          if (t < HALO15) tile[c * TILE3 + hti] = vh[c];
        }
      }
      const uint16_t m = mn;
      __syncthreads();
      if (bb + 1 < b1) {
        fetch(bb + 1);
        mn = g.meta[s + DBV];
      }
      T out[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) out[c] = T(0);
      const bool act = (m & D_VALID) && !(m & dmask);
      if constexpr (OP == OP_MASS) {
        // M x = (V/120) sum_k w_k x_k with integer weights w_k
        with_mask(act ? (m & 0xFF) : 0, [&](auto mk) {
          if (!act) return;
#pragma unroll
          for (int k = 0; k < 15; ++k) {
            const T wk = wconv<T>(mass_weight(mk, k));
            if constexpr (V4) {
              const float4 v = tile4[ti + c_toff[k]];
              out[0] += wk * v.x;
              out[1] += wk * v.y;
              out[2] += wk * v.z;
            } else {
#pragma unroll
              for (int c = 0; c < NC; ++c) out[c] += wk * tile[c * TILE3 + ti + c_toff[k]];
            }
          }
          const T f3 = stencil_factors<T>(g, bb)[3];
#pragma unroll
          for (int c = 0; c < NC; ++c) out[c] *= f3;
        });
      } else {
        if (act) {
#pragma unroll
          for (int k = 0; k < 15; ++k) {
            const T ck = coef[(int64_t)k * g.nslots + s];
#pragma unroll
            for (int c = 0; c < NC; ++c) out[c] += ck * tval(c, ti + c_toff[k]);
          }
        }
        if constexpr (SYM && NC == 3) {   // symmetric viscous form
            with_mask(act ? (m & 0xFF) : 0, [&](auto mk) {
              if (!act) return;
              const int inst = g.binst[bb];
              add_transpose<T>(mk, stencil_factors<T>(g, bb), T(g.pdt[inst] * g.pnu[inst]),
                               [&](int k, T (&v)[3]) {
#pragma unroll
                                 for (int c = 0; c < 3; ++c) v[c] = tval(c, ti + c_toff[k]);
                               },
                               out);
            });
        }
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const T own = tval(c, ti);
        if (m & D_VALID) {   // brick padding stays zero: no store
          y[(int64_t)c * g.nslots + s] = out[c];
          if (FUSEP) pnew[(int64_t)c * g.nslots + s] = own;
        }
        if (FUSEP) acc[c] += own * out[c];
      }
      __syncthreads();
    }
  }
  if (post != POST_CG_ALPHA) return;
  double* out = partials + (int64_t)gridDim.x * NC;
  if (!grid_sum_last<T, NC>(acc, partials, counter, PB ? g.bseg : g.cseg, g.ninst, out)) return;
  for (int i = threadIdx.x; i < g.ninst; i += blockDim.x)
    for (int c = 0; c < NC; ++c) {
      KState& k = ks[i * NC + c];
      if (k.done) continue;
      const double pq = out[i * NC + c];
      k.pq = pq;
      if (!(pq > 0.0) || !isfinite(pq)) { k.done = 1; k.status = 5; k.alpha = 0.0; k.af = 0.f; continue; }
      k.alpha = k.rz / pq;
      k.af = float(k.alpha);
    }
}

// FP32 momentum operator, 3 components (the inner BiCGStab of the mixed path),
// one CTA per brick, four CTAs per SM:
//  * the 15 coefficient planes are stored compactly (valid slots only; per
//    brick a run starting on a 16-byte boundary); warp 0 copies them into
//    shared memory with bulk asynchronous copies (cp.async.bulk, completion on
//    an mbarrier) issued first, so they are in flight together with the
//    brick's x values and halo, and no register holds a coefficient in transit;
//  * the tile holds one float4 per node (3 components and a pad), so each
//    stencil neighbour is one 16-byte shared load.
// Same arithmetic, in the same order, as k_apply15<float, OP_COEF, 3>.
// SYM adds the transpose-gradient couplings of the symmetric viscous form
// (two CTAs per SM: the couplings need more than 32 registers).
template <bool SYM>
__global__ void __launch_bounds__(512, SYM ? 2 : 4) k_apply15_mom32(DevGrid g, const float* __restrict__ x,
                                                                   float* __restrict__ y,
                                                                   const float* __restrict__ coef, uint16_t dmask) {
  KCOUNT();
  __shared__ __align__(16) float cf[15 * DBV];
  __shared__ float4 tile[TILE3];
  __shared__ __align__(8) uint64_t bar;
  const int b = blockIdx.x, t = threadIdx.x;
  const int32_t c0 = g.cwo[16 * b];
  if (t < 32) {
    const uint32_t bytes = uint32_t(g.cwo[16 * (b + 1)] - c0) * 4u;   // a multiple of 16, at most 2 KB
    if (t == 0) {
      mbar_init(&bar);
      mbar_arrive_expect_tx(&bar, 15u * bytes);
    }
    __syncwarp();
    if (t < 15 && bytes) bulk_g2s(cf + t * DBV, coef + (int64_t)t * g.ncomp + c0, bytes, &bar);
  }
  const int64_t s = (int64_t)b * DBV + t;
  const uint16_t m = g.meta[s];
  const int ti = tile_index(t & 7, (t >> 3) & 7, t >> 6);
  int hnb = 13, hli = 0, hti = 0;
  if (t < HALO15) halo15(t, hnb, hli, hti);
  float vo[3], vh[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int c = 0; c < 3; ++c) vo[c] = x[(int64_t)c * g.nslots + s];
  if (t < HALO15) {
    const int nb = g.bnbr[27 * b + hnb];
    if (nb >= 0) {
      const int64_t hs = (int64_t)nb * DBV + hli;
#pragma unroll
      for (int c = 0; c < 3; ++c) vh[c] = x[(int64_t)c * g.nslots + hs];
    }
  }
  tile[ti] = make_float4(vo[0], vo[1], vo[2], 0.f);
  if (t < HALO15) tile[hti] = make_float4(vh[0], vh[1], vh[2], 0.f);
  const bool valid = (m & D_VALID) != 0;
  const int32_t r = compact_index(g, b, t, valid) - c0;
  // one thread waits for the copies (every thread spinning on the mbarrier
  // would crowd the shared-memory pipe); the CTA barrier then orders the
  // copied coefficients before every thread's reads
  if (t == 0) mbar_wait_or_flag(&bar, 0, g.aerr + g.binst[b]);
  __syncthreads();
  float out[3] = {0.f, 0.f, 0.f};
  const bool act = valid && !(m & dmask);
  if (act) {
#pragma unroll
    for (int k = 0; k < 15; ++k) {
      const float ck = cf[k * DBV + r];
      const float4 v = tile[ti + c_toff[k]];
      out[0] += ck * v.x;
      out[1] += ck * v.y;
      out[2] += ck * v.z;
    }
  }
  if constexpr (SYM)
    with_mask(act ? (m & 0xFF) : 0, [&](auto mk) {
      if (!act) return;
      const int inst = g.binst[b];
      add_transpose<float>(mk, stencil_factors<float>(g, b), float(g.pdt[inst] * g.pnu[inst]),
                           [&](int k, float (&v)[3]) {
                             const float4 t4 = tile[ti + c_toff[k]];
                             v[0] = t4.x;
                             v[1] = t4.y;
                             v[2] = t4.z;
                           },
                           out);
    });
  if (valid) {   // brick padding stays zero: no store
#pragma unroll
    for (int c = 0; c < 3; ++c) y[(int64_t)c * g.nslots + s] = out[c];
  }
}

// y_i(a) -= dt nu sum_e w_e x_j(b_e) on the natural boundary rows of the
// symmetric viscous form (outlet and pressure-inlet faces), one thread per
// row; runs after the stencil apply and before the interface sums.
template <typename T>
__global__ void k_natural_bterm(DevGrid g, const T* __restrict__ x, T* __restrict__ y) {
  KCOUNT();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.n_nat) return;
  const int32_t a = g.nat_slot[r];
  const int inst = g.binst[a / DBV];
  const T* w = sizeof(T) == 4 ? reinterpret_cast<const T*>(g.nat_w32) : reinterpret_cast<const T*>(g.nat_w64);
  T acc[3] = {T(0), T(0), T(0)};
  for (int e = g.nat_off[r]; e < g.nat_off[r + 1]; ++e) {
    const int ij = g.nat_comp[e];
    const int i = ij / 3, j = ij - 3 * (ij / 3);
    const T v = w[e] * x[(int64_t)j * g.nslots + g.nat_ent[e]];
    if (i == 0) acc[0] += v;
    else if (i == 1) acc[1] += v;
    else acc[2] += v;
  }
  const T dtnu = T(g.pdt[inst] * g.pnu[inst]);
#pragma unroll
  for (int i = 0; i < 3; ++i) y[(int64_t)i * g.nslots + a] -= dtnu * acc[i];
}

template <typename T, int NC, bool FUSEP = false>
static void launch_apply(const DevGrid& g, int op, const T* x, T* y, const T* coef, uint16_t dmask, int post,
                         KState* ks, RedBuf rb, cudaStream_t st, const T* zf = nullptr, T* pnew = nullptr) {
  // the Poisson operator is scalar; its CG form (fused direction update and
  // p.q) is k_poisson_cg<T, true>, launched by fe_apply_cg
  if (op == OP_POISSON) {
    if (!launch_p7<T, false>(g, x, (const T*)nullptr, (T*)nullptr, y, dmask, (KState*)nullptr, (double*)nullptr,
                             (unsigned*)nullptr, (const uint8_t*)nullptr, st))
      IBG_LAUNCH((k_poisson_cg<T, false>), g.nchunks, DBV, 0, st, g, x, (const T*)nullptr, (T*)nullptr, y, dmask,
                 (KState*)nullptr, (double*)nullptr, (unsigned*)nullptr, (const uint8_t*)nullptr);
  }
  else if (op == OP_MASS && FUSEP)
    IBG_LAUNCH((k_apply15<T, OP_MASS, NC, FUSEP, false>), g.nchunks, DBV, 0, st, g, x, y, coef, dmask, post, ks,
               rb.partials, rb.counter, zf, pnew);
  else if (op == OP_MASS)
    IBG_LAUNCH((k_apply15<T, OP_MASS, NC, FUSEP, true>), g.nbricks, DBV, 0, st, g, x, y, coef, dmask, post, ks,
               rb.partials, rb.counter, zf, pnew);
  else {
    if constexpr (sizeof(T) == 4 && NC == 3 && !FUSEP) {
      if (g.sym) IBG_LAUNCH(k_apply15_mom32<true>, g.nbricks, DBV, 0, st, g, x, y, coef, dmask);
      else IBG_LAUNCH(k_apply15_mom32<false>, g.nbricks, DBV, 0, st, g, x, y, coef, dmask);
    } else if (NC == 3 && g.sym) {
      IBG_LAUNCH((k_apply15<T, OP_COEF, NC, FUSEP, true, true>), g.nbricks, DBV, 0, st, g, x, y, coef, dmask, post,
                 ks, rb.partials, rb.counter, zf, pnew);
    } else {
      IBG_LAUNCH((k_apply15<T, OP_COEF, NC, FUSEP, true>), g.nbricks, DBV, 0, st, g, x, y, coef, dmask, post, ks,
                 rb.partials, rb.counter, zf, pnew);
    }
    if (NC == 3 && g.sym && g.n_nat > 0)
      IBG_LAUNCH(k_natural_bterm<T>, (g.n_nat + 127) / 128, 128, 0, st, g, x, y);
  }
}

template <typename T>
void fe_apply_cg(const DevGrid& g, const OpDesc<T>& A, int nc, const T* z, const T* pold, T* pnew, T* q, KState* ks,
                 RedBuf rb, cudaStream_t st) {
  if (nc == 1 && A.op == OP_POISSON) {
    if (!launch_p7<T, true>(g, z, pold, pnew, q, A.dmask, ks, rb.partials, rb.counter, (const uint8_t*)nullptr, st))
      IBG_LAUNCH((k_poisson_cg<T, true>), g.nchunks, DBV, 0, st, g, z, pold, pnew, q, A.dmask, ks, rb.partials,
                 rb.counter, (const uint8_t*)nullptr);
  }
  else if (nc == 1) launch_apply<T, 1, true>(g, A.op, pold, q, A.coef, A.dmask, POST_CG_ALPHA, ks, rb, st, z, pnew);
  else launch_apply<T, 3, true>(g, A.op, pold, q, A.coef, A.dmask, POST_CG_ALPHA, ks, rb, st, z, pnew);
}

template <typename T>
void fe_poisson_apply(const DevGrid& g, const T* x, T* q, uint16_t dmask, KState* ks, const uint8_t* on,
                      cudaStream_t st) {
  if (!launch_p7<T, false>(g, x, (const T*)nullptr, (T*)nullptr, q, dmask, ks, (double*)nullptr, (unsigned*)nullptr,
                           on, st))
    IBG_LAUNCH((k_poisson_cg<T, false>), g.nchunks, DBV, 0, st, g, x, (const T*)nullptr, (T*)nullptr, q, dmask, ks,
               (double*)nullptr, (unsigned*)nullptr, on);
}

template <typename T>
void fe_sync(const DevGrid& g, int nc, T* y, uint16_t dmask, cudaStream_t st) {
  if (g.n_if == 0) return;
  int bl = (g.n_if + 255) / 256;
  if (nc == 1) IBG_LAUNCH((k_sync<T, 1>), bl, 256, 0, st, g, y, dmask);
  else IBG_LAUNCH((k_sync<T, 3>), bl, 256, 0, st, g, y, dmask);
}

template <typename T>
void fe_expand2(const DevGrid& g, int nc, T* x, T* x2, cudaStream_t st) {
  if (g.n_hang == 0) return;
  int bl = (g.n_hang + 255) / 256;
  if (nc == 1) IBG_LAUNCH((k_expand<T, 1>), bl, 256, 0, st, g, x, x2);
  else IBG_LAUNCH((k_expand<T, 3>), bl, 256, 0, st, g, x, x2);
}

template <typename T>
void fe_expand(const DevGrid& g, int nc, T* x, cudaStream_t st) {
  fe_expand2<T>(g, nc, x, (T*)nullptr, st);
}

template <typename T>
void fe_apply_local(const DevGrid& g, const OpDesc<T>& A, int nc, const T* x, T* y, cudaStream_t st) {
  RedBuf none;
  if (nc == 1) launch_apply<T, 1>(g, A.op, x, y, A.coef, A.dmask, POST_NONE, nullptr, none, st);
  else launch_apply<T, 3>(g, A.op, x, y, A.coef, A.dmask, POST_NONE, nullptr, none, st);
}

template <typename T>
void fe_apply(const DevGrid& g, const OpDesc<T>& A, int nc, const T* x, T* y, cudaStream_t st) {
  RedBuf none;
  if (nc == 1) launch_apply<T, 1>(g, A.op, x, y, A.coef, A.dmask, POST_NONE, nullptr, none, st);
  else launch_apply<T, 3>(g, A.op, x, y, A.coef, A.dmask, POST_NONE, nullptr, none, st);
  fe_sync<T>(g, nc, y, A.dmask, st);
}

void fe_apply_resid(const DevGrid& g, const OpDesc<double>& A, int nc, const double* x, double* y,
                    const float* chi, const float* clo, cudaStream_t st) {
  const float* none = nullptr;
  if (A.op == OP_POISSON && nc == 1)
    IBG_LAUNCH(k_apply_ff<OP_POISSON>, g.nbricks, DBV, 0, st, g, x, y, none, none, A.dmask);
  else if (A.op == OP_MASS && nc == 3)
    IBG_LAUNCH(k_apply_ff<OP_MASS>, g.nbricks, DBV, 0, st, g, x, y, none, none, A.dmask);
  else if (A.op == OP_COEF && nc == 3 && !g.sym && chi && clo)
    IBG_LAUNCH(k_apply_ff<OP_COEF>, g.nbricks, DBV, 0, st, g, x, y, chi, clo, A.dmask);
  else {
    fe_apply<double>(g, A, nc, x, y, st);
    return;
  }
  fe_sync<double>(g, nc, y, A.dmask, st);
}

template <typename T>
void fe_jacobi(const DevGrid& g, int op, const T* coef, uint16_t dmask, T* diag, T* dinv, cudaStream_t st) {
  if (op == OP_POISSON) IBG_LAUNCH((k_diag<T, OP_POISSON>), g.nbricks, DBV, 0, st, g, coef, diag);
  else if (op == OP_MASS) IBG_LAUNCH((k_diag<T, OP_MASS>), g.nbricks, DBV, 0, st, g, coef, diag);
  else IBG_LAUNCH((k_diag<T, OP_COEF>), g.nbricks, DBV, 0, st, g, coef, diag);
  fe_sync<T>(g, 1, diag, 0, st);
  IBG_LAUNCH((k_dinv<T>), g.nbricks, DBV, 0, st, g, diag, dinv, dmask);
}

void fe_cast_d2f(int64_t n, const double* a, float* b, cudaStream_t st) { IBG_LAUNCH(k_cast_d2f, nblk(n), 256, 0, st, n, a, b); }
void fe_add_f2d(int64_t n, const float* a, double* b, cudaStream_t st) { IBG_LAUNCH(k_add_f2d, nblk(n), 256, 0, st, n, a, b); }
void fe_copy_d(int64_t n, const double* a, double* b, cudaStream_t st) { IBG_LAUNCH(k_copy_d, nblk(n), 256, 0, st, n, a, b); }
void fe_add_d(int64_t n, const double* a, double* b, cudaStream_t st) { IBG_LAUNCH(k_add_d, nblk(n), 256, 0, st, n, a, b); }
template <typename T>
void fe_zero(int64_t n, T* a, cudaStream_t st) { IBG_LAUNCH((k_zero<T>), nblk(n), 256, 0, st, n, a); }

void fe_rhs_mass_grad(const DevGrid& g, const double* u, const double* p, double* out, cudaStream_t st, bool pairs) {
  if (pairs) IBG_LAUNCH(k_rhs_mass_grad_ff, g.nbricks, DBV, 0, st, g, u, p, out);
  else IBG_LAUNCH(k_rhs_mass_grad, g.nbricks, DBV, 0, st, g, u, p, out);
}
void fe_rhs_div(const DevGrid& g, const double* u, double* out, cudaStream_t st, bool pairs) {
  if (pairs) IBG_LAUNCH(k_rhs_div_ff, g.nbricks, DBV, 0, st, g, u, out);
  else IBG_LAUNCH(k_rhs_div, g.nbricks, DBV, 0, st, g, u, out);
}
cudaError_t fe_configure() {
  // four 46 KB CTAs per SM: prefer the largest shared-memory carveout
  cudaError_t e = cudaFuncSetAttribute(k_apply15_mom32<false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       int(cudaSharedmemCarveoutMaxShared));
  if (e != cudaSuccess) return e;
  for (auto k : {k_poisson7_staged<true>, k_poisson7_staged<false>, k_poisson7_persist<true>,
                 k_poisson7_persist<false>}) {
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  int(cudaSharedmemCarveoutMaxShared))) != cudaSuccess)
      return e;
    const size_t mx = std::max(std::max(p7_smem<1>(), p7_smem<2>()), std::max(p7p_smem<1>(), p7p_smem<2>()));
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(mx))) != cudaSuccess)
      return e;
  }
  return cudaFuncSetAttribute(k_apply15_mom32<true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              int(cudaSharedmemCarveoutMaxShared));
}

void fe_momentum_coef_ff(const DevGrid& g, const double* u, float* coef32, float* coeflo, cudaStream_t st) {
  IBG_LAUNCH(k_mom_coef_ff, g.nbricks, DBV, 0, st, g, u, coef32, coeflo);
}

void fe_momentum_coef(const DevGrid& g, const double* u, double* coef64, float* coef32, cudaStream_t st) {
  // the mixed path (coef32 given) evaluates the convection part in FP32
  if (coef32) IBG_LAUNCH(k_mom_coef<float>, g.nbricks, DBV, 0, st, g, u, coef64, coef32);
  else IBG_LAUNCH(k_mom_coef<double>, g.nbricks, DBV, 0, st, g, u, coef64, coef32);
}

template <typename T>
void fe_gather_canon(int64_t N, const int32_t* cs, int nc, int64_t nslots, const T* x, T* out, cudaStream_t st) {
  IBG_LAUNCH((k_gather_canon<T>), nblk(N), 256, 0, st, N, cs, nc, nslots, x, out);
}
void fe_scatter_canon(const DevGrid& g, int64_t N, const int32_t* cs, int nc, const double* in, double* x,
                      cudaStream_t st) {
  IBG_LAUNCH(k_scatter_canon, nblk(N), 256, 0, st, N, cs, nc, g.nslots, in, x);
  if (g.n_if) IBG_LAUNCH(k_copy_to_fine, (g.n_if + 255) / 256, 256, 0, st, g, nc, x);
  fe_expand<double>(g, nc, x, st);
}

void fe_set_pinlet(int64_t n, const int32_t* slot, const int32_t* port, const PortDev* ports, const double* t,
                   const double* p, double* phi, cudaStream_t st) {
  IBG_LAUNCH(k_set_pinlet, nblk(n), 256, 0, st, n, slot, port, ports, t, p, phi);
}
void fe_set_inlet(int64_t n, const int32_t* slot, const int32_t* port, const double* shape, const PortDev* ports,
                  const double* t, int64_t nslots, double* u, cudaStream_t st) {
  if (n == 0) return;
  IBG_LAUNCH(k_set_inlet, nblk(n), 256, 0, st, n, slot, port, shape, ports, t, nslots, u);
}
void fe_time_advance(double* tc, double* tn, const double* dt, int n, int commit, const int32_t* ok,
                     cudaStream_t st) {
  IBG_LAUNCH(k_time, (n + 127) / 128, 128, 0, st, tc, tn, dt, n, commit, ok);
}

// explicit instantiations
template void fe_apply<double>(const DevGrid&, const OpDesc<double>&, int, const double*, double*, cudaStream_t);
template void fe_apply<float>(const DevGrid&, const OpDesc<float>&, int, const float*, float*, cudaStream_t);
template void fe_jacobi<double>(const DevGrid&, int, const double*, uint16_t, double*, double*, cudaStream_t);
template void fe_jacobi<float>(const DevGrid&, int, const float*, uint16_t, float*, float*, cudaStream_t);
template void fe_zero<double>(int64_t, double*, cudaStream_t);
template void fe_zero<float>(int64_t, float*, cudaStream_t);
template void fe_expand<double>(const DevGrid&, int, double*, cudaStream_t);
template void fe_expand2<double>(const DevGrid&, int, double*, double*, cudaStream_t);
template void fe_expand2<float>(const DevGrid&, int, float*, float*, cudaStream_t);
template void fe_apply_cg<double>(const DevGrid&, const OpDesc<double>&, int, const double*, const double*, double*,
                                  double*, KState*, RedBuf, cudaStream_t);
template void fe_apply_cg<float>(const DevGrid&, const OpDesc<float>&, int, const float*, const float*, float*,
                                 float*, KState*, RedBuf, cudaStream_t);
template void fe_expand<float>(const DevGrid&, int, float*, cudaStream_t);
template void fe_apply_local<float>(const DevGrid&, const OpDesc<float>&, int, const float*, float*, cudaStream_t);
template void fe_apply_local<double>(const DevGrid&, const OpDesc<double>&, int, const double*, double*,
                                     cudaStream_t);
template void fe_poisson_apply<float>(const DevGrid&, const float*, float*, uint16_t, KState*, const uint8_t*,
                                      cudaStream_t);
template void fe_poisson_apply<double>(const DevGrid&, const double*, double*, uint16_t, KState*, const uint8_t*,
                                       cudaStream_t);
template void fe_sync<double>(const DevGrid&, int, double*, uint16_t, cudaStream_t);
template void fe_sync<float>(const DevGrid&, int, float*, uint16_t, cudaStream_t);
template void fe_gather_canon<double>(int64_t, const int32_t*, int, int64_t, const double*, double*, cudaStream_t);

}  // namespace ibg
