// Device rebuild of the immersed-boundary structures after the Lagrangian
// points move (see ibmove.hpp).  Counts use atomics; the order of every list is
// then fixed by sorting it, so the result does not depend on the atomics.
#include "device.cuh"
#include "ibmove.hpp"

namespace ibg {

IBG_KCOUNT_DEFINE
unsigned long long move_kcount() {
  unsigned long long v = 0;
  cudaMemcpyFromSymbol(&v, g_kcount, sizeof(v));
  return v;
}

// ---------------------------------------------------------------- scan
constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// out[i] = sum of in[0..i-1] within the tile for i in [0, n] (in[n] reads as 0);
// sums[tile] = the tile's total
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tile(const int32_t* __restrict__ in, int32_t* __restrict__ out,
                                                           int64_t n, int32_t* __restrict__ sums) {
  KCOUNT();
  __shared__ int32_t wsum[SCAN_THREADS / 32];
  const int t = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)t * SCAN_ITEMS;
  int32_t v[SCAN_ITEMS];
  int32_t run = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const int64_t i = base + k;
    v[k] = (i < n) ? in[i] : 0;
    run += v[k];
  }
  // inclusive warp scan of the thread totals
  const int lane = t & 31, warp = t >> 5;
  int32_t inc = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int32_t w = lane < SCAN_THREADS / 32 ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < SCAN_THREADS / 32) wsum[lane] = w;   // inclusive over warps
  }
  __syncthreads();
  int32_t acc = inc - run + (warp > 0 ? wsum[warp - 1] : 0);
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const int64_t i = base + k;
    if (i <= n) out[i] = acc;
    acc += v[k];
  }
  if (t == SCAN_THREADS - 1) sums[blockIdx.x] = acc;
}

__global__ void k_scan_add(int32_t* __restrict__ out, int64_t n, const int32_t* __restrict__ offs) {
  KCOUNT();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= n) out[i] += offs[i / SCAN_TILE];
}

static int64_t ntiles(int64_t n) { return (n + 1 + SCAN_TILE - 1) / SCAN_TILE; }   // n + 1 outputs

int64_t scan_scratch_len(int64_t n) {
  int64_t len = 0;
  for (int64_t t = ntiles(n); t > 1; t = ntiles(t)) len += 2 * (t + 1);
  return len + 4;
}

void scan_excl(const int32_t* in, int32_t* out, int64_t n, int32_t* scratch, cudaStream_t st) {
  const int64_t nt = ntiles(n);
  int32_t* sums = scratch;                 // nt tile totals
  int32_t* offs = scratch + (nt + 1);      // their exclusive scan (nt + 1)
  IBG_LAUNCH(k_scan_tile, unsigned(nt), SCAN_THREADS, 0, st, in, out, n, sums);
  if (nt == 1) return;
  scan_excl(sums, offs, nt, scratch + 2 * (nt + 1), st);
  IBG_LAUNCH(k_scan_add, unsigned((n + 1 + 255) / 256), 256, 0, st, out, n, (const int32_t*)offs);
}

// ---------------------------------------------------------------- supports
__device__ __forceinline__ int64_t fdiv4(int64_t a) { return a >= 0 ? a / 4 : -((-a + 3) / 4); }

__global__ void k_mv_supports(MoveGrid G, int64_t M, const double* __restrict__ X, int32_t* __restrict__ org,
                              int32_t* __restrict__ slot, uint64_t* __restrict__ freeb, int32_t* __restrict__ err) {
  KCOUNT();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  int64_t o[3];
  bool inside = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double x = (X[3 * i + a] - G.origin[a]) / G.hf[a];
    if (!(x >= 0.0 && x <= double(G.nf[a]))) inside = false;
    o[a] = inside ? int64_t(floor(x)) - 1 : 0;
    org[3 * i + a] = int32_t(o[a]);
  }
  uint64_t fb = 0;
  int32_t code = inside ? MV_OK : MV_OUTSIDE;
  for (int a = 0; a < 64; ++a) {
    const int64_t q[3] = {o[0] + (a & 3), o[1] + ((a >> 2) & 3), o[2] + (a >> 4)};
    int32_t s = -1;
    if (inside && q[0] >= 0 && q[1] >= 0 && q[2] >= 0 && q[0] <= G.nf[0] && q[1] <= G.nf[1] && q[2] <= G.nf[2]) {
      const int64_t bx = q[0] / DBS, by = q[1] / DBS, bz = q[2] / DBS;
      const int32_t b = G.bmap[(bz * G.nb[1] + by) * G.nb[0] + bx];
      if (b >= 0) {
        const int64_t t = ((q[2] % DBS) * DBS + (q[1] % DBS)) * DBS + (q[0] % DBS);
        const int64_t sl = (int64_t)b * DBV + t;
        const uint16_t m = G.meta[sl];
        if (m & D_VALID) {
          if (m & (D_HANG | D_DUP)) code = max(code, int32_t(MV_COARSE));
          s = int32_t(sl);
          if (!(m & (D_VDIR | D_TAX))) fb |= uint64_t(1) << a;
        }
      }
      if (s < 0) {   // no finest-level node here: is it a vertex of an active coarser cell?
        const int64_t F = int64_t(1) << G.L;
        for (int c = 0; c < 8; ++c) {
          int64_t cc[3];
          bool ok = true;
          for (int d = 0; d < 3; ++d) {
            const int64_t lo = (c >> d) & 1;   // 0: cell holding q, 1: the cell below when q is on its face
            cc[d] = q[d] / F - lo;
            if (lo && q[d] % F != 0) ok = false;
            if (cc[d] < 0 || cc[d] >= G.n[d]) ok = false;
          }
          if (!ok) continue;
          const int lev = G.cell_level[(cc[2] * G.n[1] + cc[1]) * G.n[0] + cc[0]];
          if (lev >= G.L) continue;   // inactive (255) or finest
          const int64_t step = int64_t(1) << (G.L - lev);
          if (q[0] % step == 0 && q[1] % step == 0 && q[2] % step == 0) code = max(code, int32_t(MV_COARSE));
        }
      }
    }
    slot[64 * i + a] = s;
  }
  if (inside && fb == 0) code = max(code, int32_t(MV_NOFREE));
  freeb[i] = fb;
  if (code != MV_OK) atomicMax(err, code);
}

void mv_supports(const MoveGrid& G, int64_t M, const double* X, int32_t* org, int32_t* slot, uint64_t* freeb,
                 int32_t* err, cudaStream_t st) {
  if (M == 0) return;
  IBG_LAUNCH(k_mv_supports, unsigned((M + 127) / 128), 128, 0, st, G, M, X, org, slot, freeb, err);
}

// ---------------------------------------------------------------- A_F pattern
// bins of 4 finest cells; origins lie in [-1, nf], so bin coordinates in
// [-1, nf / 4], shifted by one
struct BinDims {
  int64_t d[3];
};
__host__ __device__ inline BinDims bin_dims(const MoveGrid& G) {
  BinDims b;
  for (int a = 0; a < 3; ++a) b.d[a] = G.nf[a] / 4 + 3;
  return b;
}
int64_t mv_nbins(const MoveGrid& G) {
  const BinDims b = bin_dims(G);
  return b.d[0] * b.d[1] * b.d[2];
}
__device__ __forceinline__ int64_t bin_of(const BinDims& B, const int32_t* o) {
  return ((fdiv4(o[2]) + 1) * B.d[1] + (fdiv4(o[1]) + 1)) * B.d[0] + (fdiv4(o[0]) + 1);
}

__global__ void k_mv_bin_count(MoveGrid G, int64_t M, const int32_t* __restrict__ org, int32_t* __restrict__ cnt) {
  KCOUNT();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  atomicAdd(cnt + bin_of(bin_dims(G), org + 3 * i), 1);
}

__global__ void k_mv_bin_fill(MoveGrid G, int64_t M, const int32_t* __restrict__ org,
                              const int32_t* __restrict__ start, int32_t* __restrict__ fill,
                              int32_t* __restrict__ pts) {
  KCOUNT();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const int64_t b = bin_of(bin_dims(G), org + 3 * i);
  pts[start[b] + atomicAdd(fill + b, 1)] = int32_t(i);
}

// rows i < M: the points k whose origins differ by at most 3 on every axis
// (overlapping supports); FILL writes them (then sorts the row), else counts
template <bool FILL>
__global__ void k_mv_af_rows(MoveGrid G, int64_t M, int64_t Mt, const int32_t* __restrict__ org,
                             const int32_t* __restrict__ start, const int32_t* __restrict__ pts,
                             int32_t* __restrict__ rcnt, const int32_t* __restrict__ rowptr,
                             int32_t* __restrict__ col) {
  KCOUNT();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Mt) return;
  if (i >= M) {
    if (!FILL) rcnt[i] = 0;
    return;
  }
  const BinDims B = bin_dims(G);
  const int32_t* oi = org + 3 * i;
  const int64_t bx = fdiv4(oi[0]) + 1, by = fdiv4(oi[1]) + 1, bz = fdiv4(oi[2]) + 1;
  int32_t n = 0;
  const int64_t r0 = FILL ? rowptr[i] : 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int64_t x = bx + dx, y = by + dy, z = bz + dz;
        if (x < 0 || y < 0 || z < 0 || x >= B.d[0] || y >= B.d[1] || z >= B.d[2]) continue;
        const int64_t b = (z * B.d[1] + y) * B.d[0] + x;
        for (int32_t e = start[b]; e < start[b + 1]; ++e) {
          const int32_t k = pts[e];
          const int32_t* ok = org + 3 * k;
          if (abs(ok[0] - oi[0]) > 3 || abs(ok[1] - oi[1]) > 3 || abs(ok[2] - oi[2]) > 3) continue;
          if (FILL) col[r0 + n] = k;
          ++n;
        }
      }
  if constexpr (!FILL) {
    rcnt[i] = n;
  } else {
    for (int a = 1; a < n; ++a) {   // insertion sort of the row (a few dozen entries)
      const int32_t v = col[r0 + a];
      int b = a - 1;
      while (b >= 0 && col[r0 + b] > v) {
        col[r0 + b + 1] = col[r0 + b];
        --b;
      }
      col[r0 + b + 1] = v;
    }
  }
}

void mv_af_count(const MoveGrid& G, int64_t M, int64_t Mt, const int32_t* org, int32_t* bins, int32_t* rcnt,
                 int32_t* rowptr, int32_t* scratch, cudaStream_t st) {
  const int64_t nb = mv_nbins(G);
  int32_t* cnt = bins;
  int32_t* start = bins + (nb + 1);
  int32_t* fill = bins + 2 * (nb + 1);
  int32_t* pts = bins + 3 * (nb + 1);
  cudaMemsetAsync(cnt, 0, (nb + 1) * sizeof(int32_t), st);
  cudaMemsetAsync(fill, 0, (nb + 1) * sizeof(int32_t), st);
  if (M) IBG_LAUNCH(k_mv_bin_count, unsigned((M + 255) / 256), 256, 0, st, G, M, (const int32_t*)org, cnt);
  scan_excl(cnt, start, nb, scratch, st);
  if (M) IBG_LAUNCH(k_mv_bin_fill, unsigned((M + 255) / 256), 256, 0, st, G, M, (const int32_t*)org,
                    (const int32_t*)start, fill, pts);
  if (Mt)
    IBG_LAUNCH(k_mv_af_rows<false>, unsigned((Mt + 127) / 128), 128, 0, st, G, M, Mt, (const int32_t*)org,
               (const int32_t*)start, (const int32_t*)pts, rcnt, (const int32_t*)nullptr, (int32_t*)nullptr);
  scan_excl(rcnt, rowptr, Mt, scratch, st);
}

void mv_af_fill(const MoveGrid& G, int64_t M, const int32_t* org, const int32_t* bins, const int32_t* rowptr,
                int32_t* col, cudaStream_t st) {
  if (M == 0) return;
  const int64_t nb = mv_nbins(G);
  const int32_t* start = bins + (nb + 1);
  const int32_t* pts = bins + 3 * (nb + 1);
  IBG_LAUNCH(k_mv_af_rows<true>, unsigned((M + 127) / 128), 128, 0, st, G, M, M, org, start, pts,
             (int32_t*)nullptr, rowptr, col);
}

// ---------------------------------------------------------------- spreading lists
__global__ void k_mv_sp_count(int64_t M, const int32_t* __restrict__ slot, const uint64_t* __restrict__ freeb,
                              int32_t* __restrict__ cnt) {
  KCOUNT();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * 64) return;
  if (freeb[e >> 6] >> (e & 63) & 1) atomicAdd(cnt + slot[e], 1);
}

__global__ void k_mv_sp_fill(int64_t M, const int32_t* __restrict__ slot, const uint64_t* __restrict__ freeb,
                             const int32_t* __restrict__ start, int32_t* __restrict__ fill,
                             int32_t* __restrict__ ent) {
  KCOUNT();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * 64) return;
  if (!(freeb[e >> 6] >> (e & 63) & 1)) return;
  const int32_t s = slot[e];
  ent[start[s] + atomicAdd(fill + s, 1)] = int32_t(e);
}

// sort each slot's entries; flag the slots that have any
__global__ void k_mv_sp_sort(int64_t ns, const int32_t* __restrict__ start, int32_t* __restrict__ ent,
                             int32_t* __restrict__ flag) {
  KCOUNT();
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  const int32_t a0 = start[s], a1 = start[s + 1];
  flag[s] = a1 > a0 ? 1 : 0;
  for (int32_t a = a0 + 1; a < a1; ++a) {
    const int32_t v = ent[a];
    int32_t b = a - 1;
    while (b >= a0 && ent[b] > v) {
      ent[b + 1] = ent[b];
      --b;
    }
    ent[b + 1] = v;
  }
}

__global__ void k_mv_sp_compact(int64_t ns, const int32_t* __restrict__ start, const int32_t* __restrict__ flag,
                                const int32_t* __restrict__ idx, int32_t* __restrict__ sp_slot,
                                int32_t* __restrict__ sp_off) {
  KCOUNT();
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s > ns) return;
  if (s == ns) {
    sp_off[idx[ns]] = start[ns];
    return;
  }
  if (flag[s]) {
    sp_slot[idx[s]] = int32_t(s);
    sp_off[idx[s]] = start[s];
  }
}

void mv_spread(int64_t M, int64_t ns, const int32_t* slot, const uint64_t* freeb, int32_t* cnt, int32_t* start,
               int32_t* fill, int32_t* flag, int32_t* idx, int32_t* ent, int32_t* sp_slot, int32_t* sp_off,
               int32_t* scratch, cudaStream_t st) {
  cudaMemsetAsync(cnt, 0, (ns + 1) * sizeof(int32_t), st);
  cudaMemsetAsync(fill, 0, (ns + 1) * sizeof(int32_t), st);
  const unsigned ge = unsigned((M * 64 + 255) / 256), gs = unsigned((ns + 1 + 255) / 256);
  if (M) IBG_LAUNCH(k_mv_sp_count, ge, 256, 0, st, M, slot, freeb, cnt);
  scan_excl(cnt, start, ns, scratch, st);
  if (M) IBG_LAUNCH(k_mv_sp_fill, ge, 256, 0, st, M, slot, freeb, (const int32_t*)start, fill, ent);
  IBG_LAUNCH(k_mv_sp_sort, gs, 256, 0, st, ns, (const int32_t*)start, ent, flag);
  scan_excl(flag, idx, ns, scratch, st);
  IBG_LAUNCH(k_mv_sp_compact, gs, 256, 0, st, ns, (const int32_t*)start, (const int32_t*)flag,
             (const int32_t*)idx, sp_slot, sp_off);
}

}  // namespace ibg
