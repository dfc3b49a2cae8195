// Device-side view of the composite grid and shared helpers.
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

namespace ibg {

// Every kernel launch of the library goes through launch_kernel, which counts
// it (ib_info.kernel_launches).  Launches allow programmatic dependent launch:
// a kernel's CTAs may be scheduled while the previous kernel on the stream
// drains, and every kernel waits at its first statement (KCOUNT) until the
// previous one has completed and its writes are visible.  This hides the
// launch gap between the many short kernels of a step.
extern std::atomic<long long> g_launches;

template <typename... KArgs, typename... Args>
inline void launch_kernel(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                          Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}
// Every kernel starts with KCOUNT(): the wait for the previous kernel of the
// stream (programmatic dependent launch), then the device-side count of
// executed kernels, one relaxed atomic from thread 0 of block 0 (one counter
// per translation unit).  (An explicit early trigger, letting the next
// kernel's CTAs take SMs as this one's last CTAs drain, measured slower: 56.0
// against 51.9 ms for a batched step of 8 serving requests.)
#define IBG_KCOUNT_DEFINE static __device__ unsigned long long g_kcount = 0ULL;
#define KCOUNT()                                                  \
  do {                                                            \
    asm volatile("griddepcontrol.wait;" ::: "memory");            \
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&g_kcount, 1ULL); \
  } while (0)

// A cooperative launch (every CTA resident at once, for kernels whose CTAs
// wait on one another), without programmatic dependent launch.
template <typename... KArgs, typename... Args>
inline void launch_cooperative(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                               Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

#define IBG_LAUNCH(k, grid, block, smem, st, ...) \
  ::ibg::launch_kernel(k, dim3(grid), dim3(block), size_t(smem), st, __VA_ARGS__)

constexpr int DBS = 8;          // brick edge (nodes)
constexpr int DBV = 512;        // nodes per brick = threads per brick CTA
constexpr int TILE = 10;        // brick plus a one-node halo
constexpr int TILE3 = 1000;
constexpr int SF_STRIDE = 16;   // stencil factors per instance and level

// Brick padding: a slot without D_VALID (no active leaf cell of its level
// touches it) is zero in every vector of the library.  Every kernel writes only
// zeros there or skips it, so the streaming kernels neither read nor write
// such slots.
//
// per-slot metadata bits (mirror of setup.hpp)
constexpr uint16_t D_VALID = 1u << 8, D_HANG = 1u << 9, D_DUP = 1u << 10,
                   D_VDIR = 1u << 11, D_PDIR = 1u << 12, D_IFACE = 1u << 13;
// bits 14-15: 1 + the normal axis of a port node whose tangential velocity
// components are Dirichlet (zero); the normal component stays free
constexpr uint16_t D_TAX = 3u << 14;
// component c of a velocity solve (dmask holds D_VDIR) is Dirichlet at a
// slot with metadata m through the tangential port condition
__device__ __forceinline__ bool tan_dir(uint16_t m, uint16_t dmask, int c) {
  const int ax = (m >> 14) & 3;
  return (dmask & D_VDIR) && ax != 0 && c != ax - 1;
}

// One or several problem instances stored side by side: every brick belongs to
// one instance, and the bricks of an instance are contiguous
// ([bseg[i], bseg[i+1])), so reductions are segmented per instance.
struct DevGrid {
  int32_t nbricks;
  int64_t nslots;
  int32_t ninst;
  const int32_t* __restrict__ blev;   // [nbricks]
  const int32_t* __restrict__ binst;  // [nbricks] instance of each brick
  const int32_t* __restrict__ bseg;   // [ninst + 1] brick range of each instance
  const int32_t* __restrict__ bnbr;   // [nbricks][27]
  // chunks: runs of up to 8 consecutive bricks of one instance, one CTA each
  // for the streaming Krylov kernels; cseg gives each instance's chunk range
  int32_t nchunks;
  const int32_t* __restrict__ cbrick; // [nchunks + 1] first brick of each chunk
  const int32_t* __restrict__ cseg;   // [ninst + 1]
  // streaming chunks for the per-slot kernels (no halo): runs of up to 8
  // bricks (measured best of 4, 8 and 16 on the refined 64x64x256 tube)
  int32_t nschunks;
  const int32_t* __restrict__ scbrick; // [nschunks + 1]
  const int32_t* __restrict__ scseg;   // [ninst + 1]
  const uint16_t* __restrict__ meta;  // [nslots]
  const double* __restrict__ hl;      // [ninst][4][3] cell spacing per instance and level
  // stencil factors per instance and level, [ninst][4][SF_STRIDE]:
  //   (V/6)/hx^2, (V/6)/hy^2, (V/6)/hz^2, V/120, (V/24)/hx, (V/24)/hy, (V/24)/hz, 0,
  //   (V/6)/(hx hy), (V/6)/(hy hz), (V/6)/(hx hz), 0 ...
  const double* __restrict__ sf64;
  const float* __restrict__ sf32;
  const double* __restrict__ pdt;     // [ninst] time step
  const double* __restrict__ pnu;     // [ninst] kinematic viscosity
  // nodes stored on two levels: coarse owner, fine copy, hanging children
  int32_t n_if;
  const int32_t* __restrict__ if_c;
  const int32_t* __restrict__ if_f;
  const int32_t* __restrict__ if_off;
  const int32_t* __restrict__ if_kid;
  const int32_t* __restrict__ if_of_slot;   // [nslots] entry of an interface copy
  // hanging nodes and their parents (fine-level slots)
  int32_t n_hang;
  const int32_t* __restrict__ hg;
  const int32_t* __restrict__ hp1;
  const int32_t* __restrict__ hp2;
  // compact per-slot arrays (valid slots only, brick by brick): cwo[16 b + w]
  // is the index of the first valid slot of warp w of brick b; a brick's run
  // starts on a multiple of 4 entries (16 bytes in FP32) and ends where the
  // next brick's starts; cwo[16 nbricks] = ncomp, the plane stride
  const int32_t* __restrict__ cwo;    // [16 (nbricks + 1)]
  int64_t ncomp;
  // per-instance error word of the step (ASYNC_TIMEOUT when a bounded wait ran out)
  int32_t* aerr;                      // [ninst]
  // symmetric viscous form (every instance): transpose-gradient couplings in
  // the momentum operator and the natural boundary term on outlet and
  // pressure-inlet rows (row r: slot nat_slot[r], entries nat_off[r] ..
  // nat_off[r+1], trial slot nat_ent, 3 test + trial component nat_comp)
  int32_t sym;
  int32_t n_nat;
  const int32_t* __restrict__ nat_slot;
  const int32_t* __restrict__ nat_off;
  const int32_t* __restrict__ nat_ent;
  const int8_t* __restrict__ nat_comp;
  const double* __restrict__ nat_w64;
  const float* __restrict__ nat_w32;
  // launch choice: 2 selects the register-pipelined FP32 Poisson stencil, 3
  // the persistent staged one
  int32_t poisson_kernel;
  // schedule of the persistent Poisson stencil (launch choice 3): p7_ctas CTAs (a whole
  // number of CTAs per SM); CTA c walks the chunks c, c + p7_ctas, ... and
  // their bricks, one 64-byte P7Hdr per brick in that order, positions
  // [p7_off[c], p7_off[c + 1])
  int32_t p7_ctas;
  const int32_t* __restrict__ p7_off;   // [p7_ctas + 1]
  const int4* __restrict__ p7_hdr;      // [nbricks][4]
};

// Per brick of the persistent Poisson schedule: the brick, its face neighbours
// (-x, +x, -y, +y, -z, +z; -1 where missing), its instance, its chunk and
// whether it is the chunk's last brick, and the FP32 stencil factors
// (V/6)/h_a^2 of its level.  Written once per grid by the host.
struct P7Hdr {
  int32_t b, nb[6], inst;
  int32_t chunk, last, pad0, pad1;
  float fac[3], pad2;
};
static_assert(sizeof(P7Hdr) == 64, "P7Hdr is four 16-byte pieces");

// Index in the compact arrays of thread t's slot of brick b (a valid slot);
// every lane of the warp must call it (warp ballot).
__device__ __forceinline__ int32_t compact_index(const DevGrid& g, int b, int t, bool valid) {
  const unsigned bal = __ballot_sync(0xffffffffu, valid);
  unsigned lt;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
  return g.cwo[16 * b + (t >> 5)] + __popc(bal & lt);
}

// Krylov scalars of one right-hand side (one velocity component or Phi).
struct KState {
  double rz, rz_new, pq, alpha, beta, rr, bb, tol2;
  double rho, omega, rv, ts, tt;
  int32_t iter, max_iter, done, status;   // status: 0 ok, 4 no convergence, 5 breakdown
  float af, bf, of;                       // alpha, beta, omega rounded once for FP32 kernels
  float pad;
};

// scalar of KState in the kernel's precision (FP32 kernels read the mirror)
template <typename T> __device__ __forceinline__ T k_alpha(const KState& k) {
  if constexpr (sizeof(T) == 4) return k.af; else return k.alpha;
}
template <typename T> __device__ __forceinline__ T k_beta(const KState& k) {
  if constexpr (sizeof(T) == 4) return k.bf; else return k.beta;
}
template <typename T> __device__ __forceinline__ T k_omega(const KState& k) {
  if constexpr (sizeof(T) == 4) return k.of; else return k.omega;
}

// FP64 defect-correction loop around an inner solve (mixed precision).
struct OState {
  double ref[3];     // max(||b||^2, ||r_0||^2) per component, set on the first pass
  int32_t sexp[3];   // the pass's inner right-hand side is r * 2^-sexp (norm in [0.5, 1))
  int32_t spad;
  double rel2;       // max_c ||r||^2 / ref
  double prev2;      // rel2 of the previous pass
  double tol2;
  int32_t iter, max_iter, done, status, inner_status, nc;
};

// Per-solve record of a step, read by the host after the step.
struct SolveRec {
  int32_t iters[3];
  int32_t status;
  int32_t outer;
  int32_t pad;
  double relres;
};

__device__ __forceinline__ int tile_index(int lx, int ly, int lz) {   // l in [-1, 8]
  return ((lz + 1) * TILE + (ly + 1)) * TILE + (lx + 1);
}

// Load x (ncomp components, component stride cs) of this brick plus a one-node
// halo into tile[c*1000 + ...]; missing neighbours read as zero.
template <typename T>
__device__ __forceinline__ void load_tile(T* tile, const T* __restrict__ x, int64_t cs, int ncomp,
                                          const int32_t* __restrict__ nb27) {
  for (int t = threadIdx.x; t < TILE3; t += blockDim.x) {
    int hx = t % TILE, hy = (t / TILE) % TILE, hz = t / (TILE * TILE);
    int lx = hx - 1, ly = hy - 1, lz = hz - 1;
    int ox = lx < 0 ? -1 : (lx > 7 ? 1 : 0);
    int oy = ly < 0 ? -1 : (ly > 7 ? 1 : 0);
    int oz = lz < 0 ? -1 : (lz > 7 ? 1 : 0);
    int nb = nb27[(oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)];
    int64_t s = (int64_t)nb * DBV + (((lz & 7) * DBS + (ly & 7)) * DBS + (lx & 7));
    for (int c = 0; c < ncomp; ++c) tile[c * TILE3 + t] = nb >= 0 ? x[c * cs + s] : T(0);
  }
}

template <typename T>
__device__ __forceinline__ const T* stencil_factors(const DevGrid& g, int b) {
  const int idx = (g.binst[b] * 4 + g.blev[b]) * SF_STRIDE;
  if constexpr (sizeof(T) == 4) return reinterpret_cast<const T*>(g.sf32) + idx;
  else return reinterpret_cast<const T*>(g.sf64) + idx;
}

// Block-wide sum of NV values of type T (blockDim.x a multiple of 32, <= 1024);
// the total is valid in thread 0.
template <typename T, int NV>
__device__ __forceinline__ void block_sum(T (&v)[NV], T* sh /* [32*NV] */) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  __syncthreads();
  if (lane == 0)
    for (int k = 0; k < NV; ++k) sh[k * 32 + w] = v[k];
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      v[k] = lane < nw ? sh[k * 32 + lane] : T(0);
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
  }
}

// The second half of grid_sum_last, for kernels that write their partials
// themselves (partials[NV * p + k] for p over the instances' partial ranges
// seg[i] .. seg[i+1]): every CTA arrives once; the last one sums, for every
// instance, its partials in FP64 with all its threads (thread t takes the
// relative partials t, t + blockDim, ...; then a fixed tree) into
// out[i * NV + k], and returns true after a __syncthreads that makes out
// visible to all its threads.  The counter is reset.  The caller's partial
// writes must come from thread 0.
template <int NV>
__device__ __forceinline__ bool segment_sums_last(const double* __restrict__ partials, unsigned* __restrict__ counter,
                                                  const int32_t* __restrict__ seg, int nseg,
                                                  double* __restrict__ out) {
  __shared__ double shd[32 * NV];
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  for (int i = 0; i < nseg; ++i) {
    double acc[NV];
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    for (int64_t b = seg[i] + threadIdx.x; b < seg[i + 1]; b += blockDim.x)
      for (int k = 0; k < NV; ++k) acc[k] += __ldcg(partials + b * NV + k);
    block_sum<double, NV>(acc, shd);
    if (threadIdx.x == 0)
      for (int k = 0; k < NV; ++k) out[(int64_t)i * NV + k] = acc[k];
  }
  __threadfence_block();
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// Deterministic segmented grid reduction.  Every block sums its threads' NV
// contributions in the kernel's precision T (FP32 kernels: FP32 within the
// block; the GB300 FP64 rate would otherwise dominate) and writes the block
// totals in FP64; the last block to arrive sums, for every instance i, the
// partials of blocks [seg[i], seg[i+1]) in FP64 (segment_sums_last) and
// stores the totals in out[i * NV + k].  Returns true in that block only,
// after a __syncthreads that makes out visible to all its threads.  The
// counter is reset.  An instance's totals depend only on its own blocks and
// their order, so they are bitwise the same alone and next to other instances.
template <typename T, int NV>
__device__ __forceinline__ bool grid_sum_last(T (&v)[NV], double* __restrict__ partials,
                                              unsigned* __restrict__ counter, const int32_t* __restrict__ seg,
                                              int nseg, double* __restrict__ out) {
  __shared__ T sht[32 * NV];
  block_sum<T, NV>(v, sht);
  if (threadIdx.x == 0)
    for (int k = 0; k < NV; ++k) partials[(int64_t)blockIdx.x * NV + k] = double(v[k]);
  return segment_sums_last<NV>(partials, counter, seg, nseg, out);
}

}  // namespace ibg
