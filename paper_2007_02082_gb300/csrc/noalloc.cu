// Allocation-free field read of a parked problem.
//
// ib_fields_get on a deferred handle that no batch holds gathers the stored
// node copies of U, P or Phi into canonical node order in a temporary device
// buffer, then copies that buffer out.  The variant here gathers into a fixed
// scratch array that belongs to this module instead, so the read needs no
// device allocation.
//
// Setup: the first call on a device, with that device current, resolves the
// scratch's device address with cudaGetSymbolAddress (which can load this
// module's device code on that device) and keeps it for later calls.
//
// Zero state: none.  The gather writes every scratch value that the copy out
// reads, within the same call; nothing has to start at zero.
//
// Overlap: there is one scratch array per device in a process.  Two calls that
// overlapped in time on one device would race on it, so every call holds a
// process-wide lock from the gather until its copy out has completed.
#include <mutex>

#include "noalloc.hpp"

namespace ibg {

namespace {

constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_noalloc_scratch[NOALLOC_MAX_VALUES];

std::mutex g_noalloc_mu;               // guards g_scratch_ptr and every use of the scratch
double* g_scratch_ptr[kMaxDevices] = {};

__global__ void k_gather_canon_scratch(int64_t N, const int32_t* __restrict__ cs, int nc, int64_t nslots,
                                       const double* __restrict__ x, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    for (int c = 0; c < nc; ++c) out[i * nc + c] = x[c * nslots + cs[i]];
}

// Scratch address on the current device (resolved once per device).
ib_status scratch_on_current_device(double** out, std::string& err) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { err = std::string("cudaGetDevice: ") + cudaGetErrorString(e); return IB_ECUDA; }
  if (dev < 0 || dev >= kMaxDevices) { err = "device index out of range for the no-allocation scratch"; return IB_EINVAL; }
  if (!g_scratch_ptr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      err = std::string("cudaGetSymbolAddress of the no-allocation scratch: ") + cudaGetErrorString(e);
      return IB_ECUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return IB_OK;
}

}  // namespace

ib_status noalloc_gather_canon(int64_t N, const int32_t* canon, int nc, int64_t nslots, const double* src,
                               void* dst, size_t bytes, int dst_on_device, cudaStream_t st, std::string& err) {
  if (N < 0 || nc < 1 || int64_t(bytes) != int64_t(nc) * N * 8) { err = "bad size"; return IB_EINVAL; }
  if (int64_t(nc) * N > NOALLOC_MAX_VALUES) {
    err = "field of " + std::to_string(int64_t(nc) * N) + " values exceeds the no-allocation scratch of " +
          std::to_string(NOALLOC_MAX_VALUES) + " doubles (8 MiB); read it with ib_fields_get";
    return IB_EINVAL;
  }
  if (N == 0) return IB_OK;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  double* scratch = nullptr;
  ib_status s = scratch_on_current_device(&scratch, err);
  if (s != IB_OK) return s;
  const int threads = 256;
  const int64_t want = (N + threads - 1) / threads;
  const int blocks = int(want < 65536 ? want : 65536);
  k_gather_canon_scratch<<<blocks, threads, 0, st>>>(N, canon, nc, nslots, src, scratch);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dst, scratch, bytes, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { err = std::string("no-allocation field read: ") + cudaGetErrorString(e); return IB_ECUDA; }
  return IB_OK;
}

}  // namespace ibg
