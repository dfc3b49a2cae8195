// Device-driven loops inside CUDA graphs.
//
// A Krylov loop whose trip count is decided on the device is captured as a
// conditional WHILE node: the body is captured on a side stream into the
// node's body graph, and kernels in the body set the loop condition with
// cudaGraphSetConditional.  When the stream is not capturing, the same body is
// run by a host loop that polls a device flag instead (profiling path).
#pragma once

#include <cuda_runtime.h>

#include <vector>

namespace ibg {

// Handle passed to kernels that decide a loop condition.
struct Cond {
  cudaGraphConditionalHandle h = 0;
  int use = 0;   // 0: not inside a graph (host-driven loop)
};

__device__ __forceinline__ void set_cond(const Cond& c, bool v) {
  if (c.use) cudaGraphSetConditional(c.h, v ? 1u : 0u);
}

// Side streams for nested body captures (one per nesting depth).
struct CaptureCtx {
  bool capturing = false;
  std::vector<cudaStream_t> side;
  int depth = 0;
  cudaError_t err = cudaSuccess;
  cudaStream_t next() { return side[depth]; }
};

inline bool stream_capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  return cs == cudaStreamCaptureStatusActive;
}

// New conditional handle in the graph that `st` is capturing into.
inline cudaError_t cond_handle(cudaStream_t st, unsigned defval, Cond* out) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, nullptr, nullptr, nullptr);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  out->use = 1;
  return cudaGraphConditionalHandleCreate(&out->h, graph, defval, cudaGraphCondAssignDefault);
}

// Append a conditional node (WHILE or IF) to the capture of `st` and capture
// body(s) into its body graph on the side stream of the current depth.
template <typename F>
cudaError_t cond_node(CaptureCtx& cc, cudaStream_t st, const Cond& c, cudaGraphConditionalNodeType type,
                      F&& body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t graph = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, &deps, &ed, &nd);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = c.h;
  np.conditional.type = type;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if ((e = cudaGraphAddNode(&node, graph, deps, ed, nd, &np)) != cudaSuccess) return e;
  cudaGraph_t bg = np.conditional.phGraph_out[0];
  if (cc.depth >= int(cc.side.size())) return cudaErrorInvalidValue;
  cudaStream_t s = cc.side[cc.depth];
  if ((e = cudaStreamBeginCaptureToGraph(s, bg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
    return e;
  cc.depth++;
  body(s);
  cc.depth--;
  cudaGraph_t out = nullptr;
  e = cudaStreamEndCapture(s, &out);
  if (e != cudaSuccess) return e;
  return cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

}  // namespace ibg
