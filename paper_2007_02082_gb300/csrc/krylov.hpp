// Krylov solvers of the step (krylov.cu): PCG, BiCGStab and the FP64
// defect-correction loop of the mixed-precision path.  Every loop runs either
// as a conditional WHILE node of a captured CUDA graph (the device decides the
// trip count) or, when the stream is not capturing, as a host loop that polls
// the device state (used when kernel launches are timed individually).
#pragma once

#include "fe.hpp"
#include "graph.hpp"
#include "mgdev.hpp"

namespace ibg {

struct SolveArgs {
  const DevGrid* g = nullptr;
  int op = OP_POISSON;
  int nc = 1;
  uint16_t dmask = 0;
  bool bicg = false;       // BiCGStab (nonsymmetric) instead of CG
  bool mixed = false;      // FP32 iterations inside FP64 defect correction
  bool coupled = false;    // BiCGStab on the NC components as one system (shared scalars)
  const double* coef64 = nullptr;
  const double* dinv64 = nullptr;
  const float* coef32 = nullptr;
  const float* coeflo32 = nullptr;   // lo parts of the momentum coefficient pairs (mixed, gradient form)
  const float* dinv32 = nullptr;
  const double* b = nullptr;   // FP64 right-hand side (DOF rows; copies equal)
  double* x = nullptr;         // FP64 solution (initial guess in, hanging-consistent)
  double rtol = 1e-13, rtol_inner = 1e-4;
  int max_iter = 20000, max_outer = 30;
  // workspaces
  double* w64 = nullptr;       // FP64 Krylov work (8 * 3 * nslots)
  float* w32 = nullptr;        // FP32 Krylov work (8 * 3 * nslots), mixed only
  double* y64 = nullptr;       // 3 * nslots
  double* r64 = nullptr;       // 3 * nslots: the outer residual, each entry a pair of FP32 numbers (hi, lo)
  float* r32 = nullptr;        // 3 * nslots
  float* e32 = nullptr;        // 3 * nslots
  KState* ks = nullptr;        // 3 device states per instance
  OState* os = nullptr;        // 1 device state per instance
  SolveRec* rec = nullptr;     // device record of this solve, instance i at rec[4 i]
  RedBuf rb;
  Prof* prof = nullptr;
  int pbase = 0;
  // multigrid preconditioner of the Poisson CG (nullptr or no problem on: Jacobi)
  const MGDev<float>* mg32 = nullptr;
  const MGDev<double>* mg64 = nullptr;
  KState* ks_host = nullptr;   // pinned host mirrors for the polling path
  OState* os_host = nullptr;
};

// Enqueue one complete solve on st (captured into cc's graph when st is capturing).
cudaError_t solve_enqueue(const SolveArgs& a, cudaStream_t st, CaptureCtx* cc);

// Zero a record array (n records).
void rec_clear(SolveRec* rec, int n, cudaStream_t st);

// Runs body(stream, cond) until every component of ks is done.
template <typename Body>
cudaError_t run_loop(CaptureCtx* cc, cudaStream_t st, const Cond& cond, const KState* ks, KState* ks_host, int nc,
                     int max_iter, int chunk0, int chunk_max, Body&& body) {
  if (cc && cc->capturing)
    return cond_node(*cc, st, cond, cudaGraphCondTypeWhile, [&](cudaStream_t s) { body(s, cond); });
  int it = 0, chunk = chunk0;
  const Cond none;
  for (;;) {
    cudaMemcpyAsync(ks_host, ks, nc * sizeof(KState), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    bool done = true;
    for (int c = 0; c < nc; ++c) done = done && ks_host[c].done;
    if (done || it > max_iter + 2 * chunk_max) break;
    for (int k = 0; k < chunk; ++k) body(st, none);
    it += chunk;
    chunk = chunk * 2 > chunk_max ? chunk_max : chunk * 2;
  }
  return cudaSuccess;
}

// Device-side helpers shared with the IB solver.
__global__ void k_init_states(KState* ks, int nc, double tol2, int max_iter);
__global__ void k_collect(const KState* ks, int nc, int ninst, SolveRec* rec, OState* os);
__global__ void k_init_outer(OState* os, int ninst, int nc, double tol2, int max_outer);
__global__ void k_collect_outer(const OState* os, int ninst, SolveRec* rec);

}  // namespace ibg
