// Host-side interface of the BCE-IB kernels (ib.cu), Sec. 2.3.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "device.cuh"
#include "fe.hpp"
#include "graph.hpp"

namespace ibg {

// Points of all instances, each instance's rows padded to a multiple of 256
// (padding rows have no support and no A_F entries), so that both the
// thread-per-row (256 rows per block) and warp-per-row (8 rows per block)
// kernels have whole blocks per instance for segmented reductions.
struct IBDev {
  int64_t M;               // padded total
  int32_t ninst;
  const int32_t* pinst;    // [M] instance of each row
  const int32_t* seg_t;    // [ninst + 1] block range, 256 rows per block
  const int32_t* seg_w;    // [ninst + 1] block range, 8 rows per block
  const int32_t* seg_g;    // [ninst + 1] block range, 32 rows per block
  const double* pscale;    // [M] dt / (rho h^3) of the row's instance
  float* val32 = nullptr;  // FP32 copies of val and dinv (mixed path)
  float* dinv32 = nullptr;
  const double* iorigin;   // [ninst][3] box origin
  const double* ihf;       // [ninst][3] finest spacing
  const double* icoef;     // [ninst] spreading coefficient dt / (rho h^3)
  const int32_t* binst;    // [nbricks] instance of a brick (for spreading)
  const double* X;         // [M][3]
  const int32_t* org;      // [M][3] support origin, finest grid
  const int32_t* slot;     // [M][64] slot of support node a (-1 missing)
  const uint64_t* freeb;   // [M] bit a: support node a free
  double* W;               // [M][64] delta weights (0 where missing)
  const int32_t* rowptr;   // A_F pattern
  const int32_t* col;
  double* val;             // S = (dt / (rho h^3)) W_f W_f^T values
  double* dinv;            // [M] 1 / diag(S)
  const int32_t* sp_slot;  // spreading CSR
  const int32_t* sp_off;
  const int32_t* sp_ent;
  int64_t n_sp;
  // after a device rebuild (moving points): the list length lives on the
  // device and launches cover sp_cap entries, so a captured step stays valid
  const int32_t* n_sp_dev = nullptr;
  int64_t sp_cap = 0;
};

// Eq. 17-18: W[i][a] = phi((x_a - X_i)/hx) phi((y_a - Y_i)/hy) phi((z_a - Z_i)/hz).
void ib_weights(const IBDev& ib, cudaStream_t st);
// S = (dt/(rho h^3)) W_f W_f^T over free nodes (Eq. 22); dinv = 1/diag.
void ib_assemble(const IBDev& ib, cudaStream_t st);
// B_F = U_B - W u (Eq. 23), u on the finest level ([3][nslots]).
void ib_gather(const IBDev& ib, const double* u, int64_t nslots, const double* UB, double* BF, cudaStream_t st);
// PCG on S G = B_F for the 3 components ([M][3]); G holds the warm start.  The
// loop is a graph WHILE node when st is capturing; the result goes to rec.
cudaError_t ib_solve(const IBDev& ib, const double* BF, double* G, double* work /* 5*3*M */, KState* ks,
                     KState* ks_host, RedBuf rb, double rtol, int max_iter, SolveRec* rec, cudaStream_t st,
                     CaptureCtx* cc);
// After a mixed force solve: the FP64 PCG (warm-started from G) for the
// instances whose FP32-inner defect correction failed (A_F too
// ill-conditioned for FP32: points denser than the grid, Sec. 2.5); the
// others start converged and stop at once.  A device-side IF node in a graph.
cudaError_t ib_fp64_fallback(const IBDev& ib, const double* BF, double* G, double* work, KState* ks,
                             KState* ks_host, const OState* os, OState* os_host, RedBuf rb, double rtol, int max_iter,
                             SolveRec* rec, cudaStream_t st, CaptureCtx* cc);
// The same solve in mixed precision: FP64 defect correction (r = B_F - S G,
// FP64 norms, relative tolerance rtol) around FP32 PCG iterations on the FP32
// copy of S (relative tolerance rtol_inner).  y64: 3*M doubles; w32: 7*3*M
// floats; os: one outer state per instance.
cudaError_t ib_solve_mixed(const IBDev& ib, const double* BF, double* G, double* y64, float* w32, KState* ks,
                           KState* ks_host, OState* os, OState* os_host, RedBuf rb, double rtol, double rtol_inner,
                           int max_iter, int max_outer, SolveRec* rec, cudaStream_t st, CaptureCtx* cc);
// u_j += coef * sum_i W[i][a(j)] G_i on free support nodes (Eq. 19, Eq. 14).
void ib_spread(const IBDev& ib, const double* G, double* u, int64_t nslots, cudaStream_t st);

}  // namespace ibg
