// Host-side interface of the finite-element and Krylov kernels (fe.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include <vector>

#include "device.cuh"

namespace ibg {

enum Op : int { OP_POISSON = 0, OP_MASS = 1, OP_COEF = 2 };

// Scratch for deterministic grid reductions.
struct RedBuf {
  double* partials = nullptr;   // >= nblocks * 16 + ninst * 16 doubles
  unsigned* counter = nullptr;  // one zero-initialised word
};

// Optional CUDA-event timing of solver kernel launches, by class:
//   base + 0 operator apply, base + 1 vector update (with its reduction),
//   base + 2 search-direction update; base = 0 Poisson, 3 mass, 6 momentum.
struct Prof {
  static constexpr int K = 12;
  bool on = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> cls;
  int used = 0;
  double ms[K] = {};
  int64_t n[K] = {};
  void begin(int c, cudaStream_t st);
  void end(cudaStream_t st);
  void collect();          // after the stream has been synchronised
  void release();
};

// One linear operator on the composite grid: the Poisson stiffness K, the mass
// matrix M (both from incident-cell-mask tables) or a per-slot 15-point
// coefficient stencil (the momentum operator).  coef is [15][nslots].
template <typename T>
struct OpDesc {
  int op;
  const T* coef;
  uint16_t dmask;       // Dirichlet bit (D_VDIR or D_PDIR) of this solve
  const T* dinv;        // Jacobi inverse diagonal, 0 on non-DOF slots
  Prof* prof = nullptr; // optional launch timing
  int pbase = 0;        // profiling class base
};

struct SolveStats {
  int iters[3] = {0, 0, 0};
  int status = 0;       // 0 ok, 4 no convergence, 5 breakdown
  double relres = 0.0;  // max over components of sqrt(rr / bb)
};

// Upload the Kuhn tables to this device's constant memory (idempotent).
cudaError_t fe_init_tables();

// y = A x (NC components, stride nslots) followed by the interface sum.
template <typename T>
void fe_apply(const DevGrid& g, const OpDesc<T>& A, int nc, const T* x, T* y, cudaStream_t st);
// the mixed path's FP64 outer-residual product y = A x, the stencil sums in
// double-FP32 (the symmetric viscous form keeps the FP64 kernels)
// (momentum: the coefficients as the compact FP32 pairs chi + clo of
// fe_momentum_coef_ff; nullptr selects the FP64 kernel on A.coef)
void fe_apply_resid(const DevGrid& g, const OpDesc<double>& A, int nc, const double* x, double* y,
                    const float* chi, const float* clo, cudaStream_t st);

// y = A x per level only: copies of interface nodes hold their level's part
// (readers add the interface sums).
template <typename T>
void fe_apply_local(const DevGrid& g, const OpDesc<T>& A, int nc, const T* x, T* y, cudaStream_t st);

// Local diagonal of A, summed over stored copies, then dinv = 1 / diag on DOFs.
template <typename T>
void fe_jacobi(const DevGrid& g, int op, const T* coef, uint16_t dmask, T* diag, T* dinv, cudaStream_t st);

// CG iteration kernel: p_new = z + beta p_old (stored), q = A p_new local per
// level (no interface sum), fused p.q -> alpha in ks.
template <typename T>
void fe_apply_cg(const DevGrid& g, const OpDesc<T>& A, int nc, const T* z, const T* pold, T* pnew, T* q, KState* ks,
                 RedBuf rb, cudaStream_t st);

// Elementwise helpers over nc * nslots elements.
void fe_cast_d2f(int64_t n, const double* a, float* b, cudaStream_t st);
void fe_add_f2d(int64_t n, const float* a, double* b, cudaStream_t st);
void fe_copy_d(int64_t n, const double* a, double* b, cudaStream_t st);
void fe_add_d(int64_t n, const double* a, double* b, cudaStream_t st);   // b += a
template <typename T> void fe_zero(int64_t n, T* a, cudaStream_t st);

// q = K x for the Poisson stencil (local per level; consumers add the interface
// sums), over the chunks of problems not done that use multigrid (on[i] != 0).
template <typename T>
void fe_poisson_apply(const DevGrid& g, const T* x, T* q, uint16_t dmask, KState* ks, const uint8_t* on,
                      cudaStream_t st);

// Hanging nodes take the mean of their parents (nc components; x2 optional).
template <typename T>
void fe_expand(const DevGrid& g, int nc, T* x, cudaStream_t st);
template <typename T>
void fe_expand2(const DevGrid& g, int nc, T* x, T* x2, cudaStream_t st);

// The interface sum: copies of a node get the sum of their local values plus
// half of each hanging child's; rows with a dmask bit are zeroed.
template <typename T>
void fe_sync(const DevGrid& g, int nc, T* y, uint16_t dmask, cudaStream_t st);

// Right-hand sides and operators built from fields (FP64):
//   out_c = (M u_c) - dt (G_c p)                              (Eq. 9 / velocity correction)
//   out   = -(1/dt) (div u, q)                                (Eq. 12)
//   coef  = M + dt C(u) + dt nu K  as a 15-point stencil       (Eq. 9 operator)
// with each instance's dt and nu.
// All are local per level; callers apply fe_sync.
// right-hand sides in FP64; pairs: the mixed path's double-FP32 stencil sums
// (FP64 inputs and outputs, sums accurate to about 2^-44 of their terms' magnitudes)
void fe_rhs_mass_grad(const DevGrid& g, const double* u, const double* p, double* out, cudaStream_t st, bool pairs);
void fe_rhs_div(const DevGrid& g, const double* u, double* out, cudaStream_t st, bool pairs);
void fe_momentum_coef(const DevGrid& g, const double* u, double* coef64, float* coef32, cudaStream_t st);
// the mixed path's momentum coefficients (gradient viscous form) as compact
// FP32 pairs: coef32 (the inner FP32 operator) + coeflo, no FP64 plane
void fe_momentum_coef_ff(const DevGrid& g, const double* u, float* coef32, float* coeflo, cudaStream_t st);
// once per process and device: kernel attributes (shared-memory carveout)
cudaError_t fe_configure();
// CTAs per SM of the persistent staged Poisson kernels (0 if the query fails)
int fe_p7_ctas_per_sm();

// Copy canonical node values (owner slots) out / in; in also writes the fine
// copy of every interface node.
template <typename T>
void fe_gather_canon(int64_t N, const int32_t* canon_slot, int nc, int64_t nslots, const T* x, T* out,
                     cudaStream_t st);
void fe_scatter_canon(const DevGrid& g, int64_t N, const int32_t* canon_slot, int nc, const double* in,
                      double* x, cudaStream_t st);

// Inlet profile u_max(t) * shape on every inlet slot (component = port axis).
struct PortDev {
  int32_t axis, nh, inst, pad;
  double a0, a[8], b[8], period;
};
void fe_set_inlet(int64_t n, const int32_t* slot, const int32_t* port, const double* shape, const PortDev* ports,
                  const double* t, int64_t nslots, double* u, cudaStream_t st);
void fe_set_pinlet(int64_t n, const int32_t* slot, const int32_t* port, const PortDev* ports, const double* t,
                   const double* p, double* phi, cudaStream_t st);
void fe_time_advance(double* t_commit, double* t_next, const double* dt, int n, int commit, const int32_t* ok,
                     cudaStream_t st);

}  // namespace ibg
