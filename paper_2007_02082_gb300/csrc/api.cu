// C ABI (include/ib.h): handle lifetime, device buffers and the IPCS step driver.
//
// One step (combined algorithm of Sec. 2.4):
//   1. tentative velocity: (M + dt C(u^n) + dt nu K) u~ = M u^n - dt G p^n   (Eq. 9)
//      with the inlet profile at t^{n+1} and no-slip walls; BiCGStab.
//   2-4. B_F = U_B - W u~ (Eq. 23); S G = B_F (Eq. 21-22, G = dS F); PCG;
//      u = u~ + (dt/rho) h^-3 W_f^T G (Eq. 19 and Eq. 14).
//   5. (grad Phi, grad q) = -(1/dt)(div u, q), Phi = 0 on outlet nodes (Eq. 12); PCG.
//   6. (u^{n+1}, v) = (u, v) - dt (grad Phi, v) with the velocity conditions;
//      p^{n+1} = p^n + Phi; PCG on the consistent mass matrix.
// The step is committed (buffers swapped, time advanced) only when every solve
// converged.  With precision IB_MIXED each solve runs FP32 Krylov iterations
// (FP32 operator and Jacobi preconditioner) inside an FP64 defect-correction
// loop whose residual b - A x is formed in FP64.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "fe.hpp"
#include "ib.h"
#include "ib.hpp"
#include "setup.hpp"

using namespace ibg;

struct ib_grid {
  ib_grid_desc d{};
  std::string err;
  bool ready = false;
  cudaStream_t st = nullptr;
  HostGrid H;
  DevGrid g{};
  IBDev ib{};
  std::vector<void*> allocs;
  int64_t dev_bytes = 0;
  // topology
  int32_t* canon = nullptr;
  int32_t *in_slot = nullptr, *in_port = nullptr;
  double* in_shape = nullptr;
  PortDev* ports = nullptr;
  double *tc = nullptr, *tn = nullptr;
  // fields, [3][nslots] for vectors
  double *u = nullptr, *un = nullptr, *p = nullptr, *pn = nullptr, *phi = nullptr, *ut = nullptr, *uib = nullptr;
  // FP64 work
  double *rhs3 = nullptr, *y64 = nullptr, *r64 = nullptr, *w64 = nullptr;
  double *coef64 = nullptr, *diag64 = nullptr, *dK64 = nullptr, *dM64 = nullptr, *dA64 = nullptr;
  // FP32 work (mixed)
  float *coef32 = nullptr, *diag32 = nullptr, *dK32 = nullptr, *dM32 = nullptr, *dA32 = nullptr;
  float *r32 = nullptr, *e32 = nullptr, *w32 = nullptr;
  // IB
  double *X = nullptr, *dS = nullptr, *UB = nullptr, *BF = nullptr, *Gf = nullptr, *ibw = nullptr;
  // solver state
  KState* ks = nullptr;
  KState ks_host[3];
  RedBuf rb{};
  double* host_rrbb = nullptr;
  Prof prof;
  int64_t n_valid = 0;
  // committed state
  int64_t step = 0;
  double time = 0.0;
  ib_info last{};
};

namespace {

#define CK(x)                                                                      \
  do {                                                                             \
    cudaError_t e_ = (x);                                                          \
    if (e_ != cudaSuccess) {                                                       \
      g->err = std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #x;         \
      return IB_ECUDA;                                                             \
    }                                                                              \
  } while (0)

template <typename T>
ib_status dalloc(ib_grid* g, T** p, int64_t n) {
  size_t bytes = size_t(std::max<int64_t>(n, 1)) * sizeof(T);
  void* ptr = nullptr;
  if (g->d.dev_alloc) {
    ptr = g->d.dev_alloc(bytes, g->d.alloc_ctx);
    if (!ptr) { g->err = "device allocator returned NULL"; return IB_ENOMEM; }
  } else {
    cudaError_t e = cudaMalloc(&ptr, bytes);
    if (e != cudaSuccess) { g->err = std::string("cudaMalloc: ") + cudaGetErrorString(e); return IB_ENOMEM; }
  }
  g->allocs.push_back(ptr);
  g->dev_bytes += int64_t(bytes);
  *p = static_cast<T*>(ptr);
  return IB_OK;
}

template <typename T>
ib_status upload(ib_grid* g, T** p, const std::vector<T>& v) {
  ib_status s = dalloc(g, p, int64_t(v.size()));
  if (s != IB_OK) return s;
  if (!v.empty()) CK(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, g->st));
  return IB_OK;
}

void free_all(ib_grid* g) {
  if (g->st) cudaStreamSynchronize(g->st);
  for (void* p : g->allocs) {
    if (g->d.dev_free) g->d.dev_free(p, g->d.alloc_ctx);
    else cudaFree(p);
  }
  g->allocs.clear();
  g->dev_bytes = 0;
  g->prof.release();
  for (int k = 0; k < Prof::K; ++k) { g->prof.ms[k] = 0.0; g->prof.n[k] = 0; }
  if (g->host_rrbb) { cudaFreeHost(g->host_rrbb); g->host_rrbb = nullptr; }
  g->ready = false;
}

#define TRY(x)                         \
  do {                                 \
    ib_status s_ = (x);                \
    if (s_ != IB_OK) return s_;        \
  } while (0)

ib_status allocate_and_upload(ib_grid* g) {
  HostGrid& H = g->H;
  const int64_t ns = H.nbricks * BV;
  DevGrid& dg = g->g;
  dg = DevGrid();
  dg.nbricks = int32_t(H.nbricks);
  dg.nslots = ns;
  for (int l = 0; l <= H.L; ++l)
    for (int a = 0; a < 3; ++a) dg.h[l][a] = H.levels[l].h[a];
  int32_t *blev, *bnbr, *ifc, *iff, *ifo, *ifk, *hg, *hp1, *hp2;
  uint16_t* meta;
  TRY(upload(g, &blev, H.brick_level));
  TRY(upload(g, &bnbr, H.brick_nbr));
  TRY(upload(g, &meta, H.meta));
  std::vector<int32_t> ifo_v = H.if_child_off;
  if (ifo_v.empty()) ifo_v.push_back(0);
  TRY(upload(g, &ifc, H.if_coarse));
  TRY(upload(g, &iff, H.if_fine));
  TRY(upload(g, &ifo, ifo_v));
  TRY(upload(g, &ifk, H.if_child));
  TRY(upload(g, &hg, H.hang_slot));
  TRY(upload(g, &hp1, H.hang_p1));
  TRY(upload(g, &hp2, H.hang_p2));
  dg.blev = blev; dg.bnbr = bnbr; dg.meta = meta;
  dg.n_if = int32_t(H.if_coarse.size());
  dg.if_c = ifc; dg.if_f = iff; dg.if_off = ifo; dg.if_kid = ifk;
  dg.n_hang = int32_t(H.hang_slot.size());
  dg.hg = hg; dg.hp1 = hp1; dg.hp2 = hp2;
  TRY(upload(g, &g->canon, H.canon_slot));
  TRY(upload(g, &g->in_slot, H.inlet_slot));
  TRY(upload(g, &g->in_port, H.inlet_port));
  TRY(upload(g, &g->in_shape, H.inlet_shape));
  std::vector<PortDev> pd(std::max(1, int(g->d.n_ports)));
  for (int p = 0; p < g->d.n_ports; ++p) {
    const ib_port& P = g->d.ports[p];
    pd[p] = PortDev();
    pd[p].axis = P.axis;
    pd[p].nh = std::min(P.n_harm, 8);
    pd[p].a0 = P.a0;
    pd[p].period = P.period > 0 ? P.period : 1.0;
    for (int k = 0; k < 8; ++k) { pd[p].a[k] = P.a[k]; pd[p].b[k] = P.b[k]; }
  }
  TRY(upload(g, &g->ports, pd));
  TRY(dalloc(g, &g->tc, 1));
  TRY(dalloc(g, &g->tn, 1));
  // fields and FP64 work
  const bool mixed = g->d.precision == IB_MIXED;
  TRY(dalloc(g, &g->u, 3 * ns));
  TRY(dalloc(g, &g->un, 3 * ns));
  TRY(dalloc(g, &g->ut, 3 * ns));
  TRY(dalloc(g, &g->uib, 3 * ns));
  TRY(dalloc(g, &g->p, ns));
  TRY(dalloc(g, &g->pn, ns));
  TRY(dalloc(g, &g->phi, ns));
  TRY(dalloc(g, &g->rhs3, 3 * ns));
  TRY(dalloc(g, &g->y64, 3 * ns));
  TRY(dalloc(g, &g->r64, 3 * ns));
  TRY(dalloc(g, &g->w64, mixed ? 3 * ns : 8 * 3 * ns));
  TRY(dalloc(g, &g->coef64, 15 * ns));
  TRY(dalloc(g, &g->diag64, ns));
  TRY(dalloc(g, &g->dK64, ns));
  TRY(dalloc(g, &g->dM64, ns));
  TRY(dalloc(g, &g->dA64, ns));
  if (mixed) {
    TRY(dalloc(g, &g->coef32, 15 * ns));
    TRY(dalloc(g, &g->diag32, ns));
    TRY(dalloc(g, &g->dK32, ns));
    TRY(dalloc(g, &g->dM32, ns));
    TRY(dalloc(g, &g->dA32, ns));
    TRY(dalloc(g, &g->r32, 3 * ns));
    TRY(dalloc(g, &g->e32, 3 * ns));
    TRY(dalloc(g, &g->w32, 8 * 3 * ns));
  }
  // IB
  const int64_t M = H.M;
  IBDev& ib = g->ib;
  ib = IBDev();
  ib.M = M;
  int32_t *org, *slot, *rp, *col, *sps, *spo, *spe;
  uint64_t* fb;
  TRY(upload(g, &g->X, H.X));
  TRY(upload(g, &g->dS, H.dS));
  TRY(upload(g, &g->UB, H.UB));
  TRY(upload(g, &org, H.ib_origin));
  TRY(upload(g, &slot, H.ib_slot));
  TRY(upload(g, &fb, H.ib_free));
  std::vector<int32_t> rpv = H.af_rowptr;
  if (rpv.empty()) rpv.push_back(0);
  TRY(upload(g, &rp, rpv));
  TRY(upload(g, &col, H.af_col));
  std::vector<int32_t> spov = H.sp_off;
  if (spov.empty()) spov.push_back(0);
  TRY(upload(g, &sps, H.sp_slot));
  TRY(upload(g, &spo, spov));
  TRY(upload(g, &spe, H.sp_ent));
  ib.X = g->X; ib.org = org; ib.slot = slot; ib.freeb = fb; ib.rowptr = rp; ib.col = col;
  ib.sp_slot = sps; ib.sp_off = spo; ib.sp_ent = spe; ib.n_sp = int64_t(H.sp_slot.size());
  TRY(dalloc(g, &ib.W, 64 * M));
  TRY(dalloc(g, &ib.val, int64_t(H.af_col.size())));
  TRY(dalloc(g, &ib.dinv, M));
  TRY(dalloc(g, &g->BF, 3 * M));
  TRY(dalloc(g, &g->Gf, 3 * M));
  TRY(dalloc(g, &g->ibw, 4 * 3 * M));
  // reductions
  int64_t maxblk = std::max<int64_t>(H.nbricks, (M * 32 + 255) / 256 + 1);
  TRY(dalloc(g, &g->rb.partials, maxblk * 16 + 64));
  TRY(dalloc(g, &g->rb.counter, 1));
  TRY(dalloc(g, &g->ks, 3));
  CK(cudaMemsetAsync(g->rb.counter, 0, sizeof(unsigned), g->st));
  CK(cudaMallocHost(&g->host_rrbb, 16 * sizeof(double)));
  return IB_OK;
}

ib_status reset_state(ib_grid* g) {
  const int64_t ns = g->g.nslots;
  CK(cudaMemsetAsync(g->u, 0, 3 * ns * sizeof(double), g->st));
  CK(cudaMemsetAsync(g->un, 0, 3 * ns * sizeof(double), g->st));
  CK(cudaMemsetAsync(g->ut, 0, 3 * ns * sizeof(double), g->st));
  CK(cudaMemsetAsync(g->uib, 0, 3 * ns * sizeof(double), g->st));
  CK(cudaMemsetAsync(g->p, 0, ns * sizeof(double), g->st));
  CK(cudaMemsetAsync(g->pn, 0, ns * sizeof(double), g->st));
  CK(cudaMemsetAsync(g->phi, 0, ns * sizeof(double), g->st));
  CK(cudaMemsetAsync(g->tc, 0, sizeof(double), g->st));
  CK(cudaMemsetAsync(g->tn, 0, sizeof(double), g->st));
  if (g->H.M) {
    CK(cudaMemsetAsync(g->Gf, 0, 3 * g->H.M * sizeof(double), g->st));
    CK(cudaMemsetAsync(g->BF, 0, 3 * g->H.M * sizeof(double), g->st));
  }
  g->step = 0;
  g->time = 0.0;
  return IB_OK;
}

struct Tols {
  double mom, p, corr, ib, inner;
  int max_iter;
};

Tols tolerances(const ib_grid* g) {
  const bool mixed = g->d.precision == IB_MIXED;
  Tols t;
  t.mom = g->d.rtol_mom > 0 ? g->d.rtol_mom : (mixed ? 1e-10 : 1e-13);
  t.p = g->d.rtol_p > 0 ? g->d.rtol_p : (mixed ? 1e-10 : 1e-13);
  t.corr = g->d.rtol_corr > 0 ? g->d.rtol_corr : (mixed ? 1e-10 : 1e-13);
  t.ib = g->d.rtol_ib > 0 ? g->d.rtol_ib : 1e-13;
  t.inner = 1e-4;
  t.max_iter = g->d.max_iter > 0 ? g->d.max_iter : 20000;
  return t;
}

// One linear solve, FP64 or FP32-inside-FP64 defect correction.
SolveStats solve(ib_grid* g, int op, bool bicg, int nc, uint16_t dmask, const double* coef64, const double* dinv64,
                 const float* coef32, const float* dinv32, const double* b, double* x, double rtol, int max_iter,
                 int* outer_out) {
  const DevGrid& dg = g->g;
  const int pbase = op == OP_POISSON ? 0 : op == OP_MASS ? 3 : 6;
  Prof* pf = g->prof.on ? &g->prof : nullptr;
  OpDesc<double> A64{op, coef64, dmask, dinv64, pf, pbase};
  if (g->d.precision != IB_MIXED) {
    *outer_out = 1;
    return bicg ? fe_bicgstab<double>(dg, A64, nc, b, x, g->w64, g->ks, g->ks_host, g->rb, rtol, max_iter, g->st)
                : fe_cg<double>(dg, A64, nc, b, x, g->w64, g->ks, g->ks_host, g->rb, rtol, max_iter, g->st);
  }
  OpDesc<float> A32{op, coef32, dmask, dinv32, pf, pbase};
  const int64_t n = int64_t(nc) * dg.nslots;
  SolveStats tot;
  const int max_outer = 30;
  int outer = 0;
  double ref[3] = {0.0, 0.0, 0.0};   // max(||b||^2, ||r0||^2) per component
  for (; outer < max_outer; ++outer) {
    fe_residual64(dg, A64, nc, b, x, g->y64, g->r64, g->rb, g->host_rrbb, g->st);
    double rel = 0.0;
    for (int c = 0; c < nc; ++c) {
      double rr = g->host_rrbb[2 * c], bb = g->host_rrbb[2 * c + 1];
      if (outer == 0) ref[c] = std::max(bb, rr);
      rel = std::max(rel, ref[c] > 0 ? std::sqrt(rr / ref[c]) : 0.0);
    }
    tot.relres = rel;
    if (!std::isfinite(rel)) { tot.status = 5; break; }
    if (rel <= rtol) break;
    fe_cast_d2f(n, g->r64, g->r32, g->st);
    fe_zero<float>(n, g->e32, g->st);
    const double rin = std::max(tolerances(g).inner, rtol);
    SolveStats in = bicg ? fe_bicgstab<float>(dg, A32, nc, g->r32, g->e32, g->w32, g->ks, g->ks_host, g->rb, rin,
                                              max_iter, g->st)
                         : fe_cg<float>(dg, A32, nc, g->r32, g->e32, g->w32, g->ks, g->ks_host, g->rb, rin, max_iter,
                                        g->st);
    for (int c = 0; c < 3; ++c) tot.iters[c] += in.iters[c];
    if (in.status == 5) { tot.status = 5; break; }
    fe_add_f2d(n, g->e32, x, g->st);
  }
  if (outer >= max_outer) tot.status = 4;
  *outer_out = outer;
  return tot;
}

ib_status step_once(ib_grid* g) {
  const DevGrid& dg = g->g;
  const int64_t ns = dg.nslots;
  const double dt = g->d.dt, nu = g->d.nu, rho = g->d.rho;
  const bool mixed = g->d.precision == IB_MIXED;
  const Tols tl = tolerances(g);
  cudaStream_t st = g->st;
  ib_info& I = g->last;
  int status = 0;

  fe_time_advance(g->tc, g->tn, dt, 0, st);
  // ---- Step 1: tentative velocity (Eq. 9)
  fe_momentum_coef(dg, g->u, dt, nu, g->coef64, mixed ? g->coef32 : nullptr, st);
  fe_jacobi<double>(dg, OP_COEF, g->coef64, D_VDIR, g->diag64, g->dA64, st);
  if (mixed) fe_jacobi<float>(dg, OP_COEF, g->coef32, D_VDIR, g->diag32, g->dA32, st);
  fe_rhs_mass_grad(dg, g->u, g->p, dt, g->rhs3, st);
  fe_sync<double>(dg, 3, g->rhs3, D_VDIR, st);
  fe_copy_d(3 * ns, g->u, g->ut, st);
  fe_set_inlet(int64_t(g->H.inlet_slot.size()), g->in_slot, g->in_port, g->in_shape, g->ports, g->tn, ns, g->ut, st);
  fe_expand<double>(dg, 3, g->ut, st);
  int outer = 0;
  SolveStats sm = solve(g, OP_COEF, true, 3, D_VDIR, g->coef64, g->dA64, g->coef32, g->dA32, g->rhs3, g->ut, tl.mom,
                        tl.max_iter, &outer);
  for (int c = 0; c < 3; ++c) I.iters_mom[c] = sm.iters[c];
  I.outer_mom = outer;
  I.res_mom = sm.relres;
  if (sm.status) status = sm.status;

  // ---- Steps 2-4: BCE-IB force and correction (Eq. 14, 19-23)
  fe_copy_d(3 * ns, g->ut, g->uib, st);
  if (g->H.M) {
    ib_gather(g->ib, g->ut, ns, g->UB, g->BF, st);
    SolveStats si = ib_solve(g->ib, g->BF, g->Gf, g->ibw, g->ks, g->ks_host, g->rb, tl.ib, tl.max_iter, st);
    I.iters_ib = std::max(si.iters[0], std::max(si.iters[1], si.iters[2]));
    I.res_ib = si.relres;
    if (si.status && !status) status = si.status;
    const double h3 = g->H.hf[0] * g->H.hf[1] * g->H.hf[2];
    ib_spread(g->ib, g->Gf, dt / (rho * h3), g->uib, ns, st);
  }

  // ---- Step 5: pressure increment (Eq. 12)
  double* rhs1 = g->rhs3;   // component 0 of the RHS buffer
  fe_rhs_div(dg, g->uib, -1.0 / dt, rhs1, st);
  fe_sync<double>(dg, 1, rhs1, D_PDIR, st);
  SolveStats sp = solve(g, OP_POISSON, false, 1, D_PDIR, nullptr, g->dK64, nullptr, g->dK32, rhs1, g->phi, tl.p,
                        tl.max_iter, &outer);
  I.iters_p = sp.iters[0];
  I.outer_p = outer;
  I.res_p = sp.relres;
  if (sp.status && !status) status = sp.status;

  // ---- Step 6: velocity correction and pressure update
  fe_rhs_mass_grad(dg, g->uib, g->phi, dt, g->rhs3, st);
  fe_sync<double>(dg, 3, g->rhs3, D_VDIR, st);
  fe_copy_d(3 * ns, g->uib, g->un, st);
  SolveStats sc = solve(g, OP_MASS, false, 3, D_VDIR, nullptr, g->dM64, nullptr, g->dM32, g->rhs3, g->un, tl.corr,
                        tl.max_iter, &outer);
  for (int c = 0; c < 3; ++c) I.iters_corr[c] = sc.iters[c];
  I.outer_corr = outer;
  I.res_corr = sc.relres;
  if (sc.status && !status) status = sc.status;
  fe_copy_d(ns, g->p, g->pn, st);
  fe_add_d(ns, g->phi, g->pn, st);

  CK(cudaStreamSynchronize(st));
  CK(cudaGetLastError());
  if (g->prof.on) g->prof.collect();
  if (status) {
    g->err = status == 5 ? "Krylov breakdown in a step solve" : "a step solve did not converge";
    return status == 5 ? IB_EBREAKDOWN : IB_ENOCONV;
  }
  std::swap(g->u, g->un);
  std::swap(g->p, g->pn);
  fe_time_advance(g->tc, g->tn, dt, 1, st);
  g->step += 1;
  g->time += dt;
  return IB_OK;
}

int64_t field_bytes(const ib_grid* g, int f) {
  const int64_t N = int64_t(g->H.canon_slot.size()), M = g->H.M;
  const int64_t nc = g->H.n[0] * g->H.n[1] * g->H.n[2];
  switch (f) {
    case IB_FIELD_U: case IB_FIELD_U_TENT: case IB_FIELD_U_IB: return N * 3 * 8;
    case IB_FIELD_P: case IB_FIELD_PHI: return N * 8;
    case IB_FIELD_F_LAG: case IB_FIELD_B_F: return M * 3 * 8;
    case IB_FIELD_NODE_Q: return N * 3 * 4;
    case IB_FIELD_NODE_FLAGS: return N;
    case IB_FIELD_ACTIVE: case IB_FIELD_LEVEL: return nc;
    case IB_FIELD_IB_ORIGIN: return M * 3 * 4;
    case IB_FIELD_IB_WEIGHTS: return M * 64 * 8;
    case IB_FIELD_IB_FREE: return M * 64;
    default: return -1;
  }
}

}  // namespace

extern "C" {

ib_status ib_grid_create(const ib_grid_desc* d, ib_grid** out) {
  if (!d || !out) return IB_EINVAL;
  *out = nullptr;
  auto bad = [](const char*) { return IB_EINVAL; };
  for (int a = 0; a < 3; ++a)
    if (d->n[a] <= 0 || !(d->extent[a] > 0) || !std::isfinite(d->origin[a])) return bad("grid");
  if (d->max_level < 0 || d->max_level > IB_MAX_LEVEL) return bad("max_level");
  if (d->max_level > 0 && d->refine_band < 1) return bad("refine_band");
  if (!(d->nu > 0) || !(d->rho > 0) || !(d->dt > 0)) return bad("nu/rho/dt");
  if (d->precision != IB_FP64 && d->precision != IB_MIXED) return bad("precision");
  if (d->n_ports < 1 || d->n_ports > IB_MAX_PORTS) return bad("ports");
  bool outlet = false;
  for (int p = 0; p < d->n_ports; ++p) {
    const ib_port& P = d->ports[p];
    if (P.axis < 0 || P.axis > 2 || (P.side != 0 && P.side != 1) || !(P.radius > 0)) return bad("port");
    if (P.kind != IB_INLET_VELOCITY && P.kind != IB_OUTLET_ZERO_P) return bad("port kind");
    if (P.n_harm < 0 || P.n_harm > IB_MAX_HARMONICS) return bad("harmonics");
    if (P.kind == IB_OUTLET_ZERO_P) outlet = true;
  }
  if (!outlet) return bad("no outlet");
  int64_t nf = int64_t(d->n[0]) * d->n[1] * d->n[2] << (3 * d->max_level);
  if (nf > (int64_t(1) << 40)) return bad("too large");
  ib_grid* g = new (std::nothrow) ib_grid();
  if (!g) return IB_ENOMEM;
  g->d = *d;
  g->st = static_cast<cudaStream_t>(d->stream);
  cudaError_t e = fe_init_tables();
  if (e != cudaSuccess) {
    delete g;
    return IB_ECUDA;
  }
  *out = g;
  return IB_OK;
}

ib_status ib_set_boundary(ib_grid* g, int64_t M, const double* X, const double* dS, const double* UB,
                          const uint8_t* inside) {
  if (!g) return IB_EINVAL;
  if (M < 0 || (M > 0 && (!X || !dS))) { g->err = "bad point arrays"; return IB_EINVAL; }
  free_all(g);
  ib_status s = build_host_grid(g->d, M, X, dS, UB, inside, g->H, g->err);
  if (s != IB_OK) return s;
  s = allocate_and_upload(g);
  if (s != IB_OK) { free_all(g); return s; }
  const DevGrid& dg = g->g;
  cudaStream_t st = g->st;
  // constant preconditioners, IB weights and force matrix
  fe_jacobi<double>(dg, OP_POISSON, nullptr, D_PDIR, g->diag64, g->dK64, st);
  fe_jacobi<double>(dg, OP_MASS, nullptr, D_VDIR, g->diag64, g->dM64, st);
  if (g->d.precision == IB_MIXED) {
    fe_jacobi<float>(dg, OP_POISSON, nullptr, D_PDIR, g->diag32, g->dK32, st);
    fe_jacobi<float>(dg, OP_MASS, nullptr, D_VDIR, g->diag32, g->dM32, st);
  }
  ib_weights(g->ib, g->H.origin, g->H.hf, st);
  const double h3 = g->H.hf[0] * g->H.hf[1] * g->H.hf[2];
  ib_assemble(g->ib, g->d.dt / (g->d.rho * h3), st);
  s = reset_state(g);
  if (s != IB_OK) { free_all(g); return s; }
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    g->err = std::string("CUDA: ") + cudaGetErrorString(e);
    free_all(g);
    return IB_ECUDA;
  }
  g->n_valid = 0;
  for (uint16_t m : g->H.meta)
    if (m & M_VALID) g->n_valid++;
  g->prof.on = g->d.profile != 0;
  g->ready = true;
  g->err.clear();
  return IB_OK;
}

ib_status ipcs_step(ib_grid* g, int32_t nsteps) {
  if (!g) return IB_EINVAL;
  if (!g->ready) { g->err = "ib_set_boundary has not succeeded"; return IB_ESTATE; }
  if (nsteps < 0) { g->err = "nsteps < 0"; return IB_EINVAL; }
  for (int32_t k = 0; k < nsteps; ++k) {
    ib_status s = step_once(g);
    if (s != IB_OK) return s;
  }
  return IB_OK;
}

ib_status ib_fields_get(ib_grid* g, int32_t field, void* dst, size_t bytes, int32_t dst_on_device) {
  if (!g || !dst) return IB_EINVAL;
  if (!g->ready) { g->err = "ib_set_boundary has not succeeded"; return IB_ESTATE; }
  int64_t need = field_bytes(g, field);
  if (need < 0 || int64_t(bytes) != need) { g->err = "bad field id or byte count"; return IB_EINVAL; }
  const HostGrid& H = g->H;
  const int64_t N = int64_t(H.canon_slot.size()), M = H.M, ns = g->g.nslots;
  cudaStream_t st = g->st;
  const cudaMemcpyKind k_out = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const cudaMemcpyKind h_out = dst_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
  auto host_copy = [&](const void* src) -> ib_status {
    CK(cudaMemcpyAsync(dst, src, bytes, h_out, st));
    CK(cudaStreamSynchronize(st));
    return IB_OK;
  };
  switch (field) {
    case IB_FIELD_U: case IB_FIELD_U_TENT: case IB_FIELD_U_IB: case IB_FIELD_P: case IB_FIELD_PHI: {
      const double* src = field == IB_FIELD_U ? g->u : field == IB_FIELD_U_TENT ? g->ut
                        : field == IB_FIELD_U_IB ? g->uib : field == IB_FIELD_P ? g->p : g->phi;
      int nc = (field == IB_FIELD_P || field == IB_FIELD_PHI) ? 1 : 3;
      double* tmp = g->y64;   // scratch of 3 * nslots >= nc * N
      fe_gather_canon<double>(N, g->canon, nc, ns, src, tmp, st);
      CK(cudaMemcpyAsync(dst, tmp, bytes, k_out, st));
      CK(cudaStreamSynchronize(st));
      return IB_OK;
    }
    case IB_FIELD_B_F: {
      CK(cudaMemcpyAsync(dst, g->BF, bytes, k_out, st));
      CK(cudaStreamSynchronize(st));
      return IB_OK;
    }
    case IB_FIELD_F_LAG: {
      std::vector<double> G(3 * M);
      if (M) CK(cudaMemcpyAsync(G.data(), g->Gf, bytes, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (int64_t i = 0; i < M; ++i)
        for (int c = 0; c < 3; ++c) G[3 * i + c] /= H.dS[i];
      return host_copy(G.data());
    }
    case IB_FIELD_NODE_Q: return host_copy(H.canon_q.data());
    case IB_FIELD_NODE_FLAGS: return host_copy(H.canon_flags.data());
    case IB_FIELD_ACTIVE: return host_copy(H.active.data());
    case IB_FIELD_LEVEL: return host_copy(H.level.data());
    case IB_FIELD_IB_ORIGIN: return host_copy(H.ib_origin.data());
    case IB_FIELD_IB_WEIGHTS: {
      CK(cudaMemcpyAsync(dst, g->ib.W, bytes, k_out, st));
      CK(cudaStreamSynchronize(st));
      return IB_OK;
    }
    case IB_FIELD_IB_FREE: {
      std::vector<uint8_t> f(64 * M);
      for (int64_t i = 0; i < M; ++i)
        for (int a = 0; a < 64; ++a)
          f[64 * i + a] = (H.ib_free[i] >> a & 1) ? 1 : (H.ib_slot[64 * i + a] >= 0 ? 2 : 0);
      return host_copy(f.data());
    }
  }
  g->err = "field not readable";
  return IB_EINVAL;
}

ib_status ib_fields_set(ib_grid* g, int32_t field, const void* src, size_t bytes, int32_t src_on_device) {
  if (!g || !src) return IB_EINVAL;
  if (!g->ready) { g->err = "ib_set_boundary has not succeeded"; return IB_ESTATE; }
  if (field != IB_FIELD_U && field != IB_FIELD_P) { g->err = "only U and P can be set"; return IB_EINVAL; }
  if (int64_t(bytes) != field_bytes(g, field)) { g->err = "bad byte count"; return IB_EINVAL; }
  const int64_t N = int64_t(g->H.canon_slot.size());
  const int nc = field == IB_FIELD_U ? 3 : 1;
  double* tmp = g->y64;
  CK(cudaMemcpyAsync(tmp, src, bytes, src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->st));
  fe_scatter_canon(g->g, N, g->canon, nc, tmp, field == IB_FIELD_U ? g->u : g->p, g->st);
  CK(cudaStreamSynchronize(g->st));
  return IB_OK;
}

ib_status ib_grid_info(const ib_grid* g, ib_info* out) {
  if (!g || !out) return IB_EINVAL;
  if (!g->ready) return IB_ESTATE;
  const HostGrid& H = g->H;
  ib_info I = g->last;
  I.n_nodes = int64_t(H.canon_slot.size());
  I.n_dof = H.n_dof;
  I.n_hanging = int64_t(H.hang_slot.size());
  I.n_leaf_cells = 0;
  for (int l = 0; l <= IB_MAX_LEVEL; ++l) {
    I.n_leaf_cells_level[l] = H.leaf_per_level[l];
    I.n_leaf_cells += H.leaf_per_level[l];
  }
  I.n_active_coarse = H.n_active_coarse;
  I.n_bricks = H.nbricks;
  I.n_slots = H.nbricks * BV;
  I.n_interface = int64_t(H.if_coarse.size());
  I.n_points = H.M;
  I.af_nnz = int64_t(H.af_col.size());
  double mdS = 0.0;
  for (double v : H.dS) mdS += v;
  mdS = H.M ? mdS / double(H.M) : 0.0;
  for (int a = 0; a < 3; ++a) I.a_ratio[a] = std::sqrt(mdS) / H.hf[a];
  I.step = g->step;
  I.time = g->time;
  I.device_bytes = g->dev_bytes;
  I.n_valid_slots = g->n_valid;
  I.kernel_launches = g_launches.load();
  for (int k = 0; k < Prof::K; ++k) {
    I.prof_ms[k] = g->prof.ms[k];
    I.prof_launches[k] = g->prof.n[k];
  }
  *out = I;
  return IB_OK;
}

const char* ib_last_error(const ib_grid* g) { return g ? g->err.c_str() : "null handle"; }

void ib_grid_destroy(ib_grid* g) {
  if (!g) return;
  free_all(g);
  delete g;
}

}  // extern "C"
