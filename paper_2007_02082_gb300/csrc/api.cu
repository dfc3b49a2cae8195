// C ABI (include/ib.h): handles, batches, device buffers and the IPCS step driver.
//
// One step (combined algorithm of Sec. 2.4):
//   1. tentative velocity: (M + dt C(u^n) + dt nu K) u~ = M u^n - dt G p^n   (Eq. 9)
//      with the inlet profile at t^{n+1} and no-slip walls; BiCGStab.
//   2-4. B_F = U_B - W u~ (Eq. 23); S G = B_F (Eq. 21-22, G = dS F); PCG;
//      u = u~ + (dt/rho) h^-3 W_f^T G (Eq. 19 and Eq. 14).
//   5. (grad Phi, grad q) = -(1/dt)(div u, q), Phi = 0 on outlet nodes (Eq. 12); PCG.
//   6. (u^{n+1}, v) = (u, v) - dt (grad Phi, v) with the velocity conditions;
//      p^{n+1} = p^n + Phi; PCG on the consistent mass matrix.
// With precision IB_MIXED each solve runs FP32 Krylov iterations (FP32 operator
// and Jacobi preconditioner) inside an FP64 defect-correction loop whose
// residual b - A x is formed in FP64.
//
// Engine.  The device state of one or several problem instances laid out side
// by side: bricks, slots and Lagrangian rows of instance i follow those of
// instance i - 1, so every kernel runs once over all instances and every
// reduction is segmented per instance (each instance's scalars depend only on
// its own data).  A standalone handle owns an engine of one instance; a batch
// is an engine over several deferred handles.
//
// Execution: the whole step is captured once into a CUDA graph (two graphs, one
// per ping-pong parity of the u/p buffers) in which every Krylov loop and the
// FP64 outer loop are conditional WHILE nodes decided on the device; a step is
// one graph launch and one host synchronisation (to read the solve records).
// With desc.profile the same launches run eagerly, loops polled from the host,
// and every solver kernel is timed with CUDA events.  A step is committed per
// instance: an instance whose solves failed keeps its previous state.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "async.cuh"
#include "fe.hpp"
#include "ib.h"
#include "ib.hpp"
#include "ibmove.hpp"
#include "wss.hpp"
#include "krylov.hpp"
#include "mg.hpp"
#include "noalloc.hpp"
#include "setup.hpp"

using namespace ibg;

namespace ibg {
unsigned long long fe_kcount();
unsigned long long krylov_kcount();
unsigned long long ib_kcount();
unsigned long long mg_kcount();
unsigned long long move_kcount();
unsigned long long wss_kcount();
}

namespace {

struct Tols {
  double mom, p, corr, ib, inner, inner_p;
  int max_iter;
};

Tols tolerances(const ib_grid_desc& d) {
  const bool mixed = d.precision == IB_MIXED;
  Tols t;
  t.mom = d.rtol_mom > 0 ? d.rtol_mom : (mixed ? 1e-10 : 1e-13);
  t.p = d.rtol_p > 0 ? d.rtol_p : (mixed ? 1e-10 : 1e-13);
  t.corr = d.rtol_corr > 0 ? d.rtol_corr : (mixed ? 1e-10 : 1e-13);
  t.ib = d.rtol_ib > 0 ? d.rtol_ib : (mixed ? 1e-10 : 1e-13);
  t.inner = 1e-5;
  t.inner_p = 1e-3;
  t.max_iter = d.max_iter > 0 ? d.max_iter : 20000;
  return t;
}

struct Engine {
  std::vector<const HostGrid*> H;
  std::vector<const MGHost*> MG;   // multigrid hierarchy of each problem (ok = false: Jacobi)
  std::vector<ib_grid_desc> D;
  int ninst = 0;
  bool mixed = false;
  bool sym = false;   // symmetric viscous form (all members)
  Tols tol{};
  cudaStream_t st = nullptr;
  void* (*alloc)(size_t, void*) = nullptr;
  void (*freef)(void*, void*) = nullptr;
  void* actx = nullptr;
  std::vector<void*> allocs;
  int64_t bytes = 0;
  std::string err;
  // layout
  std::vector<int64_t> brick0, slot0, ns_i, row0, canon0;
  int64_t nbricks = 0, ns = 0, Mtot = 0, n_inlet = 0, n_pinlet = 0, n_valid = 0, ncomp = 0;
  DevGrid g{};
  IBDev ib{};
  int32_t* canon = nullptr;        // concatenated canonical -> global slot
  int32_t *in_slot = nullptr, *in_port = nullptr;
  double* in_shape = nullptr;
  int32_t *pin_slot = nullptr, *pin_port = nullptr;   // pressure-inlet copies and their ports
  PortDev* ports = nullptr;
  double *tc = nullptr, *tn = nullptr, *pdt = nullptr;
  int32_t* ok = nullptr;
  int32_t* aerr = nullptr;        // [ninst] device error word of the step
  int32_t* aerr_host = nullptr;   // pinned copy
  // moving points (standalone engines): finest-level brick map and rebuild buffers
  bool mv_ready = false;
  int32_t* mv_bmap = nullptr;
  uint8_t* mv_cells = nullptr;    // coarse cells: level when active, 255 otherwise
  int32_t mv_nb[3] = {0, 0, 0};
  int64_t mv_nf[3] = {0, 0, 0};
  int32_t *mv_bins = nullptr, *mv_rcnt = nullptr, *mv_scratch = nullptr, *mv_err = nullptr;
  int32_t *mv_scnt = nullptr, *mv_sstart = nullptr, *mv_sfill = nullptr, *mv_sflag = nullptr, *mv_sidx = nullptr;
  double *mv_xprev = nullptr, *mv_ubprev = nullptr;
  int64_t af_cap = 0;             // capacity of ib.col / ib.val
  bool mv_graph_stale = false;    // a rebuild reallocated a list the step graphs hold
  double *wss_n = nullptr, *wss_w = nullptr, *wss_g = nullptr;   // wall shear stress buffers
  // fields [3][ns] / [ns]
  double *ubuf[2] = {nullptr, nullptr}, *pbuf[2] = {nullptr, nullptr};
  double *u = nullptr, *un = nullptr, *p = nullptr, *pn = nullptr, *phi = nullptr, *ut = nullptr, *uib = nullptr;
  double *rhs3 = nullptr, *y64 = nullptr, *r64 = nullptr, *w64 = nullptr;
  double *coef64 = nullptr, *diag64 = nullptr, *dK64 = nullptr, *dM64 = nullptr, *dA64 = nullptr;
  float *coef32 = nullptr, *diag32 = nullptr, *dK32 = nullptr, *dM32 = nullptr, *dA32 = nullptr;
  // mixed path, gradient viscous form: the lo parts of the momentum
  // coefficient pairs (coef32 holds the hi parts); coef64 is not held then
  float* coeflo32 = nullptr;
  float *r32 = nullptr, *e32 = nullptr, *w32 = nullptr;
  double *X = nullptr, *dS = nullptr, *UB = nullptr, *BF = nullptr, *Gf = nullptr, *ibw = nullptr;
  double* ib_y64 = nullptr;       // mixed force solve: FP64 S G
  float* ib_w32 = nullptr;        // mixed force solve: FP32 work (7 x 3 M)
  // solver state
  KState* ks = nullptr;
  KState* ks_host = nullptr;
  OState* os = nullptr;
  OState* os_host = nullptr;
  SolveRec* recs = nullptr;
  SolveRec* recs_host = nullptr;
  int32_t* ok_host = nullptr;
  RedBuf rb{};
  MGDev<float> mg32;
  MGDev<double> mg64;
  Prof prof;
  bool use_graph = true;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  cudaStream_t cap_st = nullptr;
  CaptureCtx cc;
  // per-instance host counters
  std::vector<int64_t> step;
  std::vector<double> time;
  std::vector<ib_info> last;
  std::vector<int> status;
};

}  // namespace

// device snapshot of a deferred handle's state in its own slot layout
struct Snapshot {
  double* u = nullptr;    // [3][ns]
  double* p = nullptr;    // [ns]
  double* phi = nullptr;  // [ns]
  double* G = nullptr;    // [M][3]
  int32_t* canon = nullptr;
  int64_t step = 0;
  double time = 0.0;
  bool valid = false;
};

struct ib_grid {
  ib_grid_desc d{};
  std::string err;
  bool ready = false;
  HostGrid H;
  MGHost mg;                    // Poisson multigrid hierarchy (host)
  Engine* eng = nullptr;        // standalone handle
  Snapshot snap;                // deferred handle
  std::vector<void*> snap_allocs;
  int64_t snap_bytes = 0;
  ib_batch* batch = nullptr;    // batch currently holding a deferred handle
  int batch_index = -1;
  int device = -1;              // CUDA device current at ib_grid_create
};

struct ib_batch {
  std::vector<ib_grid*> members;
  Engine E;
};

namespace {

#define CK(x)                                                                      \
  do {                                                                             \
    cudaError_t e_ = (x);                                                          \
    if (e_ != cudaSuccess) {                                                       \
      E.err = std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #x;          \
      return IB_ECUDA;                                                             \
    }                                                                              \
  } while (0)

#define TRY(x)                         \
  do {                                 \
    ib_status s_ = (x);                \
    if (s_ != IB_OK) return s_;        \
  } while (0)

void* raw_alloc(void* (*al)(size_t, void*), void* ctx, size_t bytes) {
  void* ptr = nullptr;
  if (al) return al(bytes, ctx);
  if (cudaMalloc(&ptr, bytes) != cudaSuccess) return nullptr;
  return ptr;
}
void raw_free(void (*fr)(void*, void*), void* ctx, void* p) {
  if (fr) fr(p, ctx);
  else cudaFree(p);
}

template <typename T>
ib_status dalloc(Engine& E, T** p, int64_t n, bool zero = false) {
  size_t bytes = size_t(std::max<int64_t>(n, 1)) * sizeof(T);
  void* ptr = raw_alloc(E.alloc, E.actx, bytes);
  if (!ptr) { E.err = "device allocation failed"; return IB_ENOMEM; }
  E.allocs.push_back(ptr);
  if (reinterpret_cast<uintptr_t>(ptr) % 256) { E.err = "device allocator returned a block not 256-byte aligned"; return IB_ENOMEM; }
  E.bytes += int64_t(bytes);
  *p = static_cast<T*>(ptr);
  if (zero) CK(cudaMemsetAsync(ptr, 0, bytes, E.st));
  return IB_OK;
}

template <typename T>
ib_status upload(Engine& E, T** p, const std::vector<T>& v) {
  TRY(dalloc(E, p, int64_t(v.size())));
  if (!v.empty()) CK(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, E.st));
  return IB_OK;
}

void engine_free(Engine& E) {
  if (E.st) cudaStreamSynchronize(E.st);
  for (int k = 0; k < 2; ++k)
    if (E.gexec[k]) { cudaGraphExecDestroy(E.gexec[k]); E.gexec[k] = nullptr; }
  for (void* p : E.allocs) raw_free(E.freef, E.actx, p);
  E.allocs.clear();
  E.bytes = 0;
  E.prof.release();
  for (cudaStream_t s : E.cc.side) cudaStreamDestroy(s);
  E.cc.side.clear();
  if (E.cap_st) { cudaStreamDestroy(E.cap_st); E.cap_st = nullptr; }
  if (E.ks_host) { cudaFreeHost(E.ks_host); E.ks_host = nullptr; }
  if (E.os_host) { cudaFreeHost(E.os_host); E.os_host = nullptr; }
  if (E.recs_host) { cudaFreeHost(E.recs_host); E.recs_host = nullptr; }
  if (E.ok_host) { cudaFreeHost(E.ok_host); E.ok_host = nullptr; }
  if (E.aerr_host) { cudaFreeHost(E.aerr_host); E.aerr_host = nullptr; }
}

// Concatenate the members' multigrid hierarchies level by level and upload
// them in the engine's Krylov precision T.
// Level 0's weight-free transfer tables (MGHost::lat0 and following),
// concatenated over the problems with multigrid.
template <typename T>
ib_status mg_upload_level0(Engine& E, const std::vector<uint8_t>& on, const std::vector<int32_t>& noff0,
                           MGLevelDev<T>& L) {
  const int n = E.ninst;
  std::vector<int32_t> bco, lat, latn(3 * n, 0), pbase, fbr, r0slot, r0ptr(1, 0), r0idx, fnode;
  std::vector<int64_t> latoff(n, 0), fbase;
  int64_t npart = 0;
  for (int i = 0; i < n; ++i) {
    const HostGrid& H = *E.H[i];
    bco.insert(bco.end(), H.brick_coord.begin(), H.brick_coord.end());
    const int32_t B0 = int32_t(E.brick0[i]);
    if (!on[i]) {
      pbase.insert(pbase.end(), size_t(H.nbricks), -1);
      fbase.insert(fbase.end(), size_t(H.nbricks), int64_t(0));
      continue;
    }
    const MGHost& m = *E.MG[i];
    latoff[i] = int64_t(lat.size());
    lat.insert(lat.end(), m.lat0.begin(), m.lat0.end());
    for (int a = 0; a < 3; ++a) latn[3 * i + a] = int32_t(m.lat_n[a]);
    for (int32_t b = 0; b < int32_t(H.nbricks); ++b) {
      const int32_t pb = m.pbase[b];
      pbase.push_back(pb >= 0 ? int32_t(pb + npart) : -1);
      if (pb >= 0) fbr.push_back(b + B0);
      // prolongation footprint: the G0 nodes the brick's slots interpolate from
      fbase.push_back(int64_t(fnode.size()));
      const int l = H.brick_level[b], sc = 1 << l;
      const int nt = l == 0 ? BS : mg_targets_per_axis(l);
      int64_t q0[3];
      for (int a = 0; a < 3; ++a) {
        q0[a] = int64_t(H.brick_coord[3 * b + a]) * BS / sc;
        if (l > 0) q0[a] = std::min<int64_t>(q0[a], m.lat_n[a] - 2);
      }
      for (int tz = 0; tz < nt; ++tz)
        for (int ty = 0; ty < nt; ++ty)
          for (int tx = 0; tx < nt; ++tx) {
            const int64_t q[3] = {q0[0] + tx, q0[1] + ty, q0[2] + tz};
            int32_t id = -1;
            if (q[0] < m.lat_n[0] && q[1] < m.lat_n[1] && q[2] < m.lat_n[2]) {
              const int32_t v = m.lat0[(q[2] * m.lat_n[1] + q[1]) * m.lat_n[0] + q[0]];
              if (v >= 0) id = v + noff0[i];
            }
            fnode.push_back(id);
          }
    }
    for (size_t j = 0; j < m.r0slot.size(); ++j) {
      r0slot.push_back(m.r0slot[j] >= 0 ? int32_t(m.r0slot[j] + E.slot0[i]) : -1);
      for (int32_t e = m.r0ptr[j]; e < m.r0ptr[j + 1]; ++e) r0idx.push_back(int32_t(m.r0idx[e] + npart));
      r0ptr.push_back(int32_t(r0idx.size()));
    }
    npart += m.npart;
  }
  if (npart >= (int64_t(1) << 31) || int64_t(r0slot.size()) != int64_t(noff0[n])) {
    E.err = "multigrid transfer tables do not match the G0 levels";
    return IB_EINVAL;
  }
  int32_t *d_bco, *d_lat, *d_latn, *d_pbase, *d_fbr, *d_r0slot, *d_r0ptr, *d_r0idx, *d_fnode;
  int64_t *d_latoff, *d_fbase;
  T *d_part, *d_fp;
  TRY(upload(E, &d_fbase, fbase));
  TRY(upload(E, &d_fnode, fnode));
  TRY(dalloc(E, &d_fp, std::max<int64_t>(int64_t(fnode.size()), 1), true));
  L.fbase = d_fbase; L.fnode = d_fnode; L.fp = d_fp; L.nfp = int64_t(fnode.size());
  TRY(upload(E, &d_bco, bco));
  TRY(upload(E, &d_lat, lat));
  TRY(upload(E, &d_latoff, latoff));
  TRY(upload(E, &d_latn, latn));
  TRY(upload(E, &d_pbase, pbase));
  TRY(upload(E, &d_fbr, fbr));
  TRY(upload(E, &d_r0slot, r0slot));
  TRY(upload(E, &d_r0ptr, r0ptr));
  TRY(upload(E, &d_r0idx, r0idx));
  TRY(dalloc(E, &d_part, std::max<int64_t>(npart, 1), true));
  L.bco = d_bco; L.lat = d_lat; L.lat_off = d_latoff; L.lat_n = d_latn; L.pbase = d_pbase;
  L.fbr = d_fbr; L.nfb = int32_t(fbr.size()); L.part = d_part;
  L.r0slot = d_r0slot; L.r0ptr = d_r0ptr; L.r0idx = d_r0idx;
  return IB_OK;
}

template <typename T>
ib_status mg_upload(Engine& E, MGDev<T>& D) {
  const int n = E.ninst;
  D = MGDev<T>();
  D.ninst = n;
  if (E.D[0].tune[IB_TUNE_MG_SWEEPS] > 0) D.nu = E.D[0].tune[IB_TUNE_MG_SWEEPS];
  std::vector<uint8_t> on(n, 0);
  std::vector<int32_t> small(n, -1), coarsest(n, -1);
  std::vector<int64_t> coff(n, 0);
  std::vector<T> cinv;
  int nlev = 0;
  for (int i = 0; i < n; ++i) {
    const MGHost* m = E.MG[i];
    if (!m || !m->ok || int(m->lev.size()) > MG_LEVELS_MAX) continue;
    on[i] = 1;
    small[i] = m->small_start;
    coarsest[i] = int(m->lev.size()) - 1;
    nlev = std::max(nlev, int(m->lev.size()));
    D.max_big = std::max(D.max_big, m->small_start);
    coff[i] = int64_t(cinv.size());
    const int64_t nk = m->lev.back().nn;
    for (int64_t r = 0; r < nk; ++r)   // symmetrised: the preconditioner stays symmetric
      for (int64_t c = 0; c < nk; ++c) cinv.push_back(T(0.5 * (m->cinv[r * nk + c] + m->cinv[c * nk + r])));
    D.any = true;
  }
  D.nlev = nlev;
  if (!D.any) return IB_OK;
  std::vector<std::vector<int32_t>> noff(nlev, std::vector<int32_t>(n + 1, 0));
  for (int k = 0; k < nlev; ++k)
    for (int i = 0; i < n; ++i) {
      const MGHost* m = E.MG[i];
      const int64_t nn = (on[i] && k < int(m->lev.size())) ? m->lev[k].nn : 0;
      noff[k][i + 1] = int32_t(noff[k][i] + nn);
    }
  for (int k = 0; k < nlev; ++k) {
    MGLevelDev<T>& L = D.lev[k];
    const int64_t N = noff[k][n];
    L.n = N;
    std::vector<int32_t> inst, nbr, rptr(1, 0), rcol, pptr(1, 0), pcol;
    std::vector<T> offd, diag, dinv, rw, pw;
    inst.reserve(N);
    for (int i = 0; i < n; ++i) {
      if (!on[i] || k >= int(E.MG[i]->lev.size())) continue;
      const MGLevelHost& M = E.MG[i]->lev[k];
      const int32_t o = noff[k][i];
      for (int64_t j = 0; j < M.nn; ++j) {
        inst.push_back(i);
        for (int d = 0; d < 6; ++d) {
          const int32_t nb = M.nbr[6 * j + d];
          nbr.push_back(nb >= 0 ? nb + o : -1);
          offd.push_back(T(M.offd[6 * j + d]));
        }
        diag.push_back(T(M.diag[j]));
        dinv.push_back(T(1.0 / M.diag[j]));
        if (k > 0)   // level 0 computes its transfers from lattice positions
          for (int32_t e = M.r_ptr[j]; e < M.r_ptr[j + 1]; ++e) {
            rcol.push_back(M.r_col[e] + noff[k - 1][i]);
            rw.push_back(T(M.r_w[e]));
          }
        rptr.push_back(int32_t(rcol.size()));
      }
    }
    if (k == 0) TRY(mg_upload_level0<T>(E, on, noff[0], L));
    // prolongation rows over the finer index space: the nodes of level k-1
    // (level 0 computes its transfers from lattice positions)
    const int64_t nrows = k == 0 ? 0 : int64_t(noff[k - 1][n]);
    pptr.assign(nrows + 1, 0);
    for (int i = 0; i < n && k > 0; ++i) {
      const int64_t r0 = noff[k - 1][i];
      const int64_t r1 = noff[k - 1][i + 1];
      const bool has = on[i] && k < int(E.MG[i]->lev.size());
      for (int64_t r = r0; r < r1; ++r) {
        if (has) {
          const MGLevelHost& M = E.MG[i]->lev[k];
          const int64_t lr = r - r0;
          for (int32_t e = M.p_ptr[lr]; e < M.p_ptr[lr + 1]; ++e) {
            pcol.push_back(M.p_col[e] + noff[k][i]);
            pw.push_back(T(M.p_w[e]));
          }
        }
        pptr[r + 1] = int32_t(pcol.size());
      }
    }
    int32_t *d_inst, *d_noff, *d_nbr, *d_rptr, *d_rcol, *d_pptr, *d_pcol;
    T *d_offd, *d_diag, *d_dinv, *d_rw, *d_pw;
    TRY(upload(E, &d_inst, inst));
    TRY(upload(E, &d_noff, noff[k]));
    TRY(upload(E, &d_nbr, nbr));
    TRY(upload(E, &d_offd, offd));
    TRY(upload(E, &d_diag, diag));
    TRY(upload(E, &d_dinv, dinv));
    TRY(upload(E, &d_rptr, rptr));
    TRY(upload(E, &d_rcol, rcol));
    TRY(upload(E, &d_rw, rw));
    TRY(upload(E, &d_pptr, pptr));
    TRY(upload(E, &d_pcol, pcol));
    TRY(upload(E, &d_pw, pw));
    L.inst = d_inst; L.noff = d_noff; L.nbr = d_nbr; L.offd = d_offd; L.diag = d_diag; L.dinv = d_dinv;
    L.rptr = d_rptr; L.rcol = d_rcol; L.rw = d_rw; L.pptr = d_pptr; L.pcol = d_pcol; L.pw = d_pw;
    TRY(dalloc(E, &L.b, N, true));
    TRY(dalloc(E, &L.xa, N, true));
    TRY(dalloc(E, &L.xb, N, true));
    TRY(dalloc(E, &L.res, N, true));
  }
  std::vector<MGLevelDev<T>> lv(D.lev, D.lev + nlev);
  MGLevelDev<T>* d_lev;
  TRY(upload(E, &d_lev, lv));
  D.dlev = d_lev;
  uint8_t* d_on;
  int32_t *d_small, *d_coarsest;
  int64_t* d_coff;
  T* d_cinv;
  TRY(upload(E, &d_on, on));
  TRY(upload(E, &d_small, small));
  TRY(upload(E, &d_coarsest, coarsest));
  TRY(upload(E, &d_coff, coff));
  TRY(upload(E, &d_cinv, cinv));
  D.on = d_on; D.small = d_small; D.coarsest = d_coarsest; D.cinv_off = d_coff; D.cinv = d_cinv;
  if (E.D[0].tune[IB_TUNE_MG_PERSIST] == 2) {
    D.lv_ctas = mg_levels_ctas<T>();
    if (D.lv_ctas <= 0) { E.err = "no resident grid for the cooperative multigrid kernel"; return IB_ECUDA; }
    TRY(dalloc(E, &D.bar, 2, true));
  }
  return IB_OK;
}

// Concatenate the members' host grids, upload, and build the constant
// preconditioners and the IB force matrices.
ib_status engine_build(Engine& E) {
  const int n = E.ninst;
  E.mixed = E.D[0].precision == IB_MIXED;
  E.sym = E.D[0].viscous_form == IB_VISCOUS_SYM;
  E.tol = tolerances(E.D[0]);
  E.brick0.assign(n + 1, 0);
  E.slot0.assign(n + 1, 0);
  E.ns_i.assign(n, 0);
  E.row0.assign(n + 1, 0);
  E.canon0.assign(n + 1, 0);
  int64_t nif = 0, nkid = 0, nport = 0;
  for (int i = 0; i < n; ++i) {
    const HostGrid& H = *E.H[i];
    E.brick0[i + 1] = E.brick0[i] + H.nbricks;
    E.slot0[i + 1] = E.brick0[i + 1] * BV;
    E.ns_i[i] = H.nbricks * BV;
    E.row0[i + 1] = E.row0[i] + ((H.M + 255) / 256) * 256;
    E.canon0[i + 1] = E.canon0[i] + int64_t(H.canon_slot.size());
  }
  E.nbricks = E.brick0[n];
  E.ns = E.slot0[n];
  E.Mtot = E.row0[n];
  const int64_t ns = E.ns, Mt = E.Mtot;
  if (E.ns > (int64_t(1) << 31) - 1) { E.err = "too many node slots for 32-bit indices"; return IB_EINVAL; }

  // ---- concatenated topology
  std::vector<int32_t> blev, binst, bseg(n + 1), bnbr, ifc, iff, ifo(1, 0), ifk, ifos, hg, hp1, hp2, canon, ins, inp, pins, pinp;
  std::vector<uint16_t> meta;
  std::vector<double> hl(size_t(n) * 12, 0.0), sf(size_t(n) * 4 * SF_STRIDE, 0.0), pdt(n), pnu(n), insh;
  // natural boundary rows of the symmetric viscous form
  std::vector<int32_t> natslot, natoff(1, 0), natent;
  std::vector<int8_t> natcomp;
  std::vector<double> natw;
  std::vector<PortDev> ports;
  for (int i = 0; i < n; ++i) {
    const HostGrid& H = *E.H[i];
    const ib_grid_desc& d = E.D[i];
    const int32_t B0 = int32_t(E.brick0[i]);
    const int64_t S0 = E.slot0[i];
    bseg[i] = B0;
    for (int32_t b = 0; b < H.nbricks; ++b) {
      blev.push_back(H.brick_level[b]);
      binst.push_back(i);
      for (int k = 0; k < 27; ++k) {
        int32_t v = H.brick_nbr[27 * int64_t(b) + k];
        bnbr.push_back(v >= 0 ? v + B0 : -1);
      }
    }
    meta.insert(meta.end(), H.meta.begin(), H.meta.end());
    for (int l = 0; l <= H.L; ++l) {
      const double* h = H.levels[l].h;
      const double V = h[0] * h[1] * h[2];
      double* f = &sf[(i * 4 + l) * SF_STRIDE];
      for (int a = 0; a < 3; ++a) {
        hl[(i * 4 + l) * 3 + a] = h[a];
        f[a] = V / (6.0 * h[a] * h[a]);
        f[4 + a] = V / (24.0 * h[a]);
      }
      f[3] = V / 120.0;
      f[8] = V / (6.0 * h[0] * h[1]);
      f[9] = V / (6.0 * h[1] * h[2]);
      f[10] = V / (6.0 * h[0] * h[2]);
    }
    if (E.sym) {
      NaturalRows R;
      build_natural_rows(d, H, R);
      for (size_t r = 0; r < R.row_slot.size(); ++r) {
        natslot.push_back(int32_t(R.row_slot[r] + S0));
        for (int32_t e = R.row_off[r]; e < R.row_off[r + 1]; ++e) {
          natent.push_back(int32_t(R.ent_slot[e] + S0));
          natcomp.push_back(R.ent_comp[e]);
          natw.push_back(R.ent_w[e]);
        }
        natoff.push_back(int32_t(natent.size()));
      }
    }
    pdt[i] = d.dt;
    pnu[i] = d.nu;
    const int32_t E0 = int32_t(nif);
    for (size_t e = 0; e < H.if_coarse.size(); ++e) {
      ifc.push_back(int32_t(H.if_coarse[e] + S0));
      iff.push_back(int32_t(H.if_fine[e] + S0));
      ifo.push_back(int32_t(nkid + H.if_child_off[e + 1]));
    }
    for (int32_t k : H.if_child) ifk.push_back(int32_t(k + S0));
    for (int32_t v : H.if_of_slot) ifos.push_back(v >= 0 ? v + E0 : -1);
    nif += int64_t(H.if_coarse.size());
    nkid += int64_t(H.if_child.size());
    for (size_t h = 0; h < H.hang_slot.size(); ++h) {
      hg.push_back(int32_t(H.hang_slot[h] + S0));
      hp1.push_back(int32_t(H.hang_p1[h] + S0));
      hp2.push_back(int32_t(H.hang_p2[h] + S0));
    }
    for (int32_t s : H.canon_slot) canon.push_back(int32_t(s + S0));
    for (size_t k = 0; k < H.inlet_slot.size(); ++k) {
      ins.push_back(int32_t(H.inlet_slot[k] + S0));
      inp.push_back(int32_t(H.inlet_port[k] + nport));
      insh.push_back(H.inlet_shape[k]);
    }
    for (size_t k = 0; k < H.pinlet_slot.size(); ++k) {
      pins.push_back(int32_t(H.pinlet_slot[k] + S0));
      pinp.push_back(int32_t(H.pinlet_port[k] + nport));
    }
    for (int q = 0; q < d.n_ports; ++q) {
      const ib_port& P = d.ports[q];
      PortDev pd{};
      pd.axis = P.axis;
      pd.nh = std::min(P.n_harm, 8);
      pd.inst = i;
      pd.a0 = P.a0;
      pd.period = P.period > 0 ? P.period : 1.0;
      for (int k = 0; k < 8; ++k) { pd.a[k] = P.a[k]; pd.b[k] = P.b[k]; }
      ports.push_back(pd);
    }
    nport += d.n_ports;
  }
  bseg[n] = int32_t(E.nbricks);
  // chunks of up to 8 bricks, never straddling two instances
  std::vector<int32_t> cbrick, cseg(n + 1);
  for (int i = 0; i < n; ++i) {
    cseg[i] = int32_t(cbrick.size());
    for (int32_t b = bseg[i]; b < bseg[i + 1]; b += 8) cbrick.push_back(b);
  }
  cseg[n] = int32_t(cbrick.size());
  cbrick.push_back(int32_t(E.nbricks));
  // streaming chunks: a launch choice (IB_TUNE_STREAM_CHUNK), 8 bricks by default
  const int sch = E.D[0].tune[IB_TUNE_STREAM_CHUNK] > 0 ? E.D[0].tune[IB_TUNE_STREAM_CHUNK] : 8;
  std::vector<int32_t> scbrick, scseg(n + 1);
  for (int i = 0; i < n; ++i) {
    scseg[i] = int32_t(scbrick.size());
    for (int32_t b = bseg[i]; b < bseg[i + 1]; b += sch) scbrick.push_back(b);
  }
  scseg[n] = int32_t(scbrick.size());
  scbrick.push_back(int32_t(E.nbricks));
  E.n_inlet = int64_t(ins.size());
  E.n_pinlet = int64_t(pins.size());
  E.n_valid = 0;
  for (uint16_t m : meta)
    if (m & M_VALID) E.n_valid++;
  // compact arrays: per brick a run of its valid slots, starting on a multiple of 4
  std::vector<int32_t> cwo(16 * (E.nbricks + 1));
  int64_t ncomp = 0;
  for (int64_t b = 0; b < E.nbricks; ++b) {
    ncomp = (ncomp + 3) & ~int64_t(3);
    for (int w = 0; w < 16; ++w) {
      cwo[16 * b + w] = int32_t(ncomp);
      for (int l = 0; l < 32; ++l) ncomp += (meta[b * 512 + w * 32 + l] & M_VALID) ? 1 : 0;
    }
  }
  ncomp = (ncomp + 3) & ~int64_t(3);
  if (ncomp >= (int64_t(1) << 31) / 15) { E.err = "grid too large for the compact coefficient arrays"; return IB_EINVAL; }
  for (int w = 0; w < 16; ++w) cwo[16 * E.nbricks + w] = int32_t(ncomp);
  E.ncomp = ncomp;

  DevGrid& g = E.g;
  g = DevGrid();
  g.nbricks = int32_t(E.nbricks);
  g.nslots = ns;
  g.ninst = n;
  int32_t *d_blev, *d_binst, *d_bseg, *d_bnbr, *d_ifc, *d_iff, *d_ifo, *d_ifk, *d_ifos, *d_hg, *d_hp1, *d_hp2;
  uint16_t* d_meta;
  double *d_hl, *d_pnu, *d_sf64;
  float* d_sf32;
  std::vector<float> sf32(sf.begin(), sf.end());
  TRY(upload(E, &d_blev, blev));
  TRY(upload(E, &d_binst, binst));
  TRY(upload(E, &d_bseg, bseg));
  TRY(upload(E, &d_bnbr, bnbr));
  TRY(upload(E, &d_meta, meta));
  TRY(upload(E, &d_hl, hl));
  int32_t *d_cbrick, *d_cseg, *d_scbrick, *d_scseg;
  TRY(upload(E, &d_cbrick, cbrick));
  TRY(upload(E, &d_cseg, cseg));
  TRY(upload(E, &d_scbrick, scbrick));
  TRY(upload(E, &d_scseg, scseg));
  TRY(upload(E, &d_sf64, sf));
  TRY(upload(E, &d_sf32, sf32));
  TRY(upload(E, &E.pdt, pdt));
  TRY(upload(E, &d_pnu, pnu));
  TRY(upload(E, &d_ifc, ifc));
  TRY(upload(E, &d_iff, iff));
  TRY(upload(E, &d_ifo, ifo));
  TRY(upload(E, &d_ifk, ifk));
  TRY(upload(E, &d_ifos, ifos));
  TRY(upload(E, &d_hg, hg));
  TRY(upload(E, &d_hp1, hp1));
  TRY(upload(E, &d_hp2, hp2));
  int32_t* d_cwo;
  TRY(upload(E, &d_cwo, cwo));
  {
    int32_t *d_ns, *d_no, *d_ne;
    int8_t* d_nc;
    double* d_nw;
    float* d_nw32;
    std::vector<float> natw32(natw.begin(), natw.end());
    TRY(upload(E, &d_ns, natslot));
    TRY(upload(E, &d_no, natoff));
    TRY(upload(E, &d_ne, natent));
    TRY(upload(E, &d_nc, natcomp));
    TRY(upload(E, &d_nw, natw));
    TRY(upload(E, &d_nw32, natw32));
    g.sym = E.sym ? 1 : 0;
    g.n_nat = int32_t(natslot.size());
    g.nat_slot = d_ns;
    g.nat_off = d_no;
    g.nat_ent = d_ne;
    g.nat_comp = d_nc;
    g.nat_w64 = d_nw;
    g.nat_w32 = d_nw32;
  }
  TRY(dalloc(E, &E.aerr, n, true));
  g.cwo = d_cwo;
  g.ncomp = E.ncomp;
  g.aerr = E.aerr;
  g.blev = d_blev; g.binst = d_binst; g.bseg = d_bseg; g.bnbr = d_bnbr; g.meta = d_meta;
  g.nchunks = int32_t(cbrick.size()) - 1;
  g.cbrick = d_cbrick;
  g.cseg = d_cseg;
  g.nschunks = int32_t(scbrick.size()) - 1;
  g.scbrick = d_scbrick;
  g.scseg = d_scseg;
  g.poisson_kernel = E.D[0].tune[IB_TUNE_POISSON_KERNEL];
  g.hl = d_hl; g.pdt = E.pdt; g.pnu = d_pnu; g.sf64 = d_sf64; g.sf32 = d_sf32;
  g.n_if = int32_t(ifc.size());
  g.if_c = d_ifc; g.if_f = d_iff; g.if_off = d_ifo; g.if_kid = d_ifk; g.if_of_slot = d_ifos;
  g.n_hang = int32_t(hg.size());
  g.hg = d_hg; g.hp1 = d_hp1; g.hp2 = d_hp2;
  TRY(upload(E, &E.canon, canon));
  TRY(upload(E, &E.in_slot, ins));
  TRY(upload(E, &E.in_port, inp));
  TRY(upload(E, &E.in_shape, insh));
  TRY(upload(E, &E.pin_slot, pins));
  TRY(upload(E, &E.pin_port, pinp));
  TRY(upload(E, &E.ports, ports));
  TRY(dalloc(E, &E.tc, n, true));
  TRY(dalloc(E, &E.tn, n, true));
  TRY(dalloc(E, &E.ok, n, true));

  // ---- fields and work
  TRY(dalloc(E, &E.ubuf[0], 3 * ns, true));
  TRY(dalloc(E, &E.ubuf[1], 3 * ns, true));
  TRY(dalloc(E, &E.pbuf[0], ns, true));
  TRY(dalloc(E, &E.pbuf[1], ns, true));
  E.u = E.ubuf[0]; E.un = E.ubuf[1]; E.p = E.pbuf[0]; E.pn = E.pbuf[1];
  TRY(dalloc(E, &E.phi, ns, true));
  TRY(dalloc(E, &E.ut, 3 * ns, true));
  TRY(dalloc(E, &E.uib, 3 * ns, true));
  TRY(dalloc(E, &E.rhs3, 3 * ns, true));
  TRY(dalloc(E, &E.y64, 3 * ns, true));
  TRY(dalloc(E, &E.r64, 3 * ns, true));
  TRY(dalloc(E, &E.w64, E.mixed ? 1 : 8 * 3 * ns, true));
  // the FP64 momentum coefficients: FP64 path, and the symmetric form's FP64
  // residual on the mixed path; otherwise the mixed path keeps FP32 pairs
  const bool coef_pairs = E.mixed && !E.sym;
  if (!coef_pairs) TRY(dalloc(E, &E.coef64, 15 * ns, true));
  TRY(dalloc(E, &E.diag64, ns, true));
  TRY(dalloc(E, &E.dK64, ns, true));
  TRY(dalloc(E, &E.dM64, ns, true));
  TRY(dalloc(E, &E.dA64, ns, true));
  if (E.mixed) {
    TRY(dalloc(E, &E.coef32, 15 * E.ncomp, true));   // compact layout (valid slots only)
    if (coef_pairs) TRY(dalloc(E, &E.coeflo32, 15 * E.ncomp, true));
    TRY(dalloc(E, &E.diag32, ns, true));
    TRY(dalloc(E, &E.dK32, ns, true));
    TRY(dalloc(E, &E.dM32, ns, true));
    TRY(dalloc(E, &E.dA32, ns, true));
    TRY(dalloc(E, &E.r32, 3 * ns, true));
    TRY(dalloc(E, &E.e32, 3 * ns, true));
    TRY(dalloc(E, &E.w32, 8 * 3 * ns, true));
  }

  // ---- Poisson multigrid, in the precision of the inner Krylov iterations
  CK(fe_configure());
  {
    // schedule of the persistent staged Poisson stencil: a whole number of
    // CTAs per SM (never more than chunks); CTA c takes the chunks c, c + G, ...
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int per_sm = fe_p7_ctas_per_sm();
    const int nch = g.nchunks;
    const int G = std::min<int64_t>(int64_t(nsm) * per_sm, nch);
    std::vector<int32_t> poff(size_t(std::max(G, 0)) + 1, 0);
    std::vector<P7Hdr> phdr;
    phdr.reserve(size_t(E.nbricks));
    static const int face27[6] = {12, 14, 10, 16, 4, 22};   // -x, +x, -y, +y, -z, +z
    for (int c0 = 0; c0 < G; ++c0) {
      for (int c = c0; c < nch; c += G)
        for (int32_t b = cbrick[c]; b < cbrick[c + 1]; ++b) {
          P7Hdr h{};
          h.b = b;
          for (int f = 0; f < 6; ++f) h.nb[f] = bnbr[27 * int64_t(b) + face27[f]];
          h.inst = binst[b];
          h.chunk = c;
          h.last = b == cbrick[c + 1] - 1;
          for (int a = 0; a < 3; ++a) h.fac[a] = sf32[size_t((binst[b] * 4 + blev[b]) * SF_STRIDE + a)];
          phdr.push_back(h);
        }
      poff[c0 + 1] = int32_t(phdr.size());
    }
    int32_t* d_poff;
    TRY(upload(E, &d_poff, poff));
    P7Hdr* d_phdr;
    TRY(upload(E, &d_phdr, phdr));
    g.p7_ctas = G;
    g.p7_off = d_poff;
    g.p7_hdr = reinterpret_cast<const int4*>(d_phdr);
  }
  if (E.mixed) TRY(mg_upload<float>(E, E.mg32));
  else TRY(mg_upload<double>(E, E.mg64));

  // ---- IB, rows padded per instance to whole 256-row blocks
  std::vector<double> X(3 * Mt, 0.0), dSv(Mt, 1.0), UB(3 * Mt, 0.0), pscale(Mt, 0.0), iorg(3 * n), ihf(3 * n),
      icoef(n);
  std::vector<int32_t> org(3 * Mt, 0), slot(64 * Mt, -1), pinst(Mt, 0), rowptr(Mt + 1, 0), col, segt(n + 1),
      segw(n + 1), segg(n + 1), sps, spo(1, 0), spe;
  std::vector<uint64_t> fb(Mt, 0);
  for (int i = 0; i < n; ++i) {
    const HostGrid& H = *E.H[i];
    const int64_t R0 = E.row0[i], S0 = E.slot0[i];
    const double h3 = H.hf[0] * H.hf[1] * H.hf[2];
    const double sc = E.D[i].dt / (E.D[i].rho * h3);
    segt[i] = int32_t(R0 / 256);
    segw[i] = int32_t(R0 / 8);
    segg[i] = int32_t(R0 / 32);
    for (int a = 0; a < 3; ++a) { iorg[3 * i + a] = H.origin[a]; ihf[3 * i + a] = H.hf[a]; }
    icoef[i] = sc;
    for (int64_t r = R0; r < E.row0[i + 1]; ++r) { pinst[r] = i; pscale[r] = sc; }
    for (int64_t k = 0; k < H.M; ++k) {
      const int64_t r = R0 + k;
      for (int a = 0; a < 3; ++a) {
        X[3 * r + a] = H.X[3 * k + a];
        UB[3 * r + a] = H.UB[3 * k + a];
        org[3 * r + a] = H.ib_origin[3 * k + a];
      }
      dSv[r] = H.dS[k];
      fb[r] = H.ib_free[k];
      for (int a = 0; a < 64; ++a) {
        int32_t s = H.ib_slot[64 * k + a];
        slot[64 * r + a] = s >= 0 ? int32_t(s + S0) : -1;
      }
    }
  }
  segt[n] = int32_t(Mt / 256);
  segw[n] = int32_t(Mt / 8);
  segg[n] = int32_t(Mt / 32);
  for (int i = 0; i < n; ++i) {   // A_F pattern and spreading lists with global rows and slots
    const HostGrid& H = *E.H[i];
    const int64_t R0 = E.row0[i];
    for (int64_t k = 0; k < H.M; ++k) {
      for (int32_t e = H.af_rowptr[k]; e < H.af_rowptr[k + 1]; ++e) col.push_back(int32_t(H.af_col[e] + R0));
      rowptr[R0 + k + 1] = int32_t(col.size());
    }
    for (int64_t r = R0 + H.M; r < E.row0[i + 1]; ++r) rowptr[r + 1] = int32_t(col.size());
    for (size_t q = 0; q < H.sp_slot.size(); ++q) {
      sps.push_back(int32_t(H.sp_slot[q] + E.slot0[i]));
      for (int32_t e = H.sp_off[q]; e < H.sp_off[q + 1]; ++e) {
        const int32_t ent = H.sp_ent[e];
        spe.push_back(int32_t(((ent >> 6) + R0) * 64 + (ent & 63)));
      }
      spo.push_back(int32_t(spe.size()));
    }
  }
  IBDev& ib = E.ib;
  ib = IBDev();
  ib.M = Mt;
  ib.ninst = n;
  int32_t *d_org, *d_slot, *d_rp, *d_col, *d_sps, *d_spo, *d_spe, *d_pinst, *d_segt, *d_segw, *d_segg;
  uint64_t* d_fb;
  double *d_pscale, *d_iorg, *d_ihf, *d_icoef;
  TRY(upload(E, &E.X, X));
  TRY(upload(E, &E.dS, dSv));
  TRY(upload(E, &E.UB, UB));
  TRY(upload(E, &d_org, org));
  TRY(upload(E, &d_slot, slot));
  TRY(upload(E, &d_fb, fb));
  TRY(upload(E, &d_rp, rowptr));
  TRY(upload(E, &d_col, col));
  TRY(upload(E, &d_sps, sps));
  TRY(upload(E, &d_spo, spo));
  TRY(upload(E, &d_spe, spe));
  TRY(upload(E, &d_pinst, pinst));
  TRY(upload(E, &d_segt, segt));
  TRY(upload(E, &d_segw, segw));
  TRY(upload(E, &d_segg, segg));
  TRY(upload(E, &d_pscale, pscale));
  TRY(upload(E, &d_iorg, iorg));
  TRY(upload(E, &d_ihf, ihf));
  TRY(upload(E, &d_icoef, icoef));
  ib.X = E.X; ib.org = d_org; ib.slot = d_slot; ib.freeb = d_fb; ib.rowptr = d_rp; ib.col = d_col;
  ib.sp_slot = d_sps; ib.sp_off = d_spo; ib.sp_ent = d_spe; ib.n_sp = int64_t(sps.size());
  ib.pinst = d_pinst; ib.seg_t = d_segt; ib.seg_w = d_segw; ib.seg_g = d_segg; ib.pscale = d_pscale;
  ib.iorigin = d_iorg; ib.ihf = d_ihf; ib.icoef = d_icoef; ib.binst = d_binst;
  TRY(dalloc(E, &ib.W, 64 * Mt, true));
  TRY(dalloc(E, &ib.val, int64_t(col.size()), true));
  E.af_cap = int64_t(col.size());
  if (E.mixed) {
    TRY(dalloc(E, &ib.val32, int64_t(col.size()), true));
    TRY(dalloc(E, &ib.dinv32, Mt, true));
    TRY(dalloc(E, &E.ib_y64, 3 * Mt, true));
    TRY(dalloc(E, &E.ib_w32, 7 * 3 * Mt, true));
  }
  TRY(dalloc(E, &ib.dinv, Mt, true));
  TRY(dalloc(E, &E.BF, 3 * Mt, true));
  TRY(dalloc(E, &E.Gf, 3 * Mt, true));
  TRY(dalloc(E, &E.ibw, 5 * 3 * Mt, true));

  // ---- reductions, solver state, streams
  const int64_t maxblk = std::max<int64_t>(E.nbricks, Mt / 8 + 1);
  TRY(dalloc(E, &E.rb.partials, maxblk * 16 + int64_t(n) * 16 + 64, true));
  TRY(dalloc(E, &E.rb.counter, 1, true));
  TRY(dalloc(E, &E.ks, 3 * n, true));
  TRY(dalloc(E, &E.os, n, true));
  TRY(dalloc(E, &E.recs, 4 * n, true));
  CK(cudaMallocHost(&E.ks_host, 3 * n * sizeof(KState)));
  CK(cudaMallocHost(&E.os_host, n * sizeof(OState)));
  CK(cudaMallocHost(&E.recs_host, 4 * n * sizeof(SolveRec)));
  CK(cudaMallocHost(&E.ok_host, n * sizeof(int32_t)));
  CK(cudaMallocHost(&E.aerr_host, n * sizeof(int32_t)));
  for (int k = 0; k < 4; ++k) {
    cudaStream_t s2;
    CK(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
    E.cc.side.push_back(s2);
  }
  CK(cudaStreamCreateWithFlags(&E.cap_st, cudaStreamNonBlocking));

  // ---- constant preconditioners, IB weights and force matrix
  const DevGrid& dg = E.g;
  fe_jacobi<double>(dg, OP_POISSON, nullptr, D_PDIR, E.diag64, E.dK64, E.st);
  fe_jacobi<double>(dg, OP_MASS, nullptr, D_VDIR, E.diag64, E.dM64, E.st);
  if (E.mixed) {
    fe_jacobi<float>(dg, OP_POISSON, nullptr, D_PDIR, E.diag32, E.dK32, E.st);
    fe_jacobi<float>(dg, OP_MASS, nullptr, D_VDIR, E.diag32, E.dM32, E.st);
  }
  ib_weights(E.ib, E.st);
  ib_assemble(E.ib, E.st);
  E.step.assign(n, 0);
  E.time.assign(n, 0.0);
  E.last.assign(n, ib_info{});
  E.status.assign(n, 0);
  cudaError_t e = cudaStreamSynchronize(E.st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) { E.err = std::string("CUDA: ") + cudaGetErrorString(e); return IB_ECUDA; }
  return IB_OK;
}

SolveArgs solve_args(Engine& E, int op, bool bicg, int nc, uint16_t dmask, const double* coef64,
                     const double* dinv64, const float* coef32, const float* dinv32, const double* b, double* x,
                     double rtol, int rec) {
  SolveArgs a;
  a.g = &E.g;
  a.op = op;
  a.nc = nc;
  a.dmask = dmask;
  a.bicg = bicg;
  a.mixed = E.mixed;
  a.coupled = bicg && nc == 3 && E.sym;   // the symmetric viscous form couples the momentum components
  a.coef64 = coef64;
  a.dinv64 = dinv64;
  a.coef32 = coef32;
  a.coeflo32 = op == OP_COEF ? E.coeflo32 : nullptr;
  a.dinv32 = dinv32;
  a.b = b;
  a.x = x;
  a.rtol = rtol;
  // FP32 iterations cut the true FP64 residual by at most ~kappa * eps32 per
  // outer pass; for the ill-conditioned Poisson problem a looser inner
  // tolerance reaches that with fewer iterations
  a.rtol_inner = std::max(op == OP_POISSON ? E.tol.inner_p : E.tol.inner, rtol);
  a.max_iter = E.tol.max_iter;
  a.w64 = E.w64;
  a.w32 = E.w32;
  a.y64 = E.y64;
  a.r64 = E.r64;
  a.r32 = E.r32;
  a.e32 = E.e32;
  a.ks = E.ks;
  a.os = E.os;
  a.rec = E.recs + rec;
  a.rb = E.rb;
  a.prof = E.prof.on ? &E.prof : nullptr;
  a.pbase = op == OP_POISSON ? 0 : op == OP_MASS ? 3 : 6;
  a.ks_host = E.ks_host;
  a.os_host = E.os_host;
  if (op == OP_POISSON) {
    a.mg32 = E.mixed ? &E.mg32 : nullptr;
    a.mg64 = E.mixed ? nullptr : &E.mg64;
  }
  return a;
}

// Enqueue one step of every instance (reading u, p; writing un, pn) on st.
cudaError_t enqueue_step(Engine& E, double* u, double* un, double* p, double* pn, cudaStream_t st) {
  const DevGrid& dg = E.g;
  const int64_t ns = dg.nslots;
  const Tols& tl = E.tol;
  CaptureCtx* cc = &E.cc;
  cudaError_t e;

  rec_clear(E.recs, 4 * E.ninst, st);
  if ((e = cudaMemsetAsync(E.aerr, 0, E.ninst * sizeof(int32_t), st)) != cudaSuccess) return e;
  {
    unsigned* bar = E.mixed ? E.mg32.bar : E.mg64.bar;
    if (bar && (e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st)) != cudaSuccess) return e;
  }
  fe_time_advance(E.tc, E.tn, E.pdt, E.ninst, 0, nullptr, st);
  // ---- Step 1: tentative velocity (Eq. 9)
  // (the mixed path's FP64 outer loop needs no FP64 Jacobi diagonal)
  if (E.coeflo32) fe_momentum_coef_ff(dg, u, E.coef32, E.coeflo32, st);
  else fe_momentum_coef(dg, u, E.coef64, E.mixed ? E.coef32 : nullptr, st);
  if (!E.mixed) fe_jacobi<double>(dg, OP_COEF, E.coef64, D_VDIR, E.diag64, E.dA64, st);
  else fe_jacobi<float>(dg, OP_COEF, E.coef32, D_VDIR, E.diag32, E.dA32, st);
  fe_rhs_mass_grad(dg, u, p, E.rhs3, st, E.mixed);
  fe_sync<double>(dg, 3, E.rhs3, D_VDIR, st);
  fe_copy_d(3 * ns, u, E.ut, st);
  fe_set_inlet(E.n_inlet, E.in_slot, E.in_port, E.in_shape, E.ports, E.tn, ns, E.ut, st);
  fe_expand<double>(dg, 3, E.ut, st);
  e = solve_enqueue(solve_args(E, OP_COEF, true, 3, D_VDIR, E.coef64, E.dA64, E.coef32, E.dA32, E.rhs3, E.ut,
                               tl.mom, 0), st, cc);
  if (e != cudaSuccess) return e;

  // ---- Steps 2-4: BCE-IB force and correction (Eq. 14, 19-23)
  fe_copy_d(3 * ns, E.ut, E.uib, st);
  if (E.Mtot) {
    ib_gather(E.ib, E.ut, ns, E.UB, E.BF, st);
    if (E.mixed) {   // FP32 iterations inside FP64 defect correction, as the field solves
      e = ib_solve_mixed(E.ib, E.BF, E.Gf, E.ib_y64, E.ib_w32, E.ks, E.ks_host, E.os, E.os_host, E.rb, tl.ib,
                         std::max(tl.inner, tl.ib), tl.max_iter, 30, E.recs + 1, st, cc);
      if (e == cudaSuccess)
        e = ib_fp64_fallback(E.ib, E.BF, E.Gf, E.ibw, E.ks, E.ks_host, E.os, E.os_host, E.rb, tl.ib, tl.max_iter,
                             E.recs + 1, st, cc);
    } else
      e = ib_solve(E.ib, E.BF, E.Gf, E.ibw, E.ks, E.ks_host, E.rb, tl.ib, tl.max_iter, E.recs + 1, st, cc);
    if (e != cudaSuccess) return e;
    ib_spread(E.ib, E.Gf, E.uib, ns, st);
  }

  // ---- Step 5: pressure increment (Eq. 12); Phi = p_in(t^{n+1}) - p^n on
  // pressure-inlet nodes (the solve keeps the Dirichlet values of its start).
  // The warm start's hanging values are reset to the mean of their parents for
  // every member, with or without a pressure inlet, so that a member's bits do
  // not depend on the batch it runs in.
  double* rhs1 = E.rhs3;   // component 0 of the RHS buffer
  fe_rhs_div(dg, E.uib, rhs1, st, E.mixed);
  fe_sync<double>(dg, 1, rhs1, D_PDIR, st);
  if (E.n_pinlet) fe_set_pinlet(E.n_pinlet, E.pin_slot, E.pin_port, E.ports, E.tn, p, E.phi, st);
  fe_expand<double>(dg, 1, E.phi, st);
  e = solve_enqueue(solve_args(E, OP_POISSON, false, 1, D_PDIR, nullptr, E.dK64, nullptr, E.dK32, rhs1, E.phi,
                               tl.p, 2), st, cc);
  if (e != cudaSuccess) return e;

  // ---- Step 6: velocity correction and pressure update
  fe_rhs_mass_grad(dg, E.uib, E.phi, E.rhs3, st, E.mixed);
  fe_sync<double>(dg, 3, E.rhs3, D_VDIR, st);
  fe_copy_d(3 * ns, E.uib, un, st);
  e = solve_enqueue(solve_args(E, OP_MASS, false, 3, D_VDIR, nullptr, E.dM64, nullptr, E.dM32, E.rhs3, un,
                               tl.corr, 3), st, cc);
  if (e != cudaSuccess) return e;
  fe_copy_d(ns, p, pn, st);
  fe_add_d(ns, E.phi, pn, st);
  e = cudaMemcpyAsync(E.aerr_host, E.aerr, E.ninst * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(E.recs_host, E.recs, 4 * E.ninst * sizeof(SolveRec), cudaMemcpyDeviceToHost, st);
}

// One step of every instance.  Returns the worst status; per-instance status
// in E.status (an instance whose solves failed keeps its previous state).
ib_status engine_step(Engine& E) {
  cudaStream_t st = E.st;
  const int par = (E.u == E.ubuf[0]) ? 0 : 1;
  if (E.use_graph) {
    if (!E.gexec[par]) {
      cudaGraph_t graph = nullptr;
      cudaStream_t cs = E.cap_st;
      CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      E.cc.capturing = true;
      E.cc.depth = 0;
      cudaError_t e = enqueue_step(E, E.u, E.un, E.p, E.pn, cs);
      E.cc.capturing = false;
      cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        E.err = std::string("graph capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2);
        return IB_ECUDA;
      }
      e = cudaGraphInstantiate(&E.gexec[par], graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        E.gexec[par] = nullptr;
        E.err = std::string("graph instantiation failed: ") + cudaGetErrorString(e);
        return IB_ECUDA;
      }
    }
    CK(cudaGraphLaunch(E.gexec[par], st));
  } else {
    E.cc.capturing = false;
    cudaError_t e = enqueue_step(E, E.u, E.un, E.p, E.pn, st);
    if (e != cudaSuccess) {
      E.err = std::string("CUDA: ") + cudaGetErrorString(e);
      return IB_ECUDA;
    }
  }
  CK(cudaStreamSynchronize(st));
  CK(cudaGetLastError());
  if (E.prof.on) E.prof.collect();
  int worst = 0;
  bool any_fail = false;
  for (int i = 0; i < E.ninst; ++i) {
    const SolveRec* R = E.recs_host + 4 * i;
    ib_info& I = E.last[i];
    int status = 0;
    for (int k = 0; k < 4; ++k) status = std::max(status, int(R[k].status));
    status = std::max(status, int(E.aerr_host[i]));   // a bounded wait that ran out
    for (int c = 0; c < 3; ++c) {
      I.iters_mom[c] = R[0].iters[c];
      I.iters_corr[c] = R[3].iters[c];
    }
    I.iters_ib = std::max(R[1].iters[0], std::max(R[1].iters[1], R[1].iters[2]));
    I.iters_p = R[2].iters[0];
    I.outer_mom = R[0].outer;
    I.outer_p = R[2].outer;
    I.outer_corr = R[3].outer;
    I.res_mom = R[0].relres;
    I.res_ib = R[1].relres;
    I.res_p = R[2].relres;
    I.res_corr = R[3].relres;
    I.status_mom = R[0].status;
    I.status_ib = R[1].status;
    I.status_p = R[2].status;
    I.status_corr = R[3].status;
    E.status[i] = status;
    E.ok_host[i] = status == 0;
    if (status) {
      any_fail = true;
      worst = std::max(worst, status);
      // keep the previous state of this instance: next buffers <- current
      const int64_t s0 = E.slot0[i], cnt = E.ns_i[i];
      for (int c = 0; c < 3; ++c)
        CK(cudaMemcpyAsync(E.un + c * E.ns + s0, E.u + c * E.ns + s0, cnt * sizeof(double),
                           cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(E.pn + s0, E.p + s0, cnt * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
      E.step[i] += 1;
      E.time[i] += E.D[i].dt;
    }
  }
  if (any_fail) CK(cudaMemcpyAsync(E.ok, E.ok_host, E.ninst * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  std::swap(E.u, E.un);
  std::swap(E.p, E.pn);
  fe_time_advance(E.tc, E.tn, E.pdt, E.ninst, 1, any_fail ? E.ok : nullptr, st);
  if (any_fail) CK(cudaStreamSynchronize(st));
  if (worst) {
    if (worst == ASYNC_TIMEOUT) {
      E.err = "internal: an asynchronous copy of a step kernel did not complete within its wait limit";
      return IB_ETIMEOUT;
    }
    E.err = worst == 5 ? "Krylov breakdown in a step solve" : "a step solve did not converge";
    return worst == 5 ? IB_EBREAKDOWN : IB_ENOCONV;
  }
  return IB_OK;
}

int64_t field_bytes(const HostGrid& H, int f) {
  const int64_t N = int64_t(H.canon_slot.size()), M = H.M;
  const int64_t nc = H.n[0] * H.n[1] * H.n[2];
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

// host-only fields of a handle
bool host_field(const HostGrid& H, int field, std::vector<uint8_t>& buf) {
  const int64_t M = H.M;
  auto put = [&](const void* p, size_t n) {
    buf.resize(n);
    if (n) std::memcpy(buf.data(), p, n);
  };
  switch (field) {
    case IB_FIELD_NODE_Q: put(H.canon_q.data(), H.canon_q.size() * 4); return true;
    case IB_FIELD_NODE_FLAGS: put(H.canon_flags.data(), H.canon_flags.size()); return true;
    case IB_FIELD_ACTIVE: put(H.active.data(), H.active.size()); return true;
    case IB_FIELD_LEVEL: put(H.level.data(), H.level.size()); return true;
    case IB_FIELD_IB_ORIGIN: put(H.ib_origin.data(), H.ib_origin.size() * 4); return true;
    case IB_FIELD_IB_FREE: {
      buf.assign(64 * M, 0);
      for (int64_t i = 0; i < M; ++i)
        for (int a = 0; a < 64; ++a)
          buf[64 * i + a] = (H.ib_free[i] >> a & 1) ? 1 : (H.ib_slot[64 * i + a] >= 0 ? 2 : 0);
      return true;
    }
    default: return false;
  }
}

ib_status engine_fields_get(Engine& E, int i, int32_t field, void* dst, size_t bytes, int32_t on_dev) {
  const HostGrid& H = *E.H[i];
  cudaStream_t st = E.st;
  const cudaMemcpyKind k_out = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  std::vector<uint8_t> hb;
  if (host_field(H, field, hb)) {
    if (bytes) CK(cudaMemcpyAsync(dst, hb.data(), bytes, on_dev ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, st));
    CK(cudaStreamSynchronize(st));
    return IB_OK;
  }
  const int64_t N = int64_t(H.canon_slot.size()), M = H.M, R0 = E.row0[i];
  switch (field) {
    case IB_FIELD_U: case IB_FIELD_U_TENT: case IB_FIELD_U_IB: case IB_FIELD_P: case IB_FIELD_PHI: {
      const double* src = field == IB_FIELD_U ? E.u : field == IB_FIELD_U_TENT ? E.ut
                        : field == IB_FIELD_U_IB ? E.uib : field == IB_FIELD_P ? E.p : E.phi;
      const int nc = (field == IB_FIELD_P || field == IB_FIELD_PHI) ? 1 : 3;
      double* tmp = E.y64;   // 3 * ns >= nc * N
      fe_gather_canon<double>(N, E.canon + E.canon0[i], nc, E.ns, src, tmp, st);
      CK(cudaMemcpyAsync(dst, tmp, bytes, k_out, st));
      break;
    }
    case IB_FIELD_B_F:
      if (bytes) CK(cudaMemcpyAsync(dst, E.BF + 3 * R0, bytes, k_out, st));
      break;
    case IB_FIELD_IB_WEIGHTS:
      if (bytes) CK(cudaMemcpyAsync(dst, E.ib.W + 64 * R0, bytes, k_out, st));
      break;
    case IB_FIELD_F_LAG: {
      std::vector<double> G(3 * M);
      if (M) CK(cudaMemcpyAsync(G.data(), E.Gf + 3 * R0, bytes, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (int64_t k = 0; k < M; ++k)
        for (int c = 0; c < 3; ++c) G[3 * k + c] /= H.dS[k];
      if (bytes) CK(cudaMemcpyAsync(dst, G.data(), bytes, on_dev ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, st));
      break;
    }
    default: E.err = "field not readable"; return IB_EINVAL;
  }
  CK(cudaStreamSynchronize(st));
  return IB_OK;
}

ib_status engine_fields_set(Engine& E, int i, int32_t field, const void* src, size_t bytes, int32_t on_dev) {
  const HostGrid& H = *E.H[i];
  const int64_t N = int64_t(H.canon_slot.size());
  const int nc = field == IB_FIELD_U ? 3 : 1;
  double* tmp = E.y64;
  CK(cudaMemcpyAsync(tmp, src, bytes, on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, E.st));
  fe_scatter_canon(E.g, N, E.canon + E.canon0[i], nc, tmp, field == IB_FIELD_U ? E.u : E.p, E.st);
  CK(cudaStreamSynchronize(E.st));
  return IB_OK;
}

void fill_info(const HostGrid& H, const MGHost* mg, const Engine* E, int64_t dev_bytes, ib_info& I) {
  I.n_nodes = int64_t(H.canon_slot.size());
  I.mg_levels = (mg && mg->ok) ? int32_t(mg->lev.size()) : 0;
  I.mg_coarsest = (mg && mg->ok) ? int32_t(mg->lev.back().nn) : 0;
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
  int64_t nv = 0;
  for (uint16_t m : H.meta)
    if (m & M_VALID) nv++;
  I.n_valid_slots = nv;
  I.device_bytes = dev_bytes;
  I.kernel_launches = int64_t(fe_kcount() + krylov_kcount() + ib_kcount() + mg_kcount() + move_kcount() + wss_kcount());
  if (E) {
    for (int k = 0; k < Prof::K; ++k) {
      I.prof_ms[k] = E->prof.ms[k];
      I.prof_launches[k] = E->prof.n[k];
    }
  }
}

ib_status validate_desc(const ib_grid_desc* d) {
  for (int a = 0; a < 3; ++a)
    if (d->n[a] <= 0 || !(d->extent[a] > 0) || !std::isfinite(d->origin[a])) return IB_EINVAL;
  if (d->max_level < 0 || d->max_level > IB_MAX_LEVEL) return IB_EINVAL;
  if (d->max_level > 0 && d->refine_band < 1) return IB_EINVAL;
  if (!(d->nu > 0) || !(d->rho > 0) || !(d->dt > 0)) return IB_EINVAL;
  if (d->precision != IB_FP64 && d->precision != IB_MIXED) return IB_EINVAL;
  if (d->poisson_pc != IB_PC_MULTIGRID && d->poisson_pc != IB_PC_JACOBI) return IB_EINVAL;
  if (d->viscous_form != IB_VISCOUS_GRAD && d->viscous_form != IB_VISCOUS_SYM) return IB_EINVAL;
  if (d->n_ports < 1 || d->n_ports > IB_MAX_PORTS) return IB_EINVAL;
  bool outlet = false;
  for (int p = 0; p < d->n_ports; ++p) {
    const ib_port& P = d->ports[p];
    if (P.axis < 0 || P.axis > 2 || (P.side != 0 && P.side != 1) || !(P.radius > 0)) return IB_EINVAL;
    if (P.kind != IB_INLET_VELOCITY && P.kind != IB_OUTLET_ZERO_P && P.kind != IB_INLET_PRESSURE) return IB_EINVAL;
    if (P.n_harm < 0 || P.n_harm > IB_MAX_HARMONICS) return IB_EINVAL;
    if (P.profile != IB_PARABOLIC) return IB_EINVAL;
    if (P.kind != IB_INLET_VELOCITY) outlet = true;   // a port that fixes Phi
  }
  if (!outlet) return IB_EINVAL;
  int64_t nf = (int64_t(d->n[0]) * d->n[1] * d->n[2]) << (3 * d->max_level);
  if (nf > (int64_t(1) << 40)) return IB_EINVAL;
  const int32_t* tu = d->tune;
  if (tu[IB_TUNE_POISSON_KERNEL] < 0 || tu[IB_TUNE_POISSON_KERNEL] > 3) return IB_EINVAL;
  if (tu[IB_TUNE_STREAM_CHUNK] != 0 && tu[IB_TUNE_STREAM_CHUNK] != 4 && tu[IB_TUNE_STREAM_CHUNK] != 8) return IB_EINVAL;
  if (tu[IB_TUNE_MG_SMALL] != 0 && (tu[IB_TUNE_MG_SMALL] < 64 || tu[IB_TUNE_MG_SMALL] > (1 << 20))) return IB_EINVAL;
  if (tu[IB_TUNE_MG_SWEEPS] < 0 || tu[IB_TUNE_MG_SWEEPS] > 4) return IB_EINVAL;
  if (tu[IB_TUNE_MG_PERSIST] < 0 || tu[IB_TUNE_MG_PERSIST] > 2) return IB_EINVAL;
  if (d->port_tangential != IB_TANGENTIAL_FREE && d->port_tangential != IB_TANGENTIAL_ZERO) return IB_EINVAL;
  return IB_OK;
}

void snap_free(ib_grid* g) {
  for (void* p : g->snap_allocs) raw_free(g->d.dev_free, g->d.alloc_ctx, p);
  g->snap_allocs.clear();
  g->snap_bytes = 0;
  g->snap = Snapshot();
}

// allocate a deferred handle's snapshot (zero state)
ib_status snap_alloc(ib_grid* g) {
  snap_free(g);
  cudaStream_t st = static_cast<cudaStream_t>(g->d.stream);
  const int64_t ns = g->H.nbricks * BV, M = g->H.M;
  auto al = [&](void** p, size_t bytes) -> bool {
    const size_t b = std::max<size_t>(bytes, 8);
    *p = raw_alloc(g->d.dev_alloc, g->d.alloc_ctx, b);
    if (!*p) return false;
    g->snap_allocs.push_back(*p);
    g->snap_bytes += int64_t(b);
    return cudaMemsetAsync(*p, 0, b, st) == cudaSuccess;
  };
  if (!al((void**)&g->snap.u, 3 * ns * 8) || !al((void**)&g->snap.p, ns * 8) || !al((void**)&g->snap.phi, ns * 8) ||
      !al((void**)&g->snap.G, 3 * M * 8) || !al((void**)&g->snap.canon, g->H.canon_slot.size() * 4)) {
    g->err = "device allocation failed";
    return IB_ENOMEM;
  }
  if (!g->H.canon_slot.empty())
    cudaMemcpyAsync(g->snap.canon, g->H.canon_slot.data(), g->H.canon_slot.size() * 4, cudaMemcpyHostToDevice, st);
  g->snap.valid = true;
  return cudaStreamSynchronize(st) == cudaSuccess ? IB_OK : IB_ECUDA;
}

// engine instance i <-> member snapshot (u, p, Phi, G, time, step)
ib_status snap_transfer(Engine& E, int i, ib_grid* m, bool to_engine) {
  const int64_t s0 = E.slot0[i], n = E.ns_i[i], R0 = E.row0[i], M = m->H.M;
  cudaStream_t st = E.st;
  const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
  for (int c = 0; c < 3; ++c) {
    double* a = E.u + c * E.ns + s0;
    double* b = m->snap.u + c * n;
    CK(cudaMemcpyAsync(to_engine ? a : b, to_engine ? b : a, n * 8, k, st));
  }
  CK(cudaMemcpyAsync(to_engine ? E.p + s0 : m->snap.p, to_engine ? m->snap.p : E.p + s0, n * 8, k, st));
  CK(cudaMemcpyAsync(to_engine ? E.phi + s0 : m->snap.phi, to_engine ? m->snap.phi : E.phi + s0, n * 8, k, st));
  if (M) CK(cudaMemcpyAsync(to_engine ? E.Gf + 3 * R0 : m->snap.G, to_engine ? m->snap.G : E.Gf + 3 * R0, 3 * M * 8, k, st));
  if (to_engine) {
    E.step[i] = m->snap.step;
    E.time[i] = m->snap.time;
    CK(cudaMemcpyAsync(E.tc + i, &E.time[i], 8, cudaMemcpyHostToDevice, st));
  } else {
    m->snap.step = E.step[i];
    m->snap.time = E.time[i];
  }
  CK(cudaStreamSynchronize(st));
  return IB_OK;
}

}  // namespace

extern "C" {

ib_status ib_grid_create(const ib_grid_desc* d, ib_grid** out) {
  if (!d || !out) return IB_EINVAL;
  *out = nullptr;
  if (validate_desc(d) != IB_OK) return IB_EINVAL;
  ib_grid* g = new (std::nothrow) ib_grid();
  if (!g) return IB_ENOMEM;
  g->d = *d;
  if (cudaGetDevice(&g->device) != cudaSuccess || fe_init_tables() != cudaSuccess) {
    delete g;
    return IB_ECUDA;
  }
  *out = g;
  return IB_OK;
}

ib_status ib_set_boundary(ib_grid* g, int64_t M, const double* X, const double* dS, const double* UB,
                          const uint8_t* inside) {
  if (!g) return IB_EINVAL;
  if (g->batch) { g->err = "the handle is held by a batch"; return IB_ESTATE; }
  if (M < 0 || (M > 0 && (!X || !dS))) { g->err = "bad point arrays"; return IB_EINVAL; }
  if (g->eng) { engine_free(*g->eng); delete g->eng; g->eng = nullptr; }
  snap_free(g);
  g->ready = false;
  ib_status s = build_host_grid(g->d, M, X, dS, UB, inside, g->H, g->err);
  if (s != IB_OK) return s;
  g->mg = MGHost();
  if (g->d.poisson_pc == IB_PC_MULTIGRID)
    build_mg(g->H, g->mg, g->d.tune[IB_TUNE_MG_SMALL] > 0 ? g->d.tune[IB_TUNE_MG_SMALL] : MG_SMALL_NODES);
  if (g->d.deferred) {
    s = snap_alloc(g);
    if (s != IB_OK) return s;
    g->ready = true;
    g->err.clear();
    return IB_OK;
  }
  Engine* E = new (std::nothrow) Engine();
  if (!E) return IB_ENOMEM;
  E->H.push_back(&g->H);
  E->MG.push_back(&g->mg);
  E->D.push_back(g->d);
  E->ninst = 1;
  E->st = static_cast<cudaStream_t>(g->d.stream);
  E->alloc = g->d.dev_alloc;
  E->freef = g->d.dev_free;
  E->actx = g->d.alloc_ctx;
  s = engine_build(*E);
  if (s != IB_OK) {
    g->err = E->err;
    engine_free(*E);
    delete E;
    return s;
  }
  E->prof.on = g->d.profile != 0;
  E->use_graph = !E->prof.on;
  g->eng = E;
  g->ready = true;
  g->err.clear();
  return IB_OK;
}

ib_status ipcs_step(ib_grid* g, int32_t nsteps) {
  if (!g) return IB_EINVAL;
  if (!g->ready) { g->err = "ib_set_boundary has not succeeded"; return IB_ESTATE; }
  if (!g->eng) { g->err = "a deferred handle is stepped through a batch"; return IB_ESTATE; }
  if (nsteps < 0) { g->err = "nsteps < 0"; return IB_EINVAL; }
  for (int32_t k = 0; k < nsteps; ++k) {
    ib_status s = engine_step(*g->eng);
    if (s != IB_OK) { g->err = g->eng->err; return s; }
  }
  return IB_OK;
}

ib_status ib_fields_get(ib_grid* g, int32_t field, void* dst, size_t bytes, int32_t dst_on_device) {
  if (!g) return IB_EINVAL;
  if (!g->ready) { g->err = "ib_set_boundary has not succeeded"; return IB_ESTATE; }
  int64_t need = field_bytes(g->H, field);
  if (need < 0 || int64_t(bytes) != need) { g->err = "bad field id or byte count"; return IB_EINVAL; }
  if (!dst && bytes) return IB_EINVAL;
  if (g->batch) return ib_batch_fields_get(g->batch, g->batch_index, field, dst, bytes, dst_on_device);
  if (g->eng) {
    ib_status s = engine_fields_get(*g->eng, 0, field, dst, bytes, dst_on_device);
    if (s != IB_OK) g->err = g->eng->err;
    return s;
  }
  // deferred handle outside a batch: host fields and the state snapshot
  cudaStream_t st = static_cast<cudaStream_t>(g->d.stream);
  std::vector<uint8_t> hb;
  if (host_field(g->H, field, hb)) {
    if (bytes) cudaMemcpyAsync(dst, hb.data(), bytes, dst_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, st);
    return cudaStreamSynchronize(st) == cudaSuccess ? IB_OK : IB_ECUDA;
  }
  const int64_t N = int64_t(g->H.canon_slot.size()), ns = g->H.nbricks * BV;
  if (field == IB_FIELD_U || field == IB_FIELD_P || field == IB_FIELD_PHI) {
    const int nc = field == IB_FIELD_U ? 3 : 1;
    const double* src = field == IB_FIELD_U ? g->snap.u : field == IB_FIELD_P ? g->snap.p : g->snap.phi;
    double* tmp = static_cast<double*>(raw_alloc(g->d.dev_alloc, g->d.alloc_ctx, size_t(std::max<int64_t>(nc * N, 1)) * 8));
    if (!tmp) return IB_ENOMEM;
    fe_gather_canon<double>(N, g->snap.canon, nc, ns, src, tmp, st);
    cudaMemcpyAsync(dst, tmp, bytes, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    raw_free(g->d.dev_free, g->d.alloc_ctx, tmp);
    return e == cudaSuccess ? IB_OK : IB_ECUDA;
  }
  g->err = "field not available for a deferred handle outside a batch";
  return IB_EINVAL;
}

ib_status ib_fields_set(ib_grid* g, int32_t field, const void* src, size_t bytes, int32_t src_on_device) {
  if (!g || !src) return IB_EINVAL;
  if (!g->ready) { g->err = "ib_set_boundary has not succeeded"; return IB_ESTATE; }
  if (field != IB_FIELD_U && field != IB_FIELD_P) { g->err = "only U and P can be set"; return IB_EINVAL; }
  if (int64_t(bytes) != field_bytes(g->H, field)) { g->err = "bad byte count"; return IB_EINVAL; }
  if (!g->eng) { g->err = "the state of a deferred handle is set through its batch"; return IB_ESTATE; }
  ib_status s = engine_fields_set(*g->eng, 0, field, src, bytes, src_on_device);
  if (s != IB_OK) g->err = g->eng->err;
  return s;
}

ib_status ib_grid_info(const ib_grid* g, ib_info* out) {
  if (!g || !out) return IB_EINVAL;
  if (!g->ready) return IB_ESTATE;
  if (g->batch) return ib_batch_info(g->batch, g->batch_index, out);
  ib_info I = g->eng ? g->eng->last[0] : ib_info{};
  fill_info(g->H, &g->mg, g->eng, g->eng ? g->eng->bytes : g->snap_bytes, I);
  I.step = g->eng ? g->eng->step[0] : g->snap.step;
  I.time = g->eng ? g->eng->time[0] : g->snap.time;
  *out = I;
  return IB_OK;
}

const char* ib_last_error(const ib_grid* g) { return g ? g->err.c_str() : "null handle"; }

void ib_grid_destroy(ib_grid* g) {
  if (!g) return;
  if (g->batch) return;   // a batch still references it: destroy the batch first
  if (g->eng) {
    engine_free(*g->eng);
    delete g->eng;
  }
  snap_free(g);
  delete g;
}

// ---------------------------------------------------------------- moving points
namespace {

MoveGrid move_grid(const Engine& E) {
  MoveGrid G{};
  G.bmap = E.mv_bmap;
  for (int a = 0; a < 3; ++a) {
    G.nb[a] = E.mv_nb[a];
    G.nf[a] = E.mv_nf[a];
  }
  G.meta = E.g.meta;
  G.origin = E.ib.iorigin;
  G.hf = E.ib.ihf;
  G.cell_level = E.mv_cells;
  const HostGrid& H = *E.H[0];
  for (int a = 0; a < 3; ++a) G.n[a] = int32_t(H.n[a]);
  G.L = H.L;
  return G;
}

// finest level's brick map and the coarse cell levels (point lookups)
ib_status finest_map(Engine& E) {
  if (E.mv_bmap) return IB_OK;
  const HostGrid& H = *E.H[0];
  const HostLevel& HL = H.levels[H.L];
  for (int a = 0; a < 3; ++a) {
    E.mv_nb[a] = int32_t(HL.nb[a]);
    E.mv_nf[a] = H.n[a] << H.L;
  }
  TRY(upload(E, &E.mv_bmap, HL.brick_map));
  std::vector<uint8_t> cells(H.active.size());
  for (size_t c = 0; c < cells.size(); ++c) cells[c] = H.active[c] ? uint8_t(H.level[c]) : uint8_t(255);
  TRY(upload(E, &E.mv_cells, cells));
  if (!E.mv_err) TRY(dalloc(E, &E.mv_err, 4, true));
  return IB_OK;
}

ib_status move_alloc(Engine& E) {
  if (E.mv_ready) return IB_OK;
  TRY(finest_map(E));
  const HostGrid& H = *E.H[0];
  const MoveGrid G = move_grid(E);
  const int64_t nb = mv_nbins(G), Mt = E.Mtot, ns = E.ns, M = H.M;
  TRY(dalloc(E, &E.mv_bins, 3 * (nb + 1) + M + 1, true));
  TRY(dalloc(E, &E.mv_rcnt, Mt + 1, true));
  const int64_t sc = std::max(scan_scratch_len(nb), std::max(scan_scratch_len(Mt), scan_scratch_len(ns)));
  TRY(dalloc(E, &E.mv_scratch, sc, true));
  TRY(dalloc(E, &E.mv_scnt, ns + 1, true));
  TRY(dalloc(E, &E.mv_sstart, ns + 1, true));
  TRY(dalloc(E, &E.mv_sfill, ns + 1, true));
  TRY(dalloc(E, &E.mv_sflag, ns + 1, true));
  TRY(dalloc(E, &E.mv_sidx, ns + 1, true));
  TRY(dalloc(E, &E.mv_xprev, 3 * M + 1, true));
  TRY(dalloc(E, &E.mv_ubprev, 3 * M + 1, true));
  // spreading lists at their largest (every support node of every point free)
  int32_t *sp_ent, *sp_slot, *sp_off;
  TRY(dalloc(E, &sp_ent, 64 * M + 1, true));
  TRY(dalloc(E, &sp_slot, std::min<int64_t>(64 * M, ns) + 1, true));
  TRY(dalloc(E, &sp_off, std::min<int64_t>(64 * M, ns) + 2, true));
  E.ib.sp_ent = sp_ent;
  E.ib.sp_slot = sp_slot;
  E.ib.sp_off = sp_off;
  E.ib.sp_cap = std::min<int64_t>(64 * M, ns);
  E.ib.n_sp_dev = E.mv_sidx + ns;   // the compaction's total
  E.mv_ready = true;
  E.mv_graph_stale = true;          // the step graphs hold the host-built lists
  return IB_OK;
}

// Rebuild every structure of the IB step from the positions in E.X.
ib_status move_rebuild(Engine& E) {
  const HostGrid& H = *E.H[0];
  const int64_t M = H.M, Mt = E.Mtot, ns = E.ns;
  cudaStream_t st = E.st;
  IBDev& ib = E.ib;
  const MoveGrid G = move_grid(E);
  int32_t* org = const_cast<int32_t*>(ib.org);
  int32_t* slot = const_cast<int32_t*>(ib.slot);
  uint64_t* fb = const_cast<uint64_t*>(ib.freeb);
  int32_t* rowptr = const_cast<int32_t*>(ib.rowptr);
  CK(cudaMemsetAsync(E.mv_err, 0, sizeof(int32_t), st));
  mv_supports(G, M, E.X, org, slot, fb, E.mv_err, st);
  mv_af_count(G, M, Mt, org, E.mv_bins, E.mv_rcnt, rowptr, E.mv_scratch, st);
  int32_t hv[2] = {0, 0};
  CK(cudaMemcpyAsync(hv, E.mv_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hv + 1, rowptr + Mt, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (hv[0] != MV_OK) {
    E.err = hv[0] == MV_OUTSIDE ? "a Lagrangian point outside the box"
          : hv[0] == MV_NOFREE  ? "a Lagrangian point has no free support node"
                                : "an IB support touches a hanging node or a coarser level (the points left "
                                  "the finest refined band)";
    return IB_EINVAL;
  }
  if (hv[1] > E.af_cap) {   // more overlapping pairs than ever before: grow A_F
    const int64_t cap = int64_t(hv[1]) + int64_t(hv[1]) / 2;
    int32_t* col;
    double* val;
    TRY(dalloc(E, &col, cap, true));
    TRY(dalloc(E, &val, cap, true));
    ib.col = col;
    ib.val = val;
    if (E.mixed) {
      float* v32;
      TRY(dalloc(E, &v32, cap, true));
      ib.val32 = v32;
    }
    E.af_cap = cap;
    E.mv_graph_stale = true;
  }
  mv_af_fill(G, M, org, E.mv_bins, rowptr, const_cast<int32_t*>(ib.col), st);
  ib_weights(ib, st);
  ib_assemble(ib, st);
  mv_spread(M, ns, slot, fb, E.mv_scnt, E.mv_sstart, E.mv_sfill, E.mv_sflag, E.mv_sidx,
            const_cast<int32_t*>(ib.sp_ent), const_cast<int32_t*>(ib.sp_slot), const_cast<int32_t*>(ib.sp_off),
            E.mv_scratch, st);
  return IB_OK;   // the spreading length stays on the device (ib.n_sp_dev)
}

}  // namespace

ib_status ib_set_points(ib_grid* g, int64_t M, const double* X, const double* UB, int32_t on_device) {
  if (!g || !X) return IB_EINVAL;
  if (!g->ready) { g->err = "ib_set_boundary has not succeeded"; return IB_ESTATE; }
  if (!g->eng) { g->err = "a deferred handle keeps its geometry"; return IB_ESTATE; }
  if (M != g->H.M) { g->err = "ib_set_points keeps the number of points"; return IB_EINVAL; }
  Engine& E = *g->eng;
  cudaStream_t st = E.st;
  const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  ib_status s = move_alloc(E);
  if (s != IB_OK) { g->err = E.err; return s; }
  auto fail = [&](ib_status code) { g->err = E.err; return code; };
#define CKG(x)                                                                                    \
  do {                                                                                            \
    cudaError_t e_ = (x);                                                                         \
    if (e_ != cudaSuccess) { E.err = std::string("CUDA: ") + cudaGetErrorString(e_); return fail(IB_ECUDA); } \
  } while (0)
  if (M) {
    CKG(cudaMemcpyAsync(E.mv_xprev, E.X, 3 * M * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CKG(cudaMemcpyAsync(E.mv_ubprev, E.UB, 3 * M * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CKG(cudaMemcpyAsync(E.X, X, 3 * M * sizeof(double), kin, st));
    if (UB) CKG(cudaMemcpyAsync(E.UB, UB, 3 * M * sizeof(double), kin, st));
    else CKG(cudaMemsetAsync(E.UB, 0, 3 * M * sizeof(double), st));
  }
  s = move_rebuild(E);
  if (s == IB_EINVAL) {   // keep the previous points
    const std::string why = E.err;
    CKG(cudaMemcpyAsync(E.X, E.mv_xprev, 3 * M * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CKG(cudaMemcpyAsync(E.UB, E.mv_ubprev, 3 * M * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (move_rebuild(E) != IB_OK) return fail(IB_ECUDA);
    E.err = why;
  }
  if (s != IB_OK) return fail(s);
  // the captured step graphs read the list lengths from the device; only a
  // reallocated buffer (first move, a larger A_F) needs a new capture
  if (E.mv_graph_stale) {
    for (int k = 0; k < 2; ++k)
      if (E.gexec[k]) { cudaGraphExecDestroy(E.gexec[k]); E.gexec[k] = nullptr; }
    E.mv_graph_stale = false;
  }
  // host copies of the inputs and supports (exported by ib_fields_get)
  HostGrid& H = g->H;
  if (M) {
    CKG(cudaMemcpyAsync(H.X.data(), E.X, 3 * M * sizeof(double), cudaMemcpyDeviceToHost, st));
    CKG(cudaMemcpyAsync(H.UB.data(), E.UB, 3 * M * sizeof(double), cudaMemcpyDeviceToHost, st));
    CKG(cudaMemcpyAsync(H.ib_origin.data(), E.ib.org, 3 * M * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CKG(cudaMemcpyAsync(H.ib_slot.data(), E.ib.slot, 64 * M * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CKG(cudaMemcpyAsync(H.ib_free.data(), E.ib.freeb, M * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  }
  CKG(cudaStreamSynchronize(st));
#undef CKG
  return IB_OK;
}

ib_status ib_wss(ib_grid* g, const double* normals, double* wss, double* grad, int32_t on_device) {
  if (!g || !normals || !wss) return IB_EINVAL;
  if (!g->ready) { g->err = "ib_set_boundary has not succeeded"; return IB_ESTATE; }
  if (!g->eng) { g->err = "the wall shear stress of a deferred handle is read through its batch"; return IB_ESTATE; }
  Engine& E = *g->eng;
  const HostGrid& H = g->H;
  const int64_t M = H.M;
  if (M == 0) return IB_OK;
  cudaStream_t st = E.st;
  ib_status s = finest_map(E);
  if (s == IB_OK && !E.wss_n) {
    s = dalloc(E, &E.wss_n, 3 * M);
    if (s == IB_OK) s = dalloc(E, &E.wss_w, M);
    if (s == IB_OK) s = dalloc(E, &E.wss_g, 9 * M);
  }
  if (s != IB_OK) { g->err = E.err; return s; }
  double *dn = E.wss_n, *dw = E.wss_w, *dg = grad ? E.wss_g : nullptr;
  const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  int32_t herr = 0;
  cudaError_t e = cudaMemcpyAsync(dn, normals, 3 * M * sizeof(double), kin, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(E.mv_err, 0, sizeof(int32_t), st);
  if (e == cudaSuccess) {
    wss_compute(move_grid(E), H.hf, M, E.X, E.UB, dn, E.u, E.ns, E.D[0].nu * E.D[0].rho, dw, dg, E.mv_err, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(wss, dw, M * sizeof(double), kout, st);
  if (e == cudaSuccess && grad) e = cudaMemcpyAsync(grad, dg, 9 * M * sizeof(double), kout, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, E.mv_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { g->err = std::string("CUDA: ") + cudaGetErrorString(e); return IB_ECUDA; }
  if (herr) { g->err = "a wall point has too few fluid nodes around it for the DC-PSE moments"; return IB_EINVAL; }
  return IB_OK;
}

// ---------------------------------------------------------------- batches
ib_status ib_batch_create(ib_grid* const* members, int32_t n, ib_batch** out) {
  if (!members || n <= 0 || !out) return IB_EINVAL;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    ib_grid* m = members[i];
    if (!m || !m->ready || !m->d.deferred || m->batch) return IB_EINVAL;
    if (m->d.precision != members[0]->d.precision) return IB_EINVAL;
    if (m->d.viscous_form != members[0]->d.viscous_form) return IB_EINVAL;
    for (int j = 0; j < i; ++j)
      if (members[j] == m) return IB_EINVAL;
  }
  ib_batch* b = new (std::nothrow) ib_batch();
  if (!b) return IB_ENOMEM;
  Engine& E = b->E;
  for (int i = 0; i < n; ++i) {
    b->members.push_back(members[i]);
    E.H.push_back(&members[i]->H);
    E.MG.push_back(&members[i]->mg);
    E.D.push_back(members[i]->d);
  }
  E.ninst = n;
  E.st = static_cast<cudaStream_t>(members[0]->d.stream);
  E.alloc = members[0]->d.dev_alloc;
  E.freef = members[0]->d.dev_free;
  E.actx = members[0]->d.alloc_ctx;
  ib_status s = engine_build(E);
  for (int i = 0; i < n && s == IB_OK; ++i) s = snap_transfer(E, i, members[i], true);
  if (s != IB_OK) {
    members[0]->err = E.err;
    engine_free(E);
    delete b;
    return s;
  }
  E.prof.on = members[0]->d.profile != 0;
  E.use_graph = !E.prof.on;
  for (int i = 0; i < n; ++i) {
    members[i]->batch = b;
    members[i]->batch_index = i;
  }
  *out = b;
  return IB_OK;
}

ib_status ib_batch_step(ib_batch* b, int32_t nsteps, int32_t* status) {
  if (!b || nsteps < 0) return IB_EINVAL;
  ib_status worst = IB_OK;
  for (int32_t k = 0; k < nsteps; ++k) {
    ib_status s = engine_step(b->E);
    if (s == IB_ECUDA) return s;
    if (s != IB_OK) worst = s;
  }
  if (status)
    for (int i = 0; i < b->E.ninst; ++i) status[i] = b->E.status[i];
  return worst;
}

ib_status ib_batch_fields_get(ib_batch* b, int32_t member, int32_t field, void* dst, size_t bytes,
                              int32_t dst_on_device) {
  if (!b || member < 0 || member >= b->E.ninst) return IB_EINVAL;
  const int64_t need = field_bytes(*b->E.H[member], field);
  if (need < 0 || int64_t(bytes) != need || (!dst && bytes)) return IB_EINVAL;
  return engine_fields_get(b->E, member, field, dst, bytes, dst_on_device);
}

ib_status ib_batch_info(const ib_batch* b, int32_t member, ib_info* out) {
  if (!b || !out || member < 0 || member >= b->E.ninst) return IB_EINVAL;
  const Engine& E = b->E;
  ib_info I = E.last[member];
  fill_info(*E.H[member], E.MG[member], &E, E.bytes, I);
  I.step = E.step[member];
  I.time = E.time[member];
  *out = I;
  return IB_OK;
}

const char* ib_batch_last_error(const ib_batch* b) { return b ? b->E.err.c_str() : "null batch"; }

void ib_batch_destroy(ib_batch* b) {
  if (!b) return;
  for (size_t i = 0; i < b->members.size(); ++i) {
    snap_transfer(b->E, int(i), b->members[i], false);
    b->members[i]->batch = nullptr;
    b->members[i]->batch_index = -1;
  }
  engine_free(b->E);
  delete b;
}

ib_status ib_fields_get_noalloc(ib_grid* g, int32_t field, void* dst, size_t bytes, int32_t dst_on_device) {
  if (!g) return IB_EINVAL;
  if (!g->ready) { g->err = "ib_set_boundary has not succeeded"; return IB_ESTATE; }
  if (field != IB_FIELD_U && field != IB_FIELD_P && field != IB_FIELD_PHI) {
    g->err = "only U, P and PHI are read without allocation";
    return IB_EINVAL;
  }
  if (int64_t(bytes) != field_bytes(g->H, field)) { g->err = "bad byte count"; return IB_EINVAL; }
  if (!dst && bytes) return IB_EINVAL;
  if (g->eng || g->batch) {
    g->err = "only a deferred handle that no batch holds is read without allocation; use ib_fields_get";
    return IB_ESTATE;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != g->device) {
    // the scratch is per device and the snapshot lives on the handle's device
    g->err = "the handle was created on CUDA device " + std::to_string(g->device) + " but device " +
             std::to_string(dev) + " is current: make the handle's device current first";
    return IB_EINVAL;
  }
  const int nc = field == IB_FIELD_U ? 3 : 1;
  const double* src = field == IB_FIELD_U ? g->snap.u : field == IB_FIELD_P ? g->snap.p : g->snap.phi;
  return noalloc_gather_canon(int64_t(g->H.canon_slot.size()), g->snap.canon, nc, g->H.nbricks * BV, src, dst,
                              bytes, dst_on_device, static_cast<cudaStream_t>(g->d.stream), g->err);
}

}  // extern "C"
