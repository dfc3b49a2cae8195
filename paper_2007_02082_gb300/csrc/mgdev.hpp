// Device side of the multigrid preconditioner (mg.cu): level arrays of all
// problems of an engine, concatenated level by level, and the V-cycle.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "device.cuh"
#include "fe.hpp"
#include "graph.hpp"

namespace ibg {

constexpr int MG_LEVELS_MAX = 12;

template <typename T>
struct MGLevelDev {
  int64_t n = 0;                       // nodes of this level over all problems
  const int32_t* inst = nullptr;       // [n] problem of each node
  const int32_t* noff = nullptr;       // [ninst + 1] node range of each problem
  const int32_t* nbr = nullptr;        // [n][6] neighbours (-x,+x,-y,+y,-z,+z), -1 missing
  const T* offd = nullptr;             // [n][6]
  const T* diag = nullptr;             // [n]
  const T* dinv = nullptr;             // [n]
  // restriction into this level: rows over this level's nodes, columns are
  // composite slots (level 0) or nodes of the level below
  const int32_t* rptr = nullptr;
  const int32_t* rcol = nullptr;
  const T* rw = nullptr;
  // prolongation out of this level: rows over composite slots (level 0) or
  // over the nodes of the level below
  const int32_t* pptr = nullptr;
  const int32_t* pcol = nullptr;
  const T* pw = nullptr;
  T* b = nullptr;                      // right-hand side
  T* xa = nullptr;                     // iterate; the level's result ends here
  T* xb = nullptr;                     // second iterate buffer
  T* res = nullptr;                    // residual
  // level 0 only: the composite <-> G0 transfers computed from lattice
  // positions (no stored weights; MGHost::lat0 and following)
  const int32_t* bco = nullptr;        // [nbricks][3] brick coordinates in the brick's level lattice
  const int32_t* lat = nullptr;        // concatenated G0 lattices: local G0 node, -1 Dirichlet, -2 absent
  const int64_t* lat_off = nullptr;    // [ninst] offset of each problem's lattice
  const int32_t* lat_n = nullptr;      // [ninst][3] lattice nodes per axis
  const int32_t* pbase = nullptr;      // [nbricks] first partial restriction sum of a brick, -1 at level 0
  const int32_t* fbr = nullptr;        // [nfb] the bricks with pbase >= 0, in order
  int32_t nfb = 0;
  T* part = nullptr;                   // partial restriction sums
  const int64_t* fbase = nullptr;      // [nbricks] first footprint entry of a brick (prolongation)
  const int32_t* fnode = nullptr;      // [nfp] global G0 node of each footprint entry, -1 Dirichlet/none
  int64_t nfp = 0;
  T* fp = nullptr;                     // [nfp] the G0 values of the footprints
  const int32_t* r0slot = nullptr;     // [n] level-0 owner slot at the G0 node, -1
  const int32_t* r0ptr = nullptr;      // [n + 1] partial sums of each G0 node
  const int32_t* r0idx = nullptr;
};

template <typename T>
struct MGDev {
  int nlev = 0;                        // levels over all problems
  int ninst = 0;
  int nu = 2;                          // Jacobi sweeps before and after the coarse correction (composite, G0)
  int nu_coarse = 2;                   // the same on the levels below G0 (1 measured 2 more CG iterations per step)
  T omega = T(0.7);                    // Jacobi damping
  MGLevelDev<T> lev[MG_LEVELS_MAX];
  const MGLevelDev<T>* dlev = nullptr; // device copy of lev (read by the per-problem kernel)
  const uint8_t* on = nullptr;         // [ninst] 1: multigrid, 0: Jacobi preconditioner
  const int32_t* small = nullptr;      // [ninst] first level of the per-problem kernel
  const int32_t* coarsest = nullptr;   // [ninst] last level
  const int64_t* cinv_off = nullptr;   // [ninst] offset of the dense inverse of the coarsest level
  const T* cinv = nullptr;
  int max_big = 0;                     // max over problems of small (levels run grid-wide)
  // launch choice: the levels below the composite grid in one cooperative
  // launch of lv_ctas CTAs (all resident), barrier words bar[2] zeroed per step
  int lv_ctas = 0;
  unsigned* bar = nullptr;
  bool any = false;                    // some problem uses multigrid
};

// z = B r: one symmetric V-cycle per problem with multigrid, z = D^-1 r for
// the others.  r, z, zs, q are composite vectors (zs and q are scratch); dinv
// the composite Jacobi inverse.  Problems whose KState is done are skipped.
// With prof set, launches are timed by class: pcls + 0 the composite stencil
// applies, pcls + 1 the composite smoothing updates, pcls + 2 the rest.
// CTAs of the cooperative coarse-level kernel that fit on the device at once
// (at most two per SM), 0 if the query fails
template <typename T>
int mg_levels_ctas();

template <typename T>
void mg_vcycle(const DevGrid& g, const MGDev<T>& mg, const T* r, T* z, T* zs, T* q, const T* dinv, uint16_t dmask,
               const KState* ks, cudaStream_t st, Prof* prof = nullptr, int pcls = 0);

}  // namespace ibg
