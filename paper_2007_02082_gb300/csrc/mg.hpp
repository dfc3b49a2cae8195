// Geometric multigrid hierarchy for the pressure-increment Poisson problem
// (Eq. 12): host construction (mg.cpp) and the device V-cycle (mg.cu).
//
// Levels.  The composite grid (all refinement levels, hanging nodes) is the
// finest level.  G0 is the uniform P1 mesh of Kuhn tetrahedra on every active
// coarse cell (spacing h0); since refinement is nested (Sec. 3.2) the G0 space
// is a subspace of the composite space.  G(k+1) is G(k) coarsened by two per
// axis: a G(k+1) cell exists where any of its eight children does.
//
// Operators.  Every G(k) operator is the Galerkin product of the composite
// operator.  Because P1 gradients are constant on a tetrahedron and the Kuhn
// stiffness couples only the three axis edges of each tetrahedron, the
// Galerkin operator of G(k) is a 7-point stencil in which each tetrahedron's
// edge term is weighted by the fraction of the tetrahedron's volume covered by
// the active domain.  The fractions are summed up the hierarchy, 8 child
// tetrahedra per parent tetrahedron.  Pressure-Dirichlet nodes (outlets) are
// left out of every level.  A G0 node, and a coarser node where the outlet
// lies on its lattice, is Dirichlet when the finer node at its position is
// (this departs from Galerkin only next to the outlet and gave the fewest CG
// iterations); where an outlet plane falls between the coarse lattice planes,
// a coarse node is Dirichlet when its interpolation reaches any finer
// Dirichlet node, so the coarse space lies inside the finer one and the
// operator is the exact Galerkin product on every row.
//
// Transfers.  Prolongation is P1 interpolation on the coarse Kuhn tetrahedron
// that holds the fine node (barycentric weights, multiples of 2^-L, exact in
// floating point); restriction is its transpose.  Both are stored as CSR
// gathers so that every sum has one fixed order.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "setup.hpp"

namespace ibg {

constexpr int MG_MAX_LEVELS = 12;
constexpr int64_t MG_MAX_COARSEST = 1024;   // nodes of the coarsest level (dense inverse)
constexpr int64_t MG_SMALL_NODES = 8192;    // levels at most this size run in one CTA per problem

struct MGLevelHost {
  int64_t n[3] = {0, 0, 0};         // cells per axis
  double h[3] = {0, 0, 0};          // spacing
  int64_t nn = 0;                   // nodes (Dirichlet nodes excluded)
  std::vector<int32_t> coord;       // [nn][3] lattice coordinates of each node
  std::vector<int32_t> dir_coord;   // [nd][3] lattice coordinates of the Dirichlet nodes
  std::vector<int32_t> nbr;         // [nn][6]: -x, +x, -y, +y, -z, +z neighbour node or -1
  std::vector<double> offd;         // [nn][6] off-diagonal coefficients
  std::vector<double> diag;         // [nn]
  // restriction into this level: for each node, (finer index, weight); the
  // finer index is a composite slot for G0, a G(k-1) node otherwise
  std::vector<int32_t> r_ptr, r_col;
  std::vector<double> r_w;
  // prolongation out of this level: for each finer node / composite slot,
  // (node of this level, weight)
  std::vector<int32_t> p_ptr, p_col;
  std::vector<double> p_w;
};

struct MGHost {
  bool ok = false;
  std::string why;                  // reason when !ok
  std::vector<MGLevelHost> lev;     // G0 .. G(K)
  int small_start = 0;              // first level with at most MG_SMALL_NODES nodes
  std::vector<double> cinv;         // dense inverse of the G(K) operator, [nn_K][nn_K]
  // Composite <-> G0 transfers without stored weights (the device computes
  // each weight from lattice positions; the CSR of lev[0] is the reference):
  //   lat0      G0 lattice, [(n2+1)][(n1+1)][(n0+1)]: G0 node, -1 Dirichlet, -2 absent
  //   pbase     per composite brick of level >= 1, the first of its partial
  //             restriction sums (one per G0 node of its footprint, T^3 with
  //             T = (6 + 2^l) / 2^l + 1 per axis), -1 for level-0 bricks
  //   r0slot    per G0 node, the level-0 owner slot at its position, or -1
  //   r0ptr/idx per G0 node, the partial sums that make up its restriction,
  //             in brick order
  std::vector<int32_t> lat0;
  int64_t lat_n[3] = {0, 0, 0};
  std::vector<int32_t> pbase;
  int64_t npart = 0;
  std::vector<int32_t> r0slot, r0ptr, r0idx;
};

// Footprint of a level-l brick in G0 nodes per axis (see MGHost::pbase).
inline int mg_targets_per_axis(int l) { return (6 + (1 << l)) / (1 << l) + 1; }

// Build the hierarchy of one composite grid; levels with at most small_nodes
// nodes run in one CTA per problem (small_start).  On failure (no outlet node at
// all, or a transfer weight that points at a missing node) ok = false and the
// Poisson solve of that problem keeps the Jacobi preconditioner.
void build_mg(const HostGrid& G, MGHost& mg, int64_t small_nodes = MG_SMALL_NODES);

}  // namespace ibg
