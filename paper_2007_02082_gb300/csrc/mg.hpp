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
};

// Build the hierarchy of one composite grid.  On failure (no outlet node at
// all, or a transfer weight that points at a missing node) ok = false and the
// Poisson solve of that problem keeps the Jacobi preconditioner.
void build_mg(const HostGrid& G, MGHost& mg);

}  // namespace ibg
