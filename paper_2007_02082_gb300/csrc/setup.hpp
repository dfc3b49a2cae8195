// Host-side construction of the composite grid and the IB structures.
//
// Storage model.  Every refinement level l has its own Cartesian node lattice
// (n * 2^l + 1 nodes per axis), stored sparsely in bricks of 8x8x8 nodes.  Only
// bricks that hold a vertex of an active leaf cell of that level exist; all
// levels' bricks are concatenated, so a node is addressed by one "slot"
// (brick * 512 + local index).  A physical node on the interface between two
// levels is stored twice (once per level); the coarse copy owns it.  A hanging
// node (midpoint of a coarse edge or Kuhn face diagonal, Sec. 3.2 refinement)
// exists only on the fine level and is constrained to the mean of its parents.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "ib.h"

namespace ibg {

constexpr int BS = 8;        // brick edge, nodes
constexpr int BV = 512;      // nodes per brick

// Per-slot metadata (uint16): low byte = incident-cell mask (bit dz*4+dy*2+dx
// set when the level cell with lower corner node-1+(dx,dy,dz) is an active leaf
// of this level), high byte = flags.
enum : uint16_t {
  M_VALID = 1u << 8,   // a vertex of an active leaf cell of this level
  M_HANG = 1u << 9,    // hanging node (value = mean of its two parents)
  M_DUP = 1u << 10,    // non-owner copy of a node stored on two levels
  M_VDIR = 1u << 11,   // velocity Dirichlet (wall or inlet)
  M_PDIR = 1u << 12,   // pressure-increment Dirichlet (outlet port)
  M_IFACE = 1u << 13,  // either copy of a node stored on two levels
  // bits 14-15: 1 + the normal axis of an outlet or pressure-inlet port node
  // whose tangential velocity components are held at zero (0: none)
  M_TAX = 3u << 14,
};

// Canonical node flag bits (IB_FIELD_NODE_FLAGS).
enum : uint8_t { C_HANG = 1, C_VDIR = 2, C_PDIR = 4, C_INLET = 8, C_BOUNDARY = 16 };

struct HostLevel {
  int lev = 0;
  int64_t nn[3] = {0, 0, 0};   // nodes per axis
  int64_t nb[3] = {0, 0, 0};   // bricks per axis
  double h[3] = {0, 0, 0};     // cell spacing
  std::vector<int32_t> brick_map;   // dense brick index -> global brick (-1)
  int32_t brick_begin = 0, brick_end = 0;
};

struct HostGrid {
  // description
  int L = 0;
  int64_t n[3] = {0, 0, 0};
  double origin[3] = {0, 0, 0}, extent[3] = {0, 0, 0};
  double h0[3] = {0, 0, 0}, hf[3] = {0, 0, 0};
  // coarse maps [nz][ny][nx]
  std::vector<int32_t> dist;
  std::vector<uint8_t> level, active;
  int64_t n_active_coarse = 0;
  int64_t leaf_per_level[IB_MAX_LEVEL + 1] = {0, 0, 0, 0};
  // bricks
  std::vector<HostLevel> levels;
  int64_t nbricks = 0;
  std::vector<int32_t> brick_level;   // [nbricks]
  std::vector<int32_t> brick_coord;   // [nbricks][3] brick lattice coords
  std::vector<int32_t> brick_nbr;     // [nbricks][27] neighbour brick (same level) or -1
  std::vector<uint16_t> meta;         // [nbricks*512]
  // interface (node stored on two levels) and hanging constraints
  std::vector<int32_t> if_coarse, if_fine;       // [n_if]
  std::vector<int32_t> if_child_off, if_child;   // CSR of hanging children (fine slots)
  std::vector<int32_t> if_of_slot;               // [nslots] interface entry of a copy, -1 else
  std::vector<int32_t> hang_slot, hang_p1, hang_p2;
  // canonical order
  std::vector<int32_t> canon_slot;    // [N] owner slot
  std::vector<int32_t> canon_q;       // [N][3] finest coordinates
  std::vector<uint8_t> canon_flags;   // [N]
  int64_t n_dof = 0;
  // inlet Dirichlet entries (every stored copy)
  std::vector<int32_t> inlet_slot;
  std::vector<int32_t> inlet_port;
  std::vector<double> inlet_shape;    // (1 - r^2/R^2) * (+1 low face, -1 high face)
  // pressure-inlet Phi Dirichlet entries (every stored copy)
  std::vector<int32_t> pinlet_slot;
  std::vector<int32_t> pinlet_port;
  // IB
  int64_t M = 0;
  std::vector<double> X, dS, UB;      // copies of the inputs
  std::vector<int32_t> ib_origin;     // [M][3]
  std::vector<int32_t> ib_slot;       // [M][64] (-1 missing)
  std::vector<uint64_t> ib_free;      // [M] bit a: support node a exists and is free
  std::vector<int32_t> af_rowptr, af_col;   // pattern of A_F (sorted columns)
  std::vector<int32_t> sp_slot, sp_off, sp_ent;   // spreading CSR: node -> (i*64+a)
};

// Builds everything; returns IB_OK or IB_EINVAL with a message in err.
ib_status build_host_grid(const ib_grid_desc& d, int64_t M, const double* X, const double* dS,
                          const double* UB, const uint8_t* inside, HostGrid& G, std::string& err);

// Natural boundary term of the symmetric viscous form: ((grad u)^T n, phi_a)
// over the tetrahedron faces in the plane of an outlet or pressure-inlet port
// (n the outward normal).  One row per stored slot without a velocity
// condition that is a vertex of such a face, at that slot's level; entry e
// adds w_e * u_{comp_e % 3}(slot_e) to component comp_e / 3 of the row's term
// (test component, trial component).  The step subtracts nu times the term.
struct NaturalRows {
  std::vector<int32_t> row_slot;   // [rows]
  std::vector<int32_t> row_off;    // [rows + 1]
  std::vector<int32_t> ent_slot;   // trial slot
  std::vector<int8_t> ent_comp;    // 3 * test component + trial component
  std::vector<double> ent_w;
};
void build_natural_rows(const ib_grid_desc& d, const HostGrid& G, NaturalRows& out);

}  // namespace ibg
