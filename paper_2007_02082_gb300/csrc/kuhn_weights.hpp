// Integer weights of the P1 Kuhn-tetrahedron operators at a node, from the
// node's incident-cell mask (bit dz*4 + dy*2 + dx set when the cell with lower
// corner node - 1 + (dx, dy, dz) is an active leaf of the node's level).
//
// A cell is cut into six Kuhn tetrahedra v0 = lower corner, v1 = v0 + e_a1,
// v2 = v1 + e_a2, v3 = upper corner (one per axis order), so
//   * an axis edge lies in two tetrahedra of a cell when it starts at the
//     cell's lower corner or ends at its upper corner, else in one;
//   * a face diagonal in the direction e_a + e_b (both signs equal) lies in two
//     tetrahedra of each of the two cells that hold it; the main diagonal in
//     all six tetrahedra of its cell;
//   * the cell's lower and upper corners belong to all six tetrahedra, the
//     other six corners to two each.
// With V the cell volume and h_a the spacing, the P1 stiffness couples axis
// neighbours only, K[n, n +- e_a] = -(V/6) / h_a^2 * (tetrahedra holding the
// edge), and the consistent mass is M[n, m] = (V/120) * (tetrahedra holding
// both n and m) * (2 if m = n else 1).
#pragma once

#if defined(__CUDACC__)
#define IBG_HD __host__ __device__ __forceinline__
#else
#define IBG_HD inline
#endif

namespace ibg {

IBG_HD int kbit(int mask, int c) { return (mask >> c) & 1; }

// Tetrahedra holding the axis edge from the node to node + s * e_a (s = +1 or -1).
IBG_HD int stiff_edge_count(int mask, int a, int s) {
  // cells on the +a side have bit a set; of the four, the two whose other two
  // offsets are both 1 (edge at their lower corner) or both 0 (edge ending at
  // their upper corner) hold the edge twice
  const int b1 = 1 << ((a + 1) % 3), b2 = 1 << ((a + 2) % 3), ba = 1 << a;
  const int side = s > 0 ? ba : 0;
  return 2 * kbit(mask, side) + kbit(mask, side | b1) + kbit(mask, side | b2) + 2 * kbit(mask, side | b1 | b2);
}

// Mass weight (units V/120) of stencil offset k of the 15-point Kuhn stencil, in
// the order: 0 self; 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z; 7 +x+y, 8 -x-y,
// 9 +y+z, 10 -y-z, 11 +x+z, 12 -x-z; 13 +x+y+z, 14 -x-y-z.
IBG_HD int mass_weight(int mask, int k) {
  switch (k) {
    case 0: {
      int t = 6 * (kbit(mask, 0) + kbit(mask, 7));
      for (int c = 1; c < 7; ++c) t += 2 * kbit(mask, c);
      return 2 * t;
    }
    case 1: return stiff_edge_count(mask, 0, +1);
    case 2: return stiff_edge_count(mask, 0, -1);
    case 3: return stiff_edge_count(mask, 1, +1);
    case 4: return stiff_edge_count(mask, 1, -1);
    case 5: return stiff_edge_count(mask, 2, +1);
    case 6: return stiff_edge_count(mask, 2, -1);
    case 7: return 2 * (kbit(mask, 3) + kbit(mask, 7));
    case 8: return 2 * (kbit(mask, 0) + kbit(mask, 4));
    case 9: return 2 * (kbit(mask, 6) + kbit(mask, 7));
    case 10: return 2 * (kbit(mask, 0) + kbit(mask, 1));
    case 11: return 2 * (kbit(mask, 5) + kbit(mask, 7));
    case 12: return 2 * (kbit(mask, 0) + kbit(mask, 2));
    case 13: return 6 * kbit(mask, 7);
    default: return 6 * kbit(mask, 0);
  }
}

// Stencil offset index (0..14, order as in mass_weight) of a neighbour offset
// (each coordinate in -1..1), -1 if it is not in the 15-point Kuhn stencil.
IBG_HD int stencil_index(int rx, int ry, int rz) {
  const int key = (rz + 1) * 9 + (ry + 1) * 3 + (rx + 1);
  switch (key) {
    case 13: return 0;
    case 14: return 1;
    case 12: return 2;
    case 16: return 3;
    case 10: return 4;
    case 22: return 5;
    case 4: return 6;
    case 17: return 7;
    case 9: return 8;
    case 25: return 9;
    case 1: return 10;
    case 23: return 11;
    case 3: return 12;
    case 26: return 13;
    case 0: return 14;
    default: return -1;
  }
}

// Gradient coupling of one incident cell: for the cell of mask bit c, the sum
// over its Kuhn tetrahedra that hold both the node and its stencil neighbour k
// of the (integer) gradient of the neighbour's P1 function along axis a, in
// units 1/h_a.  (phi_m, d_a phi_n summed over tetrahedra is this times |T|/4.)
// Barycentric gradients of tetrahedron (a1, a2, a3): v0: -e_a1, v1: e_a1 - e_a2,
// v2: e_a2 - e_a3, v3: e_a3.
IBG_HD int grad_cell_weight(int c, int k, int a) {
  const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
  const int qb = (1 - dx) | ((1 - dy) << 1) | ((1 - dz) << 2);   // the node's corner in the cell
  const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  int sum = 0;
  for (int p = 0; p < 6; ++p) {
    const int a1 = perm[p][0], a2 = perm[p][1], a3 = perm[p][2];
    const int vb[4] = {0, 1 << a1, (1 << a1) | (1 << a2), 7};
    bool has = false;
    for (int v = 0; v < 4; ++v) has = has || vb[v] == qb;
    if (!has) continue;
    for (int v = 0; v < 4; ++v) {
      const int rx = dx - 1 + (vb[v] & 1), ry = dy - 1 + ((vb[v] >> 1) & 1), rz = dz - 1 + ((vb[v] >> 2) & 1);
      if (stencil_index(rx, ry, rz) != k) continue;
      int gvec[3] = {0, 0, 0};
      if (v == 0) gvec[a1] = -1;
      else if (v == 1) { gvec[a1] = 1; gvec[a2] = -1; }
      else if (v == 2) { gvec[a2] = 1; gvec[a3] = -1; }
      else gvec[a3] = 1;
      sum += gvec[a];
    }
  }
  return sum;
}

}  // namespace ibg
