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

// Gradient coupling of a node and its stencil neighbour k along axis a: the sum,
// over the Kuhn tetrahedra of the active incident cells that hold both, of the
// neighbour's barycentric gradient (integer, units 1/h_a).  Barycentric
// gradients of tetrahedron (a1, a2, a3): v0: -e_a1, v1: e_a1 - e_a2,
// v2: e_a2 - e_a3, v3: e_a3.  Each coupling is a fixed integer combination of
// the mask bits (one term per incident cell); (phi_n, d_a phi_m) summed over
// tetrahedra is this times |T|/4.
IBG_HD int grad_weight(int mask, int k, int a) {
  auto b = [mask](int c) { return (mask >> c) & 1; };
  switch (k * 3 + a) {
    case 0: return 2 * b(0) - 2 * b(1) + b(2) - b(3) + b(4) - b(5) + 2 * b(6) - 2 * b(7);
    case 1: return 2 * b(0) + b(1) - 2 * b(2) - b(3) + b(4) + 2 * b(5) - b(6) - 2 * b(7);
    case 2: return 2 * b(0) + b(1) + b(2) + 2 * b(3) - 2 * b(4) - b(5) - b(6) - 2 * b(7);
    case 3: return 2 * b(1) + b(3) + b(5) + 2 * b(7);
    case 4: return -b(3) - b(7);
    case 5: return -b(5) - b(7);
    case 6: return -2 * b(0) - b(2) - b(4) - 2 * b(6);
    case 7: return b(0) + b(4);
    case 8: return b(0) + b(2);
    case 9: return -b(3) - b(7);
    case 10: return 2 * b(2) + b(3) + b(6) + 2 * b(7);
    case 11: return -b(6) - b(7);
    case 12: return b(0) + b(4);
    case 13: return -2 * b(0) - b(1) - b(4) - 2 * b(5);
    case 14: return b(0) + b(1);
    case 15: return -b(5) - b(7);
    case 16: return -b(6) - b(7);
    case 17: return 2 * b(4) + b(5) + b(6) + 2 * b(7);
    case 18: return b(0) + b(2);
    case 19: return b(0) + b(1);
    case 20: return -2 * b(0) - b(1) - b(2) - 2 * b(3);
    case 21: return b(3) + b(7);
    case 22: return b(3) + b(7);
    case 23: return -2 * b(7);
    case 24: return -b(0) - b(4);
    case 25: return -b(0) - b(4);
    case 26: return 2 * b(0);
    case 27: return -2 * b(7);
    case 28: return b(6) + b(7);
    case 29: return b(6) + b(7);
    case 30: return 2 * b(0);
    case 31: return -b(0) - b(1);
    case 32: return -b(0) - b(1);
    case 33: return b(5) + b(7);
    case 34: return -2 * b(7);
    case 35: return b(5) + b(7);
    case 36: return -b(0) - b(2);
    case 37: return 2 * b(0);
    case 38: return -b(0) - b(2);
    case 39: return 2 * b(7);
    case 40: return 2 * b(7);
    case 41: return 2 * b(7);
    case 42: return -2 * b(0);
    case 43: return -2 * b(0);
    case 44: return -2 * b(0);
    default: return 0;
  }
}

// Transpose-gradient coupling of a node and its stencil neighbour k: the sum,
// over the Kuhn tetrahedra of the active incident cells that hold both, of
// (d_j phi_node)(d_i phi_neighbour), in units 1/(h_i h_j).  It is the block
// (test component i, trial component j) of (grad u^T, grad v) per |T|, the
// term the symmetric viscous form 2 (eps(u), eps(v)) adds to (grad u, grad v).
// Each tetrahedron belongs to one cell, so the sum is linear in the mask bits.
IBG_HD int trans_weight(int mask, int k, int i, int j) {
  auto b = [mask](int c) { return (mask >> c) & 1; };
  switch (k * 9 + i * 3 + j) {
    case 0: return 2 * b(0) + 2 * b(1) + b(2) + b(3) + b(4) + b(5) + 2 * b(6) + 2 * b(7);
    case 1: return -b(1) - b(2) - b(5) - b(6);
    case 2: return -b(1) - b(3) - b(4) - b(6);
    case 3: return -b(1) - b(2) - b(5) - b(6);
    case 4: return 2 * b(0) + b(1) + 2 * b(2) + b(3) + b(4) + 2 * b(5) + b(6) + 2 * b(7);
    case 5: return -b(2) - b(3) - b(4) - b(5);
    case 6: return -b(1) - b(3) - b(4) - b(6);
    case 7: return -b(2) - b(3) - b(4) - b(5);
    case 8: return 2 * b(0) + b(1) + b(2) + 2 * b(3) + 2 * b(4) + b(5) + b(6) + 2 * b(7);
    case 9: return -2 * b(1) - b(3) - b(5) - 2 * b(7);
    case 10: return b(1) + b(5);
    case 11: return b(1) + b(3);
    case 12: return b(3) + b(7);
    case 14: return -b(3);
    case 15: return b(5) + b(7);
    case 16: return -b(5);
    case 18: return -2 * b(0) - b(2) - b(4) - 2 * b(6);
    case 19: return b(2) + b(6);
    case 20: return b(4) + b(6);
    case 21: return b(0) + b(4);
    case 23: return -b(4);
    case 24: return b(0) + b(2);
    case 25: return -b(2);
    case 28: return b(3) + b(7);
    case 29: return -b(3);
    case 30: return b(2) + b(6);
    case 31: return -2 * b(2) - b(3) - b(6) - 2 * b(7);
    case 32: return b(2) + b(3);
    case 33: return -b(6);
    case 34: return b(6) + b(7);
    case 37: return b(0) + b(4);
    case 38: return -b(4);
    case 39: return b(1) + b(5);
    case 40: return -2 * b(0) - b(1) - b(4) - 2 * b(5);
    case 41: return b(4) + b(5);
    case 42: return -b(1);
    case 43: return b(0) + b(1);
    case 46: return -b(5);
    case 47: return b(5) + b(7);
    case 48: return -b(6);
    case 50: return b(6) + b(7);
    case 51: return b(4) + b(6);
    case 52: return b(4) + b(5);
    case 53: return -2 * b(4) - b(5) - b(6) - 2 * b(7);
    case 55: return -b(2);
    case 56: return b(0) + b(2);
    case 57: return -b(1);
    case 59: return b(0) + b(1);
    case 60: return b(1) + b(3);
    case 61: return b(2) + b(3);
    case 62: return -2 * b(0) - b(1) - b(2) - 2 * b(3);
    case 64: return -b(3) - b(7);
    case 65: return b(3);
    case 66: return -b(3) - b(7);
    case 68: return b(3);
    case 69: return b(7);
    case 70: return b(7);
    case 73: return -b(0) - b(4);
    case 74: return b(4);
    case 75: return -b(0) - b(4);
    case 77: return b(4);
    case 78: return b(0);
    case 79: return b(0);
    case 82: return b(7);
    case 83: return b(7);
    case 84: return b(6);
    case 86: return -b(6) - b(7);
    case 87: return b(6);
    case 88: return -b(6) - b(7);
    case 91: return b(0);
    case 92: return b(0);
    case 93: return b(1);
    case 95: return -b(0) - b(1);
    case 96: return b(1);
    case 97: return -b(0) - b(1);
    case 100: return b(5);
    case 101: return -b(5) - b(7);
    case 102: return b(7);
    case 104: return b(7);
    case 105: return -b(5) - b(7);
    case 106: return b(5);
    case 109: return b(2);
    case 110: return -b(0) - b(2);
    case 111: return b(0);
    case 113: return b(0);
    case 114: return -b(0) - b(2);
    case 115: return b(2);
    case 118: return -b(7);
    case 119: return -b(7);
    case 120: return -b(7);
    case 122: return -b(7);
    case 123: return -b(7);
    case 124: return -b(7);
    case 127: return -b(0);
    case 128: return -b(0);
    case 129: return -b(0);
    case 131: return -b(0);
    case 132: return -b(0);
    case 133: return -b(0);
    default: return 0;
  }
}

}  // namespace ibg
