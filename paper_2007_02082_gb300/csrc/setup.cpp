// Host-side grid construction (per geometry, outside the time step).
//
// Level map and domain reduction: the level of a coarse cell follows its
// Chebyshev distance d (in coarse cells) to a cell that holds a Lagrangian
// point: max_level when d <= refine_band, one level less per further band,
// then 2:1 balanced over the 26-neighbourhood (local refinement near the
// immersed boundary, Sec. 3.2).  A coarse cell is active when it is inside the
// vessel or d <= reduce_band (domain reduction, Sec. 4.3).
//
// Compiled with -ffp-contract=off: port membership (dx^2 + dy^2 <= R^2) and
// point cells (floor((X - x0) / h)) are decided in plain FP64 with no fused
// multiply-add, so that the index sets are reproducible bit for bit.
#include "setup.hpp"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <numeric>
#include <unordered_map>

namespace ibg {
namespace {

inline int64_t cidx(const HostGrid& G, int64_t x, int64_t y, int64_t z) {
  return (z * G.n[1] + y) * G.n[0] + x;
}

// Chebyshev distance by breadth-first search over the 26-neighbourhood.
void chebyshev_bfs(HostGrid& G, const std::vector<uint8_t>& seed, int rmax) {
  const int64_t nc = G.n[0] * G.n[1] * G.n[2];
  G.dist.assign(nc, rmax + 1);
  std::deque<int64_t> q;
  for (int64_t c = 0; c < nc; ++c)
    if (seed[c]) { G.dist[c] = 0; q.push_back(c); }
  while (!q.empty()) {
    int64_t c = q.front(); q.pop_front();
    int d = G.dist[c];
    if (d >= rmax) continue;
    int64_t x = c % G.n[0], y = (c / G.n[0]) % G.n[1], z = c / (G.n[0] * G.n[1]);
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int64_t X = x + dx, Y = y + dy, Z = z + dz;
          if (X < 0 || Y < 0 || Z < 0 || X >= G.n[0] || Y >= G.n[1] || Z >= G.n[2]) continue;
          int64_t e = cidx(G, X, Y, Z);
          if (G.dist[e] > d + 1) { G.dist[e] = d + 1; q.push_back(e); }
        }
  }
}

inline bool is_leaf(const HostGrid& G, int lev, int64_t ci, int64_t cj, int64_t ck) {
  const int64_t m = int64_t(1) << lev;
  if (ci < 0 || cj < 0 || ck < 0 || ci >= G.n[0] * m || cj >= G.n[1] * m || ck >= G.n[2] * m) return false;
  int64_t c = cidx(G, ci >> lev, cj >> lev, ck >> lev);
  return G.active[c] && G.level[c] == lev;
}

inline int32_t slot_of(const HostGrid& G, int lev, int64_t i, int64_t j, int64_t k) {
  const HostLevel& H = G.levels[lev];
  if (i < 0 || j < 0 || k < 0 || i >= H.nn[0] || j >= H.nn[1] || k >= H.nn[2]) return -1;
  int64_t bi = i / BS, bj = j / BS, bk = k / BS;
  int32_t b = H.brick_map[(bk * H.nb[1] + bj) * H.nb[0] + bi];
  if (b < 0) return -1;
  int32_t s = b * BV + int32_t(((k % BS) * BS + (j % BS)) * BS + (i % BS));
  return (G.meta[s] & M_VALID) ? s : -1;
}

// Is the node at finest coordinates q on the boundary of the active region?
// Interior iff the coarse cell of each of its 8 octants is active.
bool on_boundary(const HostGrid& G, const int64_t q[3]) {
  const int64_t Lf = int64_t(1) << G.L;
  for (int s = 0; s < 8; ++s) {
    int64_t c[3];
    for (int a = 0; a < 3; ++a) {
      int64_t t = 2 * q[a] + (((s >> a) & 1) ? 1 : -1);
      c[a] = (t >= 0) ? t / (2 * Lf) : -1;   // floor for t >= -1
      if (c[a] < 0 || c[a] >= G.n[a]) return true;
    }
    if (!G.active[cidx(G, c[0], c[1], c[2])]) return true;
  }
  return false;
}

// Squared radial distance of a face node from the port axis, FP64, no FMA.
double port_r2(const HostGrid& G, const ib_port& p, const int64_t q[3]) {
  int o0 = (p.axis + 1) % 3, o1 = (p.axis + 2) % 3;
  if (o0 > o1) std::swap(o0, o1);
  double x0 = G.origin[o0] + double(q[o0]) * G.hf[o0];
  double x1 = G.origin[o1] + double(q[o1]) * G.hf[o1];
  double d0 = x0 - p.center[o0];
  double d1 = x1 - p.center[o1];
  double r2 = d0 * d0;
  r2 = r2 + d1 * d1;
  return r2;
}

}  // namespace

ib_status build_host_grid(const ib_grid_desc& d, int64_t M, const double* X, const double* dS,
                          const double* UB, const uint8_t* inside, HostGrid& G, std::string& err) {
  G = HostGrid();
  G.L = d.max_level;
  for (int a = 0; a < 3; ++a) {
    G.n[a] = d.n[a];
    G.origin[a] = d.origin[a];
    G.extent[a] = d.extent[a];
    G.h0[a] = d.extent[a] / double(d.n[a]);
    G.hf[a] = d.extent[a] / double(int64_t(d.n[a]) << G.L);
  }
  const int64_t nc = G.n[0] * G.n[1] * G.n[2];
  if (!inside && d.reduce_band >= 0) { err = "inside mask required when reduce_band >= 0"; return IB_EINVAL; }

  // ---- inputs
  G.M = M;
  G.X.assign(X, X + 3 * M);
  G.dS.assign(dS, dS + M);
  G.UB.assign(3 * M, 0.0);
  if (UB) G.UB.assign(UB, UB + 3 * M);
  std::vector<uint8_t> seed(nc, 0);
  for (int64_t i = 0; i < M; ++i) {
    for (int a = 0; a < 3; ++a) {
      double x = X[3 * i + a];
      if (!std::isfinite(x) || !std::isfinite(G.UB[3 * i + a])) { err = "non-finite point input"; return IB_EINVAL; }
    }
    if (!(dS[i] > 0.0) || !std::isfinite(dS[i])) { err = "area elements must be positive"; return IB_EINVAL; }
    int64_t c[3];
    for (int a = 0; a < 3; ++a) {
      double t = std::floor((X[3 * i + a] - G.origin[a]) / G.h0[a]);
      if (t < 0.0 || t >= double(G.n[a])) { err = "a Lagrangian point lies outside the box"; return IB_EINVAL; }
      c[a] = int64_t(t);
    }
    seed[cidx(G, c[0], c[1], c[2])] = 1;
  }

  // ---- distance, level map, active set
  const int B = std::max(1, int(d.refine_band));
  const int rb = d.reduce_band;
  const int rmax = std::max(std::max(B * G.L + 1, rb), 1);
  chebyshev_bfs(G, seed, rmax);
  G.level.assign(nc, 0);
  for (int64_t c = 0; c < nc; ++c) {
    int dd = G.dist[c];
    int k = dd <= B ? 0 : (dd - B + B - 1) / B;
    G.level[c] = uint8_t(std::max(0, G.L - k));
  }
  for (bool changed = true; changed;) {       // 2:1 balance
    changed = false;
    std::vector<uint8_t> nl = G.level;
    for (int64_t z = 0; z < G.n[2]; ++z)
      for (int64_t y = 0; y < G.n[1]; ++y)
        for (int64_t x = 0; x < G.n[0]; ++x) {
          int mx = 0;
          for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
              for (int dx = -1; dx <= 1; ++dx) {
                int64_t X2 = x + dx, Y2 = y + dy, Z2 = z + dz;
                if (X2 < 0 || Y2 < 0 || Z2 < 0 || X2 >= G.n[0] || Y2 >= G.n[1] || Z2 >= G.n[2]) continue;
                mx = std::max(mx, int(G.level[cidx(G, X2, Y2, Z2)]));
              }
          int64_t c = cidx(G, x, y, z);
          if (int(nl[c]) < mx - 1) { nl[c] = uint8_t(mx - 1); changed = true; }
        }
    G.level.swap(nl);
  }
  G.active.assign(nc, 1);
  if (rb >= 0)
    for (int64_t c = 0; c < nc; ++c) G.active[c] = (inside[c] != 0) || (G.dist[c] <= rb);
  G.n_active_coarse = 0;
  for (int64_t c = 0; c < nc; ++c)
    if (G.active[c]) {
      G.n_active_coarse++;
      G.leaf_per_level[G.level[c]] += int64_t(1) << (3 * G.level[c]);
    }

  // ---- bricks per level
  G.levels.resize(G.L + 1);
  int32_t nbr = 0;
  for (int l = 0; l <= G.L; ++l) {
    HostLevel& H = G.levels[l];
    H.lev = l;
    for (int a = 0; a < 3; ++a) {
      H.nn[a] = (G.n[a] << l) + 1;
      H.nb[a] = (H.nn[a] + BS - 1) / BS;
      H.h[a] = G.h0[a] / double(1 << l);
    }
    H.brick_map.assign(H.nb[0] * H.nb[1] * H.nb[2], -1);
    const int64_t m = int64_t(1) << l;
    for (int64_t z = 0; z < G.n[2]; ++z)
      for (int64_t y = 0; y < G.n[1]; ++y)
        for (int64_t x = 0; x < G.n[0]; ++x) {
          int64_t c = cidx(G, x, y, z);
          if (!G.active[c] || G.level[c] != l) continue;
          for (int64_t bk = (z * m) / BS; bk <= ((z + 1) * m) / BS; ++bk)
            for (int64_t bj = (y * m) / BS; bj <= ((y + 1) * m) / BS; ++bj)
              for (int64_t bi = (x * m) / BS; bi <= ((x + 1) * m) / BS; ++bi)
                H.brick_map[(bk * H.nb[1] + bj) * H.nb[0] + bi] = 1;
        }
    H.brick_begin = nbr;
    for (auto& v : H.brick_map)
      if (v >= 0) v = nbr++;
    H.brick_end = nbr;
  }
  G.nbricks = nbr;
  G.brick_level.assign(nbr, 0);
  G.brick_coord.assign(3 * int64_t(nbr), 0);
  G.brick_nbr.assign(27 * int64_t(nbr), -1);
  for (int l = 0; l <= G.L; ++l) {
    HostLevel& H = G.levels[l];
    for (int64_t bk = 0; bk < H.nb[2]; ++bk)
      for (int64_t bj = 0; bj < H.nb[1]; ++bj)
        for (int64_t bi = 0; bi < H.nb[0]; ++bi) {
          int32_t b = H.brick_map[(bk * H.nb[1] + bj) * H.nb[0] + bi];
          if (b < 0) continue;
          G.brick_level[b] = l;
          G.brick_coord[3 * b] = int32_t(bi);
          G.brick_coord[3 * b + 1] = int32_t(bj);
          G.brick_coord[3 * b + 2] = int32_t(bk);
          for (int oz = -1; oz <= 1; ++oz)
            for (int oy = -1; oy <= 1; ++oy)
              for (int ox = -1; ox <= 1; ++ox) {
                int64_t I = bi + ox, J = bj + oy, K = bk + oz;
                int32_t nbv = -1;
                if (I >= 0 && J >= 0 && K >= 0 && I < H.nb[0] && J < H.nb[1] && K < H.nb[2])
                  nbv = H.brick_map[(K * H.nb[1] + J) * H.nb[0] + I];
                G.brick_nbr[27 * int64_t(b) + (oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)] = nbv;
              }
        }
  }

  // ---- per-slot incident-cell masks
  const int64_t nslots = int64_t(nbr) * BV;
  G.meta.assign(nslots, 0);
  for (int32_t b = 0; b < nbr; ++b) {
    const int l = G.brick_level[b];
    for (int t = 0; t < BV; ++t) {
      int64_t i = int64_t(G.brick_coord[3 * b]) * BS + (t % BS);
      int64_t j = int64_t(G.brick_coord[3 * b + 1]) * BS + ((t / BS) % BS);
      int64_t k = int64_t(G.brick_coord[3 * b + 2]) * BS + (t / (BS * BS));
      uint16_t mask = 0;
      for (int c = 0; c < 8; ++c) {
        int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        if (is_leaf(G, l, i - 1 + dx, j - 1 + dy, k - 1 + dz)) mask |= uint16_t(1u << c);
      }
      if (mask) G.meta[int64_t(b) * BV + t] = uint16_t(mask | M_VALID);
    }
  }

  // ---- hanging nodes, interface copies, boundary/port flags
  std::vector<int32_t> entry_of_slot;   // interface entry of a fine (DUP) slot
  entry_of_slot.assign(nslots, -1);
  std::vector<int64_t> qf(3 * nslots, 0);
  std::vector<uint8_t> cflag(nslots, 0);
  for (int32_t b = 0; b < nbr; ++b) {
    const int l = G.brick_level[b];
    const int sh = G.L - l;
    for (int t = 0; t < BV; ++t) {
      const int64_t s = int64_t(b) * BV + t;
      if (!(G.meta[s] & M_VALID)) continue;
      int64_t ijk[3] = {int64_t(G.brick_coord[3 * b]) * BS + (t % BS),
                        int64_t(G.brick_coord[3 * b + 1]) * BS + ((t / BS) % BS),
                        int64_t(G.brick_coord[3 * b + 2]) * BS + (t / (BS * BS))};
      int64_t q[3];
      for (int a = 0; a < 3; ++a) { q[a] = ijk[a] << sh; qf[3 * s + a] = q[a]; }
      if (l >= 1) {
        int odd[3], nodd = 0;
        for (int a = 0; a < 3; ++a) { odd[a] = int(ijk[a] & 1); nodd += odd[a]; }
        if (nodd == 0) {
          int32_t sc = slot_of(G, l - 1, ijk[0] >> 1, ijk[1] >> 1, ijk[2] >> 1);
          if (sc >= 0) {
            G.meta[s] |= M_DUP;
            entry_of_slot[s] = int32_t(G.if_coarse.size());
            G.if_coarse.push_back(sc);
            G.if_fine.push_back(int32_t(s));
          }
        } else {
          bool hang = false;
          const int64_t m = int64_t(1) << l;
          for (int o = 0; o < 8 && !hang; ++o) {
            int64_t c[3];
            bool inb = true;
            for (int a = 0; a < 3; ++a) {
              int64_t tt = 2 * ijk[a] + (((o >> a) & 1) ? 1 : -1);
              c[a] = (tt >= 0) ? tt / (2 * m) : -1;
              if (c[a] < 0 || c[a] >= G.n[a]) inb = false;
            }
            if (!inb) continue;
            int64_t cc = cidx(G, c[0], c[1], c[2]);
            if (G.active[cc] && G.level[cc] < l) hang = true;
          }
          if (hang) {
            if (nodd == 3) { err = "internal: hanging node at a coarse cell centre"; return IB_EINVAL; }
            int64_t dlt[3] = {odd[0], odd[1], odd[2]};
            int32_t p1 = slot_of(G, l, ijk[0] - dlt[0], ijk[1] - dlt[1], ijk[2] - dlt[2]);
            int32_t p2 = slot_of(G, l, ijk[0] + dlt[0], ijk[1] + dlt[1], ijk[2] + dlt[2]);
            if (p1 < 0 || p2 < 0) { err = "internal: hanging node without parents"; return IB_EINVAL; }
            G.meta[s] |= M_HANG;
            G.hang_slot.push_back(int32_t(s));
            G.hang_p1.push_back(p1);
            G.hang_p2.push_back(p2);
          }
        }
      }
      bool bnd = on_boundary(G, q);
      if (bnd) cflag[s] |= C_BOUNDARY;
      if (G.meta[s] & M_HANG) { cflag[s] |= C_HANG; continue; }
      int inlet = -1, pinlet = -1, pport = -1;
      bool outlet = false;
      for (int p = 0; p < d.n_ports && bnd; ++p) {
        const ib_port& P = d.ports[p];
        int64_t plane = P.side == 0 ? 0 : (G.n[P.axis] << G.L);
        if (q[P.axis] != plane) continue;
        double r2 = port_r2(G, P, q);
        if (!(r2 <= P.radius * P.radius)) continue;
        if (P.kind == IB_INLET_VELOCITY) { inlet = p; break; }
        pport = p;
        if (P.kind == IB_INLET_PRESSURE) { pinlet = p; break; }
        outlet = true;
        break;
      }
      if (outlet || pinlet >= 0) { G.meta[s] |= M_PDIR; cflag[s] |= C_PDIR; }
      if ((outlet || pinlet >= 0) && d.port_tangential == IB_TANGENTIAL_ZERO)
        G.meta[s] |= uint16_t((d.ports[pport].axis + 1) << 14);
      if ((bnd && !outlet && pinlet < 0) || inlet >= 0) { G.meta[s] |= M_VDIR; cflag[s] |= C_VDIR; }
      if (pinlet >= 0) {
        cflag[s] |= C_INLET;
        G.pinlet_slot.push_back(int32_t(s));
        G.pinlet_port.push_back(pinlet);
      }
      if (inlet >= 0) {
        const ib_port& P = d.ports[inlet];
        cflag[s] |= C_INLET;
        double r2 = port_r2(G, P, q);
        double shape = 1.0 - r2 / (P.radius * P.radius);
        G.inlet_slot.push_back(int32_t(s));
        G.inlet_port.push_back(inlet);
        G.inlet_shape.push_back(P.side == 0 ? shape : -shape);
      }
    }
  }
  // hanging parents must be interface copies; gather children per entry
  std::vector<std::vector<int32_t>> kids(G.if_coarse.size());
  for (size_t h = 0; h < G.hang_slot.size(); ++h) {
    int32_t e1 = entry_of_slot[G.hang_p1[h]], e2 = entry_of_slot[G.hang_p2[h]];
    if (e1 < 0 || e2 < 0) { err = "internal: hanging parent is not an interface node"; return IB_EINVAL; }
    kids[e1].push_back(G.hang_slot[h]);
    kids[e2].push_back(G.hang_slot[h]);
  }
  G.if_of_slot.assign(nslots, -1);
  for (size_t e = 0; e < G.if_coarse.size(); ++e) {
    G.if_of_slot[G.if_coarse[e]] = int32_t(e);
    G.if_of_slot[G.if_fine[e]] = int32_t(e);
    G.meta[G.if_coarse[e]] |= M_IFACE;
    G.meta[G.if_fine[e]] |= M_IFACE;
  }
  G.if_child_off.assign(kids.size() + 1, 0);
  for (size_t e = 0; e < kids.size(); ++e) {
    std::sort(kids[e].begin(), kids[e].end());
    G.if_child_off[e + 1] = G.if_child_off[e] + int32_t(kids[e].size());
    G.if_child.insert(G.if_child.end(), kids[e].begin(), kids[e].end());
  }

  // ---- canonical order: owner copies sorted by (z, y, x) finest coordinates
  {
    const int64_t nfx = (G.n[0] << G.L) + 1, nfy = (G.n[1] << G.L) + 1;
    std::vector<std::pair<int64_t, int32_t>> keys;
    for (int64_t s = 0; s < nslots; ++s) {
      if (!(G.meta[s] & M_VALID) || (G.meta[s] & M_DUP)) continue;
      keys.emplace_back((qf[3 * s + 2] * nfy + qf[3 * s + 1]) * nfx + qf[3 * s], int32_t(s));
    }
    std::sort(keys.begin(), keys.end());
    G.canon_slot.resize(keys.size());
    G.canon_q.resize(3 * keys.size());
    G.canon_flags.resize(keys.size());
    for (size_t i = 0; i < keys.size(); ++i) {
      int32_t s = keys[i].second;
      G.canon_slot[i] = s;
      for (int a = 0; a < 3; ++a) G.canon_q[3 * i + a] = int32_t(qf[3 * s + a]);
      G.canon_flags[i] = cflag[s];
      if (!(G.meta[s] & M_HANG)) G.n_dof++;
    }
  }
  bool any_pdir = false;
  for (int64_t s = 0; s < nslots && !any_pdir; ++s) any_pdir = (G.meta[s] & M_PDIR) != 0;
  if (!any_pdir) {
    err = "no outlet or pressure-inlet node: the pressure Poisson problem would be singular";
    return IB_EINVAL;
  }

  // ---- IB supports on the finest level (Eq. 17: 4x4x4 nodes per point)
  G.ib_origin.assign(3 * M, 0);
  G.ib_slot.assign(64 * M, -1);
  G.ib_free.assign(M, 0);
  const int64_t nf[3] = {G.n[0] << G.L, G.n[1] << G.L, G.n[2] << G.L};
  for (int64_t i = 0; i < M; ++i) {
    int64_t o[3];
    for (int a = 0; a < 3; ++a) {
      o[a] = int64_t(std::floor((X[3 * i + a] - G.origin[a]) / G.hf[a])) - 1;
      G.ib_origin[3 * i + a] = int32_t(o[a]);
    }
    bool anyfree = false;
    for (int a = 0; a < 64; ++a) {
      int64_t q[3] = {o[0] + (a & 3), o[1] + ((a >> 2) & 3), o[2] + (a >> 4)};
      if (q[0] < 0 || q[1] < 0 || q[2] < 0 || q[0] > nf[0] || q[1] > nf[1] || q[2] > nf[2]) continue;
      int32_t s = slot_of(G, G.L, q[0], q[1], q[2]);
      if (s < 0) continue;
      if (G.meta[s] & (M_HANG | M_DUP)) {
        err = "an IB support touches a hanging node or a coarser level (widen refine_band)";
        return IB_EINVAL;
      }
      G.ib_slot[64 * i + a] = s;
      if (!(G.meta[s] & (M_VDIR | M_TAX))) { G.ib_free[i] |= (uint64_t(1) << a); anyfree = true; }
    }
    if (!anyfree) { err = "a Lagrangian point has no free support node"; return IB_EINVAL; }
  }
  // A_F pattern: points whose supports overlap (|o_i - o_k|_inf <= 3)
  {
    std::unordered_map<int64_t, std::vector<int32_t>> bucket;
    auto bkey = [&](int64_t x, int64_t y, int64_t z) {
      return ((z + 4) * (nf[1] / 4 + 8) + (y + 4)) * (nf[0] / 4 + 8) + (x + 4);
    };
    auto fdiv = [](int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); };
    for (int64_t i = 0; i < M; ++i)
      bucket[bkey(fdiv(G.ib_origin[3 * i], 4), fdiv(G.ib_origin[3 * i + 1], 4), fdiv(G.ib_origin[3 * i + 2], 4))]
          .push_back(int32_t(i));
    G.af_rowptr.assign(M + 1, 0);
    std::vector<int32_t> cols;
    for (int64_t i = 0; i < M; ++i) {
      int64_t bx = fdiv(G.ib_origin[3 * i], 4), by = fdiv(G.ib_origin[3 * i + 1], 4), bz = fdiv(G.ib_origin[3 * i + 2], 4);
      std::vector<int32_t> row;
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            auto it = bucket.find(bkey(bx + dx, by + dy, bz + dz));
            if (it == bucket.end()) continue;
            for (int32_t k : it->second) {
              bool ok = true;
              for (int a = 0; a < 3; ++a)
                if (std::abs(G.ib_origin[3 * i + a] - G.ib_origin[3 * k + a]) > 3) ok = false;
              if (ok) row.push_back(k);
            }
          }
      std::sort(row.begin(), row.end());
      cols.insert(cols.end(), row.begin(), row.end());
      G.af_rowptr[i + 1] = int32_t(cols.size());
    }
    G.af_col.swap(cols);
  }
  // spreading: free support node -> list of (point, local index), sorted
  {
    std::vector<std::pair<int32_t, int32_t>> ent;   // (slot, i*64+a)
    for (int64_t i = 0; i < M; ++i)
      for (int a = 0; a < 64; ++a)
        if (G.ib_free[i] >> a & 1) ent.emplace_back(G.ib_slot[64 * i + a], int32_t(i * 64 + a));
    std::sort(ent.begin(), ent.end());
    G.sp_off.push_back(0);
    for (size_t e = 0; e < ent.size(); ++e) {
      if (e == 0 || ent[e].first != ent[e - 1].first) {
        if (e) G.sp_off.push_back(int32_t(e));
        G.sp_slot.push_back(ent[e].first);
      }
      G.sp_ent.push_back(ent[e].second);
    }
    if (!ent.empty()) G.sp_off.push_back(int32_t(ent.size()));
  }
  return IB_OK;
}

void build_natural_rows(const ib_grid_desc& d, const HostGrid& G, NaturalRows& out) {
  out = NaturalRows();
  out.row_off.push_back(0);
  const int L = G.L;
  for (int l = 0; l <= L; ++l) {
    const HostLevel& HL = G.levels[l];
    const double* h = HL.h;
    for (int32_t b = HL.brick_begin; b < HL.brick_end; ++b) {
      for (int t = 0; t < BV; ++t) {
        const int64_t s = int64_t(b) * BV + t;
        const uint16_t m = G.meta[s];
        if (!(m & M_VALID) || (m & M_VDIR)) continue;
        const int64_t q[3] = {int64_t(G.brick_coord[3 * b]) * BS + (t % BS),
                              int64_t(G.brick_coord[3 * b + 1]) * BS + ((t / BS) % BS),
                              int64_t(G.brick_coord[3 * b + 2]) * BS + t / (BS * BS)};
        std::map<std::pair<int32_t, int>, double> acc;   // (trial slot, 3 i + j) -> weight
        for (int p = 0; p < d.n_ports; ++p) {
          const ib_port& P = d.ports[p];
          if (P.kind == IB_INLET_VELOCITY) continue;
          const int ax = P.axis;
          const int64_t plane = P.side == 0 ? 0 : (G.n[ax] << l);   // in level-l lattice units
          if (q[ax] != plane) continue;
          const double nrm = P.side == 0 ? -1.0 : 1.0;
          const int u = (ax + 1) % 3, v = (ax + 2) % 3;
          const double area = 0.5 * h[u] * h[v];
          for (int c = 0; c < 8; ++c) {
            if (!((m >> c) & 1)) continue;   // incident cell c (bit order x, y, z) active
            const int64_t lo[3] = {q[0] + (c & 1) - 1, q[1] + ((c >> 1) & 1) - 1, q[2] + ((c >> 2) & 1) - 1};
            static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
            for (const auto& pm : perms) {
              int64_t vx[4][3];
              for (int a = 0; a < 3; ++a) vx[0][a] = lo[a];
              for (int k = 1; k < 4; ++k) {
                for (int a = 0; a < 3; ++a) vx[k][a] = vx[k - 1][a];
                vx[k][pm[k - 1]] += 1;
              }
              int self = -1, nplane = 0;
              for (int k = 0; k < 4; ++k) {
                if (vx[k][0] == q[0] && vx[k][1] == q[1] && vx[k][2] == q[2]) self = k;
                if (vx[k][ax] == plane) nplane++;
              }
              if (self < 0 || nplane != 3) continue;   // no face of this tetrahedron in the plane at the node
              // barycentric gradients in units 1/h: -e_p0, e_p0 - e_p1, e_p1 - e_p2, e_p2
              int gv[4][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
              gv[0][pm[0]] = -1;
              gv[1][pm[0]] = 1;
              gv[1][pm[1]] = -1;
              gv[2][pm[1]] = 1;
              gv[2][pm[2]] = -1;
              gv[3][pm[2]] = 1;
              for (int k = 0; k < 4; ++k) {
                const int32_t sb = slot_of(G, l, vx[k][0], vx[k][1], vx[k][2]);
                if (sb < 0) continue;
                for (int i = 0; i < 3; ++i) {
                  if (!gv[k][i]) continue;
                  acc[{sb, 3 * i + ax}] += nrm * (double(gv[k][i]) / h[i]) * area / 3.0;
                }
              }
            }
          }
        }
        if (acc.empty()) continue;
        out.row_slot.push_back(int32_t(s));
        for (const auto& kv : acc) {
          out.ent_slot.push_back(kv.first.first);
          out.ent_comp.push_back(int8_t(kv.first.second));
          out.ent_w.push_back(kv.second);
        }
        out.row_off.push_back(int32_t(out.ent_slot.size()));
      }
    }
  }
}

}  // namespace ibg
