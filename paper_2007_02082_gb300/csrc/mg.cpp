// Host construction of the geometric multigrid hierarchy (see mg.hpp).
#include "mg.hpp"

#include <algorithm>
#include <cmath>

namespace ibg {

namespace {

// Kuhn tetrahedron p of a cell: v0 = lower corner, v1 = v0 + e[a1],
// v2 = v1 + e[a2], v3 = upper corner.
const int kKuhn[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

int kuhn_index(int a1, int a2) {
  for (int p = 0; p < 6; ++p)
    if (kKuhn[p][0] == a1 && kKuhn[p][1] == a2) return p;
  return -1;
}

// Parent tetrahedron of child tetrahedron t of the child cell at offset o
// (bit a of o = offset along axis a): the parent tetrahedron holding the child's
// centroid, whose coordinates (in parent-cell units) are ordered a1 > a2 > a3.
int parent_tet(int o, int t) {
  double c[3];
  for (int a = 0; a < 3; ++a) c[a] = double((o >> a) & 1);
  // centroid of the child tetrahedron in child units: o + (3 e_a1 + 2 e_a2 + e_a3) / 4
  c[kKuhn[t][0]] += 0.75;
  c[kKuhn[t][1]] += 0.5;
  c[kKuhn[t][2]] += 0.25;
  int ord[3] = {0, 1, 2};
  std::sort(ord, ord + 3, [&](int x, int y) { return c[x] > c[y]; });
  return kuhn_index(ord[0], ord[1]);
}

// Barycentric weights of the point with cell-local coordinates f in [0,1]^3
// on the Kuhn tetrahedron holding it: (vertex offset bits, weight) x 4.
int kuhn_weights(const double f[3], int vb[4], double w[4]) {
  int ord[3] = {0, 1, 2};
  std::stable_sort(ord, ord + 3, [&](int x, int y) { return f[x] > f[y]; });
  vb[0] = 0;
  vb[1] = 1 << ord[0];
  vb[2] = vb[1] | (1 << ord[1]);
  vb[3] = 7;
  w[0] = 1.0 - f[ord[0]];
  w[1] = f[ord[0]] - f[ord[1]];
  w[2] = f[ord[1]] - f[ord[2]];
  w[3] = f[ord[2]];
  return 4;
}

constexpr int32_t LAT_ABSENT = -2, LAT_DIRICHLET = -1;

struct Lattice {
  int64_t n[3] = {0, 0, 0};   // cells per axis
  std::vector<float> frac;    // [ncells][6] covered volume fraction per tetrahedron
  std::vector<int32_t> lat;   // [(n+1)^3]: node index, LAT_DIRICHLET or LAT_ABSENT
  std::vector<uint8_t> dir;   // [(n+1)^3]: Dirichlet marker before node numbering
  int64_t nn_lat(int a) const { return n[a] + 1; }
  int64_t cell(int64_t i, int64_t j, int64_t k) const { return (k * n[1] + j) * n[0] + i; }
  int64_t node(int64_t i, int64_t j, int64_t k) const { return (k * (n[1] + 1) + j) * (n[0] + 1) + i; }
};

int32_t composite_slot(const HostGrid& G, int lev, const int64_t c[3]) {
  const HostLevel& H = G.levels[lev];
  for (int a = 0; a < 3; ++a)
    if (c[a] < 0 || c[a] >= H.nn[a]) return -1;
  const int32_t b = H.brick_map[((c[2] / BS) * H.nb[1] + c[1] / BS) * H.nb[0] + c[0] / BS];
  if (b < 0) return -1;
  const int32_t s = b * BV + int32_t(((c[2] % BS) * BS + (c[1] % BS)) * BS + (c[0] % BS));
  return (G.meta[s] & M_VALID) ? s : -1;
}

// Number the nodes touched by a tetrahedron of nonzero fraction (Dirichlet
// nodes excluded) and assemble the fraction-weighted 7-point operator.
void assemble(Lattice& Lt, MGLevelHost& M) {
  const int64_t nl = Lt.nn_lat(0) * Lt.nn_lat(1) * Lt.nn_lat(2);
  Lt.lat.assign(nl, LAT_ABSENT);
  for (int64_t k = 0; k < Lt.n[2]; ++k)
    for (int64_t j = 0; j < Lt.n[1]; ++j)
      for (int64_t i = 0; i < Lt.n[0]; ++i) {
        const float* fr = &Lt.frac[6 * Lt.cell(i, j, k)];
        for (int t = 0; t < 6; ++t) {
          if (fr[t] <= 0.f) continue;
          int vb[4] = {0, 1 << kKuhn[t][0], (1 << kKuhn[t][0]) | (1 << kKuhn[t][1]), 7};
          for (int v = 0; v < 4; ++v) {
            const int64_t id = Lt.node(i + (vb[v] & 1), j + ((vb[v] >> 1) & 1), k + ((vb[v] >> 2) & 1));
            Lt.lat[id] = Lt.dir[id] ? LAT_DIRICHLET : 0;
          }
        }
      }
  int64_t nn = 0;
  M.coord.clear();
  M.dir_coord.clear();
  for (int64_t id = 0; id < nl; ++id) {
    if (Lt.lat[id] == LAT_DIRICHLET) {
      const int64_t nx = Lt.nn_lat(0), ny = Lt.nn_lat(1);
      M.dir_coord.push_back(int32_t(id % nx));
      M.dir_coord.push_back(int32_t((id / nx) % ny));
      M.dir_coord.push_back(int32_t(id / (nx * ny)));
    }
    if (Lt.lat[id] == 0) {
      Lt.lat[id] = int32_t(nn++);
      const int64_t nx = Lt.nn_lat(0), ny = Lt.nn_lat(1);
      M.coord.push_back(int32_t(id % nx));
      M.coord.push_back(int32_t((id / nx) % ny));
      M.coord.push_back(int32_t(id / (nx * ny)));
    }
  }
  M.nn = nn;
  M.nbr.assign(6 * nn, -1);
  M.offd.assign(6 * nn, 0.0);
  M.diag.assign(nn, 0.0);
  const double V = M.h[0] * M.h[1] * M.h[2];
  for (int64_t k = 0; k < Lt.n[2]; ++k)
    for (int64_t j = 0; j < Lt.n[1]; ++j)
      for (int64_t i = 0; i < Lt.n[0]; ++i) {
        const float* fr = &Lt.frac[6 * Lt.cell(i, j, k)];
        for (int t = 0; t < 6; ++t) {
          if (fr[t] <= 0.f) continue;
          int64_t v[3] = {i, j, k};
          for (int e = 0; e < 3; ++e) {   // the three axis edges v_e -> v_{e+1}
            const int a = kKuhn[t][e];
            int64_t w[3] = {v[0], v[1], v[2]};
            w[a] += 1;
            const double kap = double(fr[t]) * (V / 6.0) / (M.h[a] * M.h[a]);
            const int32_t na = Lt.lat[Lt.node(v[0], v[1], v[2])], nb = Lt.lat[Lt.node(w[0], w[1], w[2])];
            if (na >= 0) {
              M.diag[na] += kap;
              if (nb >= 0) {
                M.nbr[6 * na + 2 * a + 1] = nb;
                M.offd[6 * na + 2 * a + 1] -= kap;
              }
            }
            if (nb >= 0) {
              M.diag[nb] += kap;
              if (na >= 0) {
                M.nbr[6 * nb + 2 * a] = na;
                M.offd[6 * nb + 2 * a] -= kap;
              }
            }
            v[a] += 1;
          }
        }
      }
}

// CSR transpose: rows of `ptr/col/w` (nrow) become rows over ncol.
void transpose(int64_t nrow, const std::vector<int32_t>& ptr, const std::vector<int32_t>& col,
               const std::vector<double>& w, int64_t ncol, std::vector<int32_t>& tptr, std::vector<int32_t>& tcol,
               std::vector<double>& tw) {
  tptr.assign(ncol + 1, 0);
  for (int32_t c : col) tptr[c + 1]++;
  for (int64_t c = 0; c < ncol; ++c) tptr[c + 1] += tptr[c];
  tcol.assign(col.size(), 0);
  tw.assign(col.size(), 0.0);
  std::vector<int32_t> fill(tptr.begin(), tptr.end() - 1);
  for (int64_t r = 0; r < nrow; ++r)   // rows in increasing order: every target row is sorted
    for (int32_t e = ptr[r]; e < ptr[r + 1]; ++e) {
      const int32_t at = fill[col[e]]++;
      tcol[at] = int32_t(r);
      tw[at] = w[e];
    }
}

// Interpolation weights of a point with lattice coordinates num/den (per axis)
// onto the nodes of Lt; appends nonzero entries.  False if a nonzero weight
// points at a node that does not exist.
bool interp_row(const Lattice& Lt, const int64_t num[3], int64_t den, std::vector<int32_t>& col,
                std::vector<double>& w) {
  int64_t c[3];
  double f[3];
  for (int a = 0; a < 3; ++a) {
    c[a] = std::min(num[a] / den, Lt.n[a] - 1);
    f[a] = double(num[a] - c[a] * den) / double(den);
  }
  int vb[4];
  double wt[4];
  kuhn_weights(f, vb, wt);
  for (int v = 0; v < 4; ++v) {
    if (wt[v] == 0.0) continue;
    const int32_t id = Lt.lat[Lt.node(c[0] + (vb[v] & 1), c[1] + ((vb[v] >> 1) & 1), c[2] + ((vb[v] >> 2) & 1))];
    if (id == LAT_DIRICHLET) continue;
    if (id < 0) return false;
    col.push_back(id);
    w.push_back(wt[v]);
  }
  return true;
}

// Mark as Dirichlet every lattice vertex of Lt that takes a nonzero
// interpolation weight at the point num/den (a Dirichlet node of the finer
// level): the coarse basis functions that remain then vanish on every finer
// Dirichlet node, so each coarse space is a subspace of the finer one.
void mark_dirichlet(Lattice& Lt, const int64_t num[3], int64_t den) {
  int64_t c[3];
  double f[3];
  for (int a = 0; a < 3; ++a) {
    c[a] = std::min(num[a] / den, Lt.n[a] - 1);
    f[a] = double(num[a] - c[a] * den) / double(den);
  }
  int vb[4];
  double wt[4];
  kuhn_weights(f, vb, wt);
  for (int v = 0; v < 4; ++v)
    if (wt[v] != 0.0) Lt.dir[Lt.node(c[0] + (vb[v] & 1), c[1] + ((vb[v] >> 1) & 1), c[2] + ((vb[v] >> 2) & 1))] = 1;
}

bool dense_inverse(const MGLevelHost& M, std::vector<double>& inv) {
  const int64_t n = M.nn;
  std::vector<double> A(n * n, 0.0);
  for (int64_t i = 0; i < n; ++i) {
    A[i * n + i] = M.diag[i];
    for (int d = 0; d < 6; ++d)
      if (M.nbr[6 * i + d] >= 0) A[i * n + M.nbr[6 * i + d]] += M.offd[6 * i + d];
  }
  // Cholesky A = L L^T (lower triangle in place)
  for (int64_t j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int64_t k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
    if (!(s > 0.0)) return false;
    const double d = std::sqrt(s);
    A[j * n + j] = d;
    for (int64_t i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int64_t k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = t / d;
    }
  }
  inv.assign(n * n, 0.0);
  std::vector<double> y(n);
  for (int64_t c = 0; c < n; ++c) {
    for (int64_t i = 0; i < n; ++i) {   // L y = e_c
      double t = (i == c) ? 1.0 : 0.0;
      for (int64_t k = 0; k < i; ++k) t -= A[i * n + k] * y[k];
      y[i] = t / A[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i) {   // L^T x = y
      double t = y[i];
      for (int64_t k = i + 1; k < n; ++k) t -= A[k * n + i] * inv[k * n + c];
      inv[i * n + c] = t / A[i * n + i];
    }
  }
  return true;
}

}  // namespace

void build_mg(const HostGrid& G, MGHost& mg, int64_t small_nodes) {
  mg = MGHost();
  const int L = G.L;
  const int64_t Lf = int64_t(1) << L;
  std::vector<Lattice> lats;

  // ---- G0: every active coarse cell, full coverage
  Lattice L0;
  for (int a = 0; a < 3; ++a) L0.n[a] = G.n[a];
  const int64_t nc0 = L0.n[0] * L0.n[1] * L0.n[2];
  L0.frac.assign(6 * nc0, 0.f);
  for (int64_t c = 0; c < nc0; ++c)
    if (G.active[c])
      for (int t = 0; t < 6; ++t) L0.frac[6 * c + t] = 1.f;
  const int64_t nl0 = (L0.n[0] + 1) * (L0.n[1] + 1) * (L0.n[2] + 1);
  L0.dir.assign(nl0, 0);
  for (int64_t k = 0; k <= L0.n[2]; ++k)
    for (int64_t j = 0; j <= L0.n[1]; ++j)
      for (int64_t i = 0; i <= L0.n[0]; ++i)
        for (int l = 0; l <= L; ++l) {   // any stored copy of the point carries the flags
          const int64_t c[3] = {i << l, j << l, k << l};
          const int32_t s = composite_slot(G, l, c);
          if (s >= 0) {
            L0.dir[L0.node(i, j, k)] = (G.meta[s] & M_PDIR) ? 1 : 0;
            break;
          }
        }
  mg.lev.emplace_back();
  for (int a = 0; a < 3; ++a) mg.lev[0].n[a] = L0.n[a], mg.lev[0].h[a] = G.h0[a];
  assemble(L0, mg.lev[0]);
  lats.push_back(std::move(L0));

  // ---- composite -> G0 transfers: prolongation rows over every composite slot
  {
    MGLevelHost& M = mg.lev[0];
    const int64_t ns = G.nbricks * BV;
    M.p_ptr.assign(ns + 1, 0);
    std::vector<int32_t> rptr(ns + 1, 0), rcol;   // restriction source rows (owner DOF slots only)
    std::vector<double> rw;
    for (int64_t s = 0; s < ns; ++s) {
      const uint16_t m = G.meta[s];
      const bool keep = (m & M_VALID) && !(m & (M_HANG | M_PDIR));
      if (keep) {
        const int32_t b = int32_t(s / BV);
        const int l = G.brick_level[b];
        const int t = int(s % BV);
        const int64_t q[3] = {(int64_t(G.brick_coord[3 * b]) * BS + (t % BS)) << (L - l),
                              (int64_t(G.brick_coord[3 * b + 1]) * BS + ((t / BS) % BS)) << (L - l),
                              (int64_t(G.brick_coord[3 * b + 2]) * BS + (t / (BS * BS))) << (L - l)};
        const size_t e0 = M.p_col.size();
        if (!interp_row(lats[0], q, Lf, M.p_col, M.p_w)) {
          mg.why = "composite node outside the G0 mesh";
          return;
        }
        if (!(m & M_DUP))
          for (size_t e = e0; e < M.p_col.size(); ++e) {
            rcol.push_back(M.p_col[e]);
            rw.push_back(M.p_w[e]);
          }
      }
      M.p_ptr[s + 1] = int32_t(M.p_col.size());
      rptr[s + 1] = int32_t(rcol.size());
    }
    transpose(ns, rptr, rcol, rw, M.nn, M.r_ptr, M.r_col, M.r_w);
  }

  // ---- the same transfers in the device's weight-free form
  {
    const Lattice& Lt = lats[0];
    const MGLevelHost& M = mg.lev[0];
    mg.lat0 = Lt.lat;
    for (int a = 0; a < 3; ++a) mg.lat_n[a] = Lt.n[a] + 1;
    mg.pbase.assign(G.nbricks, -1);
    mg.r0slot.assign(M.nn, -1);
    std::vector<int64_t> node_of, part_of;   // (G0 node, partial index) pairs in brick order
    int64_t np = 0;
    for (int32_t b = 0; b < int32_t(G.nbricks); ++b) {
      const int l = G.brick_level[b];
      const int64_t bc[3] = {G.brick_coord[3 * b], G.brick_coord[3 * b + 1], G.brick_coord[3 * b + 2]};
      if (l == 0) {
        for (int t = 0; t < BV; ++t) {
          const int64_t s = int64_t(b) * BV + t;
          const uint16_t m = G.meta[s];
          if (!(m & M_VALID) || (m & (M_HANG | M_PDIR | M_DUP))) continue;
          const int32_t id = Lt.lat[Lt.node(bc[0] * BS + t % BS, bc[1] * BS + (t / BS) % BS, bc[2] * BS + t / (BS * BS))];
          if (id >= 0) mg.r0slot[id] = int32_t(s);
        }
        continue;
      }
      const int sc = 1 << l, T = mg_targets_per_axis(l);
      mg.pbase[b] = int32_t(np);
      for (int tz = 0; tz < T; ++tz)
        for (int ty = 0; ty < T; ++ty)
          for (int tx = 0; tx < T; ++tx) {
            const int64_t q[3] = {bc[0] * BS / sc + tx, bc[1] * BS / sc + ty, bc[2] * BS / sc + tz};
            if (q[0] > Lt.n[0] || q[1] > Lt.n[1] || q[2] > Lt.n[2]) continue;
            const int32_t id = Lt.lat[Lt.node(q[0], q[1], q[2])];
            if (id < 0) continue;
            node_of.push_back(id);
            part_of.push_back(np + (tz * T + ty) * T + tx);
          }
      np += int64_t(T) * T * T;
    }
    mg.npart = np;
    if (np >= (int64_t(1) << 31)) { mg.why = "too many partial restriction sums"; return; }
    mg.r0ptr.assign(M.nn + 1, 0);
    for (int64_t id : node_of) mg.r0ptr[id + 1]++;
    for (int64_t j = 0; j < M.nn; ++j) mg.r0ptr[j + 1] += mg.r0ptr[j];
    mg.r0idx.assign(node_of.size(), 0);
    std::vector<int32_t> fill(mg.r0ptr.begin(), mg.r0ptr.end() - 1);
    for (size_t e = 0; e < node_of.size(); ++e) mg.r0idx[fill[node_of[e]]++] = int32_t(part_of[e]);
  }

  // ---- coarser levels
  int ptab[8][6];
  for (int o = 0; o < 8; ++o)
    for (int t = 0; t < 6; ++t) ptab[o][t] = parent_tet(o, t);
  for (;;) {
    const int k = int(mg.lev.size()) - 1;
    if (mg.lev[k].nn <= MG_MAX_COARSEST / 2) break;
    const Lattice& F = lats[k];
    if (F.n[0] < 2 && F.n[1] < 2 && F.n[2] < 2) break;
    if (int(mg.lev.size()) >= MG_MAX_LEVELS) break;
    Lattice C;
    for (int a = 0; a < 3; ++a) C.n[a] = (F.n[a] + 1) / 2;
    const int64_t ncc = C.n[0] * C.n[1] * C.n[2];
    C.frac.assign(6 * ncc, 0.f);
    for (int64_t kk = 0; kk < C.n[2]; ++kk)
      for (int64_t jj = 0; jj < C.n[1]; ++jj)
        for (int64_t ii = 0; ii < C.n[0]; ++ii) {
          double acc[6] = {0, 0, 0, 0, 0, 0};
          for (int o = 0; o < 8; ++o) {
            const int64_t ci = 2 * ii + (o & 1), cj = 2 * jj + ((o >> 1) & 1), ck = 2 * kk + ((o >> 2) & 1);
            if (ci >= F.n[0] || cj >= F.n[1] || ck >= F.n[2]) continue;
            const float* fr = &F.frac[6 * F.cell(ci, cj, ck)];
            for (int t = 0; t < 6; ++t) acc[ptab[o][t]] += fr[t];
          }
          for (int t = 0; t < 6; ++t) C.frac[6 * C.cell(ii, jj, kk) + t] = float(acc[t] / 8.0);
        }
    const int64_t nlc = (C.n[0] + 1) * (C.n[1] + 1) * (C.n[2] + 1);
    // coarse Dirichlet nodes: by injection (the finer node at the same position
    // is Dirichlet) when the outlet lies on the coarse lattice; otherwise every
    // coarse node whose interpolation reaches a finer Dirichlet node
    C.dir.assign(nlc, 0);
    int64_t ndir = 0;
    for (int64_t kk = 0; kk <= C.n[2]; ++kk)
      for (int64_t jj = 0; jj <= C.n[1]; ++jj)
        for (int64_t ii = 0; ii <= C.n[0]; ++ii) {
          if (2 * ii > F.n[0] || 2 * jj > F.n[1] || 2 * kk > F.n[2]) continue;
          if (F.lat[F.node(2 * ii, 2 * jj, 2 * kk)] == LAT_DIRICHLET) {
            C.dir[C.node(ii, jj, kk)] = 1;
            ++ndir;
          }
        }
    if (ndir == 0)
      for (int64_t kk = 0; kk <= F.n[2]; ++kk)
        for (int64_t jj = 0; jj <= F.n[1]; ++jj)
          for (int64_t ii = 0; ii <= F.n[0]; ++ii)
            if (F.lat[F.node(ii, jj, kk)] == LAT_DIRICHLET) {
              const int64_t p[3] = {ii, jj, kk};
              mark_dirichlet(C, p, 2);
              ++ndir;
            }
    if (ndir == 0) break;   // a coarse level without Dirichlet node would be singular
    MGLevelHost M;
    for (int a = 0; a < 3; ++a) M.n[a] = C.n[a], M.h[a] = 2.0 * mg.lev[k].h[a];
    assemble(C, M);
    // prolongation rows over the G(k) nodes, then restriction = transpose
    const MGLevelHost& Fm = mg.lev[k];
    M.p_ptr.assign(Fm.nn + 1, 0);
    {
      for (int64_t f = 0; f < Fm.nn; ++f) {
        const int64_t fc[3] = {Fm.coord[3 * f], Fm.coord[3 * f + 1], Fm.coord[3 * f + 2]};
        if (!interp_row(C, fc, 2, M.p_col, M.p_w)) {
          mg.why = "coarse transfer weight on a missing node";
          return;
        }
        M.p_ptr[f + 1] = int32_t(M.p_col.size());
      }
    }
    transpose(Fm.nn, M.p_ptr, M.p_col, M.p_w, M.nn, M.r_ptr, M.r_col, M.r_w);
    mg.lev.push_back(std::move(M));
    lats.push_back(std::move(C));
  }
  const MGLevelHost& K = mg.lev.back();
  if (mg.lev.size() < 1 || K.nn > MG_MAX_COARSEST || K.nn == 0) {
    mg.why = "coarsest level too large for a dense solve";
    return;
  }
  if (!dense_inverse(K, mg.cinv)) {
    mg.why = "coarsest operator not positive definite";
    return;
  }
  mg.small_start = int(mg.lev.size()) - 1;
  for (int k = 0; k < int(mg.lev.size()); ++k)
    if (mg.lev[k].nn <= small_nodes) { mg.small_start = k; break; }
  mg.ok = true;
}

}  // namespace ibg
