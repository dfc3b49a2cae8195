// Test driver for the host-side multigrid hierarchy builder (no GPU needed).
// Reads   <in>:  the same input as host_grid_probe.cpp
// Writes  <out>: int64 ok, nlev, small_start, nslots, N; canon_slot (int32 N);
//                slot_q (int32 nslots*3, finest coordinates, -1 for empty slots);
//                then per level: int64 nn, nd, nr, np, n[3]; double h[3];
//                coord (int32 nn*3), dir_coord (int32 nd*3), nbr (int32 nn*6),
//                offd (double nn*6), diag (double nn), r_ptr (int32 nn+1),
//                r_col/r_w (nr), p_ptr (int32 rows+1), p_col/p_w (np);
//                then (hierarchy built) nbricks, meta (uint16 nslots), brick_level,
//                brick_coord, lat_n[3], nlat, lat0, npart, pbase, r0slot, r0ptr,
//                nidx, r0idx
#include <cstdio>
#include <string>
#include <vector>

#include "mg.hpp"
#include "setup.hpp"

template <typename T>
static void put(FILE* o, const std::vector<T>& v) {
  if (!v.empty()) std::fwrite(v.data(), sizeof(T), v.size(), o);
}

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 3;
  ib_grid_desc d;
  int64_t M = 0;
  if (std::fread(&d, sizeof(d), 1, f) != 1 || std::fread(&M, 8, 1, f) != 1) return 4;
  std::vector<double> X(3 * M), dS(M), UB(3 * M);
  const int64_t nc = int64_t(d.n[0]) * d.n[1] * d.n[2];
  std::vector<uint8_t> inside(nc);
  if (std::fread(X.data(), 8, X.size(), f) != X.size() || std::fread(dS.data(), 8, dS.size(), f) != dS.size() ||
      std::fread(UB.data(), 8, UB.size(), f) != UB.size() || std::fread(inside.data(), 1, nc, f) != size_t(nc))
    return 5;
  std::fclose(f);
  ibg::HostGrid G;
  std::string err;
  if (ibg::build_host_grid(d, M, X.data(), dS.data(), UB.data(), inside.data(), G, err) != IB_OK) {
    std::fprintf(stderr, "%s\n", err.c_str());
    return 10;
  }
  ibg::MGHost mg;
  ibg::build_mg(G, mg);
  if (!mg.ok) std::fprintf(stderr, "%s\n", mg.why.c_str());
  FILE* o = std::fopen(argv[2], "wb");
  const int64_t ns = G.nbricks * ibg::BV, N = int64_t(G.canon_slot.size());
  const int64_t hdr[5] = {mg.ok ? 1 : 0, int64_t(mg.lev.size()), mg.small_start, ns, N};
  std::fwrite(hdr, 8, 5, o);
  put(o, G.canon_slot);
  std::vector<int32_t> q(3 * ns, -1);
  for (int64_t s = 0; s < ns; ++s) {
    if (!(G.meta[s] & ibg::M_VALID)) continue;
    const int64_t b = s / ibg::BV, t = s % ibg::BV, l = G.brick_level[b];
    q[3 * s] = int32_t((G.brick_coord[3 * b] * ibg::BS + t % ibg::BS) << (G.L - l));
    q[3 * s + 1] = int32_t((G.brick_coord[3 * b + 1] * ibg::BS + (t / ibg::BS) % ibg::BS) << (G.L - l));
    q[3 * s + 2] = int32_t((G.brick_coord[3 * b + 2] * ibg::BS + t / (ibg::BS * ibg::BS)) << (G.L - l));
  }
  put(o, q);
  for (const auto& L : mg.lev) {
    const int64_t h2[7] = {L.nn, int64_t(L.dir_coord.size() / 3), int64_t(L.r_col.size()), int64_t(L.p_col.size()),
                           L.n[0], L.n[1], L.n[2]};
    std::fwrite(h2, 8, 7, o);
    std::fwrite(L.h, 8, 3, o);
    put(o, L.coord);
    put(o, L.dir_coord);
    put(o, L.nbr);
    put(o, L.offd);
    put(o, L.diag);
    put(o, L.r_ptr);
    put(o, L.r_col);
    put(o, L.r_w);
    const int64_t np_rows = int64_t(L.p_ptr.size());
    std::fwrite(&np_rows, 8, 1, o);
    put(o, L.p_ptr);
    put(o, L.p_col);
    put(o, L.p_w);
  }
  // the weight-free form of the composite <-> G0 transfers
  if (mg.ok) {
    const int64_t nb = G.nbricks, nl = mg.lat_n[0] * mg.lat_n[1] * mg.lat_n[2];
    std::fwrite(&nb, 8, 1, o);
    put(o, G.meta);
    put(o, G.brick_level);
    put(o, G.brick_coord);
    std::fwrite(mg.lat_n, 8, 3, o);
    std::fwrite(&nl, 8, 1, o);
    put(o, mg.lat0);
    std::fwrite(&mg.npart, 8, 1, o);
    put(o, mg.pbase);
    put(o, mg.r0slot);
    put(o, mg.r0ptr);
    const int64_t ni = int64_t(mg.r0idx.size());
    std::fwrite(&ni, 8, 1, o);
    put(o, mg.r0idx);
  }
  std::fclose(o);
  return 0;
}
