// Test driver for the library's natural-boundary rows of the symmetric viscous
// form (setup.cpp, build_natural_rows); no GPU needed.
// Reads   <in>:  ib_grid_desc bytes, int64 M, X[M][3], dS[M], UB[M][3], inside[n2][n1][n0]
// Writes  <out>: int64 rows, then per row int64 q[3] (finest coordinates of
//                the row's slot), int64 entries, and per entry int64 q[3] of
//                the trial slot, int64 (3 test + trial component), double weight
#include <cstdio>
#include <string>
#include <vector>

#include "setup.hpp"

static void finest(const ibg::HostGrid& G, int32_t s, int64_t q[3]) {
  const int32_t b = s / ibg::BV, t = s % ibg::BV;
  const int l = G.brick_level[b], sh = G.L - l;
  q[0] = (int64_t(G.brick_coord[3 * b]) * ibg::BS + t % ibg::BS) << sh;
  q[1] = (int64_t(G.brick_coord[3 * b + 1]) * ibg::BS + (t / ibg::BS) % ibg::BS) << sh;
  q[2] = (int64_t(G.brick_coord[3 * b + 2]) * ibg::BS + t / (ibg::BS * ibg::BS)) << sh;
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
    return 6;
  }
  ibg::NaturalRows R;
  ibg::build_natural_rows(d, G, R);
  FILE* o = std::fopen(argv[2], "wb");
  const int64_t nr = int64_t(R.row_slot.size());
  std::fwrite(&nr, 8, 1, o);
  for (int64_t r = 0; r < nr; ++r) {
    int64_t q[3];
    finest(G, R.row_slot[r], q);
    std::fwrite(q, 8, 3, o);
    const int64_t ne = R.row_off[r + 1] - R.row_off[r];
    std::fwrite(&ne, 8, 1, o);
    for (int32_t e = R.row_off[r]; e < R.row_off[r + 1]; ++e) {
      finest(G, R.ent_slot[e], q);
      std::fwrite(q, 8, 3, o);
      const int64_t comp = R.ent_comp[e];
      std::fwrite(&comp, 8, 1, o);
      std::fwrite(&R.ent_w[e], 8, 1, o);
    }
  }
  std::fclose(o);
  return 0;
}
