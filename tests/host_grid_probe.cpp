// Test driver for the library's host-side grid builder (no GPU needed).
// Reads   <in>:  ib_grid_desc bytes, int64 M, X[M][3], dS[M], UB[M][3], inside[n2][n1][n0]
// Writes  <out>: int64 N, M, nc, n_hang, n_if, nbricks, then canon_q (int32 N*3),
//                canon_flags (uint8 N), active (uint8 nc), level (uint8 nc),
//                ib_origin (int32 M*3), ib_free (uint8 M*64: 1 free, 2 non-free, 0 missing)
#include <cstdio>
#include <string>
#include <vector>

#include "setup.hpp"

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
  ib_status s = ibg::build_host_grid(d, M, X.data(), dS.data(), UB.data(), inside.data(), G, err);
  if (s != IB_OK) {
    std::fprintf(stderr, "%s\n", err.c_str());
    return 10 + int(s);
  }
  FILE* o = std::fopen(argv[2], "wb");
  const int64_t N = int64_t(G.canon_slot.size());
  const int64_t hdr[6] = {N, M, nc, int64_t(G.hang_slot.size()), int64_t(G.if_coarse.size()), G.nbricks};
  std::fwrite(hdr, 8, 6, o);
  std::fwrite(G.canon_q.data(), 4, G.canon_q.size(), o);
  std::fwrite(G.canon_flags.data(), 1, G.canon_flags.size(), o);
  std::fwrite(G.active.data(), 1, G.active.size(), o);
  std::fwrite(G.level.data(), 1, G.level.size(), o);
  std::fwrite(G.ib_origin.data(), 4, G.ib_origin.size(), o);
  std::vector<uint8_t> fr(64 * M);
  for (int64_t i = 0; i < M; ++i)
    for (int a = 0; a < 64; ++a) fr[64 * i + a] = (G.ib_free[i] >> a & 1) ? 1 : (G.ib_slot[64 * i + a] >= 0 ? 2 : 0);
  std::fwrite(fr.data(), 1, fr.size(), o);
  std::fclose(o);
  return 0;
}
