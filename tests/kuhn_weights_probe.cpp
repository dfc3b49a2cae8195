// Test driver: prints the library's incident-cell-mask weights (kuhn_weights.hpp)
// for every mask: 15 mass weights, the 6 axis-edge counts (+x -x +y -y +z -z),
// then the 45 gradient couplings (stencil offset major, axis minor), then the
// 135 transpose-gradient couplings (offset, test component, trial component).
#include <cstdio>

#include "kuhn_weights.hpp"

int main() {
  for (int m = 0; m < 256; ++m) {
    for (int k = 0; k < 15; ++k) std::printf("%d ", ibg::mass_weight(m, k));
    for (int a = 0; a < 3; ++a)
      for (int s = 1; s >= -1; s -= 2) std::printf("%d ", ibg::stiff_edge_count(m, a, s));
    for (int k = 0; k < 15; ++k)       // gradient couplings
      for (int a = 0; a < 3; ++a) std::printf("%d ", ibg::grad_weight(m, k, a));
    for (int k = 0; k < 15; ++k)       // transpose-gradient couplings
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) std::printf("%d ", ibg::trans_weight(m, k, i, j));
    std::printf("\n");
  }
  return 0;
}
