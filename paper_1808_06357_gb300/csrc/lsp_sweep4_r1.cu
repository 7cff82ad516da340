// Kernel instantiations of the four-sweep Strang step for rank-1 lattices of
// n = 2^m points, rows of N1 = 4096 points and columns of N2 = n / 4096
// (see lsp_sweep4.cuh).
#include "lsp_sweep4.cuh"

namespace lsp {

template <typename T> static bool lookup(int m, S4Kernels* k) {
  switch (m) {
    case 20: *k = s4_kernels<T, 8, 12, true>(); return true;
    case 22: *k = s4_kernels<T, 10, 12, true>(); return true;
    case 23: *k = s4_kernels<T, 11, 12, true>(); return true;
    case 24: *k = s4_kernels<T, 12, 12, true>(); return true;
    case 25: *k = s4_kernels<T, 13, 12, true>(); return true;
    default: return false;
  }
}

bool s4_kernels_rank1(int prec, int m, S4Kernels* k) {
  return prec == LSP_C64 ? lookup<float2>(m, k) : lookup<double2>(m, k);
}

}  // namespace lsp
