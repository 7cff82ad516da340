// Kernel instantiations of the four-sweep Strang step for rank-2 lattices
// n1 x n2 = 2^m1 x 2^m2 (see lsp_sweep4.cuh).
#include "lsp_sweep4.cuh"

namespace lsp {

template <typename T> static bool lookup(int m1, int m2, S4Kernels* k) {
  if (m1 == 14 && m2 == 12) { *k = s4_kernels<T, 14, 12, false>(); return true; }
  if (m1 == 12 && m2 == 10) { *k = s4_kernels<T, 12, 10, false>(); return true; }
  if (m1 == 11 && m2 == 9) { *k = s4_kernels<T, 11, 9, false>(); return true; }
  if (m1 == 10 && m2 == 8) { *k = s4_kernels<T, 10, 8, false>(); return true; }
  return false;
}

bool s4_kernels_rank2(int prec, int m1, int m2, S4Kernels* k) {
  return prec == LSP_C64 ? lookup<float2>(m1, m2, k) : lookup<double2>(m1, m2, k);
}

}  // namespace lsp
