// Kernel instantiations of the multipass Strang step: float2 state, lattice sizes 2^m for m in {18 19 20 21 22 23}.
// One kernel per size keeps every line length compile-time (see lsp_mp.cuh).
#include "lsp_mp.cuh"

namespace lsp {

bool mp_kernels_c64_hi(int m, MPKernels* k) {
  switch (m) {
    case 18: *k = mp_kernels_for<float2, 18>(); return true;
    case 19: *k = mp_kernels_for<float2, 19>(); return true;
    case 20: *k = mp_kernels_for<float2, 20>(); return true;
    case 21: *k = mp_kernels_for<float2, 21>(); return true;
    case 22: *k = mp_kernels_for<float2, 22>(); return true;
#if LSP_MP_NT_C64 >= 512   // rows of 2^13 points need 8192-point tiles
    case 23: *k = mp_kernels_for<float2, 23>(); return true;
#endif
    default: return false;
  }
}

}  // namespace lsp
