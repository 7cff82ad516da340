// Kernel instantiations of the multipass Strang step: float2 state, lattice sizes 2^m for m in {13 14 15 16 17}.
// One kernel per size keeps every line length compile-time (see lsp_mp.cuh).
#include "lsp_mp.cuh"

namespace lsp {

bool mp_kernels_c64_lo(int m, MPKernels* k) {
  switch (m) {
    case 13: *k = mp_kernels_for<float2, 13>(); return true;
    case 14: *k = mp_kernels_for<float2, 14>(); return true;
    case 15: *k = mp_kernels_for<float2, 15>(); return true;
    case 16: *k = mp_kernels_for<float2, 16>(); return true;
    case 17: *k = mp_kernels_for<float2, 17>(); return true;
    default: return false;
  }
}

}  // namespace lsp
