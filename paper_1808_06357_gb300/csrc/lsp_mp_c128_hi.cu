// Kernel instantiations of the multipass Strang step: double2 state, lattice sizes 2^m for m in {18 19 20 21 22}.
// One kernel per size keeps every line length compile-time (see lsp_mp.cuh).
#include "lsp_mp.cuh"

namespace lsp {

bool mp_kernels_c128_hi(int m, MPKernels* k) {
  switch (m) {
    case 18: *k = mp_kernels_for<double2, 18>(); return true;
    case 19: *k = mp_kernels_for<double2, 19>(); return true;
    case 20: *k = mp_kernels_for<double2, 20>(); return true;
    case 21: *k = mp_kernels_for<double2, 21>(); return true;
    case 22: *k = mp_kernels_for<double2, 22>(); return true;
    default: return false;
  }
}

}  // namespace lsp
