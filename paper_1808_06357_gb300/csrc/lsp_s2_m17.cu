// Kernels of the TMA two-sweep path for n = 2^17 (every schedule), in a translation unit
// of their own so that the sizes compile in parallel.
#include "lsp_s2.cuh"

namespace lsp {
bool s2_kernels_17(int v, S2Kernels* k) { return s2_kernels_m<17>(v, k); }
}  // namespace lsp
