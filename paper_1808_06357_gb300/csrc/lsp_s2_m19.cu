// Kernels of the TMA two-sweep path for n = 2^19 (every schedule), in a translation unit
// of their own so that the sizes compile in parallel.
#include "lsp_s2.cuh"

namespace lsp {
bool s2_kernels_19(int v, S2Kernels* k) { return s2_kernels_m<19>(v, k); }
}  // namespace lsp
