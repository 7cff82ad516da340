// Kernels of the TMA two-sweep path for n = 2^24 (every schedule), in a translation unit
// of their own so that the sizes compile in parallel.
#include "lsp_s2.cuh"

namespace lsp {
bool s2_kernels_24(int v, S2Kernels* k) { return s2_kernels_m<24>(v, k); }
}  // namespace lsp
