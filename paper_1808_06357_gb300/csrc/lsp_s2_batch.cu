// Kernels of batched TMA two-sweep steps over instances of 2^16 .. 2^23 points (every size
// inside each kernel, dispatched per tile), in a translation unit of their own.
#include "lsp_s2.cuh"

namespace lsp {

S2BatchKernels s2_batch_kernels() {
  S2BatchKernels K;
  K.k[kS2Head] = (const void*)s2_batch_sweep<kS2Head>;
  K.k[kS2Mid] = (const void*)s2_batch_sweep<kS2Mid>;
  K.k[kS2Tail] = (const void*)s2_batch_sweep<kS2Tail>;
  K.k[kS2Row] = (const void*)s2_batch_sweep<kS2Row>;
  K.smem[kS2Head] = S2BatchSmem<kS2Head>::BYTES;
  K.smem[kS2Mid] = S2BatchSmem<kS2Mid>::BYTES;
  K.smem[kS2Tail] = S2BatchSmem<kS2Tail>::BYTES;
  K.smem[kS2Row] = S2BatchSmem<kS2Row>::BYTES;
  return K;
}

}  // namespace lsp
