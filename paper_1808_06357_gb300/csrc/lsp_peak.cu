// Arithmetic-throughput probe: the measured FMA rate that the complex128 path
// (FP64 arithmetic on GB300's small FP64 units) and the complex64 path (FP32)
// are compared against.  Every thread runs kChains independent FMA chains, so the
// pipes stay full without memory traffic; the rate is flops (2 per FMA) over the
// CUDA-event time of the launch.
#include "lsp_internal.cuh"

namespace lsp {

constexpr int kChains = 8;

template <typename R>
__global__ void __launch_bounds__(256) fma_probe(R* out, int iters, R mul, R add) {
  R a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = (R)(threadIdx.x + c) * (R)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], mul, add);
  }
  R sum = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) sum += a[c];
  if (sum == (R)-1.2345e30) out[0] = sum;            // never true: keeps the chains live
}

template <typename R> static int probe(int device, double* tflops, double* ms_out) {
  int sms = 0;
  LSP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  R* out = nullptr;
  if (cudaMalloc(&out, sizeof(R)) != cudaSuccess) { cudaGetLastError(); return LSP_ERR_OOM; }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = LSP_OK;
  const int blocks = sms * 8, threads = 256;
  const int iters = sizeof(R) == 8 ? 1 << 14 : 1 << 16;
  // (1 - 2^-20) and a small addend: the chains approach a fixed point and never overflow
  const R mul = (R)(1.0 - 1.0 / 1048576.0), add = (R)1e-6;
  do {
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) { rc = LSP_ERR_CUDA; break; }
    fma_probe<R><<<blocks, threads>>>(out, iters / 8, mul, add);          // warm-up
    if (cudaEventRecord(e0) != cudaSuccess) { rc = LSP_ERR_CUDA; break; }
    fma_probe<R><<<blocks, threads>>>(out, iters, mul, add);
    if (cudaEventRecord(e1) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) { rc = LSP_ERR_CUDA; break; }
    if (cudaGetLastError() != cudaSuccess) { rc = LSP_ERR_CUDA; break; }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f) { rc = LSP_ERR_CUDA; break; }
    const double flops = 2.0 * kChains * (double)iters * (double)blocks * (double)threads;
    *tflops = flops / ((double)ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return rc;
}

}  // namespace lsp

extern "C" int lsp_fma_rate(int device, int prec, double* tflops, double* ms) {
  using namespace lsp;
  if (!tflops || (prec != LSP_C64 && prec != LSP_C128)) return LSP_ERR_BAD_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) { cudaGetLastError(); return LSP_ERR_CUDA; }
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return LSP_ERR_CUDA;
  const int rc = prec == LSP_C128 ? probe<double>(device, tflops, ms) : probe<float>(device, tflops, ms);
  cudaSetDevice(prev);
  return rc;
}
