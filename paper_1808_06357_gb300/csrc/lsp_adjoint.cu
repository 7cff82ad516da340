// Adjoint of N Strang steps: gradients of a real objective J(u_N) with respect
// to the potential samples v and the initial state u_0.  Not in the paper.
//
// One step is S = P . F^{-1} K F . P with unitary diagonal factors, so the
// cotangent recursion is lambda_k = S^H lambda_{k+1} = S(-dt) lambda_{k+1}
// (P(-dt) = conj P, K(-dt) = conj K): an ordinary Strang step with -dt.
// Differentiating P = exp(-i a v), a = dt / (2 gamma), at both half steps of
// step k and using |P| = 1 leaves only boundary states:
//   dJ/dv += a [ Im(conj(lambda_{k+1}) u_{k+1}) + Im(conj(lambda_k) u_k) ],
// hence dJ/dv = a [ f(N) + f(0) + 2 sum_{0<j<N} f(j) ], f(j) = Im(conj(lambda_j) u_j).
// Forward states are recomputed per segment from checkpoints stored every
// ckpt_stride steps (default ceil(sqrt(N))).
#include <math.h>

#include <vector>

#include "lsp_internal.cuh"

using namespace lsp;

namespace {

struct DeviceGuard {
  int prev = 0;
  explicit DeviceGuard(int dev) { cudaGetDevice(&prev); cudaSetDevice(dev); }
  ~DeviceGuard() { cudaSetDevice(prev); }
};

// grad[k] += w * Im(conj(lam_k) u_k)
template <typename T>
__global__ void grad_accum(double* __restrict__ grad, const T* __restrict__ lam, const T* __restrict__ u,
                           double w, long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const double lr = lam[k].x, li = lam[k].y, ur = u[k].x, ui = u[k].y;
    grad[k] += w * (lr * ui - li * ur);
  }
}

int steps_on(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s) { return path_steps_on(p, state, nsteps, s); }

}  // namespace

extern "C" int lsp_adjoint(lsp_plan p, double dt, int64_t nsteps, const void* lamT, double* grad_v, void* grad_u0,
                           int64_t ckpt_stride, void* stream) {
  if (!p || !lamT || !grad_v || !grad_u0 || nsteps < 0 || !isfinite(dt) || ckpt_stride < 0) return LSP_ERR_BAD_ARG;
  if (*p->err_host != 0) return *p->err_host;
  DeviceGuard g(p->device);
  cudaStream_t s = (cudaStream_t)stream;
  const long long n = p->ntot;
  const size_t sb = (size_t)n * (p->prec == LSP_C64 ? sizeof(float2) : sizeof(double2));
  LSP_CUDA_TRY(cudaMemsetAsync(grad_v, 0, (size_t)n * sizeof(double), s));
  if (nsteps == 0) {
    LSP_CUDA_TRY(cudaMemcpyAsync(grad_u0, lamT, sb, cudaMemcpyDeviceToDevice, s));
    return LSP_OK;
  }
  const long long N = nsteps;
  long long c = ckpt_stride > 0 ? ckpt_stride : (long long)ceil(sqrt((double)N));
  if (c > N) c = N;
  const long long nseg = (N + c - 1) / c;
  // buffers: checkpoints u_{k c}, segment states, adjoint state
  char* ck = nullptr;
  char* seg = nullptr;
  void* lam = nullptr;
  if (cudaMallocAsync((void**)&ck, sb * nseg, s) != cudaSuccess ||
      cudaMallocAsync((void**)&seg, sb * c, s) != cudaSuccess || cudaMallocAsync(&lam, sb, s) != cudaSuccess) {
    cudaGetLastError();
    if (ck) cudaFreeAsync(ck, s);
    if (seg) cudaFreeAsync(seg, s);
    return LSP_ERR_OOM;
  }
  const int grid = (int)((n + 255) / 256 < 152 * 16 ? (n + 255) / 256 : 152 * 16);
  const double a = dt / (2.0 * p->gamma);
  auto accum = [&](const void* u, double w) {
    if (p->prec == LSP_C64)
      grad_accum<float2><<<grid, 256, 0, s>>>(grad_v, (const float2*)lam, (const float2*)u, w * a, n);
    else
      grad_accum<double2><<<grid, 256, 0, s>>>(grad_v, (const double2*)lam, (const double2*)u, w * a, n);
  };
  int rc = LSP_OK;
  do {
    // forward with checkpoints; the plan's state ends at u_N
    if ((rc = build_phase_tables(p, dt, s))) break;
    for (long long k = 0; k < nseg && !rc; ++k) {
      if (cudaMemcpyAsync(ck + k * sb, p->u, sb, cudaMemcpyDeviceToDevice, s) != cudaSuccess) { rc = LSP_ERR_CUDA; break; }
      const long long len = (k + 1) * c <= N ? c : N - k * c;
      rc = steps_on(p, p->u, len, s);
    }
    if (rc) break;
    // lambda_N and the j = N term
    if (cudaMemcpyAsync(lam, lamT, sb, cudaMemcpyDeviceToDevice, s) != cudaSuccess) { rc = LSP_ERR_CUDA; break; }
    accum(p->u, 1.0);
    for (long long k = nseg - 1; k >= 0 && !rc; --k) {
      const long long s0 = k * c, e = (k + 1) * c <= N ? (k + 1) * c : N;
      // forward states u_{s0} .. u_{e-1}
      if ((rc = build_phase_tables(p, dt, s))) break;
      if (cudaMemcpyAsync(seg, ck + k * sb, sb, cudaMemcpyDeviceToDevice, s) != cudaSuccess) { rc = LSP_ERR_CUDA; break; }
      for (long long j = s0 + 1; j < e && !rc; ++j) {
        char* dst = seg + (j - s0) * sb;
        if (cudaMemcpyAsync(dst, dst - sb, sb, cudaMemcpyDeviceToDevice, s) != cudaSuccess) { rc = LSP_ERR_CUDA; break; }
        rc = steps_on(p, dst, 1, s);
      }
      if (rc) break;
      // backward through the segment: lambda_j = S(-dt) lambda_{j+1}
      if ((rc = build_phase_tables(p, -dt, s))) break;
      for (long long j = e - 1; j >= s0 && !rc; --j) {
        rc = steps_on(p, lam, 1, s);
        if (!rc) accum(seg + (j - s0) * sb, j == 0 ? 1.0 : 2.0);
      }
    }
    if (rc) break;
    if (cudaMemcpyAsync(grad_u0, lam, sb, cudaMemcpyDeviceToDevice, s) != cudaSuccess) { rc = LSP_ERR_CUDA; break; }
    if (cudaGetLastError() != cudaSuccess) rc = LSP_ERR_CUDA;
  } while (0);
  cudaFreeAsync(ck, s);
  cudaFreeAsync(seg, s);
  cudaFreeAsync(lam, s);
  if (!rc && cudaMemcpyAsync(p->err_host, p->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    rc = LSP_ERR_CUDA;
  return rc;
}
