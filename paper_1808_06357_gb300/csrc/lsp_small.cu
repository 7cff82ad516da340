// SMEM-resident Strang loop for small lattices (2 n complex values fit in
// shared memory): one CTA per instance runs every step without leaving the
// SM except for the phase tables, which stay L1/L2 resident.
//
// The r-dimensional DFT of Thm 1(iii) / eq. Fnx is computed axis by axis by
// mixed-radix Stockham passes over any factorisation of n_i (odd primes
// such as 31 included): output o of a radix-R pass with span Ns is
//   y[o] = sum_r x[j + r len/R] W_len^{r (j mod Ns + Ns s) (len / (Ns R))},
// with s = (o / Ns) mod R and j = (o / (Ns R)) Ns + o mod Ns.
// One step follows Algorithm 1 in physical form with merged half steps:
//   u <- P . F^{-1} K F u   (P_half before the first and after the last step).
#include <string.h>

#include <algorithm>

#include "lsp_internal.cuh"
#include "lsp_tile.cuh"
#include "lsp_pass.cuh"

namespace lsp {

template <typename T> struct SmallDesc {
  using R = decltype(T{}.x);
  T* u;
  const T* Ph;
  const T* Pf;
  const T* K;        // chi order
  const T* tw;       // per-axis W_len^k tables (complex64: hi parts, then lo parts)
  double2* spec;     // spectral output (chi order)
  int tw_lo;         // offset of the lo parts (complex64)
  int n;
  int naxes;
  SmallAxis axes[kMaxRank];
  R inv_n;           // 1/n rounded
  R inv_n_lo;        // 1/n - inv_n
  const T* twl;      // rank 1, n = 2^logn with a line kernel: its per-pass twiddles (else null)
  int logn;
};

// Full r-D DFT (DIR = -1 forward, +1 inverse, unnormalised); returns the buffer with the result.
template <int DIR, typename T>
__device__ T* small_dft(const SmallDesc<T>& S, T* a, T* b) {
  T* src = a;
  T* dst = b;
  for (int ai = 0; ai < S.naxes; ++ai) {
    const SmallAxis& ax = S.axes[ai];
    int Ns = 1;
    for (int f = 0; f < ax.nfac; ++f) {
      small_pass<DIR>(ax, S.tw, S.tw_lo, ax.fac[f], Ns, S.n, src, dst);
      __syncthreads();
      Ns *= ax.fac[f];
      T* t = src; src = dst; dst = t;
    }
  }
  return src;
}

// The Strang loop on a state already in shared memory (buffer a; b is the
// second buffer): P_half, then per step F, K, F^{-1}, 1/n and P (P_full between
// steps, P_half after the last); the result is written back to S.u.
template <typename T>
__device__ void small_steps_body(const SmallDesc<T>& S, T* a, T* b, long long nsteps) {
  const int n = S.n;
  for (int k = threadIdx.x; k < n; k += blockDim.x) a[k] = apply_phase(a[k], __ldg(S.Ph + k));
  __syncthreads();
  T* cur = a;
  for (long long step = 0; step < nsteps; ++step) {
    T* oth = cur == a ? b : a;
    cur = small_dft<-1>(S, cur, oth);
    for (int k = threadIdx.x; k < n; k += blockDim.x) cur[k] = apply_phase(cur[k], __ldg(S.K + k));
    __syncthreads();
    oth = cur == a ? b : a;
    cur = small_dft<+1>(S, cur, oth);
    const T* P = step + 1 < nsteps ? S.Pf : S.Ph;
    // 1/n as hi + lo: for n not a power of two a rounded 1/n would scale the
    // norm by the same factor every step
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      T x = cur[k];
      x = cmake(fma(x.x, S.inv_n, x.x * S.inv_n_lo), fma(x.y, S.inv_n, x.y * S.inv_n_lo));
      cur[k] = apply_phase(x, __ldg(P + k));
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < n; k += blockDim.x) S.u[k] = cur[k];
}

template <typename T>
__global__ void __launch_bounds__(kSmallThreads) small_kernel(const SmallDesc<T>* D, long long nsteps,
                                                              int spectral) {
  const SmallDesc<T>& S = D[blockIdx.x];
  extern __shared__ __align__(16) unsigned char smraw[];
  T* a = reinterpret_cast<T*>(smraw);
  T* b = a + S.n;
  const int n = S.n;
  for (int k = threadIdx.x; k < n; k += blockDim.x) a[k] = S.u[k];
  __syncthreads();
  if (spectral) {
    T* c = small_dft<-1>(S, a, b);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      T x = cscale(c[k], S.inv_n);
      S.spec[k] = make_double2((double)x.x, (double)x.y);
    }
    return;
  }
  if (nsteps <= 0) return;
  small_steps_body(S, a, b, nsteps);
}

// --------------------------------------------------------------------------
// Rank 1, n = 2^m (2^11 .. 2^13): the whole lattice is one line of the tile FFT
// (16 points per thread, NT = n / 16 threads), held in registers across all
// steps; shared memory only carries the exchanges between radix-16 passes.
// Per step: forward line DFT (natural bin order out), K by bin, inverse line DFT
// (back to the load pattern), 1/n (exact) and the potential phase.
// --------------------------------------------------------------------------
template <typename T> constexpr bool small_line_ok(int logn) {
  return logn >= 11 && logn <= (sizeof(T) == 8 ? 13 : 12);
}

template <typename T, int LOGN>
__global__ void __launch_bounds__(1 << (LOGN - 4)) small_line_kernel(const SmallDesc<T>* D, long long nsteps) {
  constexpr int NT = 1 << (LOGN - 4);
  using G = Line<T, NT, LOGN, true>;
  constexpr int LR1 = G::LOGR1, R1 = G::R1;
  const SmallDesc<T>& S = D[blockIdx.x];
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  if (nsteps <= 0) return;
  const T* __restrict__ tw = S.twl;
  // element index of register q*R1+r in the load pattern, and of register q in natural order
  auto in_at = [](int q, int r) { int b, j; G::template bm<LR1>(q, b, j); return j + (r << (LOGN - LR1)); };
  int bn, jn;
  G::template bm<4>(0, bn, jn);
  T v[16];
#pragma unroll
  for (int q = 0; q < 16 / R1; ++q)
#pragma unroll
    for (int r = 0; r < R1; ++r) {
      const int i = in_at(q, r);
      v[q * R1 + r] = apply_phase(S.u[i], __ldg(S.Ph + i));
    }
  const auto inv_n = S.inv_n;                         // exact: n is a power of two
  for (long long step = 0; step < nsteps; ++step) {
    T kv[16], pv[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) kv[q] = __ldg(S.K + jn + (q << (LOGN - 4)));
    G::dft(sm, tw, v);
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = apply_phase(v[q], kv[q]);
    const T* P = step + 1 < nsteps ? S.Pf : S.Ph;
#pragma unroll
    for (int q = 0; q < 16 / R1; ++q)
#pragma unroll
      for (int r = 0; r < R1; ++r) pv[q * R1 + r] = __ldg(P + in_at(q, r));
    G::idft(sm, tw, v);
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = apply_phase(cscale(v[k], inv_n), pv[k]);
  }
#pragma unroll
  for (int q = 0; q < 16 / R1; ++q)
#pragma unroll
    for (int r = 0; r < R1; ++r) S.u[in_at(q, r)] = v[q * R1 + r];
}

template <typename T> static int small_line_launch(const void* desc, int count, int logn, long long nsteps, cudaStream_t s) {
  const void* fn = nullptr;
  switch (logn) {
    case 11: fn = (const void*)small_line_kernel<T, 11>; break;
    case 12: fn = (const void*)small_line_kernel<T, 12>; break;
    case 13: if constexpr (small_line_ok<T>(13)) fn = (const void*)small_line_kernel<T, 13>; break;
    default: break;
  }
  if (!fn) return LSP_ERR_UNSUPPORTED;
  const size_t smem = ((size_t)1 << logn) * sizeof(T);
  LSP_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const void* d = desc;
  void* args[] = {(void*)&d, (void*)&nsteps};
  LSP_CUDA_TRY(cudaLaunchKernel(fn, dim3(count), dim3(1u << (logn - 4)), args, smem, s));
  return LSP_OK;
}

bool small_line_supported(int prec, int r, int logn) {
  return r == 1 && (prec == LSP_C64 ? small_line_ok<float2>(logn) : small_line_ok<double2>(logn));
}

template <typename T> static SmallDesc<T> make_small(lsp_plan p) {
  SmallDesc<T> S{};
  S.u = (T*)p->u;
  S.Ph = (const T*)p->Ph;
  S.Pf = (const T*)p->Pf;
  S.K = (const T*)p->K;
  S.tw = (const T*)p->tw_small;
  S.tw_lo = p->tw_lo;
  S.spec = (double2*)p->stage;
  S.n = (int)p->ntot;
  S.naxes = p->naxes;
  for (int i = 0; i < kMaxRank; ++i) S.axes[i] = p->axes[i];
  S.inv_n = (decltype(S.inv_n))(1.0 / (double)p->ntot);
  S.inv_n_lo = (decltype(S.inv_n))(1.0 / (double)p->ntot - (double)S.inv_n);
  S.twl = (const T*)p->tw_pass;
  S.logn = p->tw_pass ? p->logn : 0;
  return S;
}

int small_desc_bytes(int prec) {
  return prec == LSP_C64 ? (int)sizeof(SmallDesc<float2>) : (int)sizeof(SmallDesc<double2>);
}

template <typename T> static int small_upload_impl(lsp_plan p, cudaStream_t s) {
  SmallDesc<T> S = make_small<T>(p);
  LSP_CUDA_TRY(cudaMemcpyAsync(p->desc, &S, sizeof(S), cudaMemcpyHostToDevice, s));
  return LSP_OK;
}

int small_upload_desc(lsp_plan p, cudaStream_t s) {
  return p->prec == LSP_C64 ? small_upload_impl<float2>(p, s) : small_upload_impl<double2>(p, s);
}

template <typename T>
static int small_launch(const void* desc, int count, int max_n, long long nsteps, int spectral, cudaStream_t s) {
  const size_t smem = 2 * (size_t)max_n * sizeof(T);
  LSP_CUDA_TRY(cudaFuncSetAttribute(small_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  small_kernel<T><<<count, kSmallThreads, smem, s>>>((const SmallDesc<T>*)desc, nsteps, spectral);
  return cuda_status(cudaGetLastError());
}

// Steps of `count` instances from a descriptor array: the line kernel when line_logn > 0
// (every instance of that size), else the mixed-radix kernel.
template <typename T>
static int small_steps_launch(const void* desc, int count, int max_n, int line_logn, long long nsteps, cudaStream_t s) {
  if (line_logn > 0) return small_line_launch<T>(desc, count, line_logn, nsteps, s);
  return small_launch<T>(desc, count, max_n, nsteps, 0, s);
}

int small_steps(lsp_plan p, int64_t nsteps, cudaStream_t s) {
  const int ll = p->tw_pass ? p->logn : 0;
  return p->prec == LSP_C64 ? small_steps_launch<float2>(p->desc, 1, (int)p->ntot, ll, nsteps, s)
                            : small_steps_launch<double2>(p->desc, 1, (int)p->ntot, ll, nsteps, s);
}

int small_spectral(lsp_plan p, cudaStream_t s) {
  return p->prec == LSP_C64 ? small_launch<float2>(p->desc, 1, (int)p->ntot, 0, 1, s)
                            : small_launch<double2>(p->desc, 1, (int)p->ntot, 0, 1, s);
}

// Steps on another state buffer of the plan's geometry (descriptor slot 1),
// with the plan's current phase tables.
template <typename T> static int small_steps_on_impl(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s) {
  SmallDesc<T> S = make_small<T>(p);
  S.u = (T*)state;
  SmallDesc<T>* d = (SmallDesc<T>*)p->desc + 1;
  LSP_CUDA_TRY(cudaMemcpyAsync(d, &S, sizeof(S), cudaMemcpyHostToDevice, s));
  return small_steps_launch<T>(d, 1, (int)p->ntot, S.logn, nsteps, s);
}

int small_steps_on(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s) {
  return p->prec == LSP_C64 ? small_steps_on_impl<float2>(p, state, nsteps, s)
                            : small_steps_on_impl<double2>(p, state, nsteps, s);
}

// Batching: descriptors of many plans in one device array, one CTA per instance.
int small_desc_size(int prec) { return small_desc_bytes(prec); }

void small_fill_desc(lsp_plan p, void* host_out) {
  if (p->prec == LSP_C64) {
    SmallDesc<float2> S = make_small<float2>(p);
    memcpy(host_out, &S, sizeof(S));
  } else {
    SmallDesc<double2> S = make_small<double2>(p);
    memcpy(host_out, &S, sizeof(S));
  }
}

int small_line_logn(lsp_plan p) { return p->tw_pass ? p->logn : 0; }

int small_batch_launch(int prec, const void* ddesc, int count, int max_n, int line_logn, int64_t nsteps,
                       cudaStream_t s) {
  return prec == LSP_C64 ? small_steps_launch<float2>(ddesc, count, max_n, line_logn, nsteps, s)
                         : small_steps_launch<double2>(ddesc, count, max_n, line_logn, nsteps, s);
}

}  // namespace lsp

// ===========================================================================
// Allocation-free entry point: the SMEM-resident Strang loop with its
// scratch (phase and twiddle tables) in a fixed file-scope device array.
// For callers that must not allocate device memory -- code running under a
// host allocator that forbids cudaMalloc, a caller that pre-plans all memory
// (embedded or real-time use), or a context where an allocation could fail
// mid-run.  The paper has no counterpart; this is a deployment convenience.
// ===========================================================================
namespace lsp {

constexpr long long kNoAllocMaxN = 8192;   // largest lattice (points) the fixed scratch holds
constexpr int kNoAllocMaxDev = 64;

// Ph[n], Pf[n], K[n], tw[n], tw_lo[n] of the plan precision: 5 * 8192 * 16 B = 640 KiB,
// held by every device that loads the library until the process exits.
static __device__ __align__(256) double2 g_noalloc_scratch[5 * kNoAllocMaxN];
static void* g_noalloc_addr[kNoAllocMaxDev];

template <typename T>
__global__ void noalloc_tables(const double* __restrict__ v, const int32_t* __restrict__ norm2, T* Ph, T* Pf,
                               T* K, T* tw, T* twlo, int n, double turns_v, double turns_k) {
  using R = decltype(T{}.x);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double th = v[i] * turns_v;
    T a, b, c;
    encode_phase_pair(th, &a, &b);            // as the plan path's build_tables
    encode_phase(turns_k * (double)norm2[i], &c);
    Ph[i] = a;
    Pf[i] = b;
    K[i] = c;
    // W_n^i = exp(-2 pi i i / n), FP64 then rounded (and its residue for FP32)
    double s, co;
    sincospi(-2.0 * (double)i / (double)n, &s, &co);
    T w, wl;
    w.x = (R)co;
    w.y = (R)s;
    wl.x = (R)(co - (double)w.x);
    wl.y = (R)(s - (double)w.y);
    tw[i] = w;
    if (twlo) twlo[i] = wl;
  }
}

template <typename T>
__global__ void __launch_bounds__(kSmallThreads) small_kernel_noalloc(const __grid_constant__ SmallDesc<T> S,
                                                                      long long nsteps) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* a = reinterpret_cast<T*>(smraw);
  T* b = a + S.n;
  for (int k = threadIdx.x; k < S.n; k += blockDim.x) a[k] = S.u[k];
  __syncthreads();
  if (nsteps <= 0) return;
  small_steps_body(S, a, b, nsteps);
}

template <typename T>
static int noalloc_run(void* scratch, long long n, double gamma, double dt, long long nsteps, const double* v,
                       const int32_t* norm2, void* u, cudaStream_t s) {
  T* base = (T*)scratch;
  SmallDesc<T> S{};
  S.u = (T*)u;
  S.Ph = base;
  S.Pf = base + n;
  S.K = base + 2 * n;
  S.tw = base + 3 * n;
  S.tw_lo = (int)n;                       // lo parts follow the n hi parts
  S.spec = nullptr;
  S.n = (int)n;
  S.naxes = 1;
  S.axes[0].len = (int)n;
  S.axes[0].stride = 1;
  S.axes[0].tw_off = 0;
  if (!factorize_axis((int)n, S.axes[0])) return LSP_ERR_TOO_LARGE;
  S.inv_n = (decltype(S.inv_n))(1.0 / (double)n);
  S.inv_n_lo = (decltype(S.inv_n))(1.0 / (double)n - (double)S.inv_n);
  const double turns_v = -dt / (4.0 * M_PI * gamma);
  const double turns_k = -M_PI * gamma * dt;
  const int grid = (int)std::min<long long>((n + 255) / 256, 64);
  noalloc_tables<T><<<grid, 256, 0, s>>>(v, norm2, base, base + n, base + 2 * n, base + 3 * n,
                                         sizeof(T) == 8 ? base + 4 * n : nullptr, (int)n, turns_v, turns_k);
  LSP_CUDA_TRY(cudaGetLastError());
  const size_t smem = 2 * (size_t)n * sizeof(T);
  LSP_CUDA_TRY(cudaFuncSetAttribute(small_kernel_noalloc<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  small_kernel_noalloc<T><<<1, kSmallThreads, smem, s>>>(S, nsteps);
  return cuda_status(cudaGetLastError());
}

}  // namespace lsp

extern "C" int lsp_strang_steps_noalloc(int prec, int64_t n, double gamma, double dt, int64_t nsteps,
                                        const double* v, const int32_t* norm2, void* u, void* stream) {
  using namespace lsp;
  if ((prec != LSP_C64 && prec != LSP_C128) || !v || !norm2 || !u) return LSP_ERR_BAD_ARG;
  if (!(gamma > 0.0) || !isfinite(dt) || nsteps < 0 || n < 1) return LSP_ERR_BAD_ARG;
  // limits: the fixed scratch (8192 points) and two state copies in shared memory
  const size_t csz = prec == LSP_C64 ? sizeof(float2) : sizeof(double2);
  if (n > kNoAllocMaxN || 2 * (size_t)n * csz > (size_t)kSmallSmemBytes) return LSP_ERR_TOO_LARGE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDev) return LSP_ERR_CUDA;
  if (!g_noalloc_addr[dev]) {
    // first call on this device (nsteps = 0 included): device address of the file-scope
    // scratch.  With lazy module loading this also loads this file's module, which
    // reserves the array, so the first call belongs before the allocation-free phase.
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return LSP_ERR_CUDA;
    g_noalloc_addr[dev] = ptr;
  }
  if (nsteps == 0) return LSP_OK;
  cudaStream_t s = (cudaStream_t)stream;
  return prec == LSP_C64 ? noalloc_run<float2>(g_noalloc_addr[dev], n, gamma, dt, nsteps, v, norm2, u, s)
                         : noalloc_run<double2>(g_noalloc_addr[dev], n, gamma, dt, nsteps, v, norm2, u, s);
}
