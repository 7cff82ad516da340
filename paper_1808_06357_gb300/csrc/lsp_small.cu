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
#include <algorithm>

#include "lsp_internal.cuh"

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
  SmallAxis axes[2];
  R inv_n;           // 1/n rounded
  R inv_n_lo;        // 1/n - inv_n
};

template <int DIR, typename T>
__device__ void small_pass(const SmallAxis& ax, const T* tw, int tw_lo, int R, int Ns, int n, const T* x, T* y) {
  const int len = ax.len, st = ax.stride;
  const int m = len / (Ns * R);          // len / (Ns R)
  const int lenR = len / R;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int inner = e % st;
    const int ia = (e / st) % len;
    const int outer = e / (st * len);
    const int jm = ia % Ns;
    const int s = (ia / Ns) % R;
    const int j = (ia / (Ns * R)) * Ns + jm;
    const int base = outer * st * len + inner;
    const int step = jm + Ns * s;
    T acc;
    acc.x = 0;
    acc.y = 0;
    int kk = 0;                            // (r * step) mod (Ns R)
    const int NsR = Ns * R;
    for (int r = 0; r < R; ++r) {
      T xv = x[base + (j + r * lenR) * st];
      T w = __ldg(tw + ax.tw_off + kk * m);
      if (DIR > 0) w.y = -w.y;
      if constexpr (sizeof(T) == 8) {
        // FP32: twiddle as hi + lo so the fixed rounding of each table entry
        // does not accumulate over the steps
        T wl = __ldg(tw + tw_lo + ax.tw_off + kk * m);
        if (DIR > 0) wl.y = -wl.y;
        const float tr = fmaf(xv.x, wl.x, -xv.y * wl.y), ti = fmaf(xv.x, wl.y, xv.y * wl.x);
        acc.x = fmaf(xv.x, w.x, fmaf(-xv.y, w.y, acc.x + tr));
        acc.y = fmaf(xv.x, w.y, fmaf(xv.y, w.x, acc.y + ti));
      } else {
        acc = cadd(acc, cmul(xv, w));
      }
      kk += step;
      if (kk >= NsR) kk -= NsR;
    }
    y[e] = acc;
  }
}

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
  S.axes[0] = p->axes[0];
  S.axes[1] = p->axes[1];
  S.inv_n = (decltype(S.inv_n))(1.0 / (double)p->ntot);
  S.inv_n_lo = (decltype(S.inv_n))(1.0 / (double)p->ntot - (double)S.inv_n);
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

int small_steps(lsp_plan p, int64_t nsteps, cudaStream_t s) {
  return p->prec == LSP_C64 ? small_launch<float2>(p->desc, 1, (int)p->ntot, nsteps, 0, s)
                            : small_launch<double2>(p->desc, 1, (int)p->ntot, nsteps, 0, s);
}

int small_spectral(lsp_plan p, cudaStream_t s) {
  return p->prec == LSP_C64 ? small_launch<float2>(p->desc, 1, (int)p->ntot, 0, 1, s)
                            : small_launch<double2>(p->desc, 1, (int)p->ntot, 0, 1, s);
}

}  // namespace lsp
