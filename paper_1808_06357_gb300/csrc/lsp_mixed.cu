// Mixed-radix two-sweep path (path 5): rank-1 lattices whose n is not a power of two (or any n)
// beyond the SMEM-resident size, n = N1 N2 with both factors at most 4096 points.
//
// The length-n DFT (Thm 1(iii)) is split four-step style (eq. Fnx): point k = k1 + N1 k2,
// bin xi = xi2 + N2 xi1, W_n^{k xi} = W_n^{k1 xi2} W_N1^{k1 xi1} W_N2^{k2 xi2}.  One Strang step
// (eq. StrangTDSE in physical form, Algorithm 1, adjacent potential half-steps merged) is two
// sweeps over the state:
//   column sweep (tile: C adjacent columns k1, N2 points each, stride N1):
//       conj W_n^{k1 xi2}, IDFT_N2, 1/n, P, DFT_N2, W_n^{k1 xi2}
//   row sweep (tile: R adjacent rows xi2 of N1 contiguous points):  DFT_N1, K, IDFT_N1
// with K in the row sweep's native order (position xi1 + N1 xi2 holds bin xi2 + N2 xi1).  The
// line transforms are the mixed-radix passes of the SMEM-resident path (any radix per factor)
// on a tile in shared memory; the four-step twiddle comes from FP64 tables
// (W_n^a = W_N1^{a div N2} W_n^{a mod N2}) and is applied in FP64, and 1/n as a hi + lo pair, so
// that neither rounds the norm the same way every step.  One CTA per tile, plain launches.
#include <algorithm>

#include "lsp_internal.cuh"
#include "lsp_pass.cuh"
#include "lsp_tile.cuh"

namespace lsp {

constexpr int kMxTile = 4096;        // points per tile (two buffers in shared memory)
constexpr int kMxThreads = 512;
constexpr int kMxMaxLine = 4096;     // largest N1, N2

enum MxKind { kMxHead = 0, kMxMid, kMxTail, kMxColFwd, kMxRow, kMxRowFwd };

template <typename T> struct MxDesc {
  using Rl = decltype(T{}.x);
  T* u;
  const T* Ph;
  const T* Pf;
  const T* K;            // row sweep's native order
  const T* tw;           // per-axis W_len^k (row axis, then column axis); complex64: lo parts at tw_lo
  const double2* twc;    // W_N1^q, q < N1
  const double2* twf;    // W_n^r, r < N2
  double2* spec;         // spectral output (chi order), row forward sweep
  SmallAxis row, col;    // lengths N1 and N2 with their radix factors and table offsets
  int tw_lo;
  int N1, N2, C, R;      // columns per column tile, rows per row tile
  long long n;
  Rl inv_n, inv_n_lo;    // 1/n as hi + lo
};

// x * W_n^{+-a} in FP64 (a = k1 xi2 mod n)
template <int DIR, typename T>
__device__ __forceinline__ T mx_twiddle(const MxDesc<T>& D, T x, long long a) {
  const double2 c = __ldg(D.twc + a / D.N2), f = __ldg(D.twf + a % D.N2);
  double wr = c.x * f.x - c.y * f.y, wi = c.x * f.y + c.y * f.x;
  if (DIR > 0) wi = -wi;
  const double xr = (double)x.x, xi = (double)x.y;
  T y;
  y.x = (decltype(y.x))(xr * wr - xi * wi);
  y.y = (decltype(y.y))(xr * wi + xi * wr);
  return y;
}

// Line transform of every line of axis `ax` in a tile of `cnt` elements; returns the buffer
// that holds the result.
template <int DIR, typename T>
__device__ T* mx_dft(const MxDesc<T>& D, const SmallAxis& ax, int cnt, T* a, T* b) {
  T* src = a;
  T* dst = b;
  int Ns = 1;
  for (int f = 0; f < ax.nfac; ++f) {
    small_pass<DIR>(ax, D.tw, D.tw_lo, ax.fac[f], Ns, cnt, src, dst);
    __syncthreads();
    Ns *= ax.fac[f];
    T* t = src; src = dst; dst = t;
  }
  return src;
}

template <typename T, int KIND>
__global__ void __launch_bounds__(kMxThreads) mx_col(const __grid_constant__ MxDesc<T> D) {
  extern __shared__ __align__(16) unsigned char mx_smem[];
  T* a = reinterpret_cast<T*>(mx_smem);
  T* b = a + kMxTile;
  const int c0 = (int)blockIdx.x * D.C;
  const int cc = min(D.C, D.N1 - c0);          // columns in this tile (the last may be ragged)
  const int cnt = D.N2 * cc;
  SmallAxis ax = D.col;
  ax.stride = cc;                              // tile layout: element (column b, row i) at i cc + b
  constexpr bool INV = KIND == kMxMid || KIND == kMxTail;
  constexpr bool FWD = KIND == kMxHead || KIND == kMxMid || KIND == kMxColFwd;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int i = e / cc, k1 = c0 + e % cc;
    T x = D.u[k1 + (long long)i * D.N1];
    if (INV) x = mx_twiddle<+1>(D, x, ((long long)k1 * i) % D.n);
    if (KIND == kMxHead) x = apply_phase(x, __ldg(D.Ph + k1 + (long long)i * D.N1));
    a[e] = x;
  }
  __syncthreads();
  T* cur = a;
  if constexpr (INV) {
    cur = mx_dft<+1>(D, ax, cnt, a, b);
    const T* P = KIND == kMxMid ? D.Pf : D.Ph;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int i = e / cc, k1 = c0 + e % cc;
      T x = cur[e];
      x = cmake(fma(x.x, D.inv_n, x.x * D.inv_n_lo), fma(x.y, D.inv_n, x.y * D.inv_n_lo));
      cur[e] = apply_phase(x, __ldg(P + k1 + (long long)i * D.N1));
    }
    __syncthreads();
  }
  if constexpr (FWD) cur = mx_dft<-1>(D, ax, cnt, cur, cur == a ? b : a);
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int i = e / cc, k1 = c0 + e % cc;
    T x = cur[e];
    if (FWD) x = mx_twiddle<-1>(D, x, ((long long)k1 * i) % D.n);
    D.u[k1 + (long long)i * D.N1] = x;
  }
}

template <typename T, int KIND>
__global__ void __launch_bounds__(kMxThreads) mx_row(const __grid_constant__ MxDesc<T> D) {
  extern __shared__ __align__(16) unsigned char mx_smem[];
  T* a = reinterpret_cast<T*>(mx_smem);
  T* b = a + kMxTile;
  const int r0 = (int)blockIdx.x * D.R;
  const int rr = min(D.R, D.N2 - r0);
  const int cnt = D.N1 * rr;
  const long long base = (long long)r0 * D.N1;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) a[e] = D.u[base + e];
  __syncthreads();
  T* cur = mx_dft<-1>(D, D.row, cnt, a, b);
  if constexpr (KIND == kMxRowFwd) {
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const long long xi2 = r0 + e / D.N1, xi1 = e % D.N1;
      const T x = cur[e];
      const double s = 1.0 / (double)D.n;
      D.spec[xi2 + (long long)D.N2 * xi1] = make_double2((double)x.x * s, (double)x.y * s);
    }
  } else {
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) cur[e] = apply_phase(cur[e], __ldg(D.K + base + e));
    __syncthreads();
    cur = mx_dft<+1>(D, D.row, cnt, cur, cur == a ? b : a);
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) D.u[base + e] = cur[e];
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

// n = N1 N2 with N2 <= N1 <= 4096, both factorisable into the passes' radices, N2 as large as
// possible (the column sweep's tiles then hold the fewest, longest-run columns).
bool mixed_geometry(long long n, int* N1, int* N2) {
  for (long long b = (long long)std::sqrt((double)n) + 1; b >= 1; --b) {
    if (n % b || b > kMxMaxLine) continue;
    const long long a = n / b;
    if (a < b || a > kMxMaxLine) continue;
    SmallAxis t1, t2;
    if (!factorize_axis((int)a, t1) || !factorize_axis((int)b, t2)) continue;
    *N1 = (int)a;
    *N2 = (int)b;
    return true;
  }
  return false;
}

template <typename T> static MxDesc<T> mx_desc(lsp_plan p, void* state) {
  MxDesc<T> D{};
  D.u = (T*)state;
  D.Ph = (const T*)p->Ph;
  D.Pf = (const T*)p->Pf;
  D.K = (const T*)p->K;
  D.tw = (const T*)p->tw_small;
  D.tw_lo = p->tw_lo;
  D.twc = (const double2*)p->tw_coarse;
  D.twf = (const double2*)p->tw_fine;
  D.spec = (double2*)p->stage;
  D.row = p->axes[0];
  D.col = p->axes[1];
  D.N1 = p->N1;
  D.N2 = p->N2;
  D.C = std::max(1, kMxTile / p->N2);
  D.R = std::max(1, kMxTile / p->N1);
  D.n = p->ntot;
  const double inv = 1.0 / (double)p->ntot;
  D.inv_n = (decltype(D.inv_n))inv;
  D.inv_n_lo = (decltype(D.inv_n))(inv - (double)D.inv_n);
  return D;
}

template <typename T> static int mx_launch(int kind, const MxDesc<T>& D, cudaStream_t s) {
  const size_t smem = 2 * (size_t)kMxTile * sizeof(T);
  const unsigned cols = (unsigned)((D.N1 + D.C - 1) / D.C), rows = (unsigned)((D.N2 + D.R - 1) / D.R);
  auto go = [&](const void* fn, unsigned grid) -> int {
    LSP_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    void* args[] = {(void*)&D};
    LSP_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(kMxThreads), args, smem, s));
    return LSP_OK;
  };
  switch (kind) {
    case kMxHead: return go((const void*)mx_col<T, kMxHead>, cols);
    case kMxMid: return go((const void*)mx_col<T, kMxMid>, cols);
    case kMxTail: return go((const void*)mx_col<T, kMxTail>, cols);
    case kMxColFwd: return go((const void*)mx_col<T, kMxColFwd>, cols);
    case kMxRow: return go((const void*)mx_row<T, kMxRow>, rows);
    default: return go((const void*)mx_row<T, kMxRowFwd>, rows);
  }
}

template <typename T> static int mx_steps(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s) {
  const MxDesc<T> D = mx_desc<T>(p, state);
  int rc = mx_launch<T>(kMxHead, D, s);
  for (int64_t st = 0; st < nsteps && !rc; ++st) {
    rc = mx_launch<T>(kMxRow, D, s);
    if (!rc) rc = mx_launch<T>(st + 1 < nsteps ? kMxMid : kMxTail, D, s);
  }
  return rc;
}

template <typename T> static int mx_spectral(lsp_plan p, cudaStream_t s) {
  LSP_CUDA_TRY(cudaMemcpyAsync(p->work, p->u, (size_t)p->ntot * sizeof(T), cudaMemcpyDeviceToDevice, s));
  const MxDesc<T> D = mx_desc<T>(p, p->work);
  int rc = mx_launch<T>(kMxColFwd, D, s);
  if (!rc) rc = mx_launch<T>(kMxRowFwd, D, s);
  return rc;
}

int mixed_steps_on(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s) {
  return p->prec == LSP_C64 ? mx_steps<float2>(p, state, nsteps, s) : mx_steps<double2>(p, state, nsteps, s);
}

int mixed_spectral(lsp_plan p, cudaStream_t s) {
  return p->prec == LSP_C64 ? mx_spectral<float2>(p, s) : mx_spectral<double2>(p, s);
}

}  // namespace lsp
