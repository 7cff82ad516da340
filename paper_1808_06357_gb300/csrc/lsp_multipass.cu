// Multipass Strang step for rank-1 lattices with n = N1 * N2 = 2^m points.
//
// The length-n DFT of Thm 1(iii) is split four-step style: with
// k = k1 + N1 k2 (point index) and xi = xi2 + N2 xi1 (bin index),
//   W_n^{k xi} = W_n^{k1 xi2} W_N1^{k1 xi1} W_N2^{k2 xi2}.
// One Strang step (eq. StrangTDSE in physical form, adjacent potential
// half-steps merged) then costs two sweeps over the state:
//   column pass (per k1, stride N1):  conj-twiddle . IDFT_N2 . P . DFT_N2 . twiddle
//   row pass    (per xi2, contiguous): DFT_N1 . K . IDFT_N1
// where P = exp(-i dt v / gamma) (exp(-i dt v / (2 gamma)) at the ends) and
// K_xi = exp(-i gamma 2 pi^2 ||h_xi||^2 dt) is stored in the row pass'
// native order (position xi1 + N1 xi2 holds bin xi2 + N2 xi1).
// A persistent cooperative kernel runs all 2N+1 sweeps of N steps, with a
// bounded grid barrier between sweeps.
#include <cooperative_groups.h>

#include <algorithm>

#include "lsp_tile.cuh"

namespace lsp {

enum PassKind { kHead = 0, kMid = 1, kTail = 2, kRow = 3, kColFwd = 4, kRowFwd = 5 };

template <typename T> struct MPInst {
  using R = decltype(T{}.x);
  T* u;                 // state (in place)
  const T* Ph;          // half potential phase (kappa order)
  const T* Pf;          // full potential phase (kappa order)
  const T* K;           // kinetic phase (row-pass native order)
  const T* twl;         // W_Lmax^k
  const T* twf;         // W_n^k, k < n / Lmax
  double2* spec;        // spectral output (chi order), kRowFwd only
  int logN1, logN2, logn, logLmax;
  int logCc, logCr;     // log2 lines per column / row tile
  int logR1c, pc;       // column-line radix plan (length N2)
  int logR1r, pr;       // row-line radix plan (length N1)
  int ncol, nrow;       // tiles per sweep
  R inv_n;
};

template <typename T> struct MPParams {
  const MPInst<T>* inst;    // device array (ninst entries)
  const int2* colmap;       // sweep tile -> (instance, local tile); null when ninst == 1
  const int2* rowmap;
  int ninst;
  int total_col, total_row;
  long long nsteps;
  int kind;                 // single-sweep kernels only
  unsigned* bar;
  int* err;
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T ldst(const T* p) { return __ldcg(p); }
template <typename T> __device__ __forceinline__ void stst(T* p, T v) { __stcg(p, v); }
template <typename T> __device__ __forceinline__ T ldtab(const T* p) { return __ldcs(p); }

// W_n^{a} for a = k1 * xi2 mod n from the two-level table.
template <typename T>
__device__ __forceinline__ T big_tw(const MPInst<T>& I, unsigned k1, unsigned xi2) {
  unsigned a = (k1 * xi2) & ((1u << I.logn) - 1u);
  int sh = I.logn - I.logLmax;
  T hi = __ldg(I.twl + (a >> sh));
  T lo = __ldg(I.twf + (a & ((1u << sh) - 1u)));
  return cmul(hi, lo);
}

template <typename T> __device__ __forceinline__ T scale_if(T x, bool s, decltype(T{}.x) f) {
  return s ? cscale(x, f) : x;
}

// ---------------------------------------------------------------------------
// Column pass (lines = columns k1 of length N2, stride N1)
// ---------------------------------------------------------------------------
template <typename T, int NT>
__device__ void col_pass(const MPInst<T>& I, int tile, int kind, T* sm) {
  Geo g{I.logN2, I.logCc, 0, I.logR1c, I.pc, I.logLmax};
  const int c0 = tile << I.logCc;
  T* __restrict__ u = I.u;
  const bool inv = (kind == kMid || kind == kTail);
  const bool fwd = (kind == kHead || kind == kMid || kind == kColFwd);
  const T* ptab = kind == kMid ? I.Pf : (kind == kColFwd ? nullptr : I.Ph);
  T v[16];

  if (inv) {
    // load in the last-pass pattern (radix 16), conj twiddle W_n^{-k1 xi2}
    const int lLR = g.logL - 4;
    const int nb = 1 << (g.logC + lLR);
    int beta = threadIdx.x;
    if (beta < nb) {
      int b, j; bmap(g, beta, lLR, b, j);
      const unsigned k1 = c0 + b;
_Pragma("unroll")
      for (int t = 0; t < 16; ++t) {
        unsigned xi2 = j + (t << lLR);
        T x = ldst(u + k1 + ((size_t)xi2 << I.logN1));
        v[t] = cmulc(x, big_tw(I, k1, xi2));
      }
    }
    line_idft<NT>(g, sm, I.twl, v);
  } else {
    LSP_R1_DISPATCH(g.logR1, {
      constexpr int LR = (RR == 2 ? 1 : RR == 4 ? 2 : RR == 8 ? 3 : 4);
      const int lLR = g.logL - LR;
      const int nb = 1 << (g.logC + lLR);
_Pragma("unroll")
      for (int q = 0; q < 16 / RR; ++q) {
        int beta = threadIdx.x + NT * q;
        if (beta < nb) {
          int b, j; bmap(g, beta, lLR, b, j);
_Pragma("unroll")
          for (int r = 0; r < RR; ++r)
            v[q * RR + r] = ldst(u + (c0 + b) + ((size_t)(j + (r << lLR)) << I.logN1));
        }
      }
    });
  }

  // potential phase on the pass-1 input pattern (physical samples)
  if (ptab) {
    const bool sc = inv;
    const auto f = I.inv_n;
    LSP_R1_DISPATCH(g.logR1, {
      constexpr int LR = (RR == 2 ? 1 : RR == 4 ? 2 : RR == 8 ? 3 : 4);
      const int lLR = g.logL - LR;
      const int nb = 1 << (g.logC + lLR);
_Pragma("unroll")
      for (int q = 0; q < 16 / RR; ++q) {
        int beta = threadIdx.x + NT * q;
        if (beta < nb) {
          int b, j; bmap(g, beta, lLR, b, j);
_Pragma("unroll")
          for (int r = 0; r < RR; ++r) {
            size_t pos = (c0 + b) + ((size_t)(j + (r << lLR)) << I.logN1);
            v[q * RR + r] = apply_phase(scale_if(v[q * RR + r], sc, f), ldtab(ptab + pos));
          }
        }
      }
    });
  }

  if (fwd) {
    line_dft<NT>(g, sm, I.twl, v);
    const int lLR = g.logL - 4;
    const int nb = 1 << (g.logC + lLR);
    int beta = threadIdx.x;
    if (beta < nb) {
      int b, j; bmap(g, beta, lLR, b, j);
      const unsigned k1 = c0 + b;
_Pragma("unroll")
      for (int t = 0; t < 16; ++t) {
        unsigned xi2 = j + (t << lLR);
        stst(u + k1 + ((size_t)xi2 << I.logN1), cmul(v[t], big_tw(I, k1, xi2)));
      }
    }
  } else {
    LSP_R1_DISPATCH(g.logR1, {
      constexpr int LR = (RR == 2 ? 1 : RR == 4 ? 2 : RR == 8 ? 3 : 4);
      const int lLR = g.logL - LR;
      const int nb = 1 << (g.logC + lLR);
_Pragma("unroll")
      for (int q = 0; q < 16 / RR; ++q) {
        int beta = threadIdx.x + NT * q;
        if (beta < nb) {
          int b, j; bmap(g, beta, lLR, b, j);
_Pragma("unroll")
          for (int r = 0; r < RR; ++r)
            stst(u + (c0 + b) + ((size_t)(j + (r << lLR)) << I.logN1), v[q * RR + r]);
        }
      }
    });
  }
}

// ---------------------------------------------------------------------------
// Row pass (lines = rows xi2 of length N1, contiguous)
// ---------------------------------------------------------------------------
template <typename T, int NT>
__device__ void row_pass(const MPInst<T>& I, int tile, int kind, T* sm) {
  Geo g{I.logN1, I.logCr, 1, I.logR1r, I.pr, I.logLmax};
  const int r0 = tile << I.logCr;
  T* __restrict__ u = I.u;
  T v[16];

  LSP_R1_DISPATCH(g.logR1, {
    constexpr int LR = (RR == 2 ? 1 : RR == 4 ? 2 : RR == 8 ? 3 : 4);
    const int lLR = g.logL - LR;
    const int nb = 1 << (g.logC + lLR);
_Pragma("unroll")
    for (int q = 0; q < 16 / RR; ++q) {
      int beta = threadIdx.x + NT * q;
      if (beta < nb) {
        int b, j; bmap(g, beta, lLR, b, j);
_Pragma("unroll")
        for (int r = 0; r < RR; ++r)
          v[q * RR + r] = ldst(u + ((size_t)(r0 + b) << I.logN1) + j + (r << lLR));
      }
    }
  });

  line_dft<NT>(g, sm, I.twl, v);

  const int lLR = g.logL - 4;
  const int nb = 1 << (g.logC + lLR);
  if (kind == kRowFwd) {
    // spectral output: bin xi = xi2 + N2 xi1, scaled by 1/n (eq. approx_uhat)
    int beta = threadIdx.x;
    if (beta < nb) {
      int b, j; bmap(g, beta, lLR, b, j);
      const size_t xi2 = r0 + b;
_Pragma("unroll")
      for (int t = 0; t < 16; ++t) {
        size_t xi1 = j + (t << lLR);
        T x = cscale(v[t], I.inv_n);
        I.spec[xi2 + (xi1 << I.logN2)] = make_double2((double)x.x, (double)x.y);
      }
    }
    return;
  }
  {
    int beta = threadIdx.x;
    if (beta < nb) {
      int b, j; bmap(g, beta, lLR, b, j);
      const size_t rowbase = (size_t)(r0 + b) << I.logN1;
_Pragma("unroll")
      for (int t = 0; t < 16; ++t) v[t] = apply_phase(v[t], ldtab(I.K + rowbase + j + (t << lLR)));
    }
  }
  line_idft<NT>(g, sm, I.twl, v);

  LSP_R1_DISPATCH(g.logR1, {
    constexpr int LR = (RR == 2 ? 1 : RR == 4 ? 2 : RR == 8 ? 3 : 4);
    const int lLR2 = g.logL - LR;
    const int nb2 = 1 << (g.logC + lLR2);
_Pragma("unroll")
    for (int q = 0; q < 16 / RR; ++q) {
      int beta = threadIdx.x + NT * q;
      if (beta < nb2) {
        int b, j; bmap(g, beta, lLR2, b, j);
_Pragma("unroll")
        for (int r = 0; r < RR; ++r)
          stst(u + ((size_t)(r0 + b) << I.logN1) + j + (r << lLR2), v[q * RR + r]);
      }
    }
  });
}

// ---------------------------------------------------------------------------
// Bounded grid barrier (all CTAs co-resident: cooperative launch).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned& target, int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    target += gridDim.x;
    __threadfence();
    atomicAdd(bar, 1u);
    int ok = 1;
    long long spins = 0;
    while ((int)(ld_acquire(bar) - target) < 0) {
      if (*(volatile int*)err != 0) { ok = 0; break; }
      if (++spins > kSpinLimit) { atomicCAS(err, 0, LSP_ERR_TIMEOUT); ok = 0; break; }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename T>
__device__ __forceinline__ void tile_of(const MPParams<T>& P, const int2* map, int t, int& inst, int& local) {
  if (map) { int2 m = map[t]; inst = m.x; local = m.y; }
  else { inst = 0; local = t; }
}

#ifndef LSP_MP_MINBLOCKS
#define LSP_MP_MINBLOCKS 1
#endif

// Sweeps 0..2N of N steps: even sweeps are column passes (head, mid..., tail),
// odd sweeps row passes; a bounded grid barrier separates consecutive sweeps.
template <typename T, int NT>
__global__ void __launch_bounds__(NT, LSP_MP_MINBLOCKS) mp_persistent(const __grid_constant__ MPParams<T> P) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  unsigned target = 0;
  const long long nsweep = 2 * P.nsteps + 1;
  for (long long sw = 0; sw < nsweep; ++sw) {
    const bool col = (sw & 1) == 0;
    const int kind = !col ? kRow : (sw == 0 ? kHead : (sw == nsweep - 1 ? kTail : kMid));
    const int total = col ? P.total_col : P.total_row;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
      int i, l;
      tile_of(P, col ? P.colmap : P.rowmap, t, i, l);
      if (col) col_pass<T, NT>(P.inst[i], l, kind, sm);
      else row_pass<T, NT>(P.inst[i], l, kind, sm);
    }
    if (sw + 1 < nsweep && !grid_barrier(P.bar, target, P.err)) return;
  }
}

// One sweep per launch (spectral output and the non-cooperative fallback).
template <typename T, int NT>
__global__ void __launch_bounds__(NT, LSP_MP_MINBLOCKS) mp_sweep(const __grid_constant__ MPParams<T> P) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const bool col = P.kind != kRow && P.kind != kRowFwd;
  const int total = col ? P.total_col : P.total_row;
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    int i, l;
    if (col) { tile_of(P, P.colmap, t, i, l); col_pass<T, NT>(P.inst[i], l, P.kind, sm); }
    else { tile_of(P, P.rowmap, t, i, l); row_pass<T, NT>(P.inst[i], l, P.kind, sm); }
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <typename T> struct Cfg;
template <> struct Cfg<float2> { static constexpr int NT = kThreadsC64, TILE = kTileC64; };
template <> struct Cfg<double2> { static constexpr int NT = kThreadsC128, TILE = kTileC128; };

static int ilog2i(long long x) { int l = 0; while ((1ll << l) < x) ++l; return l; }

template <typename T> static void radix_plan(int logL, int& logR1, int& p) {
  int rem = logL % 4;
  logR1 = rem == 0 ? 4 : rem;
  p = (logL - logR1) / 4 + 1;
}

template <typename T>
static MPInst<T> make_inst(lsp_plan pl, double2* spec) {
  MPInst<T> I{};
  constexpr int TILE = Cfg<T>::TILE;
  I.u = (T*)pl->u;
  I.Ph = (const T*)pl->Ph;
  I.Pf = (const T*)pl->Pf;
  I.K = (const T*)pl->K;
  I.twl = (const T*)pl->tw_line;
  I.twf = (const T*)pl->tw_fine;
  I.spec = spec;
  I.logN1 = pl->logN1; I.logN2 = pl->logN2; I.logn = pl->logn; I.logLmax = pl->logLmax;
  const int logTile = ilog2i(TILE);
  I.logCc = std::min(logTile - pl->logN2, pl->logN1);
  I.logCr = std::min(logTile - pl->logN1, pl->logN2);
  radix_plan<T>(pl->logN2, I.logR1c, I.pc);
  radix_plan<T>(pl->logN1, I.logR1r, I.pr);
  I.ncol = 1 << (pl->logN1 - I.logCc);
  I.nrow = 1 << (pl->logN2 - I.logCr);
  I.inv_n = (decltype(I.inv_n))(1.0 / (double)pl->ntot);
  return I;
}

template <typename T> static int max_coresident(int& grid) {
  constexpr int NT = Cfg<T>::NT;
  const size_t smem = (size_t)Cfg<T>::TILE * sizeof(T);
  static int cached = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  LSP_CUDA_TRY(cudaFuncSetAttribute(mp_persistent<T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  LSP_CUDA_TRY(cudaFuncSetAttribute(mp_sweep<T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (cached < 0) {
    int per_sm = 0, sms = 0;
    LSP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mp_persistent<T, NT>, NT, smem));
    LSP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cached = per_sm * sms;
  }
  grid = cached;
  return grid > 0 ? LSP_OK : LSP_ERR_CUDA;
}

// Run the persistent kernel over the instances described by the device array `dinst`.
template <typename T>
static int run_persistent(const MPInst<T>* dinst, const int2* colmap, const int2* rowmap, int ninst,
                          int total_col, int total_row, int64_t nsteps, unsigned* bar, int* err,
                          cudaStream_t s) {
  constexpr int NT = Cfg<T>::NT;
  const size_t smem = (size_t)Cfg<T>::TILE * sizeof(T);
  int grid = 0;
  int rc = max_coresident<T>(grid);
  if (rc) return rc;
  grid = std::min(grid, std::max(total_col, total_row));
  MPParams<T> P{dinst, colmap, rowmap, ninst, total_col, total_row, (long long)nsteps, 0, bar, err};
  LSP_CUDA_TRY(cudaMemsetAsync(bar, 0, sizeof(unsigned), s));
  void* args[] = {&P};
  LSP_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)mp_persistent<T, NT>, dim3(grid), dim3(NT), args,
                                           smem, s));
  return LSP_OK;
}

template <typename T>
static int run_sweep(const MPInst<T>* dinst, const int2* colmap, const int2* rowmap, int ninst,
                     int total_col, int total_row, int kind, cudaStream_t s) {
  constexpr int NT = Cfg<T>::NT;
  const size_t smem = (size_t)Cfg<T>::TILE * sizeof(T);
  int grid = 0;
  int rc = max_coresident<T>(grid);
  if (rc) return rc;
  const bool col = kind != kRow && kind != kRowFwd;
  grid = std::min(grid, col ? total_col : total_row);
  MPParams<T> P{dinst, colmap, rowmap, ninst, total_col, total_row, 0, kind, nullptr, nullptr};
  mp_sweep<T, NT><<<grid, NT, smem, s>>>(P);
  return cuda_status(cudaGetLastError());
}

int multipass_desc_bytes(int prec) {
  return prec == LSP_C64 ? (int)sizeof(MPInst<float2>) : (int)sizeof(MPInst<double2>);
}

// Descriptor slot 0: the plan's state; slot 1: the spectral-transform copy.
template <typename T>
static int upload_desc_impl(lsp_plan p, cudaStream_t s) {
  MPInst<T> I[2] = {make_inst<T>(p, nullptr), make_inst<T>(p, (double2*)p->stage)};
  I[1].u = (T*)p->work;
  LSP_CUDA_TRY(cudaMemcpyAsync(p->desc, I, sizeof(I), cudaMemcpyHostToDevice, s));
  return LSP_OK;
}

int multipass_upload_desc(lsp_plan p, cudaStream_t s) {
  return p->prec == LSP_C64 ? upload_desc_impl<float2>(p, s) : upload_desc_impl<double2>(p, s);
}

template <typename T>
static int steps_impl(lsp_plan p, int64_t nsteps, cudaStream_t s) {
  MPInst<T> I = make_inst<T>(p, nullptr);
  return run_persistent<T>((const MPInst<T>*)p->desc, nullptr, nullptr, 1, I.ncol, I.nrow, nsteps,
                           p->bar, p->err, s);
}

// Spectral coefficients (eq. approx_uhat) of the current state into the
// plan's staging buffer in chi order: column DFT + twiddle, then row DFT / n,
// on a copy of the state.
template <typename T>
static int spectral_impl(lsp_plan p, cudaStream_t s) {
  const size_t bytes = (size_t)p->ntot * sizeof(T);
  LSP_CUDA_TRY(cudaMemcpyAsync(p->work, p->u, bytes, cudaMemcpyDeviceToDevice, s));
  MPInst<T> I = make_inst<T>(p, nullptr);
  const MPInst<T>* d = (const MPInst<T>*)p->desc + 1;
  int rc = run_sweep<T>(d, nullptr, nullptr, 1, I.ncol, I.nrow, kColFwd, s);
  if (!rc) rc = run_sweep<T>(d, nullptr, nullptr, 1, I.ncol, I.nrow, kRowFwd, s);
  return rc;
}

int multipass_steps(lsp_plan p, int64_t nsteps, cudaStream_t s) {
  return p->prec == LSP_C64 ? steps_impl<float2>(p, nsteps, s) : steps_impl<double2>(p, nsteps, s);
}

int multipass_spectral(lsp_plan p, cudaStream_t s) {
  return p->prec == LSP_C64 ? spectral_impl<float2>(p, s) : spectral_impl<double2>(p, s);
}

}  // namespace lsp
