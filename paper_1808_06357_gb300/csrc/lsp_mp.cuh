// Multipass Strang step for rank-1 lattices with n = N1 * N2 = 2^M points.
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
//
// N steps = a head sweep, a persistent cooperative kernel running sweeps
// 1..2N-1 (row, mid, ..., row) with a bounded grid barrier between sweeps, and
// a tail sweep.  Inside the persistent kernel each CTA prefetches its next
// tile with bulk asynchronous copies (cp.async.bulk, completion on an
// mbarrier) while it transforms the current one, and keeps the twiddle tables
// in shared memory when they fit.
#pragma once

#include <algorithm>

#include "lsp_async.cuh"
#include "lsp_tile.cuh"

namespace lsp {

enum PassKind { kHead = 0, kMid = 1, kTail = 2, kRow = 3, kColFwd = 4, kRowFwd = 5 };

template <typename T> struct MPInst {
  using R = decltype(T{}.x);
  T* u;                 // state (in place)
  const T* Ph;          // half potential phase (kappa order)
  const T* Pf;          // full potential phase (kappa order)
  const T* K;           // kinetic phase (row-pass native order)
  const T* twr;         // per-pass twiddles of the row lines (length N1)
  const T* twc;         // per-pass twiddles of the column lines (length N2)
  const T* twl;         // W_N1^k, k < N1 (coarse factor of W_n^{k1 xi2})
  const T* twf;         // W_n^k, k < N2 (fine factor of W_n^{k1 xi2})
  double2* spec;        // spectral output (chi order), kRowFwd only
  int logN1, logN2, logn, logLmax;
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
  long long spin_limit;     // polls of a bounded wait before it gives up (persistent kernel)
};

#ifndef LSP_MINB_C64
#define LSP_MINB_C64 1
#endif
#ifndef LSP_MINB_C128
#define LSP_MINB_C128 1
#endif
// NT threads per worker, NW workers per CTA, TILE elements per worker tile
// (16 per thread), minimum resident CTAs per SM (register budget).
template <typename T> struct Cfg;
#ifndef LSP_MP_NT_C64
#define LSP_MP_NT_C64 512
#endif
#ifndef LSP_MP_TW_SMEM
#define LSP_MP_TW_SMEM 1
#endif
template <> struct Cfg<float2> {
  static constexpr int NT = LSP_MP_NT_C64, NW = 1, TILE = 16 * NT, MINB = LSP_MINB_C64;
};
template <> struct Cfg<double2> {
  static constexpr int NT = 256, NW = 1, TILE = 4096, MINB = LSP_MINB_C128;
};

// Line lengths of a 2^M-point lattice: N2 = 2^min(10, M/2) (column), N1 = n / N2 (row).
template <int M> struct Split {
  static constexpr int LN2 = M / 2 < 10 ? M / 2 : 10;
  static constexpr int LN1 = M - LN2;
};

template <typename T, int M> using RowLine = Line<T, Cfg<T>::NT, Split<M>::LN1, true, Cfg<T>::NW>;
template <typename T, int M> using ColLine = Line<T, Cfg<T>::NT, Split<M>::LN2, false, Cfg<T>::NW>;

// Shared memory of the persistent kernel: exchange buffer, prefetch buffer
// and (when everything fits in 227 KiB) the twiddle tables.
template <typename T, int M> struct SmemLayout {
  static constexpr int TILE = Cfg<T>::TILE, NW = Cfg<T>::NW;
  static constexpr int work(int w) { return 2 * TILE * w; }
  static constexpr int pre(int w) { return 2 * TILE * w + TILE; }
  static constexpr int twr = 2 * TILE * NW;
  static constexpr int twc = twr + RowLine<T, M>::TW_ENTRIES;
  static constexpr int twl = twc + ColLine<T, M>::TW_ENTRIES;
  static constexpr int twf = twl + (1 << Split<M>::LN1);
  static constexpr int elems_all = twf + (1 << Split<M>::LN2);
  static constexpr bool tw_in_smem = LSP_MP_TW_SMEM && (size_t)elems_all * sizeof(T) <= 227u * 1024u - 256u;
  static constexpr size_t bytes = (size_t)(tw_in_smem ? elems_all : twr) * sizeof(T);
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------

// W_n^{a} for a = k1 * xi2 mod n from the two-level table (global or shared).
template <typename T, int M>
__device__ __forceinline__ T big_tw(const T* twl, const T* twf, unsigned k1, unsigned xi2) {
  const unsigned a = (k1 * xi2) & ((1u << M) - 1u);
  constexpr int sh = M - Split<M>::LN1;
  return twprod(twl[a >> sh], twf[a & ((1u << sh) - 1u)]);
}

// Twiddle tables a pass uses (shared or global).
template <typename T> struct Tw {
  const T* line;   // per-pass table of this pass' lines
  const T* l;      // W_N1^k
  const T* f;      // W_n^k, k < N2
};

enum Src { kFromGlobal = 0, kFromPre = 1 };

// Bulk copies of a tile into the prefetch buffer, issued after the barrier that follows
// the buffer's last reads (completed reads: the copies need no proxy fence before them).
template <typename T, int NT, int M, bool COL>
__device__ __forceinline__ void prefetch_tile(const MPInst<T>& I, int tile, T* pre, unsigned long long* mb);

// ---------------------------------------------------------------------------
// Column pass (lines = columns k1 of length N2, stride N1).  kFromPre: the
// tile sits in the prefetch buffer in natural order (element (b, i) at
// i * C + b); after reading it the pass refills the buffer with tile `nxt`.
// ---------------------------------------------------------------------------
template <typename T, int NT, int M, int KIND, int FROM>
__device__ __forceinline__ void col_pass(const MPInst<T>& I, int tile, T* sm, T* pre, Tw<T> tw,
                                         const MPInst<T>* In = nullptr, int nxt = -1,
                                         unsigned long long* mb = nullptr) {
  constexpr int LOGL = Split<M>::LN2, lN1 = Split<M>::LN1;
  using G = Line<T, NT, LOGL, false, Cfg<T>::NW>;
  constexpr int LR1 = G::LOGR1, R1 = G::R1;
  constexpr bool inv = (KIND == kMid || KIND == kTail);
  constexpr bool fwd = (KIND == kHead || KIND == kMid || KIND == kColFwd);
  const int c0 = tile << G::LOGC;
  T* __restrict__ u = I.u;
  T v[16];

  if constexpr (inv) {
    // last-pass pattern (radix 16): rows xi2 = j + t L/16; conj twiddle W_n^{-k1 xi2}
    int b, j; G::template bm<4>(0, b, j);
    const unsigned k1 = c0 + b;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const unsigned xi2 = j + (t << (LOGL - 4));
      T x = FROM == kFromPre ? pre[(xi2 << G::LOGC) + b] : ldst(u + (k1 + (xi2 << lN1)));
      v[t] = twmulc(x, big_tw<T, M>(tw.l, tw.f, k1, xi2));
    }
  } else {
#pragma unroll
    for (int q = 0; q < 16 / R1; ++q) {
      int b, j; G::template bm<LR1>(q, b, j);
#pragma unroll
      for (int r = 0; r < R1; ++r) {
        const int i = j + (r << (LOGL - LR1));
        v[q * R1 + r] = FROM == kFromPre ? pre[(i << G::LOGC) + b] : ldst(u + ((c0 + b) + (i << lN1)));
      }
    }
  }
  if constexpr (FROM == kFromPre) {
    G::sync();                                           // prefetch buffer free: refill it
    if (nxt >= 0) { prefetch_tile<T, NT, M, true>(*In, nxt, pre, mb); }
  }
  if constexpr (inv) G::idft(sm, tw.line, v);

  if constexpr (KIND != kColFwd) {
    // potential phase on the pass-1 pattern (physical samples k2 = j + r L/R1)
    const T* ptab = KIND == kMid ? I.Pf : I.Ph;
    const auto f = I.inv_n;
#pragma unroll
    for (int q = 0; q < 16 / R1; ++q) {
      int b, j; G::template bm<LR1>(q, b, j);
#pragma unroll
      for (int r = 0; r < R1; ++r) {
        T x = v[q * R1 + r];
        if constexpr (inv) x = cscale(x, f);
        v[q * R1 + r] = apply_phase(x, ldtab(ptab + ((c0 + b) + ((j + (r << (LOGL - LR1))) << lN1))));
      }
    }
  }

  if constexpr (fwd) {
    G::dft(sm, tw.line, v);
    int b, j; G::template bm<4>(0, b, j);
    const unsigned k1 = c0 + b;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const unsigned xi2 = j + (t << (LOGL - 4));
      stst(u + (k1 + (xi2 << lN1)), twmul(v[t], big_tw<T, M>(tw.l, tw.f, k1, xi2)));
    }
  } else {
#pragma unroll
    for (int q = 0; q < 16 / R1; ++q) {
      int b, j; G::template bm<LR1>(q, b, j);
#pragma unroll
      for (int r = 0; r < R1; ++r) stst(u + ((c0 + b) + ((j + (r << (LOGL - LR1))) << lN1)), v[q * R1 + r]);
    }
  }
}

// ---------------------------------------------------------------------------
// Row pass (lines = rows xi2 of length N1, contiguous).  kFromPre: the tile
// sits in the prefetch buffer row-major (b * L + i).
// ---------------------------------------------------------------------------
template <typename T, int NT, int M, int KIND, int FROM>
__device__ __forceinline__ void row_pass(const MPInst<T>& I, int tile, T* sm, T* pre, Tw<T> tw,
                                         const MPInst<T>* In = nullptr, int nxt = -1,
                                         unsigned long long* mb = nullptr) {
  constexpr int LOGL = Split<M>::LN1, lN2 = Split<M>::LN2;
  using G = Line<T, NT, LOGL, true, Cfg<T>::NW>;
  constexpr int LR1 = G::LOGR1, R1 = G::R1;
  const int r0 = tile << G::LOGC;
  T* __restrict__ u = I.u;
  T v[16];

#pragma unroll
  for (int q = 0; q < 16 / R1; ++q) {
    int bb, jj; G::template bm<LR1>(q, bb, jj);
#pragma unroll
    for (int r = 0; r < R1; ++r) {
      const int off = (bb << LOGL) + jj + (r << (LOGL - LR1));
      v[q * R1 + r] = FROM == kFromPre ? pre[off] : ldst(u + ((r0 << LOGL) + off));
    }
  }
  if constexpr (FROM == kFromPre) {
    G::sync();
    if (nxt >= 0) { prefetch_tile<T, NT, M, false>(*In, nxt, pre, mb); }
  }

  G::dft(sm, tw.line, v);

  int b, j; G::template bm<4>(0, b, j);
  if constexpr (KIND == kRowFwd) {
    // spectral output: bin xi = xi2 + N2 xi1, scaled by 1/n (eq. approx_uhat)
    const int xi2 = r0 + b;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const int xi1 = j + (t << (LOGL - 4));
      T x = cscale(v[t], I.inv_n);
      I.spec[xi2 + (xi1 << lN2)] = make_double2((double)x.x, (double)x.y);
    }
  } else {
    const int base = ((r0 + b) << LOGL) + j;
#pragma unroll
    for (int t = 0; t < 16; ++t) v[t] = apply_phase(v[t], ldtab(I.K + base + (t << (LOGL - 4))));
    G::idft(sm, tw.line, v);
#pragma unroll
    for (int q = 0; q < 16 / R1; ++q) {
      int bb, jj; G::template bm<LR1>(q, bb, jj);
#pragma unroll
      for (int r = 0; r < R1; ++r) stst(u + (((r0 + bb) << LOGL) + jj + (r << (LOGL - LR1))), v[q * R1 + r]);
    }
  }
}

// ---------------------------------------------------------------------------
// Bounded grid barrier (all CTAs co-resident: cooperative launch).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned& target, int* err, long long limit) {
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
      if (++spins > limit) { atomicCAS(err, 0, LSP_ERR_TIMEOUT); ok = 0; break; }
      __nanosleep(32);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Sweep tile t -> (instance, local tile); a null map means a single instance.
template <typename T>
__device__ __forceinline__ void tile_of(const int2* map, int t, int& inst, int& local) {
  if (map) { const int2 m = map[t]; inst = m.x; local = m.y; }
  else { inst = 0; local = t; }
}

// Issue the bulk copies of one tile into the prefetch buffer (all threads).
template <typename T, int NT, int M, bool COL>
__device__ __forceinline__ void prefetch_tile(const MPInst<T>& I, int tile, T* pre, unsigned long long* mb) {
  constexpr int TILE = Cfg<T>::TILE;
  if constexpr (COL) {
    constexpr int LOGL = Split<M>::LN2, lN1 = Split<M>::LN1;
    using G = Line<T, NT, LOGL, false, Cfg<T>::NW>;
    constexpr int LOGC = G::LOGC;
    constexpr int L = 1 << LOGL, C = 1 << LOGC;
    const T* src = I.u + (tile << LOGC);
    for (int i = G::tid(); i < L; i += NT)
      bulk_g2s(pre + i * C, src + ((size_t)i << lN1), C * (unsigned)sizeof(T), mb);
  } else {
    constexpr int CHUNK = 4096 / (int)sizeof(T);   // 4 KiB per copy
    constexpr int LOGL = Split<M>::LN1;
    using G = Line<T, NT, LOGL, true, Cfg<T>::NW>;
    constexpr int LOGC = G::LOGC;
    const T* src = I.u + ((size_t)tile << (LOGL + LOGC));
    for (int c = G::tid(); c < TILE / CHUNK; c += NT)
      bulk_g2s(pre + c * CHUNK, src + c * CHUNK, CHUNK * (unsigned)sizeof(T), mb);
  }
}

// Bounded wait on the prefetch mbarrier; false (error word set) after `limit` polls.
// The copy in flight is then still waited for (bounded by kSpinLimit polls) so that
// no copy lands in shared memory after the CTA has left.
__device__ __forceinline__ bool wait_prefetch(unsigned long long* mb, unsigned parity, int* err, long long limit) {
  long long spins = 0;
  while (!mbar_try_wait(mb, parity)) {
    if (++spins > limit) {
      atomicCAS(err, 0, LSP_ERR_TIMEOUT);
      // keep waiting (bounded again) so that no copy is in flight when the CTA leaves
      for (long long k = 0; k < kSpinLimit && !mbar_try_wait(mb, parity); ++k) __nanosleep(64);
      return false;
    }
  }
  return true;
}

// One sweep inside the persistent kernel for this thread's worker: every
// tile of the worker, the copy of the next tile in flight while the current
// one is transformed.  Returns false (uniformly per worker) if a bounded wait
// expired.
template <typename T, int NT, int M, bool COL>
__device__ __forceinline__ bool persistent_sweep(const MPParams<T>& P, T* smem, Tw<T> tw,
                                                 unsigned long long* mb, unsigned& parity, int* fail) {
  using SL = SmemLayout<T, M>;
  using G = Line<T, NT, COL ? Split<M>::LN2 : Split<M>::LN1, !COL, Cfg<T>::NW>;
  constexpr int NW = Cfg<T>::NW;
  constexpr unsigned TILE_BYTES = Cfg<T>::TILE * (unsigned)sizeof(T);
  const int w = NW == 1 ? 0 : (int)(threadIdx.x / NT);
  T* sm = smem + SL::work(w);
  T* pre = smem + SL::pre(w);
  const int2* map = COL ? P.colmap : P.rowmap;
  const int total = COL ? P.total_col : P.total_row;
  const int stride = (int)gridDim.x * NW;
  int t = (int)blockIdx.x * NW + w;
  if (t >= total) return true;
  int i, l;
  tile_of<T>(map, t, i, l);
  if (G::tid() == 0) mbar_arrive_expect_tx(mb, TILE_BYTES);
  G::sync();
  prefetch_tile<T, NT, M, COL>(P.inst[i], l, pre, mb);
  for (; t < total; t += stride) {
    if (!wait_prefetch(mb, parity, P.err, P.spin_limit)) fail[w] = 1;
    G::sync();
    if (fail[w]) return false;
    parity ^= 1u;
    int in = 0, ln = -1;
    if (t + stride < total) tile_of<T>(map, t + stride, in, ln);
    if (G::tid() == 0 && ln >= 0) mbar_arrive_expect_tx(mb, TILE_BYTES);
    if constexpr (COL) col_pass<T, NT, M, kMid, kFromPre>(P.inst[i], l, sm, pre, tw, &P.inst[in], ln, mb);
    else row_pass<T, NT, M, kRow, kFromPre>(P.inst[i], l, sm, pre, tw, &P.inst[in], ln, mb);
    i = in;
    l = ln;
  }
  return true;
}

// Sweeps 1..2N-1 of N steps, after a head sweep: row, mid, row, ..., mid, row;
// a bounded grid barrier separates consecutive sweeps.  A worker whose wait
// expired skips to the barrier, where the error word stops every CTA.
template <typename T, int NT, int M>
__global__ void __launch_bounds__(NT * Cfg<T>::NW, Cfg<T>::MINB) mp_persistent(const __grid_constant__ MPParams<T> P) {
  using SL = SmemLayout<T, M>;
  constexpr int NW = Cfg<T>::NW;
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ __align__(8) unsigned long long mb[NW];
  __shared__ int fail[NW];
  T* smem = reinterpret_cast<T*>(smraw);
  const MPInst<T>& I = P.inst[0];
  Tw<T> twr{I.twr, I.twl, I.twf}, twc{I.twc, I.twl, I.twf};
  constexpr int CT = NT * NW;
  if constexpr (SL::tw_in_smem) {
    for (int k = threadIdx.x; k < RowLine<T, M>::TW_ENTRIES; k += CT) smem[SL::twr + k] = I.twr[k];
    for (int k = threadIdx.x; k < ColLine<T, M>::TW_ENTRIES; k += CT) smem[SL::twc + k] = I.twc[k];
    for (int k = threadIdx.x; k < (1 << Split<M>::LN1); k += CT) smem[SL::twl + k] = I.twl[k];
    for (int k = threadIdx.x; k < (1 << Split<M>::LN2); k += CT) smem[SL::twf + k] = I.twf[k];
    twr = Tw<T>{smem + SL::twr, smem + SL::twl, smem + SL::twf};
    twc = Tw<T>{smem + SL::twc, smem + SL::twl, smem + SL::twf};
  }
  if (threadIdx.x < NW) {
    mbar_init(&mb[threadIdx.x], 1);
    fail[threadIdx.x] = 0;
  }
  __syncthreads();
  const int w = NW == 1 ? 0 : (int)(threadIdx.x / NT);
  unsigned target = 0, parity = 0;
  for (long long step = 0; step < P.nsteps; ++step) {
    persistent_sweep<T, NT, M, false>(P, smem, twr, &mb[w], parity, fail);
    if (step + 1 == P.nsteps) break;
    if (!grid_barrier(P.bar, target, P.err, P.spin_limit)) return;
    persistent_sweep<T, NT, M, true>(P, smem, twc, &mb[w], parity, fail);
    if (!grid_barrier(P.bar, target, P.err, P.spin_limit)) return;
  }
}

// One sweep of kind KIND per launch (head and tail sweeps, spectral output),
// reading the tiles and the twiddle tables from global memory.
template <typename T, int NT, int M, int KIND>
__global__ void __launch_bounds__(NT * Cfg<T>::NW, Cfg<T>::MINB) mp_sweep(const __grid_constant__ MPParams<T> P) {
  constexpr int NW = Cfg<T>::NW;
  extern __shared__ __align__(128) unsigned char smraw[];
  const int w = NW == 1 ? 0 : (int)(threadIdx.x / NT);
  T* sm = reinterpret_cast<T*>(smraw) + w * Cfg<T>::TILE;
  constexpr bool col = KIND != kRow && KIND != kRowFwd;
  const int total = col ? P.total_col : P.total_row;
  for (int t = (int)blockIdx.x * NW + w; t < total; t += (int)gridDim.x * NW) {
    int i, l;
    tile_of<T>(col ? P.colmap : P.rowmap, t, i, l);
    const MPInst<T>& I = P.inst[i];
    if constexpr (col) col_pass<T, NT, M, KIND, kFromGlobal>(I, l, sm, nullptr, Tw<T>{I.twc, I.twl, I.twf});
    else row_pass<T, NT, M, KIND, kFromGlobal>(I, l, sm, nullptr, Tw<T>{I.twr, I.twl, I.twf});
  }
}

// Kernel entry points of one lattice size.
struct MPKernels {
  const void* persistent = nullptr;
  const void* sweep[6] = {};      // indexed by PassKind
  size_t persistent_smem = 0;
};

template <typename T, int M> MPKernels mp_kernels_for() {
  constexpr int NT = Cfg<T>::NT;
  MPKernels k;
  k.persistent = (const void*)mp_persistent<T, NT, M>;
  k.persistent_smem = SmemLayout<T, M>::bytes;
  k.sweep[kHead] = (const void*)mp_sweep<T, NT, M, kHead>;
  k.sweep[kTail] = (const void*)mp_sweep<T, NT, M, kTail>;
  k.sweep[kColFwd] = (const void*)mp_sweep<T, NT, M, kColFwd>;
  k.sweep[kRowFwd] = (const void*)mp_sweep<T, NT, M, kRowFwd>;
  return k;
}

// Defined by the per-size translation units; false if m is not theirs.
bool mp_kernels_c64_lo(int m, MPKernels* k);
bool mp_kernels_c64_hi(int m, MPKernels* k);
bool mp_kernels_c128_lo(int m, MPKernels* k);
bool mp_kernels_c128_hi(int m, MPKernels* k);

}  // namespace lsp
