// Strang step on a rank-2 lattice Lambda(Z, (n1, n2)) in canonical form with
// n1 = 2^m1, n2 = 2^m2 (Def. 1; Sec. 2.5: Algorithm 1 with the 2-D DFT).
//
// Points are ordered kappa = kappa1 n2 + kappa2 and bins chi = xi1 n2 + xi2
// (lexicographic, Sec. 2.5); the lattice DFT is the n1 x n2 2-D DFT of
// Thm 1(iii), with no twiddle between the two axes.  Rows (kappa2, contiguous,
// length n2) fit a tile; the kappa1 axis is split four-step style with
// n1 = A B, A = 2^ceil(m1/2):  kappa1 = a + A b,  xi1 = g + B e,
//   W_n1^{kappa1 xi1} = W_n1^{a g} W_A^{a e} W_B^{b g}.
// One Strang step is four sweeps over the state:
//   rows : IDFT_n2 . P . DFT_n2            (P_half at the ends of a run)
//   A    : DFT_B over b, then W_n1^{a g}   (lines of stride A n2)
//   B    : DFT_A . K . IDFT_A over a       (lines of stride n2)
//   A^-1 : conj W_n1^{a g}, then IDFT_B
// K is stored in the native order of sweep B: position (e + A g) n2 + xi2
// holds bin (g + B e) n2 + xi2.  Column tiles hold 2^13 / B (c64) adjacent
// kappa2 columns, so every global access is a run of >= 256 bytes.
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "lsp_tile.cuh"

namespace lsp {

template <typename T> struct R2Inst {
  using R = decltype(T{}.x);
  T* u;
  const T* Ph;
  const T* Pf;
  const T* K;
  const T* tw_rows;   // per-pass twiddles, lines of length n2
  const T* tw_a;      // ... of length LA
  const T* tw_b;      // ... of length LB
  const T* tw_n1;     // W_n1^k, k < n1
  double2* spec;
  R inv_n;
};

template <typename T> struct R2Cfg;
template <> struct R2Cfg<float2> { static constexpr int NT = 512, TILE = 8192; };
template <> struct R2Cfg<double2> { static constexpr int NT = 256, TILE = 4096; };

template <int M1, int M2> struct R2Geo {
  static constexpr int LA = (M1 + 1) / 2;   // log2 A
  static constexpr int LB = M1 - LA;        // log2 B
};

enum R2Kind { kR2Head = 0, kR2Mid = 1, kR2Tail = 2, kR2RowFwd = 3, kR2A = 4, kR2AInv = 5, kR2B = 6, kR2BFwd = 7 };

template <typename T> __device__ __forceinline__ T g_ld(const T* p) { return __ldcg(p); }
template <typename T> __device__ __forceinline__ void g_st(T* p, T v) { __stcg(p, v); }

// Rows: contiguous lines kappa2 of length n2; IDFT . P . DFT (head: P . DFT,
// tail: IDFT . P, row-forward: DFT only).
template <typename T, int M1, int M2, int KIND>
__global__ void __launch_bounds__(R2Cfg<T>::NT) r2_rows(const __grid_constant__ R2Inst<T> I) {
  constexpr int NT = R2Cfg<T>::NT;
  using G = Line<T, NT, M2, true>;
  constexpr int LR1 = G::LOGR1, R1 = G::R1;
  constexpr bool inv = KIND == kR2Mid || KIND == kR2Tail;
  constexpr bool fwd = KIND != kR2Tail;
  extern __shared__ __align__(128) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int ntiles = (1 << M1) >> G::LOGC;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int r0 = tile << G::LOGC;
    T v[16];
    if constexpr (inv) {
      int b, j; G::template bm<4>(0, b, j);
#pragma unroll
      for (int t = 0; t < 16; ++t) v[t] = g_ld(I.u + (((r0 + b) << M2) + j + (t << (M2 - 4))));
      G::idft(sm, I.tw_rows, v);
    } else {
#pragma unroll
      for (int q = 0; q < 16 / R1; ++q) {
        int b, j; G::template bm<LR1>(q, b, j);
#pragma unroll
        for (int r = 0; r < R1; ++r) v[q * R1 + r] = g_ld(I.u + (((r0 + b) << M2) + j + (r << (M2 - LR1))));
      }
    }
    if constexpr (KIND != kR2RowFwd) {
      const T* P = KIND == kR2Mid ? I.Pf : I.Ph;
#pragma unroll
      for (int q = 0; q < 16 / R1; ++q) {
        int b, j; G::template bm<LR1>(q, b, j);
#pragma unroll
        for (int r = 0; r < R1; ++r) {
          T x = v[q * R1 + r];
          if constexpr (inv) x = cscale(x, I.inv_n);
          v[q * R1 + r] = apply_phase(x, __ldcs(P + (((r0 + b) << M2) + j + (r << (M2 - LR1)))));
        }
      }
    }
    if constexpr (fwd) {
      G::dft(sm, I.tw_rows, v);
      int b, j; G::template bm<4>(0, b, j);
#pragma unroll
      for (int t = 0; t < 16; ++t) g_st(I.u + (((r0 + b) << M2) + j + (t << (M2 - 4))), v[t]);
    } else {
#pragma unroll
      for (int q = 0; q < 16 / R1; ++q) {
        int b, j; G::template bm<LR1>(q, b, j);
#pragma unroll
        for (int r = 0; r < R1; ++r) g_st(I.u + (((r0 + b) << M2) + j + (r << (M2 - LR1))), v[q * R1 + r]);
      }
    }
    __syncthreads();
  }
}

// Pass A (forward or inverse): lines (a, kappa2), elements b at stride LA n2.
template <typename T, int M1, int M2, int KIND>
__global__ void __launch_bounds__(R2Cfg<T>::NT) r2_colA(const __grid_constant__ R2Inst<T> I) {
  constexpr int NT = R2Cfg<T>::NT;
  constexpr int LA = R2Geo<M1, M2>::LA, LB = R2Geo<M1, M2>::LB;
  using G = Line<T, NT, LB, false>;
  static_assert(G::LOGC <= M2, "tile wider than a row");
  constexpr int LR1 = G::LOGR1, R1 = G::R1;
  constexpr int STRIDE = LA + M2;                       // log2 of the element stride
  extern __shared__ __align__(128) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  constexpr int per_a = 1 << (M2 - G::LOGC);            // tiles per a
  const int ntiles = per_a << LA;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int a = tile / per_a;
    const int c0 = (tile % per_a) << G::LOGC;
    const size_t base = ((size_t)a << M2) + c0;
    T v[16];
    if constexpr (KIND == kR2A) {
      // DFT over b (pass-1 pattern), then W_n1^{a g} on the outputs g = j + t LB/16
#pragma unroll
      for (int q = 0; q < 16 / R1; ++q) {
        int b, j; G::template bm<LR1>(q, b, j);
#pragma unroll
        for (int r = 0; r < R1; ++r) v[q * R1 + r] = g_ld(I.u + base + b + ((size_t)(j + (r << (LB - LR1))) << STRIDE));
      }
      G::dft(sm, I.tw_b, v);
      int b, j; G::template bm<4>(0, b, j);
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const int g = j + (t << (LB - 4));
        g_st(I.u + base + b + ((size_t)g << STRIDE), cmul(v[t], __ldg(I.tw_n1 + a * g)));
      }
    } else {
      int b, j; G::template bm<4>(0, b, j);
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const int g = j + (t << (LB - 4));
        v[t] = cmulc(g_ld(I.u + base + b + ((size_t)g << STRIDE)), __ldg(I.tw_n1 + a * g));
      }
      G::idft(sm, I.tw_b, v);
#pragma unroll
      for (int q = 0; q < 16 / R1; ++q) {
        int bb, jj; G::template bm<LR1>(q, bb, jj);
#pragma unroll
        for (int r = 0; r < R1; ++r)
          g_st(I.u + base + bb + ((size_t)(jj + (r << (LB - LR1))) << STRIDE), v[q * R1 + r]);
      }
    }
    __syncthreads();
  }
}

// Pass B: lines (g, kappa2), elements a at stride n2: DFT . K . IDFT (or DFT and
// spectral output in chi order).
template <typename T, int M1, int M2, int KIND>
__global__ void __launch_bounds__(R2Cfg<T>::NT) r2_colB(const __grid_constant__ R2Inst<T> I) {
  constexpr int NT = R2Cfg<T>::NT;
  constexpr int LA = R2Geo<M1, M2>::LA, LB = R2Geo<M1, M2>::LB;
  using G = Line<T, NT, LA, false>;
  static_assert(G::LOGC <= M2, "tile wider than a row");
  constexpr int LR1 = G::LOGR1, R1 = G::R1;
  extern __shared__ __align__(128) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  constexpr int per_g = 1 << (M2 - G::LOGC);
  const int ntiles = per_g << LB;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int g = tile / per_g;
    const int c0 = (tile % per_g) << G::LOGC;
    const size_t base = ((size_t)g << (LA + M2)) + c0;  // element a of line (g, c) at base + c + a n2
    T v[16];
#pragma unroll
    for (int q = 0; q < 16 / R1; ++q) {
      int b, j; G::template bm<LR1>(q, b, j);
#pragma unroll
      for (int r = 0; r < R1; ++r) v[q * R1 + r] = g_ld(I.u + base + b + ((size_t)(j + (r << (LA - LR1))) << M2));
    }
    G::dft(sm, I.tw_a, v);
    int b, j; G::template bm<4>(0, b, j);
    if constexpr (KIND == kR2BFwd) {
      // bin chi = (g + LB e) n2 + xi2, coefficient = DFT / n
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const int e = j + (t << (LA - 4));
        T x = cscale(v[t], I.inv_n);
        I.spec[((size_t)(g + (e << LB)) << M2) + c0 + b] = make_double2((double)x.x, (double)x.y);
      }
    } else {
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const int e = j + (t << (LA - 4));
        v[t] = apply_phase(v[t], __ldcs(I.K + base + b + ((size_t)e << M2)));
      }
      G::idft(sm, I.tw_a, v);
#pragma unroll
      for (int q = 0; q < 16 / R1; ++q) {
        int bb, jj; G::template bm<LR1>(q, bb, jj);
#pragma unroll
        for (int r = 0; r < R1; ++r)
          g_st(I.u + base + bb + ((size_t)(jj + (r << (LA - LR1))) << M2), v[q * R1 + r]);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct R2Kernels {
  const void* k[8] = {};
};

template <typename T, int M1, int M2> static R2Kernels r2_kernels() {
  R2Kernels K;
  K.k[kR2Head] = (const void*)r2_rows<T, M1, M2, kR2Head>;
  K.k[kR2Mid] = (const void*)r2_rows<T, M1, M2, kR2Mid>;
  K.k[kR2Tail] = (const void*)r2_rows<T, M1, M2, kR2Tail>;
  K.k[kR2RowFwd] = (const void*)r2_rows<T, M1, M2, kR2RowFwd>;
  K.k[kR2A] = (const void*)r2_colA<T, M1, M2, kR2A>;
  K.k[kR2AInv] = (const void*)r2_colA<T, M1, M2, kR2AInv>;
  K.k[kR2B] = (const void*)r2_colB<T, M1, M2, kR2B>;
  K.k[kR2BFwd] = (const void*)r2_colB<T, M1, M2, kR2BFwd>;
  return K;
}

// Supported lattice shapes (n1, n2) = (2^m1, 2^m2).
template <typename T> static bool r2_lookup(int m1, int m2, R2Kernels* K) {
  if (m1 == 14 && m2 == 12) { *K = r2_kernels<T, 14, 12>(); return true; }
  if (m1 == 12 && m2 == 10) { *K = r2_kernels<T, 12, 10>(); return true; }
  if (m1 == 11 && m2 == 9) { *K = r2_kernels<T, 11, 9>(); return true; }
  if (m1 == 10 && m2 == 8) { *K = r2_kernels<T, 10, 8>(); return true; }
  return false;
}

bool r2_supports(int prec, int m1, int m2) {
  R2Kernels K;
  return prec == LSP_C64 ? r2_lookup<float2>(m1, m2, &K) : r2_lookup<double2>(m1, m2, &K);
}

template <typename T> static R2Inst<T> r2_inst(lsp_plan p, void* state) {
  R2Inst<T> I{};
  I.u = (T*)state;
  I.Ph = (const T*)p->Ph;
  I.Pf = (const T*)p->Pf;
  I.K = (const T*)p->K;
  const T* tw = (const T*)p->tw_pass;
  I.tw_rows = tw;
  I.tw_a = tw + p->twr_entries;
  I.tw_b = tw + p->twr_entries + p->twa_entries;
  I.tw_n1 = (const T*)p->tw_line;
  I.spec = (double2*)p->stage;
  I.inv_n = (decltype(I.inv_n))(1.0 / (double)p->ntot);
  return I;
}

// Grid of one sweep kernel: as many CTAs as fit on the device at once (at most
// one per tile), computed once per (device, kernel).
static int r2_grid(const void* fn, int nt, size_t smem, int* grid) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> cache;
  int dev = 0;
  LSP_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find({dev, fn});
  if (it != cache.end()) { *grid = it->second; return LSP_OK; }
  int per_sm = 0, sms = 0;
  LSP_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  LSP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nt, smem));
  LSP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (per_sm < 1) return LSP_ERR_UNSUPPORTED;
  *grid = per_sm * sms;
  cache[{dev, fn}] = *grid;
  return LSP_OK;
}

template <typename T> static int r2_launch(const void* fn, const R2Inst<T>& I, int ntiles, cudaStream_t s) {
  constexpr int NT = R2Cfg<T>::NT;
  const size_t smem = (size_t)R2Cfg<T>::TILE * sizeof(T);
  int grid = 0;
  int rc = r2_grid(fn, NT, smem, &grid);
  if (rc) return rc;
  grid = std::max(1, std::min(ntiles, grid));
  void* args[] = {(void*)&I};
  LSP_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(NT), args, smem, s));
  return LSP_OK;
}

template <typename T> static int r2_steps_impl(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s) {
  R2Kernels K;
  const int m1 = p->logN1, m2 = p->logN2;
  if (!r2_lookup<T>(m1, m2, &K)) return LSP_ERR_UNSUPPORTED;
  R2Inst<T> I = r2_inst<T>(p, state);
  const int la = (m1 + 1) / 2, lb = m1 - la;
  const int logTile = R2Cfg<T>::TILE == 8192 ? 13 : 12;
  const int rows_tiles = (1 << m1) >> (logTile - m2);
  const int a_tiles = (1 << (m2 - (logTile - lb))) << la;
  const int b_tiles = (1 << (m2 - (logTile - la))) << lb;
  int rc = LSP_OK;
  for (int64_t st = 0; st < nsteps && !rc; ++st) {
    rc = r2_launch<T>(K.k[st == 0 ? kR2Head : kR2Mid], I, rows_tiles, s);
    if (!rc) rc = r2_launch<T>(K.k[kR2A], I, a_tiles, s);
    if (!rc) rc = r2_launch<T>(K.k[kR2B], I, b_tiles, s);
    if (!rc) rc = r2_launch<T>(K.k[kR2AInv], I, a_tiles, s);
  }
  if (!rc) rc = r2_launch<T>(K.k[kR2Tail], I, rows_tiles, s);
  return rc;
}

template <typename T> static int r2_spectral_impl(lsp_plan p, cudaStream_t s) {
  R2Kernels K;
  const int m1 = p->logN1, m2 = p->logN2;
  if (!r2_lookup<T>(m1, m2, &K)) return LSP_ERR_UNSUPPORTED;
  LSP_CUDA_TRY(cudaMemcpyAsync(p->work, p->u, (size_t)p->ntot * sizeof(T), cudaMemcpyDeviceToDevice, s));
  R2Inst<T> I = r2_inst<T>(p, p->work);
  const int la = (m1 + 1) / 2, lb = m1 - la;
  const int logTile = R2Cfg<T>::TILE == 8192 ? 13 : 12;
  int rc = r2_launch<T>(K.k[kR2RowFwd], I, (1 << m1) >> (logTile - m2), s);
  if (!rc) rc = r2_launch<T>(K.k[kR2A], I, (1 << (m2 - (logTile - lb))) << la, s);
  if (!rc) rc = r2_launch<T>(K.k[kR2BFwd], I, (1 << (m2 - (logTile - la))) << lb, s);
  return rc;
}

int r2_steps_on(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s) {
  return p->prec == LSP_C64 ? r2_steps_impl<float2>(p, state, nsteps, s) : r2_steps_impl<double2>(p, state, nsteps, s);
}

int r2_spectral(lsp_plan p, cudaStream_t s) {
  return p->prec == LSP_C64 ? r2_spectral_impl<float2>(p, s) : r2_spectral_impl<double2>(p, s);
}

}  // namespace lsp
