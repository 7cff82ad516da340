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

#include "lsp_mp.cuh"

namespace lsp {

template <typename T> struct R2Inst {
  using R = decltype(T{}.x);
  T* u;
  const T* Ph;
  const T* Pf;
  const T* K;
  const T* tw_rows;   // per-pass twiddles, lines of length n2
  const T* tw_a;      // ... of length A
  const T* tw_b;      // ... of length B
  const T* tw_n1;     // W_n1^k, k < n1
  double2* spec;
  int* err;           // sticky device error word
  R inv_n;
};

#ifndef LSP_R2_NT_C64
#define LSP_R2_NT_C64 256
#endif
#ifndef LSP_R2_MINB
#define LSP_R2_MINB 3
#endif
#ifndef LSP_R2_MINB_2T
#define LSP_R2_MINB_2T 3
#endif
#ifndef LSP_R2_MINB_C128
#define LSP_R2_MINB_C128 1
#endif
#ifndef LSP_R2_PREFETCH
#define LSP_R2_PREFETCH 0
#endif
// NT threads of 16 elements each per CTA, at least MINB CTAs per SM (register
// cap); PRE: stage the next tile with bulk asynchronous copies instead of
// loading it directly.  Measured on the 2^14 x 2^12 lattice (complex64), three
// 256-thread CTAs per SM with direct loads beat one or two 512-thread CTAs
// per SM with or without staging: independent CTAs overlap one another's load
// and transform phases.
template <typename T> struct R2Cfg;
template <> struct R2Cfg<float2> {
  static constexpr int NT = LSP_R2_NT_C64, TILE = 16 * NT, MINB = LSP_R2_MINB, MINB_2T = LSP_R2_MINB_2T;
  static constexpr bool PRE = LSP_R2_PREFETCH != 0;
};
template <> struct R2Cfg<double2> {
  static constexpr int NT = 256, TILE = 4096, MINB = LSP_R2_MINB_C128, MINB_2T = LSP_R2_MINB_C128;
  static constexpr bool PRE = LSP_R2_PREFETCH != 0;
};

enum R2Kind { kR2Head = 0, kR2Mid = 1, kR2Tail = 2, kR2RowFwd = 3, kR2A = 4, kR2AInv = 5, kR2B = 6, kR2BFwd = 7 };

// Compile-time geometry of one sweep kind: which lines a tile holds and where
// element i of line b of tile t sits in the state.
template <typename T, int M1, int M2, int KIND> struct R2Geo {
  static constexpr int NT = R2Cfg<T>::NT, TILE = R2Cfg<T>::TILE;
  static constexpr int LA = (M1 + 1) / 2;   // log2 A
  static constexpr int LB = M1 - LA;        // log2 B
  static constexpr bool ROW = KIND <= kR2RowFwd;
  static constexpr bool SWEEP_A = KIND == kR2A || KIND == kR2AInv;
  static constexpr int LOGL = ROW ? M2 : SWEEP_A ? LB : LA;
  using G = Line<T, NT, LOGL, ROW>;
  static constexpr int LOGC = G::LOGC;
  static_assert(ROW ? LOGC <= M1 : LOGC <= M2, "tile larger than the lattice");
  // log2 of the element stride along a line
  static constexpr int ISTRIDE = ROW ? 0 : SWEEP_A ? LA + M2 : M2;
  static constexpr int PER = ROW ? 1 : 1 << (M2 - LOGC);   // column tiles per outer index
  static constexpr int NTILES = ROW ? (1 << M1) >> LOGC : PER << (SWEEP_A ? LA : LB);
  // first element of tile t (line b adds b, or b << M2 for rows)
  static __device__ __forceinline__ size_t base(int t, int& outer) {
    if constexpr (ROW) { outer = 0; return (size_t)t << (LOGC + M2); }
    else {
      outer = t / PER;
      const int c0 = (t % PER) << LOGC;
      return (SWEEP_A ? ((size_t)outer << M2) : ((size_t)outer << (LA + M2))) + c0;
    }
  }
  static __device__ __forceinline__ size_t off(int b, int i) {
    return ROW ? ((size_t)b << M2) + i : (size_t)b + ((size_t)i << ISTRIDE);
  }
  // element (b, i) in the prefetch buffer: rows in natural order, columns i-major
  static __device__ __forceinline__ int pidx(int b, int i) { return ROW ? (b << M2) + i : (i << LOGC) + b; }
};

// Bulk copies of tile t into the prefetch buffer (all threads issue a share).
template <typename T, int M1, int M2, int KIND>
__device__ __forceinline__ void r2_prefetch(const T* u, int t, T* pre, unsigned long long* mb) {
  using Geo = R2Geo<T, M1, M2, KIND>;
  int outer;
  const T* src = u + Geo::base(t, outer);
  if constexpr (Geo::ROW) {
    constexpr int CHUNK = 4096 / (int)sizeof(T);
    for (int c = threadIdx.x; c < Geo::TILE / CHUNK; c += Geo::NT)
      bulk_g2s(pre + c * CHUNK, src + c * CHUNK, CHUNK * (unsigned)sizeof(T), mb);
  } else {
    constexpr int L = 1 << Geo::LOGL, C = 1 << Geo::LOGC;
    for (int i = threadIdx.x; i < L; i += Geo::NT)
      bulk_g2s(pre + i * C, src + ((size_t)i << Geo::ISTRIDE), C * (unsigned)sizeof(T), mb);
  }
}

// One sweep.  Each CTA walks its tiles; the next tile's bulk copy is in flight
// while the current one is transformed.
//   rows (Head/Mid/Tail/RowFwd): [IDFT_n2, 1/n, P] then DFT_n2 (Tail: no DFT)
//   A   : DFT_B over b, times W_n1^{a g}      AInv: times conj W_n1^{a g}, IDFT_B
//   B   : DFT_A, K, IDFT_A                    BFwd: DFT_A, 1/n, to chi order (c128)
template <typename T, int M1, int M2, int KIND>
__global__ void __launch_bounds__(R2Cfg<T>::NT, (KIND == kR2Mid || KIND == kR2B) ? R2Cfg<T>::MINB_2T : R2Cfg<T>::MINB)
    r2_sweep(const __grid_constant__ R2Inst<T> I) {
  using Geo = R2Geo<T, M1, M2, KIND>;
  using G = typename Geo::G;
  constexpr int LOGL = Geo::LOGL, LR1 = G::LOGR1, R1 = G::R1, TILE = Geo::TILE;
  constexpr int LA = Geo::LA, LB = Geo::LB;
  constexpr unsigned TILE_BYTES = TILE * (unsigned)sizeof(T);
  // natural-order input: registers hold v[t] = x[j + t L/16] (bm<4>); else the pass-1 pattern
  constexpr bool nat_in = KIND == kR2Mid || KIND == kR2Tail || KIND == kR2AInv;
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ __align__(8) unsigned long long mb;
  __shared__ int s_fail;
  T* sm = reinterpret_cast<T*>(smraw);
  T* pre = sm + TILE;
  const T* tw_line = Geo::ROW ? I.tw_rows : Geo::SWEEP_A ? I.tw_b : I.tw_a;

  constexpr bool PRE = R2Cfg<T>::PRE;
  int t = blockIdx.x;
  if (t >= Geo::NTILES) return;
  unsigned parity = 0;
  if constexpr (PRE) {
    if (threadIdx.x == 0) {
      mbar_init(&mb, 1);
      s_fail = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_arrive_expect_tx(&mb, TILE_BYTES);
    __syncthreads();
    fence_proxy_async();
    r2_prefetch<T, M1, M2, KIND>(I.u, t, pre, &mb);
  }
  for (; t < Geo::NTILES; t += gridDim.x) {
    if constexpr (PRE) {
      if (!wait_prefetch(&mb, parity, I.err)) s_fail = 1;
      __syncthreads();
      if (s_fail) return;
      parity ^= 1u;
    }
    int outer;
    const size_t base = Geo::base(t, outer);
    // element (b, i) of the tile: from the prefetch buffer, or straight from the state
    auto ld = [&](int b, int i) { return PRE ? pre[Geo::pidx(b, i)] : ldst(I.u + base + Geo::off(b, i)); };
    T v[16];
    if constexpr (nat_in) {
      int b, j; G::template bm<4>(0, b, j);
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = ld(b, j + (q << (LOGL - 4)));
    } else {
#pragma unroll
      for (int q = 0; q < 16 / R1; ++q) {
        int b, j; G::template bm<LR1>(q, b, j);
#pragma unroll
        for (int r = 0; r < R1; ++r) v[q * R1 + r] = ld(b, j + (r << (LOGL - LR1)));
      }
    }
    if constexpr (PRE) {
      const bool more = t + (int)gridDim.x < Geo::NTILES;
      if (more && threadIdx.x == 0) mbar_arrive_expect_tx(&mb, TILE_BYTES);
      __syncthreads();                                  // prefetch buffer free: refill it
      if (more) {
        fence_proxy_async();
        r2_prefetch<T, M1, M2, KIND>(I.u, t + gridDim.x, pre, &mb);
      }
    } else {
      __syncthreads();                                  // previous tile's exchange reads done
    }

    if constexpr (Geo::ROW) {
      if constexpr (nat_in) G::idft(sm, tw_line, v);
      if constexpr (KIND != kR2RowFwd) {
        const T* P = KIND == kR2Mid ? I.Pf : I.Ph;
#pragma unroll
        for (int q = 0; q < 16 / R1; ++q) {
          int b, j; G::template bm<LR1>(q, b, j);
#pragma unroll
          for (int r = 0; r < R1; ++r) {
            T x = v[q * R1 + r];
            if constexpr (nat_in) x = cscale(x, I.inv_n);
            v[q * R1 + r] = apply_phase(x, ldtab(P + base + Geo::off(b, j + (r << (LOGL - LR1)))));
          }
        }
      }
      if constexpr (KIND != kR2Tail) {
        G::dft(sm, tw_line, v);
        int b, j; G::template bm<4>(0, b, j);
#pragma unroll
        for (int q = 0; q < 16; ++q) stst(I.u + base + Geo::off(b, j + (q << (LOGL - 4))), v[q]);
      } else {
#pragma unroll
        for (int q = 0; q < 16 / R1; ++q) {
          int b, j; G::template bm<LR1>(q, b, j);
#pragma unroll
          for (int r = 0; r < R1; ++r) stst(I.u + base + Geo::off(b, j + (r << (LOGL - LR1))), v[q * R1 + r]);
        }
      }
    } else if constexpr (KIND == kR2A) {
      G::dft(sm, tw_line, v);
      int b, j; G::template bm<4>(0, b, j);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int g = j + (q << (LB - 4));
        stst(I.u + base + Geo::off(b, g), cmul(v[q], __ldg(I.tw_n1 + outer * g)));
      }
    } else if constexpr (KIND == kR2AInv) {
      {
        int b, j; G::template bm<4>(0, b, j);
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = cmulc(v[q], __ldg(I.tw_n1 + outer * (j + (q << (LB - 4)))));
      }
      G::idft(sm, tw_line, v);
#pragma unroll
      for (int q = 0; q < 16 / R1; ++q) {
        int b, j; G::template bm<LR1>(q, b, j);
#pragma unroll
        for (int r = 0; r < R1; ++r) stst(I.u + base + Geo::off(b, j + (r << (LOGL - LR1))), v[q * R1 + r]);
      }
    } else {
      G::dft(sm, tw_line, v);
      int b, j; G::template bm<4>(0, b, j);
      if constexpr (KIND == kR2BFwd) {
        // bin chi = (g + B e) n2 + xi2 with g = outer; coefficient = DFT / n
        const int c0 = (t % Geo::PER) << Geo::LOGC;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int e = j + (q << (LA - 4));
          T x = cscale(v[q], I.inv_n);
          I.spec[((size_t)(outer + (e << LB)) << M2) + c0 + b] = make_double2((double)x.x, (double)x.y);
        }
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = apply_phase(v[q], ldtab(I.K + base + Geo::off(b, j + (q << (LA - 4)))));
        G::idft(sm, tw_line, v);
#pragma unroll
        for (int q = 0; q < 16 / R1; ++q) {
          int bb, jj; G::template bm<LR1>(q, bb, jj);
#pragma unroll
          for (int r = 0; r < R1; ++r) stst(I.u + base + Geo::off(bb, jj + (r << (LOGL - LR1))), v[q * R1 + r]);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct R2Kernels {
  const void* k[8] = {};
  int ntiles[3] = {};   // tiles of a row sweep, an A sweep, a B sweep
};

template <typename T, int M1, int M2> static R2Kernels r2_kernels() {
  R2Kernels K;
  K.k[kR2Head] = (const void*)r2_sweep<T, M1, M2, kR2Head>;
  K.k[kR2Mid] = (const void*)r2_sweep<T, M1, M2, kR2Mid>;
  K.k[kR2Tail] = (const void*)r2_sweep<T, M1, M2, kR2Tail>;
  K.k[kR2RowFwd] = (const void*)r2_sweep<T, M1, M2, kR2RowFwd>;
  K.k[kR2A] = (const void*)r2_sweep<T, M1, M2, kR2A>;
  K.k[kR2AInv] = (const void*)r2_sweep<T, M1, M2, kR2AInv>;
  K.k[kR2B] = (const void*)r2_sweep<T, M1, M2, kR2B>;
  K.k[kR2BFwd] = (const void*)r2_sweep<T, M1, M2, kR2BFwd>;
  K.ntiles[0] = R2Geo<T, M1, M2, kR2Mid>::NTILES;
  K.ntiles[1] = R2Geo<T, M1, M2, kR2A>::NTILES;
  K.ntiles[2] = R2Geo<T, M1, M2, kR2B>::NTILES;
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
  I.err = p->err;
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

// Dynamic shared memory of a sweep: exchange buffer (and prefetch buffer).
template <typename T> constexpr size_t r2_smem() {
  return (R2Cfg<T>::PRE ? 2 : 1) * (size_t)R2Cfg<T>::TILE * sizeof(T);
}

template <typename T> static int r2_launch(const void* fn, const R2Inst<T>& I, int ntiles, cudaStream_t s) {
  constexpr int NT = R2Cfg<T>::NT;
  int grid = 0;
  int rc = r2_grid(fn, NT, r2_smem<T>(), &grid);
  if (rc) return rc;
  grid = std::max(1, std::min(ntiles, grid));
  void* args[] = {(void*)&I};
  LSP_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(NT), args, r2_smem<T>(), s));
  return LSP_OK;
}

template <typename T> static int r2_steps_impl(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s) {
  R2Kernels K;
  if (!r2_lookup<T>(p->logN1, p->logN2, &K)) return LSP_ERR_UNSUPPORTED;
  const R2Inst<T> I = r2_inst<T>(p, state);
  int rc = LSP_OK;
  for (int64_t st = 0; st < nsteps && !rc; ++st) {
    rc = r2_launch<T>(K.k[st == 0 ? kR2Head : kR2Mid], I, K.ntiles[0], s);
    if (!rc) rc = r2_launch<T>(K.k[kR2A], I, K.ntiles[1], s);
    if (!rc) rc = r2_launch<T>(K.k[kR2B], I, K.ntiles[2], s);
    if (!rc) rc = r2_launch<T>(K.k[kR2AInv], I, K.ntiles[1], s);
  }
  if (!rc) rc = r2_launch<T>(K.k[kR2Tail], I, K.ntiles[0], s);
  return rc;
}

template <typename T> static int r2_spectral_impl(lsp_plan p, cudaStream_t s) {
  R2Kernels K;
  if (!r2_lookup<T>(p->logN1, p->logN2, &K)) return LSP_ERR_UNSUPPORTED;
  LSP_CUDA_TRY(cudaMemcpyAsync(p->work, p->u, (size_t)p->ntot * sizeof(T), cudaMemcpyDeviceToDevice, s));
  const R2Inst<T> I = r2_inst<T>(p, p->work);
  int rc = r2_launch<T>(K.k[kR2RowFwd], I, K.ntiles[0], s);
  if (!rc) rc = r2_launch<T>(K.k[kR2A], I, K.ntiles[1], s);
  if (!rc) rc = r2_launch<T>(K.k[kR2BFwd], I, K.ntiles[2], s);
  return rc;
}

int r2_steps_on(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s) {
  return p->prec == LSP_C64 ? r2_steps_impl<float2>(p, state, nsteps, s) : r2_steps_impl<double2>(p, state, nsteps, s);
}

int r2_spectral(lsp_plan p, cudaStream_t s) {
  return p->prec == LSP_C64 ? r2_spectral_impl<float2>(p, s) : r2_spectral_impl<double2>(p, s);
}

}  // namespace lsp
