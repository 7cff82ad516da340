// Four-sweep Strang step: every sweep is one launch over tiles of 4096 points,
// lines of one axis per tile.
//
// Two lattice families use it.  In both, a 2^(M1 + M2)-point array is viewed as
// 2^M1 rows of 2^M2 contiguous points; the strided axis (2^M1 points, stride
// 2^M2) is split four-step style, 2^M1 = A B with A = 2^ceil(M1/2):
// index a + A b on the way in, g + B e on the way out, and
//   W_{2^M1}^{(a + A b)(g + B e)} = W_{2^M1}^{a g} W_A^{a e} W_B^{b g}.
//
// Rank-2 lattice Lambda(Z, (n1, n2)) in canonical form, n1 = 2^M1, n2 = 2^M2
// (Def. 1; Sec. 2.5: Algorithm 1 with the 2-D DFT of Thm 1(iii), which has
// no twiddle between the axes).  Points kappa = kappa1 n2 + kappa2, bins
// chi = xi1 n2 + xi2.  One Strang step is
//   rows : IDFT_n2 . P . DFT_n2            (P_half at the ends of a run)
//   A    : DFT_B over b, then W_n1^{a g}   (lines of stride A n2)
//   B    : DFT_A . K . IDFT_A over a       (lines of stride n2)
//   A^-1 : conj W_n1^{a g}, then IDFT_B
// with K in sweep B's native order: position (e + A g) n2 + xi2 holds bin
// (g + B e) n2 + xi2.
//
// Rank-1 lattice with n = N1 N2, N1 = 2^M2 (rows), N2 = 2^M1 (columns), for n
// too large for the two-sweep kernels (Sec. 2.2, eq. Fnx as a three-stage
// four-step FFT): k = k1 + N1 (a + A b), xi = (g + B e) + N2 xi1,
//   W_n^{k xi} = W_N2^{(a + A b)(g + B e)} W_n^{k1 (g + B e)} W_N1^{k1 xi1}.
// One Strang step is
//   X    : conj W_N2^{a g}, IDFT_B, 1/n, P, DFT_B, W_N2^{a g}   (lines of stride A N1)
//   Y    : DFT_A over a, then W_n^{k1 xi2}                      (lines of stride N1)
//   Z    : DFT_N1 . K . IDFT_N1 over k1                          (rows, contiguous)
//   Y^-1 : conj W_n^{k1 xi2}, IDFT_A
// with K in sweep Z's native order: position xi1 + N1 (e + A g) holds bin
// (g + B e) + N2 xi1.  W_n^{k1 xi2} comes from two tables, W_N1^{c >> M1} times
// W_n^{c mod N2} for c = k1 xi2 mod n.
//
// Column tiles hold TILE / L adjacent columns of lines of L points (256-byte or
// longer runs); each CTA walks its tiles, loading each tile straight into
// registers, and several CTAs share an SM so that one's loads overlap another's
// transforms.
#pragma once

#include "lsp_tile.cuh"

namespace lsp {

template <typename T> struct S4Inst {
  using R = decltype(T{}.x);
  T* u;
  const T* Ph;
  const T* Pf;
  const T* K;
  const T* tw_rows;   // per-pass twiddles, lines of 2^M2 points
  const T* tw_a;      // ... of A points
  const T* tw_b;      // ... of B points
  const T* tw_col;    // W_{2^M1}^k, k < 2^M1
  const T* tw_bl;     // rank-1: W_N1^k, k < N1 (coarse factor of W_n^{k1 xi2})
  const T* tw_bf;     // rank-1: W_n^k, k < N2 (fine factor)
  double2* spec;      // spectral output (chi order)
  int* err;           // sticky device error word
  const uint8_t* kidx;  // K sweeps: ||h||^2 per native position (null: read K)
  const T* klut;        // K per value of ||h||^2, nlut entries (<= 256)
  int nlut;
  R inv_n;
};

#ifndef LSP_S4_MINB
#define LSP_S4_MINB 4
#endif
#ifndef LSP_S4_MINB_2T
#define LSP_S4_MINB_2T 2
#endif
#ifndef LSP_S4_MINB_C128
#define LSP_S4_MINB_C128 1
#endif
// 256 threads of 16 points each per CTA, at least MINB CTAs per SM (register
// cap), MINB_2T for the sweeps that run two transforms.  Measured on the
// 2^14 x 2^12 lattice (complex64): two-transform sweeps at two CTAs per SM
// and the others at four beat one 512-thread CTA per SM (with or without
// bulk-copy staging of the next tile) and three CTAs per SM for every sweep.
template <typename T> struct S4Cfg;
template <> struct S4Cfg<float2> {
  static constexpr int NT = 256, TILE = 16 * NT, MINB = LSP_S4_MINB, MINB_2T = LSP_S4_MINB_2T;
};
template <> struct S4Cfg<double2> {
  static constexpr int NT = 256, TILE = 16 * NT, MINB = LSP_S4_MINB_C128, MINB_2T = LSP_S4_MINB_C128;
};

enum S4Kind {
  // rank-2
  kR2Head = 0, kR2Mid, kR2Tail, kR2RowFwd, kR2A, kR2AInv, kR2B, kR2BFwd,
  // rank-1, four sweeps
  kXHead, kXMid, kXTail, kXFwd, kY, kYInv, kZ, kZFwd,
  kS4Kinds
};

// What one sweep kind does, in order: [conj twiddle, IDFT] [1/n, P] [DFT] [twiddle | K, IDFT | spectral out].
template <int KIND> struct S4Ops {
  static constexpr bool ROW = KIND <= kR2RowFwd || KIND == kZ || KIND == kZFwd;
  static constexpr bool SWEEP_A = (KIND >= kR2A && KIND <= kR2AInv) || (KIND >= kXHead && KIND <= kXFwd);
  static constexpr bool RANK1 = KIND >= kXHead;
  // inverse transform first (input in the forward's natural output order)
  static constexpr bool INV_IN = KIND == kR2Mid || KIND == kR2Tail || KIND == kR2AInv || KIND == kXMid ||
                                 KIND == kXTail || KIND == kYInv;
  static constexpr bool CONJ_COL = KIND == kR2AInv || KIND == kXMid || KIND == kXTail;
  static constexpr bool CONJ_BIG = KIND == kYInv;
  static constexpr bool HAS_P = (KIND <= kR2Tail) || (KIND >= kXHead && KIND <= kXTail);
  static constexpr bool FULL_P = KIND == kR2Mid || KIND == kXMid;
  static constexpr bool FWD = !(KIND == kR2Tail || KIND == kR2AInv || KIND == kXTail || KIND == kYInv);
  static constexpr bool COL_TW = KIND == kR2A || KIND == kXHead || KIND == kXMid || KIND == kXFwd;
  static constexpr bool BIG_TW = KIND == kY;
  static constexpr bool KIN = KIND == kR2B || KIND == kZ;
  static constexpr bool SPEC = KIND == kR2BFwd || KIND == kZFwd;
  // result left in the forward's natural order (else in the pass-1 pattern)
  static constexpr bool NAT_OUT = FWD && !KIN && !SPEC;
  static constexpr bool TWO = (INV_IN && FWD) || KIN;
};

// Compile-time geometry of one sweep kind: which lines a tile holds and where
// element i of line b of tile t sits in the array.
template <typename T, int M1, int M2, int KIND> struct S4Geo {
  using Ops = S4Ops<KIND>;
  static constexpr int NT = S4Cfg<T>::NT, TILE = S4Cfg<T>::TILE;
  static constexpr int LA = (M1 + 1) / 2;   // log2 A
  static constexpr int LB = M1 - LA;        // log2 B
  static constexpr bool ROW = Ops::ROW, SWEEP_A = Ops::SWEEP_A;
  static constexpr int LOGL = ROW ? M2 : SWEEP_A ? LB : LA;
  using G = Line<T, NT, LOGL, ROW>;
  static constexpr int LOGC = G::LOGC;
  static_assert(ROW ? LOGC <= M1 : LOGC <= M2, "tile larger than the array");
  static constexpr int ISTRIDE = ROW ? 0 : SWEEP_A ? LA + M2 : M2;   // log2 of the stride along a line
  static constexpr int PER = ROW ? 1 : 1 << (M2 - LOGC);              // column tiles per outer index
  static constexpr int NTILES = ROW ? (1 << M1) >> LOGC : PER << (SWEEP_A ? LA : LB);
  // first element of tile t; outer = a (sweep A / X) or g (sweep B / Y); c0 = first column
  static __device__ __forceinline__ size_t base(int t, int& outer, int& c0) {
    if constexpr (ROW) {
      outer = 0;
      c0 = 0;
      return (size_t)t << (LOGC + M2);
    } else {
      outer = t / PER;
      c0 = (t % PER) << LOGC;
      return (SWEEP_A ? ((size_t)outer << M2) : ((size_t)outer << (LA + M2))) + c0;
    }
  }
  static __device__ __forceinline__ size_t off(int b, int i) {
    return ROW ? ((size_t)b << M2) + i : (size_t)b + ((size_t)i << ISTRIDE);
  }
};

// W_n^{k1 xi2} for the rank-1 Y sweeps, n = 2^(M1 + M2), from the coarse and fine tables.
template <typename T, int M1, int M2>
__device__ __forceinline__ T big_twiddle(const S4Inst<T>& I, unsigned k1, unsigned xi2) {
  const unsigned c = (k1 * xi2) & ((1u << (M1 + M2)) - 1u);
  return twprod(__ldg(I.tw_bl + (c >> M1)), __ldg(I.tw_bf + (c & ((1u << M1) - 1u))));
}

// K value of byte index k from the per-norm table (shared memory, or global in batches).
template <typename T, bool SMEM> __device__ __forceinline__ T kval(const T* lut, unsigned k) {
  if constexpr (SMEM) return lut[k];
  else return __ldg(lut + k);
}

// One tile of one sweep.  KIDX (K sweeps only): K comes from lut[kidx[i]] (one byte per
// point) instead of the K table.
template <typename T, int M1, int M2, int KIND, bool KIDX, bool LUT_SMEM>
__device__ __forceinline__ void sweep4_tile(const S4Inst<T>& I, int t, T* sm, const T* lut) {
  using Ops = S4Ops<KIND>;
  using Geo = S4Geo<T, M1, M2, KIND>;
  using G = typename Geo::G;
  constexpr int LOGL = Geo::LOGL, LR1 = G::LOGR1, R1 = G::R1;
  constexpr int LA = Geo::LA, LB = Geo::LB;
  const T* tw_line = Geo::ROW ? I.tw_rows : Geo::SWEEP_A ? I.tw_b : I.tw_a;
  int outer, c0;
  const size_t base = Geo::base(t, outer, c0);
  T v[16];
  int bn, jn;                                          // this thread's natural-order line and butterfly
  G::template bm<4>(0, bn, jn);
  if constexpr (Ops::INV_IN) {
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = ldst(I.u + base + Geo::off(bn, jn + (q << (LOGL - 4))));
  } else {
#pragma unroll
    for (int q = 0; q < 16 / R1; ++q) {
      int b, j; G::template bm<LR1>(q, b, j);
#pragma unroll
      for (int r = 0; r < R1; ++r) v[q * R1 + r] = ldst(I.u + base + Geo::off(b, j + (r << (LOGL - LR1))));
    }
  }
  __syncthreads();                                     // previous tile's exchange reads done

  // ---- inverse half: natural order in, pass-1 pattern out ----
  if constexpr (Ops::CONJ_COL) {
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = twmulc(v[q], __ldg(I.tw_col + outer * (jn + (q << (LB - 4)))));
  }
  if constexpr (Ops::CONJ_BIG) {
#pragma unroll
    for (int q = 0; q < 16; ++q)
      v[q] = twmulc(v[q], big_twiddle<T, M1, M2>(I, c0 + bn, outer + ((jn + (q << (LA - 4))) << LB)));
  }
  if constexpr (Ops::INV_IN) G::idft(sm, tw_line, v);

  // ---- physical samples: 1/n and the potential phase ----
  if constexpr (Ops::HAS_P) {
    const T* P = Ops::FULL_P ? I.Pf : I.Ph;
#pragma unroll
    for (int q = 0; q < 16 / R1; ++q) {
      int b, j; G::template bm<LR1>(q, b, j);
#pragma unroll
      for (int r = 0; r < R1; ++r) {
        T x = v[q * R1 + r];
        if constexpr (Ops::INV_IN) x = cscale(x, I.inv_n);
        v[q * R1 + r] = apply_phase(x, ldtab(P + base + Geo::off(b, j + (r << (LOGL - LR1)))));
      }
    }
  }

  // ---- forward half: pass-1 pattern in, natural order out ----
  // K is loaded before the transform so that its latency hides behind it (measured: a
  // quarter of the four-sweep step's time at 2^22 when loaded after the transform)
  T kv[KIDX ? 1 : 16];
  unsigned kb[4];                                       // 16 byte indices, packed
  if constexpr (Ops::KIN && KIDX) {
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      unsigned x = 0;
#pragma unroll
      for (int e = 0; e < 4; ++e)
        x |= (unsigned)ldtab(I.kidx + base + Geo::off(bn, jn + ((4 * w + e) << (LOGL - 4)))) << (8 * e);
      kb[w] = x;
    }
  } else if constexpr (Ops::KIN) {
#pragma unroll
    for (int q = 0; q < 16; ++q) kv[q] = ldtab(I.K + base + Geo::off(bn, jn + (q << (LOGL - 4))));
  }
  if constexpr (Ops::FWD) G::dft(sm, tw_line, v);
  if constexpr (Ops::COL_TW) {
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = twmul(v[q], __ldg(I.tw_col + outer * (jn + (q << (LB - 4)))));
  }
  if constexpr (Ops::BIG_TW) {
#pragma unroll
    for (int q = 0; q < 16; ++q)
      v[q] = twmul(v[q], big_twiddle<T, M1, M2>(I, c0 + bn, outer + ((jn + (q << (LA - 4))) << LB)));
  }
  if constexpr (Ops::KIN) {
    if constexpr (KIDX) {
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = apply_phase(v[q], kval<T, LUT_SMEM>(lut, (kb[q >> 2] >> (8 * (q & 3))) & 255u));
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = apply_phase(v[q], kv[q]);
    }
    G::idft(sm, tw_line, v);
  }
  if constexpr (Ops::SPEC) {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const T x = cscale(v[q], I.inv_n);
      size_t chi;
      if constexpr (KIND == kR2BFwd) {
        // bin (g + B e) n2 + xi2, g = outer, e = output index, xi2 = column
        const int e = jn + (q << (LA - 4));
        chi = ((size_t)(outer + (e << LB)) << M2) + c0 + bn;
      } else {
        // row r = e + A g of the rank-1 array; bin (g + B e) + N2 xi1, xi1 = output index
        const int r = (t << Geo::LOGC) + bn;
        const int e = r & ((1 << LA) - 1), g = r >> LA;
        chi = (size_t)(g + (e << LB)) + ((size_t)(jn + (q << (LOGL - 4))) << M1);
      }
      I.spec[chi] = make_double2((double)x.x, (double)x.y);
    }
  } else if constexpr (Ops::NAT_OUT) {
#pragma unroll
    for (int q = 0; q < 16; ++q) stst(I.u + base + Geo::off(bn, jn + (q << (LOGL - 4))), v[q]);
  } else {
#pragma unroll
    for (int q = 0; q < 16 / R1; ++q) {
      int b, j; G::template bm<LR1>(q, b, j);
#pragma unroll
      for (int r = 0; r < R1; ++r) stst(I.u + base + Geo::off(b, j + (r << (LOGL - LR1))), v[q * R1 + r]);
    }
  }
}

template <typename T, int M1, int M2, int KIND, bool KIDX = false>
__global__ void __launch_bounds__(S4Cfg<T>::NT, S4Ops<KIND>::TWO ? S4Cfg<T>::MINB_2T : S4Cfg<T>::MINB)
    sweep4(const __grid_constant__ S4Inst<T> I) {
  using Geo = S4Geo<T, M1, M2, KIND>;
  extern __shared__ __align__(128) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  // K sweeps: K from a table of at most 256 values indexed by one byte per point
  __shared__ T klut[S4Ops<KIND>::KIN && KIDX ? 256 : 1];
  if constexpr (S4Ops<KIND>::KIN && KIDX) {
    for (int i = threadIdx.x; i < I.nlut; i += Geo::NT) klut[i] = I.klut[i];
    __syncthreads();
  }
  for (int t = blockIdx.x; t < Geo::NTILES; t += gridDim.x) sweep4_tile<T, M1, M2, KIND, KIDX, true>(I, t, sm, klut);
}

// Several instances of one array shape in one launch: tile t of the launch is local tile
// map[t].y of instance map[t].x (each instance with its own state, tables and step size).
template <typename T> struct S4Batch {
  const S4Inst<T>* inst;
  const int2* map;
  int ntiles;
};

template <typename T, int M1, int M2, int KIND, bool KIDX = false>
__global__ void __launch_bounds__(S4Cfg<T>::NT, S4Ops<KIND>::TWO ? S4Cfg<T>::MINB_2T : S4Cfg<T>::MINB)
    sweep4_batch(const __grid_constant__ S4Batch<T> B) {
  extern __shared__ __align__(128) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  for (int t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
    const int2 m = B.map[t];
    const S4Inst<T> I = B.inst[m.x];
    sweep4_tile<T, M1, M2, KIND, KIDX, false>(I, m.y, sm, I.klut);
  }
}

// Kernel entry points of one array shape, indexed by S4Kind, and the tile
// count of each geometry (rows, A / X, B / Y).
struct S4Kernels {
  const void* k[kS4Kinds] = {};
  const void* k_kidx = nullptr;   // the K sweep reading K through kidx
  const void* b[kS4Kinds] = {};   // rank-1 shapes up to 2^22: the multi-instance (batch) kernels
  const void* b_kidx = nullptr;
  int ntiles[3] = {};
};

template <typename T, int M1, int M2, bool RANK1> S4Kernels s4_kernels() {
  S4Kernels K;
  if constexpr (!RANK1) {
    K.k[kR2Head] = (const void*)sweep4<T, M1, M2, kR2Head>;
    K.k[kR2Mid] = (const void*)sweep4<T, M1, M2, kR2Mid>;
    K.k[kR2Tail] = (const void*)sweep4<T, M1, M2, kR2Tail>;
    K.k[kR2RowFwd] = (const void*)sweep4<T, M1, M2, kR2RowFwd>;
    K.k[kR2A] = (const void*)sweep4<T, M1, M2, kR2A>;
    K.k[kR2AInv] = (const void*)sweep4<T, M1, M2, kR2AInv>;
    K.k[kR2B] = (const void*)sweep4<T, M1, M2, kR2B>;
    K.k[kR2BFwd] = (const void*)sweep4<T, M1, M2, kR2BFwd>;
    K.k_kidx = (const void*)sweep4<T, M1, M2, kR2B, true>;
    K.ntiles[0] = S4Geo<T, M1, M2, kR2Mid>::NTILES;
    K.ntiles[1] = S4Geo<T, M1, M2, kR2A>::NTILES;
    K.ntiles[2] = S4Geo<T, M1, M2, kR2B>::NTILES;
  } else {
    K.k[kXHead] = (const void*)sweep4<T, M1, M2, kXHead>;
    K.k[kXMid] = (const void*)sweep4<T, M1, M2, kXMid>;
    K.k[kXTail] = (const void*)sweep4<T, M1, M2, kXTail>;
    K.k[kXFwd] = (const void*)sweep4<T, M1, M2, kXFwd>;
    K.k[kY] = (const void*)sweep4<T, M1, M2, kY>;
    K.k[kYInv] = (const void*)sweep4<T, M1, M2, kYInv>;
    K.k[kZ] = (const void*)sweep4<T, M1, M2, kZ>;
    K.k[kZFwd] = (const void*)sweep4<T, M1, M2, kZFwd>;
    K.k_kidx = (const void*)sweep4<T, M1, M2, kZ, true>;
    if constexpr (M1 + M2 <= 22) {   // larger instances fill the GPU one at a time
      K.b[kXHead] = (const void*)sweep4_batch<T, M1, M2, kXHead>;
      K.b[kXMid] = (const void*)sweep4_batch<T, M1, M2, kXMid>;
      K.b[kXTail] = (const void*)sweep4_batch<T, M1, M2, kXTail>;
      K.b[kY] = (const void*)sweep4_batch<T, M1, M2, kY>;
      K.b[kYInv] = (const void*)sweep4_batch<T, M1, M2, kYInv>;
      K.b[kZ] = (const void*)sweep4_batch<T, M1, M2, kZ>;
      K.b_kidx = (const void*)sweep4_batch<T, M1, M2, kZ, true>;
    }
    K.ntiles[0] = S4Geo<T, M1, M2, kZ>::NTILES;
    K.ntiles[1] = S4Geo<T, M1, M2, kXMid>::NTILES;
    K.ntiles[2] = S4Geo<T, M1, M2, kY>::NTILES;
  }
  return K;
}

// Defined by the instantiation units; false for shapes they do not hold.
bool s4_kernels_rank2(int prec, int m1, int m2, S4Kernels* k);
bool s4_kernels_rank1(int prec, int m, S4Kernels* k);

}  // namespace lsp
