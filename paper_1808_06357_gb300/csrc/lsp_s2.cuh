// Two-sweep Strang step for rank-1 lattices of n = 2^M points (complex64), with
// every tile brought on chip by the TMA engine.
//
// The length-n DFT of Thm 1(iii) is split four-step style (eq. Fnx) into rows of
// N1 = 4096 contiguous points and columns of N2 = n / 4096 points (stride N1):
// point k = k1 + N1 k2, bin xi = xi2 + N2 xi1,
//   W_n^{k xi} = W_n^{k1 xi2} W_N1^{k1 xi1} W_N2^{k2 xi2}.
// One Strang step (eq. StrangTDSE in physical form, Algorithm 1, adjacent
// potential half-steps merged) is two sweeps over the state:
//   column sweep (tile: C = 4096 / N2 adjacent columns k1):
//       IDFT_N2, 1/n, P, DFT_N2
//   row sweep (tile: one row xi2):  W_n^{k1 xi2}, DFT_N1, K, IDFT_N1, conj W_n^{k1 xi2}
// with K in the row sweep's native order (row xi2 of the table holds the bins
// xi2 + N2 xi1 in the order in which the row transform's threads hold them, S2Row
// below).  The four-step twiddle sits in the row sweep, where the row
// xi2 is fixed: thread j holds k1 = j + 256 r (r = 0..15), so
//   W_n^{k1 xi2} = W_n^{j xi2} W_n^{256 r xi2},
// one table value per thread and sixteen per tile (shared memory) instead of a
// scattered table lookup per point.  A call of N steps runs a head column sweep
// (P_half, forward half only), N row sweeps and N - 1 mid column sweeps in
// between, and a tail column sweep (inverse half, P_half): 2 N + 1 launches,
// replayed as a graph.
//
// Each CTA (256 threads, 16 points each, two CTAs per SM) walks its tiles with
// the next tile's copy in flight: column tiles of the state are 2-D tensor copies
// (boxes of C columns x up to 256 rows), row tiles one 32 KiB bulk copy, the K byte
// index a 4 KiB bulk copy into the same slot.  The potential-phase tables are stored
// tile by tile in the order in which the column transform's threads use them, so a
// column tile's phases are one 32 KiB bulk copy too.  A slot
// that has been read into registers serves as the tile's exchange buffer for
// the radix-16 passes, so two slots (and one potential-phase buffer for the
// column sweeps, whose copy is issued at the start of the tile and consumed
// after the inverse transform) are all the shared memory a CTA holds.  Column
// tiles with short rows (n >= 2^21) leave through that buffer too: the result is
// written there in the tile's layout and sent out by tensor stores.  Waits on the
// copies are bounded: on expiry the sticky error word is set and the CTA leaves at
// the next tile boundary with no load in flight (and its stores completed).
#pragma once

#include "lsp_async.cuh"
#include "lsp_tile.cuh"

namespace lsp {

// Per-instance descriptor in device memory.
struct S2Inst {                 // 128-byte aligned through its tensor maps
  CUtensorMap tu;            // state as {N1 (inner), N2} of 8-byte elements, box {C, BR}
  float2* u;
  const float2* Ph;          // P_half, P_full: 4096 values per column tile, in the order of the
  const float2* Pf;          // column transform's threads (16 per thread, 16-byte pairs swizzled)
  const float2* K;           // K in the row sweep's native order (when kidx is null): row xi2,
                             // position j + 256 q holds the bin of thread j's forward output q
  const uint8_t* kidx;       // ||h||^2 per row position, thread-major within a row (max < 256)
  const float2* klut;        // K per value of ||h||^2
  const float2* tw_rows;     // per-pass twiddles of the 4096-point rows
  const float2* tw_cols;     // per-pass twiddles of the N2-point columns
  const float2* tw_coarse;   // W_N1^k, k < N1 (coarse factor of W_n^a)
  const float2* tw_fine;     // W_n^k, k < N2 (fine factor)
  double2* spec;             // spectral output (chi order)
  int nlut;
  float inv_n;
  int m;                     // log2 n
};

struct S2Params {
  const S2Inst* inst;        // device array
  const int2* map;           // launch tile -> (instance, local tile); null for one instance
  int ntiles;
  int* err;
  long long spin_limit;      // polls of a copy wait before it gives up
};

enum S2Kind { kS2Head = 0, kS2Mid, kS2Tail, kS2ColFwd, kS2Row, kS2RowFwd, kS2Kinds };

constexpr int kS2NT = 256, kS2Tile = 4096, kS2LogN1 = 12;
constexpr unsigned kS2TileBytes = kS2Tile * 8u;

// Tiles of a lattice of 2^M points: 4096 points (one row, or C = 4096 / N2 columns) on 256
// threads; from 2^24 (N2 >= 4096: a 4096-point column tile would be one column, below the
// tensor copies' 16-byte rows) 8192 points (two rows, or two columns) on 512 threads, one CTA
// per SM, each row of a row tile transformed by one 256-thread half.
constexpr int kS2WideLog = 24;
template <int M> struct S2Tiles {
  static constexpr bool WIDE = M >= kS2WideLog;
  static constexpr int NT = WIDE ? 512 : 256;
  static constexpr int LOGT = WIDE ? 13 : 12;           // log2 points per tile
  static constexpr int TILE = 1 << LOGT;
  static constexpr unsigned BYTES = (unsigned)TILE * 8u;
  static constexpr int ROWS = TILE >> kS2LogN1;         // rows per row tile
  static constexpr int MINB = WIDE ? 1 : 2;             // CTAs per SM
};
__host__ __device__ __forceinline__ int s2_logtile(int m) { return m >= kS2WideLog ? 13 : 12; }

// Schedules of the kernels (the autotuner's choice per lattice size); all run two
// CTAs per SM and bring the potential-phase tile of the column sweeps in by TMA:
//   0: the line twiddles of each radix-16 pass read (through L1) where they are used
//   1: each pass' twiddles loaded before the barriers and the exchange that precede
//      the pass, so that their latency overlaps the wait
//   2: as 1, with the column lines' twiddle table copied into shared memory
template <int V> struct S2Sched;
template <> struct S2Sched<0> { static constexpr bool PRE = false, TWS_COL = false; };
template <> struct S2Sched<1> { static constexpr bool PRE = true, TWS_COL = false; };
template <> struct S2Sched<2> { static constexpr bool PRE = true, TWS_COL = true; };
static_assert(kS2NumScheds == 3, "schedule count as declared for the host");
constexpr int kS2MinBlocks = 2;
// Column tiles of lattices of at least 2^kS2TmaStoreMinLog points leave through tensor stores
// (their rows are C <= 8 elements, 64 bytes or less: as plain stores every warp instruction
// writes eight or more separate short row segments); larger tiles' rows store coalesced.
#ifndef LSP_S2_TMASTORE_MIN
#define LSP_S2_TMASTORE_MIN 21
#endif
constexpr int kS2TmaStoreMinLog = LSP_S2_TMASTORE_MIN;
template <int M> constexpr bool s2_tma_store() { return M >= kS2TmaStoreMinLog; }

template <int M, int KIND> struct S2Geo {
  static constexpr bool COL = KIND <= kS2ColFwd;
  static constexpr int LN2 = M - kS2LogN1;
  static constexpr int LOGL = COL ? LN2 : kS2LogN1;
  using T = S2Tiles<M>;
  static constexpr int NT = T::NT;
  using G = Line<float2, NT, LOGL, !COL, 1, COL ? col_swizzle(LOGL) : 0>;
  static constexpr int LOGC = G::LOGC;                  // lines per tile
  static constexpr int C = 1 << LOGC;
  static constexpr int BR = COL ? ((1 << LN2) < 256 ? (1 << LN2) : 256) : 0;   // rows per tensor box
  static constexpr bool INV_IN = KIND == kS2Mid || KIND == kS2Tail;
  static constexpr bool FWD = KIND == kS2Head || KIND == kS2Mid || KIND == kS2ColFwd;
  static constexpr bool HAS_P = KIND == kS2Head || KIND == kS2Mid || KIND == kS2Tail;
  static_assert(!COL || C >= 2, "a column tile needs at least 16-byte rows (two columns)");
};

// Shared memory of one CTA: two tile slots (+ the K byte index of a row), the
// potential-phase tile, the column twiddles (schedule 2), the K table per norm value,
// the sixteen per-tile twiddles of a row.
template <int M, int KIND, bool KIDX, int V> struct S2Smem {
  using Geo = S2Geo<M, KIND>;
  static constexpr bool TWS = Geo::COL && S2Sched<V>::TWS_COL;
  using T = typename Geo::T;
  static constexpr unsigned KIDX_BYTES = (!Geo::COL && KIDX) ? (unsigned)T::TILE : 0u;
  static constexpr unsigned SLOT = T::BYTES + KIDX_BYTES;
  static constexpr unsigned PBUF = 2 * SLOT;
  static constexpr unsigned TWT = PBUF + (Geo::HAS_P ? T::BYTES : 0u);
  static constexpr unsigned LUT = TWT + (TWS ? (unsigned)Geo::G::TW_ENTRIES * 8u : 0u);
  static constexpr unsigned TWR = LUT + ((!Geo::COL && KIDX) ? 256u * 8u : 0u);   // 2 x W_n^{256 r xi2}, r < 16, per row
  static constexpr unsigned USED = TWR + (Geo::COL ? 0u : 2u * (unsigned)T::ROWS * 16u * 8u);
  static constexpr unsigned BYTES = USED + 128u;        // room to align the base to 128 bytes (tensor copies)
};

// 4096-point row transform (radix 16, 16, 16) with one block-wide exchange per
// direction.  Butterfly j of pass s reads x[j + 256 r] and writes
// y[(j / Ns) 16 Ns + j mod Ns + Ns t] (Ns = 1, 16, 256), as the Line passes do; what
// differs is which thread runs which butterfly, and the exchange layouts.  Pass 2's
// butterfly 16 c + e writes positions 256 c + 16 t + e, which are read by pass 3's
// butterflies 16 t + e only: the pass-2 -> pass-3 exchange joins butterflies of one e.
// So warp w runs e in {2w, 2w + 1} with c (pass 2) or t (pass 3) = lane mod 16, and that
// exchange never leaves the 512 buffer positions the warp read after pass 1; __syncwarp
// orders it.  Pass 1 keeps butterfly j = thread (the tile's coalesced input and output
// pattern).  Layouts, conflict-free for every access of a warp:
//   pass 1 -> 2: y at y ^ ((y >> 4) & 15)
//   pass 2 -> 3: element (c, t, e) at 256 c + 16 (c ^ t) + (e ^ c ^ t)
// Twiddles: pass 2's W_256^{e r} from the row table's [r-1][jm] part; pass 3's
// W_4096^{(16 t + e) r} stored [r-1][e][t] (the host's row table permutes that part),
// so that a warp's 32 loads of one r are contiguous.  On CTAs of NT = 512 threads each
// 256-thread half transforms its own row, synchronised by a named barrier of its own.
template <int NT> struct S2Row {
  static constexpr int kTw3 = 15 * 16;                  // start of pass 3's table
  static __device__ __forceinline__ int lt() { return (int)(threadIdx.x & 255u); }
  static __device__ __forceinline__ void sync() {
    if constexpr (NT == 256) __syncthreads();
    else asm volatile("bar.sync %0, 256;" ::"r"(1 + (int)(threadIdx.x >> 8)) : "memory");
  }
  static __device__ __forceinline__ int e_of() { return ((lt() >> 5) << 1) | ((lt() >> 4) & 1); }
  static __device__ __forceinline__ int c_of() { return (int)(threadIdx.x & 15u); }
  // pass-3 butterfly of this thread: the forward's output t is bin xi1 = jn3() + 256 t
  static __device__ __forceinline__ int jn3() { return (c_of() << 4) | e_of(); }
  static __device__ __forceinline__ void load_tw2(const float2* __restrict__ tw, int e, float2 (&w)[15]) {
#pragma unroll
    for (int r = 1; r < 16; ++r) w[r - 1] = tw[((r - 1) << 4) + e];
  }
  static __device__ __forceinline__ void load_tw3(const float2* __restrict__ tw, int e, int c, float2 (&w)[15]) {
    const float2* tq = tw + kTw3 + (e << 4) + c;
#pragma unroll
    for (int r = 1; r < 16; ++r) w[r - 1] = tq[(r - 1) << 8];
  }
  template <int DIR> static __device__ __forceinline__ void butterfly(float2 (&v)[16]) {
    float2 o[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) o[i] = v[i];
    bfly<16, DIR>(o);
#pragma unroll
    for (int t = 0; t < 16; ++t) v[t] = o[out_at<16>(t)];
  }

  // v[r] = x[j + 256 r] (j = thread of the half)  ->  v[t] = X[jn3() + 256 t]
  static __device__ __forceinline__ void fwd(float2* sm, const float2* __restrict__ tw, float2 (&v)[16]) {
    const int j = lt(), c = c_of(), e = e_of();
    const int a2 = (c << 4) | (e ^ c), b2 = (c << 8) | a2;
    float2 w[15];
    load_tw2(tw, e, w);
    butterfly<-1>(v);
    sync();                                             // every thread has read its tile input
#pragma unroll
    for (int t = 0; t < 16; ++t) sm[(j << 4) | (t ^ (j & 15))] = v[t];
    sync();
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = sm[(r << 8) + a2];
#pragma unroll
    for (int r = 1; r < 16; ++r) v[r] = twmul(v[r], w[r - 1]);
    load_tw3(tw, e, c, w);
    butterfly<-1>(v);
    __syncwarp();
#pragma unroll
    for (int t = 0; t < 16; ++t) sm[b2 ^ (17 * t)] = v[t];
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = sm[a2 ^ (273 * r)];
#pragma unroll
    for (int r = 1; r < 16; ++r) v[r] = twmul(v[r], w[r - 1]);
    butterfly<-1>(v);
  }

  // v[t] = X[jn3() + 256 t]  ->  v[r] = unnormalised inverse DFT at x[j + 256 r]
  static __device__ __forceinline__ void inv(float2* sm, const float2* __restrict__ tw, float2 (&v)[16]) {
    const int j = lt(), c = c_of(), e = e_of();
    const int a2 = (c << 4) | (e ^ c), b2 = (c << 8) | a2;
    float2 w[15];
    load_tw3(tw, e, c, w);
    butterfly<+1>(v);
#pragma unroll
    for (int r = 1; r < 16; ++r) v[r] = twmulc(v[r], w[r - 1]);
    load_tw2(tw, e, w);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; ++r) sm[a2 ^ (273 * r)] = v[r];
    __syncwarp();
#pragma unroll
    for (int t = 0; t < 16; ++t) v[t] = sm[b2 ^ (17 * t)];
    butterfly<+1>(v);
#pragma unroll
    for (int r = 1; r < 16; ++r) v[r] = twmulc(v[r], w[r - 1]);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; ++r) sm[(r << 8) + a2] = v[r];
    sync();
#pragma unroll
    for (int t = 0; t < 16; ++t) v[t] = sm[(j << 4) | (t ^ (j & 15))];
    butterfly<+1>(v);
  }
};

// Forward / inverse line transform of a tile under schedule V.
template <typename G, int V>
__device__ __forceinline__ void s2_dft(float2* sm, const float2* tw, float2 (&v)[16]) {
  if constexpr (S2Sched<V>::PRE) G::dft_pre(sm, tw, v);
  else G::dft(sm, tw, v);
}
template <typename G, int V>
__device__ __forceinline__ void s2_idft(float2* sm, const float2* tw, float2 (&v)[16]) {
  if constexpr (S2Sched<V>::PRE) G::idft_pre(sm, tw, v);
  else G::idft(sm, tw, v);
}

// Bounded wait for phase `parity` of mbarrier b: at most `limit` non-blocking polls
// ~32 ns apart.  On expiry the error word is set and *fail raised, and the wait goes
// on (bounded again) so that the copy has landed before the CTA moves on.
__device__ __forceinline__ void s2_wait(unsigned long long* b, unsigned parity, long long limit, int* err,
                                       int* fail) {
  long long spins = 0;
  while (!mbar_test_wait(b, parity)) {
    __nanosleep(32);
    if (++spins > limit) {
      atomicCAS(err, 0, LSP_ERR_TIMEOUT);
      *(volatile int*)fail = 1;
      for (long long k = 0; k < kSpinLimit && !mbar_try_wait(b, parity); ++k) __nanosleep(64);
      return;
    }
  }
}

// The copies below overwrite shared memory whose last ordinary accesses (the previous
// tile's reads, and its exchange writes, each read back by other threads) completed
// before the CTA barrier that precedes the issue; no proxy fence is needed for that
// order (a fence here stalls the issuing warp on its own outstanding global stores, and
// every other warp with it at the tile's next barrier).
//
// Column tile t of an n = 2^m array (tensor map `map`): C = tile / N2 columns, boxes of
// min(N2, 256) rows, into dst (thread 0 only).
__device__ __forceinline__ void s2_issue_cols(const CUtensorMap* map, int m, int t, unsigned char* dst,
                                              unsigned long long* b) {
  const int ln2 = m - kS2LogN1, lt = s2_logtile(m);
  const int c = 1 << (lt - ln2);
  const int br = (1 << ln2) < 256 ? (1 << ln2) : 256;
  const int nb = (1 << ln2) / br;
  mbar_arrive_expect_tx(b, 8u << lt);
  for (int k = 0; k < nb; ++k) tma_load_2d(dst + (size_t)k * br * c * 8, map, t * c, k * br, b);
}

// Column tile t of the state from src (the tile row-major, as the loads leave it) back to
// global memory: tensor stores in thread 0's bulk group, after every thread's writes of src,
// their proxy fence and a CTA barrier.
__device__ __forceinline__ void s2_store_cols(const CUtensorMap* map, int m, int t, const unsigned char* src) {
  const int ln2 = m - kS2LogN1, lt = s2_logtile(m);
  const int c = 1 << (lt - ln2);
  const int br = (1 << ln2) < 256 ? (1 << ln2) : 256;
  const int nb = (1 << ln2) / br;
  for (int k = 0; k < nb; ++k) tma_store_2d(map, t * c, k * br, src + (size_t)k * br * c * 8);
  bulk_commit();
}

// Issue the copies of local tile t of instance I into slot `dst` (thread 0 only): a column
// tile, or a row tile (one or two rows) with its K byte index when the instance has one and
// the slot has room for it (KIDX).
template <bool COL, bool KIDX>
__device__ __forceinline__ void s2_issue_tile(const S2Inst& I, int t, unsigned char* dst, unsigned long long* b) {
  if constexpr (COL) {
    s2_issue_cols(&I.tu, I.m, t, dst, b);
  } else {
    const int lt = s2_logtile(I.m);
    const bool kx = KIDX && I.kidx != nullptr;
    mbar_arrive_expect_tx(b, (8u << lt) + (kx ? 1u << lt : 0u));
    bulk_g2s(dst, I.u + ((size_t)t << lt), 8u << lt, b);
    if (kx) bulk_g2s(dst + (8u << lt), I.kidx + ((size_t)t << lt), 1u << lt, b);
  }
}

// The potential-phase tile of column tile t: the tile's phases, contiguous in the tables'
// tile order (32 or 64 KiB).
template <int KIND>
__device__ __forceinline__ void s2_issue_p(const S2Inst& I, int t, unsigned char* dst, unsigned long long* b) {
  const int lt = s2_logtile(I.m);
  mbar_arrive_expect_tx(b, 8u << lt);
  bulk_g2s(dst, (KIND == kS2Mid ? I.Pf : I.Ph) + ((size_t)t << lt), 8u << lt, b);
}

// W_n^a (a < n) from the two-level table: W_N1^{a >> LN2} W_n^{a mod N2}.
template <int M>
__device__ __forceinline__ float2 s2_wn(const S2Inst& I, unsigned a) {
  constexpr int LN2 = M - kS2LogN1;
  return twprod(__ldg(I.tw_coarse + (a >> LN2)), __ldg(I.tw_fine + (a & ((1u << LN2) - 1u))));
}

// One column tile: lines = columns k1 = c0 + b of N2 points; slot holds the tile row-major
// (element (b, i) at i C + b), pbuf the potential-phase tile in its threads' order.
template <int M, int KIND, int V>
__device__ __forceinline__ void s2_col_tile(const S2Inst& I, int t, float2* slot, const float2* tw, float2* pbuf,
                                            unsigned long long* mbp, unsigned pparity, const S2Params& P,
                                            int* fail) {
  using Geo = S2Geo<M, KIND>;
  using G = typename Geo::G;
  constexpr int LOGL = Geo::LOGL, LOGC = Geo::LOGC, LR1 = G::LOGR1, R1 = G::R1;
  const int c0 = t << LOGC;
  float2 v[16];
  int bn, jn;
  G::template bm<4>(0, bn, jn);
  if constexpr (Geo::INV_IN) {
    // natural order (the forward transform's output): rows xi2 = jn + q L/16
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = slot[((jn + (q << (LOGL - 4))) << LOGC) + bn];
  } else {
#pragma unroll
    for (int q = 0; q < 16 / R1; ++q) {
      int b, j; G::template bm<LR1>(q, b, j);
#pragma unroll
      for (int r = 0; r < R1; ++r) v[q * R1 + r] = slot[((j + (r << (LOGL - LR1))) << LOGC) + b];
    }
  }
  // the slot becomes the exchange buffer: the transform's first barrier precedes its first write
  if constexpr (Geo::INV_IN) s2_idft<G, V>(slot, tw, v);
  if constexpr (Geo::HAS_P) {
    // this thread's 16 phases (register order) as eight 16-byte pairs, pair x at x ^ (thread mod 8)
    s2_wait(mbp, pparity, P.spin_limit, P.err, fail);
    const float4* pp = reinterpret_cast<const float4*>(pbuf) + 8 * threadIdx.x;
#pragma unroll
    for (int x = 0; x < 8; ++x) {
      const float4 pr = pp[x ^ (threadIdx.x & 7u)];
      float2 a = v[2 * x], c = v[2 * x + 1];
      if constexpr (Geo::INV_IN) { a = cscale(a, I.inv_n); c = cscale(c, I.inv_n); }
      v[2 * x] = apply_phase(a, make_float2(pr.x, pr.y));
      v[2 * x + 1] = apply_phase(c, make_float2(pr.z, pr.w));
    }
  }
  if constexpr (Geo::FWD) s2_dft<G, V>(slot, tw, v);
  if constexpr (Geo::HAS_P && s2_tma_store<M>()) {
    // the result into the phase buffer, in the tile's row-major layout, then tensor stores by
    // thread 0; the buffer is free once every thread has read its phases: after the forward
    // transform's first barrier, or (tail sweep, one-pass lines) after a barrier of its own
    if constexpr (!Geo::FWD || G::P == 1) __syncthreads();
    if constexpr (Geo::FWD) {
#pragma unroll
      for (int q = 0; q < 16; ++q) pbuf[((jn + (q << (LOGL - 4))) << LOGC) + bn] = v[q];
    } else {
#pragma unroll
      for (int q = 0; q < 16 / R1; ++q) {
        int b, j; G::template bm<LR1>(q, b, j);
#pragma unroll
        for (int r = 0; r < R1; ++r) pbuf[((j + (r << (LOGL - LR1))) << LOGC) + b] = v[q * R1 + r];
      }
    }
    fence_proxy_async_shared();
    __syncthreads();
    if (threadIdx.x == 0) s2_store_cols(&I.tu, I.m, t, reinterpret_cast<const unsigned char*>(pbuf));
  } else if constexpr (Geo::FWD) {
#pragma unroll
    for (int q = 0; q < 16; ++q) stst(I.u + (c0 + bn) + ((size_t)(jn + (q << (LOGL - 4))) << kS2LogN1), v[q]);
  } else {
#pragma unroll
    for (int q = 0; q < 16 / R1; ++q) {
      int b, j; G::template bm<LR1>(q, b, j);
#pragma unroll
      for (int r = 0; r < R1; ++r)
        stst(I.u + (c0 + b) + ((size_t)(j + (r << (LOGL - LR1))) << kS2LogN1), v[q * R1 + r]);
    }
  }
}

// One row tile: ROWS rows xi2 = t ROWS + g of 4096 contiguous points, row g transformed by
// threads 256 g .. 256 g + 255; the K byte index of the rows sits after the state in the slot,
// thread-major within each row (thread jn's 16 bytes, for its forward outputs q = 0..15,
// together).
// W_n^{256 r xi2}, r < 16, of the tile's rows into twr (16 per row; threads 0 .. 16 ROWS - 1).
template <int M>
__device__ __forceinline__ void s2_row_twr(const S2Inst& I, int t, float2* twr) {
  constexpr int ROWS = S2Tiles<M>::ROWS;
  if (threadIdx.x < 16u * ROWS) {
    const unsigned row = (unsigned)(t * ROWS) + (threadIdx.x >> 4), r = threadIdx.x & 15u;
    twr[threadIdx.x] = s2_wn<M>(I, (row * (r << (kS2LogN1 - 4))) & ((1u << M) - 1u));
  }
}

template <int M, int KIND, bool KIDX, int V>
__device__ __forceinline__ void s2_row_tile(const S2Inst& I, int t, float2* slot, const float2* tw, const float2* lut,
                                            const float2* twr) {
  using T = S2Tiles<M>;
  using R = S2Row<T::NT>;
  constexpr int LOGL = kS2LogN1;
  constexpr unsigned NMASK = (1u << M) - 1u;
  float2 v[16];
  const int g = T::ROWS == 1 ? 0 : (int)(threadIdx.x >> 8);
  const int rt = t * T::ROWS + g;                       // this half's row xi2
  float2* sl = slot + (g << LOGL);
  twr += 16 * g;
  const int jn = R::lt(), j3 = R::jn3();
  // pass-1 pattern: register r holds k1 = jn + 256 r of row rt
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = sl[jn + (r << (LOGL - 4))];
  uint4 kb = make_uint4(0, 0, 0, 0);
  float2 kv[(KIND == kS2Row && !KIDX) ? 16 : 1];
  if constexpr (KIND == kS2Row) {
    if constexpr (KIDX) {
      kb = reinterpret_cast<const uint4*>(reinterpret_cast<const unsigned char*>(slot) + T::BYTES + (g << LOGL))[jn];
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) kv[q] = ldtab(I.K + ((size_t)rt << LOGL) + jn + (q << (LOGL - 4)));
    }
  }
  // the slot becomes the exchange buffer: the transform's first barrier precedes its first write
  // four-step twiddle W_n^{k1 rt} = W_n^{j rt} W_n^{256 r rt} (twr written before the tile's barrier)
  const float2 wb = s2_wn<M>(I, ((unsigned)rt * (unsigned)jn) & NMASK);
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = twmul(twmul(v[r], twr[r]), wb);
  R::fwd(sl, tw, v);                                    // v[q] = bin xi1 = j3 + 256 q of row rt
  if constexpr (KIND == kS2RowFwd) {
    const int N2 = 1 << (M - kS2LogN1);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int xi1 = j3 + (q << (LOGL - 4));
      const float2 x = cscale(v[q], I.inv_n);
      I.spec[rt + (size_t)xi1 * N2] = make_double2((double)x.x, (double)x.y);
    }
  } else {
    if constexpr (KIDX) {
      const unsigned w[4] = {kb.x, kb.y, kb.z, kb.w};
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = apply_phase(v[q], lut[(w[q >> 2] >> (8 * (q & 3))) & 255u]);
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = apply_phase(v[q], kv[q]);
    }
    R::inv(sl, tw, v);
#pragma unroll
    for (int r = 0; r < 16; ++r) stst(I.u + ((size_t)rt << LOGL) + jn + (r << (LOGL - 4)), twmulc(twmulc(v[r], wb), twr[r]));
  }
}

template <int M, int KIND, bool KIDX, int V>
__global__ void __launch_bounds__(S2Tiles<M>::NT, S2Tiles<M>::MINB) s2_sweep(const __grid_constant__ S2Params P) {
  using Geo = S2Geo<M, KIND>;
  using SM = S2Smem<M, KIND, KIDX, V>;
  extern __shared__ __align__(128) unsigned char smdyn[];
  unsigned char* smraw = smdyn + ((128u - (smem_u32(smdyn) & 127u)) & 127u);
  __shared__ __align__(8) unsigned long long mb[3];    // slot 0, slot 1, potential-phase tile
  __shared__ int fail;
  const int G = (int)gridDim.x;
  if (threadIdx.x == 0) {
    mbar_init(&mb[0], 1);
    mbar_init(&mb[1], 1);
    mbar_init(&mb[2], 1);
    fail = 0;
    fence_mbar_init();
  }
  float2* lut = reinterpret_cast<float2*>(smraw + SM::LUT);
  // line twiddles: shared-memory copy (schedule 2, columns) or the table in global memory;
  // every instance of a launch has the same line length, hence the same table
  const float2* tw = Geo::COL ? P.inst[0].tw_cols : P.inst[0].tw_rows;
  if constexpr (SM::TWS) {
    float2* tws = reinterpret_cast<float2*>(smraw + SM::TWT);
    for (int k = threadIdx.x; k < Geo::G::TW_ENTRIES; k += Geo::NT) tws[k] = __ldg(tw + k);
    tw = tws;
  }
  auto inst_of = [&](int tt, int& local) -> const S2Inst& {
    if (P.map) { const int2 m = P.map[tt]; local = m.y; return P.inst[m.x]; }
    local = tt;
    return P.inst[0];
  };
  if constexpr (!Geo::COL && KIDX) {
    // one instance: its K table once; a batch reloads the table of each tile's instance below
    if (!P.map)
      for (int k = threadIdx.x; k < P.inst[0].nlut; k += Geo::NT) lut[k] = P.inst[0].klut[k];
  }
  __syncthreads();
  float2* twr = reinterpret_cast<float2*>(smraw + SM::TWR);   // row sweeps: per-tile twiddles, by tile parity
  constexpr int TWR_SET = 16 * Geo::T::ROWS;
  int t = (int)blockIdx.x;
  if (t >= P.ntiles) return;
  {
    int l;
    const S2Inst& I0 = inst_of(t, l);
    if (threadIdx.x == 0) s2_issue_tile<Geo::COL, KIDX>(I0, l, smraw, &mb[0]);
    if constexpr (!Geo::COL) s2_row_twr<M>(I0, l, twr);
  }
  for (int i = 0; t < P.ntiles; ++i, t += G) {
    const int s = i & 1;
    unsigned char* slot = smraw + (size_t)s * SM::SLOT;
    s2_wait(&mb[s], (unsigned)(i >> 1) & 1u, P.spin_limit, P.err, &fail);
    int l;
    const S2Inst& I = inst_of(t, l);
    if constexpr (!Geo::COL && KIDX) {
      if (P.map) {                                       // batch: this instance's K table
        __syncthreads();
        for (int k = threadIdx.x; k < I.nlut; k += Geo::NT) lut[k] = I.klut[k];
      }
    }
    __syncthreads();                                    // tile i - 1 done; the wait above ended in every thread
    if (*(volatile int*)&fail) break;                   // no copy is in flight here
    if (t + G < P.ntiles) {
      int ln;
      const S2Inst& In = inst_of(t + G, ln);
      if (threadIdx.x == 0) s2_issue_tile<Geo::COL, KIDX>(In, ln, smraw + (size_t)(s ^ 1) * SM::SLOT, &mb[s ^ 1]);
      // the next row's twiddles: the buffer of parity i + 1 was last read in tile i - 1
      if constexpr (!Geo::COL) s2_row_twr<M>(In, ln, twr + TWR_SET * (s ^ 1));
    }
    if constexpr (Geo::HAS_P) {
      if (threadIdx.x == 0) {
        if constexpr (s2_tma_store<M>()) bulk_wait_read();   // tile i - 1's stores have read the buffer
        s2_issue_p<KIND>(I, l, smraw + SM::PBUF, &mb[2]);
      }
    }
    if constexpr (Geo::COL)
      s2_col_tile<M, KIND, V>(I, l, reinterpret_cast<float2*>(slot), tw,
                              reinterpret_cast<float2*>(smraw + SM::PBUF), &mb[2], (unsigned)i & 1u, P, &fail);
    else
      s2_row_tile<M, KIND, KIDX, V>(I, l, reinterpret_cast<float2*>(slot), tw, lut, twr + TWR_SET * s);
  }
  if constexpr (Geo::HAS_P && s2_tma_store<M>()) {
    if (threadIdx.x == 0) bulk_wait_all();              // the last tile's stores, before the CTA ends
  }
}

// Kernel entry points of one lattice size and schedule.
struct S2Kernels {
  const void* k[kS2Kinds] = {};
  const void* row_kidx = nullptr;
  size_t smem[kS2Kinds] = {};
  size_t smem_row_kidx = 0;
  int ntiles = 0;                                       // tiles per sweep (both geometries)
  int nt = kS2NT;                                       // threads per CTA
};

template <int M, int V> S2Kernels s2_kernels_v() {
  S2Kernels K;
  K.k[kS2Head] = (const void*)s2_sweep<M, kS2Head, false, V>;
  K.k[kS2Mid] = (const void*)s2_sweep<M, kS2Mid, false, V>;
  K.k[kS2Tail] = (const void*)s2_sweep<M, kS2Tail, false, V>;
  K.k[kS2ColFwd] = (const void*)s2_sweep<M, kS2ColFwd, false, V>;
  K.k[kS2Row] = (const void*)s2_sweep<M, kS2Row, false, V>;
  K.k[kS2RowFwd] = (const void*)s2_sweep<M, kS2RowFwd, false, V>;
  K.row_kidx = (const void*)s2_sweep<M, kS2Row, true, V>;
  K.smem[kS2Head] = S2Smem<M, kS2Head, false, V>::BYTES;
  K.smem[kS2Mid] = S2Smem<M, kS2Mid, false, V>::BYTES;
  K.smem[kS2Tail] = S2Smem<M, kS2Tail, false, V>::BYTES;
  K.smem[kS2ColFwd] = S2Smem<M, kS2ColFwd, false, V>::BYTES;
  K.smem[kS2Row] = S2Smem<M, kS2Row, false, V>::BYTES;
  K.smem[kS2RowFwd] = S2Smem<M, kS2RowFwd, false, V>::BYTES;
  K.smem_row_kidx = S2Smem<M, kS2Row, true, V>::BYTES;
  K.ntiles = 1 << (M - S2Tiles<M>::LOGT);
  K.nt = S2Tiles<M>::NT;
  return K;
}

template <int M> bool s2_kernels_m(int v, S2Kernels* k) {
  switch (v) {
    case 0: *k = s2_kernels_v<M, 0>(); return true;
    case 1: *k = s2_kernels_v<M, 1>(); return true;
    case 2: *k = s2_kernels_v<M, 2>(); return true;
    default: return false;
  }
}

// Defined by the instantiation units (one per lattice size); false for other sizes.
bool s2_kernels_for(int m, int v, S2Kernels* k);

// ---------------------------------------------------------------------------
// Batches of instances of uneven size: one launch per sweep kind covers every tile
// of every instance with 2^16 <= n <= 2^23 points (tiles of 4096 points in all of
// them); a tile's instance fixes its geometry (column length, twiddle tables, K form,
// step size through its tables), dispatched per tile.  Schedule 1 (twiddles loaded
// ahead of the barriers), two CTAs per SM, slots sized for the K byte index.
// ---------------------------------------------------------------------------
constexpr int kS2BatchMinLog = 16, kS2BatchMaxLog = 23;
constexpr int kS2BatchSched = 1;

// Shared memory of a batch CTA: two slots (rows: with room for the K byte index), the
// potential-phase tile, two K tables and two sets of row twiddles (by tile parity).
template <int KIND> struct S2BatchSmem {
  static constexpr bool COL = KIND <= kS2ColFwd;
  static constexpr bool HAS_P = KIND == kS2Head || KIND == kS2Mid || KIND == kS2Tail;
  static constexpr unsigned SLOT = kS2TileBytes + (COL ? 0u : 4096u);
  static constexpr unsigned PBUF = 2 * SLOT;
  static constexpr unsigned LUT = PBUF + (HAS_P ? kS2TileBytes : 0u);
  static constexpr unsigned TWR = LUT + (COL ? 0u : 2u * 256u * 8u);
  static constexpr unsigned USED = TWR + (COL ? 0u : 2u * 16u * 8u);
  static constexpr unsigned BYTES = USED + 128u;
};

template <int KIND, int MM = kS2BatchMinLog>
__device__ __forceinline__ void s2_batch_tile(const S2Inst& I, int l, unsigned char* slot, unsigned char* smraw,
                                              float2* lut, const float2* twr, unsigned long long* mbp,
                                              unsigned pparity, const S2Params& P, int* fail) {
  if constexpr (MM <= kS2BatchMaxLog) {
    if (I.m != MM) {
      s2_batch_tile<KIND, MM + 1>(I, l, slot, smraw, lut, twr, mbp, pparity, P, fail);
      return;
    }
    using Geo = S2Geo<MM, KIND>;
    using SM = S2BatchSmem<KIND>;
    if constexpr (Geo::COL) {
      s2_col_tile<MM, KIND, kS2BatchSched>(I, l, reinterpret_cast<float2*>(slot), I.tw_cols,
                                           reinterpret_cast<float2*>(smraw + SM::PBUF), mbp, pparity, P, fail);
    } else if (I.kidx) {
      s2_row_tile<MM, KIND, true, kS2BatchSched>(I, l, reinterpret_cast<float2*>(slot), I.tw_rows, lut, twr);
    } else {
      s2_row_tile<MM, KIND, false, kS2BatchSched>(I, l, reinterpret_cast<float2*>(slot), I.tw_rows, lut, twr);
    }
  }
}

// Row twiddles W_n^{256 r t} of a tile of any batch size.
template <int MM = kS2BatchMinLog>
__device__ __forceinline__ void s2_batch_twr(const S2Inst& I, int l, float2* twr) {
  if constexpr (MM <= kS2BatchMaxLog) {
    if (I.m != MM) s2_batch_twr<MM + 1>(I, l, twr);
    else s2_row_twr<MM>(I, l, twr);
  }
}

// K table of instance I into lut (all threads; nlut <= 256 when the instance has a byte index).
__device__ __forceinline__ void s2_batch_lut(const S2Inst& I, float2* lut) {
  if (I.kidx)
    for (int k = threadIdx.x; k < I.nlut; k += kS2NT) lut[k] = I.klut[k];
}

template <int KIND>
__global__ void __launch_bounds__(kS2NT, kS2MinBlocks) s2_batch_sweep(const __grid_constant__ S2Params P) {
  using SM = S2BatchSmem<KIND>;
  constexpr bool COL = SM::COL;
  extern __shared__ __align__(128) unsigned char smdyn[];
  unsigned char* smraw = smdyn + ((128u - (smem_u32(smdyn) & 127u)) & 127u);
  __shared__ __align__(8) unsigned long long mb[3];    // slot 0, slot 1, potential-phase tile
  __shared__ int fail;
  const int G = (int)gridDim.x;
  if (threadIdx.x == 0) {
    mbar_init(&mb[0], 1);
    mbar_init(&mb[1], 1);
    mbar_init(&mb[2], 1);
    fail = 0;
    fence_mbar_init();
  }
  // rows: the K table and the per-row twiddles of tile i sit in buffer i & 1, written for
  // tile i + 1 while tile i runs (the buffer of parity i + 1 was last read in tile i - 1)
  float2* lut = reinterpret_cast<float2*>(smraw + SM::LUT);
  float2* twr = reinterpret_cast<float2*>(smraw + SM::TWR);
  int t = (int)blockIdx.x;
  if (t < P.ntiles) {
    const int2 m0 = P.map[t];
    const S2Inst& I0 = P.inst[m0.x];
    if (threadIdx.x == 0) s2_issue_tile<COL, !COL>(I0, m0.y, smraw, &mb[0]);
    if constexpr (!COL) {
      s2_batch_twr(I0, m0.y, twr);
      s2_batch_lut(I0, lut);
    }
  }
  __syncthreads();
  if (t >= P.ntiles) return;
  for (int i = 0; t < P.ntiles; ++i, t += G) {
    const int s = i & 1;
    unsigned char* slot = smraw + (size_t)s * SM::SLOT;
    s2_wait(&mb[s], (unsigned)(i >> 1) & 1u, P.spin_limit, P.err, &fail);
    const int2 mt = P.map[t];
    const S2Inst& I = P.inst[mt.x];
    __syncthreads();                                    // tile i - 1 done; the wait above ended in every thread
    if (*(volatile int*)&fail) break;                   // no copy is in flight here
    if (t + G < P.ntiles) {
      const int2 mn = P.map[t + G];
      const S2Inst& In = P.inst[mn.x];
      if (threadIdx.x == 0) s2_issue_tile<COL, !COL>(In, mn.y, smraw + (size_t)(s ^ 1) * SM::SLOT, &mb[s ^ 1]);
      if constexpr (!COL) {
        s2_batch_twr(In, mn.y, twr + 16 * (s ^ 1));
        s2_batch_lut(In, lut + 256 * (s ^ 1));
      }
    }
    if constexpr (SM::HAS_P) {
      if (threadIdx.x == 0) {
        bulk_wait_read();                               // tile i - 1's stores (if any) have read the buffer
        s2_issue_p<KIND>(I, mt.y, smraw + SM::PBUF, &mb[2]);
      }
    }
    s2_batch_tile<KIND>(I, mt.y, slot, smraw, lut + 256 * s, twr + 16 * s, &mb[2], (unsigned)i & 1u, P, &fail);
  }
  if constexpr (SM::HAS_P) {
    if (threadIdx.x == 0) bulk_wait_all();              // the last tile's stores (if any), before the CTA ends
  }
}

// Batch kernels by sweep kind (kS2Row reads K through the byte index where an instance has one).
struct S2BatchKernels {
  const void* k[kS2Kinds] = {};
  size_t smem[kS2Kinds] = {};
};
S2BatchKernels s2_batch_kernels();

}  // namespace lsp
