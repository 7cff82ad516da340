// Tile FFT building blocks for the multipass Strang step.
//
// A CTA owns a tile of C lines of length L, C * L = 16 * NT elements (16 per
// thread).  Lines are rows (contiguous; "major" thread mapping: consecutive
// threads take consecutive elements of one line) or columns (stride N1;
// consecutive threads take adjacent columns).  L, C and the radix plan are
// compile-time constants so that every index, shift and shared-memory offset
// folds into immediates.
//
// Line transforms are Stockham decimation-in-time passes (the O(n log n)
// FFT of Sec. 2.2, eq. Fnx): pass s has radix R_s and span Ns_s; butterfly j
// reads x[j + r L/R], applies W_{Ns R}^{(j mod Ns) r}, does a radix-R DFT and
// writes y[(j/Ns) Ns R + (j mod Ns) + t Ns].  The radix plan is R_1 in
// {2,4,8,16} followed by radix-16 passes, so the last pass is radix 16.
// The inverse runs the passes backward, each the conjugate transpose of its
// forward pass (butterfly, then conjugate twiddle), so the inverse's output
// pattern equals the forward's input pattern: the two meet in registers.
#pragma once

#include "lsp_internal.cuh"

namespace lsp {

// ---------------------------------------------------------------------------
// Radix butterflies on registers (DIR = -1 forward, +1 inverse)
// ---------------------------------------------------------------------------
// Constants of the radix-8/16 butterflies.  In FP32 they are applied with a
// hi/lo split (fma(x, hi, x * lo)) so that their rounding error, shared by
// every element of every pass, does not bias the norm.
struct K16 {
  static constexpr double c1 = 0.92387953251128675613;   // cos(pi/8)
  static constexpr double s1 = 0.38268343236508977173;   // sin(pi/8)
  static constexpr double r2 = 0.70710678118654752440;   // 1/sqrt(2)
};

__device__ __forceinline__ float mulk(float x, float hi, float lo) { return fmaf(x, hi, x * lo); }
__device__ __forceinline__ double mulk(double x, double hi, double) { return x * hi; }

template <typename R> struct KC {
  static constexpr R c1h = (R)K16::c1, c1l = (R)(K16::c1 - (double)(R)K16::c1);
  static constexpr R s1h = (R)K16::s1, s1l = (R)(K16::s1 - (double)(R)K16::s1);
  static constexpr R r2h = (R)K16::r2, r2l = (R)(K16::r2 - (double)(R)K16::r2);
};

// x * exp(DIR * i * pi / 4)
template <int DIR, typename T> __device__ __forceinline__ T mul_w8(T x) {
  using R = decltype(x.x);
  R a = DIR < 0 ? x.x + x.y : x.x - x.y;
  R b = DIR < 0 ? x.y - x.x : x.y + x.x;
  return cmake(mulk(a, KC<R>::r2h, KC<R>::r2l), mulk(b, KC<R>::r2h, KC<R>::r2l));
}
// x * exp(DIR * i * 3 pi / 4)
template <int DIR, typename T> __device__ __forceinline__ T mul_w8_3(T x) {
  using R = decltype(x.x);
  R a = DIR < 0 ? x.y - x.x : -x.x - x.y;
  R b = DIR < 0 ? -x.y - x.x : x.x - x.y;
  return cmake(mulk(a, KC<R>::r2h, KC<R>::r2l), mulk(b, KC<R>::r2h, KC<R>::r2l));
}
// x * (c + DIR i s) for a (cos, sin) pair given as hi/lo parts
template <int DIR>
__device__ __forceinline__ float2 mul_cs(float2 x, float ch, float cl, float sh, float sl) {
  const float s_h = DIR < 0 ? -sh : sh, s_l = DIR < 0 ? -sl : sl;
  float re = fmaf(x.x, ch, fmaf(-x.y, s_h, fmaf(x.x, cl, -x.y * s_l)));
  float im = fmaf(x.x, s_h, fmaf(x.y, ch, fmaf(x.x, s_l, x.y * cl)));
  return make_float2(re, im);
}
template <int DIR>
__device__ __forceinline__ double2 mul_cs(double2 x, double ch, double, double sh, double) {
  const double s = DIR < 0 ? -sh : sh;
  return make_double2(fma(x.x, ch, -x.y * s), fma(x.x, s, x.y * ch));
}
// x * exp(DIR * i * 2 pi k / 16) for k in {1, 3, 9}
template <int DIR, int K, typename T> __device__ __forceinline__ T mul_w16(T x) {
  using R = decltype(x.x);
  if constexpr (K == 1) return mul_cs<DIR>(x, KC<R>::c1h, KC<R>::c1l, KC<R>::s1h, KC<R>::s1l);
  else if constexpr (K == 3) return mul_cs<DIR>(x, KC<R>::s1h, KC<R>::s1l, KC<R>::c1h, KC<R>::c1l);
  else {  // K == 9: -exp(DIR i pi/8)
    T y = mul_cs<DIR>(x, KC<R>::c1h, KC<R>::c1l, KC<R>::s1h, KC<R>::s1l);
    return cmake(-y.x, -y.y);
  }
}

template <typename T> __device__ __forceinline__ void bfly2(T& a, T& b) {
  T t = a; a = cadd(t, b); b = csub(t, b);
}
template <int DIR, typename T> __device__ __forceinline__ void bfly4(T& a0, T& a1, T& a2, T& a3) {
  T t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = cmul_i<DIR>(csub(a1, a3));
  a0 = cadd(t0, t2); a2 = csub(t0, t2); a1 = cadd(t1, t3); a3 = csub(t1, t3);
}

// Radix-R DFT y_t = sum_r v_r exp(DIR 2 pi i r t / R) in place; output t is
// left in register out_at<R>(t).
template <int R> __host__ __device__ constexpr int out_at(int t) {
  return R == 8 ? 2 * (t & 3) + (t >> 2) : R == 16 ? (t >> 2) + 4 * (t & 3) : t;
}

template <int R, int DIR, typename T> __device__ __forceinline__ void bfly(T* v) {
  if constexpr (R == 2) {
    bfly2(v[0], v[1]);
  } else if constexpr (R == 4) {
    bfly4<DIR>(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 8) {
    // r = r1 + 2 r2, t = t2 + 4 t1
    bfly4<DIR>(v[0], v[2], v[4], v[6]);
    bfly4<DIR>(v[1], v[3], v[5], v[7]);
    v[3] = mul_w8<DIR>(v[3]);
    v[5] = cmul_i<DIR>(v[5]);
    v[7] = mul_w8_3<DIR>(v[7]);
    bfly2(v[0], v[1]); bfly2(v[2], v[3]); bfly2(v[4], v[5]); bfly2(v[6], v[7]);
  } else {
    // r = r1 + 4 r2, t = t2 + 4 t1
    bfly4<DIR>(v[0], v[4], v[8], v[12]);
    bfly4<DIR>(v[1], v[5], v[9], v[13]);
    bfly4<DIR>(v[2], v[6], v[10], v[14]);
    bfly4<DIR>(v[3], v[7], v[11], v[15]);
    v[5] = mul_w16<DIR, 1>(v[5]);
    v[9] = mul_w8<DIR>(v[9]);
    v[13] = mul_w16<DIR, 3>(v[13]);
    v[6] = mul_w8<DIR>(v[6]);
    v[10] = cmul_i<DIR>(v[10]);
    v[14] = mul_w8_3<DIR>(v[14]);
    v[7] = mul_w16<DIR, 3>(v[7]);
    v[11] = mul_w8_3<DIR>(v[11]);
    v[15] = mul_w16<DIR, 9>(v[15]);
    bfly4<DIR>(v[0], v[1], v[2], v[3]);
    bfly4<DIR>(v[4], v[5], v[6], v[7]);
    bfly4<DIR>(v[8], v[9], v[10], v[11]);
    bfly4<DIR>(v[12], v[13], v[14], v[15]);
  }
}

// Exchange-buffer swizzles: XOR the position within a 128-byte bank row with higher
// index bits so that the threads of a warp hit distinct banks.  SW = 0 is the
// swizzle of every line geometry below; SW = 1..3 are complex64 swizzles for column
// lines of 256 threads (consecutive threads on adjacent columns), chosen per line
// length by a bank model of every exchange pattern (conflict-free for 2^4..2^11
// points, where SW = 0 costs up to 1.5x the minimum wavefronts at 2^10).
template <typename T, int SW = 0> struct Swz;
template <> struct Swz<float2, 0> {   // 16 x 8 B per 128 B bank row
  static __device__ __forceinline__ int f(int e) { return e ^ ((e >> 4) & 15); }
};
template <> struct Swz<float2, 1> {
  static __device__ __forceinline__ int f(int e) { return e ^ ((e >> 2) & 15); }
};
template <> struct Swz<float2, 2> {
  static __device__ __forceinline__ int f(int e) { return e ^ (((e >> 2) ^ (e >> 3)) & 15); }
};
template <> struct Swz<float2, 3> {
  static __device__ __forceinline__ int f(int e) { return e ^ (((e >> 2) ^ (e >> 1)) & 15); }
};
template <> struct Swz<double2, 0> {  // 8 x 16 B per 128 B bank row
  static __device__ __forceinline__ int f(int e) { return e ^ ((e >> 3) & 7); }
};
// SW for a complex64 column line of 2^LOGL points on 256 threads; the 4096-point column lines
// (two per tile, 512 threads) take SW = 0, the one conflict-free there (SW = 1 costs 1.75x the
// minimum wavefronts by the same model)
constexpr int col_swizzle(int logl) { return logl == 12 ? 0 : logl == 11 ? 2 : logl == 9 ? 3 : 1; }
// Each swizzle changes only bits 0..3 (float2; 0..2 for double2) as a function of the bits
// below its granule: f(e + OFF) = f(e) + OFF for every OFF that is a multiple of the granule.
template <typename T, int SW> struct SwzGranule;
template <> struct SwzGranule<float2, 0> { static constexpr int G = 256; };   // bits 4..7
template <> struct SwzGranule<float2, 1> { static constexpr int G = 64; };    // bits 2..5
template <> struct SwzGranule<float2, 2> { static constexpr int G = 128; };   // bits 2..6
template <> struct SwzGranule<float2, 3> { static constexpr int G = 64; };    // bits 1..5
template <> struct SwzGranule<double2, 0> { static constexpr int G = 64; };   // bits 3..5

// State and phase-table loads and state stores bypass L1 (each point is touched
// once per sweep) but stay in L2 with normal priority: when state and tables fit
// in L2 (2^22 complex64: 32 MiB state, 32 MiB P, 4 MiB K index) they are found
// there on the next step.  (Evict-first table loads measured 3.5 % slower at 2^22.)
template <typename T> __device__ __forceinline__ T ldst(const T* p) { return __ldcg(p); }
template <typename T> __device__ __forceinline__ void stst(T* p, T v) { __stcg(p, v); }
template <typename T> __device__ __forceinline__ T ldtab(const T* p) { return __ldcg(p); }

// ---------------------------------------------------------------------------
// Compile-time line geometry
// ---------------------------------------------------------------------------
// NW independent workers of NT threads share a CTA; each transforms its own
// tile and synchronises on its own named barrier (id 1 + worker).
template <typename T, int NT, int LOGL, bool MAJOR, int NW = 1, int SW = 0>
struct Line {
  static constexpr int L = 1 << LOGL;
  static __device__ __forceinline__ int tid() { return NW == 1 ? (int)threadIdx.x : (int)(threadIdx.x & (NT - 1)); }
  static __device__ __forceinline__ void sync() {
    if constexpr (NW == 1) {
      __syncthreads();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)(threadIdx.x / NT)), "r"(NT) : "memory");
    }
  }
  static constexpr int LOGNT = NT == 512 ? 9 : NT == 256 ? 8 : NT == 128 ? 7 : 10;
  static constexpr int LOGC = LOGNT + 4 - LOGL;      // lines per tile
  static constexpr int C = 1 << LOGC;
  static constexpr int LOGR1 = LOGL % 4 == 0 ? 4 : LOGL % 4;
  static constexpr int R1 = 1 << LOGR1;
  static constexpr int P = (LOGL - LOGR1) / 4 + 1;   // passes
  static_assert(LOGC >= 0, "line longer than a tile");
  static_assert(LOGL >= 4, "line shorter than 16");

  // log2 Ns of pass S (1-based)
  static constexpr int lns(int S) { return S == 1 ? 0 : LOGR1 + 4 * (S - 2); }
  static constexpr int radix_log(int S) { return S == 1 ? LOGR1 : 4; }
  // Per-pass twiddle tables: pass S >= 2 (radix 16) owns 15 Ns entries laid
  // out [r-1][jm] = W_{16 Ns}^{jm r}, so that threads with consecutive jm read
  // consecutive words.  tw_off(S) is the start of pass S's table.
  static constexpr int tw_off(int S) {
    int o = 0;
    for (int s = 2; s < S; ++s) o += 15 << lns(s);
    return o;
  }
  static constexpr int TW_ENTRIES = tw_off(P + 1);

  // q-th butterfly of this thread for radix 2^LR -> (line b, butterfly j)
  template <int LR>
  static __device__ __forceinline__ void bm(int q, int& b, int& j) {
    const int beta = tid() + NT * q;
    if constexpr (MAJOR) { j = beta & ((1 << (LOGL - LR)) - 1); b = beta >> (LOGL - LR); }
    else { b = beta & (C - 1); j = beta >> LOGC; }
  }
  static __device__ __forceinline__ int sidx(int b, int i) {
    return Swz<T, SW>::f(MAJOR ? (b << LOGL) + i : (i << LOGC) + b);
  }
  // swizzled position of element (b, i0 + DI) for a compile-time DI: one swizzle of the
  // thread's base position plus an immediate when DI's offset is a multiple of the granule
  template <int DI>
  static __device__ __forceinline__ int sidx_at(int b, int i0) {
    constexpr int OFF = MAJOR ? DI : DI << LOGC;
    if constexpr (OFF % SwzGranule<T, SW>::G == 0) return sidx(b, i0) + OFF;
    else return sidx(b, i0 + DI);
  }

  // ---- forward pass S: registers hold inputs x[j + r L/R] ----
  template <int S>
  static __device__ __forceinline__ void fwd_body(const T* __restrict__ tw, T (&v)[16]) {
    constexpr int LR = radix_log(S), R = 1 << LR, LNS = lns(S);
#pragma unroll
    for (int q = 0; q < 16 / R; ++q) {
      if constexpr (S > 1) {
        int b, j; bm<LR>(q, b, j);
        const T* tq = tw + tw_off(S) + (j & ((1 << LNS) - 1));
#pragma unroll
        for (int r = 1; r < R; ++r) v[q * R + r] = twmul(v[q * R + r], tq[(r - 1) << LNS]);
      }
      bfly<R, -1>(&v[q * R]);
    }
  }
  // element index t * STEP of a butterfly (t < R) at base i0, as compile-time offsets
  template <int STEP, int R, typename F>
  static __device__ __forceinline__ void for_offsets(int b, int i0, F&& f) {
    for_offsets_impl<STEP, R, 0>(b, i0, f);
  }
  template <int STEP, int R, int K, typename F>
  static __device__ __forceinline__ void for_offsets_impl(int b, int i0, F& f) {
    if constexpr (K < R) {
      f(K, sidx_at<K * STEP>(b, i0));
      for_offsets_impl<STEP, R, K + 1>(b, i0, f);
    }
  }
  template <int S>
  static __device__ __forceinline__ void write_out(T* sm, const T (&v)[16]) {
    constexpr int LR = radix_log(S), R = 1 << LR, LNS = lns(S);
#pragma unroll
    for (int q = 0; q < 16 / R; ++q) {
      int b, j; bm<LR>(q, b, j);
      const int ob = ((j >> LNS) << (LNS + LR)) + (j & ((1 << LNS) - 1));
      for_offsets<(1 << LNS), R>(b, ob, [&](int t, int pos) { sm[pos] = v[q * R + out_at<R>(t)]; });
    }
  }
  template <int S>
  static __device__ __forceinline__ void read_in(const T* sm, T (&v)[16]) {
    constexpr int LR = radix_log(S), R = 1 << LR;
#pragma unroll
    for (int q = 0; q < 16 / R; ++q) {
      int b, j; bm<LR>(q, b, j);
      for_offsets<(1 << (LOGL - LR)), R>(b, j, [&](int r, int pos) { v[q * R + r] = sm[pos]; });
    }
  }
  // ---- inverse pass S (conjugate transpose of forward pass S) ----
  template <int S>
  static __device__ __forceinline__ void read_out(const T* sm, T (&v)[16]) {
    constexpr int LR = radix_log(S), R = 1 << LR, LNS = lns(S);
#pragma unroll
    for (int q = 0; q < 16 / R; ++q) {
      int b, j; bm<LR>(q, b, j);
      const int ob = ((j >> LNS) << (LNS + LR)) + (j & ((1 << LNS) - 1));
      for_offsets<(1 << LNS), R>(b, ob, [&](int t, int pos) { v[q * R + t] = sm[pos]; });
    }
  }
  template <int S>
  static __device__ __forceinline__ void inv_body(const T* __restrict__ tw, T (&v)[16]) {
    constexpr int LR = radix_log(S), R = 1 << LR, LNS = lns(S);
#pragma unroll
    for (int q = 0; q < 16 / R; ++q) {
      T w[R];
#pragma unroll
      for (int t = 0; t < R; ++t) w[t] = v[q * R + t];
      bfly<R, +1>(w);
#pragma unroll
      for (int r = 0; r < R; ++r) v[q * R + r] = w[out_at<R>(r)];
      if constexpr (S > 1) {
        int b, j; bm<LR>(q, b, j);
        const T* tq = tw + tw_off(S) + (j & ((1 << LNS) - 1));
#pragma unroll
        for (int r = 1; r < R; ++r) v[q * R + r] = twmulc(v[q * R + r], tq[(r - 1) << LNS]);
      }
    }
  }
  template <int S>
  static __device__ __forceinline__ void write_in(T* sm, const T (&v)[16]) {
    constexpr int LR = radix_log(S), R = 1 << LR;
#pragma unroll
    for (int q = 0; q < 16 / R; ++q) {
      int b, j; bm<LR>(q, b, j);
      for_offsets<(1 << (LOGL - LR)), R>(b, j, [&](int r, int pos) { sm[pos] = v[q * R + r]; });
    }
  }

  // Forward line DFT: registers in the pass-1 input pattern -> last-pass
  // outputs in natural order (v[t] = element j + t L/16 of the thread's
  // radix-16 butterfly).
  template <int S = 1>
  static __device__ __forceinline__ void dft(T* sm, const T* tw, T (&v)[16]) {
    if constexpr (S > 1) {
      sync();
      read_in<S>(sm, v);
    }
    fwd_body<S>(tw, v);
    if constexpr (S < P) {
      sync();
      write_out<S>(sm, v);
      dft<S + 1>(sm, tw, v);
    } else {
      constexpr int R = 1 << radix_log(S);
      T w[16];
#pragma unroll
      for (int q = 0; q < 16 / R; ++q)
#pragma unroll
        for (int t = 0; t < R; ++t) w[q * R + t] = v[q * R + out_at<R>(t)];
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = w[i];
    }
  }
  // Twiddles of the thread's radix-16 butterfly in pass S >= 2 (one butterfly per
  // thread there): w[r - 1] = W_{16 Ns}^{jm r}, r = 1..15.
  template <int S>
  static __device__ __forceinline__ void load_tw(const T* __restrict__ tw, T (&w)[15]) {
    static_assert(S > 1 && radix_log(S) == 4, "passes after the first are radix 16");
    constexpr int LNS = lns(S);
    int b, j;
    bm<4>(0, b, j);
    const T* tq = tw + tw_off(S) + (j & ((1 << LNS) - 1));
#pragma unroll
    for (int r = 1; r < 16; ++r) w[r - 1] = tq[(r - 1) << LNS];
  }
  // dft / idft with each pass' twiddles loaded before the barriers and the exchange
  // that precede the pass, so that their latency overlaps the wait and the reads.
  template <int S = 1>
  static __device__ __forceinline__ void dft_pre(T* sm, const T* tw, T (&v)[16]) {
    fwd_body<S>(tw, v);
    if constexpr (S < P) {
      T w[15];
      load_tw<S + 1>(tw, w);
      sync();
      write_out<S>(sm, v);
      sync();
      read_in<S + 1>(sm, v);
#pragma unroll
      for (int r = 1; r < 16; ++r) v[r] = twmul(v[r], w[r - 1]);
      dft_pre_tail<S + 1>(sm, tw, v);
    } else {
      constexpr int R = 1 << radix_log(S);
      T o[16];
#pragma unroll
      for (int q = 0; q < 16 / R; ++q)
#pragma unroll
        for (int t = 0; t < R; ++t) o[q * R + t] = v[q * R + out_at<R>(t)];
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = o[i];
    }
  }
  // pass S >= 2 of dft_pre after its twiddles: the butterfly, then as dft_pre
  template <int S>
  static __device__ __forceinline__ void dft_pre_tail(T* sm, const T* tw, T (&v)[16]) {
    bfly<16, -1>(v);
    if constexpr (S < P) {
      T w[15];
      load_tw<S + 1>(tw, w);
      sync();
      write_out<S>(sm, v);
      sync();
      read_in<S + 1>(sm, v);
#pragma unroll
      for (int r = 1; r < 16; ++r) v[r] = twmul(v[r], w[r - 1]);
      dft_pre_tail<S + 1>(sm, tw, v);
    } else {
      T o[16];
#pragma unroll
      for (int t = 0; t < 16; ++t) o[t] = v[out_at<16>(t)];
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = o[i];
    }
  }
  template <int S = P>
  static __device__ __forceinline__ void idft_pre(T* sm, const T* tw, T (&v)[16]) {
    if constexpr (S > 1) {
      T w[15];
      load_tw<S>(tw, w);
      if constexpr (S < P) {
        sync();
        read_out<S>(sm, v);
      }
      T o[16];
#pragma unroll
      for (int t = 0; t < 16; ++t) o[t] = v[t];
      bfly<16, +1>(o);
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = o[out_at<16>(r)];
#pragma unroll
      for (int r = 1; r < 16; ++r) v[r] = twmulc(v[r], w[r - 1]);
      sync();
      write_in<S>(sm, v);
      idft_pre<S - 1>(sm, tw, v);
    } else {
      if constexpr (S < P) {
        sync();
        read_out<S>(sm, v);
      }
      inv_body<S>(tw, v);
    }
  }

  // Inverse line DFT (unnormalised): registers holding the last forward
  // pass' outputs in natural order -> the pass-1 input pattern.
  template <int S = P>
  static __device__ __forceinline__ void idft(T* sm, const T* tw, T (&v)[16]) {
    if constexpr (S < P) {
      sync();
      read_out<S>(sm, v);
    }
    inv_body<S>(tw, v);
    if constexpr (S > 1) {
      sync();
      write_in<S>(sm, v);
      idft<S - 1>(sm, tw, v);
    }
  }
};

}  // namespace lsp
