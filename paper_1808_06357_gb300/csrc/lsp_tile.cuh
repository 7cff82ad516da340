// Tile FFT building blocks for the multipass Strang step.
//
// A CTA owns a tile of C lines of length L (16 * NT elements).  Lines are
// either rows (contiguous, "line-major" thread mapping: consecutive threads
// take consecutive elements of a line) or columns (stride N1, "line-minor":
// consecutive threads take consecutive lines, i.e. adjacent columns).
//
// Line transforms are Stockham decimation-in-time passes (paper eq. Fnx, the
// O(n log n) FFT of Sec. 2.2): pass s has radix R_s and span Ns_s; butterfly j
// reads x[j + r L/R], applies W_{Ns R}^{(j mod Ns) r}, does a radix-R DFT and
// writes y[(j/Ns) Ns R + (j mod Ns) + s Ns].  The radix plan is R_1 in
// {2,4,8,16} then radix 16, so the last pass is always radix 16.
// The inverse transform runs the same passes backward, each one the
// conjugate transpose of its forward pass (butterfly, then conjugate
// twiddle), so the inverse's output pattern equals the forward's input
// pattern and the two meet in registers with no shared-memory round trip.
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
  // (1 + DIR i)/sqrt(2): (xr - DIR xi, xi + DIR xr) / sqrt(2)
  R a = DIR < 0 ? x.x + x.y : x.x - x.y;
  R b = DIR < 0 ? x.y - x.x : x.y + x.x;
  return cmake(mulk(a, KC<R>::r2h, KC<R>::r2l), mulk(b, KC<R>::r2h, KC<R>::r2l));
}
// x * exp(DIR * i * 3 pi / 4)
template <int DIR, typename T> __device__ __forceinline__ T mul_w8_3(T x) {
  using R = decltype(x.x);
  // (-1 + DIR i)/sqrt(2): (-xr - DIR xi, -xi + DIR xr) / sqrt(2)
  R a = DIR < 0 ? x.y - x.x : -x.x - x.y;
  R b = DIR < 0 ? -x.y - x.x : x.x - x.y;
  return cmake(mulk(a, KC<R>::r2h, KC<R>::r2l), mulk(b, KC<R>::r2h, KC<R>::r2l));
}
// x * (c + DIR i s) for the (cos, sin) pair given as hi/lo parts
__device__ __forceinline__ float2 mul_cs(float2 x, float ch, float cl, float sh, float sl, int dir) {
  float s_h = dir < 0 ? -sh : sh, s_l = dir < 0 ? -sl : sl;
  float re = fmaf(x.x, ch, fmaf(-x.y, s_h, fmaf(x.x, cl, -x.y * s_l)));
  float im = fmaf(x.x, s_h, fmaf(x.y, ch, fmaf(x.x, s_l, x.y * cl)));
  return make_float2(re, im);
}
__device__ __forceinline__ double2 mul_cs(double2 x, double ch, double, double sh, double, int dir) {
  double s = dir < 0 ? -sh : sh;
  return make_double2(fma(x.x, ch, -x.y * s), fma(x.x, s, x.y * ch));
}
// x * exp(DIR * i * 2 pi k / 16) for k in {1, 3, 9}
template <int DIR, int K, typename T> __device__ __forceinline__ T mul_w16(T x) {
  using R = decltype(x.x);
  if (K == 1) return mul_cs(x, KC<R>::c1h, KC<R>::c1l, KC<R>::s1h, KC<R>::s1l, DIR);
  if (K == 3) return mul_cs(x, KC<R>::s1h, KC<R>::s1l, KC<R>::c1h, KC<R>::c1l, DIR);
  // K == 9: -exp(DIR i pi/8)
  T y = mul_cs(x, KC<R>::c1h, KC<R>::c1l, KC<R>::s1h, KC<R>::s1l, DIR);
  return cmake(-y.x, -y.y);
}

template <int DIR, typename T> __device__ __forceinline__ void bfly2(T& a, T& b) {
  T t = a; a = cadd(t, b); b = csub(t, b);
}
template <int DIR, typename T> __device__ __forceinline__ void bfly4(T& a0, T& a1, T& a2, T& a3) {
  T t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = cmul_i<DIR>(csub(a1, a3));
  a0 = cadd(t0, t2); a2 = csub(t0, t2); a1 = cadd(t1, t3); a3 = csub(t1, t3);
}

// Radix-R DFT of v[0..R-1] in place: y_s = sum_r v_r exp(DIR 2 pi i r s / R).
// Output s is left in register OUT<R>(s).
template <int R> struct Out;
template <> struct Out<2> { static __device__ __forceinline__ constexpr int at(int s) { return s; } };
template <> struct Out<4> { static __device__ __forceinline__ constexpr int at(int s) { return s; } };
template <> struct Out<8> { static __device__ __forceinline__ constexpr int at(int s) { return 2 * (s & 3) + (s >> 2); } };
template <> struct Out<16> { static __device__ __forceinline__ constexpr int at(int s) { return (s >> 2) + 4 * (s & 3); } };

template <int R, int DIR, typename T> __device__ __forceinline__ void bfly(T* v) {
  if constexpr (R == 2) {
    bfly2<DIR>(v[0], v[1]);
  } else if constexpr (R == 4) {
    bfly4<DIR>(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 8) {
    // r = r1 + 2 r2, s = s2 + 4 s1
    bfly4<DIR>(v[0], v[2], v[4], v[6]);
    bfly4<DIR>(v[1], v[3], v[5], v[7]);
    v[3] = mul_w8<DIR>(v[3]);
    v[5] = cmul_i<DIR>(v[5]);
    v[7] = mul_w8_3<DIR>(v[7]);
    bfly2<DIR>(v[0], v[1]); bfly2<DIR>(v[2], v[3]); bfly2<DIR>(v[4], v[5]); bfly2<DIR>(v[6], v[7]);
  } else {
    // r = r1 + 4 r2, s = s2 + 4 s1
    bfly4<DIR>(v[0], v[4], v[8], v[12]);
    bfly4<DIR>(v[1], v[5], v[9], v[13]);
    bfly4<DIR>(v[2], v[6], v[10], v[14]);
    bfly4<DIR>(v[3], v[7], v[11], v[15]);
    // twiddle W16^{r1 s2} on v[r1 + 4 s2]
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

// ---------------------------------------------------------------------------
// Tile geometry
// ---------------------------------------------------------------------------
struct Geo {
  int logL;        // line length L = 2^logL
  int logC;        // lines in the tile
  int major;       // 1: rows (j fastest over threads), 0: columns (line fastest)
  int logR1;       // log2 of the first-pass radix
  int p;           // number of passes
  int logLmax;     // size of the line-twiddle table
};

template <typename T> struct Swz;
template <> struct Swz<float2> {
  static __device__ __forceinline__ int f(int e) { return e ^ ((e >> 4) & 15); }
};
template <> struct Swz<double2> {
  static __device__ __forceinline__ int f(int e) { return e ^ ((e >> 3) & 7); }
};

template <typename T> __device__ __forceinline__ int sidx(const Geo& g, int b, int i) {
  int e = g.major ? ((b << g.logL) + i) : ((i << g.logC) + b);
  return Swz<T>::f(e);
}

// Butterfly beta of a pass with log2(L/R) = lLR -> (line b, butterfly j).
__device__ __forceinline__ void bmap(const Geo& g, int beta, int lLR, int& b, int& j) {
  if (g.major) { j = beta & ((1 << lLR) - 1); b = beta >> lLR; }
  else { b = beta & ((1 << g.logC) - 1); j = beta >> g.logC; }
}

// log2 of Ns for pass s (1-based): Ns_1 = 1, Ns_s = R1 * 16^(s-2)
__device__ __forceinline__ int log_ns(const Geo& g, int s) { return s == 1 ? 0 : g.logR1 + 4 * (s - 2); }

template <typename T> __device__ __forceinline__ T ldtw(const T* tw, int k) { return __ldg(tw + k); }

// ---------------------------------------------------------------------------
// Passes.  Register layout: v[q * R + r] holds element r of the thread's q-th
// butterfly (16 / R butterflies per thread, 16 elements).
// ---------------------------------------------------------------------------

// Read pass-s inputs x[j + r L/R] from shared memory.
template <int R, int NT, typename T>
__device__ __forceinline__ void read_in(const Geo& g, const T* sm, T (&v)[16]) {
  constexpr int LR = (R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4);
  const int lLR = g.logL - LR;
  const int nb = 1 << (g.logC + lLR);
#pragma unroll
  for (int q = 0; q < 16 / R; ++q) {
    int beta = threadIdx.x + NT * q;
    if (beta < nb) {
      int b, j; bmap(g, beta, lLR, b, j);
#pragma unroll
      for (int r = 0; r < R; ++r) v[q * R + r] = sm[sidx<T>(g, b, j + (r << lLR))];
    }
  }
}

// Forward pass s body on registers: twiddle (s > 1) then butterfly.
template <int R, int NT, typename T>
__device__ __forceinline__ void fwd_body(const Geo& g, int s, const T* twl, T (&v)[16]) {
  constexpr int LR = (R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4);
  const int lLR = g.logL - LR;
  const int nb = 1 << (g.logC + lLR);
  const int lns = log_ns(g, s);
#pragma unroll
  for (int q = 0; q < 16 / R; ++q) {
    int beta = threadIdx.x + NT * q;
    if (beta < nb) {
      if (s > 1) {
        int b, j; bmap(g, beta, lLR, b, j);
        int jm = j & ((1 << lns) - 1);
        int sh = g.logLmax - lns - LR;
#pragma unroll
        for (int r = 1; r < R; ++r) v[q * R + r] = cmul(v[q * R + r], ldtw(twl, (jm * r) << sh));
      }
      bfly<R, -1>(&v[q * R]);
    }
  }
}

// Write forward pass-s outputs y[(j/Ns) Ns R + (j mod Ns) + s Ns] to shared memory.
template <int R, int NT, typename T>
__device__ __forceinline__ void write_out(const Geo& g, int s, T* sm, const T (&v)[16]) {
  constexpr int LR = (R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4);
  const int lLR = g.logL - LR;
  const int nb = 1 << (g.logC + lLR);
  const int lns = log_ns(g, s);
#pragma unroll
  for (int q = 0; q < 16 / R; ++q) {
    int beta = threadIdx.x + NT * q;
    if (beta < nb) {
      int b, j; bmap(g, beta, lLR, b, j);
      int jm = j & ((1 << lns) - 1);
      int ob = ((j >> lns) << (lns + LR)) + jm;
#pragma unroll
      for (int t = 0; t < R; ++t) sm[sidx<T>(g, b, ob + (t << lns))] = v[q * R + Out<R>::at(t)];
    }
  }
}

// Read inverse pass-s inputs (the forward pass' output positions) into natural order.
template <int R, int NT, typename T>
__device__ __forceinline__ void read_out(const Geo& g, int s, const T* sm, T (&v)[16]) {
  constexpr int LR = (R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4);
  const int lLR = g.logL - LR;
  const int nb = 1 << (g.logC + lLR);
  const int lns = log_ns(g, s);
#pragma unroll
  for (int q = 0; q < 16 / R; ++q) {
    int beta = threadIdx.x + NT * q;
    if (beta < nb) {
      int b, j; bmap(g, beta, lLR, b, j);
      int jm = j & ((1 << lns) - 1);
      int ob = ((j >> lns) << (lns + LR)) + jm;
#pragma unroll
      for (int t = 0; t < R; ++t) v[q * R + t] = sm[sidx<T>(g, b, ob + (t << lns))];
    }
  }
}

// Inverse pass-s body: butterfly (conjugate) then conjugate twiddle (s > 1).
// Output element r of butterfly q ends in v[q * R + r] (natural order).
template <int R, int NT, typename T>
__device__ __forceinline__ void inv_body(const Geo& g, int s, const T* twl, T (&v)[16]) {
  constexpr int LR = (R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4);
  const int lLR = g.logL - LR;
  const int nb = 1 << (g.logC + lLR);
  const int lns = log_ns(g, s);
#pragma unroll
  for (int q = 0; q < 16 / R; ++q) {
    int beta = threadIdx.x + NT * q;
    if (beta < nb) {
      T w[R];
#pragma unroll
      for (int t = 0; t < R; ++t) w[t] = v[q * R + t];
      bfly<R, +1>(w);
#pragma unroll
      for (int r = 0; r < R; ++r) v[q * R + r] = w[Out<R>::at(r)];
      if (s > 1) {
        int b, j; bmap(g, beta, lLR, b, j);
        int jm = j & ((1 << lns) - 1);
        int sh = g.logLmax - lns - LR;
#pragma unroll
        for (int r = 1; r < R; ++r) v[q * R + r] = cmulc(v[q * R + r], ldtw(twl, (jm * r) << sh));
      }
    }
  }
}

// Write inverse pass-s outputs x[j + r L/R] to shared memory.
template <int R, int NT, typename T>
__device__ __forceinline__ void write_in(const Geo& g, T* sm, const T (&v)[16]) {
  constexpr int LR = (R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4);
  const int lLR = g.logL - LR;
  const int nb = 1 << (g.logC + lLR);
#pragma unroll
  for (int q = 0; q < 16 / R; ++q) {
    int beta = threadIdx.x + NT * q;
    if (beta < nb) {
      int b, j; bmap(g, beta, lLR, b, j);
#pragma unroll
      for (int r = 0; r < R; ++r) sm[sidx<T>(g, b, j + (r << lLR))] = v[q * R + r];
    }
  }
}

// Permute forward-pass outputs held in registers (register Out<R>(t) holds
// output t) into natural order, so that an inverse pass can consume them.
template <int R, typename T> __device__ __forceinline__ void out_to_nat(T (&v)[16]) {
  T w[16];
#pragma unroll
  for (int q = 0; q < 16 / R; ++q)
#pragma unroll
    for (int t = 0; t < R; ++t) w[q * R + t] = v[q * R + Out<R>::at(t)];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = w[i];
}

// Dispatch helpers on the runtime first-pass radix.
#define LSP_R1_DISPATCH(logR1, ...)                          \
  switch (logR1) {                                           \
    case 1: { constexpr int RR = 2; __VA_ARGS__; } break;    \
    case 2: { constexpr int RR = 4; __VA_ARGS__; } break;    \
    case 3: { constexpr int RR = 8; __VA_ARGS__; } break;    \
    default: { constexpr int RR = 16; __VA_ARGS__; } break;  \
  }

// Radix of pass s (1-based): R1 for s = 1, else 16.
// Full forward line DFT from registers (loaded in the pass-1 input pattern);
// ends with the last pass' outputs in registers in natural output order
// (element j + t L/16 of butterfly q in v[q*16 + t]).
template <int NT, typename T>
__device__ __forceinline__ void line_dft(const Geo& g, T* sm, const T* twl, T (&v)[16]) {
  for (int s = 1; s <= g.p; ++s) {
    if (s > 1) {
      __syncthreads();
      read_in<16, NT>(g, sm, v);
      fwd_body<16, NT>(g, s, twl, v);
    } else {
      LSP_R1_DISPATCH(g.logR1, fwd_body<RR, NT>(g, 1, twl, v));
    }
    if (s < g.p) {
      __syncthreads();                            // earlier readers of sm are done
      if (s == 1) { LSP_R1_DISPATCH(g.logR1, write_out<RR, NT>(g, 1, sm, v)); }
      else write_out<16, NT>(g, s, sm, v);
    }
  }
  if (g.p == 1) { LSP_R1_DISPATCH(g.logR1, out_to_nat<RR>(v)); }
  else out_to_nat<16>(v);
}

// Full inverse line DFT (unnormalised) from registers holding the last
// forward pass' outputs in natural order; ends with the pass-1 input pattern
// in registers.
template <int NT, typename T>
__device__ __forceinline__ void line_idft(const Geo& g, T* sm, const T* twl, T (&v)[16]) {
  for (int s = g.p; s >= 1; --s) {
    if (s < g.p) {
      __syncthreads();                            // writes of the previous pass visible
      if (s == 1) { LSP_R1_DISPATCH(g.logR1, read_out<RR, NT>(g, 1, sm, v)); }
      else read_out<16, NT>(g, s, sm, v);
    }
    if (s == 1) { LSP_R1_DISPATCH(g.logR1, inv_body<RR, NT>(g, 1, twl, v)); }
    else inv_body<16, NT>(g, s, twl, v);
    if (s > 1) {
      __syncthreads();                            // all reads of this pass done
      write_in<16, NT>(g, sm, v);
    }
  }
}

}  // namespace lsp
