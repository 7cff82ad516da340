// One mixed-radix Stockham pass of a line transform held in shared memory, for lines of any
// length (the radix factors of an axis, SmallAxis) at any stride: the building block of the
// SMEM-resident path's r-D transform (Sec. 2.5) and of the mixed-radix multipass path's line
// transforms (eq. Fnx for n that is not a power of two).
#pragma once

#include "lsp_internal.cuh"

namespace lsp {

// Pass of radix R and span Ns over the n elements of x (every line of axis `ax`, element e of
// the buffer at line position (e / stride) mod len): y = one Stockham stage (DIR = -1 forward,
// +1 inverse).  tw holds W_len^k per axis (tw_off); complex64 adds the rounding residue of each
// entry at tw_lo, applied so that the fixed rounding of an entry does not accumulate over steps.
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

}  // namespace lsp
