// Internal definitions shared by the translation units of the lattice
// Strang-splitting library: plan layout, complex helpers, phase-factor
// encodings and kernel-launch declarations.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "lsp.h"

namespace lsp {

// --------------------------------------------------------------------------
// Geometry limits
// --------------------------------------------------------------------------
// Multipass tiles: a CTA owns TILE elements (16 per thread).  c64 tiles hold
// 8192 elements (64 KiB), c128 tiles 4096 (64 KiB).
constexpr int kTileC64 = 8192;
constexpr int kThreadsC64 = 512;
constexpr int kTileC128 = 4096;
constexpr int kThreadsC128 = 256;
// Column tiles need at least this many adjacent columns for 64-byte segments.
constexpr int kMinColsC64 = 8;
constexpr int kMinColsC128 = 4;
// SMEM-resident path: two state copies must fit in shared memory.
constexpr int kSmallSmemBytes = 200 * 1024;
constexpr int kSmallThreads = 512;
// Largest ||h||^2 for which K is tabulated per norm value.
constexpr long long kKLutMax = 1ll << 20;
// The four-sweep kernels read K as klut[kidx[i]] (one byte per point) below this norm.
constexpr long long kKIdxMax = 256;
// Bounded device-side waits (grid barrier): spins of ~100 ns each.
constexpr long long kSpinLimit = 1ll << 25;

// Execution paths (lsp_plan_info [3]): rank-1 two-sweep multipass (persistent kernel),
// SMEM-resident, rank-2 four-sweep, rank-1 four-sweep, rank-1 two-sweep with TMA-fed tiles.
enum PathKind {
  kPathMultipass = 0, kPathSmall = 1, kPathRank2 = 2, kPathRank1x4 = 3, kPathRank1x2 = 4, kPathMixed = 5,
  kNumPaths = 6
};

// --------------------------------------------------------------------------
// Plan
// --------------------------------------------------------------------------
// Largest lattice rank (Sec. 2.5: rank-r lattices, an r-D transform): every rank runs on the
// SMEM-resident path; ranks 1 and 2 also on the multipass paths.
constexpr int kMaxRank = 4;

struct SmallAxis {
  int len;          // axis length n_i
  int stride;       // element stride of the axis in kappa / chi order
  int nfac;         // radix factors of len, applied in order
  int fac[24];
  int tw_off;       // offset of this axis' twiddle table in tw_small
};

// Radix factors of an axis of length len for the SMEM-resident passes: 16, 8, 4,
// 2 first, then odd factors in increasing order (a prime above the last tried
// factor stays whole).  False when the factors would not fit ax.fac.
inline bool factorize_axis(int len, SmallAxis& ax) {
  const int cap = (int)(sizeof(ax.fac) / sizeof(ax.fac[0]));
  ax.nfac = 0;
  int rem = len;
  const int pref[] = {16, 8, 4, 2};
  for (int f : pref)
    while (rem % f == 0) {
      if (ax.nfac >= cap) return false;
      ax.fac[ax.nfac++] = f;
      rem /= f;
    }
  for (int f = 3; f <= rem; f += 2)
    while (rem % f == 0) {
      if (ax.nfac >= cap) return false;
      ax.fac[ax.nfac++] = f;
      rem /= f;
    }
  if (rem > 1) {
    if (ax.nfac >= cap) return false;
    ax.fac[ax.nfac++] = rem;
  }
  return true;
}

}  // namespace lsp

struct lsp_plan_s {
  int device = 0;
  int d = 0, r = 0;
  int64_t n[lsp::kMaxRank] = {1, 1, 1, 1};    // n_1..n_r, then 1
  int64_t ntot = 0;
  std::vector<int64_t> Z;        // d*r, row-major (component j of z_i at j*r + i)
  int prec = LSP_C64;
  double gamma = 1.0;
  int aa_mode = LSP_AA_MINL2;
  int path = lsp::kPathSmall;

  // multipass geometry: rank-1 n = N1 * N2 with rows of N1 contiguous points
  // (two-sweep and four-sweep paths); rank-2 four-sweep: logN1 = log2 n_1,
  // logN2 = log2 n_2 (rows of n_2 points), N1 = n_2, N2 = n_1
  int logn = 0, N1 = 1, N2 = 1, logN1 = 0, logN2 = 0, logLmax = 0;

  // SMEM-resident geometry
  int naxes = 0;
  lsp::SmallAxis axes[lsp::kMaxRank];
  int tw_lo = 0;              // complex64: offset of the lo parts of tw_small

  // device buffers
  void* u = nullptr;          // state, n complex (plan precision)
  double* v = nullptr;        // potential samples
  int32_t* norm2 = nullptr;   // ||h_chi||^2 in chi order
  void* Ph = nullptr;         // exp(-i dt v / (2 gamma)), kappa order, encoded
  void* Pf = nullptr;         // exp(-i dt v / gamma), kappa order, encoded
  void* K = nullptr;          // exp(-i gamma 2 pi^2 |h|^2 dt) in the kernel's bin order
  void* klut = nullptr;       // K per value of ||h||^2 = 0..max_norm2 (when max_norm2 < kKLutMax)
  uint8_t* kidx = nullptr;    // four-sweep paths: ||h||^2 in the K sweep's native order (max_norm2 < kKIdxMax)
  bool norms_ready = false;   // norm2 / max_norm2 computed
  void* tw_line = nullptr;    // W_Lmax^k, k < Lmax (two-sweep); W_{2^M1}^k (four-sweep: n1 or N2 points)
  void* tw_fine = nullptr;    // W_n^k, k < n / Lmax (two-sweep); W_n^k, k < N2 (rank-1 four-sweep)
  void* tw_coarse = nullptr;  // W_N1^k, k < N1 (rank-1 four-sweep)
  void* tw_pass = nullptr;    // per-pass line twiddles: row lines, then column lines
  int twr_entries = 0;        // entries of the row-line part of tw_pass
  int twa_entries = 0;        // four-sweep: entries of the second part (the third follows)
  void* tw_small = nullptr;   // per-axis W_len^k tables (SMEM-resident path)
  void* stage = nullptr;      // n complex128 staging buffer (conversions, spectral output)
  void* work = nullptr;       // n complex (plan precision): scratch copy for spectral output
  void* desc = nullptr;       // device copies of the multipass kernel descriptors
  void* s2desc = nullptr;     // TMA two-sweep path: descriptors (state, spectral copy, other buffer)
  std::vector<unsigned char> s2host0;   // host copy of descriptor slot 0
  int s2_sched = 1;                     // kernel schedule of the TMA two-sweep path (autotuned)
  int* err_host = nullptr;    // pinned mirror of the device error word
  unsigned* bar = nullptr;    // grid-barrier counter
  int* err = nullptr;         // device error word
  size_t bytes = 0;

  int dp_box = 0;
  int64_t max_norm2 = 0;
  // four-sweep paths: the launch sequence of the last call, captured as a CUDA graph and
  // replayed while the call's parameters are unchanged (key: nsteps and the kernel arguments)
  cudaGraphExec_t s4_graph = nullptr;
  std::vector<unsigned char> s4_graph_key;
  cudaStream_t capture = nullptr;   // private stream for graph capture
  double tables_dt = 0.0;     // dt of the current phase tables (NaN: none)
  bool tables_valid = false;
  long long spin_limit = lsp::kSpinLimit;   // polls of a bounded device wait (lsp_plan_set_wait_limit)
};

struct lsp_batch_s {
  std::vector<lsp_plan> plans;   // borrowed
  int prec = LSP_C64;
  std::vector<int> seq_ids;      // four-sweep instances, stepped one after another
  std::vector<int> paths;        // each plan's execution path when the batch was made
  int device = 0;
  // SMEM-resident instances: one CTA each, one launch per group (the line kernel's
  // instances by size, line_logn = log2 n; all others together, line_logn = 0)
  struct SmallGroup {
    int line_logn = 0;
    std::vector<int> ids;
    void* desc = nullptr;        // device array of their kernel descriptors
    int max_n = 0;
  };
  std::vector<SmallGroup> smalls;
  // multipass instances grouped by lattice size 2^m (one kernel per size)
  struct Class {
    int m = 0;
    std::vector<int> ids;
    void* desc = nullptr;        // device array of descriptors
    int2* colmap = nullptr;      // sweep tile -> (instance in class, local tile)
    int2* rowmap = nullptr;
    int total_col = 0, total_row = 0;
  };
  std::vector<Class> classes;
  // rank-1 four-sweep instances of one size (and K form): one launch per sweep for all
  struct S4Class {
    int m = 0;
    bool kidx = false;           // K sweeps read K through the byte index
    std::vector<int> ids;
    void* inst = nullptr;        // device array of sweep descriptors
    std::vector<unsigned char> inst_host;   // its host copy
    int2* map[3] = {};           // launch tile -> (instance in class, local tile), per geometry
    int total[3] = {};
  };
  std::vector<S4Class> s4classes;
  // rank-1 instances on the TMA two-sweep path (2^16 .. 2^23 points, any mix of sizes):
  // one launch per sweep over all their tiles, replayed as a CUDA graph
  struct S2Group {
    std::vector<int> ids;
    void* inst = nullptr;                   // device array of descriptors
    std::vector<unsigned char> inst_host;   // its host copy
    int2* map = nullptr;                    // launch tile -> (instance in group, local tile)
    int total = 0;
    cudaGraphExec_t graph = nullptr;
    std::vector<unsigned char> graph_key;
    cudaStream_t capture = nullptr;
  };
  S2Group s2group;
  cudaGraphExec_t s4_graph = nullptr;       // the four-sweep classes' launches of one call
  std::vector<unsigned char> s4_graph_key;
  cudaStream_t capture = nullptr;
  unsigned* bar = nullptr;       // grid-barrier counter (reused by every class)
  int* err = nullptr;            // device error word
  int* err_host = nullptr;       // pinned mirror
};

namespace lsp {

// --------------------------------------------------------------------------
// Complex helpers
// --------------------------------------------------------------------------
template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

__device__ __forceinline__ float2 cmake(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 cmake(double a, double b) { return make_double2(a, b); }
template <typename T> __device__ __forceinline__ T cadd(T a, T b) { return cmake(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ T csub(T a, T b) { return cmake(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ T cscale(T a, decltype(a.x) s) { return cmake(a.x * s, a.y * s); }
// a * b
template <typename T> __device__ __forceinline__ T cmul(T a, T b) {
  return cmake(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
template <typename T> __device__ __forceinline__ T cmulc(T a, T b) {
  return cmake(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
// Twiddle factors of the multipass tables.  complex64 tables hold m = w - 1 =
// (cos t - 1, sin t), accurate for small angles, applied as x + x m with the
// same four FMAs as a complex multiply; rounding cos t itself would leave
// |w| > 1 for every small angle and bias the norm a little every step.
// complex128 tables hold w = (cos t, sin t).
__device__ __forceinline__ float2 twmul(float2 x, float2 m) {
  return make_float2(fmaf(x.x, m.x, fmaf(-x.y, m.y, x.x)), fmaf(x.x, m.y, fmaf(x.y, m.x, x.y)));
}
__device__ __forceinline__ float2 twmulc(float2 x, float2 m) {   // x conj(1 + m)
  return make_float2(fmaf(x.x, m.x, fmaf(x.y, m.y, x.x)), fmaf(x.y, m.x, fmaf(-x.x, m.y, x.y)));
}
// product of two table entries, in the tables' form: (1 + a)(1 + b) - 1 = a + b + a b
__device__ __forceinline__ float2 twprod(float2 a, float2 b) {
  return make_float2(a.x + b.x + fmaf(a.x, b.x, -a.y * b.y), a.y + b.y + fmaf(a.x, b.y, a.y * b.x));
}
// a * (DIR * i):  DIR = -1 -> -i,  DIR = +1 -> +i
template <int DIR, typename T> __device__ __forceinline__ T cmul_i(T a) {
  return DIR < 0 ? cmake(a.y, -a.x) : cmake(-a.y, a.x);
}
__device__ __forceinline__ double2 twmul(double2 x, double2 w) { return cmul(x, w); }
__device__ __forceinline__ double2 twmulc(double2 x, double2 w) { return cmulc(x, w); }
__device__ __forceinline__ double2 twprod(double2 a, double2 b) { return cmul(a, b); }

// --------------------------------------------------------------------------
// Phase-factor encodings (applied as u <- w u)
// --------------------------------------------------------------------------
// complex128: (cos, sin) in FP64.
// complex64 : w = (-1)^h (1 + c + i s) stored as (c', s) in FP32 with
//   c = cos(phi) - 1 <= 0 (accurate for small phi), |phi| <= pi/2, and the
//   half-turn flag h in the sign bit of c' (sign set <=> h = 0).  Keeping
//   w - 1 instead of cos(phi) avoids the |w| > 1 bias that rounding cos(phi)
//   to 1 would give for small angles; applying it costs the same four FMAs.
__host__ __device__ inline void encode_phase(double turns, double2* out) {
  double r = turns - rint(turns);            // [-1/2, 1/2]
#ifdef __CUDA_ARCH__
  double s, c;
  sincospi(2.0 * r, &s, &c);
#else
  double s = sin(2.0 * 3.14159265358979323846 * r), c = cos(2.0 * 3.14159265358979323846 * r);
#endif
  *out = double2{c, s};
}

__host__ __device__ inline float2 encode_half_angle(double r, double sh, double ch);

__host__ __device__ inline void encode_phase(double turns, float2* out) {
  const double r = turns - rint(turns);      // [-1/2, 1/2]
  // one FP64 sine/cosine pair of the half angle: sin(phi) = 2 sin(phi/2) cos(phi/2)
#ifdef __CUDA_ARCH__
  double sh, ch;
  sincospi(r, &sh, &ch);                     // phi = 2 pi r
#else
  double sh = sin(3.14159265358979323846 * r), ch = cos(3.14159265358979323846 * r);
#endif
  *out = encode_half_angle(r, sh, ch);
}

// The pair (phi, 2 phi) from one FP64 sine/cosine evaluation, as encode_phase
// of turns and of 2 turns (the half and full potential steps).
//   complex128: (cos 2 phi, sin 2 phi) from (cos phi, sin phi) by the double-angle formulas.
//   complex64 : from sin(pi r), cos(pi r), r = turns reduced to [-1/2, 1/2]:
//     sin(2 pi r) and cos(2 pi r) are the half-angle pair of 2 r, shifted by
//     rint(2 r) half turns; the half-turn fold of encode_phase is applied to each.
__host__ __device__ inline void encode_phase_pair(double turns, double2* half, double2* full) {
  double r = turns - rint(turns);
#ifdef __CUDA_ARCH__
  double s, c;
  sincospi(2.0 * r, &s, &c);
#else
  double s = sin(2.0 * 3.14159265358979323846 * r), c = cos(2.0 * 3.14159265358979323846 * r);
#endif
  *half = double2{c, s};
  *full = double2{1.0 - 2.0 * s * s, 2.0 * s * c};
}

__host__ __device__ inline float2 encode_half_angle(double r, double sh, double ch) {
  // r in [-1/2, 1/2], sh = sin(pi r), ch = cos(pi r)
  int h = 0;
  if (r > 0.25) { const double t = sh; sh = -ch; ch = t; h = 1; }        // r - 1/2
  else if (r < -0.25) { const double t = sh; sh = ch; ch = -t; h = 1; }  // r + 1/2
  const double s = 2.0 * sh * ch;
  const double c = -2.0 * sh * sh;
  const float af = fabsf((float)c);
  return float2{h ? af : -af, (float)s};
}

__host__ __device__ inline void encode_phase_pair(double turns, float2* half, float2* full) {
  const double r = turns - rint(turns);
#ifdef __CUDA_ARCH__
  double sh, ch;
  sincospi(r, &sh, &ch);
#else
  double sh = sin(3.14159265358979323846 * r), ch = cos(3.14159265358979323846 * r);
#endif
  *half = encode_half_angle(r, sh, ch);
  const double k = rint(2.0 * r);                  // -1, 0 or 1
  const double r2 = 2.0 * r - k;                   // 2 turns reduced, exactly
  const double sg = k == 0.0 ? 1.0 : -1.0;
  *full = encode_half_angle(r2, sg * 2.0 * sh * ch, sg * (1.0 - 2.0 * sh * sh));
}

__device__ __forceinline__ float2 apply_phase(float2 x, float2 e) {
  unsigned cb = __float_as_uint(e.x);
  float c = __uint_as_float(cb | 0x80000000u);          // -|c'|
  unsigned flip = (~cb) & 0x80000000u;                   // h = 1 -> negate
  float yr = fmaf(x.x, c, fmaf(-x.y, e.y, x.x));
  float yi = fmaf(x.y, c, fmaf(x.x, e.y, x.y));
  return make_float2(__uint_as_float(__float_as_uint(yr) ^ flip),
                     __uint_as_float(__float_as_uint(yi) ^ flip));
}
__device__ __forceinline__ double2 apply_phase(double2 x, double2 e) { return cmul(x, e); }

// --------------------------------------------------------------------------
// Launch entry points implemented in the kernel translation units
// --------------------------------------------------------------------------
int multipass_desc_bytes(int prec);
bool multipass_supports(int prec, int m);
int multipass_upload_desc(lsp_plan p, cudaStream_t s);
int multipass_steps(lsp_plan p, int64_t nsteps, cudaStream_t s);
int multipass_spectral(lsp_plan p, cudaStream_t s);       // -> p->stage (chi order, c128)
int small_steps(lsp_plan p, int64_t nsteps, cudaStream_t s);
int small_spectral(lsp_plan p, cudaStream_t s);           // -> p->stage (chi order, c128)
int build_phase_tables(lsp_plan p, double dt, cudaStream_t s);
// steps of the plan's kernels on another state buffer of the same geometry
int multipass_steps_on(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s);
int small_steps_on(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s);
// batching hooks: descriptor bytes of a plan, and launches over descriptor arrays
int small_desc_size(int prec);
void small_fill_desc(lsp_plan p, void* host_out);
// line_logn > 0: all `count` instances are rank 1 with n = 2^line_logn and run the line kernel
int small_batch_launch(int prec, const void* ddesc, int count, int max_n, int line_logn, int64_t nsteps,
                       cudaStream_t s);
bool small_line_supported(int prec, int r, int logn);   // rank 1, n = 2^logn: line kernel exists
int small_line_logn(lsp_plan p);                        // log2 n if the plan runs the line kernel, else 0
int multipass_desc_size(int prec);
void multipass_fill_desc(lsp_plan p, void* host_out, int* ncol, int* nrow);
int multipass_batch_steps(int prec, int m, const void* ddesc, const int2* colmap, const int2* rowmap, int ninst,
                          int total_col, int total_row, int64_t nsteps, unsigned* bar, int* err, cudaStream_t s);

// four-sweep paths: rank-2 (n_1 = 2^m1, n_2 = 2^m2) and rank-1 (n = 2^m)
bool s4_supports_rank2(int prec, int m1, int m2);
bool s4_supports_rank1(int prec, int m);
int s4_steps_on(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s);
// Batches of rank-1 four-sweep plans of one size (lsp_batch.cu): whether a plan has
// multi-instance kernels; descriptor upload (sets *changed when the descriptors moved);
// the launches of nsteps steps; release.
bool s4_batchable(lsp_plan p);
int s4_class_init(lsp_batch_s::S4Class& c, const std::vector<lsp_plan>& plans);
int s4_class_sync(lsp_batch_s::S4Class& c, const std::vector<lsp_plan>& plans, bool* changed, cudaStream_t s);
int s4_class_steps(const lsp_batch_s::S4Class& c, int prec, int64_t nsteps, cudaStream_t s);
void s4_class_free(lsp_batch_s::S4Class& c);
int s4_spectral(lsp_plan p, cudaStream_t s);               // -> p->stage (chi order, c128)
// TMA-fed two-sweep rank-1 path (lsp_s2.cu)
constexpr int kS2NumScheds = 3;                            // kernel schedules (lsp_s2.cuh, S2Sched)
bool s2_supports(int prec, int m);
int s2_upload_desc(lsp_plan p);                            // after the tables or the K form changed
int s2_steps_on(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s);
int s2_spectral(lsp_plan p, cudaStream_t s);               // -> p->stage (chi order, c128)

// mixed-radix two-sweep path (rank 1, n = N1 N2 with N2 <= N1 <= 4096)
bool mixed_geometry(long long n, int* N1, int* N2);
int mixed_steps_on(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s);
int mixed_spectral(lsp_plan p, cudaStream_t s);            // -> p->stage (chi order, c128)
int s2_sweep_times(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s, double* ms);
bool s2_batchable(lsp_plan p);
int s2_group_init(lsp_batch_s::S2Group& g, const std::vector<lsp_plan>& plans);
int s2_group_steps(lsp_batch_s::S2Group& g, const std::vector<lsp_plan>& plans, int64_t nsteps, int* err,
                   cudaStream_t s);
void s2_group_free(lsp_batch_s::S2Group& g);
// steps of the plan's current path on a state buffer of the plan's geometry
int path_steps_on(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s);

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? LSP_OK : LSP_ERR_CUDA; }

}  // namespace lsp

#define LSP_CUDA_TRY(call)                                   \
  do {                                                       \
    cudaError_t _e = (call);                                 \
    if (_e != cudaSuccess) return LSP_ERR_CUDA;              \
  } while (0)
