// Host side of the multipass Strang step: kernel selection per lattice size,
// descriptors, cooperative persistent launches and single-sweep launches.
#include <string.h>

#include <algorithm>

#include "lsp_mp.cuh"

namespace lsp {

static int ilog2i(long long x) { int l = 0; while ((1ll << l) < x) ++l; return l; }

static bool kernels_for(int prec, int m, MPKernels* k) {
  if (prec == LSP_C64) return mp_kernels_c64_lo(m, k) || mp_kernels_c64_hi(m, k);
  return mp_kernels_c128_lo(m, k) || mp_kernels_c128_hi(m, k);
}

bool multipass_supports(int prec, int m) {
  MPKernels k;
  return kernels_for(prec, m, &k);
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
  I.twr = (const T*)pl->tw_pass;
  I.twc = (const T*)pl->tw_pass + pl->twr_entries;
  I.spec = spec;
  I.logN1 = pl->logN1; I.logN2 = pl->logN2; I.logn = pl->logn; I.logLmax = pl->logLmax;
  const int logTile = ilog2i(TILE);
  const int logCc = logTile - pl->logN2;   // columns per column tile
  const int logCr = logTile - pl->logN1;   // rows per row tile
  I.ncol = pl->logN1 > logCc ? 1 << (pl->logN1 - logCc) : 1;
  I.nrow = pl->logN2 > logCr ? 1 << (pl->logN2 - logCr) : 1;
  I.inv_n = (decltype(I.inv_n))(1.0 / (double)pl->ntot);
  return I;
}

// Co-resident CTA count of a kernel (cached per kernel pointer).
template <typename T> static int coresident(const void* fn, size_t smem, int& grid) {
  constexpr int NT = Cfg<T>::NT * Cfg<T>::NW;
  static const void* cfn[64] = {};
  static int cval[64] = {};
  for (int i = 0; i < 64; ++i)
    if (cfn[i] == fn) { grid = cval[i]; return LSP_OK; }
  int dev = 0, per_sm = 0, sms = 0;
  LSP_CUDA_TRY(cudaGetDevice(&dev));
  LSP_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  LSP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NT, smem));
  LSP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  grid = per_sm * sms;
  for (int i = 0; i < 64; ++i)
    if (!cfn[i]) { cfn[i] = fn; cval[i] = grid; break; }
  return grid > 0 ? LSP_OK : LSP_ERR_CUDA;
}

template <typename T>
int launch_persistent(int m, const MPInst<T>* dinst, const int2* colmap, const int2* rowmap, int ninst,
                      int total_col, int total_row, int64_t nsteps, unsigned* bar, int* err, long long spin_limit,
                      cudaStream_t s) {
  MPKernels k;
  if (!kernels_for(sizeof(T) == 8 ? LSP_C64 : LSP_C128, m, &k)) return LSP_ERR_TOO_LARGE;
  constexpr int NT = Cfg<T>::NT * Cfg<T>::NW;
  const size_t smem = k.persistent_smem;
  int grid = 0;
  int rc = coresident<T>(k.persistent, smem, grid);
  if (rc) return rc;
  grid = std::min(grid, (std::max(total_col, total_row) + Cfg<T>::NW - 1) / Cfg<T>::NW);
  MPParams<T> P{dinst, colmap, rowmap, ninst, total_col, total_row, (long long)nsteps, 0, bar, err, spin_limit};
  LSP_CUDA_TRY(cudaMemsetAsync(bar, 0, sizeof(unsigned), s));
  void* args[] = {&P};
  LSP_CUDA_TRY(cudaLaunchCooperativeKernel(k.persistent, dim3(grid), dim3(NT), args, smem, s));
  return LSP_OK;
}

template <typename T>
int launch_sweep(int m, const MPInst<T>* dinst, const int2* colmap, const int2* rowmap, int ninst,
                 int total_col, int total_row, int kind, cudaStream_t s) {
  MPKernels k;
  if (!kernels_for(sizeof(T) == 8 ? LSP_C64 : LSP_C128, m, &k)) return LSP_ERR_TOO_LARGE;
  constexpr int NT = Cfg<T>::NT * Cfg<T>::NW;
  const size_t smem = (size_t)Cfg<T>::TILE * Cfg<T>::NW * sizeof(T);
  int grid = 0;
  int rc = coresident<T>(k.sweep[kind], smem, grid);
  if (rc) return rc;
  const bool col = kind != kRow && kind != kRowFwd;
  grid = std::min(grid, ((col ? total_col : total_row) + Cfg<T>::NW - 1) / Cfg<T>::NW);
  MPParams<T> P{dinst, colmap, rowmap, ninst, total_col, total_row, 0, kind, nullptr, nullptr, kSpinLimit};
  void* args[] = {&P};
  LSP_CUDA_TRY(cudaLaunchKernel(k.sweep[kind], dim3(grid), dim3(NT), args, smem, s));
  return LSP_OK;
}

template int launch_sweep<float2>(int, const MPInst<float2>*, const int2*, const int2*, int, int, int, int,
                                  cudaStream_t);
template int launch_sweep<double2>(int, const MPInst<double2>*, const int2*, const int2*, int, int, int, int,
                                   cudaStream_t);

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

// Sweeps 1..2N-1 of N steps (row, mid, ..., row): one persistent cooperative launch.
template <typename T>
static int middle_sweeps(int m, const MPInst<T>* d, const int2* colmap, const int2* rowmap, int ninst, int total_col,
                         int total_row, int64_t nsteps, unsigned* bar, int* err, cudaStream_t s,
                         long long spin_limit = kSpinLimit) {
  return launch_persistent<T>(m, d, colmap, rowmap, ninst, total_col, total_row, nsteps, bar, err, spin_limit, s);
}

// head sweep, sweeps 1..2N-1, tail sweep
template <typename T>
static int steps_impl(lsp_plan p, int64_t nsteps, cudaStream_t s) {
  MPInst<T> I = make_inst<T>(p, nullptr);
  const MPInst<T>* d = (const MPInst<T>*)p->desc;
  int rc = launch_sweep<T>(p->logn, d, nullptr, nullptr, 1, I.ncol, I.nrow, kHead, s);
  if (!rc) rc = middle_sweeps<T>(p->logn, d, nullptr, nullptr, 1, I.ncol, I.nrow, nsteps, p->bar, p->err, s,
                                 p->spin_limit);
  if (!rc) rc = launch_sweep<T>(p->logn, d, nullptr, nullptr, 1, I.ncol, I.nrow, kTail, s);
  return rc;
}

// Steps on another state buffer of the plan's geometry (descriptor slot 2),
// with the plan's current phase tables.
template <typename T>
static int steps_on_impl(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s) {
  MPInst<T> I = make_inst<T>(p, nullptr);
  I.u = (T*)state;
  MPInst<T>* d = (MPInst<T>*)p->desc + 2;
  LSP_CUDA_TRY(cudaMemcpyAsync(d, &I, sizeof(I), cudaMemcpyHostToDevice, s));
  int rc = launch_sweep<T>(p->logn, d, nullptr, nullptr, 1, I.ncol, I.nrow, kHead, s);
  if (!rc) rc = middle_sweeps<T>(p->logn, d, nullptr, nullptr, 1, I.ncol, I.nrow, nsteps, p->bar, p->err, s,
                                 p->spin_limit);
  if (!rc) rc = launch_sweep<T>(p->logn, d, nullptr, nullptr, 1, I.ncol, I.nrow, kTail, s);
  return rc;
}

int multipass_steps_on(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s) {
  return p->prec == LSP_C64 ? steps_on_impl<float2>(p, state, nsteps, s)
                            : steps_on_impl<double2>(p, state, nsteps, s);
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
  int rc = launch_sweep<T>(p->logn, d, nullptr, nullptr, 1, I.ncol, I.nrow, kColFwd, s);
  if (!rc) rc = launch_sweep<T>(p->logn, d, nullptr, nullptr, 1, I.ncol, I.nrow, kRowFwd, s);
  return rc;
}

int multipass_steps(lsp_plan p, int64_t nsteps, cudaStream_t s) {
  return p->prec == LSP_C64 ? steps_impl<float2>(p, nsteps, s) : steps_impl<double2>(p, nsteps, s);
}

int multipass_spectral(lsp_plan p, cudaStream_t s) {
  return p->prec == LSP_C64 ? spectral_impl<float2>(p, s) : spectral_impl<double2>(p, s);
}

// Batching: descriptors of many same-size plans in one device array; the tile
// maps enumerate (instance, local tile) over all of them.
int multipass_desc_size(int prec) { return multipass_desc_bytes(prec); }

void multipass_fill_desc(lsp_plan p, void* host_out, int* ncol, int* nrow) {
  if (p->prec == LSP_C64) {
    MPInst<float2> I = make_inst<float2>(p, nullptr);
    memcpy(host_out, &I, sizeof(I));
    *ncol = I.ncol; *nrow = I.nrow;
  } else {
    MPInst<double2> I = make_inst<double2>(p, nullptr);
    memcpy(host_out, &I, sizeof(I));
    *ncol = I.ncol; *nrow = I.nrow;
  }
}

template <typename T>
static int batch_impl(int m, const void* ddesc, const int2* colmap, const int2* rowmap, int ninst, int total_col,
                      int total_row, int64_t nsteps, unsigned* bar, int* err, cudaStream_t s) {
  const MPInst<T>* d = (const MPInst<T>*)ddesc;
  int rc = launch_sweep<T>(m, d, colmap, rowmap, ninst, total_col, total_row, kHead, s);
  if (!rc) rc = middle_sweeps<T>(m, d, colmap, rowmap, ninst, total_col, total_row, nsteps, bar, err, s);
  if (!rc) rc = launch_sweep<T>(m, d, colmap, rowmap, ninst, total_col, total_row, kTail, s);
  return rc;
}

int multipass_batch_steps(int prec, int m, const void* ddesc, const int2* colmap, const int2* rowmap, int ninst,
                          int total_col, int total_row, int64_t nsteps, unsigned* bar, int* err, cudaStream_t s) {
  return prec == LSP_C64 ? batch_impl<float2>(m, ddesc, colmap, rowmap, ninst, total_col, total_row, nsteps, bar, err, s)
                         : batch_impl<double2>(m, ddesc, colmap, rowmap, ninst, total_col, total_row, nsteps, bar, err, s);
}

}  // namespace lsp
