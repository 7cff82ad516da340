// Host side of the four-sweep Strang step (rank-2 lattices, and rank-1
// lattices on the four-sweep schedule): descriptors, launches, step driver,
// spectral output.
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "lsp_sweep4.cuh"

namespace lsp {

// Template shape of a plan: rank-2 (M1, M2) = (log2 n1, log2 n2); rank-1
// (M1, M2) = (log2 N2, log2 N1), rows of N1 points.
static bool s4_lookup(lsp_plan p, S4Kernels* k) {
  if (p->path == kPathRank2) return s4_kernels_rank2(p->prec, p->logN1, p->logN2, k);
  if (p->path == kPathRank1x4) return s4_kernels_rank1(p->prec, p->logn, k);
  return false;
}

bool s4_supports_rank2(int prec, int m1, int m2) {
  S4Kernels k;
  return s4_kernels_rank2(prec, m1, m2, &k);
}

bool s4_supports_rank1(int prec, int m) {
  S4Kernels k;
  return s4_kernels_rank1(prec, m, &k);
}

template <typename T> static S4Inst<T> s4_inst(lsp_plan p, void* state) {
  S4Inst<T> I;
  memset(&I, 0, sizeof(I));   // padding too: descriptors are compared bytewise
  I.u = (T*)state;
  I.Ph = (const T*)p->Ph;
  I.Pf = (const T*)p->Pf;
  I.K = (const T*)p->K;
  const T* tw = (const T*)p->tw_pass;
  I.tw_rows = tw;
  I.tw_a = tw + p->twr_entries;
  I.tw_b = tw + p->twr_entries + p->twa_entries;
  I.tw_col = (const T*)p->tw_line;
  I.tw_bl = (const T*)p->tw_coarse;
  I.tw_bf = (const T*)p->tw_fine;
  I.spec = (double2*)p->stage;
  I.err = p->err;
  I.kidx = p->kidx;
  I.klut = (const T*)p->klut;
  I.nlut = p->klut ? (int)p->max_norm2 + 1 : 0;
  I.inv_n = (decltype(I.inv_n))(1.0 / (double)p->ntot);
  return I;
}

// Grid of one sweep kernel: as many CTAs as fit on the device at once (at most
// one per tile), computed once per (device, kernel).
static int s4_grid(const void* fn, int nt, size_t smem, int* grid) {
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

template <typename T> static int s4_launch(const void* fn, const S4Inst<T>& I, int ntiles, cudaStream_t s) {
  constexpr int NT = S4Cfg<T>::NT;
  constexpr size_t smem = (size_t)S4Cfg<T>::TILE * sizeof(T);   // exchange buffer
  int grid = 0;
  int rc = s4_grid(fn, NT, smem, &grid);
  if (rc) return rc;
  grid = std::max(1, std::min(ntiles, grid));
  void* args[] = {(void*)&I};
  LSP_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(NT), args, smem, s));
  return LSP_OK;
}

// N steps: P-sweep head, then per step the three other sweeps and the next
// P-sweep (mid), and the P-sweep tail.  Sweep geometries: rows (0), A / X (1), B / Y (2).
template <typename T> static int s4_launch_steps(lsp_plan p, const S4Inst<T>& I, int64_t nsteps, cudaStream_t s) {
  S4Kernels K;
  if (!s4_lookup(p, &K)) return LSP_ERR_UNSUPPORTED;
  const bool r2 = p->path == kPathRank2;
  // kernel, geometry of each sweep of a step in order
  const int head = r2 ? kR2Head : kXHead, mid = r2 ? kR2Mid : kXMid, tail = r2 ? kR2Tail : kXTail;
  const int pg = r2 ? 0 : 1;                                       // geometry of the P sweep
  const int seq[3] = {r2 ? kR2A : kY, r2 ? kR2B : kZ, r2 ? kR2AInv : kYInv};
  const int geo[3] = {r2 ? 1 : 2, r2 ? 2 : 0, r2 ? 1 : 2};
  int rc = LSP_OK;
  const void* kin = I.kidx ? K.k_kidx : K.k[seq[1]];                // the K sweep
  for (int64_t st = 0; st < nsteps && !rc; ++st) {
    rc = s4_launch<T>(K.k[st == 0 ? head : mid], I, K.ntiles[pg], s);
    for (int i = 0; i < 3 && !rc; ++i) rc = s4_launch<T>(i == 1 ? kin : K.k[seq[i]], I, K.ntiles[geo[i]], s);
  }
  if (!rc) rc = s4_launch<T>(K.k[tail], I, K.ntiles[pg], s);
  return rc;
}

// The same launches as s4_launch_steps with an event recorded after each one, for
// per-sweep durations: ms[0] P sweeps between steps (rows / X mid), ms[1] A / Y,
// ms[2] the K sweep (B / Z), ms[3] A^-1 / Y^-1, each the mean over the call.
template <typename T> static int s4_sweep_times_impl(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s,
                                                     double* ms) {
  S4Kernels K;
  if (!s4_lookup(p, &K)) return LSP_ERR_UNSUPPORTED;
  const S4Inst<T> I = s4_inst<T>(p, state);
  const bool r2 = p->path == kPathRank2;
  const int head = r2 ? kR2Head : kXHead, mid = r2 ? kR2Mid : kXMid, tail = r2 ? kR2Tail : kXTail;
  const int pg = r2 ? 0 : 1;
  const int seq[3] = {r2 ? kR2A : kY, r2 ? kR2B : kZ, r2 ? kR2AInv : kYInv};
  const int geo[3] = {r2 ? 1 : 2, r2 ? 2 : 0, r2 ? 1 : 2};
  const void* kin = I.kidx ? K.k_kidx : K.k[seq[1]];
  std::vector<cudaEvent_t> ev((size_t)(4 * nsteps + 2), nullptr);
  int rc = LSP_OK;
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) { rc = LSP_ERR_CUDA; break; }
  std::vector<int> kind;                                // sweep class of launch i (-1: head / tail)
  size_t k = 0;
  if (!rc) rc = cudaEventRecord(ev[k++], s) == cudaSuccess ? LSP_OK : LSP_ERR_CUDA;
  for (int64_t st = 0; st < nsteps && !rc; ++st) {
    rc = s4_launch<T>(K.k[st == 0 ? head : mid], I, K.ntiles[pg], s);
    kind.push_back(st == 0 ? -1 : 0);
    if (!rc) rc = cudaEventRecord(ev[k++], s) == cudaSuccess ? LSP_OK : LSP_ERR_CUDA;
    for (int i = 0; i < 3 && !rc; ++i) {
      rc = s4_launch<T>(i == 1 ? kin : K.k[seq[i]], I, K.ntiles[geo[i]], s);
      kind.push_back(1 + i);
      if (!rc) rc = cudaEventRecord(ev[k++], s) == cudaSuccess ? LSP_OK : LSP_ERR_CUDA;
    }
  }
  if (!rc) {
    rc = s4_launch<T>(K.k[tail], I, K.ntiles[pg], s);
    kind.push_back(-1);
    if (!rc) rc = cudaEventRecord(ev[k++], s) == cudaSuccess ? LSP_OK : LSP_ERR_CUDA;
  }
  if (!rc && cudaEventSynchronize(ev[k - 1]) != cudaSuccess) rc = LSP_ERR_CUDA;
  if (!rc) {
    double sum[4] = {0, 0, 0, 0};
    int cnt[4] = {0, 0, 0, 0};
    for (size_t i = 0; i < kind.size(); ++i) {
      if (kind[i] < 0) continue;
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
      sum[kind[i]] += t;
      cnt[kind[i]] += 1;
    }
    for (int c = 0; c < 4; ++c) ms[c] = cnt[c] ? sum[c] / cnt[c] : -1.0;
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  return rc;
}

int s4_sweep_times(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s, double* ms) {
  return p->prec == LSP_C64 ? s4_sweep_times_impl<float2>(p, state, nsteps, s, ms)
                            : s4_sweep_times_impl<double2>(p, state, nsteps, s, ms);
}

constexpr int64_t kGraphMinSteps = 16;

// The 4 N + 1 launches of a call, captured once as a CUDA graph on a private
// stream and replayed on the caller's stream while (nsteps, kernel arguments) are
// unchanged: the sweeps then follow one another without per-launch host work.
template <typename T> static int s4_steps_impl(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s) {
  const S4Inst<T> I = s4_inst<T>(p, state);
  if (nsteps < kGraphMinSteps) return s4_launch_steps<T>(p, I, nsteps, s);   // short calls (adjoint, stages)
  std::vector<unsigned char> key(sizeof(I) + sizeof(nsteps) + sizeof(int));
  memcpy(key.data(), &I, sizeof(I));
  memcpy(key.data() + sizeof(I), &nsteps, sizeof(nsteps));
  memcpy(key.data() + sizeof(I) + sizeof(nsteps), &p->path, sizeof(int));
  if (!p->s4_graph || key != p->s4_graph_key) {
    if (p->s4_graph) { cudaGraphExecDestroy(p->s4_graph); p->s4_graph = nullptr; }
    if (!p->capture) LSP_CUDA_TRY(cudaStreamCreateWithFlags(&p->capture, cudaStreamNonBlocking));
    // kernel attributes and grid sizes are set and cached before the capture
    S4Kernels K;
    if (!s4_lookup(p, &K)) return LSP_ERR_UNSUPPORTED;
    int grid = 0, rc = LSP_OK;
    for (const void* fn : K.k)
      if (fn && (rc = s4_grid(fn, S4Cfg<T>::NT, (size_t)S4Cfg<T>::TILE * sizeof(T), &grid))) return rc;
    if (K.k_kidx && (rc = s4_grid(K.k_kidx, S4Cfg<T>::NT, (size_t)S4Cfg<T>::TILE * sizeof(T), &grid))) return rc;
    LSP_CUDA_TRY(cudaStreamBeginCapture(p->capture, cudaStreamCaptureModeThreadLocal));
    rc = s4_launch_steps<T>(p, I, nsteps, p->capture);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(p->capture, &g);
    if (rc || ec != cudaSuccess) { if (g) cudaGraphDestroy(g); return rc ? rc : LSP_ERR_CUDA; }
    const cudaError_t ei = cudaGraphInstantiate(&p->s4_graph, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) { p->s4_graph = nullptr; return LSP_ERR_CUDA; }
    p->s4_graph_key = key;
  }
  LSP_CUDA_TRY(cudaGraphLaunch(p->s4_graph, s));
  return LSP_OK;
}

// Spectral coefficients of the current state into p->stage (chi order, c128),
// on a scratch copy of the state.
template <typename T> static int s4_spectral_impl(lsp_plan p, cudaStream_t s) {
  S4Kernels K;
  if (!s4_lookup(p, &K)) return LSP_ERR_UNSUPPORTED;
  LSP_CUDA_TRY(cudaMemcpyAsync(p->work, p->u, (size_t)p->ntot * sizeof(T), cudaMemcpyDeviceToDevice, s));
  const S4Inst<T> I = s4_inst<T>(p, p->work);
  int rc;
  if (p->path == kPathRank2) {
    rc = s4_launch<T>(K.k[kR2RowFwd], I, K.ntiles[0], s);
    if (!rc) rc = s4_launch<T>(K.k[kR2A], I, K.ntiles[1], s);
    if (!rc) rc = s4_launch<T>(K.k[kR2BFwd], I, K.ntiles[2], s);
  } else {
    rc = s4_launch<T>(K.k[kXFwd], I, K.ntiles[1], s);
    if (!rc) rc = s4_launch<T>(K.k[kY], I, K.ntiles[2], s);
    if (!rc) rc = s4_launch<T>(K.k[kZFwd], I, K.ntiles[0], s);
  }
  return rc;
}

// --------------------------------------------------------------------------
// Batches: all instances of one rank-1 size in each sweep's launch
// --------------------------------------------------------------------------
bool s4_batchable(lsp_plan p) {
  S4Kernels K;
  return p->path == kPathRank1x4 && s4_lookup(p, &K) && K.b[kXHead] != nullptr;
}

int s4_class_init(lsp_batch_s::S4Class& c, const std::vector<lsp_plan>& plans) {
  S4Kernels K;
  if (c.ids.empty() || !s4_lookup(plans[c.ids[0]], &K)) return LSP_ERR_UNSUPPORTED;
  for (int g = 0; g < 3; ++g) {
    std::vector<int2> map;
    for (size_t k = 0; k < c.ids.size(); ++k)
      for (int t = 0; t < K.ntiles[g]; ++t) map.push_back(make_int2((int)k, t));
    c.total[g] = (int)map.size();
    if (cudaMalloc(&c.map[g], map.size() * sizeof(int2)) != cudaSuccess) return LSP_ERR_OOM;
    LSP_CUDA_TRY(cudaMemcpy(c.map[g], map.data(), map.size() * sizeof(int2), cudaMemcpyHostToDevice));
  }
  // kernel attributes and grid sizes are set and cached here, outside any graph capture
  static_assert(S4Cfg<float2>::NT == S4Cfg<double2>::NT && S4Cfg<float2>::TILE == S4Cfg<double2>::TILE, "");
  const size_t smem = (size_t)S4Cfg<float2>::TILE * (plans[c.ids[0]]->prec == LSP_C64 ? 8 : 16);
  int grid = 0, rc = LSP_OK;
  for (const void* fn : K.b)
    if (fn && (rc = s4_grid(fn, S4Cfg<float2>::NT, smem, &grid))) return rc;
  if (K.b_kidx && (rc = s4_grid(K.b_kidx, S4Cfg<float2>::NT, smem, &grid))) return rc;
  return LSP_OK;
}

template <typename T>
static int s4_class_sync_impl(lsp_batch_s::S4Class& c, const std::vector<lsp_plan>& plans, bool* changed,
                              cudaStream_t s) {
  std::vector<unsigned char> h(c.ids.size() * sizeof(S4Inst<T>));
  for (size_t k = 0; k < c.ids.size(); ++k) {
    lsp_plan p = plans[c.ids[k]];
    if ((p->kidx != nullptr) != c.kidx) return LSP_ERR_BAD_ARG;   // K form changed since creation
    const S4Inst<T> I = s4_inst<T>(p, p->u);
    memcpy(h.data() + k * sizeof(I), &I, sizeof(I));
  }
  *changed = h != c.inst_host;
  if (!*changed) return LSP_OK;
  // Launches of an earlier call on this stream may still read the old descriptors: the
  // copy is ordered after them on the call's stream (a pageable-source copy returns once
  // the source is staged, so h may go out of scope).  Not capturable into a graph.
  if (!c.inst && cudaMalloc(&c.inst, h.size()) != cudaSuccess) return LSP_ERR_OOM;
  LSP_CUDA_TRY(cudaMemcpyAsync(c.inst, h.data(), h.size(), cudaMemcpyHostToDevice, s));
  c.inst_host = h;
  return LSP_OK;
}

int s4_class_sync(lsp_batch_s::S4Class& c, const std::vector<lsp_plan>& plans, bool* changed, cudaStream_t s) {
  const int prec = plans[c.ids[0]]->prec;
  return prec == LSP_C64 ? s4_class_sync_impl<float2>(c, plans, changed, s)
                         : s4_class_sync_impl<double2>(c, plans, changed, s);
}

template <typename T> static int s4b_launch(const void* fn, const lsp_batch_s::S4Class& c, int g, cudaStream_t s) {
  constexpr int NT = S4Cfg<T>::NT;
  constexpr size_t smem = (size_t)S4Cfg<T>::TILE * sizeof(T);
  int grid = 0;
  int rc = s4_grid(fn, NT, smem, &grid);
  if (rc) return rc;
  grid = std::max(1, std::min(c.total[g], grid));
  S4Batch<T> B{(const S4Inst<T>*)c.inst, c.map[g], c.total[g]};
  void* args[] = {(void*)&B};
  LSP_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(NT), args, smem, s));
  return LSP_OK;
}

// The same sweep order as one instance's steps (s4_launch_steps), over all instances.
template <typename T> static int s4_class_steps_impl(const lsp_batch_s::S4Class& c, int64_t nsteps, cudaStream_t s) {
  S4Kernels K;
  if (!s4_kernels_rank1(sizeof(T) == 8 ? LSP_C64 : LSP_C128, c.m, &K) || !K.b[kXHead]) return LSP_ERR_UNSUPPORTED;
  const void* kin = c.kidx ? K.b_kidx : K.b[kZ];
  int rc = LSP_OK;
  for (int64_t st = 0; st < nsteps && !rc; ++st) {
    rc = s4b_launch<T>(K.b[st == 0 ? kXHead : kXMid], c, 1, s);
    if (!rc) rc = s4b_launch<T>(K.b[kY], c, 2, s);
    if (!rc) rc = s4b_launch<T>(kin, c, 0, s);
    if (!rc) rc = s4b_launch<T>(K.b[kYInv], c, 2, s);
  }
  if (!rc) rc = s4b_launch<T>(K.b[kXTail], c, 1, s);
  return rc;
}

int s4_class_steps(const lsp_batch_s::S4Class& c, int prec, int64_t nsteps, cudaStream_t s) {
  return prec == LSP_C64 ? s4_class_steps_impl<float2>(c, nsteps, s) : s4_class_steps_impl<double2>(c, nsteps, s);
}

void s4_class_free(lsp_batch_s::S4Class& c) {
  cudaFree(c.inst);
  for (int g = 0; g < 3; ++g) cudaFree(c.map[g]);
  c.inst = nullptr;
}

int s4_steps_on(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s) {
  return p->prec == LSP_C64 ? s4_steps_impl<float2>(p, state, nsteps, s) : s4_steps_impl<double2>(p, state, nsteps, s);
}

int s4_spectral(lsp_plan p, cudaStream_t s) {
  return p->prec == LSP_C64 ? s4_spectral_impl<float2>(p, s) : s4_spectral_impl<double2>(p, s);
}

}  // namespace lsp
