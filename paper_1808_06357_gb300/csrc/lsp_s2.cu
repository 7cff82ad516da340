// Host side of the TMA-fed two-sweep rank-1 path: tensor maps, descriptors,
// launches, the step driver (replayed as a CUDA graph) and spectral output.
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include <cudaTypedefs.h>

#include "lsp_s2.cuh"

namespace lsp {

constexpr int kS2MinLog = 16, kS2MaxLog = 24;

bool s2_kernels_16(int v, S2Kernels* k);
bool s2_kernels_17(int v, S2Kernels* k);
bool s2_kernels_18(int v, S2Kernels* k);
bool s2_kernels_19(int v, S2Kernels* k);
bool s2_kernels_20(int v, S2Kernels* k);
bool s2_kernels_21(int v, S2Kernels* k);
bool s2_kernels_22(int v, S2Kernels* k);
bool s2_kernels_23(int v, S2Kernels* k);
bool s2_kernels_24(int v, S2Kernels* k);

bool s2_kernels_for(int m, int v, S2Kernels* k) {
  switch (m) {
    case 16: return s2_kernels_16(v, k);
    case 17: return s2_kernels_17(v, k);
    case 18: return s2_kernels_18(v, k);
    case 19: return s2_kernels_19(v, k);
    case 20: return s2_kernels_20(v, k);
    case 21: return s2_kernels_21(v, k);
    case 22: return s2_kernels_22(v, k);
    case 23: return s2_kernels_23(v, k);
    case 24: return s2_kernels_24(v, k);
    default: return false;
  }
}

static bool s2_lookup(lsp_plan p, S2Kernels* k) { return s2_kernels_for(p->logn, p->s2_sched, k); }

bool s2_supports(int prec, int m) { return prec == LSP_C64 && m >= kS2MinLog && m <= kS2MaxLog; }

static PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
  });
  return fn;
}

// 2-D map of an n-point complex64 array viewed as N2 rows of N1 = 4096 elements of 8
// bytes, copied in boxes of C columns x BR rows.
static int encode_cols(CUtensorMap* map, const void* base, int m) {
  auto fn = encode_tiled();
  if (!fn) return LSP_ERR_CUDA;
  const int ln2 = m - kS2LogN1;
  const cuuint64_t dims[2] = {(cuuint64_t)1 << kS2LogN1, (cuuint64_t)1 << ln2};
  const cuuint64_t strides[1] = {((cuuint64_t)1 << kS2LogN1) * 8};
  const cuuint32_t box[2] = {(cuuint32_t)((1 << s2_logtile(m)) >> ln2), (cuuint32_t)std::min(1 << ln2, 256)};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? LSP_OK : LSP_ERR_CUDA;
}

static int s2_inst(lsp_plan p, void* state, double2* spec, S2Inst* I) {
  memset(I, 0, sizeof(*I));
  const int rc = encode_cols(&I->tu, state, p->logn);
  if (rc) return rc;
  I->u = (float2*)state;
  I->Ph = (const float2*)p->Ph;
  I->Pf = (const float2*)p->Pf;
  I->K = (const float2*)p->K;
  I->kidx = p->kidx;
  I->klut = (const float2*)p->klut;
  I->tw_rows = (const float2*)p->tw_pass;
  I->tw_cols = (const float2*)p->tw_pass + p->twr_entries;
  I->tw_coarse = (const float2*)p->tw_coarse;
  I->tw_fine = (const float2*)p->tw_fine;
  I->spec = spec;
  I->nlut = p->klut ? (int)p->max_norm2 + 1 : 0;
  I->inv_n = (float)(1.0 / (double)p->ntot);
  I->m = p->logn;
  return LSP_OK;
}

// Descriptor slots in p->s2desc: 0 the plan's state, 1 the spectral copy (p->work),
// 2 any other state buffer (rewritten per call, stream-ordered).
int s2_upload_desc(lsp_plan p) {
  if (!p->s2desc && cudaMalloc(&p->s2desc, 3 * sizeof(S2Inst)) != cudaSuccess) { cudaGetLastError(); return LSP_ERR_OOM; }
  S2Inst I[2];
  int rc = s2_inst(p, p->u, nullptr, &I[0]);
  if (!rc) rc = s2_inst(p, p->work, (double2*)p->stage, &I[1]);
  if (rc) return rc;
  LSP_CUDA_TRY(cudaMemcpy(p->s2desc, I, sizeof(I), cudaMemcpyHostToDevice));
  p->s2host0.assign((const unsigned char*)&I[0], (const unsigned char*)&I[0] + sizeof(S2Inst));
  return LSP_OK;
}

// Grid of one kernel: CTAs resident at once (cached per device and kernel).
static int s2_grid(const void* fn, size_t smem, int* grid, int nt = kS2NT) {
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

static int s2_launch(const void* fn, size_t smem, const S2Inst* inst, const int2* map, int ntiles, int* err,
                     long long spin_limit, cudaStream_t s, int nt = kS2NT) {
  int grid = 0;
  int rc = s2_grid(fn, smem, &grid, nt);
  if (rc) return rc;
  grid = std::max(1, std::min(ntiles, grid));
  S2Params P{inst, map, ntiles, err, spin_limit};
  void* args[] = {(void*)&P};
  LSP_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(nt), args, smem, s));
  return LSP_OK;
}

// Kernel attributes and grids of every kernel of size m, set outside any capture.
static int s2_prepare(const S2Kernels& K) {
  int grid = 0, rc = LSP_OK;
  for (int k = 0; k < kS2Kinds && !rc; ++k) rc = s2_grid(K.k[k], K.smem[k], &grid, K.nt);
  if (!rc) rc = s2_grid(K.row_kidx, K.smem_row_kidx, &grid, K.nt);
  return rc;
}

// N steps on the instance(s) of `inst`: head, N row sweeps with N - 1 mid sweeps between them, tail.
static int s2_launch_steps(const S2Kernels& K, bool kidx, const S2Inst* inst, const int2* map, int ntiles, int* err,
                           long long spin_limit, int64_t nsteps, cudaStream_t s) {
  const void* row = kidx ? K.row_kidx : K.k[kS2Row];
  const size_t row_smem = kidx ? K.smem_row_kidx : K.smem[kS2Row];
  int rc = s2_launch(K.k[kS2Head], K.smem[kS2Head], inst, map, ntiles, err, spin_limit, s, K.nt);
  for (int64_t st = 0; st < nsteps && !rc; ++st) {
    rc = s2_launch(row, row_smem, inst, map, ntiles, err, spin_limit, s, K.nt);
    if (!rc) rc = st + 1 < nsteps ? s2_launch(K.k[kS2Mid], K.smem[kS2Mid], inst, map, ntiles, err, spin_limit, s, K.nt)
                                  : s2_launch(K.k[kS2Tail], K.smem[kS2Tail], inst, map, ntiles, err, spin_limit, s, K.nt);
  }
  return rc;
}

constexpr int64_t kS2GraphMinSteps = 16;

// Steps on `state` (the plan's own state: descriptor slot 0, replayed from a captured graph
// for calls of 16 steps or more; another buffer: slot 2, plain launches).
int s2_steps_on(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s) {
  S2Kernels K;
  if (!s2_lookup(p, &K)) return LSP_ERR_UNSUPPORTED;
  int rc = s2_prepare(K);
  if (rc) return rc;
  const S2Inst* d = (const S2Inst*)p->s2desc;
  const bool kidx = p->kidx != nullptr;
  S2Inst I;
  if ((rc = s2_inst(p, state, nullptr, &I))) return rc;
  if (state != p->u || p->s2host0.size() != sizeof(I) || memcmp(p->s2host0.data(), &I, sizeof(I)) != 0) {
    // another buffer, or other phase tables (composed steps): descriptor slot 2, stream-ordered
    LSP_CUDA_TRY(cudaMemcpyAsync((S2Inst*)p->s2desc + 2, &I, sizeof(I), cudaMemcpyHostToDevice, s));
    return s2_launch_steps(K, kidx, d + 2, nullptr, K.ntiles, p->err, p->spin_limit, nsteps, s);
  }
  if (nsteps < kS2GraphMinSteps) return s2_launch_steps(K, kidx, d, nullptr, K.ntiles, p->err, p->spin_limit, nsteps, s);
  // graph key: nsteps, K form and wait limit (the descriptor itself lives at a fixed address)
  std::vector<unsigned char> key(sizeof(nsteps) + sizeof(int) + sizeof(long long) + sizeof(void*));
  const int form = kidx ? 1 : 0;
  memcpy(key.data(), &nsteps, sizeof(nsteps));
  memcpy(key.data() + sizeof(nsteps), &form, sizeof(int));
  memcpy(key.data() + sizeof(nsteps) + sizeof(int), &p->spin_limit, sizeof(long long));
  memcpy(key.data() + sizeof(nsteps) + sizeof(int) + sizeof(long long), &p->s2desc, sizeof(void*));
  key.push_back((unsigned char)p->s2_sched);           // the schedule's kernels
  key.push_back(0x52);                                  // distinct from the four-sweep paths' keys
  if (!p->s4_graph || key != p->s4_graph_key) {
    if (p->s4_graph) { cudaGraphExecDestroy(p->s4_graph); p->s4_graph = nullptr; }
    if (!p->capture) LSP_CUDA_TRY(cudaStreamCreateWithFlags(&p->capture, cudaStreamNonBlocking));
    LSP_CUDA_TRY(cudaStreamBeginCapture(p->capture, cudaStreamCaptureModeThreadLocal));
    rc = s2_launch_steps(K, kidx, d, nullptr, K.ntiles, p->err, p->spin_limit, nsteps, p->capture);
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

// Spectral coefficients of the current state into p->stage (chi order, c128), on p->work.
int s2_spectral(lsp_plan p, cudaStream_t s) {
  S2Kernels K;
  if (!s2_lookup(p, &K)) return LSP_ERR_UNSUPPORTED;
  int rc = s2_prepare(K);
  if (rc) return rc;
  LSP_CUDA_TRY(cudaMemcpyAsync(p->work, p->u, (size_t)p->ntot * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  const S2Inst* d = (const S2Inst*)p->s2desc + 1;
  rc = s2_launch(K.k[kS2ColFwd], K.smem[kS2ColFwd], d, nullptr, K.ntiles, p->err, p->spin_limit, s, K.nt);
  if (!rc) rc = s2_launch(K.k[kS2RowFwd], K.smem[kS2RowFwd], d, nullptr, K.ntiles, p->err, p->spin_limit, s, K.nt);
  return rc;
}

}  // namespace lsp

namespace lsp {

// The launches of s2 steps on `state` with an event after each: ms[0] the mean of the
// mid column sweeps, ms[2] of the row (K) sweeps; ms[1] = ms[3] = -1 (no such sweeps).
int s2_sweep_times(lsp_plan p, void* state, int64_t nsteps, cudaStream_t s, double* ms) {
  S2Kernels K;
  if (!s2_lookup(p, &K)) return LSP_ERR_UNSUPPORTED;
  int rc = s2_prepare(K);
  if (rc) return rc;
  S2Inst I;
  if ((rc = s2_inst(p, state, nullptr, &I))) return rc;
  S2Inst* d = (S2Inst*)p->s2desc + 2;
  LSP_CUDA_TRY(cudaMemcpyAsync(d, &I, sizeof(I), cudaMemcpyHostToDevice, s));
  const bool kidx = p->kidx != nullptr;
  const void* row = kidx ? K.row_kidx : K.k[kS2Row];
  const size_t row_smem = kidx ? K.smem_row_kidx : K.smem[kS2Row];
  std::vector<cudaEvent_t> ev((size_t)(2 * nsteps + 2), nullptr);
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) { rc = LSP_ERR_CUDA; break; }
  std::vector<int> kind;                    // 0 mid column sweep, 2 row sweep, -1 head / tail
  // The launches with an event after each, captured into a CUDA graph (events as event-record
  // nodes) and replayed, so that the sweeps follow one another as in a graph-replayed call.
  auto issue = [&](cudaStream_t st, unsigned flags) {
    size_t k = 0;
    kind.clear();
    auto rec = [&]() { return cudaEventRecordWithFlags(ev[k++], st, flags) == cudaSuccess ? LSP_OK : LSP_ERR_CUDA; };
    int r = rec();
    if (!r) r = s2_launch(K.k[kS2Head], K.smem[kS2Head], d, nullptr, K.ntiles, p->err, p->spin_limit, st, K.nt);
    kind.push_back(-1);
    if (!r) r = rec();
    for (int64_t step = 0; step < nsteps && !r; ++step) {
      r = s2_launch(row, row_smem, d, nullptr, K.ntiles, p->err, p->spin_limit, st, K.nt);
      kind.push_back(2);
      if (!r) r = rec();
      const bool last = step + 1 == nsteps;
      if (!r) r = s2_launch(K.k[last ? kS2Tail : kS2Mid], K.smem[last ? kS2Tail : kS2Mid], d, nullptr, K.ntiles,
                            p->err, p->spin_limit, st, K.nt);
      kind.push_back(last ? -1 : 0);
      if (!r) r = rec();
    }
    return r;
  };
  cudaGraphExec_t exec = nullptr;
  if (!rc) {
    cudaStream_t cap = nullptr;
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      const int r = issue(cap, cudaEventRecordExternal);
      ok = cudaStreamEndCapture(cap, &g) == cudaSuccess && r == LSP_OK &&
           cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
    }
    if (g) cudaGraphDestroy(g);
    if (cap) cudaStreamDestroy(cap);
    if (!ok) {                                           // no event nodes: plain launches
      cudaGetLastError();
      if (exec) { cudaGraphExecDestroy(exec); exec = nullptr; }
    }
  }
  if (!rc) rc = exec ? (cudaGraphLaunch(exec, s) == cudaSuccess ? LSP_OK : LSP_ERR_CUDA) : issue(s, cudaEventRecordDefault);
  if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = LSP_ERR_CUDA;
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
  if (exec) cudaGraphExecDestroy(exec);
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  return rc;
}

}  // namespace lsp

// --------------------------------------------------------------------------
// Batches: every path-4 instance (2^16 .. 2^23 points, mixed sizes) in one launch per sweep
// --------------------------------------------------------------------------
namespace lsp {

bool s2_batchable(lsp_plan p) {
  return p->path == kPathRank1x2 && p->logn >= kS2BatchMinLog && p->logn <= kS2BatchMaxLog;
}

int s2_group_init(lsp_batch_s::S2Group& g, const std::vector<lsp_plan>& plans) {
  // Instances in size order, so that the tiles that the CTAs hold at any one time are mostly of
  // one size (one code path, one twiddle table, the same tile set-up): C3's 140 instances of
  // 2^16 .. 2^20 points took 349 ms per 500-step call in size order, 386 ms in arbitrary order.
  std::stable_sort(g.ids.begin(), g.ids.end(), [&](int a, int b) { return plans[a]->logn < plans[b]->logn; });
  std::vector<int2> map;
  for (size_t k = 0; k < g.ids.size(); ++k) {
    const int nt = 1 << (plans[g.ids[k]]->logn - kS2LogN1);
    for (int t = 0; t < nt; ++t) map.push_back(make_int2((int)k, t));
  }
  g.total = (int)map.size();
  if (cudaMalloc(&g.map, map.size() * sizeof(int2)) != cudaSuccess ||
      cudaMalloc(&g.inst, g.ids.size() * sizeof(S2Inst)) != cudaSuccess) { cudaGetLastError(); return LSP_ERR_OOM; }
  LSP_CUDA_TRY(cudaMemcpy(g.map, map.data(), map.size() * sizeof(int2), cudaMemcpyHostToDevice));
  // kernel attributes and grids, outside any capture
  const S2BatchKernels K = s2_batch_kernels();
  int grid = 0;
  for (int k = 0; k < kS2Kinds; ++k) {
    if (!K.k[k]) continue;
    int rc = s2_grid(K.k[k], K.smem[k], &grid);
    if (rc) return rc;
  }
  return LSP_OK;
}

void s2_group_free(lsp_batch_s::S2Group& g) {
  cudaFree(g.inst);
  cudaFree(g.map);
  if (g.graph) cudaGraphExecDestroy(g.graph);
  if (g.capture) cudaStreamDestroy(g.capture);
  g = lsp_batch_s::S2Group();
}

// The group's launches of one call: one launch per sweep over every tile of every size.  (Each
// size's whole call in turn, so that the small sizes' state stays in L2, measured slower: 366
// against 349 ms per C3 call.)
static int s2_group_launches(const lsp_batch_s::S2Group& g, int64_t nsteps, int* err, cudaStream_t s) {
  const S2BatchKernels K = s2_batch_kernels();
  const S2Inst* d = (const S2Inst*)g.inst;
  auto go = [&](int kind) { return s2_launch(K.k[kind], K.smem[kind], d, g.map, g.total, err, kSpinLimit, s); };
  int rc = go(kS2Head);
  for (int64_t st = 0; st < nsteps && !rc; ++st) {
    rc = go(kS2Row);
    if (!rc) rc = go(st + 1 < nsteps ? kS2Mid : kS2Tail);
  }
  return rc;
}

// nsteps steps of every instance of the group; descriptors are refreshed (stream-ordered)
// when a plan's tables or state buffer moved, and calls of 16 steps or more replay a graph.
int s2_group_steps(lsp_batch_s::S2Group& g, const std::vector<lsp_plan>& plans, int64_t nsteps, int* err,
                   cudaStream_t s) {
  std::vector<unsigned char> h(g.ids.size() * sizeof(S2Inst));
  for (size_t k = 0; k < g.ids.size(); ++k) {
    lsp_plan p = plans[g.ids[k]];
    S2Inst I;
    int rc = s2_inst(p, p->u, nullptr, &I);
    if (rc) return rc;
    memcpy(h.data() + k * sizeof(S2Inst), &I, sizeof(I));
  }
  if (h != g.inst_host) {
    LSP_CUDA_TRY(cudaMemcpyAsync(g.inst, h.data(), h.size(), cudaMemcpyHostToDevice, s));
    g.inst_host = h;
  }
  if (nsteps < kS2GraphMinSteps) return s2_group_launches(g, nsteps, err, s);
  std::vector<unsigned char> key(sizeof(nsteps) + sizeof(err));
  memcpy(key.data(), &nsteps, sizeof(nsteps));
  memcpy(key.data() + sizeof(nsteps), &err, sizeof(err));
  if (!g.graph || key != g.graph_key) {
    if (g.graph) { cudaGraphExecDestroy(g.graph); g.graph = nullptr; }
    if (!g.capture) LSP_CUDA_TRY(cudaStreamCreateWithFlags(&g.capture, cudaStreamNonBlocking));
    LSP_CUDA_TRY(cudaStreamBeginCapture(g.capture, cudaStreamCaptureModeThreadLocal));
    const int rc = s2_group_launches(g, nsteps, err, g.capture);
    cudaGraph_t gr = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(g.capture, &gr);
    if (rc || ec != cudaSuccess) { if (gr) cudaGraphDestroy(gr); return rc ? rc : LSP_ERR_CUDA; }
    const cudaError_t ei = cudaGraphInstantiate(&g.graph, gr, 0);
    cudaGraphDestroy(gr);
    if (ei != cudaSuccess) { g.graph = nullptr; return LSP_ERR_CUDA; }
    g.graph_key = key;
  }
  LSP_CUDA_TRY(cudaGraphLaunch(g.graph, s));
  return LSP_OK;
}

}  // namespace lsp
