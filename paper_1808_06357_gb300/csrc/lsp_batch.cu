// Batched Strang stepping: many independent instances (uneven n, d and dt)
// advanced together.  Instances are grouped once at creation:
//  * SMEM-resident instances: one CTA per instance running all steps; one launch
//    per power-of-two size with the line kernel, one for all the others;
//  * multipass instances: one group per lattice size 2^m (kernels are
//    specialised per size); each group is a head sweep, one persistent
//    cooperative launch over the tiles of all its instances, and a tail sweep;
//  * rank-1 four-sweep instances of up to 2^22 points: one group per (size, K
//    form); each sweep is one launch over the tiles of all the group's instances,
//    and a call of 16 steps or more replays the groups' launches as a CUDA graph;
//  * other four-sweep instances (rank-2, larger rank-1; each fills the GPU by
//    itself): stepped one after another.
// Each instance's phase tables are built with its own dt on every call.
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <vector>

#include "lsp_internal.cuh"

using namespace lsp;

namespace {

struct DeviceGuard {
  int prev = 0;
  explicit DeviceGuard(int dev) { cudaGetDevice(&prev); cudaSetDevice(dev); }
  ~DeviceGuard() { cudaSetDevice(prev); }
};

void free_batch(lsp_batch b) {
  if (!b) return;
  for (auto& g : b->smalls) cudaFree(g.desc);
  for (auto& c : b->classes) {
    cudaFree(c.desc);
    cudaFree(c.colmap);
    cudaFree(c.rowmap);
  }
  for (auto& c : b->s4classes) s4_class_free(c);
  s2_group_free(b->s2group);
  if (b->s4_graph) cudaGraphExecDestroy(b->s4_graph);
  if (b->capture) cudaStreamDestroy(b->capture);
  cudaFree(b->bar);
  cudaFree(b->err);
  if (b->err_host) cudaFreeHost(b->err_host);
  delete b;
}

constexpr int64_t kGraphMinSteps = 16;

// The four-sweep groups' launches of one call: direct for short calls, else a CUDA
// graph captured on a private stream while (nsteps, descriptors) are unchanged.
int s4_batch_steps(lsp_batch b, int64_t nsteps, cudaStream_t s) {
  std::vector<unsigned char> key(sizeof(nsteps));
  memcpy(key.data(), &nsteps, sizeof(nsteps));
  for (auto& c : b->s4classes) {
    bool changed = false;
    int rc = s4_class_sync(c, b->plans, &changed, s);
    if (rc) return rc;
    key.insert(key.end(), c.inst_host.begin(), c.inst_host.end());
  }
  auto launch_all = [&](cudaStream_t st) {
    for (auto& c : b->s4classes) {
      int rc = s4_class_steps(c, b->prec, nsteps, st);
      if (rc) return rc;
    }
    return (int)LSP_OK;
  };
  if (nsteps < kGraphMinSteps) return launch_all(s);
  if (!b->s4_graph || key != b->s4_graph_key) {
    if (b->s4_graph) { cudaGraphExecDestroy(b->s4_graph); b->s4_graph = nullptr; }
    if (!b->capture) LSP_CUDA_TRY(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking));
    LSP_CUDA_TRY(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
    const int rc = launch_all(b->capture);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->capture, &g);
    if (rc || ec != cudaSuccess) { if (g) cudaGraphDestroy(g); return rc ? rc : LSP_ERR_CUDA; }
    const cudaError_t ei = cudaGraphInstantiate(&b->s4_graph, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) { b->s4_graph = nullptr; return LSP_ERR_CUDA; }
    b->s4_graph_key = key;
  }
  LSP_CUDA_TRY(cudaGraphLaunch(b->s4_graph, s));
  return LSP_OK;
}

}  // namespace

extern "C" {

int lsp_batch_create(lsp_batch* out, const lsp_plan* plans, int count) {
  if (!out) return LSP_ERR_BAD_ARG;
  *out = nullptr;
  if (!plans || count < 1) return LSP_ERR_BAD_ARG;
  for (int i = 0; i < count; ++i)
    if (!plans[i]) return LSP_ERR_BAD_ARG;
  const int prec = plans[0]->prec, dev = plans[0]->device;
  for (int i = 1; i < count; ++i)
    if (plans[i]->prec != prec || plans[i]->device != dev) return LSP_ERR_UNSUPPORTED;

  lsp_batch b = new (std::nothrow) lsp_batch_s();
  if (!b) return LSP_ERR_OOM;
  b->plans.assign(plans, plans + count);
  for (int i = 0; i < count; ++i) b->paths.push_back(plans[i]->path);
  b->prec = prec;
  b->device = dev;
  DeviceGuard g(dev);
  auto fail = [&](int code) { free_batch(b); return code; };

  std::map<int, std::vector<int>> by_m, by_line;
  std::map<std::pair<int, bool>, std::vector<int>> by_m4;
  for (int i = 0; i < count; ++i) {
    if (plans[i]->path == kPathMultipass) by_m[plans[i]->logn].push_back(i);
    else if (s2_batchable(plans[i])) b->s2group.ids.push_back(i);
    else if (s4_batchable(plans[i])) by_m4[{plans[i]->logn, plans[i]->kidx != nullptr}].push_back(i);
    else if (plans[i]->path == kPathRank2 || plans[i]->path == kPathRank1x4 || plans[i]->path == kPathRank1x2 ||
             plans[i]->path == kPathMixed)
      b->seq_ids.push_back(i);
    else by_line[small_line_logn(plans[i])].push_back(i);
  }
  for (auto& kv : by_m4) {
    b->s4classes.emplace_back();
    lsp_batch_s::S4Class& c = b->s4classes.back();
    c.m = kv.first.first;
    c.kidx = kv.first.second;
    c.ids = kv.second;
    int rc = s4_class_init(c, b->plans);
    bool changed = false;
    if (!rc) rc = s4_class_sync(c, b->plans, &changed, nullptr);
    if (!rc && cudaStreamSynchronize(nullptr) != cudaSuccess) rc = LSP_ERR_CUDA;
    if (rc) return fail(rc);
  }
  if (!b->s2group.ids.empty()) {
    int rc = s2_group_init(b->s2group, b->plans);
    if (rc) return fail(rc);
  }
  // SMEM-resident groups
  for (auto& kv : by_line) {
    b->smalls.emplace_back();
    lsp_batch_s::SmallGroup& sg = b->smalls.back();
    sg.line_logn = kv.first;
    sg.ids = kv.second;
    const size_t ds = (size_t)small_desc_size(prec);
    std::vector<unsigned char> host(ds * sg.ids.size());
    for (size_t k = 0; k < sg.ids.size(); ++k) {
      lsp_plan p = plans[sg.ids[k]];
      small_fill_desc(p, host.data() + k * ds);
      sg.max_n = std::max(sg.max_n, (int)p->ntot);
    }
    if (cudaMalloc(&sg.desc, host.size()) != cudaSuccess) return fail(LSP_ERR_OOM);
    if (cudaMemcpy(sg.desc, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(LSP_ERR_CUDA);
  }
  // one class per lattice size
  const size_t ds = (size_t)multipass_desc_size(prec);
  for (auto& kv : by_m) {
    lsp_batch_s::Class c;
    c.m = kv.first;
    c.ids = kv.second;
    std::vector<unsigned char> host(ds * c.ids.size());
    std::vector<int2> cm, rm;
    for (size_t k = 0; k < c.ids.size(); ++k) {
      int ncol = 0, nrow = 0;
      multipass_fill_desc(plans[c.ids[k]], host.data() + k * ds, &ncol, &nrow);
      for (int t = 0; t < ncol; ++t) cm.push_back(make_int2((int)k, t));
      for (int t = 0; t < nrow; ++t) rm.push_back(make_int2((int)k, t));
    }
    c.total_col = (int)cm.size();
    c.total_row = (int)rm.size();
    b->classes.push_back(c);
    lsp_batch_s::Class& cc = b->classes.back();
    if (cudaMalloc(&cc.desc, host.size()) != cudaSuccess || cudaMalloc(&cc.colmap, cm.size() * sizeof(int2)) != cudaSuccess ||
        cudaMalloc(&cc.rowmap, rm.size() * sizeof(int2)) != cudaSuccess)
      return fail(LSP_ERR_OOM);
    if (cudaMemcpy(cc.desc, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(cc.colmap, cm.data(), cm.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(cc.rowmap, rm.data(), rm.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(LSP_ERR_CUDA);
  }
  if (cudaMalloc(&b->bar, 256) != cudaSuccess || cudaMalloc(&b->err, 256) != cudaSuccess) return fail(LSP_ERR_OOM);
  if (cudaMemset(b->err, 0, 256) != cudaSuccess) return fail(LSP_ERR_CUDA);
  if (cudaHostAlloc((void**)&b->err_host, sizeof(int), cudaHostAllocDefault) != cudaSuccess) return fail(LSP_ERR_OOM);
  *b->err_host = 0;
  *out = b;
  return LSP_OK;
}

int lsp_batch_steps(lsp_batch b, const double* dt, int64_t nsteps, void* stream) {
  if (!b || !dt || nsteps < 0) return LSP_ERR_BAD_ARG;
  for (size_t i = 0; i < b->plans.size(); ++i)
    if (!isfinite(dt[i]) || b->plans[i]->path != b->paths[i]) return LSP_ERR_BAD_ARG;
  if (*b->err_host != 0) return *b->err_host;
  if (nsteps == 0) return LSP_OK;
  DeviceGuard g(b->device);
  cudaStream_t s = (cudaStream_t)stream;
  for (size_t i = 0; i < b->plans.size(); ++i) {
    int rc = build_phase_tables(b->plans[i], dt[i], s);
    if (rc) return rc;
  }
  for (auto& sg : b->smalls) {
    int rc = small_batch_launch(b->prec, sg.desc, (int)sg.ids.size(), sg.max_n, sg.line_logn, nsteps, s);
    if (rc) return rc;
  }
  if (!b->s4classes.empty()) {
    int rc = s4_batch_steps(b, nsteps, s);
    if (rc) return rc;
  }
  if (!b->s2group.ids.empty()) {
    int rc = s2_group_steps(b->s2group, b->plans, nsteps, b->err, s);
    if (rc) return rc;
  }
  for (int i : b->seq_ids) {     // each fills the GPU by itself
    lsp_plan p = b->plans[i];
    int rc = path_steps_on(p, p->u, nsteps, s);
    if (rc) return rc;
    LSP_CUDA_TRY(cudaMemcpyAsync(p->err_host, p->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  }
  for (auto& c : b->classes) {
    int rc = multipass_batch_steps(b->prec, c.m, c.desc, c.colmap, c.rowmap, (int)c.ids.size(), c.total_col,
                                   c.total_row, nsteps, b->bar, b->err, s);
    if (rc) return rc;
  }
  LSP_CUDA_TRY(cudaMemcpyAsync(b->err_host, b->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  return LSP_OK;
}

int lsp_batch_status(lsp_batch b, void* stream) {
  if (!b) return LSP_ERR_BAD_ARG;
  DeviceGuard g(b->device);
  LSP_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  if (*b->err_host) return *b->err_host;
  for (int i : b->seq_ids)                 // instances stepped by their own plan's kernels
    if (*b->plans[i]->err_host) return *b->plans[i]->err_host;
  return LSP_OK;
}

void lsp_batch_destroy(lsp_batch b) {
  if (!b) return;
  DeviceGuard g(b->device);
  cudaDeviceSynchronize();
  free_batch(b);
}

}  // extern "C"
