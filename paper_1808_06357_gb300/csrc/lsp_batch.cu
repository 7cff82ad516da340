// Batched Strang stepping: many independent instances (uneven n, d and dt)
// advanced together.  Instances are grouped once at creation:
//  * SMEM-resident instances: one launch, one CTA per instance, all steps;
//  * multipass instances: one group per lattice size 2^m (kernels are
//    specialised per size); each group is a head sweep, one persistent
//    cooperative launch over the tiles of all its instances, and a tail sweep;
//  * four-sweep instances (rank-2, and rank-1 beyond the two-sweep sizes;
//    2^24 points and more, each enough to fill the GPU): stepped one after another.
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
  cudaFree(b->small_desc);
  for (auto& c : b->classes) {
    cudaFree(c.desc);
    cudaFree(c.colmap);
    cudaFree(c.rowmap);
  }
  cudaFree(b->bar);
  cudaFree(b->err);
  if (b->err_host) cudaFreeHost(b->err_host);
  delete b;
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

  std::map<int, std::vector<int>> by_m;
  for (int i = 0; i < count; ++i) {
    if (plans[i]->path == kPathMultipass) by_m[plans[i]->logn].push_back(i);
    else if (plans[i]->path == kPathRank2 || plans[i]->path == kPathRank1x4) b->seq_ids.push_back(i);
    else b->small_ids.push_back(i);
  }
  // SMEM-resident group
  if (!b->small_ids.empty()) {
    const size_t ds = (size_t)small_desc_size(prec);
    std::vector<unsigned char> host(ds * b->small_ids.size());
    for (size_t k = 0; k < b->small_ids.size(); ++k) {
      lsp_plan p = plans[b->small_ids[k]];
      small_fill_desc(p, host.data() + k * ds);
      b->small_max_n = std::max(b->small_max_n, (int)p->ntot);
    }
    if (cudaMalloc(&b->small_desc, host.size()) != cudaSuccess) return fail(LSP_ERR_OOM);
    if (cudaMemcpy(b->small_desc, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess)
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
  if (!b->small_ids.empty()) {
    int rc = small_batch_launch(b->prec, b->small_desc, (int)b->small_ids.size(), b->small_max_n, nsteps, s);
    if (rc) return rc;
  }
  for (int i : b->seq_ids) {     // each fills the GPU by itself
    int rc = s4_steps_on(b->plans[i], b->plans[i]->u, nsteps, s);
    if (rc) return rc;
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
  return *b->err_host;
}

void lsp_batch_destroy(lsp_batch b) {
  if (!b) return;
  DeviceGuard g(b->device);
  cudaDeviceSynchronize();
  free_batch(b);
}

}  // extern "C"
