// Component-by-component construction of a reconstructing lattice (Sec. 3.1:
// lattices are built one generating-vector component at a time; the acceptance
// test is injectivity of h -> bin on the index set, Def. 2 / Thm 1(iii)).
//
// One launch tests one candidate: every row h of I computes its bin and claims
// the bin's slot in a table of one 8-byte word per bin, (tag << 32) | (row + 1),
// where the tag is a per-launch stamp (slots holding another tag are free, so the
// table is cleared once per call, not per candidate).  A row that finds its slot
// taken by a row with a different projection onto the first j + 1 coordinates
// reports a collision; rows with equal projections share a slot legitimately.
#include <string.h>

#include <algorithm>
#include <vector>

#include "lsp_internal.cuh"

namespace lsp {

constexpr int kCasRetries = 4096;   // bound of one row's claim loop (in practice <= 2 rounds)

__device__ __forceinline__ long long mod_nonneg(long long a, long long n) {
  long long x = a % n;
  return x < 0 ? x + n : x;
}

// status bit 0: collision; bit 1: a claim loop gave up
__global__ void cbc_check(const int32_t* __restrict__ I, long long m, int d, int j, int r,
                          const long long* __restrict__ Z, long long c1, long long c2, long long n1, long long n2,
                          unsigned long long* table, unsigned tag, int* status) {
  for (long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x; row < m;
       row += (long long)gridDim.x * blockDim.x) {
    const int32_t* h = I + row * d;
    long long a1 = 0, a2 = 0;
    for (int i = 0; i < j; ++i) {
      a1 = mod_nonneg(a1 + mod_nonneg(h[i], n1) * Z[i * r], n1);
      if (r == 2) a2 = mod_nonneg(a2 + mod_nonneg(h[i], n2) * Z[i * r + 1], n2);
    }
    a1 = mod_nonneg(a1 + mod_nonneg(h[j], n1) * c1, n1);
    if (r == 2) a2 = mod_nonneg(a2 + mod_nonneg(h[j], n2) * c2, n2);
    const long long bin = r == 2 ? a1 * n2 + a2 : a1;
    const unsigned long long mine = ((unsigned long long)tag << 32) | (unsigned long long)(row + 1);
    unsigned long long* slot = table + bin;
    bool done = false;
    for (int it = 0; it < kCasRetries && !done; ++it) {
      const unsigned long long old = *((volatile unsigned long long*)slot);
      if ((unsigned)(old >> 32) != tag) {
        if (atomicCAS(slot, old, mine) == old) done = true;   // claimed; else retry (someone else wrote)
        continue;
      }
      const long long other = (long long)(old & 0xffffffffull) - 1;
      const int32_t* g = I + other * d;
      bool same = true;
      for (int i = 0; i <= j; ++i) same = same && g[i] == h[i];
      if (!same) atomicOr(status, 1);
      done = true;
    }
    if (!done) atomicOr(status, 2);
  }
}

}  // namespace lsp

using namespace lsp;

extern "C" int lsp_cbc_reconstructing(const int32_t* I, int64_t m, int d, int r, const int64_t* n,
                                      const int64_t* cand, int64_t ncand, int64_t* Z_out, int* fixed,
                                      int device) {
  if (!I || !n || !cand || !Z_out || m < 1 || d < 1 || (r != 1 && r != 2) || ncand < 0 || m >= (1ll << 32) - 1)
    return LSP_ERR_BAD_ARG;
  const long long n1 = n[0], n2 = r == 2 ? n[1] : 1;
  if (n1 < 1 || n2 < 1 || n1 > (1ll << 31) || n2 > (1ll << 31) || n1 * n2 > (1ll << 31)) return LSP_ERR_BAD_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) { cudaGetLastError(); return LSP_ERR_CUDA; }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  std::vector<long long> Z((size_t)d * r, 0);
  Z[0] = 1;                                           // (1) or (1, 0)
  {
    // component 0 alone: h_0 -> h_0 mod n_1 must be injective on the distinct values
    // of h_0 in I (a d = 1 lattice is accepted or rejected by this check only)
    std::vector<int32_t> h0((size_t)m);
    for (int64_t i = 0; i < m; ++i) h0[(size_t)i] = I[(size_t)i * d];
    std::sort(h0.begin(), h0.end());
    h0.erase(std::unique(h0.begin(), h0.end()), h0.end());
    if ((long long)h0.size() > n1) {
      for (int64_t i = 0; i < d * r; ++i) Z_out[i] = 0;
      if (fixed) *fixed = 0;
      return LSP_ERR_NOT_INJECTIVE;
    }
    std::vector<long long> res(h0.size());
    for (size_t i = 0; i < h0.size(); ++i) res[i] = ((long long)h0[i] % n1 + n1) % n1;
    std::sort(res.begin(), res.end());
    if (std::adjacent_find(res.begin(), res.end()) != res.end()) {
      for (int64_t i = 0; i < d * r; ++i) Z_out[i] = 0;
      if (fixed) *fixed = 0;
      return LSP_ERR_NOT_INJECTIVE;
    }
  }
  int32_t* dI = nullptr;
  long long* dZ = nullptr;
  unsigned long long* table = nullptr;
  int* dstat = nullptr;
  int rc = LSP_OK, nfixed = 1;
  const size_t nbins = (size_t)(n1 * n2);
  do {
    if (cudaMalloc(&dI, (size_t)m * d * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&dZ, Z.size() * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&table, nbins * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&dstat, sizeof(int)) != cudaSuccess) { cudaGetLastError(); rc = LSP_ERR_OOM; break; }
    if (cudaMemcpy(dI, I, (size_t)m * d * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(table, 0, nbins * sizeof(unsigned long long)) != cudaSuccess) { rc = LSP_ERR_CUDA; break; }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const long long blocks = std::min<long long>((m + 255) / 256, (long long)sms * 8);
    unsigned tag = 0;
    for (int j = 1; j < d && rc == LSP_OK; ++j) {
      if (cudaMemcpy(dZ, Z.data(), Z.size() * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess) {
        rc = LSP_ERR_CUDA;
        break;
      }
      bool found = false;
      for (int64_t t = 0; t < ncand && !found && rc == LSP_OK; ++t) {
        const int64_t* cr = cand + ((size_t)(j - 1) * ncand + t) * r;
        // candidates reduced mod n_i (an equivalent lattice; keeps h z products in int64)
        const int64_t c[2] = {((cr[0] % n1) + n1) % n1, r == 2 ? ((cr[1] % n2) + n2) % n2 : 0};
        if (++tag == 0) {                               // stamps wrapped: clear the table
          if (cudaMemset(table, 0, nbins * sizeof(unsigned long long)) != cudaSuccess) { rc = LSP_ERR_CUDA; break; }
          tag = 1;
        }
        int st = 0;
        if (cudaMemset(dstat, 0, sizeof(int)) != cudaSuccess) { rc = LSP_ERR_CUDA; break; }
        cbc_check<<<(unsigned)blocks, 256>>>(dI, m, d, j, r, dZ, c[0], r == 2 ? c[1] : 0, n1, n2, table, tag, dstat);
        if (cudaMemcpy(&st, dstat, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) { rc = LSP_ERR_CUDA; break; }
        if (st & 2) { rc = LSP_ERR_TIMEOUT; break; }
        if (!(st & 1)) {
          found = true;
          nfixed = j + 1;
          for (int q = 0; q < r; ++q) Z[(size_t)j * r + q] = c[q];
        }
      }
      if (rc == LSP_OK && !found) {
        for (int jj = j; jj < d; ++jj)
          for (int q = 0; q < r; ++q) Z[(size_t)jj * r + q] = 0;
        rc = LSP_ERR_NOT_INJECTIVE;
      }
    }
  } while (0);
  for (size_t i = 0; i < Z.size(); ++i) Z_out[i] = Z[i];
  if (fixed) *fixed = nfixed;
  cudaFree(dI);
  cudaFree(dZ);
  cudaFree(table);
  cudaFree(dstat);
  cudaSetDevice(prev);
  return rc;
}
