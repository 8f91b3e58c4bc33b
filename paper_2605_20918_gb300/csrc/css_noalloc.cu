// Graph colouring that allocates nothing: the scratch of the Jones-Plassmann rounds (degrees,
// priority keys, round counters) lives in one file-scope device array instead of the context's
// workspace, so the call needs no css_ctx and makes no device or pinned-host allocation.
//
// The array is a single device symbol; host code must not pass the symbol itself to a kernel
// (on the host it only names a stand-in, not device memory).  Its device address is looked up
// once per device with cudaGetSymbolAddress, with that device current, and cached.
#include <mutex>

#include "css_internal.cuh"

namespace {

constexpr int64_t kMaxN = CSS_NOALLOC_MAX_VERTICES;
// layout of the scratch: counters (64 int32), then deg[kMaxN] int32, then key[kMaxN] uint64
constexpr size_t kCountersBytes = 256;
constexpr size_t kDegBytes = (size_t)kMaxN * sizeof(int32_t);
constexpr size_t kScratchBytes = kCountersBytes + kDegBytes + (size_t)kMaxN * sizeof(uint64_t);

}  // namespace

static __device__ __align__(256) unsigned char css_noalloc_scratch[kScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch[kMaxDevices] = {};

__device__ __forceinline__ bool na_higher(int32_t du, uint64_t ku, int32_t u, int32_t dv, uint64_t kv, int32_t v) {
  if (du != dv) return du > dv;
  if (ku != kv) return ku > kv;
  return u < v;
}

__global__ void k_na_init(int32_t n, const int32_t* __restrict__ adj_ptr, uint64_t seed, unsigned char* scratch,
                          int32_t* __restrict__ colour) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t* deg = reinterpret_cast<int32_t*>(scratch + kCountersBytes);
  uint64_t* key = reinterpret_cast<uint64_t*>(scratch + kCountersBytes + kDegBytes);
  deg[i] = adj_ptr[i + 1] - adj_ptr[i];
  key[i] = css_splitmix64(seed, (uint64_t)i);
  colour[i] = -1;
}

// one Jones-Plassmann round: a vertex whose higher-priority neighbours are all coloured takes
// the smallest colour none of them uses; the others count themselves into *remaining
__global__ void k_na_round(int32_t n, const int32_t* __restrict__ adj_ptr, const int32_t* __restrict__ adj,
                           unsigned char* scratch, int32_t* colour, int32_t slot) {
  int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  int32_t* counters = reinterpret_cast<int32_t*>(scratch);
  const int32_t* deg = reinterpret_cast<const int32_t*>(scratch + kCountersBytes);
  const uint64_t* key = reinterpret_cast<const uint64_t*>(scratch + kCountersBytes + kDegBytes);
  if (__ldcg(&colour[v]) >= 0) return;
  const int32_t dv = deg[v];
  const uint64_t kv = key[v];
  const int32_t s = adj_ptr[v], e = adj_ptr[v + 1];
  for (int32_t k = s; k < e; ++k) {
    int32_t u = adj[k];
    if (na_higher(deg[u], key[u], u, dv, kv, v) && __ldcg(&colour[u]) < 0) {
      atomicAdd(&counters[slot], 1);
      return;
    }
  }
  for (int32_t base = 0;; base += 64) {
    uint64_t used = 0;
    for (int32_t k = s; k < e; ++k) {
      int32_t u = adj[k];
      if (!na_higher(deg[u], key[u], u, dv, kv, v)) continue;
      int32_t c = __ldcg(&colour[u]) - base;
      if (c >= 0 && c < 64) used |= 1ull << c;
    }
    if (~used) {
      colour[v] = base + __ffsll((long long)~used) - 1;
      return;
    }
  }
}

// adj_ptr[0] = 0, adj_ptr non-decreasing and every neighbour in [0, n), else counters[40] != 0
__global__ void k_na_check(int32_t n, const int32_t* __restrict__ adj_ptr, const int32_t* __restrict__ adj,
                           unsigned char* scratch) {
  int32_t* counters = reinterpret_cast<int32_t*>(scratch);
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t s = adj_ptr[i], e = adj_ptr[i + 1];
  if ((i == 0 && s != 0) || e < s) {
    atomicOr(&counters[40], 1);
    return;
  }
  for (int32_t k = s; k < e; ++k) {
    const int32_t u = adj[k];
    if (u < 0 || u >= n) {
      atomicOr(&counters[40], 1);
      return;
    }
  }
}

__global__ void k_na_max(int32_t n, const int32_t* __restrict__ colour, unsigned char* scratch) {
  int32_t* counters = reinterpret_cast<int32_t*>(scratch);
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  int32_t c = i < n ? colour[i] : -1;
  for (int o = 16; o > 0; o >>= 1) c = max(c, __shfl_xor_sync(0xffffffffu, c, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&counters[32], c);
}

css_status na_error(cudaError_t e) { return e == cudaErrorMemoryAllocation ? CSS_ERR_NOMEM : CSS_ERR_CUDA; }

}  // namespace

extern "C" {

css_status css_color_graph_noalloc(int32_t n, const int32_t* adj_ptr, const int32_t* adj, uint64_t seed,
                                   int32_t* colour, int32_t* n_colours, void* stream) {
  if (n < 1 || !adj_ptr || !colour || !n_colours) return CSS_ERR_INVALID_ARG;
  if ((int64_t)n > kMaxN) return CSS_ERR_INVALID_ARG;  // larger graphs: css_color_graph
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_error(e);
  if (dev < 0 || dev >= kMaxDevices) return CSS_ERR_UNSUPPORTED;
  unsigned char* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, css_noalloc_scratch);  // device `dev` is current here
      if (e != cudaSuccess || !p) return na_error(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
      g_scratch[dev] = p;
    }
    scratch = static_cast<unsigned char*>(g_scratch[dev]);
  }
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned nbk = (unsigned)((n + 255) / 256);
  int32_t* counters = reinterpret_cast<int32_t*>(scratch);
  // a malformed graph is refused before any round reads through it (the flag keeps the previous
  // call's value, so it is cleared first)
  int32_t bad = 0;
  if ((e = cudaMemsetAsync(counters + 40, 0, sizeof(int32_t), st)) != cudaSuccess) return na_error(e);
  k_na_check<<<nbk, 256, 0, st>>>(n, adj_ptr, adj, scratch);
  if ((e = cudaGetLastError()) != cudaSuccess) return na_error(e);
  if ((e = cudaMemcpyAsync(&bad, counters + 40, sizeof(int32_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return na_error(e);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return na_error(e);
  if (bad) return CSS_ERR_INVALID_ARG;
  k_na_init<<<nbk, 256, 0, st>>>(n, adj_ptr, seed, scratch, colour);
  if ((e = cudaGetLastError()) != cudaSuccess) return na_error(e);
  const int group = 8;
  int32_t remaining = 0;
  for (int64_t rounds = 0;; rounds += group) {
    // the counters keep the previous call's values: clear them for these rounds
    if ((e = cudaMemsetAsync(counters, 0, sizeof(int32_t) * group, st)) != cudaSuccess) return na_error(e);
    for (int r = 0; r < group; ++r) {
      k_na_round<<<nbk, 256, 0, st>>>(n, adj_ptr, adj, scratch, colour, r);
      if ((e = cudaGetLastError()) != cudaSuccess) return na_error(e);
    }
    if ((e = cudaMemcpyAsync(&remaining, counters + group - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
      return na_error(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return na_error(e);
    if (remaining == 0) break;
    if (rounds > (int64_t)n + group) return CSS_ERR_INVALID_ARG;
  }
  if ((e = cudaMemsetAsync(counters + 32, 0xff, sizeof(int32_t), st)) != cudaSuccess) return na_error(e);
  k_na_max<<<nbk, 256, 0, st>>>(n, colour, scratch);
  if ((e = cudaGetLastError()) != cudaSuccess) return na_error(e);
  int32_t maxc = -1;
  if ((e = cudaMemcpyAsync(&maxc, counters + 32, sizeof(int32_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return na_error(e);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return na_error(e);
  *n_colours = maxc + 1;
  return CSS_OK;
}

}  // extern "C"
