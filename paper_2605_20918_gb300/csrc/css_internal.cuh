// Internal declarations shared by the CUDA translation units of the CSS library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "css.h"

#define CSS_MAX_B 32

// ---------------------------------------------------------------- error handling
#define CSS_TRY(expr)                       \
  do {                                      \
    css_status _st = (expr);                \
    if (_st != CSS_OK) return _st;          \
  } while (0)

#define CSS_CU(ctx, call)                                                             \
  do {                                                                                \
    cudaError_t _e = (call);                                                          \
    if (_e != cudaSuccess) return css_set_cuda_error((ctx), _e, #call, __FILE__, __LINE__); \
  } while (0)

#define CSS_LAUNCHED(ctx)        \
  do {                           \
    ++(ctx)->kernel_launches;    \
    CSS_CU(ctx, cudaGetLastError()); \
  } while (0)

struct css_buf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct css_ctx {
  int device = 0;
  int n_sm = 0;
  bool timing = false;
  int debug_eig = 0;  // 1: eigen stage returns its FP32 shifts instead of refined eigenvalues
  int64_t kernel_launches = 0;  // kernels this context has launched (all calls)
  // where the last density call left its Ritz data (device)
  const double* last_lam = nullptr;
  const double* last_wgt = nullptr;
  const int32_t* last_nblk = nullptr;
  const double* last_A = nullptr;
  const double* last_B = nullptr;
  int32_t last_m = 0;
  int32_t last_ncol = 0, last_b = 0, last_nmax = 0;
  std::string last_error;
  css_info info{};
  // named, grow-only device workspace
  std::vector<std::pair<std::string, css_buf>> bufs;
  int64_t ws_bytes = 0;
  // pinned host staging for scalars read back at the end of a call
  void* host_pinned = nullptr;
  size_t host_pinned_bytes = 0;
  // H * V autotuner: launch variant chosen per (precision, block width, column count, rows)
  std::vector<std::pair<uint64_t, int>> spmm_tune;
  // env CSS_SPMM_VARIANT = 0..4: the padded FP32 kernel (also for b = 6 and 23) with that variant
  int spmm_variant = -1;
  int spmm_dup_variant = -1;  // env CSS_SPMM_DUP_VARIANT = 0..3 fixes the exact-width kernel's variant
  // failure injection for tests (env CSS_TEST_SPMM_EMPTY_EXTRA = k at css_create): the "empty"
  // barriers of the exact-width H * V wait for k warps more than a CTA has, so the copying
  // thread's bounded wait runs out and the call returns CSS_ERR_TIMEOUT; 0 is the normal kernel
  int test_spmm_empty_extra = 0;
  // failure injection for tests (env CSS_TEST_MU_BARRIER_EXTRA = k at css_create): the grid
  // barrier of the mu bisection waits for k CTAs more than the launch has, so its bounded wait
  // runs out and the call returns CSS_ERR_TIMEOUT; 0 (the default) is the normal barrier
  int32_t test_mu_barrier_extra = 0;
  // FP32 H * V on the tensor cores where the block width allows it (env CSS_HV_TC=1 at
  // css_create; the default is the CUDA-core kernel)
  bool hv_tc = false;
  // env CSS_ROWS_STREAM=1 at css_create: the streaming FP32 row passes of css_rows.cu (11
  // passes per step) instead of the tiled row kernels (14 passes, faster as measured)
  bool rows_stream = false;
  // side streams (and their fork / join events) on which the per-system block-Lanczos passes
  // of a batch run concurrently; created on first use, destroyed with the context
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> side_ev;
  // the block-Lanczos phase of a css_density call (every system, colour batch and step) is
  // captured from the stream into one CUDA graph and launched at once; the executable graph of
  // each pass mode (0 no retention, 1 stored rows, 2 regenerating pass) is kept and updated in
  // place by the next call's capture.  graph: 1 always, 0 never (the kernels one by one), -1 (the
  // default) for a single system only: a batch's thousands of small launches on the side streams
  // cost less to enqueue than to capture anew each call (env CSS_GRAPH=0 / 1 at css_create)
  int graph = -1;
  cudaStream_t cap_stream = nullptr;  // the stream the phase is captured on
  cudaGraphExec_t lz_exec[3] = {nullptr, nullptr, nullptr};
  int64_t graph_launches = 0, graph_instantiations = 0, graph_updates = 0;
  // CSS_TIMING events of the block-Lanczos phase (two per step and pass), kept across calls so
  // that a captured graph's event nodes stay the same
  std::vector<cudaEvent_t> lz_ev;
};

// CUDA events owned by the holder: destroyed when it goes out of scope, early returns included
struct css_events {
  std::vector<cudaEvent_t> ev;
  css_events() = default;
  css_events(const css_events&) = delete;
  css_events& operator=(const css_events&) = delete;
  ~css_events() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
  cudaError_t create(size_t n) {  // n more events; stops at the first failure
    for (size_t i = 0; i < n; ++i) {
      cudaEvent_t e = nullptr;
      const cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return r;
      ev.push_back(e);
    }
    return cudaSuccess;
  }
  cudaEvent_t& operator[](size_t i) { return ev[i]; }
  cudaEvent_t* data() { return ev.data(); }
};

css_status css_set_cuda_error(css_ctx* ctx, cudaError_t e, const char* what, const char* file, int line);
css_status css_set_arg_error(css_ctx* ctx, const char* what);
// Device buffer `name` with at least `bytes` bytes (grow-only; contents not preserved on growth).
css_status css_ws(css_ctx* ctx, const char* name, size_t bytes, void** out);
css_status css_pinned(css_ctx* ctx, size_t bytes, void** out);

// SplitMix64 output for state seed + (x + 1) * gamma (Steele, Lea & Flood 2014).
__host__ __device__ __forceinline__ uint64_t css_splitmix64(uint64_t seed, uint64_t x) {
  uint64_t z = seed + (x + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ int64_t css_ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ----------------------------------------------------------- internal entry points
// colouring (css_color.cu)
css_status css_color_impl(css_ctx* ctx, int32_t n, const double* xyz, double box, double r_col, uint64_t seed,
                          const int32_t* adj_ptr_in, const int32_t* adj_in, int32_t* colour, int32_t* n_colours,
                          cudaStream_t st);
// density (css_density.cu)
struct css_sys_desc {
  css_bsr H;
  const int32_t* colour;
  const int8_t* sign;
  int32_t n_colours;
  css_fermi fermi;
  double* P_val;
};
// yfull (optional, device, [N][ldy] in the vector precision, zeroed by the caller): forces the
// regenerating second pass and accumulates Y = Q_c Z_c of every colour over all rows into it
// partial: colour -1 marks molecules in no probe block (colour-partitioned builds; one system,
// unsymmetrised output, the blocks of unprobed columns written as zero)
css_status css_density_impl(css_ctx* ctx, int32_t n_sys, const css_sys_desc* sys, int32_t m, css_precision prec,
                            uint32_t flags, double* trP, double* trPH, double* mu_out, cudaStream_t st,
                            void* yfull = nullptr, int32_t ldy = 0, bool partial = false,
                            const int32_t* colour_ids = nullptr);
