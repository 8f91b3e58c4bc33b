// Context, workspace and error plumbing of the CSS library.
#include <cstdlib>

#include "css_internal.cuh"

css_status css_set_cuda_error(css_ctx* ctx, cudaError_t e, const char* what, const char* file, int line) {
  if (ctx) {
    char buf[512];
    snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    ctx->last_error = buf;
  }
  if (e == cudaErrorMemoryAllocation) return CSS_ERR_NOMEM;
  return CSS_ERR_CUDA;
}

css_status css_set_arg_error(css_ctx* ctx, const char* what) {
  if (ctx) ctx->last_error = what;
  return CSS_ERR_INVALID_ARG;
}

css_status css_ws(css_ctx* ctx, const char* name, size_t bytes, void** out) {
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255) & ~size_t(255);
  for (auto& kv : ctx->bufs) {
    if (kv.first == name) {
      if (kv.second.bytes >= bytes) {
        *out = kv.second.p;
        return CSS_OK;
      }
      cudaError_t e = cudaFree(kv.second.p);
      if (e != cudaSuccess) return css_set_cuda_error(ctx, e, "cudaFree(workspace)", __FILE__, __LINE__);
      ctx->ws_bytes -= (int64_t)kv.second.bytes;
      kv.second = css_buf{};
      e = cudaMalloc(&kv.second.p, bytes);
      if (e != cudaSuccess) {
        kv.second.p = nullptr;
        return css_set_cuda_error(ctx, e, "cudaMalloc(workspace)", __FILE__, __LINE__);
      }
      kv.second.bytes = bytes;
      ctx->ws_bytes += (int64_t)bytes;
      *out = kv.second.p;
      return CSS_OK;
    }
  }
  css_buf b;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) return css_set_cuda_error(ctx, e, "cudaMalloc(workspace)", __FILE__, __LINE__);
  b.bytes = bytes;
  ctx->ws_bytes += (int64_t)bytes;
  ctx->bufs.emplace_back(name, b);
  *out = b.p;
  return CSS_OK;
}

css_status css_pinned(css_ctx* ctx, size_t bytes, void** out) {
  if (ctx->host_pinned_bytes < bytes) {
    if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
    ctx->host_pinned = nullptr;
    ctx->host_pinned_bytes = 0;
    CSS_CU(ctx, cudaMallocHost(&ctx->host_pinned, bytes));
    ctx->host_pinned_bytes = bytes;
  }
  *out = ctx->host_pinned;
  return CSS_OK;
}

extern "C" {

css_status css_create(css_ctx** out, int device) {
  if (!out) return CSS_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return css_set_cuda_error(nullptr, e, "cudaGetDeviceCount", __FILE__, __LINE__);
  if (device < 0 || device >= ndev) return CSS_ERR_INVALID_ARG;
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return css_set_cuda_error(nullptr, e, "cudaSetDevice", __FILE__, __LINE__);
  css_ctx* ctx = new (std::nothrow) css_ctx();
  if (!ctx) return CSS_ERR_NOMEM;
  ctx->device = device;
  cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, device);
  const char* t = getenv("CSS_TIMING");
  ctx->timing = t && t[0] == '1';
  const char* sv = getenv("CSS_SPMM_VARIANT");
  if (sv && sv[0] >= '0' && sv[0] <= '4' && sv[1] == 0) ctx->spmm_variant = sv[0] - '0';
  const char* dv = getenv("CSS_SPMM_DUP_VARIANT");
  if (dv && dv[0] >= '0' && dv[0] <= '3' && dv[1] == 0) ctx->spmm_dup_variant = dv[0] - '0';
  const char* de = getenv("CSS_DEBUG_EIG");
  ctx->debug_eig = de ? atoi(de) : 0;
  const char* tb = getenv("CSS_TEST_MU_BARRIER_EXTRA");
  const int extra = tb ? atoi(tb) : 0;
  ctx->test_mu_barrier_extra = extra > 0 && extra < 64 ? extra : 0;
  const char* te = getenv("CSS_TEST_SPMM_EMPTY_EXTRA");
  const int eextra = te ? atoi(te) : 0;
  ctx->test_spmm_empty_extra = eextra > 0 && eextra < 4 ? eextra : 0;
  const char* tc = getenv("CSS_HV_TC");
  ctx->hv_tc = tc && tc[0] == '1';
  const char* rs = getenv("CSS_ROWS_STREAM");
  ctx->rows_stream = rs && rs[0] == '1';
  const char* gr = getenv("CSS_GRAPH");
  ctx->graph = gr && gr[0] == '0' ? 0 : (gr && gr[0] == '1' ? 1 : -1);
  *out = ctx;
  return CSS_OK;
}

void css_destroy(css_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (auto& kv : ctx->bufs)
    if (kv.second.p) cudaFree(kv.second.p);
  for (cudaStream_t s : ctx->side) cudaStreamDestroy(s);
  for (cudaEvent_t e : ctx->side_ev) cudaEventDestroy(e);
  for (cudaGraphExec_t g : ctx->lz_exec)
    if (g) cudaGraphExecDestroy(g);
  for (cudaEvent_t e : ctx->lz_ev) cudaEventDestroy(e);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
  delete ctx;
}

const char* css_status_str(css_status s) {
  switch (s) {
    case CSS_OK: return "CSS_OK";
    case CSS_ERR_INVALID_ARG: return "CSS_ERR_INVALID_ARG";
    case CSS_ERR_NOMEM: return "CSS_ERR_NOMEM";
    case CSS_ERR_CUDA: return "CSS_ERR_CUDA";
    case CSS_ERR_TIMEOUT: return "CSS_ERR_TIMEOUT";
    case CSS_ERR_NUMERIC: return "CSS_ERR_NUMERIC";
    case CSS_WARN_BREAKDOWN: return "CSS_WARN_BREAKDOWN";
    case CSS_ERR_UNSUPPORTED: return "CSS_ERR_UNSUPPORTED";
  }
  return "CSS_UNKNOWN_STATUS";
}

const char* css_last_error(const css_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

css_status css_get_info(const css_ctx* ctx, css_info* info) {
  if (!ctx || !info) return CSS_ERR_INVALID_ARG;
  *info = ctx->info;
  info->workspace_bytes = ctx->ws_bytes;
  info->kernel_launches = ctx->kernel_launches;
  info->graph_launches = ctx->graph_launches;
  info->graph_instantiations = ctx->graph_instantiations;
  return CSS_OK;
}

}  // extern "C"
