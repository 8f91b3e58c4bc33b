// One whole P build (colouring, probes, density) behind a single call, optionally from host
// buffers with the host<->device copies done here on the caller's stream.
#include "css_internal.cuh"

extern "C" {

css_status css_pbuild(css_ctx* ctx, const css_geom* geom, const css_bsr* H, double r_col, uint64_t colour_seed,
                      uint64_t sign_seed, const css_fermi* fermi, int32_t m, css_precision prec, uint32_t flags,
                      double* P_val, int32_t* colour_out, int32_t* n_colours, double* trP, double* trPH,
                      double* mu_out, void* stream) {
  if (!ctx || !geom || !H || !fermi || !P_val || !geom->xyz || !H->row_ptr || !H->col_idx || !H->val)
    return css_set_arg_error(ctx, "css_pbuild: null pointer");
  if (geom->n_mol != H->n_brow) return css_set_arg_error(ctx, "css_pbuild: geometry and H disagree on n_mol");
  if (H->b < 1 || H->b > CSS_MAX_B || H->nnzb < H->n_brow) return css_set_arg_error(ctx, "css_pbuild: bad H shape");
  CSS_CU(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const bool host = (flags & CSS_HOST_IO) != 0;
  const uint32_t dflags = flags & ~CSS_HOST_IO;
  const int32_t n = geom->n_mol, b = H->b, nnzb = H->nnzb;
  const size_t vbytes = (size_t)nnzb * b * b * sizeof(double);
  css_geom g = *geom;
  css_bsr h = *H;
  double* P_dev = P_val;
  int32_t* col_dev = nullptr;
  int8_t* sign_dev = nullptr;
  CSS_TRY(css_ws(ctx, "pb_colour", sizeof(int32_t) * n, (void**)&col_dev));
  CSS_TRY(css_ws(ctx, "pb_sign", (size_t)n * b, (void**)&sign_dev));
  if (host) {
    double *xyz, *val, *pd;
    int32_t *rp, *ci;
    CSS_TRY(css_ws(ctx, "pb_xyz", sizeof(double) * 3 * n, (void**)&xyz));
    CSS_TRY(css_ws(ctx, "pb_rowptr", sizeof(int32_t) * (n + 1), (void**)&rp));
    CSS_TRY(css_ws(ctx, "pb_colidx", sizeof(int32_t) * nnzb, (void**)&ci));
    CSS_TRY(css_ws(ctx, "pb_val", vbytes, (void**)&val));
    CSS_TRY(css_ws(ctx, "pb_P", vbytes, (void**)&pd));
    CSS_CU(ctx, cudaMemcpyAsync(xyz, geom->xyz, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    CSS_CU(ctx, cudaMemcpyAsync(rp, H->row_ptr, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, st));
    CSS_CU(ctx, cudaMemcpyAsync(ci, H->col_idx, sizeof(int32_t) * nnzb, cudaMemcpyHostToDevice, st));
    CSS_CU(ctx, cudaMemcpyAsync(val, H->val, vbytes, cudaMemcpyHostToDevice, st));
    g.xyz = xyz;
    h.row_ptr = rp;
    h.col_idx = ci;
    h.val = val;
    P_dev = pd;
  }
  int32_t nc = 0;
  CSS_TRY(css_color(ctx, &g, r_col, colour_seed, col_dev, &nc, stream));
  CSS_TRY(css_probes(ctx, col_dev, n, b, sign_seed, 0, sign_dev, stream));
  css_status st_d = css_density(ctx, &h, col_dev, sign_dev, nc, fermi, m, prec, dflags, P_dev, trP, trPH, mu_out,
                                stream);
  if (st_d != CSS_OK && st_d != CSS_WARN_BREAKDOWN) return st_d;
  if (host) {
    CSS_CU(ctx, cudaMemcpyAsync(P_val, P_dev, vbytes, cudaMemcpyDeviceToHost, st));
    if (colour_out) CSS_CU(ctx, cudaMemcpyAsync(colour_out, col_dev, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
    CSS_CU(ctx, cudaStreamSynchronize(st));
  } else if (colour_out) {
    CSS_CU(ctx, cudaMemcpyAsync(colour_out, col_dev, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st));
  }
  if (n_colours) *n_colours = nc;
  return st_d;
}

}  // extern "C"
