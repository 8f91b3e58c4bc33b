// Host-side interface of the block-Lanczos pass (css_lanczos.cu).
#pragma once
#include "css_internal.cuh"

struct LzArgs {
  bool fp32 = false;                 // Krylov vectors and H*V in FP32 (else FP64)
  int32_t n_brow = 0, b = 0, m = 0;  // molecules, block width, block steps
  int32_t row0 = 0;                  // first block row of this pass in the combined numbering of a
                                     // batch (row_ptr, colour, sign, Hlo_diag already offset by it;
                                     // column indices and pair molecules are global: minus row0)
  int32_t w = 0, ws = 0;             // columns of the batch (b * ncb) and row stride
  const int32_t* row_ptr = nullptr;
  const int32_t* col_idx = nullptr;
  const void* Hval = nullptr;        // [nnzb][BM][BM] transposed, zero-padded (css_spmm_prepare)
  const void* Hlo_diag = nullptr;    // FP32 mode: [n_brow][BM][BM] low parts of the diagonal blocks
  int32_t max_row_blocks = 0;        // largest block count of a row
  const int32_t* colour = nullptr;   // global colour of each molecule
  const int8_t* sign = nullptr;      // probe signs [n_brow * b]
  const double* inv_sqrt_cnt = nullptr;  // 1/sqrt|c| per global colour
  int32_t cb0 = 0, ncb = 0;          // batch = global colours [cb0, cb0 + ncb)
  void *Q0 = nullptr, *Q1 = nullptr, *W = nullptr;  // N x ws vectors
  double* Ablk = nullptr;            // [colour][m][b][b] projected diagonal blocks
  double* Bblk = nullptr;            // [colour][m][b][b] projected sub-diagonal blocks (upper)
  double* Bblk_prev = nullptr;       // [colour][b][b] scratch: B_{j-1} of the running step
  int32_t* nblk = nullptr;           // [colour] blocks used (m unless breakdown)
  int32_t* done = nullptr;           // [colour] recurrence stopped
  double* part = nullptr;            // per-chunk partial products
  double* small = nullptr;           // per-colour small matrices of the batch
  double tau = 1e-10;                // breakdown threshold relative to ||H Q_j||_F
  double shift_rel = 1e-12;          // shifted-CholeskyQR shift relative to trace(W^T W)
  uint32_t flags = 0;
  int mode = 0;                      // 0 none, 1 store sampled rows into Qs, 2 accumulate X
  void* Qs = nullptr;                // [pair][m][b][b] in the vector precision
  double* X = nullptr;               // [pair][b][b]
  const double* Z = nullptr;         // [colour][ldz][b]
  int32_t ldz = 0;
  const int32_t* pair_I = nullptr;   // pairs sorted by colour
  const int32_t* pair_c = nullptr;
  const int64_t* pair_off_h = nullptr;  // host: first pair of each colour (n_colours + 1)
  cudaEvent_t* ev_spmm = nullptr;    // when set: 2 events per step bracket each H*V launch
  void* Yfull = nullptr;             // mode 2 only: also Y += Q_j Z_c[j] over ALL rows, [N][ldy] in the
  int32_t ldy = 0;                   //   vector precision, colour c at columns [c b, c b + b)
  // general start block (non-orthogonal basis): when set, Q_1 B_0 = start (N x ws, the batch's
  // colours in their columns) by shifted CholeskyQR3 instead of Q_1 = R_c / sqrt|c|, and B_0 goes
  // to B0 [colour][b][b]
  const void* start = nullptr;
  double* B0 = nullptr;
  // when set: Vc[colour][j b + k][l] = (Q_j^T u)[k][l] for every block j (u: N x ws)
  const void* ucol = nullptr;
  double* Vc = nullptr;
  // FP32 H * V on the tensor cores (css_hv_tc.cu) when use_tc: TF32 parts of H (tc_H: every
  // block, tc_Hd3: third part of the diagonal blocks, rows numbered as in the combined matrix)
  // and the pass's group schedule (filled by css_hv_tc_schedule)
  // FP32 H * V with exact block width (css_spmm.cu) when Hdup is set: duplicated FP32 pairs of
  // every block and of the low parts of the diagonal blocks (rows as in Hlo_diag)
  const void* Hdup = nullptr;
  const void* Hlo_dup = nullptr;
  // FP64 H * V in FP32 pairs (css_spmm.cu) when Hsplit is set: hi and lo parts of every block
  const void* Hsplit = nullptr;
  bool use_tc = false;
  const void* tc_H = nullptr;
  const void* tc_Hd3 = nullptr;
  const int32_t* tc_cnt = nullptr;
  const int32_t* tc_sJ = nullptr;
  const int32_t* tc_sp = nullptr;
  int32_t tc_cap = 0, tc_groups = 0;
};

css_status css_lanczos_pass(css_ctx* ctx, const LzArgs& a, cudaStream_t st);
// choose (tune, when the shape is new) the H * V launch variant of a pass without running it
css_status css_lanczos_tune(css_ctx* ctx, const LzArgs& a, cudaStream_t st);
// tensor-core H * V (css_hv_tc.cu): FP32 mode with 16 < b <= 24
bool css_hv_tc_supported(bool fp32, int32_t b, int32_t max_row_blocks);
css_status css_hv_tc_prepare(css_ctx* ctx, int32_t b, int32_t n_brow, int32_t nnzb, const int32_t* row_ptr,
                             const int32_t* col_idx, const double* H, const void** Htc, const void** Hd3,
                             cudaStream_t st);
css_status css_hv_tc_schedule(css_ctx* ctx, LzArgs& a, cudaStream_t st);
css_status css_hv_tc(css_ctx* ctx, const LzArgs& a, const float* V, float* W, cudaStream_t st);
css_status css_hv_tc_check(css_ctx* ctx, cudaStream_t st);
// exact-width FP32 H * V (css_spmm.cu): b = 6 and b = 23
bool css_spmm_dup_supported(bool fp32, int32_t b);
int css_spmm_dup_variants();
css_status css_spmm_dup_prepare(css_ctx* ctx, int32_t b, int32_t n_brow, int32_t nnzb, const int32_t* row_ptr,
                                const int32_t* col_idx, const double* H, const void** Hd, const void** Hlod,
                                cudaStream_t st);
css_status css_spmm_dup(css_ctx* ctx, const LzArgs& a, const float* V, float* W, int variant, cudaStream_t st);
css_status css_spmm_dup_check(css_ctx* ctx, cudaStream_t st);
// FP64-accurate H * V in FP32 pairs (css_spmm.cu, precision CSS_FP64_SPLIT): b = 6 and b = 23;
// its time-out flag is the exact-width kernel's (css_spmm_dup_check)
bool css_spmm_split_supported(int32_t b);
int css_spmm_split_variants();
css_status css_spmm_split_prepare(css_ctx* ctx, int32_t b, int32_t nnzb, const double* H, const void** Hs,
                                  cudaStream_t st);
css_status css_spmm_split(css_ctx* ctx, const LzArgs& a, const double* V, double* W, int variant, cudaStream_t st);
// FP32 row passes of a Lanczos step for 16 < b <= 24 (css_rows.cu); mode 0 S1, 1 S3, 2 TRIG, 3 TRI
bool css_rowpass_supported(bool fp32, int32_t b);
css_status css_rowpass(css_ctx* ctx, int mode, int64_t N, int32_t b, int32_t ws, int32_t ncb, int32_t cb0, int first,
                       int reorth, const float* Q, const float* Qp, const float* W, float* OUT, const double* M1,
                       const double* Bprev, const double* Kp, double* part1, double* part2, cudaStream_t st);
css_status css_small_mm(css_ctx* ctx, int32_t ncb, int32_t b, const double* A, const double* B, double* Cm,
                        cudaStream_t st);
// W = M V for a BSR matrix prepared by css_spmm_prepare (a.Hval, a.Hlo_diag, a.row_ptr,
// a.col_idx, a.n_brow, a.b) and N x a.w blocks V, W of row stride a.ws in the vector precision
css_status css_spmm(css_ctx* ctx, const LzArgs& a, const void* V, void* W, cudaStream_t st);
size_t css_lanczos_part_doubles(int64_t N, int32_t b, int32_t ncb);
size_t css_lanczos_small_doubles(int32_t b, int32_t ncb);
// padded block size of the H * V kernel for block width b
int32_t css_spmm_bm(int32_t b);
// H (FP64 [nnzb][b][b]) in the layout of the H * V kernel, in the vector precision; FP32 mode
// also the low FP32 parts of the diagonal blocks.  Both live in the context's workspace.
css_status css_spmm_prepare(css_ctx* ctx, bool fp32, int32_t b, int32_t n_brow, int32_t nnzb,
                            const int32_t* row_ptr, const int32_t* col_idx, const double* H, const void** Hpad,
                            const void** Hlo_pad, cudaStream_t st);
// the same into workspace buffers of their own (named after `tag`), so that several matrices can
// be prepared at once
css_status css_spmm_prepare_as(css_ctx* ctx, const char* tag, bool fp32, int32_t b, int32_t n_brow, int32_t nnzb,
                               const int32_t* row_ptr, const int32_t* col_idx, const double* H, const void** Hpad,
                               const void** Hlo_pad, cudaStream_t st);
// probe block: out (N x ws, zeroed here) holds scale[c] * sign on orbital k of every molecule of
// colour c in column c b + k, for the colours [cb0, cb0 + ncb)
css_status css_probe_block(css_ctx* ctx, bool fp32, int32_t n_brow, int32_t b, int32_t ws, int32_t cb0, int32_t ncb,
                           const int32_t* colour, const int8_t* sign, const double* scale, void* out,
                           cudaStream_t st);
