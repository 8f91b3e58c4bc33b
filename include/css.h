/*
 * css.h — C-ABI of the GB300 (sm_103a) chromatic-superposition-state (CSS) density-matrix
 * library: graph colouring, CSS probe blocks and the block-Lanczos projection that returns
 * the sparse Kohn-Sham density matrix P = f(H) on H's sparsity pattern.
 *
 * Paper: Jiang, Xiao, Tang, Li, Sun, Xia, Ke, "High-performance linear-scaling electronic
 * structure method via chromatic superposition states" (arXiv 2605.20918).
 *
 * Conventions for every entry point
 *   - Plain C types only.  Array arguments are DEVICE pointers (cudaMalloc'd or from any
 *     CUDA allocator, e.g. torch) unless a comment says "host".  The caller owns every input
 *     and output buffer; the library never frees them.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  All device
 *     work is ordered on it.  Calls that return a scalar through a host pointer synchronise
 *     that stream before returning; the others are asynchronous unless stated.
 *   - The context owns device workspace.  It grows on demand (cudaMalloc) and is reused;
 *     once a call has run with a given shape, repeating it allocates nothing.
 *   - No C++ exception crosses this interface.  Errors are returned as css_status; a
 *     CUDA error is reported as CSS_ERR_CUDA and the message is kept for css_last_error().
 *   - css_density works in an orthogonal basis (S = I, so H' = H in the paper's Eq. 4);
 *     css_density with CSS_INV_SQRT and css_hprime give S~^(-1/2) and H' of a non-orthogonal
 *     one (Eq. 8-10).
 */
#ifndef CSS_H
#define CSS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CSS_API __attribute__((visibility("default")))
#else
#define CSS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CSS_OK = 0,
  CSS_ERR_INVALID_ARG = 1, /* a size, pointer, flag or value is out of range          */
  CSS_ERR_NOMEM = 2,       /* device workspace could not be allocated                  */
  CSS_ERR_CUDA = 3,        /* a CUDA runtime call or kernel failed                      */
  CSS_ERR_TIMEOUT = 4,     /* a bounded device wait ran out (mu grid barrier, band-reduction sweeps) */
  CSS_ERR_NUMERIC = 5,     /* NaN/Inf in the result or a non-convergent eigen-step      */
  CSS_WARN_BREAKDOWN = 6,  /* some colour's Krylov space became invariant early; result valid */
  CSS_ERR_UNSUPPORTED = 7  /* a shape the build does not support (b > 32)              */
} css_status;

typedef enum {
  CSS_FP64 = 0,        /* everything in FP64                                               */
  CSS_MIXED_FP32 = 1,  /* H*V, Krylov vectors and block products in FP32 (FP32 accumulate); */
                       /* recurrence coefficients, Cholesky, eigensolve, mu, Z and P in FP64; */
                       /* implies CSS_REORTH_LOCAL (it removes an FP32-level bias of Tr P)   */
  CSS_MIXED_3XTF32 = 2, /* as CSS_MIXED_FP32, with the H*V of the block-Lanczos recurrence on */
                        /* the tensor cores: TF32 products of split operands (x = x1 + x2, the */
                        /* on-site blocks in three parts) accumulated in FP32, for 17 <= b <= 24 */
                        /* (other b: CSS_ERR_UNSUPPORTED); the other sparse products of        */
                        /* css_hprime and css_density_nonorth stay on the FP32 FMA pipe        */
  CSS_FP64_SPLIT = 3    /* as CSS_FP64, with the H*V of the block-Lanczos recurrence on the FP32 */
                        /* FMA pipe: H and V as pairs hi + lo of FP32 numbers, each product by */
                        /* an error-free FMA split, sums by TwoSum into hi + lo (about 2^-47   */
                        /* relative per term against 2^-53); b = 6 or 23 (other b:            */
                        /* CSS_ERR_UNSUPPORTED); other sparse products stay FP64             */
} css_precision;

/* css_density flags */
#define CSS_SYMMETRIZE 1u   /* P = (P~ + P~^T)/2 on the pattern (default in the Python binding)   */
#define CSS_TWO_PASS 2u     /* regenerate the Krylov basis instead of storing its sampled rows  */
#define CSS_REORTH_LOCAL 4u /* one more orthogonalisation pass of each new block against Q_j, Q_j-1 */
#define CSS_HOST_IO 8u      /* css_pbuild only: every array argument is HOST memory            */
/* Energy-weighted density matrix instead of P (paper: the matrix rho_E = sum_i f(e_i) e_i
 * |psi_i><psi_i| that DFTB forces need, obtained in CSS as H rho~ for an orthogonal basis),
 * taken in each colour's Krylov subspace: Z_c = U Lambda f(Lambda) U^T E_1 B_0 = T_c Z_c(P).
 * mu is still fixed by f (Tr P = n_elec/2); trP and trPH then return Tr rho_E and
 * Tr(rho_E H). */
#define CSS_ENERGY_WEIGHTED 16u
/* H is an overlap matrix S (symmetric positive definite) and the matrix function is x^(-1/2)
 * instead of the Fermi function (paper, Eq. 8-10: S^(-1/2) by the same block-Lanczos
 * projection onto coloured probes, the exact diagonalisation of the projected S^K and its
 * inverse square root); fermi is ignored and mu_out returns fermi->mu; P_val receives
 * S~^(-1/2) on S's pattern, trP Tr S~^(-1/2), trPH Tr(S~^(-1/2) S).  A non-positive Ritz
 * value (S not positive definite) gives CSS_ERR_NUMERIC. */
#define CSS_INV_SQRT 32u
/* Stop after the exact diagonalisation of the projected matrices (paper, Eq. 7): css_ritz then
 * returns every colour's Ritz values and weights; mu, Z and P are not computed (P_val, trP, trPH
 * and mu_out are left untouched).  The first phase of a colour-partitioned build. */
#define CSS_RITZ_ONLY 64u
/* css_probes flags */
#define CSS_SIGNS_ONES 1u   /* all probe entries +1 instead of seeded random signs             */

typedef struct css_ctx css_ctx;

/* Molecule centres in a periodic cubic box.  xyz: n_mol x 3 doubles (Angstrom). */
typedef struct {
  int32_t n_mol;
  const double* xyz;
  double box;
} css_geom;

/* Symmetric block-sparse-row matrix with b x b blocks (b <= 32).
 * row_ptr[n_brow+1], col_idx[nnzb] (sorted within a row, diagonal present, pattern
 * structurally symmetric), val[nnzb*b*b] row-major inside each block, FP64. */
typedef struct {
  int32_t n_brow, b, nnzb;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const double* val;
} css_bsr;

/* Fermi-Dirac occupation f(x) = 1/(1+exp((x-mu)/kT)) (paper, Eq. 1); kT = 0 is the step
 * function.  solve_mu != 0: mu is taken from the Ritz quadrature N(mu) = sum_c sum_k
 * f(lambda_ck) w_ck of Tr P (P per spin): it is the midpoint of the set of mu where
 * |N(mu) - n_elec/2| <= ne_tol (each end by bisection), i.e. the root for a metal and
 * mid-gap for an insulator; ne_tol <= 0 selects 1e-4 * n_elec/2 (above the spurious Ritz
 * weight that a truncated Krylov projection leaves inside a gap, so that the ends of the set
 * are the band edges).  Otherwise `mu` is used as given. */
typedef struct {
  double mu, kT, n_elec, ne_tol;
  int32_t solve_mu;
} css_fermi;

/* Per-call diagnostics (host struct filled by css_get_info). */
typedef struct {
  int32_t n_colours, n_pairs, n_breakdown, m;
  int64_t workspace_bytes;
  double ms_color, ms_probes, ms_setup, ms_lanczos, ms_spmm, ms_eigen, ms_mu, ms_extract, ms_total;
  int64_t spmm_launches; /* H*V launches of the last css_density call                       */
  double spmm_flops;     /* algorithmic flops of one H*V launch: 2 nnzb b^2 w               */
  double spmm_bytes;     /* algorithmic bytes of one H*V launch: H once, V in, W out        */
  int64_t kernel_launches; /* kernels launched by this context since css_create            */
  double ms_rows;          /* row work of one Lanczos step between two H*V launches (three-term
                              update, reorthogonalisation, CholeskyQR3, sampled rows), averaged */
  int64_t graph_launches;  /* CUDA-graph launches of the block-Lanczos phase since css_create  */
  int64_t graph_instantiations; /* of those, graphs instantiated anew (the rest were updated in
                                   place from the previous call's graph of the same mode)     */
} css_info;

/* ------------------------------------------------------------------ context */
/* Create a context bound to CUDA device `device`.  *ctx receives the handle. */
CSS_API css_status css_create(css_ctx** ctx, int device);
/* Free the context and its workspace (synchronises the device first). */
CSS_API void css_destroy(css_ctx* ctx);
/* Static string for a status code. */
CSS_API const char* css_status_str(css_status s);
/* Message of the last CUDA/argument error seen by this context ("" if none). */
CSS_API const char* css_last_error(const css_ctx* ctx);
/* Diagnostics of the last call (host pointer).  Phase times are taken with CUDA events
 * only when the environment variable CSS_TIMING=1 was set at css_create. */
CSS_API css_status css_get_info(const css_ctx* ctx, css_info* info);

/* ---------------------------------------------------------------- colouring */
/* Greedy multicolouring of molecules (paper: CSS construction paragraph after Eq. 2; greedy
 * order after Welsh-Powell): molecules whose minimum-image centre distance is < r_col get
 * different colours.  Distances are exact: coordinates are rounded to int64 multiples of
 * 2^-20 A (llrint(x*2^20)) and compared as squared integers, strictly below
 * llrint(r_col*2^20)^2.  The order is degree descending, then SplitMix64(seed, id)
 * descending, then id ascending; each molecule takes the smallest colour not used by a
 * neighbour earlier in that order (Jones-Plassmann rounds on the GPU give exactly that
 * colouring).
 *   geom      host struct; geom->xyz is a DEVICE array of n_mol*3 doubles
 *   colour    device int32[n_mol], written
 *   n_colours host int32*, written (the call synchronises `stream`)
 * Errors: INVALID_ARG for n_mol < 1, box <= 0, r_col < 0 or box > 1000 A. */
CSS_API css_status css_color(css_ctx* ctx, const css_geom* geom, double r_col, uint64_t seed, int32_t* colour,
                     int32_t* n_colours, void* stream);

/* Same colouring rule on an explicit graph: device CSR adj_ptr[n+1], adj[adj_ptr[n]]
 * (symmetric, no self loops; neighbour order irrelevant).  The pattern is checked on the device
 * before the rounds: adj_ptr[0] != 0, a decreasing adj_ptr or a neighbour outside [0, n) gives
 * CSS_ERR_INVALID_ARG (adj must hold adj_ptr[n] entries; the call cannot check that). */
CSS_API css_status css_color_graph(css_ctx* ctx, int32_t n, const int32_t* adj_ptr, const int32_t* adj, uint64_t seed,
                           int32_t* colour, int32_t* n_colours, void* stream);

/* Conflicts of a colouring on a (new) geometry: the number of unordered molecule pairs
 * {I, J} with colour[I] == colour[J] whose minimum-image centre distance is < r_col, in the
 * same fixed-point arithmetic as css_color.  Zero means the colouring still meets the
 * condition of the CSS construction (paragraph after Eq. 2) on this geometry, so it can be
 * kept from one MD step to the next.
 *   geom        as in css_color (xyz a DEVICE array)
 *   colour      device int32[n_mol], read; values must lie in [0, n_colours)
 *   n_conflicts host int64*, written (the call synchronises `stream`)
 * Errors: INVALID_ARG for bad geometry or r_col (as css_color), n_colours < 1, or a colour
 * outside [0, n_colours) (detected on the device). */
CSS_API css_status css_color_check(css_ctx* ctx, const css_geom* geom, double r_col, const int32_t* colour,
                           int32_t n_colours, int64_t* n_conflicts, void* stream);

/* Colouring kept across MD steps: when *n_colours >= 1 and `colour` has no conflict at r_col
 * on geom (css_color_check) and all its values lie in [0, *n_colours), nothing is written
 * and *recoloured = 0; otherwise geom is coloured from scratch exactly as
 * css_color(r_col + skin, seed) does, into colour and *n_colours, and *recoloured = 1.  A
 * skin > 0 (like a neighbour-list skin) leaves same-coloured molecules room to move before
 * the colouring has to change, at the price of more colours.  Pass *n_colours = 0 for the
 * first step.
 *   skin        Angstrom, >= 0
 *   colour      device int32[n_mol], read and possibly written
 *   n_colours   host int32*, read and possibly written
 *   recoloured  host int32* or NULL
 * Blocking like css_color.  No counterpart in the paper, which colours each geometry. */
CSS_API css_status css_color_update(css_ctx* ctx, const css_geom* geom, double r_col, double skin, uint64_t seed,
                            int32_t* colour, int32_t* n_colours, int32_t* recoloured, void* stream);

/* ------------------------------------------------------------------- probes */
/* CSS probe signs (paper: same paragraph, Fig. 1c): column k of colour c's probe block holds
 * sign[J*b+k] = +-1 on orbital k of every molecule J of colour c, 0 elsewhere.  sign is -1
 * exactly when bit 0 of SplitMix64(sign_seed, J*b+k) is set (all +1 with CSS_SIGNS_ONES).
 *   colour  device int32[n_mol] (not read; the probes are implicit in colour + sign)
 *   sign    device int8[n_mol*b], written.  Asynchronous. */
CSS_API css_status css_probes(css_ctx* ctx, const int32_t* colour, int32_t n_mol, int32_t b, uint64_t sign_seed,
                      uint32_t flags, int8_t* sign, void* stream);

/* ------------------------------------------------------------------ density */
/* CSS density matrix (paper, Eq. 2 and Eq. 5-7): for every colour c a block-Lanczos
 * recurrence of depth m on R_c (block width b), the projected block-tridiagonal matrix
 * diagonalised exactly in FP64, f applied to its eigenvalues, and
 *   P~_IJ = [Q_c Z_c]_I diag(s_J),  c = colour(J),  Z_c = U f(Lambda) U^T E_1 B_0
 * written on H's pattern only; P = (P~ + P~^T)/2 with CSS_SYMMETRIZE.
 *   H          host struct of device arrays (see css_bsr)
 *   colour     device int32[n_brow] in [0, n_colours)
 *   sign       device int8[n_brow*b] (from css_probes)
 *   fermi      host struct
 *   m          Lanczos block steps (projected matrix of size m*b per colour), 1 <= m, m*b <= 4096
 *   P_val      device double[nnzb*b*b], written (same block order as H->val)
 *   trP, trPH, mu_out   host doubles, written (Tr P, Tr(P H), chemical potential); may be NULL
 * Returns CSS_WARN_BREAKDOWN when a colour's recurrence stopped early (invariant Krylov
 * space: the result is exact for that colour).  Synchronises `stream`.
 * The block-Lanczos phase of a single-system call runs as one CUDA graph, captured on a stream
 * of the context and launched on `stream` (the previous call's graph is updated in place when
 * the launch sequence has the same shape); the environment variable CSS_GRAPH=0 at css_create
 * launches its kernels one by one, CSS_GRAPH=1 captures batches too.  The results are the
 * same either way. */
CSS_API css_status css_density(css_ctx* ctx, const css_bsr* H, const int32_t* colour, const int8_t* sign, int32_t n_colours,
                       const css_fermi* fermi, int32_t m, css_precision prec, uint32_t flags, double* P_val,
                       double* trP, double* trPH, double* mu_out, void* stream);

/* H' of a non-orthogonal basis (paper, Eq. 8-10 and the paragraph after them).  With the probes
 * o of (colour, sign) -- a colouring of S's pattern at the caller's cut-off d_cut^S --
 *   Y = S^(-1/2) |o>  by block-Lanczos on S (depth m) and x^(-1/2) in the Krylov subspace,
 *   S~^(-1/2) = Y <o| extracted on S's pattern                       -> Sinv_val,
 *   H'~ extracted from S~^(-1/2) H Y <o| on H's pattern               -> Hp_val,
 * i.e. H'~_IJ = [S~^(-1/2) (H Y_c)]_I diag(o_J), c = colour(J): two SpMMs on the full
 * N x (n_colours b) block Y.  With CSS_SYMMETRIZE both outputs are symmetrised on their
 * (structurally symmetric) patterns.
 *   S, H      host structs of device arrays; same n_brow and b, patterns may differ
 *   Sinv_val  device double[S->nnzb*b*b], Hp_val device double[H->nnzb*b*b], written
 *   trHp      host double, written: Tr H'
 *   flags     CSS_SYMMETRIZE, CSS_REORTH_LOCAL
 * Workspace: three N x (n_colours b) blocks in the vector precision beyond css_density's.
 * Returns CSS_WARN_BREAKDOWN when a colour's recurrence on S stopped early.  Synchronises. */
CSS_API css_status css_hprime(css_ctx* ctx, const css_bsr* S, const css_bsr* H, const int32_t* colour,
                              const int8_t* sign, int32_t n_colours, int32_t m, css_precision prec, uint32_t flags,
                              double* Sinv_val, double* Hp_val, double* trHp, void* stream);

/* Density matrix of a NON-ORTHOGONAL basis (paper, Eq. 4-6 with S != I): the block-Krylov space
 * of H' for colour c starts at r~_c = S~^(-1/2) r_c (r_c the probe block of the colouring
 * `colour`/`sign`), r~_c = Q_1 B_0 by QR, and rho~ = S~^(-1/2) Phi_c f(T_c) E_1 B_0 <r_c|,
 * extracted on H's pattern (rho~_IJ = X_c(J)[I] diag(s_J)) and symmetrised with CSS_SYMMETRIZE.
 * The electron count of a non-orthogonal basis is Tr(rho S); mu is solved (fermi->solve_mu) on the
 * Ritz quadrature whose weights kappa_cj = (U^T Phi_c^T S~^(-1/2)^T S R_c)_j . (U^T E_1 B_0)_j make
 * it equal to the extracted Tr(rho~ S), with the rule of css_fermi.
 *   S         overlap matrix (BSR, FP64, structurally symmetric); its pattern must lie inside H's
 *   Sinv_val  S~^(-1/2) on S's pattern ([S->nnzb][b][b], e.g. from css_hprime)
 *   Hp        H' (values on H's pattern, e.g. from css_hprime) with H's row_ptr / col_idx
 *   H_val     the Hamiltonian H itself on the same pattern (for Tr(rho H))
 *   P_val     [Hp->nnzb][b][b], written;  trPS, trPH, mu_out: host double*, written
 * flags: CSS_SYMMETRIZE, CSS_REORTH_LOCAL.  Workspace: seven N x (n_colours b) blocks in the vector
 * precision (all colours at once; CSS_ERR_NOMEM when they do not fit).  After the call css_ritz
 * returns the Ritz values of H' and the weights kappa.  Synchronises. */
CSS_API css_status css_density_nonorth(css_ctx* ctx, const css_bsr* S, const double* Sinv_val, const css_bsr* Hp,
                                       const double* H_val, const int32_t* colour, const int8_t* sign,
                                       int32_t n_colours, const css_fermi* fermi, int32_t m, css_precision prec,
                                       uint32_t flags, double* P_val, double* trPS, double* trPH, double* mu_out,
                                       void* stream);

/* Many independent systems in one call (MD snapshots of uneven size).  Arrays of n_sys
 * host structs / host arrays of device pointers; mu is solved per system (fermi[s]).
 * Outputs per system: P_val[s] (device), trP[s], trPH[s], mu_out[s] (host arrays). */
CSS_API css_status css_density_batch(css_ctx* ctx, int32_t n_sys, const css_bsr* H, const int32_t* const* colour,
                             const int8_t* const* sign, const int32_t* n_colours, const css_fermi* fermi, int32_t m,
                             css_precision prec, uint32_t flags, double* const* P_val, double* trP, double* trPH,
                             double* mu_out, void* stream);

/* Colour-partitioned build of one system (paper: each colour's probe block is an independent
 * right-hand side of the shifted systems, paragraph after Eq. 4, so its block-Lanczos problem and
 * its columns of P~ need no other colour).  Only the colours with owned[c] != 0 are worked on; they
 * are renumbered 0, 1, ... in increasing c for css_ritz, and every other molecule is in no probe
 * block of this call.  A build split over ranks:
 *   1. each rank: css_density_colours(..., flags | CSS_RITZ_ONLY) for its colours, then css_ritz;
 *   2. all ranks' Ritz lists gathered in increasing colour order; css_solve_mu gives mu (the same
 *      mu, bit for bit, as one css_density call over all colours);
 *   3. each rank: css_density_colours(..., fermi->mu = that mu) writes P~_IJ = [Q_c Z_c]_I diag(s_J)
 *      for the blocks whose column molecule J has an owned colour, and ZERO for every other block;
 *   4. the ranks' P_val arrays are summed (disjoint blocks) and symmetrised by the caller.
 * Each owned colour's arithmetic is that of css_density, so the sum of the parts equals the
 * unsymmetrised P of one css_density call with the same mu bit for bit.
 *   colour, sign, H  as in css_density (colour in [0, n_colours))
 *   owned            HOST uint8[n_colours]
 *   fermi            host struct; solve_mu must be 0 (mu is an input here)
 *   flags            CSS_TWO_PASS, CSS_REORTH_LOCAL, CSS_ENERGY_WEIGHTED, CSS_RITZ_ONLY (no
 *                    CSS_SYMMETRIZE: the output is unsymmetrised)
 *   P_val, trP, trPH as in css_density (the traces cover the owned columns only)
 * Errors: INVALID_ARG for solve_mu != 0, CSS_SYMMETRIZE, no owned colour, or a colour out of range
 * (checked on the device).  Synchronises `stream`. */
CSS_API css_status css_density_colours(css_ctx* ctx, const css_bsr* H, const int32_t* colour, const int8_t* sign,
                                       int32_t n_colours, const uint8_t* owned, const css_fermi* fermi, int32_t m,
                                       css_precision prec, uint32_t flags, double* P_val, double* trP, double* trPH,
                                       void* stream);

/* mu from Ritz lists gathered from several calls (the rule of css_fermi with solve_mu: the midpoint
 * of {mu : |N(mu) - n_elec/2| <= ne_tol}, N(mu) = sum over lists t and pairs k of
 * f(lam_tk) wgt_tk; ne_tol <= 0 selects 1e-4 n_elec/2), on the GPU with the kernel of css_density.
 * Lists given in the colour order of one css_density call over all colours give exactly that call's
 * mu.
 *   n_per   HOST int32[n_lists] (pairs per list);  lam, wgt  HOST doubles, the lists concatenated
 *   mu_out  HOST double, written.  Synchronises `stream`.
 * Errors: INVALID_ARG for n_lists < 1, a negative length or kT < 0; TIMEOUT if the bounded grid
 * barrier runs out; NUMERIC for a non-finite mu. */
CSS_API css_status css_solve_mu(css_ctx* ctx, int32_t n_lists, const int32_t* n_per, const double* lam,
                                const double* wgt, double kT, double n_elec, double ne_tol, double* mu_out,
                                void* stream);

/* Ritz data of the last css_density / css_density_batch call (paper, Eq. 7: eigenvalues of
 * each colour's projected matrix and their weights w = ||Y_k||^2, Y = U^T E_1 B_0, whose
 * f-weighted sum is the quadrature of Tr P).  Host arrays: lam and wgt receive, colour by
 * colour, n_per[c] values each (n_per has n_colours entries); `capacity` is the length of
 * lam and wgt.  *n_colours receives the colour count (all systems of a batch, in order).
 * Errors: INVALID_ARG if nothing was computed yet or capacity is too small (then *n_colours
 * and n_per are still written when n_per is large enough: pass n_per = NULL to query). */
CSS_API css_status css_ritz(css_ctx* ctx, double* lam, double* wgt, int32_t* n_per, int64_t capacity,
                            int32_t* n_colours);

/* Projected block-tridiagonal matrices of the last css_density call (the Krylov-projected
 * Hamiltonian of Eq. 5-7): host arrays A and B of n_colours * m * b * b doubles ([c][j][b][b],
 * B upper triangular, sub-diagonal blocks) and nblk (n_colours; blocks in use per colour).
 * capacity = length of A and B in doubles.  INVALID_ARG if nothing was computed yet or the
 * capacity is short. */
CSS_API css_status css_projected(css_ctx* ctx, double* A, double* B, int32_t* nblk, int64_t capacity,
                                 int32_t* n_colours, int32_t* m, int32_t* b);

/* The exact-diagonalisation stage on its own (paper, Eq. 7): for each of n_col
 * block-tridiagonal projected matrices T_c (diagonal blocks A[c][j], sub-diagonal blocks
 * B[c][j] upper triangular, j < nblk[c] <= m, b x b row-major, FP64) return the eigenvalues
 * lam[c][k], the weights wgt[c][k] = |c| sum_{i<b} U[i][k]^2 (U the eigenvectors, |c| =
 * cnt[c]) and, when Z is not NULL, Z_c = U f(Lambda) U^T E_1 sqrt|c| for the given mu, kT.
 * All arrays are device arrays laid out [c][m*b] (lam, wgt) and [c][m*b][b] (Z); entries
 * beyond nblk[c]*b are zero.  Synchronises `stream`. */
CSS_API css_status css_eigen_blocks(css_ctx* ctx, int32_t n_col, int32_t b, int32_t m, const double* A, const double* B,
                                    const int32_t* nblk, const int32_t* cnt, double mu, double kT, double* lam,
                                    double* wgt, double* Z, void* stream);

/* Colouring of an explicit graph for callers that cannot allocate memory: the same colouring
 * rule and result as css_color_graph, but the call needs no css_ctx and allocates nothing
 * (no cudaMalloc, cudaFree, pinned host memory or library allocation).  Meant for code that
 * runs where new allocations are not allowed: a host application whose own allocator has
 * reserved the device memory, a latency-critical loop that must not hit cudaMalloc's implicit
 * synchronisation, or a plug-in that may use only the buffers it is handed.  The paper has no
 * counterpart; it is an operational variant of the colouring step.
 *   Scratch: one fixed device array inside this library (about 3 MB, held by every GPU that
 *   loads the library until the process exits), so n must be <= CSS_NOALLOC_MAX_VERTICES;
 *   larger graphs get CSS_ERR_INVALID_ARG (use css_color_graph).  Every call shares that
 *   array: calls that overlap on the GPU (several streams or host threads at once) race and
 *   must be serialised by the caller.
 *   The first call on a device looks the array's device address up (cudaGetSymbolAddress, with
 *   that device current) and caches it for the life of the process; make that first call before
 *   any stream capture.  The cached address does not survive cudaDeviceReset (or any other
 *   teardown of the device's primary context): do not call this entry point after one.
 *   The graph is checked as in css_color_graph (CSS_ERR_INVALID_ARG for a malformed pattern).
 *   adj_ptr, adj, colour: device arrays as in css_color_graph (colour int32[n], written);
 *   n_colours: host int32*, written; the call synchronises `stream`. */
#define CSS_NOALLOC_MAX_VERTICES 262144
CSS_API css_status css_color_graph_noalloc(int32_t n, const int32_t* adj_ptr, const int32_t* adj, uint64_t seed,
                                           int32_t* colour, int32_t* n_colours, void* stream);

/* One whole P build from a geometry and H: css_color + css_probes + css_density.  With
 * CSS_HOST_IO every array (geom->xyz, H arrays, P_val) is HOST memory and the library copies
 * in and out on `stream`; otherwise they are device arrays.  colour_out (n_mol int32,
 * same memory kind) may be NULL. */
CSS_API css_status css_pbuild(css_ctx* ctx, const css_geom* geom, const css_bsr* H, double r_col, uint64_t colour_seed,
                      uint64_t sign_seed, const css_fermi* fermi, int32_t m, css_precision prec, uint32_t flags,
                      double* P_val, int32_t* colour_out, int32_t* n_colours, double* trP, double* trPH,
                      double* mu_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CSS_H */
