/*
 * CSS density-matrix ORACLE — plain, slow, FP64 CPU code.  TEST INFRASTRUCTURE ONLY.
 *
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may load this
 * library.  It shares no code, header, table or helper with the CUDA library: it follows
 * the paper (arXiv 2605.20918, "High-performance linear-scaling electronic structure
 * method via chromatic superposition states") step by step, in the order and notation of
 * the paper, with no blocking, fusion or reordering beyond what the method states.
 *
 *   colouring   greedy multicolouring: objects closer than the cut-off get different
 *               colours (paper, CSS construction paragraph after Eq. 2; Welsh-Powell order)
 *   conflicts   same-coloured pairs closer than the cut-off on a new geometry (zero: the
 *               colouring still satisfies that condition and can be kept across MD steps)
 *   probes      |r_i> = +-1 on the indices of colour i, 0 elsewhere (same paragraph, Fig. 1c)
 *   Lanczos     block-Lanczos (Golub-Underwood) basis of K^v(H, r) (paragraph after Eq. 4)
 *   rho^K       exact diagonalisation of the projected Hamiltonian, f(lambda) (Eq. 7)
 *   extraction  rho~ = Phi rho^K <Phi|r><r| restricted to the sparse pattern (Eq. 2, Eq. 6)
 *   traces      Tr(P) and Tr(PH) = E_orbit (convergence study of Fig. 2 inset a)
 *   S^(-1/2), H' the same projection applied to an overlap S with x^(-1/2) (Eq. 8-10), and H'
 *               extracted from S~^(-1/2) H Y <o| (the paragraph after Eq. 10)
 *   non-orthogonal density  rho~ = S~^(-1/2) Phi rho^K <Phi|r~><r| from Krylov spaces of H'
 *               started at r~ = S~^(-1/2) r (Eq. 4-6 with S != I)
 *
 * Readings where the paper is silent (each one also listed in the design notes):
 *   - orthogonal basis, S = I, so H' = H and r~ = r (Eq. 4 with S = I);
 *   - one block-Lanczos per colour of MOLECULES; block width b = orbitals per molecule,
 *     column k of colour c's probe block carries orbital k of every molecule of colour c;
 *   - colour graph: min-image centre distance < R_col, in int64 fixed point
 *     q = llrint(x * 2^20); priority = (degree desc, h(seed, id) desc, id asc) with
 *     h = SplitMix64 (Steele, Lea & Flood 2014);
 *   - probe signs s[J*b+k] = -1 if bit 0 of h(sign_seed, J*b+k) is set, else +1;
 *   - Fermi-Dirac f(x) = (1 - tanh((x - mu) / (2 kT))) / 2, step function at kT = 0;
 *   - mu: the Ritz quadrature N(mu) = sum_c sum_j f(lambda_cj) w_cj of Tr P must match N_e/2;
 *     mu is the midpoint of the set where |N(mu) - N_e/2| <= ne_tol (default 1e-4 N_e/2),
 *     each end found by bisection on [min lambda - 1, max lambda + 1] until
 *     hi - lo <= 1e-13 max(1, |mid|) or 200 halvings (mid-gap for an insulator, the root for
 *     a metal; the paper works at T = 0 and does not state how mu is fixed).  The quadrature
 *     of a truncated, contaminated Krylov projection puts a thin spread of spurious Ritz weight
 *     inside the gap; ne_tol must exceed its total so that the ends of the set are the band
 *     edges, not points inside that spread;
 *   - breakdown: stop the colour's recurrence at step j when min_k R_kk of the QR of the
 *     new block is <= 1e-10 ||H Q_j||_F; its projected matrix then has j blocks;
 *   - no reorthogonalisation unless CSS_REF_REORTH_LOCAL (one more pass against Q_j, Q_j-1);
 *   - symmetrisation P = (P~ + P~^T) / 2 when CSS_REF_SYMMETRIZE is set;
 *   - CSS_REF_ENERGY_WEIGHTED: the energy-weighted density matrix (the paper's force section:
 *     rho_E = sum_i f(e_i) e_i |psi_i><psi_i|, obtained in CSS as H rho~ for an orthogonal
 *     basis), taken in each colour's Krylov subspace as Q_c T_c Z_c = Q_c U Lambda f(Lambda)
 *     U^T E_1 B_0 (H Q_c = Q_c T_c up to the Lanczos residual); mu is still fixed by f;
 *   - CSS_REF_INV_SQRT: the matrix is an overlap S (symmetric positive definite) and the
 *     function is x^(-1/2) instead of f (the paper's S^(-1/2) step, Eq. 8-10: the same
 *     block-Lanczos projection onto coloured probes, exact diagonalisation of the projected
 *     S^K and its inverse square root); no mu, Tr returns Tr S~^(-1/2) and Tr(S~^(-1/2) S).
 *   - non-orthogonal basis: the electron count is Tr(rho S) (Mulliken), evaluated as a
 *     quadrature over the Ritz pairs of H' whose weights make it equal the extracted
 *     Tr(rho~ S) exactly; mu is solved on it with the rule above.
 * Pins: the test-suite checks every function here against closed forms, dense
 * diagonalisation with LAPACK (numpy), brute force on tiny inputs and invariants; the
 * paper prints no worked numeric example, so agreement with the paper's own numbers is
 * "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* flag values of the oracle's own interface */
#define CSS_REF_SYMMETRIZE 1
#define CSS_REF_REORTH_LOCAL 4
#define CSS_REF_ENERGY_WEIGHTED 16
#define CSS_REF_INV_SQRT 32
#define CSS_REF_SIGNS_ONES 1

#define REF_OK 0
#define REF_ERR_ARG 1
#define REF_ERR_NOMEM 2
#define REF_ERR_NUMERIC 5

/* ---------------------------------------------------------------- hashing */
/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): state += golden gamma, then the
 * published 64-bit finaliser.  h(seed, x) is the output for state seed + x * gamma. */
static uint64_t ref_splitmix64(uint64_t seed, uint64_t x) {
  uint64_t z = seed + (x + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t css_ref_hash(uint64_t seed, uint64_t x) { return ref_splitmix64(seed, x); }

/* ------------------------------------------------------------ colouring */
static int64_t ref_fixed(double x) { return llrint(x * 1048576.0); }

static int64_t ref_min_image(int64_t d, int64_t Lq) {
  int64_t r = d % Lq;
  if (r > Lq / 2) r -= Lq;
  if (r < -(Lq / 2)) r += Lq;
  return r;
}

/* Colour graph: i ~ j (i != j) iff the minimum-image centre distance is < r_col.
 * Brute force over all pairs.  adj_ptr has n+1 entries; *adj is malloc'd by the oracle
 * (free with css_ref_free); neighbours are listed in increasing id. */
int css_ref_neighbours(int32_t n, const double* xyz, double box, double r_col,
                       int32_t* adj_ptr, int32_t** adj) {
  if (n < 0 || !(box > 0) || !(r_col >= 0) || !adj_ptr || !adj) return REF_ERR_ARG;
  int64_t Lq = ref_fixed(box), Rq = ref_fixed(r_col);
  int64_t R2 = Rq * Rq;
  int64_t* q = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)(n > 0 ? n : 1));
  if (!q) return REF_ERR_NOMEM;
  for (int64_t i = 0; i < 3 * (int64_t)n; ++i) q[i] = ref_fixed(xyz[i]);
  size_t cap = 1024, len = 0;
  int32_t* list = (int32_t*)malloc(sizeof(int32_t) * cap);
  if (!list) { free(q); return REF_ERR_NOMEM; }
  adj_ptr[0] = 0;
  for (int32_t i = 0; i < n; ++i) {
    for (int32_t j = 0; j < n; ++j) {
      if (j == i) continue;
      int64_t dx = ref_min_image(q[3 * i] - q[3 * j], Lq);
      int64_t dy = ref_min_image(q[3 * i + 1] - q[3 * j + 1], Lq);
      int64_t dz = ref_min_image(q[3 * i + 2] - q[3 * j + 2], Lq);
      if (dx * dx + dy * dy + dz * dz < R2) {
        if (len == cap) {
          cap *= 2;
          int32_t* t = (int32_t*)realloc(list, sizeof(int32_t) * cap);
          if (!t) { free(list); free(q); return REF_ERR_NOMEM; }
          list = t;
        }
        list[len++] = j;
      }
    }
    adj_ptr[i + 1] = (int32_t)len;
  }
  free(q);
  *adj = list;
  return REF_OK;
}

void css_ref_free(void* p) { free(p); }

/* priority order: degree desc, then key desc, then id asc */
typedef struct { int32_t id, deg; uint64_t key; } ref_prio;

static int ref_prio_cmp(const void* a, const void* b) {
  const ref_prio* x = (const ref_prio*)a;
  const ref_prio* y = (const ref_prio*)b;
  if (x->deg != y->deg) return x->deg > y->deg ? -1 : 1;
  if (x->key != y->key) return x->key > y->key ? -1 : 1;
  return x->id < y->id ? -1 : (x->id > y->id);
}

/* Sequential greedy colouring in priority order: each vertex takes the smallest colour
 * not used by an already coloured neighbour. */
int css_ref_color_graph(int32_t n, const int32_t* adj_ptr, const int32_t* adj, uint64_t seed,
                        int32_t* colour, int32_t* n_colours) {
  if (n < 0 || !adj_ptr || !colour || !n_colours) return REF_ERR_ARG;
  ref_prio* order = (ref_prio*)malloc(sizeof(ref_prio) * (size_t)(n > 0 ? n : 1));
  if (!order) return REF_ERR_NOMEM;
  for (int32_t i = 0; i < n; ++i) {
    order[i].id = i;
    order[i].deg = adj_ptr[i + 1] - adj_ptr[i];
    order[i].key = ref_splitmix64(seed, (uint64_t)i);
  }
  qsort(order, (size_t)n, sizeof(ref_prio), ref_prio_cmp);
  for (int32_t i = 0; i < n; ++i) colour[i] = -1;
  int32_t maxdeg = 0;
  for (int32_t i = 0; i < n; ++i)
    if (adj_ptr[i + 1] - adj_ptr[i] > maxdeg) maxdeg = adj_ptr[i + 1] - adj_ptr[i];
  char* used = (char*)calloc((size_t)maxdeg + 2, 1);
  if (!used) { free(order); return REF_ERR_NOMEM; }
  int32_t nc = 0;
  for (int32_t t = 0; t < n; ++t) {
    int32_t v = order[t].id;
    memset(used, 0, (size_t)maxdeg + 2);
    for (int32_t k = adj_ptr[v]; k < adj_ptr[v + 1]; ++k) {
      int32_t c = colour[adj[k]];
      if (c >= 0 && c <= maxdeg) used[c] = 1;
    }
    int32_t c = 0;
    while (used[c]) ++c;
    colour[v] = c;
    if (c + 1 > nc) nc = c + 1;
  }
  free(used);
  free(order);
  *n_colours = nc;
  return REF_OK;
}

int css_ref_color(int32_t n, const double* xyz, double box, double r_col, uint64_t seed,
                  int32_t* colour, int32_t* n_colours) {
  int32_t* adj_ptr = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
  int32_t* adj = NULL;
  if (!adj_ptr) return REF_ERR_NOMEM;
  int st = css_ref_neighbours(n, xyz, box, r_col, adj_ptr, &adj);
  if (st == REF_OK) st = css_ref_color_graph(n, adj_ptr, adj, seed, colour, n_colours);
  free(adj);
  free(adj_ptr);
  return st;
}

/* Colouring conflicts on a (new) geometry: the number of unordered pairs {i, j} that share a
 * colour although their minimum-image centre distance is < r_col, i.e. the edges of this
 * geometry's colour graph that the colouring violates.  Zero means the colouring is still a
 * valid distance-r_col colouring (the condition of the CSS construction paragraph after
 * Eq. 2), so it may be kept from one MD step to the next.  Brute force over all pairs. */
int css_ref_color_conflicts(int32_t n, const double* xyz, double box, double r_col, const int32_t* colour,
                            int64_t* count) {
  if (n < 0 || !(box > 0) || !(r_col >= 0) || !colour || !count) return REF_ERR_ARG;
  int64_t Lq = ref_fixed(box), Rq = ref_fixed(r_col);
  int64_t R2 = Rq * Rq;
  int64_t k = 0;
  for (int32_t i = 0; i < n; ++i) {
    for (int32_t j = i + 1; j < n; ++j) {
      if (colour[i] != colour[j]) continue;
      int64_t dx = ref_min_image(ref_fixed(xyz[3 * i]) - ref_fixed(xyz[3 * j]), Lq);
      int64_t dy = ref_min_image(ref_fixed(xyz[3 * i + 1]) - ref_fixed(xyz[3 * j + 1]), Lq);
      int64_t dz = ref_min_image(ref_fixed(xyz[3 * i + 2]) - ref_fixed(xyz[3 * j + 2]), Lq);
      if (dx * dx + dy * dy + dz * dz < R2) ++k;
    }
  }
  *count = k;
  return REF_OK;
}

/* --------------------------------------------------------------- probes */
int css_ref_probes(const int32_t* colour, int32_t n_mol, int32_t b, uint64_t sign_seed, int flags,
                   int8_t* sign) {
  if (n_mol < 0 || b < 1 || !sign) return REF_ERR_ARG;
  (void)colour;
  for (int64_t i = 0; i < (int64_t)n_mol * b; ++i) {
    if (flags & CSS_REF_SIGNS_ONES) sign[i] = 1;
    else sign[i] = (ref_splitmix64(sign_seed, (uint64_t)i) & 1ULL) ? (int8_t)-1 : (int8_t)1;
  }
  return REF_OK;
}

/* ------------------------------------------------------- dense helpers */
/* y (N x w) = H (BSR) x (N x w); row-major vectors with leading dimension w */
static void ref_bsr_mul(int32_t n_brow, int32_t b, const int32_t* row_ptr, const int32_t* col_idx,
                        const double* val, const double* x, double* y, int32_t w) {
  /* rows are independent; threads split them only when no outer parallel region is active */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (!omp_in_parallel())
#endif
  for (int32_t I = 0; I < n_brow; ++I) {
    for (int32_t a = 0; a < b; ++a)
      for (int32_t k = 0; k < w; ++k) y[((size_t)I * b + a) * w + k] = 0.0;
    for (int32_t p = row_ptr[I]; p < row_ptr[I + 1]; ++p) {
      int32_t J = col_idx[p];
      const double* h = val + (size_t)p * b * b;
      for (int32_t a = 0; a < b; ++a)
        for (int32_t c = 0; c < b; ++c) {
          double hac = h[a * b + c];
          for (int32_t k = 0; k < w; ++k)
            y[((size_t)I * b + a) * w + k] += hac * x[((size_t)J * b + c) * w + k];
        }
    }
  }
}

/* Householder vector of x (length n): H x = beta e_1 with H = I - tau v v^T, v[0] = 1. */
static void ref_house(int64_t n, const double* x, int64_t incx, double* v, double* tau, double* beta) {
  double sigma = 0.0;
  for (int64_t i = 1; i < n; ++i) sigma += x[i * incx] * x[i * incx];
  double x0 = x[0];
  v[0] = 1.0;
  if (sigma == 0.0) {
    for (int64_t i = 1; i < n; ++i) v[i] = 0.0;
    *tau = 0.0;
    *beta = x0;
    return;
  }
  double mu = sqrt(x0 * x0 + sigma);
  double v0 = (x0 <= 0.0) ? x0 - mu : -sigma / (x0 + mu);
  *tau = 2.0 * v0 * v0 / (sigma + v0 * v0);
  for (int64_t i = 1; i < n; ++i) v[i] = x[i * incx] / v0;
  *beta = mu;
}

/* Thin QR of W (N x b, row-major) by Householder reflections: W = Q R, diag(R) >= 0.
 * Q (N x b) and R (b x b, upper) are outputs; W is destroyed. */
static void ref_qr(int64_t N, int32_t b, double* W, double* Q, double* R, double* v) {
  double* taus = (double*)malloc(sizeof(double) * b);
  double* vs = (double*)malloc(sizeof(double) * (size_t)N * b);
  for (int32_t k = 0; k < b; ++k) {
    double tau, beta;
    ref_house(N - k, W + (size_t)k * b + k, b, v, &tau, &beta);
    for (int64_t i = 0; i < N - k; ++i) vs[(size_t)k * N + i] = v[i];
    taus[k] = tau;
    for (int32_t c = k; c < b; ++c) {  /* W[k:, c] -= tau v (v^T W[k:, c]) */
      double s = 0.0;
      for (int64_t i = 0; i < N - k; ++i) s += v[i] * W[(size_t)(k + i) * b + c];
      s *= tau;
      for (int64_t i = 0; i < N - k; ++i) W[(size_t)(k + i) * b + c] -= s * v[i];
    }
  }
  for (int32_t r = 0; r < b; ++r)
    for (int32_t c = 0; c < b; ++c) R[r * b + c] = (c >= r) ? W[(size_t)r * b + c] : 0.0;
  /* Q = H_0 ... H_{b-1} [I_b; 0] */
  for (int64_t i = 0; i < N; ++i)
    for (int32_t c = 0; c < b; ++c) Q[(size_t)i * b + c] = (i == c) ? 1.0 : 0.0;
  for (int32_t k = b - 1; k >= 0; --k) {
    const double* vk = vs + (size_t)k * N;
    for (int32_t c = 0; c < b; ++c) {
      double s = 0.0;
      for (int64_t i = 0; i < N - k; ++i) s += vk[i] * Q[(size_t)(k + i) * b + c];
      s *= taus[k];
      for (int64_t i = 0; i < N - k; ++i) Q[(size_t)(k + i) * b + c] -= s * vk[i];
    }
  }
  for (int32_t r = 0; r < b; ++r)
    if (R[r * b + r] < 0.0) {
      for (int32_t c = 0; c < b; ++c) R[r * b + c] = -R[r * b + c];
      for (int64_t i = 0; i < N; ++i) Q[(size_t)i * b + r] = -Q[(size_t)i * b + r];
    }
  free(vs);
  free(taus);
}

/* Symmetric eigen-decomposition: Householder tridiagonalisation with the orthogonal
 * factor accumulated, then implicit symmetric QR steps with Wilkinson shifts
 * (Golub & Van Loan, "Matrix Computations", Alg. 8.3.1 and 8.3.3).
 * A (n x n, row-major, symmetric) is overwritten by the eigenvectors (column j belongs to
 * w[j]); w ascending.  Returns REF_ERR_NUMERIC if the QR steps do not converge. */
int css_ref_eigh(int32_t n, double* A, double* w) {
  if (n < 1) return REF_ERR_ARG;
  double* Q = (double*)calloc((size_t)n * n, sizeof(double));
  double* d = (double*)malloc(sizeof(double) * n);
  double* e = (double*)calloc((size_t)n, sizeof(double));
  double* v = (double*)malloc(sizeof(double) * n);
  double* p = (double*)malloc(sizeof(double) * n);
  if (!Q || !d || !e || !v || !p) { free(Q); free(d); free(e); free(v); free(p); return REF_ERR_NOMEM; }
  for (int32_t i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
  /* tridiagonalisation: A <- P A P, Q <- Q P, P = I - tau v v^T acting on rows/cols k+1.. */
  for (int32_t k = 0; k + 2 < n; ++k) {
    int32_t m = n - k - 1;
    double tau, beta;
    ref_house(m, A + (size_t)(k + 1) * n + k, n, v, &tau, &beta);
    if (tau != 0.0) {
      /* p = tau A22 v ; q = p - (tau/2)(p^T v) v ; A22 -= v q^T + q v^T */
      for (int32_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int32_t j = 0; j < m; ++j) s += A[(size_t)(k + 1 + i) * n + (k + 1 + j)] * v[j];
        p[i] = tau * s;
      }
      double pv = 0.0;
      for (int32_t i = 0; i < m; ++i) pv += p[i] * v[i];
      for (int32_t i = 0; i < m; ++i) p[i] -= 0.5 * tau * pv * v[i];
      for (int32_t i = 0; i < m; ++i)
        for (int32_t j = 0; j < m; ++j)
          A[(size_t)(k + 1 + i) * n + (k + 1 + j)] -= v[i] * p[j] + p[i] * v[j];
      /* Q[:, k+1:] -= tau (Q[:, k+1:] v) v^T */
      for (int32_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t j = 0; j < m; ++j) s += Q[(size_t)i * n + (k + 1 + j)] * v[j];
        s *= tau;
        for (int32_t j = 0; j < m; ++j) Q[(size_t)i * n + (k + 1 + j)] -= s * v[j];
      }
    }
    A[(size_t)(k + 1) * n + k] = beta;
    A[(size_t)k * n + (k + 1)] = beta;
    for (int32_t i = 1; i < m; ++i) {
      A[(size_t)(k + 1 + i) * n + k] = 0.0;
      A[(size_t)k * n + (k + 1 + i)] = 0.0;
    }
  }
  for (int32_t i = 0; i < n; ++i) d[i] = A[(size_t)i * n + i];
  for (int32_t i = 0; i + 1 < n; ++i) e[i] = A[(size_t)(i + 1) * n + i];
  /* implicit symmetric QR with Wilkinson shift on (d, e); rotations accumulated into Q */
  int status = REF_OK;
  int32_t hi = n - 1;
  long iter = 0, max_iter = 60L * n + 100;
  while (hi > 0) {
    /* deflate negligible off-diagonals */
    for (int32_t i = 0; i < hi; ++i)
      if (fabs(e[i]) <= 1e-300 + 2.220446049250313e-16 * (fabs(d[i]) + fabs(d[i + 1]))) e[i] = 0.0;
    if (e[hi - 1] == 0.0) { --hi; continue; }
    int32_t lo = hi - 1;
    while (lo > 0 && e[lo - 1] != 0.0) --lo;
    if (++iter > max_iter) { status = REF_ERR_NUMERIC; break; }
    /* Wilkinson shift from the trailing 2x2 of the unreduced block [lo, hi] */
    double dd = 0.5 * (d[hi - 1] - d[hi]);
    double e2 = e[hi - 1] * e[hi - 1];
    double sgn = dd >= 0.0 ? 1.0 : -1.0;
    double mu = d[hi] - e2 / (dd + sgn * sqrt(dd * dd + e2));
    double x = d[lo] - mu, z = e[lo];
    for (int32_t k = lo; k < hi; ++k) {
      /* Givens rotation [c s; -s c] zeroing z against x */
      double r = hypot(x, z);
      double c = x / r, s = -z / r;
      /* apply G^T T G on rows/cols k, k+1 */
      if (k > lo) e[k - 1] = r;
      double dk = d[k], dk1 = d[k + 1], ek = e[k];
      d[k] = c * c * dk - 2.0 * c * s * ek + s * s * dk1;
      d[k + 1] = s * s * dk + 2.0 * c * s * ek + c * c * dk1;
      e[k] = c * s * (dk - dk1) + (c * c - s * s) * ek;
      if (k + 1 < hi) {
        x = e[k];
        z = -s * e[k + 1];
        e[k + 1] = c * e[k + 1];
      }
      for (int32_t i = 0; i < n; ++i) {
        double qa = Q[(size_t)i * n + k], qb = Q[(size_t)i * n + k + 1];
        Q[(size_t)i * n + k] = c * qa - s * qb;
        Q[(size_t)i * n + k + 1] = s * qa + c * qb;
      }
    }
  }
  /* sort ascending (selection sort, columns follow) */
  for (int32_t i = 0; i < n; ++i) {
    int32_t kmin = i;
    for (int32_t j = i + 1; j < n; ++j) if (d[j] < d[kmin]) kmin = j;
    if (kmin != i) {
      double t = d[i]; d[i] = d[kmin]; d[kmin] = t;
      for (int32_t r = 0; r < n; ++r) {
        double u = Q[(size_t)r * n + i];
        Q[(size_t)r * n + i] = Q[(size_t)r * n + kmin];
        Q[(size_t)r * n + kmin] = u;
      }
    }
  }
  memcpy(A, Q, sizeof(double) * (size_t)n * n);
  memcpy(w, d, sizeof(double) * n);
  free(Q); free(d); free(e); free(v); free(p);
  return status;
}

/* --------------------------------------------------------- block Lanczos */
typedef struct {
  int32_t n_brow, b;
  const int32_t *row_ptr, *col_idx;
  const double* val;
} ref_h;

/* Block-Lanczos for colour c (paper, paragraph after Eq. 4; Golub-Underwood):
 *   Q_1 = R_c / sqrt|c|, B_0 = sqrt|c| I, Q_0 = 0  (or Q_1 = Q1start when it is given: the
 *   orthonormal factor of a general start block, whose B_0 the caller keeps)
 *   W = H Q_j - Q_{j-1} B_{j-1}^T ;  A_j = sym(Q_j^T W) ;  W -= Q_j A_j
 *   W = Q_{j+1} B_j  (QR)
 * T (nmax x nmax, nmax = m b) receives the block-tridiagonal projected matrix
 * T[j][j] = A_j, T[j+1][j] = B_j, T[j][j+1] = B_j^T; returns the number of blocks used.
 * If Zc != NULL (pass 2) X (N x b) accumulates sum_j Q_j Zc[j-th block rows]. */
static int32_t ref_lanczos_colour(const ref_h* H, const int32_t* colour, const int8_t* sign, int32_t c,
                                  int32_t m, int flags, double* T, const double* Zc, double* X,
                                  double* Qout, const double* Q1start) {
  const int32_t b = H->b;
  const int64_t N = (int64_t)H->n_brow * b;
  const int32_t nmax = m * b;
  double* Qp = (double*)calloc((size_t)N * b, sizeof(double));
  double* Qj = (double*)calloc((size_t)N * b, sizeof(double));
  double* W = (double*)malloc(sizeof(double) * (size_t)N * b);
  double* Wc = (double*)malloc(sizeof(double) * (size_t)N * b);
  double* Bp = (double*)calloc((size_t)b * b, sizeof(double));
  double* A = (double*)malloc(sizeof(double) * b * b);
  double* R = (double*)malloc(sizeof(double) * b * b);
  double* C = (double*)malloc(sizeof(double) * b * b);
  double* v = (double*)malloc(sizeof(double) * (size_t)N);
  if (Q1start) {
    memcpy(Qj, Q1start, sizeof(double) * (size_t)N * b);
  } else {
    int64_t cnt = 0;
    for (int32_t J = 0; J < H->n_brow; ++J) cnt += (colour[J] == c);
    double sq = sqrt((double)cnt);
    for (int32_t J = 0; J < H->n_brow; ++J)
      if (colour[J] == c)
        for (int32_t k = 0; k < b; ++k) Qj[((size_t)J * b + k) * b + k] = sign[(size_t)J * b + k] / sq;
  }
  if (T) memset(T, 0, sizeof(double) * (size_t)nmax * nmax);
  if (X) memset(X, 0, sizeof(double) * (size_t)N * b);
  int32_t used = 0;
  for (int32_t j = 0; j < m; ++j) {
    if (Qout)
      for (int64_t i = 0; i < N; ++i)
        for (int32_t k = 0; k < b; ++k) Qout[(size_t)i * nmax + (size_t)j * b + k] = Qj[(size_t)i * b + k];
    if (X && Zc)  /* X += Q_j Zc[j b : (j+1) b, :] */
      for (int64_t i = 0; i < N; ++i)
        for (int32_t k = 0; k < b; ++k) {
          double s = 0.0;
          for (int32_t l = 0; l < b; ++l) s += Qj[(size_t)i * b + l] * Zc[((size_t)j * b + l) * b + k];
          X[(size_t)i * b + k] += s;
        }
    ref_bsr_mul(H->n_brow, b, H->row_ptr, H->col_idx, H->val, Qj, W, b);
    double hq = 0.0;
    for (int64_t i = 0; i < N * b; ++i) hq += W[i] * W[i];
    hq = sqrt(hq);
    for (int64_t i = 0; i < N; ++i)  /* W -= Q_{j-1} B_{j-1}^T */
      for (int32_t k = 0; k < b; ++k) {
        double s = 0.0;
        for (int32_t l = 0; l < b; ++l) s += Qp[(size_t)i * b + l] * Bp[k * b + l];
        W[(size_t)i * b + k] -= s;
      }
    for (int32_t k = 0; k < b; ++k)  /* A = Q_j^T W */
      for (int32_t l = 0; l < b; ++l) {
        double s = 0.0;
        for (int64_t i = 0; i < N; ++i) s += Qj[(size_t)i * b + k] * W[(size_t)i * b + l];
        A[k * b + l] = s;
      }
    for (int32_t k = 0; k < b; ++k)
      for (int32_t l = 0; l < k; ++l) {
        double s = 0.5 * (A[k * b + l] + A[l * b + k]);
        A[k * b + l] = s;
        A[l * b + k] = s;
      }
    for (int64_t i = 0; i < N; ++i)  /* W -= Q_j A_j */
      for (int32_t k = 0; k < b; ++k) {
        double s = 0.0;
        for (int32_t l = 0; l < b; ++l) s += Qj[(size_t)i * b + l] * A[l * b + k];
        W[(size_t)i * b + k] -= s;
      }
    if (flags & CSS_REF_REORTH_LOCAL) {  /* one more pass against Q_j, then Q_{j-1} */
      const double* bases[2] = {Qj, Qp};
      for (int t = 0; t < 2; ++t) {
        const double* Bq = bases[t];
        for (int32_t k = 0; k < b; ++k)
          for (int32_t l = 0; l < b; ++l) {
            double s = 0.0;
            for (int64_t i = 0; i < N; ++i) s += Bq[(size_t)i * b + k] * W[(size_t)i * b + l];
            C[k * b + l] = s;
          }
        for (int64_t i = 0; i < N; ++i)
          for (int32_t k = 0; k < b; ++k) {
            double s = 0.0;
            for (int32_t l = 0; l < b; ++l) s += Bq[(size_t)i * b + l] * C[l * b + k];
            W[(size_t)i * b + k] -= s;
          }
      }
    }
    if (T)
      for (int32_t k = 0; k < b; ++k)
        for (int32_t l = 0; l < b; ++l) T[((size_t)j * b + k) * nmax + (size_t)j * b + l] = A[k * b + l];
    used = j + 1;
    if (j + 1 == m) break;
    memcpy(Wc, W, sizeof(double) * (size_t)N * b);
    ref_qr(N, b, Wc, Qp /* receives Q_{j+1} */, R, v);
    double rmin = INFINITY;
    for (int32_t k = 0; k < b; ++k) if (R[k * b + k] < rmin) rmin = R[k * b + k];
    if (!(rmin > 1e-10 * hq)) break;  /* breakdown: invariant subspace reached */
    if (T)
      for (int32_t k = 0; k < b; ++k)
        for (int32_t l = 0; l < b; ++l) {
          T[((size_t)(j + 1) * b + k) * nmax + (size_t)j * b + l] = R[k * b + l];
          T[((size_t)j * b + l) * nmax + (size_t)(j + 1) * b + k] = R[k * b + l];
        }
    /* shift: Q_{j-1} <- Q_j, Q_j <- Q_{j+1} */
    double* t = Qp; Qp = Qj; Qj = t;
    memcpy(Bp, R, sizeof(double) * b * b);
  }
  free(Qp); free(Qj); free(W); free(Wc); free(Bp); free(A); free(R); free(C); free(v);
  return used;
}

/* test hook: the projected matrix of one colour, and (optionally) its Lanczos basis */
int css_ref_lanczos(int32_t n_brow, int32_t b, const int32_t* row_ptr, const int32_t* col_idx,
                    const double* val, const int32_t* colour, const int8_t* sign, int32_t c, int32_t m,
                    int flags, double* T, double* Q, int32_t* n_blocks) {
  if (n_brow < 1 || b < 1 || m < 1 || !T || !n_blocks) return REF_ERR_ARG;
  ref_h H = {n_brow, b, row_ptr, col_idx, val};
  *n_blocks = ref_lanczos_colour(&H, colour, sign, c, m, flags, T, NULL, NULL, Q, NULL);
  return REF_OK;
}

/* ----------------------------------------------------------- Fermi-Dirac */
static double ref_fermi(double x, double mu, double kT) {
  if (kT > 0.0) return 0.5 * (1.0 - tanh((x - mu) / (2.0 * kT)));
  if (x < mu) return 1.0;
  if (x > mu) return 0.0;
  return 0.5;
}

double css_ref_fermi(double x, double mu, double kT) { return ref_fermi(x, mu, kT); }

/* ------------------------------------------------------------- density */
/* Projected eigen-data of one colour: eigenvalues lambda (n), weights w_j = ||Y_j||^2 with
 * Y = U^T E_1 B_0 = sqrt|c| U[0:b, :]^T (Eq. 6-7), and U itself. */
static int ref_colour_eigen(const ref_h* H, const int32_t* colour, const int8_t* sign, int32_t c,
                            int32_t m, int flags, int32_t* n_out, double* lam, double* wgt, double* U,
                            int32_t* breakdown, int64_t cnt) {
  const int32_t b = H->b, nmax = m * b;
  double* T = (double*)malloc(sizeof(double) * (size_t)nmax * nmax);
  if (!T) return REF_ERR_NOMEM;
  int32_t blocks = ref_lanczos_colour(H, colour, sign, c, m, flags, T, NULL, NULL, NULL, NULL);
  if (blocks < m) *breakdown = 1;
  int32_t n = blocks * b;
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = 0; j < n; ++j) U[(size_t)i * n + j] = T[(size_t)i * nmax + j];
  free(T);
  int st = css_ref_eigh(n, U, lam);
  for (int32_t j = 0; j < n; ++j) {
    double s = 0.0;
    for (int32_t k = 0; k < b; ++k) s += U[(size_t)k * n + j] * U[(size_t)k * n + j];
    wgt[j] = (double)cnt * s;
  }
  *n_out = n;
  return st;
}

/* mu from a Ritz quadrature N(mu) = sum_t sum_j f(lam_tj; mu) wgt_tj (nj[t] pairs per colour,
 * stride nmax): the midpoint of the interval where |N(mu) - N_e/2| <= ne_tol, each end found
 * by bisection on [min lam - 1, max lam + 1] (lower end: smallest mu with N - N_e/2 >= -ne_tol;
 * upper end: largest mu with N - N_e/2 <= +ne_tol) until hi - lo <= 1e-13 max(1, |mid|) or 200
 * halvings.  For a metal both ends meet at the root; for an insulator the interval is the gap
 * and mu lands mid-gap instead of at a band edge. */
static double ref_solve_mu(int32_t nwork, const int32_t* nj, int32_t nmax, const double* lam, const double* wgt,
                           double kT, double n_elec, double ne_tol) {
  double lo0 = INFINITY, hi0 = -INFINITY;
  for (int32_t t = 0; t < nwork; ++t)
    for (int32_t j = 0; j < nj[t]; ++j) {
      double x = lam[(size_t)t * nmax + j];
      if (x < lo0) lo0 = x;
      if (x > hi0) hi0 = x;
    }
  lo0 -= 1.0;
  hi0 += 1.0;
  double ends[2];
  for (int side = 0; side < 2; ++side) {
    double lo = lo0, hi = hi0;
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (lo + hi);
      double g = 0.0;
      for (int32_t t = 0; t < nwork; ++t)
        for (int32_t j = 0; j < nj[t]; ++j)
          g += ref_fermi(lam[(size_t)t * nmax + j], mid, kT) * wgt[(size_t)t * nmax + j];
      g -= 0.5 * n_elec;
      if (side == 0) {
        if (g >= -ne_tol) hi = mid;
        else lo = mid;
      } else {
        if (g <= ne_tol) lo = mid;
        else hi = mid;
      }
      if (hi - lo <= 1e-13 * fmax(1.0, fabs(mid))) break;
    }
    ends[side] = 0.5 * (lo + hi);
  }
  return 0.5 * (ends[0] + ends[1]);
}

/* mu from Ritz lists gathered elsewhere (n_lists lists of n_per[t] pairs, stride nmax), with
 * the rule of css_ref_density; the lists enter the sums in the order given. */
int css_ref_solve_mu(int32_t n_lists, const int32_t* n_per, int32_t nmax, const double* lam, const double* wgt,
                     double kT, double n_elec, double ne_tol, double* mu) {
  if (n_lists < 1 || nmax < 1 || !n_per || !lam || !wgt || !mu || kT < 0.0) return REF_ERR_ARG;
  if (!(ne_tol > 0.0)) ne_tol = 1e-4 * fmax(1.0, 0.5 * n_elec);
  *mu = ref_solve_mu(n_lists, n_per, nmax, lam, wgt, kT, n_elec, ne_tol);
  return isfinite(*mu) ? REF_OK : REF_ERR_NUMERIC;
}

/* Full CSS density matrix on H's pattern.  colour_subset (n_subset entries) restricts the
 * work to those colours (then solve_mu must be 0 and only the blocks (I, J) with colour(J)
 * in the subset are written).  Returns REF_OK; *n_breakdown counts truncated colours. */
int css_ref_density(int32_t n_brow, int32_t b, int32_t nnzb, const int32_t* row_ptr, const int32_t* col_idx,
                    const double* val, const int32_t* colour, const int8_t* sign, int32_t n_colours,
                    double mu, double kT, double n_elec, double ne_tol, int solve_mu, int32_t m, int flags,
                    const int32_t* colour_subset, int32_t n_subset, double* P_val, double* trP,
                    double* trPH, double* mu_out, int32_t* n_breakdown) {
  if (n_brow < 1 || b < 1 || m < 1 || n_colours < 1 || nnzb < n_brow || !P_val) return REF_ERR_ARG;
  if (colour_subset && solve_mu) return REF_ERR_ARG;
  if (kT < 0.0) return REF_ERR_ARG;
  if (!(ne_tol > 0.0)) ne_tol = 1e-4 * fmax(1.0, 0.5 * n_elec);
  ref_h H = {n_brow, b, row_ptr, col_idx, val};
  const int64_t N = (int64_t)n_brow * b;
  const int32_t nmax = m * b;
  int32_t nwork = colour_subset ? n_subset : n_colours;
  int32_t* todo = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nwork > 0 ? nwork : 1));
  int64_t* cnt = (int64_t*)calloc((size_t)n_colours, sizeof(int64_t));
  double* lam = (double*)malloc(sizeof(double) * (size_t)nwork * nmax);
  double* wgt = (double*)malloc(sizeof(double) * (size_t)nwork * nmax);
  int32_t* nj = (int32_t*)calloc((size_t)(nwork > 0 ? nwork : 1), sizeof(int32_t));
  int32_t* brk = (int32_t*)calloc((size_t)(nwork > 0 ? nwork : 1), sizeof(int32_t));
  if (!todo || !cnt || !lam || !wgt || !nj || !brk) return REF_ERR_NOMEM;
  for (int32_t t = 0; t < nwork; ++t) todo[t] = colour_subset ? colour_subset[t] : t;
  for (int32_t J = 0; J < n_brow; ++J) {
    if (colour[J] < 0 || colour[J] >= n_colours) return REF_ERR_ARG;
    cnt[colour[J]]++;
  }
  int status = REF_OK;
  /* pass 1: Lanczos + exact diagonalisation per colour -> Ritz values and weights */
#pragma omp parallel for schedule(dynamic, 1) if (nwork > 1)
  for (int32_t t = 0; t < nwork; ++t) {
    int32_t c = todo[t];
    if (cnt[c] == 0) { nj[t] = 0; continue; }
    double* U = (double*)malloc(sizeof(double) * (size_t)nmax * nmax);
    int st = ref_colour_eigen(&H, colour, sign, c, m, flags, &nj[t], lam + (size_t)t * nmax,
                              wgt + (size_t)t * nmax, U, &brk[t], cnt[c]);
    if (st != REF_OK) {
#pragma omp critical
      status = st;
    }
    free(U);
  }
  if (status != REF_OK) return status;
  /* chemical potential from the Ritz quadrature N(mu) = sum_c sum_j f(lambda_cj; mu) w_cj */
  if (solve_mu && !(flags & CSS_REF_INV_SQRT)) mu = ref_solve_mu(nwork, nj, nmax, lam, wgt, kT, n_elec, ne_tol);
  if (mu_out) *mu_out = mu;
  /* pass 2: rebuild each colour's basis, X_c = Q_c Z_c with Z_c = U f(Lambda) U^T E_1 B_0,
   * and extract P~_IJ = X_c[I] diag(s_J) on the pattern (Eq. 2, Eq. 6) */
  int32_t* brow = (int32_t*)malloc(sizeof(int32_t) * (size_t)nnzb);
  for (int32_t I = 0; I < n_brow; ++I)
    for (int32_t p = row_ptr[I]; p < row_ptr[I + 1]; ++p) brow[p] = I;
  double* Pt = (double*)malloc(sizeof(double) * (size_t)nnzb * b * b);
  if (!brow || !Pt) return REF_ERR_NOMEM;
  for (size_t i = 0; i < (size_t)nnzb * b * b; ++i) Pt[i] = P_val[i];
#pragma omp parallel for schedule(dynamic, 1) if (nwork > 1)
  for (int32_t t = 0; t < nwork; ++t) {
    int32_t c = todo[t];
    if (cnt[c] == 0) continue;
    double* U = (double*)malloc(sizeof(double) * (size_t)nmax * nmax);
    double* lam2 = (double*)malloc(sizeof(double) * nmax);
    double* wg2 = (double*)malloc(sizeof(double) * nmax);
    double* Z = (double*)malloc(sizeof(double) * (size_t)nmax * b);
    double* fy = (double*)malloc(sizeof(double) * (size_t)nmax * b);
    double* X = (double*)malloc(sizeof(double) * (size_t)N * b);
    int32_t n = 0, bk = 0;
    ref_colour_eigen(&H, colour, sign, c, m, flags, &n, lam2, wg2, U, &bk, cnt[c]);
    double sq = sqrt((double)cnt[c]);
    for (int32_t j = 0; j < n; ++j) {  /* f(Lambda) Y (Lambda f(Lambda) Y), Y[j][k] = sqrt|c| U[k][j] */
      double fj;
      if (flags & CSS_REF_INV_SQRT)  /* S^K is positive definite: its Ritz values are > 0 */
        fj = lam2[j] > 0.0 ? 1.0 / sqrt(lam2[j]) : NAN;
      else
        fj = ref_fermi(lam2[j], mu, kT);
      if (flags & CSS_REF_ENERGY_WEIGHTED) fj *= lam2[j];
      for (int32_t k = 0; k < b; ++k) fy[(size_t)j * b + k] = fj * sq * U[(size_t)k * n + j];
    }
    for (int32_t i = 0; i < nmax; ++i)
      for (int32_t k = 0; k < b; ++k) {
        double s = 0.0;
        if (i < n)
          for (int32_t j = 0; j < n; ++j) s += U[(size_t)i * n + j] * fy[(size_t)j * b + k];
        Z[(size_t)i * b + k] = s;
      }
    ref_lanczos_colour(&H, colour, sign, c, n / b, flags, NULL, Z, X, NULL, NULL);
    for (int32_t p = 0; p < nnzb; ++p) {
      int32_t J = col_idx[p];
      if (colour[J] != c) continue;
      int32_t I = brow[p];
      for (int32_t a = 0; a < b; ++a)
        for (int32_t k = 0; k < b; ++k)
          Pt[(size_t)p * b * b + a * b + k] = X[((size_t)I * b + a) * b + k] * sign[(size_t)J * b + k];
    }
    free(U); free(lam2); free(wg2); free(Z); free(fy); free(X);
  }
  /* symmetrise on the pattern and take the traces */
  for (int32_t p = 0; p < nnzb; ++p) {
    int32_t I = brow[p], J = col_idx[p];
    int32_t q = -1;
    for (int32_t r = row_ptr[J]; r < row_ptr[J + 1]; ++r)
      if (col_idx[r] == I) { q = r; break; }
    for (int32_t a = 0; a < b; ++a)
      for (int32_t k = 0; k < b; ++k) {
        double x = Pt[(size_t)p * b * b + a * b + k];
        if ((flags & CSS_REF_SYMMETRIZE) && q >= 0) x = 0.5 * (x + Pt[(size_t)q * b * b + k * b + a]);
        P_val[(size_t)p * b * b + a * b + k] = x;
      }
  }
  /* with a colour subset the traces cover the written blocks only */
  char* inset = (char*)calloc((size_t)n_colours, 1);
  for (int32_t t = 0; t < nwork; ++t) inset[todo[t]] = 1;
  double tp = 0.0, tph = 0.0;
  for (int32_t p = 0; p < nnzb; ++p) {
    int32_t I = brow[p], J = col_idx[p];
    if (!inset[colour[J]]) continue;
    for (int32_t a = 0; a < b; ++a)
      for (int32_t k = 0; k < b; ++k) {
        double x = P_val[(size_t)p * b * b + a * b + k];
        tph += x * val[(size_t)p * b * b + a * b + k];
        if (I == J && a == k) tp += x;
      }
  }
  if (trP) *trP = tp;
  if (trPH) *trPH = tph;
  int32_t nb = 0;
  for (int32_t t = 0; t < nwork; ++t) nb += brk[t];
  if (n_breakdown) *n_breakdown = nb;
  free(inset); free(brow); free(Pt); free(todo); free(cnt); free(lam); free(wgt); free(nj); free(brk);
  if (!isfinite(tp) || !isfinite(tph)) return REF_ERR_NUMERIC;
  return REF_OK;
}

/* H' of a non-orthogonal basis (paper, Eq. 8-10 and the paragraph after them): with
 * Y = S^(-1/2) |o> from the CSS projection of the overlap S onto the probes o (block-Lanczos
 * on S, x^(-1/2) in the Krylov subspace), S~^(-1/2) = Y <o| on S's pattern, and the sparse H'
 * extracted from S~^(-1/2) H Y <o| on H's pattern:
 *   H'~_IJ = [S~^(-1/2) (H Y_c)]_I diag(o_J),  c = colour(J),
 * where the left factor is the sparse S~^(-1/2) just obtained (symmetrised when
 * CSS_REF_SYMMETRIZE is set, as is H'~).  S and H share n_brow and b; their patterns may
 * differ.  Outputs: Sinv_val (S's pattern), Hp_val (H's pattern), *trHp = Tr H'. */
int css_ref_hprime(int32_t n_brow, int32_t b, int32_t nnzb_s, const int32_t* s_row_ptr, const int32_t* s_col_idx,
                   const double* s_val, int32_t nnzb_h, const int32_t* h_row_ptr, const int32_t* h_col_idx,
                   const double* h_val, const int32_t* colour, const int8_t* sign, int32_t n_colours, int32_t m,
                   int flags, double* Sinv_val, double* Hp_val, double* trHp) {
  if (n_brow < 1 || b < 1 || m < 1 || n_colours < 1 || !Sinv_val || !Hp_val) return REF_ERR_ARG;
  const int sym = flags & CSS_REF_SYMMETRIZE;
  double t1, t2, mu0;
  int32_t nbrk;
  int st = css_ref_density(n_brow, b, nnzb_s, s_row_ptr, s_col_idx, s_val, colour, sign, n_colours, 0.0, 0.0,
                           0.0, 0.0, 0, m, (flags & (CSS_REF_SYMMETRIZE | CSS_REF_REORTH_LOCAL)) | CSS_REF_INV_SQRT,
                           NULL, 0, Sinv_val, &t1, &t2, &mu0, &nbrk);
  if (st != REF_OK) return st;
  ref_h S = {n_brow, b, s_row_ptr, s_col_idx, s_val};
  const int64_t N = (int64_t)n_brow * b;
  const int32_t nmax = m * b;
  int64_t* cnt = (int64_t*)calloc((size_t)n_colours, sizeof(int64_t));
  int32_t* brow = (int32_t*)malloc(sizeof(int32_t) * (size_t)nnzb_h);
  double* Ht = (double*)calloc((size_t)nnzb_h * b * b, sizeof(double));
  if (!cnt || !brow || !Ht) return REF_ERR_NOMEM;
  for (int32_t J = 0; J < n_brow; ++J) cnt[colour[J]]++;
  for (int32_t I = 0; I < n_brow; ++I)
    for (int32_t p = h_row_ptr[I]; p < h_row_ptr[I + 1]; ++p) brow[p] = I;
  int status = REF_OK;
#pragma omp parallel for schedule(dynamic, 1) if (n_colours > 1)
  for (int32_t c = 0; c < n_colours; ++c) {
    if (cnt[c] == 0) continue;
    double* U = (double*)malloc(sizeof(double) * (size_t)nmax * nmax);
    double* lam = (double*)malloc(sizeof(double) * nmax);
    double* wg = (double*)malloc(sizeof(double) * nmax);
    double* Z = (double*)malloc(sizeof(double) * (size_t)nmax * b);
    double* fy = (double*)malloc(sizeof(double) * (size_t)nmax * b);
    double* Y = (double*)malloc(sizeof(double) * (size_t)N * b);
    double* W1 = (double*)malloc(sizeof(double) * (size_t)N * b);
    double* W2 = (double*)malloc(sizeof(double) * (size_t)N * b);
    int32_t n = 0, bk = 0;
    int sc = ref_colour_eigen(&S, colour, sign, c, m, flags & CSS_REF_REORTH_LOCAL, &n, lam, wg, U, &bk, cnt[c]);
    double sq = sqrt((double)cnt[c]);
    for (int32_t j = 0; j < n; ++j) {  /* Lambda^(-1/2) U^T E_1 B_0 */
      double g = lam[j] > 0.0 ? 1.0 / sqrt(lam[j]) : NAN;
      for (int32_t k = 0; k < b; ++k) fy[(size_t)j * b + k] = g * sq * U[(size_t)k * n + j];
    }
    for (int32_t i = 0; i < nmax; ++i)
      for (int32_t k = 0; k < b; ++k) {
        double sum = 0.0;
        if (i < n)
          for (int32_t j = 0; j < n; ++j) sum += U[(size_t)i * n + j] * fy[(size_t)j * b + k];
        Z[(size_t)i * b + k] = sum;
      }
    ref_lanczos_colour(&S, colour, sign, c, n / b, flags & CSS_REF_REORTH_LOCAL, NULL, Z, Y, NULL, NULL);  /* Y_c */
    ref_bsr_mul(n_brow, b, h_row_ptr, h_col_idx, h_val, Y, W1, b);          /* H Y_c */
    ref_bsr_mul(n_brow, b, s_row_ptr, s_col_idx, Sinv_val, W1, W2, b);      /* S~^(-1/2) H Y_c */
    for (int32_t p = 0; p < nnzb_h; ++p) {
      int32_t J = h_col_idx[p];
      if (colour[J] != c) continue;
      int32_t I = brow[p];
      for (int32_t a = 0; a < b; ++a)
        for (int32_t k = 0; k < b; ++k)
          Ht[(size_t)p * b * b + a * b + k] = W2[((size_t)I * b + a) * b + k] * sign[(size_t)J * b + k];
    }
    if (sc != REF_OK) {
#pragma omp critical
      status = sc;
    }
    free(U); free(lam); free(wg); free(Z); free(fy); free(Y); free(W1); free(W2);
  }
  double tr = 0.0;
  for (int32_t p = 0; p < nnzb_h; ++p) {
    int32_t I = brow[p], J = h_col_idx[p];
    int32_t q = -1;
    for (int32_t r = h_row_ptr[J]; r < h_row_ptr[J + 1]; ++r)
      if (h_col_idx[r] == I) { q = r; break; }
    for (int32_t a = 0; a < b; ++a)
      for (int32_t k = 0; k < b; ++k) {
        double x = Ht[(size_t)p * b * b + a * b + k];
        if (sym && q >= 0) x = 0.5 * (x + Ht[(size_t)q * b * b + k * b + a]);
        Hp_val[(size_t)p * b * b + a * b + k] = x;
        if (I == J && a == k) tr += x;
      }
  }
  if (trHp) *trHp = tr;
  free(cnt); free(brow); free(Ht);
  if (status != REF_OK) return status;
  return isfinite(tr) ? REF_OK : REF_ERR_NUMERIC;
}

/* y (N x w) = A^T x for a BSR matrix A (the transpose of ref_bsr_mul) */
static void ref_bsr_mul_t(int32_t n_brow, int32_t b, const int32_t* row_ptr, const int32_t* col_idx,
                          const double* val, const double* x, double* y, int32_t w) {
  memset(y, 0, sizeof(double) * (size_t)n_brow * b * w);
  for (int32_t I = 0; I < n_brow; ++I)
    for (int32_t p = row_ptr[I]; p < row_ptr[I + 1]; ++p) {
      int32_t J = col_idx[p];
      const double* a = val + (size_t)p * b * b;
      for (int32_t r = 0; r < b; ++r)
        for (int32_t c = 0; c < b; ++c) {
          double arc = a[r * b + c];  /* y[J, c] += A_IJ[r][c] x[I, r] */
          for (int32_t k = 0; k < w; ++k) y[((size_t)J * b + c) * w + k] += arc * x[((size_t)I * b + r) * w + k];
        }
    }
}

/* Density matrix of a NON-ORTHOGONAL basis (paper, Eq. 4-6 with S != I): the Krylov space of
 * H' is built from r~_c = S^(-1/2) r_c, and rho~ = S^(-1/2) Phi rho^K <Phi|r~><r| (the
 * displayed form of rho~ after Eq. 5, with rho^K of Eq. 6).  Per colour c of the probes r:
 *   r~_c = S~^(-1/2) R_c,  r~_c = Q_1 B_0 (QR),  block-Lanczos on H' from Q_1 -> T_c, Phi_c
 *   T_c = U Lambda U^T,  Y = U^T E_1 B_0,  Z_c = U f(Lambda) Y
 *   X_c = S~^(-1/2) Phi_c Z_c,  rho~_IJ = X_c[I] diag(s_J) for J of colour c (H's pattern)
 * Inputs are the sparse S~^(-1/2) (sinv_val on S's pattern) and H' (hp_val on H's pattern)
 * of css_ref_hprime, S itself and H (h_val, same pattern as H').  S's pattern must lie inside
 * H's.  Electron count (reading where the paper is silent): in a non-orthogonal basis it is
 * Tr(rho S); with u_c = S~^(-1/2)^T S R_c and V_c = Phi_c^T u_c, the weights
 *   kappa_cj = (U^T V_c)_j . Y_j
 * give sum_c sum_j f(lambda_cj) kappa_cj = sum_c Tr(R_c^T S X_c), which is exactly the
 * extracted Tr(rho~ S); mu is solved on that quadrature with the rule of css_ref_density.
 * Outputs: P_val (H's pattern, symmetrised with CSS_REF_SYMMETRIZE), Tr(rho~ S), Tr(rho~ H). */
int css_ref_density_nonorth(int32_t n_brow, int32_t b, int32_t nnzb_s, const int32_t* s_row_ptr,
                            const int32_t* s_col_idx, const double* s_val, const double* sinv_val, int32_t nnzb_h,
                            const int32_t* h_row_ptr, const int32_t* h_col_idx, const double* h_val,
                            const double* hp_val, const int32_t* colour, const int8_t* sign, int32_t n_colours,
                            double mu, double kT, double n_elec, double ne_tol, int solve_mu, int32_t m, int flags,
                            double* P_val, double* trPS, double* trPH, double* mu_out, int32_t* n_breakdown) {
  if (n_brow < 1 || b < 1 || m < 1 || n_colours < 1 || nnzb_h < n_brow || !P_val || kT < 0.0) return REF_ERR_ARG;
  if (!(ne_tol > 0.0)) ne_tol = 1e-4 * fmax(1.0, 0.5 * n_elec);
  const int64_t N = (int64_t)n_brow * b;
  const int32_t nmax = m * b, bb = b * b;
  ref_h Hp = {n_brow, b, h_row_ptr, h_col_idx, hp_val};
  /* position of each S block in H's pattern (S's pattern must be inside H's) */
  int32_t* s_in_h = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnzb_s > 0 ? nnzb_s : 1));
  int64_t* cnt = (int64_t*)calloc((size_t)n_colours, sizeof(int64_t));
  double* lam = (double*)calloc((size_t)n_colours * nmax, sizeof(double));
  double* kap = (double*)calloc((size_t)n_colours * nmax, sizeof(double));
  double* Us = (double*)calloc((size_t)n_colours * nmax * nmax, sizeof(double));
  double* Ys = (double*)calloc((size_t)n_colours * nmax * b, sizeof(double));
  int32_t* nj = (int32_t*)calloc((size_t)n_colours, sizeof(int32_t));
  int32_t* brk = (int32_t*)calloc((size_t)n_colours, sizeof(int32_t));
  double** Phi = (double**)calloc((size_t)n_colours, sizeof(double*));
  if (!s_in_h || !cnt || !lam || !kap || !Us || !Ys || !nj || !brk || !Phi) return REF_ERR_NOMEM;
  int status = REF_OK;
  for (int32_t I = 0; I < n_brow && status == REF_OK; ++I)
    for (int32_t p = s_row_ptr[I]; p < s_row_ptr[I + 1]; ++p) {
      s_in_h[p] = -1;
      for (int32_t q = h_row_ptr[I]; q < h_row_ptr[I + 1]; ++q)
        if (h_col_idx[q] == s_col_idx[p]) { s_in_h[p] = q; break; }
      if (s_in_h[p] < 0) status = REF_ERR_ARG;
    }
  for (int32_t J = 0; J < n_brow && status == REF_OK; ++J) {
    if (colour[J] < 0 || colour[J] >= n_colours) status = REF_ERR_ARG;
    else cnt[colour[J]]++;
  }
  if (status != REF_OK) return status;
  /* pass 1 per colour: start block, Lanczos on H' (basis kept), eigen-data and kappa */
#pragma omp parallel for schedule(dynamic, 1) if (n_colours > 1)
  for (int32_t c = 0; c < n_colours; ++c) {
    if (cnt[c] == 0) continue;
    double* R = (double*)calloc((size_t)N * b, sizeof(double));
    double* rt = (double*)malloc(sizeof(double) * (size_t)N * b);
    double* Q1 = (double*)malloc(sizeof(double) * (size_t)N * b);
    double* SR = (double*)malloc(sizeof(double) * (size_t)N * b);
    double* u = (double*)malloc(sizeof(double) * (size_t)N * b);
    double* B0 = (double*)malloc(sizeof(double) * bb);
    double* v = (double*)malloc(sizeof(double) * (size_t)N);
    double* T = (double*)malloc(sizeof(double) * (size_t)nmax * nmax);
    double* Q = (double*)malloc(sizeof(double) * (size_t)N * nmax);
    double* V = (double*)malloc(sizeof(double) * (size_t)nmax * b);
    double* UV = (double*)malloc(sizeof(double) * (size_t)nmax * b);
    for (int32_t J = 0; J < n_brow; ++J)  /* R_c: column k = s_Jk on orbital k of each J in c */
      if (colour[J] == c)
        for (int32_t k = 0; k < b; ++k) R[((size_t)J * b + k) * b + k] = sign[(size_t)J * b + k];
    ref_bsr_mul(n_brow, b, s_row_ptr, s_col_idx, sinv_val, R, rt, b);  /* r~_c = S~^(-1/2) R_c */
    ref_bsr_mul(n_brow, b, s_row_ptr, s_col_idx, s_val, R, SR, b);     /* S R_c */
    ref_bsr_mul_t(n_brow, b, s_row_ptr, s_col_idx, sinv_val, SR, u, b); /* u_c = S~^(-1/2)^T S R_c */
    ref_qr(N, b, rt, Q1, B0, v);                                        /* r~_c = Q_1 B_0 */
    int32_t blocks = ref_lanczos_colour(&Hp, colour, sign, c, m, flags & CSS_REF_REORTH_LOCAL, T, NULL, NULL, Q, Q1);
    if (blocks < m) brk[c] = 1;
    const int32_t n = blocks * b;
    double* U = Us + (size_t)c * nmax * nmax;
    double* Y = Ys + (size_t)c * nmax * b;
    for (int32_t i = 0; i < n; ++i)
      for (int32_t j = 0; j < n; ++j) U[(size_t)i * n + j] = T[(size_t)i * nmax + j];
    int st = css_ref_eigh(n, U, lam + (size_t)c * nmax);
    for (int32_t j = 0; j < n; ++j)  /* Y = U^T E_1 B_0 */
      for (int32_t k = 0; k < b; ++k) {
        double sum = 0.0;
        for (int32_t l = 0; l <= k; ++l) sum += U[(size_t)l * n + j] * B0[l * b + k];
        Y[(size_t)j * b + k] = sum;
      }
    for (int32_t i = 0; i < n; ++i)  /* V = Phi^T u */
      for (int32_t k = 0; k < b; ++k) {
        double sum = 0.0;
        for (int64_t r = 0; r < N; ++r) sum += Q[(size_t)r * nmax + i] * u[(size_t)r * b + k];
        V[(size_t)i * b + k] = sum;
      }
    for (int32_t j = 0; j < n; ++j) {  /* kappa_j = (U^T V)_j . Y_j */
      double kj = 0.0;
      for (int32_t k = 0; k < b; ++k) {
        double sum = 0.0;
        for (int32_t i = 0; i < n; ++i) sum += U[(size_t)i * n + j] * V[(size_t)i * b + k];
        UV[(size_t)j * b + k] = sum;
        kj += sum * Y[(size_t)j * b + k];
      }
      kap[(size_t)c * nmax + j] = kj;
    }
    nj[c] = n;
    Phi[c] = Q;
    if (st != REF_OK) {
#pragma omp critical
      status = st;
    }
    free(R); free(rt); free(Q1); free(SR); free(u); free(B0); free(v); free(T); free(V); free(UV);
  }
  if (status == REF_OK && solve_mu) mu = ref_solve_mu(n_colours, nj, nmax, lam, kap, kT, n_elec, ne_tol);
  if (mu_out) *mu_out = mu;
  /* pass 2 per colour: Z_c, X_c = S~^(-1/2) Phi_c Z_c, extraction on H's pattern */
  int32_t* brow = (int32_t*)malloc(sizeof(int32_t) * (size_t)nnzb_h);
  double* Pt = (double*)calloc((size_t)nnzb_h * bb, sizeof(double));
  if (!brow || !Pt) return REF_ERR_NOMEM;
  for (int32_t I = 0; I < n_brow; ++I)
    for (int32_t p = h_row_ptr[I]; p < h_row_ptr[I + 1]; ++p) brow[p] = I;
#pragma omp parallel for schedule(dynamic, 1) if (n_colours > 1)
  for (int32_t c = 0; c < n_colours; ++c) {
    if (cnt[c] == 0 || status != REF_OK) continue;
    const int32_t n = nj[c];
    const double* U = Us + (size_t)c * nmax * nmax;
    const double* Y = Ys + (size_t)c * nmax * b;
    double* fy = (double*)malloc(sizeof(double) * (size_t)nmax * b);
    double* Z = (double*)malloc(sizeof(double) * (size_t)nmax * b);
    double* Xt = (double*)malloc(sizeof(double) * (size_t)N * b);
    double* X = (double*)malloc(sizeof(double) * (size_t)N * b);
    for (int32_t j = 0; j < n; ++j) {
      double fj = ref_fermi(lam[(size_t)c * nmax + j], mu, kT);
      for (int32_t k = 0; k < b; ++k) fy[(size_t)j * b + k] = fj * Y[(size_t)j * b + k];
    }
    for (int32_t i = 0; i < n; ++i)  /* Z = U f(Lambda) Y */
      for (int32_t k = 0; k < b; ++k) {
        double sum = 0.0;
        for (int32_t j = 0; j < n; ++j) sum += U[(size_t)i * n + j] * fy[(size_t)j * b + k];
        Z[(size_t)i * b + k] = sum;
      }
    for (int64_t r = 0; r < N; ++r)  /* X~ = Phi Z */
      for (int32_t k = 0; k < b; ++k) {
        double sum = 0.0;
        for (int32_t i = 0; i < n; ++i) sum += Phi[c][(size_t)r * nmax + i] * Z[(size_t)i * b + k];
        Xt[(size_t)r * b + k] = sum;
      }
    ref_bsr_mul(n_brow, b, s_row_ptr, s_col_idx, sinv_val, Xt, X, b);  /* X = S~^(-1/2) X~ */
    for (int32_t p = 0; p < nnzb_h; ++p) {
      int32_t J = h_col_idx[p];
      if (colour[J] != c) continue;
      int32_t I = brow[p];
      for (int32_t a = 0; a < b; ++a)
        for (int32_t k = 0; k < b; ++k)
          Pt[(size_t)p * bb + a * b + k] = X[((size_t)I * b + a) * b + k] * sign[(size_t)J * b + k];
    }
    free(fy); free(Z); free(Xt); free(X);
  }
  /* symmetrise on H's pattern and take Tr(rho~ H) and Tr(rho~ S) */
  double tph = 0.0, tps = 0.0;
  for (int32_t p = 0; p < nnzb_h; ++p) {
    int32_t I = brow[p], J = h_col_idx[p];
    int32_t q = -1;
    for (int32_t r = h_row_ptr[J]; r < h_row_ptr[J + 1]; ++r)
      if (h_col_idx[r] == I) { q = r; break; }
    for (int32_t a = 0; a < b; ++a)
      for (int32_t k = 0; k < b; ++k) {
        double x = Pt[(size_t)p * bb + a * b + k];
        if ((flags & CSS_REF_SYMMETRIZE) && q >= 0) x = 0.5 * (x + Pt[(size_t)q * bb + k * b + a]);
        P_val[(size_t)p * bb + a * b + k] = x;
        tph += x * h_val[(size_t)p * bb + a * b + k];
      }
  }
  for (int32_t p = 0; p < nnzb_s; ++p)
    for (int32_t e = 0; e < bb; ++e) tps += P_val[(size_t)s_in_h[p] * bb + e] * s_val[(size_t)p * bb + e];
  if (trPS) *trPS = tps;
  if (trPH) *trPH = tph;
  int32_t nb = 0;
  for (int32_t c = 0; c < n_colours; ++c) nb += brk[c];
  if (n_breakdown) *n_breakdown = nb;
  for (int32_t c = 0; c < n_colours; ++c) free(Phi[c]);
  free(Phi); free(s_in_h); free(cnt); free(lam); free(kap); free(Us); free(Ys); free(nj); free(brk);
  free(brow); free(Pt);
  if (status != REF_OK) return status;
  return (isfinite(tps) && isfinite(tph)) ? REF_OK : REF_ERR_NUMERIC;
}

/* Ritz data of all colours, or of the colours with want[c] != 0 when want is given (test hook):
 * lam/wgt are n_colours x (m b), n_per receives the size of each colour's projected matrix (0
 * for colours left out). */
int css_ref_ritz(int32_t n_brow, int32_t b, const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                 const int32_t* colour, const int8_t* sign, int32_t n_colours, int32_t m, int flags,
                 const int8_t* want, double* lam, double* wgt, int32_t* n_per) {
  ref_h H = {n_brow, b, row_ptr, col_idx, val};
  const int32_t nmax = m * b;
  int64_t* cnt = (int64_t*)calloc((size_t)n_colours, sizeof(int64_t));
  for (int32_t J = 0; J < n_brow; ++J) cnt[colour[J]]++;
  int status = REF_OK;
  for (int32_t c = 0; c < n_colours; ++c) {
    n_per[c] = 0;
    if (cnt[c] == 0 || (want && !want[c])) continue;
    double* U = (double*)malloc(sizeof(double) * (size_t)nmax * nmax);
    int32_t bk = 0;
    int st = ref_colour_eigen(&H, colour, sign, c, m, flags, &n_per[c], lam + (size_t)c * nmax,
                              wgt + (size_t)c * nmax, U, &bk, cnt[c]);
    if (st != REF_OK) status = st;
    free(U);
  }
  free(cnt);
  return status;
}

int css_ref_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
