// Block-Lanczos on CSS probe blocks, all colours of a batch at once (paper: paragraph after
// Eq. 4, Golub-Underwood block-Lanczos; SpMM-only cost noted after Eq. 10).
//
// Krylov blocks of a batch of colours live side by side as the columns of one N x w matrix
// (row-major, row stride ws, w = b * colours): colour c of the batch owns columns
// [c b, c b + b).  One step j is
//     W = H Q_j                        (k_spmm: every H block multiplies all w columns)
//     W -= Q_{j-1} B_{j-1}^T ; A_j = sym(Q_j^T W) ; W -= Q_j A_j      (k_threeterm, k_sub)
//     W = Q_{j+1} B_j by CholQR2: R1 = chol(W^T W), W R1^-1, R2 = chol(.), B_j = R2 R1
// Small per-colour matrices (A_j, B_j, Grams, Cholesky factors) are FP64; the per-row-chunk
// partial products are combined in FP64 in a fixed order, so every run is bitwise
// reproducible (a second pass regenerates the same basis).
#include "css_lanczos.cuh"

namespace {

// ------------------------------------------------------------------------ H * V
// One CTA per (block row I, tile of 128*TC columns); blockIdx.x runs over I so the CTAs in
// flight share one column tile and the V rows they gather stay in L2.  The row's H blocks are
// staged in shared memory (zero-padded to BM x BM), every thread keeps the b x TC outputs of
// its columns in registers and streams the b rows of V of each neighbour J.
template <typename T, int BM, int TC>
__global__ void __launch_bounds__(128) k_spmm(int32_t b, const int32_t* __restrict__ row_ptr,
                                              const int32_t* __restrict__ col_idx, const T* __restrict__ Hv,
                                              const T* __restrict__ V, T* __restrict__ W, int32_t ws, int32_t w,
                                              int32_t chunk, const T* __restrict__ Hlo) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Hs = reinterpret_cast<T*>(smem_raw);
  const int32_t I = blockIdx.x;
  const int32_t col0 = blockIdx.y * (128 * TC) + threadIdx.x;
  const int32_t p0 = row_ptr[I], p1 = row_ptr[I + 1];
  const int32_t bb = b * b;
  T acc[BM][TC];
#pragma unroll
  for (int a = 0; a < BM; ++a)
#pragma unroll
    for (int u = 0; u < TC; ++u) acc[a][u] = T(0);
  for (int32_t pc = p0; pc < p1; pc += chunk) {
    const int32_t pe = min(p1, pc + chunk);
    __syncthreads();
    for (int32_t e = threadIdx.x; e < (pe - pc) * BM * BM; e += blockDim.x) {
      int32_t blk = e / (BM * BM), r = e % (BM * BM), a = r / BM, k = r % BM;
      Hs[e] = (a < b && k < b) ? Hv[(size_t)(pc + blk) * bb + a * b + k] : T(0);
    }
    __syncthreads();
    for (int32_t p = pc; p < pe; ++p) {
      const int32_t J = col_idx[p];
      const T* Hb = Hs + (size_t)(p - pc) * BM * BM;
      const T* Vr = V + (size_t)J * b * ws;
      T v[BM][TC];
#pragma unroll
      for (int k = 0; k < BM; ++k)
#pragma unroll
        for (int u = 0; u < TC; ++u) {
          const int32_t col = col0 + 128 * u;
          v[k][u] = (k < b && col < w) ? __ldg(Vr + (size_t)k * ws + col) : T(0);
        }
#pragma unroll
      for (int a = 0; a < BM; ++a)
#pragma unroll
        for (int k = 0; k < BM; ++k) {
          const T h = Hb[a * BM + k];
#pragma unroll
          for (int u = 0; u < TC; ++u) acc[a][u] = fma(h, v[k][u], acc[a][u]);
        }
    }
  }
  if (Hlo) {
    // low part of the diagonal block (FP32 mode: H_II = hi + lo, both FP32), W_I += lo V_I
    __syncthreads();
    for (int32_t e = threadIdx.x; e < BM * BM; e += blockDim.x) {
      int32_t a = e / BM, k = e % BM;
      Hs[e] = (a < b && k < b) ? Hlo[(size_t)I * bb + a * b + k] : T(0);
    }
    __syncthreads();
    const T* Vr = V + (size_t)I * b * ws;
    T v[BM][TC];
#pragma unroll
    for (int k = 0; k < BM; ++k)
#pragma unroll
      for (int u = 0; u < TC; ++u) {
        const int32_t col = col0 + 128 * u;
        v[k][u] = (k < b && col < w) ? __ldg(Vr + (size_t)k * ws + col) : T(0);
      }
#pragma unroll
    for (int a = 0; a < BM; ++a)
#pragma unroll
      for (int k = 0; k < BM; ++k) {
        const T h = Hs[a * BM + k];
#pragma unroll
        for (int u = 0; u < TC; ++u) acc[a][u] = fma(h, v[k][u], acc[a][u]);
      }
  }
  T* Wr = W + (size_t)I * b * ws;
#pragma unroll
  for (int a = 0; a < BM; ++a)
#pragma unroll
    for (int u = 0; u < TC; ++u) {
      const int32_t col = col0 + 128 * u;
      if (a < b && col < w) Wr[(size_t)a * ws + col] = acc[a][u];
    }
}

// --------------------------------------------------------------- row-chunk kernels
// CTA = (chunk of RCH = RC * TPC rows, one colour of the batch).  The chunk is walked in
// tiles of RC rows staged in shared memory as [RC][b]; per-tile Gram products are summed in
// the vector precision and added to FP64 accumulators held in registers (thread t owns the
// entries t, t + 256, ... of the b x b block), which are written once per CTA.
constexpr int RC = 128;
constexpr int TPC = 8;
constexpr int RCH = RC * TPC;
constexpr int RT = 256;
constexpr int GACC = (CSS_MAX_B * CSS_MAX_B + RT - 1) / RT;

template <typename T>
__device__ __forceinline__ void load_tile(T* dst, const T* src, int64_t r0, int32_t nr, int32_t b, int32_t ws,
                                          int32_t c0) {
  for (int32_t e = threadIdx.x; e < nr * b; e += blockDim.x) {
    int32_t r = e / b, k = e % b;
    dst[e] = src[(size_t)(r0 + r) * ws + c0 + k];
  }
}

template <typename T>
__device__ __forceinline__ void store_tile(T* dst, const T* src, int64_t r0, int32_t nr, int32_t b, int32_t ws,
                                           int32_t c0) {
  for (int32_t e = threadIdx.x; e < nr * b; e += blockDim.x) {
    int32_t r = e / b, k = e % b;
    dst[(size_t)(r0 + r) * ws + c0 + k] = src[e];
  }
}

// acc[i] += sum_r X[r][k] Y[r][l] for entry e = threadIdx.x + RT i = k b + l
template <typename T>
__device__ __forceinline__ void tile_gram(const T* X, const T* Y, int32_t nr, int32_t b, double* acc) {
#pragma unroll
  for (int i = 0; i < GACC; ++i) {
    const int32_t e = threadIdx.x + RT * i;
    if (e < b * b) {
      const int32_t k = e / b, l = e % b;
      T s = T(0);
      for (int32_t r = 0; r < nr; ++r) s = fma(X[r * b + k], Y[r * b + l], s);
      acc[i] += (double)s;
    }
  }
}

__device__ __forceinline__ void store_acc(const double* acc, int32_t b, double* out) {
#pragma unroll
  for (int i = 0; i < GACC; ++i) {
    const int32_t e = threadIdx.x + RT * i;
    if (e < b * b) out[e] = acc[i];
  }
}

#define ROW_LOOP(N)                                                                        \
  for (int64_t r0 = (int64_t)blockIdx.x * RCH, r_end = min((int64_t)(N), r0 + RCH); r0 < r_end; \
       r0 += RC)

// W -= Qp Bp^T (skipped at the first step), partial A = Q^T W, partial ||W_in||^2
template <typename T>
__global__ void __launch_bounds__(RT) k_threeterm(int64_t N, int32_t b, int32_t ws, int32_t cb0,
                                                  const T* __restrict__ Qp, const T* __restrict__ Q,
                                                  T* __restrict__ W, const double* __restrict__ Bprev, int first,
                                                  double* __restrict__ partA, double* __restrict__ partH) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* red = reinterpret_cast<double*>(smem_raw);  // RT/32 warp sums
  T* sQ = reinterpret_cast<T*>(smem_raw + 16 * sizeof(double));
  T* sW = sQ + RC * b;
  T* sP = sW + RC * b;
  T* sB = sP + RC * b;
  const int32_t lc = blockIdx.y, c0 = lc * b;
  double acc[GACC] = {};
  double hs = 0.0;
  if (!first)
    for (int32_t e = threadIdx.x; e < b * b; e += blockDim.x) sB[e] = (T)Bprev[(size_t)(cb0 + lc) * b * b + e];
  ROW_LOOP(N) {
    const int32_t nr = (int32_t)min((int64_t)RC, N - r0);
    __syncthreads();
    load_tile(sQ, Q, r0, nr, b, ws, c0);
    load_tile(sW, W, r0, nr, b, ws, c0);
    if (!first) load_tile(sP, Qp, r0, nr, b, ws, c0);
    __syncthreads();
    for (int32_t e = threadIdx.x; e < nr * b; e += blockDim.x) hs += (double)sW[e] * (double)sW[e];
    if (!first) {
      for (int32_t e = threadIdx.x; e < nr * b; e += blockDim.x) {
        int32_t r = e / b, k = e % b;
        T s = T(0);
        for (int32_t l = 0; l < b; ++l) s = fma(sP[r * b + l], sB[k * b + l], s);
        sW[e] -= s;
      }
      __syncthreads();
      store_tile(W, sW, r0, nr, b, ws, c0);
    }
    tile_gram(sQ, sW, nr, b, acc);
  }
  const size_t o = (size_t)blockIdx.x * gridDim.y + lc;
  store_acc(acc, b, partA + o * b * b);
  for (int of = 16; of > 0; of >>= 1) hs += __shfl_xor_sync(0xffffffffu, hs, of);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = hs;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < RT / 32; ++i) t += red[i];
    partH[o] = t;
  }
}

// W -= Q M (M = A_j symmetrised, or a reorthogonalisation coefficient block), optional
// second subtraction W -= Qp M2, then partial Gram W^T W when GRAM
template <typename T, bool GRAM>
__global__ void __launch_bounds__(RT) k_sub(int64_t N, int32_t b, int32_t ws, const T* __restrict__ Q,
                                            const T* __restrict__ Qp, T* __restrict__ W,
                                            const double* __restrict__ M, const double* __restrict__ M2,
                                            double* __restrict__ partG) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sQ = reinterpret_cast<T*>(smem_raw);
  T* sW = sQ + RC * b;
  T* sP = sW + RC * b;
  T* sM = sP + RC * b;
  T* sM2 = sM + b * b;
  const int32_t lc = blockIdx.y, c0 = lc * b;
  double acc[GACC] = {};
  for (int32_t e = threadIdx.x; e < b * b; e += blockDim.x) {
    sM[e] = (T)M[(size_t)lc * b * b + e];
    if (M2) sM2[e] = (T)M2[(size_t)lc * b * b + e];
  }
  ROW_LOOP(N) {
    const int32_t nr = (int32_t)min((int64_t)RC, N - r0);
    __syncthreads();
    load_tile(sQ, Q, r0, nr, b, ws, c0);
    load_tile(sW, W, r0, nr, b, ws, c0);
    if (M2) load_tile(sP, Qp, r0, nr, b, ws, c0);
    __syncthreads();
    for (int32_t e = threadIdx.x; e < nr * b; e += blockDim.x) {
      int32_t r = e / b, k = e % b;
      T s = T(0);
      for (int32_t l = 0; l < b; ++l) s = fma(sQ[r * b + l], sM[l * b + k], s);
      if (M2)
        for (int32_t l = 0; l < b; ++l) s = fma(sP[r * b + l], sM2[l * b + k], s);
      sW[e] -= s;
    }
    __syncthreads();
    store_tile(W, sW, r0, nr, b, ws, c0);
    if (GRAM) tile_gram(sW, sW, nr, b, acc);
  }
  if (GRAM) store_acc(acc, b, partG + ((size_t)blockIdx.x * gridDim.y + lc) * b * b);
}

// partial X^T W for X = Q and X = Qp (local reorthogonalisation coefficients)
template <typename T>
__global__ void __launch_bounds__(RT) k_proj2(int64_t N, int32_t b, int32_t ws, const T* __restrict__ Q,
                                              const T* __restrict__ Qp, const T* __restrict__ W,
                                              double* __restrict__ part1, double* __restrict__ part2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sQ = reinterpret_cast<T*>(smem_raw);
  T* sW = sQ + RC * b;
  T* sP = sW + RC * b;
  const int32_t lc = blockIdx.y, c0 = lc * b;
  double a1[GACC] = {}, a2[GACC] = {};
  ROW_LOOP(N) {
    const int32_t nr = (int32_t)min((int64_t)RC, N - r0);
    __syncthreads();
    load_tile(sQ, Q, r0, nr, b, ws, c0);
    load_tile(sW, W, r0, nr, b, ws, c0);
    load_tile(sP, Qp, r0, nr, b, ws, c0);
    __syncthreads();
    tile_gram(sQ, sW, nr, b, a1);
    tile_gram(sP, sW, nr, b, a2);
  }
  const size_t o = ((size_t)blockIdx.x * gridDim.y + lc) * b * b;
  store_acc(a1, b, part1 + o);
  store_acc(a2, b, part2 + o);
}

// W <- W R^-1 (upper triangular, FP64 -> T); partial Gram of the result when GRAM; when OUT
// is non-null the result goes there instead of back into W
template <typename T, bool GRAM>
__global__ void __launch_bounds__(RT) k_apply(int64_t N, int32_t b, int32_t ws, T* __restrict__ W,
                                              T* __restrict__ OUT, const double* __restrict__ Rinv,
                                              double* __restrict__ partG) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sW = reinterpret_cast<T*>(smem_raw);
  T* sO = sW + RC * b;
  T* sR = sO + RC * b;
  const int32_t lc = blockIdx.y, c0 = lc * b;
  double acc[GACC] = {};
  for (int32_t e = threadIdx.x; e < b * b; e += blockDim.x) sR[e] = (T)Rinv[(size_t)lc * b * b + e];
  ROW_LOOP(N) {
    const int32_t nr = (int32_t)min((int64_t)RC, N - r0);
    __syncthreads();
    load_tile(sW, W, r0, nr, b, ws, c0);
    __syncthreads();
    for (int32_t e = threadIdx.x; e < nr * b; e += blockDim.x) {
      int32_t r = e / b, l = e % b;
      T s = T(0);
      for (int32_t k = 0; k <= l; ++k) s = fma(sW[r * b + k], sR[k * b + l], s);
      sO[e] = s;
    }
    __syncthreads();
    store_tile(OUT ? OUT : W, sO, r0, nr, b, ws, c0);
    if (GRAM) tile_gram(sO, sO, nr, b, acc);
  }
  if (GRAM) store_acc(acc, b, partG + ((size_t)blockIdx.x * gridDim.y + lc) * b * b);
}

// out[lc][e] = sum over chunks of part[ch][lc][e], fixed order, FP64
__global__ void k_reduce(int32_t nch, int32_t ncb, int32_t E, const double* __restrict__ part,
                         double* __restrict__ out) {
  int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncb * E) return;
  double s = 0.0;
  for (int32_t ch = 0; ch < nch; ++ch) s += part[(size_t)ch * ncb * E + t];
  out[t] = s;
}

// Store A_j = (A + A^T)/2 into the projected matrix and keep the symmetrised copy
__global__ void k_store_A(int32_t ncb, int32_t b, int32_t cb0, int32_t m, int32_t j, double* __restrict__ A,
                          double* __restrict__ Ablk) {
  int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncb * b * b) return;
  int32_t lc = t / (b * b), e = t % (b * b), k = e / b, l = e % b;
  const double* a = A + (size_t)lc * b * b;
  double v = 0.5 * (a[k * b + l] + a[l * b + k]);
  Ablk[(((size_t)(cb0 + lc)) * m + j) * b * b + e] = v;
  // the symmetrised copy goes to a second slot, so no thread reads a value changed here
  A[(size_t)ncb * b * b + t] = v;
}

// Cholesky factor and inverse of one colour's Gram matrix, one warp per colour (lane l owns
// column l).  Three uses make shifted CholeskyQR3 (Fukaya, Kannan, Nakatsukasa, Yamamoto &
// Yanagisawa, SIAM J. Sci. Comput. 2020), which keeps the new block orthonormal even when it
// is nearly rank deficient (converged Ritz directions):
//   MODE 0: R0 = chol(G + s I), s = shift_rel * trace(G)                 (regularised pass)
//   MODE 1: R1 = chol(G); stores R10 = R1 R0 in Rprod
//   MODE 2: R2 = chol(G); B_j = R2 R10 stored in the projected matrix; breakdown when
//           min_k B_kk <= tau ||H Q_j||_F (same rule as a Householder QR's R_kk)
// A colour already finished, or a failed factorisation, gives R = I and R^-1 = 0, so the
// colour's next block is zero.
template <int MODE>
__global__ void k_chol(int32_t ncb, int32_t b, int32_t cb0, int32_t m, int32_t j, const double* __restrict__ G,
                       const double* __restrict__ hq2, double tau, double shift_rel, double* __restrict__ R,
                       double* __restrict__ Rinv, double* __restrict__ Rprod, double* __restrict__ Bblk,
                       int32_t* __restrict__ done, int32_t* __restrict__ nblk) {
  __shared__ double sR[4][CSS_MAX_B][CSS_MAX_B + 1];
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t lc = blockIdx.x * 4 + warp;
  if (lc >= ncb) return;
  const int32_t c = cb0 + lc;
  double (*r)[CSS_MAX_B + 1] = sR[warp];
  const double* g = G + (size_t)lc * b * b;
  double* ro = R + (size_t)lc * b * b;
  double* ri = Rinv + (size_t)lc * b * b;
  double* rp = Rprod + (size_t)lc * b * b;
  const bool was_done = done[c] != 0;
  bool broken = was_done;
  for (int32_t i = 0; i < b; ++i)
    if (lane < b) r[i][lane] = 0.0;
  __syncwarp();
  double shift = 0.0;
  if (MODE == 0) {
    double t = (lane < b) ? g[lane * b + lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    shift = shift_rel * t;
  }
  if (!broken) {
    for (int32_t k = 0; k < b && !broken; ++k) {
      double sv = 0.0;
      if (lane < b && lane >= k) {
        sv = g[k * b + lane] + ((lane == k) ? shift : 0.0);
        for (int32_t i = 0; i < k; ++i) sv -= r[i][k] * r[i][lane];
      }
      const double piv = __shfl_sync(0xffffffffu, sv, k);
      if (!(piv > 0.0)) {
        broken = true;
        break;
      }
      const double inv = 1.0 / sqrt(piv);
      if (lane < b && lane >= k) r[k][lane] = sv * inv;
      __syncwarp();
    }
  }
  __syncwarp();
  // the new sub-diagonal block and the breakdown test
  if (MODE == 2 && !broken && lane < b) {
    for (int32_t i = 0; i < b; ++i) {
      double sv = 0.0;
      for (int32_t k2 = i; k2 <= lane; ++k2) sv += r[i][k2] * rp[k2 * b + lane];
      Bblk[(((size_t)c) * m + j) * b * b + i * b + lane] = (i <= lane) ? sv : 0.0;
    }
  }
  if (MODE == 2 && !broken) {
    double dk = 1e300;
    if (lane < b) {
      double sv = 0.0;
      for (int32_t k2 = lane; k2 < b; ++k2) sv += (k2 == lane ? r[lane][lane] : 0.0) * rp[k2 * b + lane];
      dk = sv;  // (R2 R10)_kk = R2_kk R10_kk for upper-triangular factors
    }
    for (int o = 16; o > 0; o >>= 1) dk = fmin(dk, __shfl_xor_sync(0xffffffffu, dk, o));
    if (!(dk > tau * sqrt(hq2[lc]))) broken = true;
  }
  if (broken) {
    if (lane < b)
      for (int32_t i = 0; i < b; ++i) {
        ro[i * b + lane] = (i == lane) ? 1.0 : 0.0;
        ri[i * b + lane] = 0.0;
        if (MODE == 1) rp[i * b + lane] = (i == lane) ? 1.0 : 0.0;
        if (MODE == 2) Bblk[(((size_t)c) * m + j) * b * b + i * b + lane] = 0.0;
      }
    if (!was_done && lane == 0) {
      done[c] = 1;
      nblk[c] = j + 1;
    }
    return;
  }
  // inverse of the upper-triangular factor: lane l solves R x = e_l
  if (lane < b) {
    double x[CSS_MAX_B];
    for (int32_t i = b - 1; i >= 0; --i) {
      double sv = (i == lane) ? 1.0 : 0.0;
      for (int32_t k2 = i + 1; k2 <= lane; ++k2) sv -= r[i][k2] * x[k2];
      x[i] = (i <= lane) ? sv / r[i][i] : 0.0;
    }
    for (int32_t i = 0; i < b; ++i) {
      ri[i * b + lane] = (i <= lane) ? x[i] : 0.0;
      ro[i * b + lane] = r[i][lane];
    }
  }
  __syncwarp();
  if (MODE == 1 && lane < b) {
    // R10 = R1 R0 (R0 is the factor of the previous pass, passed in Rprod's slot on entry)
    double col[CSS_MAX_B];
    for (int32_t i = 0; i < b; ++i) {
      double sv = 0.0;
      for (int32_t k2 = i; k2 <= lane; ++k2) sv += r[i][k2] * rp[k2 * b + lane];
      col[i] = (i <= lane) ? sv : 0.0;
    }
    __syncwarp();
    for (int32_t i = 0; i < b; ++i) rp[i * b + lane] = col[i];
  }
}

// Q_1 = R_c / sqrt|c| for the colours of the batch (the rest of Q is zeroed by the caller)
template <typename T>
__global__ void k_init_q1(int32_t n_brow, int32_t b, int32_t ws, int32_t cb0, int32_t ncb,
                          const int32_t* __restrict__ colour, const int8_t* __restrict__ sign,
                          const double* __restrict__ inv_sqrt_cnt, T* __restrict__ Q) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n_brow * b) return;
  int32_t J = (int32_t)(t / b), k = (int32_t)(t % b);
  int32_t c = colour[J] - cb0;
  if (c < 0 || c >= ncb) return;
  Q[(size_t)t * ws + (size_t)c * b + k] = (T)(sign[t] * inv_sqrt_cnt[cb0 + c]);
}

// Sampled rows of Q_j: Qs[p][j][a][k] = Q_j[(I_p, a), c_p block, k] for the batch's pairs
template <typename T>
__global__ void k_scatter(int64_t p_begin, int64_t p_end, int32_t b, int32_t ws, int32_t cb0, int32_t m, int32_t j,
                          const int32_t* __restrict__ pair_I, const int32_t* __restrict__ pair_c,
                          const T* __restrict__ Q, T* __restrict__ Qs) {
  const int32_t bb = b * b;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t p = p_begin + t / bb;
  if (p >= p_end) return;
  int32_t e = (int32_t)(t % bb), a = e / b, k = e % b;
  int32_t I = pair_I[p], c = pair_c[p] - cb0;
  Qs[((size_t)p * m + j) * bb + e] = Q[((size_t)I * b + a) * ws + (size_t)c * b + k];
}

// Second pass: X[p][a][kk] += sum_l Q_j[(I_p, a), c_p block, l] Z_c[j b + l][kk] (FP64)
template <typename T>
__global__ void k_accum_x(int64_t p_begin, int64_t p_end, int32_t b, int32_t ws, int32_t cb0, int32_t ldz,
                          int32_t j, const int32_t* __restrict__ pair_I, const int32_t* __restrict__ pair_c,
                          const int32_t* __restrict__ nblk, const T* __restrict__ Q, const double* __restrict__ Z,
                          double* __restrict__ X) {
  const int32_t bb = b * b;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t p = p_begin + t / bb;
  if (p >= p_end) return;
  int32_t e = (int32_t)(t % bb), a = e / b, kk = e % b;
  int32_t I = pair_I[p], cg = pair_c[p], c = cg - cb0;
  if (j >= nblk[cg]) return;
  const T* q = Q + ((size_t)I * b + a) * ws + (size_t)c * b;
  const double* z = Z + ((size_t)cg * ldz + (size_t)j * b) * b + kk;
  double s = 0.0;
  for (int32_t l = 0; l < b; ++l) s = fma((double)q[l], z[(size_t)l * b], s);
  X[(size_t)p * bb + e] += s;
}

// opt in to more than 48 KB of dynamic shared memory where a launch needs it
template <typename K>
css_status smem_optin(css_ctx* ctx, K kern, size_t bytes) {
  if (bytes > 48 * 1024) CSS_CU(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return CSS_OK;
}

template <typename T, int BM, int TC>
css_status launch_spmm_t(css_ctx* ctx, const LzArgs& a, const T* V, T* W, cudaStream_t st) {
  const int64_t smem_cap = 160 * 1024;
  int64_t cap_blocks = smem_cap / ((int64_t)BM * BM * sizeof(T));
  int32_t chunk = (int32_t)(a.max_row_blocks < cap_blocks ? a.max_row_blocks : cap_blocks);
  if (chunk < 1) chunk = 1;
  const size_t smem = (size_t)chunk * BM * BM * sizeof(T);
  auto kern = k_spmm<T, BM, TC>;
  CSS_CU(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((unsigned)a.n_brow, (unsigned)css_ceil_div(a.w, 128 * TC));
  kern<<<grid, 128, smem, st>>>(a.b, a.row_ptr, a.col_idx, (const T*)a.Hval, V, W, a.ws, a.w, chunk,
                                (const T*)a.Hlo_diag);
  CSS_LAUNCHED(ctx);
  return CSS_OK;
}

template <typename T>
css_status launch_spmm(css_ctx* ctx, const LzArgs& a, const T* V, T* W, cudaStream_t st) {
  constexpr bool F32 = sizeof(T) == 4;
  if (a.b <= 6) return launch_spmm_t<T, 6, F32 ? 4 : 2>(ctx, a, V, W, st);
  if (a.b <= 8) return launch_spmm_t<T, 8, F32 ? 4 : 2>(ctx, a, V, W, st);
  if (a.b <= 16) return launch_spmm_t<T, 16, F32 ? 2 : 1>(ctx, a, V, W, st);
  if (a.b <= 24) return launch_spmm_t<T, 24, F32 ? 2 : 1>(ctx, a, V, W, st);
  return launch_spmm_t<T, 32, 1>(ctx, a, V, W, st);
}

template <typename T>
css_status run_pass(css_ctx* ctx, const LzArgs& a, cudaStream_t st) {
  const int32_t b = a.b, bb = b * b, ncb = a.ncb, m = a.m;
  const int64_t N = (int64_t)a.n_brow * b;
  const int32_t nch = (int32_t)css_ceil_div(N, RCH);
  T* Qp = (T*)a.Q0;
  T* Qc = (T*)a.Q1;
  T* W = (T*)a.W;
  const size_t vec_bytes = (size_t)N * a.ws * sizeof(T);
  const dim3 rgrid((unsigned)nch, (unsigned)ncb);
  const size_t tile = (size_t)RC * b * sizeof(T);
  const size_t sm_three = 16 * sizeof(double) + 3 * tile + bb * sizeof(T);
  const size_t sm_sub = 3 * tile + 2 * bb * sizeof(T);
  const size_t sm_apply = 2 * tile + bb * sizeof(T);
  double* partA = a.part;
  double* partH = a.part + (size_t)nch * ncb * bb;
  double* sA = a.small;                          // [2][ncb][bb]: raw, symmetrised
  double* sH = a.small + 2 * (size_t)ncb * bb;   // [ncb]
  double* sG = sH + ncb;                         // [ncb][bb]
  double* sR1 = sG + (size_t)ncb * bb;
  double* sR1i = sR1 + (size_t)ncb * bb;
  double* sR2 = sR1i + (size_t)ncb * bb;
  double* sR2i = sR2 + (size_t)ncb * bb;
  double* sC1 = sR2i + (size_t)ncb * bb;
  double* sC2 = sC1 + (size_t)ncb * bb;
  const unsigned rblocks_bb = (unsigned)css_ceil_div((int64_t)ncb * bb, 256);
  const int64_t pb = a.pair_off_h[a.cb0], pe = a.pair_off_h[a.cb0 + ncb];
  const unsigned sblocks = (unsigned)css_ceil_div((pe - pb) * bb, 256);

  CSS_TRY(smem_optin(ctx, k_threeterm<T>, sm_three));
  CSS_TRY(smem_optin(ctx, k_sub<T, false>, sm_sub));
  CSS_TRY(smem_optin(ctx, k_sub<T, true>, sm_sub));
  CSS_TRY(smem_optin(ctx, k_proj2<T>, 3 * tile));
  CSS_TRY(smem_optin(ctx, k_apply<T, true>, sm_apply));
  CSS_TRY(smem_optin(ctx, k_apply<T, false>, sm_apply));
  CSS_CU(ctx, cudaMemsetAsync(Qp, 0, vec_bytes, st));
  CSS_CU(ctx, cudaMemsetAsync(Qc, 0, vec_bytes, st));
  k_init_q1<T><<<(unsigned)css_ceil_div(N, 256), 256, 0, st>>>(a.n_brow, b, a.ws, a.cb0, ncb, a.colour, a.sign,
                                                                a.inv_sqrt_cnt, Qc);
  CSS_LAUNCHED(ctx);
  auto sampled = [&](const T* Qj, int32_t j) -> css_status {
    if (pe <= pb) return CSS_OK;
    if (a.mode == 1) {
      k_scatter<T><<<sblocks, 256, 0, st>>>(pb, pe, b, a.ws, a.cb0, m, j, a.pair_I, a.pair_c, Qj, (T*)a.Qs);
    } else if (a.mode == 2) {
      k_accum_x<T><<<sblocks, 256, 0, st>>>(pb, pe, b, a.ws, a.cb0, a.ldz, j, a.pair_I, a.pair_c, a.nblk, Qj, a.Z,
                                            a.X);
    } else {
      return CSS_OK;
    }
    CSS_LAUNCHED(ctx);
    return CSS_OK;
  };
  CSS_TRY(sampled(Qc, 0));
  for (int32_t j = 0; j < m; ++j) {
    if (a.ev_spmm) CSS_CU(ctx, cudaEventRecord(a.ev_spmm[2 * j], st));
    CSS_TRY(launch_spmm<T>(ctx, a, Qc, W, st));
    if (a.ev_spmm) CSS_CU(ctx, cudaEventRecord(a.ev_spmm[2 * j + 1], st));
    k_threeterm<T><<<rgrid, RT, sm_three, st>>>(N, b, a.ws, a.cb0, Qp, Qc, W, a.Bblk_prev, j == 0 ? 1 : 0, partA,
                                                partH);
    CSS_LAUNCHED(ctx);
    k_reduce<<<rblocks_bb, 256, 0, st>>>(nch, ncb, bb, partA, sA);
    CSS_LAUNCHED(ctx);
    k_reduce<<<(unsigned)css_ceil_div(ncb, 256), 256, 0, st>>>(nch, ncb, 1, partH, sH);
    CSS_LAUNCHED(ctx);
    k_store_A<<<rblocks_bb, 256, 0, st>>>(ncb, b, a.cb0, m, j, sA, a.Ablk);
    CSS_LAUNCHED(ctx);
    const double* Asym = sA + (size_t)ncb * bb;
    if (j + 1 == m) break;
    if (a.flags & CSS_REORTH_LOCAL) {
      k_sub<T, false><<<rgrid, RT, sm_sub, st>>>(N, b, a.ws, Qc, Qp, W, Asym, nullptr, nullptr);
      CSS_LAUNCHED(ctx);
      k_proj2<T><<<rgrid, RT, 3 * tile, st>>>(N, b, a.ws, Qc, Qp, W, partA, partA + (size_t)nch * ncb * bb);
      CSS_LAUNCHED(ctx);
      k_reduce<<<rblocks_bb, 256, 0, st>>>(nch, ncb, bb, partA, sC1);
      CSS_LAUNCHED(ctx);
      k_reduce<<<rblocks_bb, 256, 0, st>>>(nch, ncb, bb, partA + (size_t)nch * ncb * bb, sC2);
      CSS_LAUNCHED(ctx);
      k_sub<T, true><<<rgrid, RT, sm_sub, st>>>(N, b, a.ws, Qc, Qp, W, sC1, sC2, partA);
      CSS_LAUNCHED(ctx);
    } else {
      k_sub<T, true><<<rgrid, RT, sm_sub, st>>>(N, b, a.ws, Qc, Qp, W, Asym, nullptr, partA);
      CSS_LAUNCHED(ctx);
    }
    // shifted CholeskyQR3 of W: R0 from G + sI, then two plain CholeskyQR passes
    k_reduce<<<rblocks_bb, 256, 0, st>>>(nch, ncb, bb, partA, sG);
    CSS_LAUNCHED(ctx);
    k_chol<0><<<(unsigned)css_ceil_div(ncb, 4), 128, 0, st>>>(ncb, b, a.cb0, m, j, sG, sH, a.tau, a.shift_rel, sR1, sR1i,
                                                              sC1, a.Bblk, a.done, a.nblk);
    CSS_LAUNCHED(ctx);
    CSS_CU(ctx, cudaMemcpyAsync(sC1, sR1, sizeof(double) * ncb * bb, cudaMemcpyDeviceToDevice, st));
    k_apply<T, true><<<rgrid, RT, sm_apply, st>>>(N, b, a.ws, W, nullptr, sR1i, partA);
    CSS_LAUNCHED(ctx);
    k_reduce<<<rblocks_bb, 256, 0, st>>>(nch, ncb, bb, partA, sG);
    CSS_LAUNCHED(ctx);
    k_chol<1><<<(unsigned)css_ceil_div(ncb, 4), 128, 0, st>>>(ncb, b, a.cb0, m, j, sG, sH, a.tau, 0.0, sR1, sR1i,
                                                              sC1, a.Bblk, a.done, a.nblk);
    CSS_LAUNCHED(ctx);
    k_apply<T, true><<<rgrid, RT, sm_apply, st>>>(N, b, a.ws, W, nullptr, sR1i, partA);
    CSS_LAUNCHED(ctx);
    k_reduce<<<rblocks_bb, 256, 0, st>>>(nch, ncb, bb, partA, sG);
    CSS_LAUNCHED(ctx);
    k_chol<2><<<(unsigned)css_ceil_div(ncb, 4), 128, 0, st>>>(ncb, b, a.cb0, m, j, sG, sH, a.tau, 0.0, sR2, sR2i,
                                                              sC1, a.Bblk, a.done, a.nblk);
    CSS_LAUNCHED(ctx);
    // Q_{j+1} = W R2^-1 overwrites Q_{j-1}
    k_apply<T, false><<<rgrid, RT, sm_apply, st>>>(N, b, a.ws, W, Qp, sR2i, nullptr);
    CSS_LAUNCHED(ctx);
    CSS_TRY(sampled(Qp, j + 1));
    // B_{j} for the next step's three-term update, in the batch's local layout
    CSS_CU(ctx, cudaMemcpy2DAsync(a.Bblk_prev + (size_t)a.cb0 * bb, bb * sizeof(double),
                                  a.Bblk + ((size_t)a.cb0 * m + j) * bb, (size_t)m * bb * sizeof(double),
                                  bb * sizeof(double), ncb, cudaMemcpyDeviceToDevice, st));
    T* t = Qp;
    Qp = Qc;
    Qc = t;
  }
  return CSS_OK;
}

}  // namespace

// Bblk_prev is indexed by global colour; the three-term kernel reads [cb0 + lc]
css_status css_lanczos_pass(css_ctx* ctx, const LzArgs& a, cudaStream_t st) {
  if (a.fp32) return run_pass<float>(ctx, a, st);
  return run_pass<double>(ctx, a, st);
}

size_t css_lanczos_part_doubles(int64_t N, int32_t b, int32_t ncb) {
  const int64_t nch = css_ceil_div(N, RCH);
  return (size_t)nch * ncb * b * b * 2 + (size_t)nch * ncb + 64;
}

size_t css_lanczos_small_doubles(int32_t b, int32_t ncb) { return (size_t)ncb * b * b * 10 + ncb + 64; }
