// CSS density matrix on H's pattern (paper, Eq. 2 and Eq. 5-7): set-up of the sampled
// (row, colour) pairs, the block-Lanczos passes, the eigensolve, the chemical potential, the
// reconstruction X_c = Q_c Z_c on the sampled rows and the extraction
//     P~_IJ = X_{c(J)}[I] diag(s_J),  P = (P~ + P~^T) / 2,  Tr P,  Tr(P H).
//
// "Pairs": for every block row I the distinct colours of its pattern columns.  X is needed
// exactly on those (I, c) pairs; they are stored sorted by colour, so the pairs of a colour
// batch are one contiguous range.
#include <algorithm>
#include <cmath>

#include "css_eigen.cuh"
#include "css_lanczos.cuh"

css_status css_scan_i32(css_ctx* ctx, const int32_t* in, int32_t* out, int64_t n, cudaStream_t st, int depth = 0);

namespace {

constexpr int ERR_PATTERN = 1;     // pattern not structurally symmetric / diagonal missing
constexpr int ERR_COLOUR = 2;      // colour out of range

// ----------------------------------------------------------------------- set-up
__global__ void k_concat_rowptr(int32_t n, const int32_t* __restrict__ src, int32_t row_off, int32_t blk_off,
                                int32_t* __restrict__ dst) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= n) dst[row_off + i] = src[i] + blk_off;
}

__global__ void k_offset_i32(int64_t n, const int32_t* __restrict__ src, int32_t off, int32_t* __restrict__ dst) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i] + off;
}

// colour -1 marks a molecule that is in no probe block of this call (a colour owned by another
// rank of a colour-partitioned build); allowed only when `partial` is set
__global__ void k_rows(int32_t n_brow, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                       const int32_t* __restrict__ colour, int32_t n_col, int32_t* __restrict__ brow,
                       int32_t* __restrict__ trans, int32_t* __restrict__ cnt, int32_t* __restrict__ maxrow,
                       int32_t* __restrict__ err, int partial = 0) {
  int32_t I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n_brow) return;
  const int32_t s = row_ptr[I], e = row_ptr[I + 1];
  atomicMax(maxrow, e - s);
  const int32_t cI = colour[I];
  if (cI < 0 || cI >= n_col) {
    if (!(partial && cI == -1)) atomicOr(err, ERR_COLOUR);
  } else {
    atomicAdd(&cnt[cI], 1);
  }
  bool diag = false;
  for (int32_t k = s; k < e; ++k) {
    brow[k] = I;
    const int32_t J = col_idx[k];
    if (J == I) diag = true;
    if (J < 0 || J >= n_brow) {
      atomicOr(err, ERR_PATTERN);
      trans[k] = k;
      continue;
    }
    // binary search for column I in row J
    int32_t lo = row_ptr[J], hi = row_ptr[J + 1] - 1, f = -1;
    while (lo <= hi) {
      int32_t mid = (lo + hi) >> 1, v = col_idx[mid];
      if (v == I) {
        f = mid;
        break;
      }
      if (v < I) lo = mid + 1;
      else hi = mid - 1;
    }
    if (f < 0) {
      atomicOr(err, ERR_PATTERN);
      f = k;
    }
    trans[k] = f;
  }
  if (!diag) atomicOr(err, ERR_PATTERN);
}

// empty colours are finished from the start (no blocks, no Ritz pairs)
__global__ void k_inv_sqrt(int32_t n_col, const int32_t* __restrict__ cnt, double* __restrict__ isq,
                           int32_t* __restrict__ nblk, int32_t* __restrict__ done, int32_t m) {
  int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_col) return;
  isq[c] = cnt[c] > 0 ? 1.0 / sqrt((double)cnt[c]) : 0.0;
  nblk[c] = cnt[c] > 0 ? m : 0;
  done[c] = cnt[c] > 0 ? 0 : 1;
}

// distinct colours among row I's pattern columns
__global__ void k_pair_count(int32_t n_brow, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                             const int32_t* __restrict__ colour, int32_t* __restrict__ pcount) {
  int32_t I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n_brow) return;
  const int32_t s = row_ptr[I], e = row_ptr[I + 1];
  int32_t n = 0;
  for (int32_t k = s; k < e; ++k) {
    const int32_t c = colour[col_idx[k]];
    if (c < 0) continue;  // not probed in this call
    bool seen = false;
    for (int32_t k2 = s; k2 < k; ++k2)
      if (colour[col_idx[k2]] == c) {
        seen = true;
        break;
      }
    n += !seen;
  }
  pcount[I] = n;
}

__global__ void k_pair_fill(int32_t n_brow, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                            const int32_t* __restrict__ colour, const int32_t* __restrict__ pstart,
                            int32_t* __restrict__ pr_c, int32_t* __restrict__ bpr, int32_t* __restrict__ ccount) {
  int32_t I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n_brow) return;
  const int32_t s = row_ptr[I], e = row_ptr[I + 1];
  int32_t n = 0;
  const int32_t base = pstart[I];
  for (int32_t k = s; k < e; ++k) {
    const int32_t c = colour[col_idx[k]];
    if (c < 0) {  // not probed in this call: the block gets no column
      bpr[k] = -1;
      continue;
    }
    int32_t found = -1;
    for (int32_t t = 0; t < n; ++t)
      if (pr_c[base + t] == c) {
        found = t;
        break;
      }
    if (found < 0) {
      found = n++;
      pr_c[base + found] = c;
      atomicAdd(&ccount[c], 1);
    }
    bpr[k] = base + found;
  }
}

// row-grouped pair q -> colour-sorted slot (order inside a colour is by arrival)
__global__ void k_pair_place(int32_t n_brow, const int32_t* __restrict__ pstart, const int32_t* __restrict__ pr_c,
                             const int32_t* __restrict__ coff, int32_t* __restrict__ cfill, int32_t* __restrict__ perm,
                             int32_t* __restrict__ pair_I, int32_t* __restrict__ pair_c) {
  int32_t I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n_brow) return;
  for (int32_t q = pstart[I]; q < pstart[I + 1]; ++q) {
    const int32_t c = pr_c[q];
    const int32_t pos = coff[c] + atomicAdd(&cfill[c], 1);
    perm[q] = pos;
    pair_I[pos] = I;
    pair_c[pos] = c;
  }
}

__global__ void k_pob(int32_t nnzb, const int32_t* __restrict__ bpr, const int32_t* __restrict__ perm,
                      int32_t* __restrict__ pob) {
  int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nnzb) pob[k] = bpr[k] < 0 ? -1 : perm[bpr[k]];
}

// ----------------------------------------------------------- chemical potential
// Bounded grid barrier (generation counter): every wait gives up after ~2^24 polls, sets
// *err and returns false, so the kernel always terminates.
__device__ bool grid_sync(unsigned* count, unsigned* gen, unsigned nb, int32_t* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vg = gen;
    const unsigned g = *vg;
    __threadfence();
    const unsigned arrived = atomicAdd(count, 1u) + 1u;
    ok = 1;
    if (arrived == nb) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      long long spins = 0;
      while (*vg == g) {
        if (++spins > (1ll << 24) || *(volatile int32_t*)err) {
          atomicOr(err, 4);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

constexpr int MU_T = 256;
constexpr int MU_MAXSYS = 512;

// Chemical potential of every system s from its Ritz quadrature
//     g_s(mu) = sum_{c in s} sum_k f(lam_ck; mu) w_ck - N_e,s / 2:
// mu_s is the midpoint of {mu : |g_s(mu)| <= tol_s}; its lower end (smallest mu with
// g >= -tol) and upper end (largest mu with g <= +tol) are bisected together in one
// persistent cooperative launch.  Each CTA sums a fixed range of colours in a fixed order;
// all CTAs then reduce the per-CTA partials in the same order, so every CTA holds identical
// brackets and the result is deterministic.
__global__ void __launch_bounds__(MU_T) k_mu(int32_t n_sys, int32_t n_col, int32_t nmax, const int32_t* __restrict__ nblk,
                                             int32_t b, const int32_t* __restrict__ sys_of_colour,
                                             const double* __restrict__ lam, const double* __restrict__ wgt,
                                             const double* __restrict__ kT, const double* __restrict__ half_ne,
                                             const double* __restrict__ tol, const int32_t* __restrict__ solve,
                                             const double* __restrict__ mu_in, double* __restrict__ mu_out,
                                             double* __restrict__ part, unsigned* __restrict__ bar,
                                             int32_t* __restrict__ err, int32_t nb_extra) {
  __shared__ double acc[2][MU_MAXSYS];
  __shared__ double lo[2][MU_MAXSYS], hi[2][MU_MAXSYS];
  __shared__ int conv[MU_MAXSYS];
  __shared__ double red[2][MU_T / 32];
  __shared__ int all_done;
  const unsigned G = gridDim.x;
  const int32_t per = (int32_t)((n_col + G - 1) / G);
  const int32_t c0 = blockIdx.x * per, c1 = min(n_col, c0 + per);
  double* pbuf[2] = {part, part + (size_t)2 * n_sys * G};
  // phase 0: spectrum bounds per system
  for (int32_t s = threadIdx.x; s < n_sys; s += blockDim.x) {
    lo[0][s] = 1e300;
    hi[0][s] = -1e300;
  }
  __syncthreads();
  for (int32_t c = c0; c < c1; ++c) {
    const int32_t n = nblk[c] * b;
    double mn = 1e300, mx = -1e300;
    for (int32_t k = threadIdx.x; k < n; k += blockDim.x) {
      const double x = lam[(size_t)c * nmax + k];
      mn = fmin(mn, x);
      mx = fmax(mx, x);
    }
    for (int o = 16; o > 0; o >>= 1) {
      mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = mn;
      red[1][threadIdx.x >> 5] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double t0 = 1e300, t1 = -1e300;
      for (int i = 0; i < MU_T / 32; ++i) {
        t0 = fmin(t0, red[0][i]);
        t1 = fmax(t1, red[1][i]);
      }
      const int32_t s = sys_of_colour[c];
      lo[0][s] = fmin(lo[0][s], t0);
      hi[0][s] = fmax(hi[0][s], t1);
    }
    __syncthreads();
  }
  for (int32_t s = threadIdx.x; s < n_sys; s += blockDim.x) {
    pbuf[0][(size_t)s * G + blockIdx.x] = lo[0][s];
    pbuf[0][(size_t)(n_sys + s) * G + blockIdx.x] = hi[0][s];
  }
  if (!grid_sync(bar, bar + 1, G + (unsigned)nb_extra, err)) return;
  for (int32_t s = threadIdx.x; s < n_sys; s += blockDim.x) {
    double a = 1e300, z = -1e300;
    for (unsigned g = 0; g < G; ++g) {
      a = fmin(a, __ldcg(&pbuf[0][(size_t)s * G + g]));
      z = fmax(z, __ldcg(&pbuf[0][(size_t)(n_sys + s) * G + g]));
    }
    lo[0][s] = lo[1][s] = a - 1.0;
    hi[0][s] = hi[1][s] = z + 1.0;
    conv[s] = solve[s] ? 0 : 1;
  }
  __syncthreads();
  for (int it = 0; it < 200; ++it) {
    for (int32_t s = threadIdx.x; s < n_sys; s += blockDim.x) acc[0][s] = acc[1][s] = 0.0;
    __syncthreads();
    for (int32_t c = c0; c < c1; ++c) {
      const int32_t s = sys_of_colour[c];
      if (conv[s]) continue;
      const double m0 = 0.5 * (lo[0][s] + hi[0][s]), m1 = 0.5 * (lo[1][s] + hi[1][s]);
      const double t_ = kT[s];
      const int32_t n = nblk[c] * b;
      double v0 = 0.0, v1 = 0.0;
      for (int32_t k = threadIdx.x; k < n; k += blockDim.x) {
        const double x = lam[(size_t)c * nmax + k], w = wgt[(size_t)c * nmax + k];
        v0 += css_fermi_dirac(x, m0, t_) * w;
        v1 += css_fermi_dirac(x, m1, t_) * w;
      }
      for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
      }
      if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = v0;
        red[1][threadIdx.x >> 5] = v1;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0;
        for (int i = 0; i < MU_T / 32; ++i) {
          t0 += red[0][i];
          t1 += red[1][i];
        }
        acc[0][s] += t0;
        acc[1][s] += t1;
      }
      __syncthreads();
    }
    double* pb = pbuf[(it + 1) & 1];
    for (int32_t s = threadIdx.x; s < n_sys; s += blockDim.x) {
      pb[(size_t)s * G + blockIdx.x] = acc[0][s];
      pb[(size_t)(n_sys + s) * G + blockIdx.x] = acc[1][s];
    }
    if (!grid_sync(bar, bar + 1, G + (unsigned)nb_extra, err)) return;
    if (threadIdx.x == 0) all_done = 1;
    __syncthreads();
    for (int32_t s = threadIdx.x; s < n_sys; s += blockDim.x) {
      if (conv[s]) continue;
      double g0 = 0.0, g1 = 0.0;
      for (unsigned q = 0; q < G; ++q) {
        g0 += __ldcg(&pb[(size_t)s * G + q]);
        g1 += __ldcg(&pb[(size_t)(n_sys + s) * G + q]);
      }
      g0 -= half_ne[s];
      g1 -= half_ne[s];
      const double m0 = 0.5 * (lo[0][s] + hi[0][s]), m1 = 0.5 * (lo[1][s] + hi[1][s]);
      if (g0 >= -tol[s]) hi[0][s] = m0;
      else lo[0][s] = m0;
      if (g1 <= tol[s]) lo[1][s] = m1;
      else hi[1][s] = m1;
      const bool d0 = hi[0][s] - lo[0][s] <= 1e-13 * fmax(1.0, fabs(m0));
      const bool d1 = hi[1][s] - lo[1][s] <= 1e-13 * fmax(1.0, fabs(m1));
      if (d0 && d1) conv[s] = 1;
      else all_done = 0;
    }
    __syncthreads();
    if (all_done) break;
  }
  if (blockIdx.x == 0)
    for (int32_t s = threadIdx.x; s < n_sys; s += blockDim.x)
      mu_out[s] = solve[s] ? 0.5 * (0.5 * (lo[0][s] + hi[0][s]) + 0.5 * (lo[1][s] + hi[1][s])) : mu_in[s];
}

// --------------------------------------------------------- reconstruction on pairs
__global__ void k_zsplit(int64_t n, const double* __restrict__ Z, float* __restrict__ zh, float* __restrict__ zl) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double z = Z[i];
  const float h = (float)z;
  zh[i] = h;
  zl[i] = (float)(z - (double)h);
}

// X[p][a][kk] = sum_j sum_l Qs[p][j][a][l] Z_c[j b + l][kk]; FP64 rows, or FP32 rows with a
// two-term FP32 split of Z and FP64 accumulation over the blocks j
template <typename T>
__global__ void k_xcompute(int64_t n_pairs, int32_t b, int32_t m, int32_t nmax, const int32_t* __restrict__ pair_c,
                           const int32_t* __restrict__ nblk, const T* __restrict__ Qs, const double* __restrict__ Z,
                           const float* __restrict__ zh, const float* __restrict__ zl, double* __restrict__ X) {
  const int32_t bb = b * b;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t p = t / bb;
  if (p >= n_pairs) return;
  const int32_t e = (int32_t)(t % bb), a = e / b, kk = e % b;
  const int32_t c = pair_c[p];
  const int32_t nb = nblk[c];
  const T* q = Qs + (size_t)p * m * bb + (size_t)a * b;
  double acc = 0.0;
  if (sizeof(T) == 8) {
    const double* z = Z + (size_t)c * nmax * b + kk;
    for (int32_t j = 0; j < nb; ++j)
      for (int32_t l = 0; l < b; ++l) acc = fma((double)q[(size_t)j * bb + l], z[(size_t)(j * b + l) * b], acc);
  } else {
    const float* h = zh + (size_t)c * nmax * b + kk;
    const float* lw = zl + (size_t)c * nmax * b + kk;
    for (int32_t j = 0; j < nb; ++j) {
      float sh = 0.f, sl = 0.f;
      for (int32_t l = 0; l < b; ++l) {
        const float qv = (float)q[(size_t)j * bb + l];
        sh = fmaf(qv, h[(size_t)(j * b + l) * b], sh);
        sl = fmaf(qv, lw[(size_t)(j * b + l) * b], sl);
      }
      acc += (double)sh + (double)sl;
    }
  }
  X[(size_t)p * bb + e] = acc;
}

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}

// X_p = Qs_p Z_c for the FP32 Krylov rows: for every pair p of colour c a (b x m b) x (m b x b)
// product.  A CTA takes up to XP pairs of one colour and walks the blocks j of Z_c: the
// blocks Qs_p[j] (transposed) and the FP32 hi/lo halves of Z_c[j] are staged in shared memory
// (zero padded to BP x BP; two stages filled by cp.async, the next block's copies in flight
// during the current block's multiply), and each thread owns a 4 x 4 tile of one pair's X.  The hi product
// of a block is summed in FP32 and added into an FP32 hi + lo pair by TwoSum; the lo product
// (2^-24 of the hi one) is summed in FP32 over all blocks.  The sum is widened to FP64 once.
template <int BP>
__global__ void __launch_bounds__(256) k_xtile(int32_t n_col, int32_t b, int32_t m, int32_t nmax,
                                               const int32_t* __restrict__ coff, const int32_t* __restrict__ cta_off,
                                               const int32_t* __restrict__ nblk, const float* __restrict__ Qs,
                                               const float* __restrict__ zh, const float* __restrict__ zl,
                                               double* __restrict__ X) {
  constexpr int CB = BP / 4, TPP = CB * CB, XP = 256 / TPP;
  __shared__ __align__(16) float sQ[2][XP][BP][BP];  // [stage][pair][l][a]
  __shared__ __align__(16) float sZh[2][BP][BP];     // [stage][l][k]
  __shared__ __align__(16) float sZl[2][BP][BP];
  const int32_t bid = blockIdx.x;
  if (bid >= cta_off[n_col]) return;
  int32_t lo = 0, hi = n_col - 1;  // colour c: cta_off[c] <= bid < cta_off[c + 1]
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (cta_off[mid] <= bid) lo = mid;
    else hi = mid - 1;
  }
  const int32_t c = lo;
  const int32_t p0 = coff[c] + (bid - cta_off[c]) * XP;
  const int32_t np = min(XP, coff[c + 1] - p0);
  const int32_t nb = nblk[c], bb = b * b;
  const int t = threadIdx.x;
  const int pp = t / TPP, rem = t - pp * TPP, ai = rem / CB, ki = rem - ai * CB;
  // zero both stages once: the copies write only the b x b part of each block
  for (int e = t; e < 2 * XP * BP * BP; e += 256) (&sQ[0][0][0][0])[e] = 0.0f;
  for (int e = t; e < 2 * BP * BP; e += 256) {
    (&sZh[0][0][0])[e] = 0.0f;
    (&sZl[0][0][0])[e] = 0.0f;
  }
  __syncthreads();
  // asynchronous copies of block j into stage s (Qs blocks transposed on the way)
  auto issue = [&](int32_t j, int s) {
    for (int32_t e = t; e < np * bb; e += 256) {
      const int32_t q = e / bb, r = e - q * bb, a = r / b, l = r - a * b;
      cp_async4(&sQ[s][q][l][a], Qs + ((size_t)(p0 + q) * m + j) * bb + r);
    }
    for (int32_t e = t; e < bb; e += 256) {
      const int32_t l = e / b, k = e - l * b;
      const size_t o = ((size_t)c * nmax + (size_t)j * b + l) * b + k;
      cp_async4(&sZh[s][l][k], zh + o);
      cp_async4(&sZl[s][l][k], zl + o);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  float ahi[16], alo[16], asm_[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) ahi[i] = alo[i] = asm_[i] = 0.0f;
  if (nb > 0) issue(0, 0);
  for (int32_t j = 0; j < nb; ++j) {
    const int s = j & 1;
    if (j + 1 < nb) {
      issue(j + 1, s ^ 1);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();  // block j is in stage s for every thread
    if (pp < np) {
      float ph[4][4] = {};
      for (int32_t l = 0; l < b; ++l) {
        const float4 x = *reinterpret_cast<const float4*>(&sQ[s][pp][l][ai * 4]);
        const float4 zH = *reinterpret_cast<const float4*>(&sZh[s][l][ki * 4]);
        const float4 zL = *reinterpret_cast<const float4*>(&sZl[s][l][ki * 4]);
        const float xv[4] = {x.x, x.y, x.z, x.w}, hv[4] = {zH.x, zH.y, zH.z, zH.w}, lv[4] = {zL.x, zL.y, zL.z, zL.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            ph[i][k] = fmaf(xv[i], hv[k], ph[i][k]);
            asm_[i * 4 + k] = fmaf(xv[i], lv[k], asm_[i * 4 + k]);
          }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) {  // TwoSum of the running hi sum and this block's product
          const int u = i * 4 + k;
          const float sm = __fadd_rn(ahi[u], ph[i][k]);
          const float z = __fsub_rn(sm, ahi[u]);
          alo[u] = __fadd_rn(alo[u], __fadd_rn(__fsub_rn(ahi[u], __fsub_rn(sm, z)), __fsub_rn(ph[i][k], z)));
          ahi[u] = sm;
        }
    }
    __syncthreads();  // stage s is free for block j + 2
  }
  if (pp >= np) return;
  double* xo = X + (size_t)(p0 + pp) * bb;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int32_t a = ai * 4 + i, kk = ki * 4 + k;
      const int u = i * 4 + k;
      if (a < b && kk < b) xo[a * b + kk] = (double)ahi[u] + (double)alo[u] + (double)asm_[u];
    }
}

// CTAs of k_xtile per colour (ceil(pairs / xp)), prefix-summed; one thread, in colour order
__global__ void k_xtile_plan(int32_t n_col, int32_t xp, const int32_t* __restrict__ coff, int32_t* __restrict__ cta_off) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int32_t s = 0;
  for (int32_t c = 0; c < n_col; ++c) {
    cta_off[c] = s;
    s += (coff[c + 1] - coff[c] + xp - 1) / xp;
  }
  cta_off[n_col] = s;
}

// P_val and trace partials of one system's blocks [k0, k1)
constexpr int EX_T = 256;
__global__ void __launch_bounds__(EX_T) k_extract(int32_t k0, int32_t k1, int32_t b, int32_t blk_off,
                                                  const int32_t* __restrict__ brow, const int32_t* __restrict__ col_idx,
                                                  const int32_t* __restrict__ trans, const int32_t* __restrict__ pob,
                                                  const int8_t* __restrict__ sign, const double* __restrict__ X,
                                                  const double* __restrict__ Hval, int sym, double* __restrict__ P,
                                                  double* __restrict__ part) {
  __shared__ double r1[EX_T / 32], r2[EX_T / 32];
  const int32_t bb = b * b;
  const int64_t t = (int64_t)k0 * bb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double tp = 0.0, tph = 0.0;
  if (t < (int64_t)k1 * bb) {
    const int32_t k = (int32_t)(t / bb), e = (int32_t)(t % bb), a = e / b, kk = e % b;
    const int32_t I = brow[k], J = col_idx[k];
    const int32_t pk = pob[k];  // -1: column J is not probed in this call (written as zero)
    double v = pk < 0 ? 0.0 : X[(size_t)pk * bb + e] * (double)sign[(size_t)J * b + kk];
    if (sym) {
      const int32_t kt = trans[k];
      const double w = X[(size_t)pob[kt] * bb + kk * b + a] * (double)sign[(size_t)I * b + a];
      v = 0.5 * (v + w);
    }
    P[(size_t)(k - blk_off) * bb + e] = v;
    if (I == J && a == kk) tp = v;
    tph = v * Hval[(size_t)k * bb + e];
  }
  for (int o = 16; o > 0; o >>= 1) {
    tp += __shfl_xor_sync(0xffffffffu, tp, o);
    tph += __shfl_xor_sync(0xffffffffu, tph, o);
  }
  if ((threadIdx.x & 31) == 0) {
    r1[threadIdx.x >> 5] = tp;
    r2[threadIdx.x >> 5] = tph;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, z = 0.0;
    for (int i = 0; i < EX_T / 32; ++i) {
      a += r1[i];
      z += r2[i];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = z;
  }
}

// out = sum of the (Tr P, Tr PH) partials; fixed thread-to-partial map and a fixed tree, so
// the sum is deterministic
__global__ void __launch_bounds__(1024) k_trace_sum(int32_t nparts, const double* __restrict__ part,
                                                    double* __restrict__ out) {
  __shared__ double r1[32], r2[32];
  double a = 0.0, z = 0.0;
  for (int32_t i = threadIdx.x; i < nparts; i += blockDim.x) {
    a += part[2 * i];
    z += part[2 * i + 1];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    z += __shfl_xor_sync(0xffffffffu, z, o);
  }
  if ((threadIdx.x & 31) == 0) {
    r1[threadIdx.x >> 5] = a;
    r2[threadIdx.x >> 5] = z;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tz = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      ta += r1[i];
      tz += r2[i];
    }
    out[0] = ta;
    out[1] = tz;
  }
}

__global__ void k_count_breakdown(int32_t n_col, int32_t m, const int32_t* __restrict__ nblk,
                                  const int32_t* __restrict__ cnt, int32_t* __restrict__ out) {
  int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n_col && cnt[c] > 0 && nblk[c] < m) atomicAdd(out, 1);
}

// OR of the eigen stage's per-colour status words (bit 2: a band-reduction wait gave up)
__global__ void k_status_or(int32_t n_col, const int32_t* __restrict__ status, int32_t* __restrict__ out) {
  int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n_col && (status[c] & 2)) atomicOr(out, 2);
}

template <typename Tp>
css_status ws_get(css_ctx* ctx, const char* name, size_t count, Tp** p) {
  return css_ws(ctx, name, count * sizeof(Tp), (void**)p);
}

struct Timer {
  css_ctx* ctx;
  cudaStream_t st;
  cudaEvent_t ev[16];
  int n = 0;
  bool on;
  Timer(css_ctx* c, cudaStream_t s) : ctx(c), st(s), on(c->timing) {}
  void mark() {
    if (!on || n >= 16) return;
    cudaEventCreate(&ev[n]);
    cudaEventRecord(ev[n], st);
    ++n;
  }
  double ms(int a, int b) {
    float t = 0.f;
    if (on && a < n && b < n) cudaEventElapsedTime(&t, ev[a], ev[b]);
    return t;
  }
  ~Timer() {
    for (int i = 0; i < n; ++i) cudaEventDestroy(ev[i]);
  }
};

}  // namespace

css_status css_density_impl(css_ctx* ctx, int32_t n_sys, const css_sys_desc* sys, int32_t m, css_precision prec,
                            uint32_t flags, double* trP, double* trPH, double* mu_out, cudaStream_t st,
                            void* yfull, int32_t ldy, bool partial, const int32_t* colour_ids) {
  // ------------------------------------------------------------ validation
  if (n_sys < 1 || n_sys > MU_MAXSYS) return css_set_arg_error(ctx, "css_density: n_sys out of range");
  if (prec != CSS_FP64 && prec != CSS_MIXED_FP32 && prec != CSS_MIXED_3XTF32 && prec != CSS_FP64_SPLIT)
    return css_set_arg_error(ctx, "css_density: unknown precision");
  if (flags & ~(CSS_SYMMETRIZE | CSS_TWO_PASS | CSS_REORTH_LOCAL | CSS_ENERGY_WEIGHTED | CSS_INV_SQRT | CSS_RITZ_ONLY))
    return css_set_arg_error(ctx, "css_density: unknown flag");
  if (partial && (n_sys != 1 || (flags & CSS_SYMMETRIZE)))
    return css_set_arg_error(ctx, "css_density_colours: one system, unsymmetrised output");
  const int32_t b = sys[0].H.b;
  if (b < 1) return css_set_arg_error(ctx, "css_density: b < 1");
  if (b > CSS_MAX_B) {
    ctx->last_error = "css_density: b > 32 is not supported";
    return CSS_ERR_UNSUPPORTED;
  }
  if (m < 1 || (int64_t)m * b > 4096) return css_set_arg_error(ctx, "css_density: need 1 <= m and m*b <= 4096");
  int64_t nb_tot = 0, nnz_tot = 0, nc_tot = 0;
  for (int32_t s = 0; s < n_sys; ++s) {
    const css_sys_desc& d = sys[s];
    if (d.H.b != b) return css_set_arg_error(ctx, "css_density_batch: all systems need the same b");
    if (d.H.n_brow < 1 || d.H.nnzb < d.H.n_brow || !d.H.row_ptr || !d.H.col_idx || !d.H.val || !d.colour ||
        !d.sign || !d.P_val || d.n_colours < 1)
      return css_set_arg_error(ctx, "css_density: bad H, colour, sign or P_val argument");
    if (!(d.fermi.kT >= 0.0) || !std::isfinite(d.fermi.kT) || !std::isfinite(d.fermi.mu) ||
        !std::isfinite(d.fermi.n_elec) || !std::isfinite(d.fermi.ne_tol))
      return css_set_arg_error(ctx, "css_density: kT must be finite and >= 0, mu and n_elec finite");
    nb_tot += d.H.n_brow;
    nnz_tot += d.H.nnzb;
    nc_tot += d.n_colours;
  }
  if (nb_tot > (1ll << 30) || nnz_tot > (1ll << 30) || nc_tot > (1 << 24) || nnz_tot * b * b > (1ll << 40))
    return css_set_arg_error(ctx, "css_density: problem too large for 32-bit block indices");
  const int32_t n_brow = (int32_t)nb_tot, nnzb = (int32_t)nnz_tot, n_col = (int32_t)nc_tot;
  const int64_t N = (int64_t)n_brow * b;
  const int32_t bb = b * b, nmax = m * b;
  const bool f32 = prec == CSS_MIXED_FP32 || prec == CSS_MIXED_3XTF32;
  const bool two_pass = (flags & CSS_TWO_PASS) != 0 || yfull != nullptr;
  const bool ritz_only = (flags & CSS_RITZ_ONLY) != 0;  // stop after the exact diagonalisation
  const int T = 256;
  Timer tm(ctx, st);
  tm.mark();  // 0

  // -------------------------------------------------- combined system (batch)
  const int32_t *row_ptr, *col_idx, *colour;
  const int8_t* sign;
  const double* Hval;
  double* Pout;
  int32_t *sys_of_colour, *row_off_dev;
  std::vector<int32_t> row_off(n_sys + 1), blk_off(n_sys + 1), col_off(n_sys + 1);
  row_off[0] = blk_off[0] = col_off[0] = 0;
  for (int32_t s = 0; s < n_sys; ++s) {
    row_off[s + 1] = row_off[s] + sys[s].H.n_brow;
    blk_off[s + 1] = blk_off[s] + sys[s].H.nnzb;
    col_off[s + 1] = col_off[s] + sys[s].n_colours;
  }
  CSS_TRY(ws_get(ctx, "sys_of_colour", n_col, &sys_of_colour));
  CSS_TRY(ws_get(ctx, "row_off", n_sys + 1, &row_off_dev));
  {
    std::vector<int32_t> soc(n_col);
    for (int32_t s = 0; s < n_sys; ++s)
      for (int32_t c = col_off[s]; c < col_off[s + 1]; ++c) soc[c] = s;
    int32_t* hp;
    CSS_TRY(css_pinned(ctx, sizeof(int32_t) * (n_col + n_sys + 1) + 256, (void**)&hp));
    memcpy(hp, soc.data(), sizeof(int32_t) * n_col);
    CSS_CU(ctx, cudaMemcpyAsync(sys_of_colour, hp, sizeof(int32_t) * n_col, cudaMemcpyHostToDevice, st));
    CSS_CU(ctx, cudaStreamSynchronize(st));
  }
  if (n_sys == 1) {
    row_ptr = sys[0].H.row_ptr;
    col_idx = sys[0].H.col_idx;
    colour = sys[0].colour;
    sign = sys[0].sign;
    Hval = sys[0].H.val;
    Pout = sys[0].P_val;
  } else {
    int32_t *rp, *ci, *co;
    int8_t* sg;
    double* hv;
    CSS_TRY(ws_get(ctx, "b_rowptr", n_brow + 1, &rp));
    CSS_TRY(ws_get(ctx, "b_colidx", nnzb, &ci));
    CSS_TRY(ws_get(ctx, "b_colour", n_brow, &co));
    CSS_TRY(ws_get(ctx, "b_sign", N, &sg));
    CSS_TRY(ws_get(ctx, "b_hval", (size_t)nnzb * bb, &hv));
    for (int32_t s = 0; s < n_sys; ++s) {
      const css_sys_desc& d = sys[s];
      k_concat_rowptr<<<(unsigned)css_ceil_div(d.H.n_brow + 1, T), T, 0, st>>>(d.H.n_brow, d.H.row_ptr, row_off[s],
                                                                                blk_off[s], rp);
      CSS_LAUNCHED(ctx);
      k_offset_i32<<<(unsigned)css_ceil_div(d.H.nnzb, T), T, 0, st>>>(d.H.nnzb, d.H.col_idx, row_off[s],
                                                                       ci + blk_off[s]);
      CSS_LAUNCHED(ctx);
      k_offset_i32<<<(unsigned)css_ceil_div(d.H.n_brow, T), T, 0, st>>>(d.H.n_brow, d.colour, col_off[s],
                                                                         co + row_off[s]);
      CSS_LAUNCHED(ctx);
      CSS_CU(ctx, cudaMemcpyAsync(sg + (size_t)row_off[s] * b, d.sign, (size_t)d.H.n_brow * b, cudaMemcpyDeviceToDevice,
                                  st));
      CSS_CU(ctx, cudaMemcpyAsync(hv + (size_t)blk_off[s] * bb, d.H.val, (size_t)d.H.nnzb * bb * sizeof(double),
                                  cudaMemcpyDeviceToDevice, st));
    }
    row_ptr = rp;
    col_idx = ci;
    colour = co;
    sign = sg;
    Hval = hv;
    Pout = nullptr;  // each system's blocks are written straight into its own P_val
  }

  // ------------------------------------------------------------------ set-up
  int32_t *brow, *trans, *cnt, *nblk, *done, *misc, *pcount, *pstart, *bpr, *pr_c, *ccount, *coff, *cfill;
  double* isq;
  CSS_TRY(ws_get(ctx, "brow", nnzb, &brow));
  CSS_TRY(ws_get(ctx, "trans", nnzb, &trans));
  CSS_TRY(ws_get(ctx, "cnt", n_col, &cnt));
  CSS_TRY(ws_get(ctx, "nblk", n_col, &nblk));
  CSS_TRY(ws_get(ctx, "done", n_col, &done));
  CSS_TRY(ws_get(ctx, "isq", n_col, &isq));
  CSS_TRY(ws_get(ctx, "misc", 64, &misc));
  CSS_TRY(ws_get(ctx, "pcount", n_brow + 1, &pcount));
  CSS_TRY(ws_get(ctx, "pstart", n_brow + 1, &pstart));
  CSS_TRY(ws_get(ctx, "bpr", nnzb, &bpr));
  CSS_TRY(ws_get(ctx, "ccount", n_col + 1, &ccount));
  CSS_TRY(ws_get(ctx, "coff", n_col + 1, &coff));
  CSS_TRY(ws_get(ctx, "cfill", n_col + 1, &cfill));
  CSS_CU(ctx, cudaMemsetAsync(misc, 0, 64 * sizeof(int32_t), st));
  CSS_CU(ctx, cudaMemsetAsync(cnt, 0, n_col * sizeof(int32_t), st));
  CSS_CU(ctx, cudaMemsetAsync(done, 0, n_col * sizeof(int32_t), st));
  CSS_CU(ctx, cudaMemsetAsync(ccount, 0, (n_col + 1) * sizeof(int32_t), st));
  CSS_CU(ctx, cudaMemsetAsync(cfill, 0, (n_col + 1) * sizeof(int32_t), st));
  const unsigned gb = (unsigned)css_ceil_div(n_brow, T);
  k_rows<<<gb, T, 0, st>>>(n_brow, row_ptr, col_idx, colour, n_col, brow, trans, cnt, misc + 1, misc, partial ? 1 : 0);
  CSS_LAUNCHED(ctx);
  k_inv_sqrt<<<(unsigned)css_ceil_div(n_col, T), T, 0, st>>>(n_col, cnt, isq, nblk, done, m);
  CSS_LAUNCHED(ctx);
  k_pair_count<<<gb, T, 0, st>>>(n_brow, row_ptr, col_idx, colour, pcount);
  CSS_LAUNCHED(ctx);
  CSS_TRY(css_scan_i32(ctx, pcount, pstart, n_brow, st));
  int32_t* hb;
  CSS_TRY(css_pinned(ctx, sizeof(int64_t) * (n_col + 8) + 256, (void**)&hb));
  CSS_CU(ctx, cudaMemcpyAsync(hb, misc, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CSS_CU(ctx, cudaMemcpyAsync(hb + 2, pstart + n_brow, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CSS_CU(ctx, cudaStreamSynchronize(st));
  if (hb[0] & ERR_COLOUR) return css_set_arg_error(ctx, "css_density: colour outside [0, n_colours)");
  if (hb[0] & ERR_PATTERN)
    return css_set_arg_error(ctx, "css_density: pattern not symmetric, column out of range or diagonal missing");
  const int32_t max_row = hb[1];
  const int64_t n_pairs = hb[2];
  int32_t *pair_I, *pair_c, *perm, *pob;
  CSS_TRY(ws_get(ctx, "pr_c", n_pairs + 1, &pr_c));
  CSS_TRY(ws_get(ctx, "perm", n_pairs + 1, &perm));
  CSS_TRY(ws_get(ctx, "pair_I", n_pairs + 1, &pair_I));
  CSS_TRY(ws_get(ctx, "pair_c", n_pairs + 1, &pair_c));
  CSS_TRY(ws_get(ctx, "pob", nnzb, &pob));
  k_pair_fill<<<gb, T, 0, st>>>(n_brow, row_ptr, col_idx, colour, pstart, pr_c, bpr, ccount);
  CSS_LAUNCHED(ctx);
  CSS_TRY(css_scan_i32(ctx, ccount, coff, n_col, st));
  k_pair_place<<<gb, T, 0, st>>>(n_brow, pstart, pr_c, coff, cfill, perm, pair_I, pair_c);
  CSS_LAUNCHED(ctx);
  k_pob<<<(unsigned)css_ceil_div(nnzb, T), T, 0, st>>>(nnzb, bpr, perm, pob);
  CSS_LAUNCHED(ctx);
  std::vector<int64_t> pair_off_h(n_col + 1);
  {
    CSS_CU(ctx, cudaMemcpyAsync(hb, coff, sizeof(int32_t) * (n_col + 1), cudaMemcpyDeviceToHost, st));
    CSS_CU(ctx, cudaStreamSynchronize(st));
    for (int32_t c = 0; c <= n_col; ++c) pair_off_h[c] = hb[c];
  }
  const void* Hv = nullptr;
  const void* Hlo = nullptr;
  const void* Htc = nullptr;
  const void* Hd3 = nullptr;
  const void* Hdup = nullptr;
  const void* Hlodup = nullptr;
  const bool use_tc = (prec == CSS_MIXED_3XTF32 || ctx->hv_tc) && css_hv_tc_supported(f32, b, max_row);
  if (prec == CSS_MIXED_3XTF32 && !use_tc) {
    ctx->last_error = "css_density: CSS_MIXED_3XTF32 needs 17 <= b <= 24 (and rows of at most 128 blocks)";
    return CSS_ERR_UNSUPPORTED;
  }
  const bool use_split = prec == CSS_FP64_SPLIT;
  if (use_split && !css_spmm_split_supported(b)) {
    ctx->last_error = "css_density: CSS_FP64_SPLIT needs b = 6 or b = 23";
    return CSS_ERR_UNSUPPORTED;
  }
  // FP32 with b = 6 or 23: the exact-width H * V unless a padded variant is asked for
  const bool use_dup = !use_tc && ctx->spmm_variant < 0 && css_spmm_dup_supported(f32, b);
  const void* Hsplit = nullptr;
  if (use_tc)
    CSS_TRY(css_hv_tc_prepare(ctx, b, n_brow, nnzb, row_ptr, col_idx, Hval, &Htc, &Hd3, st));
  else if (use_split)
    CSS_TRY(css_spmm_split_prepare(ctx, b, nnzb, Hval, &Hsplit, st));
  else if (use_dup)
    CSS_TRY(css_spmm_dup_prepare(ctx, b, n_brow, nnzb, row_ptr, col_idx, Hval, &Hdup, &Hlodup, st));
  else
    CSS_TRY(css_spmm_prepare(ctx, f32, b, n_brow, nnzb, row_ptr, col_idx, Hval, &Hv, &Hlo, st));
  tm.mark();  // 1

  // ----------------------------------------------------------- memory plan
  const size_t s_vec = f32 ? 4 : 8;
  double *Ablk, *Bblk, *Bprev, *X;
  CSS_TRY(ws_get(ctx, "Ablk", (size_t)n_col * m * bb, &Ablk));
  CSS_TRY(ws_get(ctx, "Bblk", (size_t)n_col * m * bb, &Bblk));
  CSS_TRY(ws_get(ctx, "Bprev", (size_t)n_col * bb, &Bprev));
  CSS_TRY(ws_get(ctx, "X", (size_t)n_pairs * bb, &X));
  void* Qs = nullptr;
  if (!two_pass && !ritz_only) CSS_TRY(css_ws(ctx, "Qs", (size_t)n_pairs * m * bb * s_vec, &Qs));
  // eigen workspace (all colours at once)
  EigArgs ea;
  ea.n_col = n_col;
  ea.b = b;
  ea.m = m;
  ea.Ablk = Ablk;
  ea.Bblk = Bblk;
  ea.nblk = nblk;
  ea.cnt = cnt;
  ea.gid = colour_ids;
  ea.rcap = nmax * (nmax / b + 2);
  CSS_TRY(ws_get(ctx, "e_AB", (size_t)n_col * nmax * (2 * b + 1), &ea.AB));
  CSS_TRY(ws_get(ctx, "e_RV", (size_t)n_col * ea.rcap * b, &ea.RV));
  CSS_TRY(ws_get(ctx, "e_RT", (size_t)n_col * ea.rcap, &ea.RT));
  CSS_TRY(ws_get(ctx, "e_RR0", (size_t)n_col * ea.rcap, &ea.RR0));
  CSS_TRY(ws_get(ctx, "e_so", (size_t)n_col * (nmax + 1), &ea.sweep_off));
  CSS_TRY(ws_get(ctx, "e_d", (size_t)n_col * nmax, &ea.d));
  CSS_TRY(ws_get(ctx, "e_e", (size_t)n_col * nmax, &ea.e));
  CSS_TRY(ws_get(ctx, "e_l32", (size_t)n_col * nmax, &ea.lam32));
  CSS_TRY(ws_get(ctx, "e_tn", (size_t)n_col, &ea.tnorm));
  CSS_TRY(ws_get(ctx, "e_U", (size_t)n_col * nmax * nmax, &ea.U));
  CSS_TRY(ws_get(ctx, "e_F", (size_t)n_col * 5 * nmax * nmax, &ea.F));
  CSS_TRY(ws_get(ctx, "e_lam", (size_t)n_col * nmax, &ea.lam));
  CSS_TRY(ws_get(ctx, "e_X0", (size_t)n_col * nmax * b, &ea.X0));
  CSS_TRY(ws_get(ctx, "e_Y", (size_t)n_col * nmax * b, &ea.Y));
  CSS_TRY(ws_get(ctx, "e_w", (size_t)n_col * nmax, &ea.wgt));
  CSS_TRY(ws_get(ctx, "e_st", (size_t)n_col, &ea.status));
  CSS_TRY(ws_get(ctx, "e_flag", (size_t)n_col * nmax, &ea.flag));
  double* Z;
  CSS_TRY(ws_get(ctx, "Z", (size_t)n_col * nmax * b, &Z));
  // Krylov vectors.  The combined matrix of a batch is block-diagonal by system, so each
  // system's colours are run on that system's rows only (per-system passes); the blocks are
  // sized for the largest system, with as many of its colours per pass as memory allows.
  int64_t Nmax = 0;
  int32_t ncmax = 0;
  for (int32_t s = 0; s < n_sys; ++s) {
    Nmax = std::max(Nmax, (int64_t)sys[s].H.n_brow * b);
    ncmax = std::max(ncmax, sys[s].n_colours);
  }
  size_t free_b = 0, total_b = 0;
  CSS_CU(ctx, cudaMemGetInfo(&free_b, &total_b));
  int32_t ncb = ncmax;
  auto vec_need = [&](int32_t k) -> size_t {
    const int32_t ws = (int32_t)css_ceil_div((int64_t)k * b, 8) * 8;
    return 3 * (size_t)Nmax * ws * s_vec + css_lanczos_part_doubles(Nmax, b, k) * 8 * 2 +
           css_lanczos_small_doubles(b, k) * 8;
  };
  const size_t reserve = (size_t)2 << 30;
  while (ncb > 1 && vec_need(ncb) + reserve > free_b) ncb = (ncb + 1) / 2;
  const int32_t ws = (int32_t)css_ceil_div((int64_t)ncb * b, 8) * 8;
  void *Q0, *Q1, *Wv;
  double *part, *small;
  CSS_TRY(css_ws(ctx, "Q0", (size_t)Nmax * ws * s_vec, &Q0));
  CSS_TRY(css_ws(ctx, "Q1", (size_t)Nmax * ws * s_vec, &Q1));
  CSS_TRY(css_ws(ctx, "W", (size_t)Nmax * ws * s_vec, &Wv));
  CSS_TRY(ws_get(ctx, "lz_part", css_lanczos_part_doubles(Nmax, b, ncb) * 2, &part));
  CSS_TRY(ws_get(ctx, "lz_small", css_lanczos_small_doubles(b, ncb), &small));

  LzArgs la;
  la.fp32 = f32;
  la.n_brow = n_brow;
  la.b = b;
  la.m = m;
  la.row_ptr = row_ptr;
  la.col_idx = col_idx;
  la.Hval = Hv;
  la.Hlo_diag = Hlo;
  la.Hdup = Hdup;
  la.Hlo_dup = Hlodup;
  la.Hsplit = Hsplit;
  la.use_tc = use_tc;
  la.tc_H = Htc;
  la.tc_Hd3 = Hd3;
  la.max_row_blocks = max_row;
  la.colour = colour;
  la.sign = sign;
  la.inv_sqrt_cnt = isq;
  la.Q0 = Q0;
  la.Q1 = Q1;
  la.W = Wv;
  la.ws = ws;
  la.Ablk = Ablk;
  la.Bblk = Bblk;
  la.Bblk_prev = Bprev;
  la.nblk = nblk;
  la.done = done;
  la.part = part;
  la.small = small;
  la.tau = f32 ? 1e-5 : 1e-10;
  la.shift_rel = f32 ? 1e-5 : 1e-12;
  // FP32 Krylov vectors lose local orthogonality at the FP32 level, which biases the trace of
  // the reconstructed P; the local reorthogonalisation pass removes that bias
  la.flags = f32 ? (flags | CSS_REORTH_LOCAL) : flags;
  la.Qs = Qs;
  la.X = X;
  la.Yfull = yfull;
  la.ldy = ldy;
  la.Z = Z;
  la.ldz = nmax;
  la.pair_I = pair_I;
  la.pair_c = pair_c;
  la.pair_off_h = pair_off_h.data();
  // timing: two events per step of every pass of the one-stream path, read after the phase
  int32_t n_pass = 0;
  for (int32_t s = 0; s < n_sys; ++s) n_pass += (int32_t)css_ceil_div(col_off[s + 1] - col_off[s], ncb);
  int64_t n_spmm = 0;
  double spmm_ms = 0.0, rows_ms = 0.0;
  int64_t n_rows = 0;
  const int32_t BMh = css_spmm_bm(b);
  const size_t dup_row = (size_t)b * (b + (b & 1)) * 4;  // bytes of one row's low-part block (exact width)
  // A batch of systems runs its per-system passes concurrently on up to kSide side streams, each
  // with its own Krylov workspace (the passes of different systems touch disjoint rows, colours
  // and sampled pairs); the call's stream waits for all of them before the eigen stage.  The
  // tensor-core H*V keeps one schedule per call and the split-FP64 H*V one split copy of V, so
  // with them the passes run in turn.
  constexpr int kSide = 8;
  int nside = (n_sys > 1 && !use_tc && !use_split) ? std::min(n_sys, kSide) : 0;
  if (nside > 0) {
    // each side stream needs one more Krylov set; take only as many as fit beside the
    // reserve (sets already held from an earlier call count as free)
    size_t free2 = 0, total2 = 0, held = 0;
    CSS_CU(ctx, cudaMemGetInfo(&free2, &total2));
    static const char* const kSideNames[] = {"sQ0_", "sQ1_", "sW_", "spart_", "ssmall_"};
    for (auto& kv : ctx->bufs)
      for (const char* pre : kSideNames)
        if (kv.first.rfind(pre, 0) == 0) held += kv.second.bytes;
    const size_t avail = free2 + held > reserve ? free2 + held - reserve : 0;
    nside = (int)std::min<size_t>((size_t)nside, avail / vec_need(ncb));
    if (nside < 2) nside = 0;
  }
  struct SideWs {
    void *Q0, *Q1, *W;
    double *part, *small;
  };
  std::vector<SideWs> sws(nside);
  if (nside > 0) {
    while ((int)ctx->side.size() < nside) {
      cudaStream_t s2;
      CSS_CU(ctx, cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
      ctx->side.push_back(s2);
    }
    while ((int)ctx->side_ev.size() < nside + 1) {
      cudaEvent_t e2;
      CSS_CU(ctx, cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
      ctx->side_ev.push_back(e2);
    }
    for (int k = 0; k < nside; ++k) {
      char nm[32];
      snprintf(nm, sizeof(nm), "sQ0_%d", k);
      CSS_TRY(css_ws(ctx, nm, (size_t)Nmax * ws * s_vec, &sws[k].Q0));
      snprintf(nm, sizeof(nm), "sQ1_%d", k);
      CSS_TRY(css_ws(ctx, nm, (size_t)Nmax * ws * s_vec, &sws[k].Q1));
      snprintf(nm, sizeof(nm), "sW_%d", k);
      CSS_TRY(css_ws(ctx, nm, (size_t)Nmax * ws * s_vec, &sws[k].W));
      snprintf(nm, sizeof(nm), "spart_%d", k);
      CSS_TRY(ws_get(ctx, nm, css_lanczos_part_doubles(Nmax, b, ncb) * 2, &sws[k].part));
      snprintf(nm, sizeof(nm), "ssmall_%d", k);
      CSS_TRY(ws_get(ctx, nm, css_lanczos_small_doubles(b, ncb), &sws[k].small));
    }
  }
  // systems by decreasing size, dealt round-robin to the side streams
  std::vector<int32_t> sys_order(n_sys);
  for (int32_t s = 0; s < n_sys; ++s) sys_order[s] = s;
  std::stable_sort(sys_order.begin(), sys_order.end(),
                   [&](int32_t x, int32_t y) { return sys[x].H.n_brow > sys[y].H.n_brow; });
  // tune == true: only choose the H * V launch variant of every pass (tuning new shapes), so that
  // the passes themselves can then be captured
  auto run_batches = [&](int mode, bool tune, cudaStream_t s0) -> css_status {
    la.mode = mode;
    if (nside > 0) {
      if (!tune) {
        CSS_CU(ctx, cudaEventRecord(ctx->side_ev[nside], s0));
        for (int k = 0; k < nside; ++k) CSS_CU(ctx, cudaStreamWaitEvent(ctx->side[k], ctx->side_ev[nside], 0));
      }
      css_status rs = CSS_OK;
      for (int32_t i = 0; i < n_sys; ++i) {
        const int32_t s = sys_order[i];
        const int k = i % nside;
        LzArgs lb = la;
        lb.Q0 = sws[k].Q0;
        lb.Q1 = sws[k].Q1;
        lb.W = sws[k].W;
        lb.part = sws[k].part;
        lb.small = sws[k].small;
        lb.row0 = row_off[s];
        lb.n_brow = sys[s].H.n_brow;
        lb.row_ptr = row_ptr + row_off[s];
        lb.colour = colour + row_off[s];
        lb.sign = sign + (size_t)row_off[s] * b;
        lb.Hlo_diag = Hlo ? (const void*)((const char*)Hlo + (size_t)row_off[s] * BMh * BMh * s_vec) : nullptr;
        lb.Hlo_dup = Hlodup ? (const void*)((const char*)Hlodup + (size_t)row_off[s] * dup_row) : nullptr;
        lb.ev_spmm = nullptr;
        for (int32_t cb0 = col_off[s]; cb0 < col_off[s + 1] && rs == CSS_OK; cb0 += ncb) {
          lb.cb0 = cb0;
          lb.ncb = min(ncb, col_off[s + 1] - cb0);
          lb.w = lb.ncb * b;
          rs = tune ? css_lanczos_tune(ctx, lb, s0) : css_lanczos_pass(ctx, lb, ctx->side[k]);
        }
        if (rs != CSS_OK) break;
      }
      if (tune) return rs;
      // joined on every path, so that no side stream still writes the workspace after return
      for (int k = 0; k < nside; ++k) {
        CSS_CU(ctx, cudaEventRecord(ctx->side_ev[k], ctx->side[k]));
        CSS_CU(ctx, cudaStreamWaitEvent(s0, ctx->side_ev[k], 0));
      }
      return rs;
    }
    int32_t p = 0;
    for (int32_t s = 0; s < n_sys; ++s) {
      la.row0 = row_off[s];
      la.n_brow = sys[s].H.n_brow;
      la.row_ptr = row_ptr + row_off[s];
      la.colour = colour + row_off[s];
      la.sign = sign + (size_t)row_off[s] * b;
      la.Hlo_diag = Hlo ? (const void*)((const char*)Hlo + (size_t)row_off[s] * BMh * BMh * s_vec) : nullptr;
      la.Hlo_dup = Hlodup ? (const void*)((const char*)Hlodup + (size_t)row_off[s] * dup_row) : nullptr;
      for (int32_t cb0 = col_off[s]; cb0 < col_off[s + 1]; cb0 += ncb, ++p) {
        la.cb0 = cb0;
        la.ncb = min(ncb, col_off[s + 1] - cb0);
        la.w = la.ncb * b;
        la.ev_spmm = (ctx->timing && !tune) ? ctx->lz_ev.data() + (size_t)p * 2 * m : nullptr;
        CSS_TRY(tune ? css_lanczos_tune(ctx, la, s0) : css_lanczos_pass(ctx, la, s0));
      }
    }
    return CSS_OK;
  };
  // H * V times and the row work between them, from the events of the one-stream path
  auto read_timing = [&]() -> css_status {
    if (!ctx->timing || nside > 0) return CSS_OK;
    CSS_CU(ctx, cudaStreamSynchronize(st));
    for (int32_t p = 0; p < n_pass; ++p) {
      const cudaEvent_t* e = ctx->lz_ev.data() + (size_t)p * 2 * m;
      for (int32_t j = 0; j < m; ++j) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, e[2 * j], e[2 * j + 1]) == cudaSuccess) {
          spmm_ms += t;
          ++n_spmm;
        }
        // the row work of step j: from the end of its H * V to the start of the next one
        if (j + 1 < m && cudaEventElapsedTime(&t, e[2 * j + 1], e[2 * j + 2]) == cudaSuccess) {
          rows_ms += t;
          ++n_rows;
        }
      }
    }
    cudaGetLastError();  // steps a breakdown skipped leave unrecorded events
    return CSS_OK;
  };
  // The block-Lanczos phase: every pass of every system (on the side streams of a batch) is
  // captured on the context's capture stream into one CUDA graph, which replaces the previous
  // call's graph of the same mode in place when the launch sequence has the same shape (else it is
  // instantiated anew), and launched at once on the call's stream: by default for a single system,
  // on request for a batch (ctx->graph).  Not when the caller's stream is itself being captured:
  // the kernels then go into the caller's graph one by one.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CSS_CU(ctx, cudaStreamIsCapturing(st, &cap));
  const bool use_graph = (ctx->graph == 1 || (ctx->graph < 0 && n_sys == 1)) && cap == cudaStreamCaptureStatusNone;
  if (use_graph && !ctx->cap_stream) CSS_CU(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  auto run_lanczos = [&](int mode) -> css_status {
    while (ctx->timing && nside == 0 && ctx->lz_ev.size() < 2 * (size_t)m * n_pass) {
      cudaEvent_t e = nullptr;
      CSS_CU(ctx, cudaEventCreate(&e));
      ctx->lz_ev.push_back(e);
    }
    if (!use_graph) {
      CSS_TRY(run_batches(mode, false, st));
      return read_timing();
    }
    CSS_TRY(run_batches(mode, true, st));
    CSS_CU(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed));
    const css_status rs = run_batches(mode, false, ctx->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &g);
    if (rs != CSS_OK || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      if (rs != CSS_OK) return rs;
      return css_set_cuda_error(ctx, ce, "cudaStreamEndCapture (block-Lanczos graph)", __FILE__, __LINE__);
    }
    cudaGraphExec_t& ex = ctx->lz_exec[mode];
    if (ex) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(ex, g, &info) == cudaSuccess) {
        ++ctx->graph_updates;
      } else {
        cudaGetLastError();
        cudaGraphExecDestroy(ex);
        ex = nullptr;
      }
    }
    cudaError_t ie = cudaSuccess;
    if (!ex) {
      ie = cudaGraphInstantiate(&ex, g, 0);
      if (ie == cudaSuccess) ++ctx->graph_instantiations;
      else ex = nullptr;
    }
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return css_set_cuda_error(ctx, ie, "cudaGraphInstantiate (block-Lanczos graph)", __FILE__, __LINE__);
    CSS_CU(ctx, cudaGraphLaunch(ex, st));
    ++ctx->graph_launches;
    return read_timing();
  };
  CSS_TRY(run_lanczos((two_pass || ritz_only) ? 0 : 1));
  tm.mark();  // 2

  // ---------------------------------------------------------- eigen + mu + Z
  CSS_TRY(css_eigen_ritz(ctx, ea, st));
  tm.mark();  // 3
  if (ritz_only) {  // Ritz values and weights only (css_ritz); mu, Z and P are not computed
    k_count_breakdown<<<(unsigned)css_ceil_div(n_col, T), T, 0, st>>>(n_col, m, nblk, cnt, misc + 16);
    CSS_LAUNCHED(ctx);
    k_status_or<<<(unsigned)css_ceil_div(n_col, T), T, 0, st>>>(n_col, ea.status, misc + 17);
    CSS_LAUNCHED(ctx);
    int32_t* hm;
    CSS_TRY(css_pinned(ctx, 64 * sizeof(int32_t), (void**)&hm));
    CSS_CU(ctx, cudaMemcpyAsync(hm, misc + 16, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CSS_CU(ctx, cudaStreamSynchronize(st));
    ctx->last_lam = ea.lam;
    ctx->last_wgt = ea.wgt;
    ctx->last_nblk = nblk;
    ctx->last_ncol = n_col;
    ctx->last_b = b;
    ctx->last_nmax = nmax;
    ctx->last_A = Ablk;
    ctx->last_B = Bblk;
    ctx->last_m = m;
    ctx->info.n_colours = n_col;
    ctx->info.n_breakdown = hm[0];
    const int32_t st_bits = hm[1];
    if (use_tc) CSS_TRY(css_hv_tc_check(ctx, st));
    if (use_dup || use_split) CSS_TRY(css_spmm_dup_check(ctx, st));
    if (st_bits & 2) {
      ctx->last_error = "css_density: a wait between pipelined band-reduction sweeps timed out";
      return CSS_ERR_TIMEOUT;
    }
    return hm[0] > 0 ? CSS_WARN_BREAKDOWN : CSS_OK;
  }
  double *dmu, *dkT, *dhalf, *dmu_in, *dtol, *mupart;
  int32_t* dsolve;
  unsigned* bar;
  CSS_TRY(ws_get(ctx, "mu", n_sys, &dmu));
  CSS_TRY(ws_get(ctx, "kT", n_sys, &dkT));
  CSS_TRY(ws_get(ctx, "half_ne", n_sys, &dhalf));
  CSS_TRY(ws_get(ctx, "mu_in", n_sys, &dmu_in));
  CSS_TRY(ws_get(ctx, "ne_tol", n_sys, &dtol));
  CSS_TRY(ws_get(ctx, "solve", n_sys, &dsolve));
  CSS_TRY(ws_get(ctx, "bar", 8, &bar));
  {
    double* hp;
    CSS_TRY(css_pinned(ctx, sizeof(double) * 5 * n_sys + 256, (void**)&hp));
    for (int32_t s = 0; s < n_sys; ++s) {
      hp[s] = sys[s].fermi.kT;
      hp[n_sys + s] = 0.5 * sys[s].fermi.n_elec;
      hp[2 * n_sys + s] = sys[s].fermi.mu;
      // no chemical potential for the inverse square root of an overlap matrix
      ((int32_t*)(hp + 3 * n_sys))[s] = (sys[s].fermi.solve_mu && !(flags & CSS_INV_SQRT)) ? 1 : 0;
      const double tl = sys[s].fermi.ne_tol;
      hp[4 * n_sys + s] = tl > 0.0 ? tl : 1e-4 * std::max(1.0, 0.5 * sys[s].fermi.n_elec);
    }
    CSS_CU(ctx, cudaMemcpyAsync(dtol, hp + 4 * n_sys, sizeof(double) * n_sys, cudaMemcpyHostToDevice, st));
    CSS_CU(ctx, cudaMemcpyAsync(dkT, hp, sizeof(double) * n_sys, cudaMemcpyHostToDevice, st));
    CSS_CU(ctx, cudaMemcpyAsync(dhalf, hp + n_sys, sizeof(double) * n_sys, cudaMemcpyHostToDevice, st));
    CSS_CU(ctx, cudaMemcpyAsync(dmu_in, hp + 2 * n_sys, sizeof(double) * n_sys, cudaMemcpyHostToDevice, st));
    CSS_CU(ctx, cudaMemcpyAsync(dsolve, hp + 3 * n_sys, sizeof(int32_t) * n_sys, cudaMemcpyHostToDevice, st));
    CSS_CU(ctx, cudaMemsetAsync(bar, 0, 8 * sizeof(unsigned), st));
    CSS_CU(ctx, cudaStreamSynchronize(st));  // the pinned staging is reused below
  }
  int occ = 0;
  CSS_CU(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mu, MU_T, 0));
  unsigned G = (unsigned)std::max(1, std::min(ctx->n_sm * std::max(occ, 1), std::max(n_col, 1)));
  if (G > (unsigned)ctx->n_sm) G = (unsigned)ctx->n_sm;
  CSS_TRY(ws_get(ctx, "mu_part", (size_t)4 * n_sys * G + 16, &mupart));  // two buffers of [2][n_sys][G]
  {
    int32_t n_sys_ = n_sys, n_col_ = n_col, nmax_ = nmax, b_ = b;
    const int32_t* nblk_ = nblk;
    const int32_t* soc_ = sys_of_colour;
    const double* lam_ = ea.lam;
    const double* w_ = ea.wgt;
    const double* kT_ = dkT;
    const double* h_ = dhalf;
    const double* tl_ = dtol;
    const int32_t* sv_ = dsolve;
    const double* mi_ = dmu_in;
    double* mo_ = dmu;
    double* pp_ = mupart;
    unsigned* bar_ = bar;
    int32_t* err_ = misc + 8;
    int32_t extra_ = ctx->test_mu_barrier_extra;
    void* args[] = {&n_sys_, &n_col_, &nmax_, &nblk_, &b_, &soc_, &lam_, &w_, &kT_, &h_, &tl_, &sv_, &mi_, &mo_, &pp_,
                    &bar_, &err_, &extra_};
    CSS_CU(ctx, cudaLaunchCooperativeKernel((void*)k_mu, dim3(G), dim3(MU_T), args, 0, st));
    ++ctx->kernel_launches;
  }
  tm.mark();  // 4
  CSS_TRY(css_eigen_z(ctx, ea, sys_of_colour, dmu, dkT, Z, st, ((flags & CSS_ENERGY_WEIGHTED) ? 1 : 0) |
                                                                     ((flags & CSS_INV_SQRT) ? 2 : 0)));

  // --------------------------------------------------------- reconstruction
  if (two_pass) {
    CSS_CU(ctx, cudaMemsetAsync(X, 0, (size_t)n_pairs * bb * sizeof(double), st));
    CSS_CU(ctx, cudaMemsetAsync(done, 0, n_col * sizeof(int32_t), st));
    k_inv_sqrt<<<(unsigned)css_ceil_div(n_col, T), T, 0, st>>>(n_col, cnt, isq, nblk, done, m);
    CSS_LAUNCHED(ctx);
    CSS_TRY(run_lanczos(2));
  } else {
    float *zh = nullptr, *zl = nullptr;
    if (f32) {
      CSS_TRY(ws_get(ctx, "zh", (size_t)n_col * nmax * b, &zh));
      CSS_TRY(ws_get(ctx, "zl", (size_t)n_col * nmax * b, &zl));
      k_zsplit<<<(unsigned)css_ceil_div((int64_t)n_col * nmax * b, T), T, 0, st>>>((int64_t)n_col * nmax * b, Z, zh,
                                                                                   zl);
      CSS_LAUNCHED(ctx);
      const int32_t BPx = b <= 8 ? 8 : b <= 16 ? 16 : b <= 24 ? 24 : 32;
      const int32_t xp = 256 / ((BPx / 4) * (BPx / 4));
      int32_t* cta_off;
      CSS_TRY(ws_get(ctx, "x_cta", (size_t)n_col + 1, &cta_off));
      k_xtile_plan<<<1, 32, 0, st>>>(n_col, xp, coff, cta_off);
      CSS_LAUNCHED(ctx);
      const unsigned nct = (unsigned)(n_pairs / xp + n_col + 1);  // >= sum over colours of ceil(pairs / xp)
      auto launch_x = [&](auto kern) { kern<<<nct, 256, 0, st>>>(n_col, b, m, nmax, coff, cta_off, nblk,
                                                                 (const float*)Qs, zh, zl, X); };
      if (BPx == 8) launch_x(k_xtile<8>);
      else if (BPx == 16) launch_x(k_xtile<16>);
      else if (BPx == 24) launch_x(k_xtile<24>);
      else launch_x(k_xtile<32>);
    } else {
      k_xcompute<double><<<(unsigned)css_ceil_div(n_pairs * bb, T), T, 0, st>>>(n_pairs, b, m, nmax, pair_c, nblk,
                                                                                 (const double*)Qs, Z, nullptr,
                                                                                 nullptr, X);
    }
    CSS_LAUNCHED(ctx);
  }
  tm.mark();  // 5
  // ------------------------------------------------------------- extraction
  const int sym = (flags & CSS_SYMMETRIZE) ? 1 : 0;
  double* tpart;
  double* tout;
  const int64_t max_parts = css_ceil_div((int64_t)nnzb * bb, EX_T) + n_sys;
  CSS_TRY(ws_get(ctx, "tr_part", 2 * (size_t)max_parts, &tpart));
  CSS_TRY(ws_get(ctx, "tr_out", 2 * (size_t)n_sys + 2, &tout));
  for (int32_t s = 0; s < n_sys; ++s) {
    const int32_t k0 = blk_off[s], k1 = blk_off[s + 1];
    const int64_t nth = (int64_t)(k1 - k0) * bb;
    const unsigned blocks = (unsigned)css_ceil_div(nth, EX_T);
    double* out_p = (n_sys == 1) ? Pout : sys[s].P_val;
    k_extract<<<blocks, EX_T, 0, st>>>(k0, k1, b, k0, brow, col_idx, trans, pob, sign, X, Hval, sym, out_p, tpart);
    CSS_LAUNCHED(ctx);
    k_trace_sum<<<1, 1024, 0, st>>>((int32_t)blocks, tpart, tout + 2 * s);
    CSS_LAUNCHED(ctx);
  }
  k_count_breakdown<<<(unsigned)css_ceil_div(n_col, T), T, 0, st>>>(n_col, m, nblk, cnt, misc + 16);
  CSS_LAUNCHED(ctx);
  k_status_or<<<(unsigned)css_ceil_div(n_col, T), T, 0, st>>>(n_col, ea.status, misc + 17);
  CSS_LAUNCHED(ctx);
  tm.mark();  // 6
  // ------------------------------------------------------------ read back
  double* hres;
  CSS_TRY(css_pinned(ctx, sizeof(double) * (3 * n_sys + 16), (void**)&hres));
  CSS_CU(ctx, cudaMemcpyAsync(hres, tout, sizeof(double) * 2 * n_sys, cudaMemcpyDeviceToHost, st));
  CSS_CU(ctx, cudaMemcpyAsync(hres + 2 * n_sys, dmu, sizeof(double) * n_sys, cudaMemcpyDeviceToHost, st));
  CSS_CU(ctx, cudaMemcpyAsync(hres + 3 * n_sys, misc + 8, sizeof(int32_t) * 16, cudaMemcpyDeviceToHost, st));
  CSS_CU(ctx, cudaStreamSynchronize(st));
  const int32_t* hmisc = (const int32_t*)(hres + 3 * n_sys);
  const int32_t mu_err = hmisc[0];
  const int32_t n_break = hmisc[8];
  bool finite = true;
  for (int32_t s = 0; s < n_sys; ++s) {
    if (trP) trP[s] = hres[2 * s];
    if (trPH) trPH[s] = hres[2 * s + 1];
    if (mu_out) mu_out[s] = hres[2 * n_sys + s];
    finite = finite && std::isfinite(hres[2 * s]) && std::isfinite(hres[2 * s + 1]) &&
             std::isfinite(hres[2 * n_sys + s]);
  }
  ctx->last_lam = ea.lam;
  ctx->last_wgt = ea.wgt;
  ctx->last_nblk = nblk;
  ctx->last_ncol = n_col;
  ctx->last_b = b;
  ctx->last_nmax = nmax;
  ctx->last_A = Ablk;
  ctx->last_B = Bblk;
  ctx->last_m = m;
  ctx->info.n_colours = n_col;
  ctx->info.n_pairs = (int32_t)n_pairs;
  ctx->info.n_breakdown = n_break;
  ctx->info.m = m;
  ctx->info.spmm_launches = n_spmm;
  const int64_t wcols = (int64_t)std::min(ncb, n_col) * b;
  ctx->info.spmm_flops = 2.0 * nnzb * (double)bb * (double)wcols;
  ctx->info.spmm_bytes = (double)nnzb * bb * s_vec + 2.0 * (double)N * wcols * s_vec;
  ctx->info.ms_spmm = n_spmm ? spmm_ms / n_spmm : 0.0;
  ctx->info.ms_rows = n_rows ? rows_ms / n_rows : 0.0;
  if (ctx->timing) {
    ctx->info.ms_setup = tm.ms(0, 1);
    ctx->info.ms_lanczos = tm.ms(1, 2);
    ctx->info.ms_eigen = tm.ms(2, 3);
    ctx->info.ms_mu = tm.ms(3, 4);
    ctx->info.ms_extract = tm.ms(4, 6);
    ctx->info.ms_total = tm.ms(0, 6);
  }
  if (use_tc) CSS_TRY(css_hv_tc_check(ctx, st));
  if (use_dup || use_split) CSS_TRY(css_spmm_dup_check(ctx, st));
  if (mu_err) {
    ctx->last_error = "css_density: grid barrier of the mu bisection timed out";
    return CSS_ERR_TIMEOUT;
  }
  if (hmisc[9] & 2) {
    ctx->last_error = "css_density: a wait between pipelined band-reduction sweeps timed out";
    return CSS_ERR_TIMEOUT;
  }
  if (!finite) {
    ctx->last_error = "css_density: non-finite trace or mu";
    return CSS_ERR_NUMERIC;
  }
  return n_break > 0 ? CSS_WARN_BREAKDOWN : CSS_OK;
}


namespace {

__global__ void k_block_rows(int32_t n_brow, const int32_t* __restrict__ row_ptr, int32_t* __restrict__ brow) {
  const int32_t I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n_brow) return;
  for (int32_t p = row_ptr[I]; p < row_ptr[I + 1]; ++p) brow[p] = I;
}

// H'~_IJ = W[I rows][c(J) block] diag(o_J) on H's pattern, symmetrised with the transpose
// element W[J rows][c(I) block] diag(o_I) when sym; per-CTA partial sums of the trace
template <typename T>
__global__ void __launch_bounds__(EX_T) k_hp_extract(int32_t nnzb, int32_t b, const int32_t* __restrict__ brow,
                                                     const int32_t* __restrict__ col_idx,
                                                     const int32_t* __restrict__ colour, const int8_t* __restrict__ sign,
                                                     const T* __restrict__ Wm, int32_t ldy, int sym,
                                                     double* __restrict__ out, double* __restrict__ part) {
  __shared__ double r1[EX_T / 32];
  const int32_t bb = b * b;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double tp = 0.0;
  if (t < (int64_t)nnzb * bb) {
    const int32_t k = (int32_t)(t / bb), e = (int32_t)(t % bb), a = e / b, kk = e % b;
    const int32_t I = brow[k], J = col_idx[k];
    double v = (double)Wm[((size_t)I * b + a) * ldy + (size_t)colour[J] * b + kk] * (double)sign[(size_t)J * b + kk];
    if (sym) {
      const double w = (double)Wm[((size_t)J * b + kk) * ldy + (size_t)colour[I] * b + a] *
                       (double)sign[(size_t)I * b + a];
      v = 0.5 * (v + w);
    }
    out[t] = v;
    if (I == J && a == kk) tp = v;
  }
  for (int o = 16; o > 0; o >>= 1) tp += __shfl_xor_sync(0xffffffffu, tp, o);
  if ((threadIdx.x & 31) == 0) r1[threadIdx.x >> 5] = tp;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int i = 0; i < EX_T / 32; ++i) a += r1[i];
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = 0.0;
  }
}

// Mt[p] = M[trans[p]]^T: the transpose of a BSR matrix on a structurally symmetric pattern
__global__ void k_block_transpose(int32_t nnzb, int32_t b, const int32_t* __restrict__ trans,
                                  const double* __restrict__ M, double* __restrict__ Mt) {
  const int32_t bb = b * b;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nnzb * bb) return;
  const int32_t p = (int32_t)(t / bb), e = (int32_t)(t % bb), i = e / b, k = e % b;
  Mt[t] = M[(size_t)trans[p] * bb + k * b + i];
}

__global__ void k_fill(int32_t n, double v, double* __restrict__ x) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

// electron-count weights kappa[c][k] = YV[c][k] . Y[c][k] (0 past the colour's projected size)
__global__ void k_kappa(int32_t n_col, int32_t b, int32_t nmax, const int32_t* __restrict__ nblk,
                        const double* __restrict__ YV, const double* __restrict__ Y, double* __restrict__ kap) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n_col * nmax) return;
  const int32_t c = (int32_t)(t / nmax), k = (int32_t)(t % nmax);
  double s = 0.0;
  if (k < nblk[c] * b)
    for (int32_t a = 0; a < b; ++a) s = fma(YV[(size_t)t * b + a], Y[(size_t)t * b + a], s);
  kap[t] = s;
}

// per-CTA partial sums of Tr(rho H) over H's blocks and of Tr(rho S) over S's blocks; each S
// block is found in H's row by bisection (columns sorted), err = 1 when it is not there
__global__ void __launch_bounds__(EX_T) k_trace_hs(int64_t nh, int64_t ns, int32_t b, const double* __restrict__ P,
                                                   const double* __restrict__ Hval, const int32_t* __restrict__ h_row_ptr,
                                                   const int32_t* __restrict__ h_col_idx,
                                                   const int32_t* __restrict__ s_brow,
                                                   const int32_t* __restrict__ s_col_idx,
                                                   const double* __restrict__ Sval, double* __restrict__ part,
                                                   int32_t* __restrict__ err) {
  __shared__ double r1[EX_T / 32], r2[EX_T / 32];
  const int32_t bb = b * b;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double th = 0.0, ts = 0.0;
  if (t < nh) th = P[t] * Hval[t];
  if (t < ns) {
    const int32_t p = (int32_t)(t / bb), e = (int32_t)(t % bb);
    const int32_t I = s_brow[p], J = s_col_idx[p];
    int32_t lo = h_row_ptr[I], hi = h_row_ptr[I + 1] - 1, q = -1;
    while (lo <= hi) {
      const int32_t mid = (lo + hi) >> 1, v = h_col_idx[mid];
      if (v == J) {
        q = mid;
        break;
      }
      if (v < J) lo = mid + 1;
      else hi = mid - 1;
    }
    if (q >= 0) ts = P[(size_t)q * bb + e] * Sval[t];
    else atomicOr(err, 1);
  }
  for (int o = 16; o > 0; o >>= 1) {
    th += __shfl_xor_sync(0xffffffffu, th, o);
    ts += __shfl_xor_sync(0xffffffffu, ts, o);
  }
  if ((threadIdx.x & 31) == 0) {
    r1[threadIdx.x >> 5] = th;
    r2[threadIdx.x >> 5] = ts;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int i = 0; i < EX_T / 32; ++i) {
      x += r1[i];
      y += r2[i];
    }
    part[2 * blockIdx.x] = x;
    part[2 * blockIdx.x + 1] = y;
  }
}

}  // namespace

extern "C" {

css_status css_ritz(css_ctx* ctx, double* lam, double* wgt, int32_t* n_per, int64_t capacity, int32_t* n_colours) {
  if (!ctx || !n_colours) return css_set_arg_error(ctx, "css_ritz: null pointer");
  if (!ctx->last_lam) return css_set_arg_error(ctx, "css_ritz: no density has been computed");
  CSS_CU(ctx, cudaSetDevice(ctx->device));
  const int32_t nc = ctx->last_ncol, nmax = ctx->last_nmax;
  *n_colours = nc;
  if (!n_per) return CSS_OK;
  std::vector<int32_t> nb(nc);
  CSS_CU(ctx, cudaDeviceSynchronize());
  CSS_CU(ctx, cudaMemcpy(nb.data(), ctx->last_nblk, sizeof(int32_t) * nc, cudaMemcpyDeviceToHost));
  int64_t total = 0;
  for (int32_t c = 0; c < nc; ++c) {
    n_per[c] = nb[c] * ctx->last_b;
    total += n_per[c];
  }
  if (!lam || !wgt || capacity < total) return css_set_arg_error(ctx, "css_ritz: capacity too small");
  int64_t o = 0;
  for (int32_t c = 0; c < nc; ++c) {
    if (n_per[c] == 0) continue;
    CSS_CU(ctx, cudaMemcpy(lam + o, ctx->last_lam + (size_t)c * nmax, sizeof(double) * n_per[c], cudaMemcpyDeviceToHost));
    CSS_CU(ctx, cudaMemcpy(wgt + o, ctx->last_wgt + (size_t)c * nmax, sizeof(double) * n_per[c], cudaMemcpyDeviceToHost));
    o += n_per[c];
  }
  return CSS_OK;
}

css_status css_projected(css_ctx* ctx, double* A, double* B, int32_t* nblk, int64_t capacity, int32_t* n_colours,
                         int32_t* m, int32_t* b) {
  if (!ctx || !n_colours || !m || !b) return css_set_arg_error(ctx, "css_projected: null pointer");
  if (!ctx->last_A) return css_set_arg_error(ctx, "css_projected: no density has been computed");
  *n_colours = ctx->last_ncol;
  *m = ctx->last_m;
  *b = ctx->last_b;
  const int64_t need = (int64_t)ctx->last_ncol * ctx->last_m * ctx->last_b * ctx->last_b;
  if (!A || !B || !nblk || capacity < need) return css_set_arg_error(ctx, "css_projected: capacity too small");
  CSS_CU(ctx, cudaSetDevice(ctx->device));
  CSS_CU(ctx, cudaDeviceSynchronize());
  CSS_CU(ctx, cudaMemcpy(A, ctx->last_A, sizeof(double) * need, cudaMemcpyDeviceToHost));
  CSS_CU(ctx, cudaMemcpy(B, ctx->last_B, sizeof(double) * need, cudaMemcpyDeviceToHost));
  CSS_CU(ctx, cudaMemcpy(nblk, ctx->last_nblk, sizeof(int32_t) * ctx->last_ncol, cudaMemcpyDeviceToHost));
  return CSS_OK;
}

css_status css_eigen_blocks(css_ctx* ctx, int32_t n_col, int32_t b, int32_t m, const double* A, const double* B,
                            const int32_t* nblk, const int32_t* cnt, double mu, double kT, double* lam, double* wgt,
                            double* Z, void* stream) {
  if (!ctx || !A || !B || !nblk || !cnt || !lam || !wgt) return css_set_arg_error(ctx, "css_eigen_blocks: null pointer");
  if (n_col < 1 || b < 1 || b > CSS_MAX_B || m < 1 || (int64_t)m * b > 4096 || !(kT >= 0.0))
    return css_set_arg_error(ctx, "css_eigen_blocks: bad size or kT");
  CSS_CU(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t nmax = m * b;
  EigArgs ea;
  ea.n_col = n_col;
  ea.b = b;
  ea.m = m;
  ea.Ablk = A;
  ea.Bblk = B;
  ea.nblk = nblk;
  ea.cnt = cnt;
  ea.rcap = nmax * (nmax / b + 2);
  CSS_TRY(ws_get(ctx, "e_AB", (size_t)n_col * nmax * (2 * b + 1), &ea.AB));
  CSS_TRY(ws_get(ctx, "e_RV", (size_t)n_col * ea.rcap * b, &ea.RV));
  CSS_TRY(ws_get(ctx, "e_RT", (size_t)n_col * ea.rcap, &ea.RT));
  CSS_TRY(ws_get(ctx, "e_RR0", (size_t)n_col * ea.rcap, &ea.RR0));
  CSS_TRY(ws_get(ctx, "e_so", (size_t)n_col * (nmax + 1), &ea.sweep_off));
  CSS_TRY(ws_get(ctx, "e_d", (size_t)n_col * nmax, &ea.d));
  CSS_TRY(ws_get(ctx, "e_e", (size_t)n_col * nmax, &ea.e));
  CSS_TRY(ws_get(ctx, "e_l32", (size_t)n_col * nmax, &ea.lam32));
  CSS_TRY(ws_get(ctx, "e_tn", (size_t)n_col, &ea.tnorm));
  CSS_TRY(ws_get(ctx, "e_U", (size_t)n_col * nmax * nmax, &ea.U));
  CSS_TRY(ws_get(ctx, "e_F", (size_t)n_col * 5 * nmax * nmax, &ea.F));
  CSS_TRY(ws_get(ctx, "e_X0", (size_t)n_col * nmax * b, &ea.X0));
  CSS_TRY(ws_get(ctx, "e_Y", (size_t)n_col * nmax * b, &ea.Y));
  CSS_TRY(ws_get(ctx, "e_st", (size_t)n_col, &ea.status));
  CSS_TRY(ws_get(ctx, "e_flag", (size_t)n_col * nmax, &ea.flag));
  ea.lam = lam;
  ea.wgt = wgt;
  CSS_CU(ctx, cudaMemsetAsync(lam, 0, sizeof(double) * n_col * nmax, st));
  CSS_TRY(css_eigen_ritz(ctx, ea, st));
  if (Z) {
    int32_t* soc;
    double* par;
    CSS_TRY(ws_get(ctx, "eb_soc", n_col, &soc));
    CSS_TRY(ws_get(ctx, "eb_par", 2, &par));
    CSS_CU(ctx, cudaMemsetAsync(soc, 0, sizeof(int32_t) * n_col, st));
    double hp[2] = {mu, kT};
    CSS_CU(ctx, cudaMemcpyAsync(par, hp, sizeof(hp), cudaMemcpyHostToDevice, st));
    CSS_TRY(css_eigen_z(ctx, ea, soc, par, par + 1, Z, st));
  }
  CSS_CU(ctx, cudaStreamSynchronize(st));
  return CSS_OK;
}

css_status css_density(css_ctx* ctx, const css_bsr* H, const int32_t* colour, const int8_t* sign, int32_t n_colours,
                       const css_fermi* fermi, int32_t m, css_precision prec, uint32_t flags, double* P_val,
                       double* trP, double* trPH, double* mu_out, void* stream) {
  if (!ctx || !H || !fermi) return css_set_arg_error(ctx, "css_density: null pointer");
  CSS_CU(ctx, cudaSetDevice(ctx->device));
  css_sys_desc d{*H, colour, sign, n_colours, *fermi, P_val};
  return css_density_impl(ctx, 1, &d, m, prec, flags, trP, trPH, mu_out, (cudaStream_t)stream);
}

// colour'(J) = map[colour(J)]: the owned colours renumbered 0.. in increasing order, -1 for the rest
__global__ void k_colour_map(int32_t n, const int32_t* __restrict__ colour, int32_t n_col, const int32_t* __restrict__ map,
                             int32_t* __restrict__ out, int32_t* __restrict__ err) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t c = colour[i];
  if (c < 0 || c >= n_col) {
    atomicOr(err, 1);
    out[i] = -1;
    return;
  }
  out[i] = map[c];
}

css_status css_density_colours(css_ctx* ctx, const css_bsr* H, const int32_t* colour, const int8_t* sign,
                               int32_t n_colours, const uint8_t* owned, const css_fermi* fermi, int32_t m,
                               css_precision prec, uint32_t flags, double* P_val, double* trP, double* trPH,
                               void* stream) {
  if (!ctx || !H || !colour || !sign || !owned || !fermi || !P_val || n_colours < 1)
    return css_set_arg_error(ctx, "css_density_colours: null pointer or n_colours < 1");
  if (fermi->solve_mu) return css_set_arg_error(ctx, "css_density_colours: mu must be given (solve_mu = 0)");
  if (flags & CSS_SYMMETRIZE) return css_set_arg_error(ctx, "css_density_colours: the output is unsymmetrised");
  CSS_CU(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int32_t> map(n_colours);
  int32_t n_own = 0;
  for (int32_t c = 0; c < n_colours; ++c) map[c] = owned[c] ? n_own++ : -1;
  if (n_own < 1) return css_set_arg_error(ctx, "css_density_colours: no colour owned");
  int32_t *dmap, *dcol, *derr, *dids, *h;
  CSS_TRY(css_ws(ctx, "part_map", sizeof(int32_t) * (2 * (size_t)n_colours + 64), (void**)&dmap));
  CSS_TRY(css_ws(ctx, "part_colour", sizeof(int32_t) * H->n_brow, (void**)&dcol));
  derr = dmap + n_colours;
  dids = derr + 64;  // the owned colours' ids in the full numbering (their eigen-stage seeds)
  CSS_TRY(css_pinned(ctx, sizeof(int32_t) * (2 * (size_t)n_colours + 64), (void**)&h));
  std::memcpy(h, map.data(), sizeof(int32_t) * n_colours);
  for (int32_t c = 0, t = 0; c < n_colours; ++c)
    if (owned[c]) h[n_colours + 64 + t++] = c;
  CSS_CU(ctx, cudaMemcpyAsync(dmap, h, sizeof(int32_t) * n_colours, cudaMemcpyHostToDevice, st));
  CSS_CU(ctx, cudaMemcpyAsync(dids, h + n_colours + 64, sizeof(int32_t) * n_own, cudaMemcpyHostToDevice, st));
  CSS_CU(ctx, cudaMemsetAsync(derr, 0, sizeof(int32_t), st));
  k_colour_map<<<(unsigned)css_ceil_div(H->n_brow, 256), 256, 0, st>>>(H->n_brow, colour, n_colours, dmap, dcol, derr);
  CSS_LAUNCHED(ctx);
  CSS_CU(ctx, cudaMemcpyAsync(h + n_colours, derr, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CSS_CU(ctx, cudaStreamSynchronize(st));  // the pinned staging is reused below
  if (h[n_colours]) return css_set_arg_error(ctx, "css_density_colours: colour outside [0, n_colours)");
  css_sys_desc d{*H, dcol, sign, n_own, *fermi, P_val};
  double mu = 0.0;
  return css_density_impl(ctx, 1, &d, m, prec, flags, trP, trPH, &mu, st, nullptr, 0, true, dids);
}

css_status css_solve_mu(css_ctx* ctx, int32_t n_lists, const int32_t* n_per, const double* lam, const double* wgt,
                        double kT, double n_elec, double ne_tol, double* mu_out, void* stream) {
  if (!ctx || !n_per || !lam || !wgt || !mu_out || n_lists < 1)
    return css_set_arg_error(ctx, "css_solve_mu: null pointer or n_lists < 1");
  if (!(kT >= 0.0) || !std::isfinite(kT) || !std::isfinite(n_elec))
    return css_set_arg_error(ctx, "css_solve_mu: kT must be finite and >= 0, n_elec finite");
  CSS_CU(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  int64_t total = 0;
  int32_t nmax = 1;
  for (int32_t t = 0; t < n_lists; ++t) {
    if (n_per[t] < 0) return css_set_arg_error(ctx, "css_solve_mu: negative list length");
    total += n_per[t];
    nmax = std::max(nmax, n_per[t]);
  }
  // the lists as the colours of one system (stride nmax, block width 1), solved by the kernel
  // and the rule of css_density
  double *dl, *dw, *dpar, *dmu;
  int32_t *dn, *dsoc, *dsolve, *derr;
  unsigned* bar;
  const size_t nn = (size_t)n_lists * nmax;
  CSS_TRY(css_ws(ctx, "smu_lam", sizeof(double) * nn, (void**)&dl));
  CSS_TRY(css_ws(ctx, "smu_wgt", sizeof(double) * nn, (void**)&dw));
  CSS_TRY(css_ws(ctx, "smu_i", sizeof(int32_t) * (2 * (size_t)n_lists + 64), (void**)&dn));
  dsoc = dn + n_lists;
  dsolve = dsoc + n_lists;
  derr = dsolve + 8;
  bar = reinterpret_cast<unsigned*>(derr + 8);
  CSS_TRY(css_ws(ctx, "smu_d", sizeof(double) * 16, (void**)&dpar));
  dmu = dpar + 8;
  double* hp;
  const size_t hbytes = sizeof(double) * 2 * nn + sizeof(int32_t) * 2 * (size_t)n_lists + 256;
  CSS_TRY(css_pinned(ctx, hbytes, (void**)&hp));
  double* hl = hp;
  double* hw = hl + nn;
  int32_t* hi = reinterpret_cast<int32_t*>(hw + nn);
  double* hd = reinterpret_cast<double*>(hi + 2 * (size_t)n_lists + 2);
  size_t o = 0;
  for (int32_t t = 0; t < n_lists; ++t) {
    for (int32_t k = 0; k < nmax; ++k) {
      hl[(size_t)t * nmax + k] = k < n_per[t] ? lam[o + k] : 0.0;
      hw[(size_t)t * nmax + k] = k < n_per[t] ? wgt[o + k] : 0.0;
    }
    o += n_per[t];
    hi[t] = n_per[t];
    hi[n_lists + t] = 0;
  }
  hd[0] = kT;
  hd[1] = 0.5 * n_elec;
  hd[2] = ne_tol > 0.0 ? ne_tol : 1e-4 * std::max(1.0, 0.5 * n_elec);
  hd[3] = 0.0;
  CSS_CU(ctx, cudaMemcpyAsync(dl, hl, sizeof(double) * nn, cudaMemcpyHostToDevice, st));
  CSS_CU(ctx, cudaMemcpyAsync(dw, hw, sizeof(double) * nn, cudaMemcpyHostToDevice, st));
  CSS_CU(ctx, cudaMemcpyAsync(dn, hi, sizeof(int32_t) * 2 * (size_t)n_lists, cudaMemcpyHostToDevice, st));
  CSS_CU(ctx, cudaMemcpyAsync(dpar, hd, sizeof(double) * 4, cudaMemcpyHostToDevice, st));
  const int32_t one = 1;
  CSS_CU(ctx, cudaMemcpyAsync(dsolve, &one, sizeof(int32_t), cudaMemcpyHostToDevice, st));
  CSS_CU(ctx, cudaMemsetAsync(derr, 0, sizeof(int32_t) * 8 + 8 * sizeof(unsigned), st));
  int occ = 0;
  CSS_CU(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mu, MU_T, 0));
  unsigned G = (unsigned)std::max(1, std::min(ctx->n_sm * std::max(occ, 1), n_lists));
  if (G > (unsigned)ctx->n_sm) G = (unsigned)ctx->n_sm;
  double* mupart;
  CSS_TRY(css_ws(ctx, "smu_part", sizeof(double) * (4 * (size_t)G + 16), (void**)&mupart));
  {
    int32_t n_sys_ = 1, n_col_ = n_lists, nmax_ = nmax, b_ = 1, extra_ = 0;
    const int32_t* nblk_ = dn;
    const int32_t* soc_ = dsoc;
    const double* lam_ = dl;
    const double* w_ = dw;
    const double* kT_ = dpar;
    const double* h_ = dpar + 1;
    const double* tl_ = dpar + 2;
    const int32_t* sv_ = dsolve;
    const double* mi_ = dpar + 3;
    double* mo_ = dmu;
    double* pp_ = mupart;
    unsigned* bar_ = bar;
    int32_t* err_ = derr;
    void* args[] = {&n_sys_, &n_col_, &nmax_, &nblk_, &b_, &soc_, &lam_, &w_, &kT_, &h_, &tl_, &sv_, &mi_, &mo_, &pp_,
                    &bar_, &err_, &extra_};
    CSS_CU(ctx, cudaLaunchCooperativeKernel((void*)k_mu, dim3(G), dim3(MU_T), args, 0, st));
    ++ctx->kernel_launches;
  }
  CSS_CU(ctx, cudaMemcpyAsync(hd + 4, dmu, sizeof(double), cudaMemcpyDeviceToHost, st));
  CSS_CU(ctx, cudaMemcpyAsync(hi, derr, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CSS_CU(ctx, cudaStreamSynchronize(st));
  if (hi[0]) {
    ctx->last_error = "css_solve_mu: grid barrier of the mu bisection timed out";
    return CSS_ERR_TIMEOUT;
  }
  *mu_out = hd[4];
  return std::isfinite(*mu_out) ? CSS_OK : CSS_ERR_NUMERIC;
}

css_status css_density_batch(css_ctx* ctx, int32_t n_sys, const css_bsr* H, const int32_t* const* colour,
                             const int8_t* const* sign, const int32_t* n_colours, const css_fermi* fermi, int32_t m,
                             css_precision prec, uint32_t flags, double* const* P_val, double* trP, double* trPH,
                             double* mu_out, void* stream) {
  if (!ctx || !H || !colour || !sign || !n_colours || !fermi || !P_val || n_sys < 1)
    return css_set_arg_error(ctx, "css_density_batch: null pointer or n_sys < 1");
  CSS_CU(ctx, cudaSetDevice(ctx->device));
  std::vector<css_sys_desc> d(n_sys);
  for (int32_t s = 0; s < n_sys; ++s) d[s] = css_sys_desc{H[s], colour[s], sign[s], n_colours[s], fermi[s], P_val[s]};
  return css_density_impl(ctx, n_sys, d.data(), m, prec, flags, trP, trPH, mu_out, (cudaStream_t)stream);
}


css_status css_hprime(css_ctx* ctx, const css_bsr* S, const css_bsr* H, const int32_t* colour, const int8_t* sign,
                      int32_t n_colours, int32_t m, css_precision prec, uint32_t flags, double* Sinv_val,
                      double* Hp_val, double* trHp, void* stream) {
  if (!ctx || !S || !H || !Sinv_val || !Hp_val) return css_set_arg_error(ctx, "css_hprime: null pointer");
  if (S->n_brow != H->n_brow || S->b != H->b || H->nnzb < H->n_brow || !H->row_ptr || !H->col_idx || !H->val)
    return css_set_arg_error(ctx, "css_hprime: S and H need the same n_brow and b, and a valid H");
  if (flags & ~(CSS_SYMMETRIZE | CSS_REORTH_LOCAL)) return css_set_arg_error(ctx, "css_hprime: unknown flag");
  if (n_colours < 1) return css_set_arg_error(ctx, "css_hprime: n_colours < 1");
  CSS_CU(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const bool f32 = prec == CSS_MIXED_FP32 || prec == CSS_MIXED_3XTF32;
  const int32_t b = S->b, n_brow = S->n_brow;
  const int64_t N = (int64_t)n_brow * b;
  const int32_t w = n_colours * b;
  const int32_t ldy = (int32_t)css_ceil_div(w, 8) * 8;
  const size_t sv = f32 ? sizeof(float) : sizeof(double);
  void *Y, *W1, *W2;
  CSS_TRY(css_ws(ctx, "hp_Y", (size_t)N * ldy * sv, &Y));
  CSS_TRY(css_ws(ctx, "hp_W1", (size_t)N * ldy * sv, &W1));
  CSS_TRY(css_ws(ctx, "hp_W2", (size_t)N * ldy * sv, &W2));
  CSS_CU(ctx, cudaMemsetAsync(Y, 0, (size_t)N * ldy * sv, st));
  // 1. S~^(-1/2) on S's pattern and Y = S^(-1/2) |o> for every colour (paper, Eq. 8-10)
  css_fermi fz{0.0, 0.0, 0.0, 0.0, 0};
  css_sys_desc d{*S, colour, sign, n_colours, fz, Sinv_val};
  double t1, t2, mu0;
  const css_status s1 = css_density_impl(ctx, 1, &d, m, prec, (flags & (CSS_SYMMETRIZE | CSS_REORTH_LOCAL)) |
                                                                    CSS_INV_SQRT, &t1, &t2, &mu0, st, Y, ldy);
  if (s1 != CSS_OK && s1 != CSS_WARN_BREAKDOWN) return s1;
  // 2. W1 = H Y, W2 = S~^(-1/2) W1 (the left factor is the sparse S~^(-1/2) just obtained)
  LzArgs la;
  la.fp32 = f32;
  la.n_brow = n_brow;
  la.b = b;
  la.w = w;
  la.ws = ldy;
  la.row_ptr = H->row_ptr;
  la.col_idx = H->col_idx;
  CSS_TRY(css_spmm_prepare(ctx, f32, b, n_brow, H->nnzb, H->row_ptr, H->col_idx, H->val, &la.Hval, &la.Hlo_diag,
                           st));
  CSS_TRY(css_spmm(ctx, la, Y, W1, st));
  la.row_ptr = S->row_ptr;
  la.col_idx = S->col_idx;
  CSS_TRY(css_spmm_prepare(ctx, f32, b, n_brow, S->nnzb, S->row_ptr, S->col_idx, Sinv_val, &la.Hval,
                           &la.Hlo_diag, st));
  CSS_TRY(css_spmm(ctx, la, W1, W2, st));
  // 3. H' on H's pattern and its trace
  int32_t* brow;
  double *part, *tout;
  const int64_t nth = (int64_t)H->nnzb * b * b;
  const unsigned blocks = (unsigned)css_ceil_div(nth, EX_T);
  CSS_TRY(css_ws(ctx, "hp_brow", sizeof(int32_t) * (size_t)H->nnzb, (void**)&brow));
  CSS_TRY(css_ws(ctx, "hp_part", sizeof(double) * 2 * (size_t)blocks, (void**)&part));
  CSS_TRY(css_ws(ctx, "hp_tout", sizeof(double) * 2, (void**)&tout));
  k_block_rows<<<(unsigned)css_ceil_div(n_brow, 256), 256, 0, st>>>(n_brow, H->row_ptr, brow);
  CSS_LAUNCHED(ctx);
  const int sym = (flags & CSS_SYMMETRIZE) ? 1 : 0;
  if (f32)
    k_hp_extract<float><<<blocks, EX_T, 0, st>>>(H->nnzb, b, brow, H->col_idx, colour, sign, (const float*)W2, ldy,
                                                 sym, Hp_val, part);
  else
    k_hp_extract<double><<<blocks, EX_T, 0, st>>>(H->nnzb, b, brow, H->col_idx, colour, sign, (const double*)W2,
                                                  ldy, sym, Hp_val, part);
  CSS_LAUNCHED(ctx);
  k_trace_sum<<<1, 1024, 0, st>>>((int32_t)blocks, part, tout);
  CSS_LAUNCHED(ctx);
  double* h;
  CSS_TRY(css_pinned(ctx, sizeof(double) * 2, (void**)&h));
  CSS_CU(ctx, cudaMemcpyAsync(h, tout, sizeof(double), cudaMemcpyDeviceToHost, st));
  CSS_CU(ctx, cudaStreamSynchronize(st));
  if (trHp) *trHp = h[0];
  if (!std::isfinite(h[0])) {
    ctx->last_error = "css_hprime: non-finite trace of H'";
    return CSS_ERR_NUMERIC;
  }
  return s1;
}

css_status css_density_nonorth(css_ctx* ctx, const css_bsr* S, const double* Sinv_val, const css_bsr* Hp,
                               const double* H_val, const int32_t* colour, const int8_t* sign, int32_t n_colours,
                               const css_fermi* fermi, int32_t m, css_precision prec, uint32_t flags, double* P_val,
                               double* trPS, double* trPH, double* mu_out, void* stream) {
  // ------------------------------------------------------------ validation
  if (!ctx || !S || !Hp || !fermi || !Sinv_val || !H_val || !colour || !sign || !P_val)
    return css_set_arg_error(ctx, "css_density_nonorth: null pointer");
  if (!S->row_ptr || !S->col_idx || !S->val || !Hp->row_ptr || !Hp->col_idx || !Hp->val)
    return css_set_arg_error(ctx, "css_density_nonorth: S or H' without pattern or values");
  if (S->n_brow != Hp->n_brow || S->b != Hp->b || S->n_brow < 1 || S->nnzb < S->n_brow || Hp->nnzb < Hp->n_brow)
    return css_set_arg_error(ctx, "css_density_nonorth: S and H' need the same n_brow and b and a diagonal");
  if (prec != CSS_FP64 && prec != CSS_MIXED_FP32 && prec != CSS_MIXED_3XTF32 && prec != CSS_FP64_SPLIT)
    return css_set_arg_error(ctx, "css_density_nonorth: unknown precision");
  if (flags & ~(CSS_SYMMETRIZE | CSS_REORTH_LOCAL)) return css_set_arg_error(ctx, "css_density_nonorth: unknown flag");
  const int32_t b = Hp->b;
  if (b < 1) return css_set_arg_error(ctx, "css_density_nonorth: b < 1");
  if (b > CSS_MAX_B) {
    ctx->last_error = "css_density_nonorth: b > 32 is not supported";
    return CSS_ERR_UNSUPPORTED;
  }
  if (m < 1 || (int64_t)m * b > 4096) return css_set_arg_error(ctx, "css_density_nonorth: need 1 <= m and m*b <= 4096");
  if (n_colours < 1 || n_colours > (1 << 24)) return css_set_arg_error(ctx, "css_density_nonorth: n_colours out of range");
  if (!(fermi->kT >= 0.0) || !std::isfinite(fermi->kT) || !std::isfinite(fermi->mu) || !std::isfinite(fermi->n_elec) ||
      !std::isfinite(fermi->ne_tol))
    return css_set_arg_error(ctx, "css_density_nonorth: kT must be finite and >= 0, mu and n_elec finite");
  if ((int64_t)Hp->nnzb * b * b > (1ll << 40) || (int64_t)S->nnzb * b * b > (1ll << 40))
    return css_set_arg_error(ctx, "css_density_nonorth: problem too large");
  CSS_CU(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const bool f32 = prec == CSS_MIXED_FP32 || prec == CSS_MIXED_3XTF32;
  const int32_t n_brow = Hp->n_brow, nc = n_colours, bb = b * b, nmax = m * b;
  const int64_t N = (int64_t)n_brow * b;
  const size_t s_vec = f32 ? 4 : 8;
  const int T = 256;
  const unsigned gb = (unsigned)css_ceil_div(n_brow, T);

  // ------------------------------------- patterns, colour counts, validation
  int32_t *hbrow, *htrans, *sbrow, *strans, *cnt, *cnt2, *nblk, *done, *misc, *soc;
  double* isq;
  CSS_TRY(ws_get(ctx, "no_hbrow", Hp->nnzb, &hbrow));
  CSS_TRY(ws_get(ctx, "no_htrans", Hp->nnzb, &htrans));
  CSS_TRY(ws_get(ctx, "no_sbrow", S->nnzb, &sbrow));
  CSS_TRY(ws_get(ctx, "no_strans", S->nnzb, &strans));
  CSS_TRY(ws_get(ctx, "no_cnt", nc, &cnt));
  CSS_TRY(ws_get(ctx, "no_cnt2", nc, &cnt2));
  CSS_TRY(ws_get(ctx, "no_nblk", nc, &nblk));
  CSS_TRY(ws_get(ctx, "no_done", nc, &done));
  CSS_TRY(ws_get(ctx, "no_soc", nc, &soc));
  CSS_TRY(ws_get(ctx, "no_isq", nc, &isq));
  CSS_TRY(ws_get(ctx, "no_misc", 64, &misc));
  CSS_CU(ctx, cudaMemsetAsync(misc, 0, 64 * sizeof(int32_t), st));
  CSS_CU(ctx, cudaMemsetAsync(cnt, 0, nc * sizeof(int32_t), st));
  CSS_CU(ctx, cudaMemsetAsync(cnt2, 0, nc * sizeof(int32_t), st));
  CSS_CU(ctx, cudaMemsetAsync(soc, 0, nc * sizeof(int32_t), st));  // one system
  k_rows<<<gb, T, 0, st>>>(n_brow, Hp->row_ptr, Hp->col_idx, colour, nc, hbrow, htrans, cnt, misc + 1, misc);
  CSS_LAUNCHED(ctx);
  k_rows<<<gb, T, 0, st>>>(n_brow, S->row_ptr, S->col_idx, colour, nc, sbrow, strans, cnt2, misc + 3, misc + 2);
  CSS_LAUNCHED(ctx);
  k_inv_sqrt<<<(unsigned)css_ceil_div(nc, T), T, 0, st>>>(nc, cnt, isq, nblk, done, m);
  CSS_LAUNCHED(ctx);
  int32_t* hb;
  CSS_TRY(css_pinned(ctx, 256, (void**)&hb));
  CSS_CU(ctx, cudaMemcpyAsync(hb, misc, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CSS_CU(ctx, cudaStreamSynchronize(st));
  if ((hb[0] | hb[2]) & ERR_COLOUR) return css_set_arg_error(ctx, "css_density_nonorth: colour outside [0, n_colours)");
  if ((hb[0] | hb[2]) & ERR_PATTERN)
    return css_set_arg_error(ctx, "css_density_nonorth: a pattern is not symmetric, has a column out of range or "
                                  "misses a diagonal block");
  const int32_t max_row = hb[1];

  // ------------------------- H', S~^(-1/2), S and S~^(-1/2)^T in the H*V layout
  double* sinvT;
  CSS_TRY(ws_get(ctx, "no_sinvT", (size_t)S->nnzb * bb, &sinvT));
  k_block_transpose<<<(unsigned)css_ceil_div((int64_t)S->nnzb * bb, T), T, 0, st>>>(S->nnzb, b, strans, Sinv_val,
                                                                                    sinvT);
  CSS_LAUNCHED(ctx);
  const void *hpv, *hplo, *siv, *silo, *sv, *slo, *sitv, *sitlo;
  CSS_TRY(css_spmm_prepare_as(ctx, "no_hp", f32, b, n_brow, Hp->nnzb, Hp->row_ptr, Hp->col_idx, Hp->val, &hpv, &hplo,
                              st));
  CSS_TRY(css_spmm_prepare_as(ctx, "no_si", f32, b, n_brow, S->nnzb, S->row_ptr, S->col_idx, Sinv_val, &siv, &silo,
                              st));
  CSS_TRY(css_spmm_prepare_as(ctx, "no_s", f32, b, n_brow, S->nnzb, S->row_ptr, S->col_idx, S->val, &sv, &slo, st));
  CSS_TRY(css_spmm_prepare_as(ctx, "no_sit", f32, b, n_brow, S->nnzb, S->row_ptr, S->col_idx, sinvT, &sitv, &sitlo,
                              st));

  // ------------------------------------------ vectors (all colours at once)
  const int32_t ws = (int32_t)css_ceil_div((int64_t)nc * b, 8) * 8;
  const size_t vbytes = (size_t)N * ws * s_vec;
  size_t free_b = 0, total_b = 0;
  CSS_CU(ctx, cudaMemGetInfo(&free_b, &total_b));
  if (7 * vbytes + ((size_t)1 << 30) > free_b + ctx->ws_bytes) {
    ctx->last_error = "css_density_nonorth: the Krylov blocks of all colours do not fit in device memory";
    return CSS_ERR_NOMEM;
  }
  void *R, *R0, *SR, *U, *Q0, *Q1, *Wv;
  CSS_TRY(css_ws(ctx, "no_R", vbytes, &R));
  CSS_TRY(css_ws(ctx, "no_start", vbytes, &R0));
  CSS_TRY(css_ws(ctx, "no_SR", vbytes, &SR));
  CSS_TRY(css_ws(ctx, "no_u", vbytes, &U));
  CSS_TRY(css_ws(ctx, "no_Q0", vbytes, &Q0));
  CSS_TRY(css_ws(ctx, "no_Q1", vbytes, &Q1));
  CSS_TRY(css_ws(ctx, "no_W", vbytes, &Wv));
  LzArgs op;  // one H*V operand at a time: pattern and prepared values
  op.fp32 = f32;
  op.n_brow = n_brow;
  op.b = b;
  op.w = nc * b;
  op.ws = ws;
  auto spmm_with = [&](const css_bsr* M, const void* val, const void* lo, const void* V, void* W) -> css_status {
    op.row_ptr = M->row_ptr;
    op.col_idx = M->col_idx;
    op.Hval = val;
    op.Hlo_diag = lo;
    return css_spmm(ctx, op, V, W, st);
  };
  // probe blocks R_c, start blocks r~_c = S~^(-1/2) R_c, and u_c = S~^(-1/2)^T S R_c
  double* ones;
  CSS_TRY(ws_get(ctx, "no_ones", nc, &ones));
  k_fill<<<(unsigned)css_ceil_div(nc, T), T, 0, st>>>(nc, 1.0, ones);
  CSS_LAUNCHED(ctx);
  CSS_TRY(css_probe_block(ctx, f32, n_brow, b, ws, 0, nc, colour, sign, ones, R, st));
  CSS_TRY(spmm_with(S, siv, silo, R, R0));
  CSS_TRY(spmm_with(S, sv, slo, R, SR));
  CSS_TRY(spmm_with(S, sitv, sitlo, SR, U));

  // ---------------------------- block-Lanczos on H' (pass 1: T_c, B_0, V_c)
  double *Ablk, *Bblk, *Bprev, *B0, *Vc, *part, *small, *Z;
  CSS_TRY(ws_get(ctx, "no_A", (size_t)nc * m * bb, &Ablk));
  CSS_TRY(ws_get(ctx, "no_B", (size_t)nc * m * bb, &Bblk));
  CSS_TRY(ws_get(ctx, "no_Bprev", (size_t)nc * bb, &Bprev));
  CSS_TRY(ws_get(ctx, "no_B0", (size_t)nc * bb, &B0));
  CSS_TRY(ws_get(ctx, "no_Vc", (size_t)nc * nmax * b, &Vc));
  CSS_TRY(ws_get(ctx, "no_part", css_lanczos_part_doubles(N, b, nc) * 2, &part));
  CSS_TRY(ws_get(ctx, "no_small", css_lanczos_small_doubles(b, nc), &small));
  CSS_TRY(ws_get(ctx, "no_Z", (size_t)nc * nmax * b, &Z));
  CSS_CU(ctx, cudaMemsetAsync(Vc, 0, sizeof(double) * nc * nmax * b, st));
  std::vector<int64_t> no_pairs((size_t)nc + 1, 0);  // nothing is sampled: X comes from whole rows
  LzArgs la;
  la.fp32 = f32;
  la.n_brow = n_brow;
  la.b = b;
  la.m = m;
  la.w = nc * b;
  la.ws = ws;
  la.row_ptr = Hp->row_ptr;
  la.col_idx = Hp->col_idx;
  la.Hval = hpv;
  la.Hlo_diag = hplo;
  la.max_row_blocks = max_row;
  la.colour = colour;
  la.sign = sign;
  la.inv_sqrt_cnt = isq;
  la.cb0 = 0;
  la.ncb = nc;
  la.Q0 = Q0;
  la.Q1 = Q1;
  la.W = Wv;
  la.Ablk = Ablk;
  la.Bblk = Bblk;
  la.Bblk_prev = Bprev;
  la.nblk = nblk;
  la.done = done;
  la.part = part;
  la.small = small;
  la.tau = f32 ? 1e-5 : 1e-10;
  la.shift_rel = f32 ? 1e-5 : 1e-12;
  la.flags = f32 ? (flags | CSS_REORTH_LOCAL) : flags;
  la.mode = 0;
  la.Z = Z;
  la.ldz = nmax;
  la.pair_off_h = no_pairs.data();
  la.start = R0;
  la.B0 = B0;
  la.ucol = U;
  la.Vc = Vc;
  CSS_TRY(css_lanczos_pass(ctx, la, st));

  // ------------------------------ eigen-data with B_0, kappa, mu and Z_c
  EigArgs ea;
  ea.n_col = nc;
  ea.b = b;
  ea.m = m;
  ea.Ablk = Ablk;
  ea.Bblk = Bblk;
  ea.nblk = nblk;
  ea.cnt = cnt;
  ea.B0 = B0;
  ea.rcap = nmax * (nmax / b + 2);
  CSS_TRY(ws_get(ctx, "e_AB", (size_t)nc * nmax * (2 * b + 1), &ea.AB));
  CSS_TRY(ws_get(ctx, "e_RV", (size_t)nc * ea.rcap * b, &ea.RV));
  CSS_TRY(ws_get(ctx, "e_RT", (size_t)nc * ea.rcap, &ea.RT));
  CSS_TRY(ws_get(ctx, "e_RR0", (size_t)nc * ea.rcap, &ea.RR0));
  CSS_TRY(ws_get(ctx, "e_so", (size_t)nc * (nmax + 1), &ea.sweep_off));
  CSS_TRY(ws_get(ctx, "e_d", (size_t)nc * nmax, &ea.d));
  CSS_TRY(ws_get(ctx, "e_e", (size_t)nc * nmax, &ea.e));
  CSS_TRY(ws_get(ctx, "e_l32", (size_t)nc * nmax, &ea.lam32));
  CSS_TRY(ws_get(ctx, "e_tn", (size_t)nc, &ea.tnorm));
  CSS_TRY(ws_get(ctx, "e_U", (size_t)nc * nmax * nmax, &ea.U));
  CSS_TRY(ws_get(ctx, "e_F", (size_t)nc * 5 * nmax * nmax, &ea.F));
  CSS_TRY(ws_get(ctx, "e_lam", (size_t)nc * nmax, &ea.lam));
  CSS_TRY(ws_get(ctx, "e_X0", (size_t)nc * nmax * b, &ea.X0));
  CSS_TRY(ws_get(ctx, "e_Y", (size_t)nc * nmax * b, &ea.Y));
  CSS_TRY(ws_get(ctx, "e_w", (size_t)nc * nmax, &ea.wgt));
  CSS_TRY(ws_get(ctx, "e_st", (size_t)nc, &ea.status));
  CSS_TRY(ws_get(ctx, "e_flag", (size_t)nc * nmax, &ea.flag));
  CSS_TRY(css_eigen_ritz(ctx, ea, st));
  double *YV, *scratch, *kap;
  CSS_TRY(ws_get(ctx, "no_YV", (size_t)nc * nmax * b, &YV));
  CSS_TRY(ws_get(ctx, "no_wsc", (size_t)nc * nmax, &scratch));
  CSS_TRY(ws_get(ctx, "no_kap", (size_t)nc * nmax, &kap));
  CSS_TRY(css_eigen_project(ctx, ea, Vc, YV, scratch, st));
  k_kappa<<<(unsigned)css_ceil_div((int64_t)nc * nmax, T), T, 0, st>>>(nc, b, nmax, nblk, YV, ea.Y, kap);
  CSS_LAUNCHED(ctx);
  double *dmu, *dkT, *dhalf, *dmu_in, *dtol, *mupart;
  int32_t* dsolve;
  unsigned* bar;
  CSS_TRY(ws_get(ctx, "no_mu", 8, &dmu));
  CSS_TRY(ws_get(ctx, "no_fermi", 8, &dkT));
  dhalf = dkT + 1;
  dmu_in = dkT + 2;
  dtol = dkT + 3;
  CSS_TRY(ws_get(ctx, "no_solve", 8, &dsolve));
  CSS_TRY(ws_get(ctx, "no_bar", 8, &bar));
  {
    double* hp;
    CSS_TRY(css_pinned(ctx, 256, (void**)&hp));
    hp[0] = fermi->kT;
    hp[1] = 0.5 * fermi->n_elec;
    hp[2] = fermi->mu;
    hp[3] = fermi->ne_tol > 0.0 ? fermi->ne_tol : 1e-4 * std::max(1.0, 0.5 * fermi->n_elec);
    ((int32_t*)(hp + 4))[0] = fermi->solve_mu ? 1 : 0;
    CSS_CU(ctx, cudaMemcpyAsync(dkT, hp, 4 * sizeof(double), cudaMemcpyHostToDevice, st));
    CSS_CU(ctx, cudaMemcpyAsync(dsolve, hp + 4, sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CSS_CU(ctx, cudaMemsetAsync(bar, 0, 8 * sizeof(unsigned), st));
    CSS_CU(ctx, cudaStreamSynchronize(st));  // the pinned staging is reused below
  }
  int occ = 0;
  CSS_CU(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mu, MU_T, 0));
  unsigned G = (unsigned)std::max(1, std::min(ctx->n_sm * std::max(occ, 1), std::max(nc, 1)));
  if (G > (unsigned)ctx->n_sm) G = (unsigned)ctx->n_sm;
  CSS_TRY(ws_get(ctx, "no_mu_part", (size_t)4 * G + 16, &mupart));
  {
    int32_t n_sys_ = 1, n_col_ = nc, nmax_ = nmax, b_ = b;
    const int32_t* nblk_ = nblk;
    const int32_t* soc_ = soc;
    const double* lam_ = ea.lam;
    const double* w_ = kap;  // the electron count is Tr(rho S)
    const double* kT_ = dkT;
    const double* h_ = dhalf;
    const double* tl_ = dtol;
    const int32_t* sv_ = dsolve;
    const double* mi_ = dmu_in;
    double* mo_ = dmu;
    double* pp_ = mupart;
    unsigned* bar_ = bar;
    int32_t* err_ = misc + 8;
    int32_t extra_ = ctx->test_mu_barrier_extra;
    void* args[] = {&n_sys_, &n_col_, &nmax_, &nblk_, &b_, &soc_, &lam_, &w_, &kT_, &h_, &tl_, &sv_, &mi_, &mo_, &pp_,
                    &bar_, &err_, &extra_};
    CSS_CU(ctx, cudaLaunchCooperativeKernel((void*)k_mu, dim3(G), dim3(MU_T), args, 0, st));
    ++ctx->kernel_launches;
  }
  CSS_TRY(css_eigen_z(ctx, ea, soc, dmu, dkT, Z, st, 0));

  // ------------- pass 2: X~ = Phi Z over all rows, X = S~^(-1/2) X~, extraction
  void* Xt = R;  // the probe blocks are no longer needed
  void* X = SR;
  CSS_CU(ctx, cudaMemsetAsync(Xt, 0, vbytes, st));
  CSS_CU(ctx, cudaMemsetAsync(done, 0, nc * sizeof(int32_t), st));
  k_inv_sqrt<<<(unsigned)css_ceil_div(nc, T), T, 0, st>>>(nc, cnt, isq, nblk, done, m);
  CSS_LAUNCHED(ctx);
  double* B0b;  // pass 2 recomputes B_0 (bitwise the same) into a scratch copy
  CSS_TRY(ws_get(ctx, "no_B0b", (size_t)nc * bb, &B0b));
  la.mode = 2;
  la.Yfull = Xt;
  la.ldy = ws;
  la.ucol = nullptr;
  la.Vc = nullptr;
  la.B0 = B0b;
  CSS_TRY(css_lanczos_pass(ctx, la, st));
  CSS_TRY(spmm_with(S, siv, silo, Xt, X));
  double *tpart, *tpart2, *tout;
  const int64_t nh = (int64_t)Hp->nnzb * bb, ns = (int64_t)S->nnzb * bb;
  const unsigned xblocks = (unsigned)css_ceil_div(nh, EX_T);
  const unsigned tblocks = (unsigned)css_ceil_div(std::max(nh, ns), EX_T);
  CSS_TRY(ws_get(ctx, "no_tpart", 2 * (size_t)xblocks + 2, &tpart));
  CSS_TRY(ws_get(ctx, "no_tpart2", 2 * (size_t)tblocks + 2, &tpart2));
  CSS_TRY(ws_get(ctx, "no_tout", 4, &tout));
  const int sym = (flags & CSS_SYMMETRIZE) ? 1 : 0;
  if (f32)
    k_hp_extract<float><<<xblocks, EX_T, 0, st>>>(Hp->nnzb, b, hbrow, Hp->col_idx, colour, sign, (const float*)X, ws,
                                                  sym, P_val, tpart);
  else
    k_hp_extract<double><<<xblocks, EX_T, 0, st>>>(Hp->nnzb, b, hbrow, Hp->col_idx, colour, sign, (const double*)X,
                                                   ws, sym, P_val, tpart);
  CSS_LAUNCHED(ctx);
  k_trace_hs<<<tblocks, EX_T, 0, st>>>(nh, ns, b, P_val, H_val, Hp->row_ptr, Hp->col_idx, sbrow, S->col_idx, S->val,
                                       tpart2, misc + 20);
  CSS_LAUNCHED(ctx);
  k_trace_sum<<<1, 1024, 0, st>>>((int32_t)tblocks, tpart2, tout);
  CSS_LAUNCHED(ctx);
  k_count_breakdown<<<(unsigned)css_ceil_div(nc, T), T, 0, st>>>(nc, m, nblk, cnt, misc + 16);
  CSS_LAUNCHED(ctx);
  k_status_or<<<(unsigned)css_ceil_div(nc, T), T, 0, st>>>(nc, ea.status, misc + 17);
  CSS_LAUNCHED(ctx);

  // -------------------------------------------------------------- read back
  double* hres;
  CSS_TRY(css_pinned(ctx, 256, (void**)&hres));
  CSS_CU(ctx, cudaMemcpyAsync(hres, tout, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CSS_CU(ctx, cudaMemcpyAsync(hres + 2, dmu, sizeof(double), cudaMemcpyDeviceToHost, st));
  CSS_CU(ctx, cudaMemcpyAsync(hres + 4, misc, 24 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CSS_CU(ctx, cudaStreamSynchronize(st));
  const int32_t* hm = (const int32_t*)(hres + 4);
  if (trPH) *trPH = hres[0];
  if (trPS) *trPS = hres[1];
  if (mu_out) *mu_out = hres[2];
  ctx->last_lam = ea.lam;
  ctx->last_wgt = kap;
  ctx->last_nblk = nblk;
  ctx->last_ncol = nc;
  ctx->last_b = b;
  ctx->last_nmax = nmax;
  ctx->last_A = Ablk;
  ctx->last_B = Bblk;
  ctx->last_m = m;
  ctx->info.n_colours = nc;
  ctx->info.n_breakdown = hm[16];
  ctx->info.m = m;
  if (hm[8]) {
    ctx->last_error = "css_density_nonorth: grid barrier of the mu bisection timed out";
    return CSS_ERR_TIMEOUT;
  }
  if (hm[17] & 2) {
    ctx->last_error = "css_density_nonorth: a wait between pipelined band-reduction sweeps timed out";
    return CSS_ERR_TIMEOUT;
  }
  if (hm[20]) return css_set_arg_error(ctx, "css_density_nonorth: S has a block outside H's pattern");
  if (!std::isfinite(hres[0]) || !std::isfinite(hres[1]) || !std::isfinite(hres[2])) {
    ctx->last_error = "css_density_nonorth: non-finite trace or mu";
    return CSS_ERR_NUMERIC;
  }
  return hm[16] > 0 ? CSS_WARN_BREAKDOWN : CSS_OK;
}

}  // extern "C"
