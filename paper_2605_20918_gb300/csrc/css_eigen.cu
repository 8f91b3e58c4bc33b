// FP64 eigen-decomposition of the projected block-tridiagonal matrices, one per colour, and
// the subspace matrix function Z = U f(Lambda) U^T E_1 B_0 (paper, Eq. 5-7: exact
// diagonalisation of the Krylov-projected Hamiltonian).
//
// GB300 runs FP64 at about 1/64 of the FP32 rate and a dependent FP64 sqrt + divide costs
// ~0.6 us, so no stage here is a long sequential FP64 chain:
//   1. band -> tridiagonal by Householder bulge chasing, up to 32 sweeps in flight (one warp
//      each, a sweep waits only for the one before it to move past its window); reflectors
//      of length <= b, and a sweep's reflectors touch disjoint rows, so their action on
//      b-column blocks is applied sweep by sweep with all of a sweep's reflectors in parallel;
//   2. eigenvalues of the tridiagonal by Sturm-count bisection in FP32 (one thread per
//      eigenvalue), used only as shifts;
//   3. FP64 Rayleigh-quotient inverse iteration: one thread per eigenvalue in lockstep, then
//      one warp per cluster of close shifts (simultaneous iteration with Gram-Schmidt and a
//      Rayleigh-Ritz step inside the cluster), which gives eigenvalues and eigenvectors to
//      FP64 accuracy;
//   4. Y = U^T (Q_band^T E_1 B_0), weights w = ||Y_k||^2, and after mu is known
//      Z = Q_band U f(Lambda) Y.
#include "css_eigen.cuh"

namespace {

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------ band storage
// AB[col * LDB + d] = T[col + d][col], d in [0, LDB), LDB = 2 kd + 1 (room for the bulge)
__global__ void k_band_build(int32_t b, int32_t m, int32_t nmax, int32_t ldb, const double* __restrict__ Ablk,
                             const double* __restrict__ Bblk, const int32_t* __restrict__ nblk,
                             double* __restrict__ AB) {
  const int32_t c = blockIdx.x;
  const int32_t n = nblk[c] * b;
  double* ab = AB + (size_t)c * nmax * ldb;
  for (int32_t t = threadIdx.x; t < nmax * ldb; t += blockDim.x) {
    int32_t col = t / ldb, d = t % ldb, row = col + d;
    double v = 0.0;
    if (col < n && row < n && d <= b) {
      int32_t jc = col / b, kc = col % b, jr = row / b, kr = row % b;
      if (jr == jc) v = Ablk[(((size_t)c * m + jc) * b + kr) * b + kc];
      else if (jr == jc + 1 && kr <= kc) v = Bblk[(((size_t)c * m + jc) * b + kr) * b + kc];
    }
    ab[t] = v;
  }
}

struct Band {
  double* ab;
  int32_t ldb;
  // lower-stored symmetric access, r >= c
  __device__ __forceinline__ double& at(int32_t r, int32_t c) const { return ab[(size_t)c * ldb + (r - c)]; }
};

// Householder vector of x[0..L) held one element per lane of warp 0: H x = beta e_0.
// Textbook construction (Golub & Van Loan, Alg. 5.1.1): v[0] = 1, tau = 2 v0^2/(sigma+v0^2).
__device__ void warp_house(double x, int32_t L, double* sv, double* stau, double* sbeta) {
  const int lane = threadIdx.x & 31;
  double x0 = __shfl_sync(0xffffffffu, x, 0);
  double sig = warp_sum((lane >= 1 && lane < L) ? x * x : 0.0);
  if (sig == 0.0) {
    if (lane < 32) sv[lane] = (lane == 0) ? 1.0 : 0.0;
    if (lane == 0) {
      *stau = 0.0;
      *sbeta = x0;
    }
    return;
  }
  double mu = sqrt(x0 * x0 + sig);
  double v0 = (x0 <= 0.0) ? x0 - mu : -sig / (x0 + mu);
  double inv = 1.0 / v0;
  sv[lane] = (lane == 0) ? 1.0 : ((lane < L) ? x * inv : 0.0);
  if (lane == 0) {
    *stau = 2.0 * v0 * v0 / (sig + v0 * v0);
    *sbeta = mu;
  }
}

// D <- H D H on the symmetric L x L diagonal block starting at r0 (H = I - tau v v^T), by one
// warp: lane i owns row i.  pw is the warp's scratch of 32 doubles.
__device__ void two_sided_w(const Band& A, int32_t r0, int32_t L, const double* v, double tau, double* pw) {
  const int lane = threadIdx.x & 31;
  if (tau == 0.0) return;
  double acc = 0.0;
  if (lane < L)
    for (int32_t j = 0; j < L; ++j)
      acc += (lane >= j ? A.at(r0 + lane, r0 + j) : A.at(r0 + j, r0 + lane)) * v[j];
  const double vi = lane < L ? v[lane] : 0.0;
  const double pi = lane < L ? tau * acc : 0.0;
  const double alpha = -0.5 * tau * warp_sum(pi * vi);
  const double wi = pi + alpha * vi;
  pw[lane] = wi;
  __syncwarp();
  if (lane < L)
    for (int32_t j = 0; j <= lane; ++j) A.at(r0 + lane, r0 + j) -= vi * pw[j] + wi * v[j];
  __syncwarp();
}

// reflectors recorded by sweep i (the type-1 reflector and one per chase step whose block has
// at least two rows), the same count the sequential order produces
__device__ int32_t sweep_refl_count(int32_t i, int32_t n, int32_t kd) {
  int32_t cnt = 1, p0 = i + 1, Lp = min(kd, n - 1 - i);
  for (;;) {
    const int32_t q0 = p0 + Lp;
    if (q0 > n - 1) break;
    const int32_t Lq = min(kd, n - q0);
    if (Lq < 2) break;
    ++cnt;
    p0 = q0;
    Lp = Lq;
  }
  return cnt;
}

// Band -> tridiagonal (one CTA of 32 warps per colour) with the sweeps pipelined: warp w runs
// sweeps w, w + 32, ...  Every step of a sweep touches the rows and columns of one window
// [lo, hi) of the matrix, and the windows of a sweep move down the band.  Sweep s runs a step
// only once sweep s - 1 has finished or its next step's window starts at or after the step's
// hi: then no later step of s - 1 touches what the step reads or writes, and (by induction)
// neither does any earlier sweep, so the result is the sequential order's.  Each warp
// publishes (sweep, start of its next window) in one 64-bit shared word.  Reflector k of
// sweep i is stored at sweep_off[i] + k, as in the sequential order.  A wait gives up after
// 2^24 polls: the colour's status gets bit 2 and the CTA stops.
__global__ void __launch_bounds__(1024) k_band_to_tri(int32_t kd, int32_t nmax, int32_t ldb, int32_t rcap,
                                                      const int32_t* __restrict__ nblk, double* __restrict__ AB,
                                                      double* __restrict__ RV, double* __restrict__ RT,
                                                      int32_t* __restrict__ RR0, int32_t* __restrict__ sweep_off,
                                                      double* __restrict__ dd, double* __restrict__ ee,
                                                      int32_t* __restrict__ status) {
  constexpr int NW = 32;
  __shared__ double sv[NW][32], svn[NW][32], spw[NW][32];
  __shared__ double stau[NW], sbeta[NW];
  __shared__ unsigned long long slot[NW];  // ((sweep + 1) << 32) | start of the next window
  __shared__ int abort_flag;
  const int32_t c = blockIdx.x;
  const int32_t n = nblk[c] * kd;
  Band A{AB + (size_t)c * nmax * ldb, ldb};
  double* rv = RV + (size_t)c * rcap * kd;
  double* rt = RT + (size_t)c * rcap;
  int32_t* rr = RR0 + (size_t)c * rcap;
  int32_t* so = sweep_off + (size_t)c * (nmax + 1);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int32_t nsweep = n > 2 ? n - 2 : 0;
  // reflector offsets of the sweeps
  for (int32_t i = threadIdx.x; i < nsweep; i += blockDim.x) so[i + 1] = sweep_refl_count(i, n, kd);
  if (threadIdx.x < NW) slot[threadIdx.x] = 0ull;
  if (threadIdx.x == 0) abort_flag = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    so[0] = 0;
    for (int32_t i = 0; i < nsweep; ++i) so[i + 1] += so[i];
    for (int32_t i = nsweep + 1; i <= n; ++i) so[i] = so[nsweep];
  }
  __syncthreads();
  double* v = sv[w];
  double* vn = svn[w];
  double* pw = spw[w];
  auto publish = [&](int32_t s, int32_t front) {
    __syncwarp();
    if (lane == 0) {
      __threadfence_block();
      *(volatile unsigned long long*)&slot[w] =
          ((unsigned long long)(uint32_t)(s + 1) << 32) | (unsigned long long)(uint32_t)front;
    }
  };
  // wait until sweep s - 1 cannot touch [.., hi) any more; false on timeout or abort
  auto wait_prev = [&](int32_t s, int32_t hi) -> bool {
    bool ok = true;
    if (s > 0 && lane == 0) {
      const int pw_ = (s - 1) % NW;
      for (uint32_t it = 0;; ++it) {
        const unsigned long long x = *(volatile unsigned long long*)&slot[pw_];
        const int32_t id = (int32_t)(x >> 32) - 1;
        const int32_t front = (int32_t)(uint32_t)(x & 0xffffffffull);
        if (id > s - 1 || (id == s - 1 && front >= hi)) break;
        if (*(volatile int*)&abort_flag) {
          ok = false;
          break;
        }
        if (it >= (1u << 24)) {
          atomicOr(&status[c], 2);
          *(volatile int*)&abort_flag = 1;
          ok = false;
          break;
        }
        __nanosleep(32);
      }
      __threadfence_block();
    }
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    __syncwarp();
    return ok;
  };
  auto record = [&](int32_t k, int32_t r0, const double* vv, double tau) {
    if (lane < kd) rv[(size_t)k * kd + lane] = vv[lane];
    if (lane == 0) {
      rt[k] = tau;
      rr[k] = r0;
    }
  };
  constexpr int32_t kDone = 0x7fffffff;
  bool dead = false;  // a wait gave up: leave the loops, still reach the final barrier
  for (int32_t i = w; i < nsweep && !dead; i += NW) {
    const int32_t r0 = i + 1;
    const int32_t L = min(kd, n - 1 - i);
    int32_t k = so[i];
    publish(i, i);  // first window starts at column i
    // type 1: annihilate column i below the sub-diagonal; window [i, r0 + L)
    if (!wait_prev(i, r0 + L)) {
      dead = true;
      break;
    }
    {
      const double x = (lane < L) ? A.at(r0 + lane, i) : 0.0;
      warp_house(x, L, v, &stau[w], &sbeta[w]);
      __syncwarp();
      if (lane < L) A.at(r0 + lane, i) = (lane == 0) ? sbeta[w] : 0.0;
      __syncwarp();
      two_sided_w(A, r0, L, v, stau[w], pw);
      record(k++, r0, v, stau[w]);
    }
    int32_t p0 = r0, Lp = L;
    double* cv = v;
    double* nv = vn;
    double tau = stau[w];
    for (;;) {
      const int32_t q0 = p0 + Lp;
      if (q0 > n - 1) break;
      const int32_t Lq = min(kd, n - q0);
      publish(i, p0);  // this chase step's window is [p0, q0 + Lq)
      if (!wait_prev(i, q0 + Lq)) {
        dead = true;
        break;
      }
      // type 2a: B = A[q0.., p0..] <- B (I - tau v v^T), lane = row of B
      if (tau != 0.0 && lane < Lq) {
        double y = 0.0;
        for (int32_t j = 0; j < Lp; ++j) y += A.at(q0 + lane, p0 + j) * cv[j];
        for (int32_t j = 0; j < Lp; ++j) A.at(q0 + lane, p0 + j) -= tau * y * cv[j];
      }
      __syncwarp();
      if (Lq < 2) break;
      // type 2b: new reflector from the bulge's first column, applied from the left
      {
        const double x = (lane < Lq) ? A.at(q0 + lane, p0) : 0.0;
        warp_house(x, Lq, nv, &stau[w], &sbeta[w]);
      }
      __syncwarp();
      const double tau2 = stau[w];
      if (tau2 != 0.0) {
        double z = 0.0;  // z[col] = nv^T B[:, col], lane = col >= 1
        if (lane >= 1 && lane < Lp)
          for (int32_t r = 0; r < Lq; ++r) z += nv[r] * A.at(q0 + r, p0 + lane);
        pw[lane] = z;
        __syncwarp();
        if (lane < Lq)
          for (int32_t j = 1; j < Lp; ++j) A.at(q0 + lane, p0 + j) -= tau2 * nv[lane] * pw[j];
        __syncwarp();
      }
      if (lane < Lq) A.at(q0 + lane, p0) = (lane == 0) ? sbeta[w] : 0.0;
      __syncwarp();
      // type 3: two-sided on the next diagonal block
      two_sided_w(A, q0, Lq, nv, tau2, pw);
      record(k++, q0, nv, tau2);
      double* t = cv;
      cv = nv;
      nv = t;
      tau = tau2;
      p0 = q0;
      Lp = Lq;
    }
    if (!dead) publish(i, kDone);
  }
  __syncthreads();
  if (abort_flag) return;
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
    dd[(size_t)c * nmax + i] = A.at(i, i);
    ee[(size_t)c * nmax + i] = (i + 1 < n) ? A.at(i + 1, i) : 0.0;
  }
}

// Apply the recorded reflectors to an n x b block X ([c][nmax][b]): FWD applies them in
// generation order (X <- Q^T X), otherwise in reverse (X <- Q X).  A sweep's reflectors act
// on disjoint rows, so one thread per (reflector of the sweep, column) works in parallel.
template <bool FWD>
__global__ void k_apply_refl(int32_t kd, int32_t b, int32_t nmax, int32_t rcap, const int32_t* __restrict__ nblk,
                             const double* __restrict__ RV, const double* __restrict__ RT,
                             const int32_t* __restrict__ RR0, const int32_t* __restrict__ sweep_off,
                             double* __restrict__ X) {
  const int32_t c = blockIdx.x;
  const int32_t n = nblk[c] * kd;
  const double* rv = RV + (size_t)c * rcap * kd;
  const double* rt = RT + (size_t)c * rcap;
  const int32_t* rr = RR0 + (size_t)c * rcap;
  const int32_t* so = sweep_off + (size_t)c * (nmax + 1);
  double* x = X + (size_t)c * nmax * b;
  const int32_t nsweep = n > 2 ? n - 2 : 0;
  for (int32_t s = 0; s < nsweep; ++s) {
    const int32_t i = FWD ? s : nsweep - 1 - s;
    const int32_t t0 = so[i], t1 = so[i + 1];
    for (int32_t t = threadIdx.x; t < (t1 - t0) * b; t += blockDim.x) {
      const int32_t r = t0 + t / b, col = t % b;
      const double tau = rt[r];
      if (tau == 0.0) continue;
      const int32_t r0 = rr[r];
      const int32_t L = min(kd, n - r0);
      const double* v = rv + (size_t)r * kd;
      double s2 = 0.0;
      for (int32_t l = 0; l < L; ++l) s2 += v[l] * x[(size_t)(r0 + l) * b + col];
      s2 *= tau;
      for (int32_t l = 0; l < L; ++l) x[(size_t)(r0 + l) * b + col] -= s2 * v[l];
    }
    __syncthreads();
  }
}

// X0 = E_1 B_0 = [B_0; 0] for a general start factor B_0 [c][b][b]
__global__ void k_x0_b0(int32_t b, int32_t nmax, const double* __restrict__ B0, double* __restrict__ X) {
  const int32_t c = blockIdx.x;
  for (int32_t t = threadIdx.x; t < nmax * b; t += blockDim.x) {
    const int32_t i = t / b, k = t % b;
    X[(size_t)c * nmax * b + t] = (i < b) ? B0[((size_t)c * b + i) * b + k] : 0.0;
  }
}

// X0 = E_1 B_0 = sqrt|c| [I_b; 0]
__global__ void k_x0(int32_t b, int32_t nmax, const int32_t* __restrict__ cnt, double* __restrict__ X) {
  const int32_t c = blockIdx.x;
  const double s = sqrt((double)cnt[c]);
  for (int32_t t = threadIdx.x; t < nmax * b; t += blockDim.x) {
    int32_t i = t / b, k = t % b;
    X[(size_t)c * nmax * b + t] = (i == k) ? s : 0.0;
  }
}

// ------------------------------------------------------------- FP32 bisection
__device__ __forceinline__ int32_t sturm32(const float* d, const float* e2, int32_t n, float x, float pivmin) {
  float qv = d[0] - x;
  int32_t cnt = qv < 0.f;
  for (int32_t i = 1; i < n; ++i) {
    if (fabsf(qv) < pivmin) qv = -pivmin;
    qv = (d[i] - x) - __fdividef(e2[i - 1], qv);
    cnt += qv < 0.f;
  }
  return cnt;
}

__global__ void k_bisect32(int32_t kd, int32_t nmax, const int32_t* __restrict__ nblk, const double* __restrict__ dd,
                           const double* __restrict__ ee, float* __restrict__ lam32, double* __restrict__ tnorm) {
  extern __shared__ float sh32[];
  const int32_t c = blockIdx.x;
  const int32_t n = nblk[c] * kd;
  float* d = sh32;
  float* e2 = sh32 + nmax;
  __shared__ double red_lo[32], red_hi[32];
  double lo = 1e300, hi = -1e300, emax = 0.0;
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
    double di = dd[(size_t)c * nmax + i];
    double el = i > 0 ? fabs(ee[(size_t)c * nmax + i - 1]) : 0.0;
    double er = i + 1 < n ? fabs(ee[(size_t)c * nmax + i]) : 0.0;
    lo = fmin(lo, di - el - er);
    hi = fmax(hi, di + el + er);
    d[i] = (float)di;
    double e = i + 1 < n ? ee[(size_t)c * nmax + i] : 0.0;
    e2[i] = (float)(e * e);
    emax = fmax(emax, e * e);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red_lo[threadIdx.x >> 5] = lo;
    red_hi[threadIdx.x >> 5] = fmax(hi, -1e300);
  }
  __shared__ double semax[32];
  if ((threadIdx.x & 31) == 0) semax[threadIdx.x >> 5] = emax;
  __syncthreads();
  double glo = 1e300, ghi = -1e300, gem = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
    glo = fmin(glo, red_lo[i]);
    ghi = fmax(ghi, red_hi[i]);
    gem = fmax(gem, semax[i]);
  }
  const double span = fmax(fabs(glo), fabs(ghi));
  if (threadIdx.x == 0) tnorm[c] = fmax(span, 1e-100);
  const float flo = (float)(glo - 1e-3 * span - 1e-30), fhi = (float)(ghi + 1e-3 * span + 1e-30);
  const float pivmin = (float)fmax(1e-30, 1e-30 * gem);
  for (int32_t k = threadIdx.x; k < n; k += blockDim.x) {
    float a = flo, z = fhi;
    for (int it = 0; it < 80; ++it) {
      float mid = 0.5f * (a + z);
      if (!(mid > a && mid < z)) break;
      if (sturm32(d, e2, n, mid, pivmin) <= k) a = mid;
      else z = mid;
    }
    lam32[(size_t)c * nmax + k] = 0.5f * (a + z);
  }
}

// ------------------------------------------------- FP64 inverse iteration
constexpr int kMaxCluster = 16;
// Convergence: the last solve (T - sigma I) y = x, ||x|| = 1, grew by ||y|| > 1 / (kResTol ||T||), so
// the returned y / ||y|| has residual ||(T - sigma I) y/||y|| || below kResTol ||T|| (128 eps);
// with the shift that close, the step damps every component outside the target eigenvector by
// at least that residual over the gap to the other eigenvalues.
constexpr double kResTol = 128.0 * 2.2e-16;

__device__ __forceinline__ double hash_unit(uint64_t a, uint64_t b) {
  uint64_t z = css_splitmix64(a * 0x9E3779B97F4A7C15ull + 0x5851F42D4C957F2Dull, b);
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// Phase 1 of the FP64 inverse iteration: one thread per eigenvalue, all threads of a colour
// in lockstep (same loop bounds, fixed four iterations: two at the FP32 shift, two with
// Rayleigh-quotient shifts), so the column-per-thread accesses to U and the scratch F are
// coalesced across a warp.  Eigenvalues whose shift lies within tol of a neighbour's (a
// cluster) and results that did not converge or left their window are flagged for phase 2.
__global__ void __launch_bounds__(128) k_inviter_p1(int32_t kd, int32_t nmax, const int32_t* __restrict__ nblk,
                                                    const double* __restrict__ dd, const double* __restrict__ ee,
                                                    const float* __restrict__ lam32, const double* __restrict__ tnorm,
                                                    double rel_cluster, double* __restrict__ U,
                                                    double* __restrict__ F, double* __restrict__ lam,
                                                    int32_t* __restrict__ flag, const int32_t* __restrict__ gid) {
  const int32_t c = blockIdx.y;
  const uint64_t cseed = gid ? (uint64_t)gid[c] : (uint64_t)c;  // the colour's own id seeds its start vectors
  const int32_t n = nblk[c] * kd;
  const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.x * blockDim.x >= n) return;  // whole block beyond this colour's size
  const double* d = dd + (size_t)c * nmax;
  const double* e = ee + (size_t)c * nmax;
  const float* l32 = lam32 + (size_t)c * nmax;
  double* u = U + (size_t)c * nmax * nmax;
  double* f_u0 = F + (size_t)c * 5 * nmax * nmax;
  double* f_u1 = f_u0 + (size_t)nmax * nmax;
  double* f_u2 = f_u1 + (size_t)nmax * nmax;
  double* f_x = f_u2 + (size_t)nmax * nmax;
  int32_t* fl = flag + (size_t)c * nmax;
  const double tn = tnorm[c];
  const double tol = rel_cluster * tn;
  const double pivmin = 2.2e-16 * tn;
  const double res_tol = kResTol * tn;
  const bool valid = k < n;
  bool in_cluster = false;
  double win_lo = 0.0, win_hi = 0.0, sigma = 0.0;
  if (valid) {
    const double lk = (double)l32[k];
    const double g_lo = k > 0 ? lk - (double)l32[k - 1] : tn;
    const double g_hi = k + 1 < n ? (double)l32[k + 1] - lk : tn;
    in_cluster = g_lo <= tol || g_hi <= tol;
    win_lo = lk - 0.25 * g_lo - 2e-6 * tn;
    win_hi = lk + 0.25 * g_hi + 2e-6 * tn;
    sigma = lk;
  }
  const bool work = valid && !in_cluster;
  // start vector, normalised
  double nrm = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    const double x = work ? hash_unit(cseed * 1000003ull + (uint64_t)k, (uint64_t)i) : 0.0;
    if (work) f_x[(size_t)i * nmax + k] = x;
    nrm += x * x;
  }
  double inv = work ? 1.0 / sqrt(nrm) : 0.0;
  double growth = 0.0;
  for (int it = 0; it < 4; ++it) {
    // factor T - sigma I with partial pivoting and eliminate on x in the same sweep; the rows
    // of U are stored, x is overwritten by L^-1 P x (scaled by inv)
    double cd = d[0] - sigma, cs = n > 1 ? e[0] : 0.0;
    double xc = work ? f_x[k] * inv : 0.0;  // current row's right-hand side
    for (int32_t i = 0; i + 1 < n; ++i) {
      const double sub = e[i], dg = d[i + 1] - sigma, sup = (i + 2 < n) ? e[i + 1] : 0.0;
      const double xn = work ? f_x[(size_t)(i + 1) * nmax + k] * inv : 0.0;
      double u0, u1, u2, rhs_i, ncd, ncs, nx;
      if (fabs(cd) >= fabs(sub)) {
        if (fabs(cd) < pivmin) cd = cd >= 0 ? pivmin : -pivmin;
        u0 = 1.0 / cd;  // the pivot's reciprocal serves the multiplier and the back substitution
        const double l = sub * u0;
        u1 = cs;
        u2 = 0.0;
        rhs_i = xc;
        ncd = dg - l * cs;
        ncs = sup;
        nx = xn - l * xc;
      } else {
        u0 = 1.0 / sub;
        const double l = cd * u0;
        u1 = dg;
        u2 = sup;
        rhs_i = xn;
        ncd = cs - l * dg;
        ncs = -l * sup;
        nx = xc - l * xn;
      }
      if (work) {
        f_u0[(size_t)i * nmax + k] = u0;
        f_u1[(size_t)i * nmax + k] = u1;
        f_u2[(size_t)i * nmax + k] = u2;
        f_x[(size_t)i * nmax + k] = rhs_i;
      }
      cd = ncd;
      cs = ncs;
      xc = nx;
    }
    if (fabs(cd) < pivmin) cd = cd >= 0 ? pivmin : -pivmin;
    // backward substitution U y = x, then the norm
    double y1 = 0.0, y2 = 0.0, ss = 0.0;
    for (int32_t i = n - 1; i >= 0; --i) {
      double r, u0;  // u0: the reciprocal of the row's pivot
      if (i == n - 1) {
        r = xc;
        u0 = 1.0 / cd;
      } else {
        r = work ? f_x[(size_t)i * nmax + k] : 0.0;
        u0 = work ? f_u0[(size_t)i * nmax + k] : 1.0;
        if (work) r -= f_u1[(size_t)i * nmax + k] * y1;
        if (work && i + 2 < n) r -= f_u2[(size_t)i * nmax + k] * y2;
      }
      const double y = work ? r * u0 : 0.0;
      if (work) f_x[(size_t)i * nmax + k] = y;
      ss += y * y;
      y2 = y1;
      y1 = y;
    }
    growth = sqrt(ss);
    inv = work ? 1.0 / growth : 0.0;
    // Rayleigh quotient of the normalised vector
    double rq = 0.0, prev = 0.0;
    for (int32_t i = 0; i < n; ++i) {
      const double xi = work ? f_x[(size_t)i * nmax + k] * inv : 0.0;
      rq += xi * (d[i] * xi + 2.0 * (i > 0 ? e[i - 1] * prev : 0.0));
      prev = xi;
    }
    if (it >= 1) sigma = rq;
  }
  if (!valid) return;
  const bool ok = work && growth * res_tol > 1.0 && sigma >= win_lo && sigma <= win_hi;
  fl[k] = ok ? 0 : 1;
  if (!ok) return;
  for (int32_t i = 0; i < n; ++i) u[(size_t)i * nmax + k] = f_x[(size_t)i * nmax + k] * inv;
  lam[(size_t)c * nmax + k] = sigma;
}

// Phase 2 of the FP64 inverse iteration: one warp per cluster of close shifts (or per single
// eigenvalue that phase 1 flagged).  Lane j < kc owns member k0 + j; its iterate is column k0 + j
// of the scratch X and its LU factors columns k0 + j of U0..U2, so the lanes of a warp touch
// contiguous addresses of a row.  Every member solves with its own shift, then the members are
// orthonormalised by modified Gram-Schmidt in member order (simultaneous inverse iteration);
// Rayleigh-Ritz inside the cluster gives the final pairs.  Every sweep over the rows loads a
// batch of rows before the batch's dependent arithmetic, so one warp keeps several loads in
// flight.
constexpr int kCB = 8;  // rows per batch

struct ClusterCols {
  const double* d;
  const double* e;
  double* u0;
  double* u1;
  double* u2;
  double* x;
  int32_t n, nmax;
};

// LU with partial pivoting of T - sigma I fused with the forward elimination of column col of
// X (scaled by scl), then the back substitution U y = x; y overwrites the column.  Returns ||y||.
// Lanes with st == false compute but store nothing.
__device__ double cl_solve(const ClusterCols& m, int32_t col, double sigma, double scl, double pivmin, bool st) {
  const int32_t n = m.n, nmax = m.nmax;
  double cd = m.d[0] - sigma, cs = n > 1 ? m.e[0] : 0.0;
  double xc = m.x[col] * scl;
  for (int32_t i0 = 0; i0 + 1 < n; i0 += kCB) {
    double sub[kCB], dg[kCB], sup[kCB], xn[kCB];
#pragma unroll
    for (int q = 0; q < kCB; ++q) {
      const int32_t i = i0 + q;
      const bool ok = i + 1 < n;
      sub[q] = ok ? m.e[i] : 1.0;
      dg[q] = ok ? m.d[i + 1] - sigma : 0.0;
      sup[q] = (i + 2 < n) ? m.e[i + 1] : 0.0;
      xn[q] = ok ? m.x[(size_t)(i + 1) * nmax + col] * scl : 0.0;
    }
#pragma unroll
    for (int q = 0; q < kCB; ++q) {
      const int32_t i = i0 + q;
      if (i + 1 >= n) break;
      double u0, u1, u2, rhs, ncd, ncs, nx;
      if (fabs(cd) >= fabs(sub[q])) {
        if (fabs(cd) < pivmin) cd = cd >= 0 ? pivmin : -pivmin;
        u0 = 1.0 / cd;  // the pivot's reciprocal serves the multiplier and the back substitution
        const double l = sub[q] * u0;
        u1 = cs;
        u2 = 0.0;
        rhs = xc;
        ncd = dg[q] - l * cs;
        ncs = sup[q];
        nx = xn[q] - l * xc;
      } else {
        u0 = 1.0 / sub[q];
        const double l = cd * u0;
        u1 = dg[q];
        u2 = sup[q];
        rhs = xn[q];
        ncd = cs - l * dg[q];
        ncs = -l * sup[q];
        nx = xc - l * xn[q];
      }
      if (st) {
        m.u0[(size_t)i * nmax + col] = u0;
        m.u1[(size_t)i * nmax + col] = u1;
        m.u2[(size_t)i * nmax + col] = u2;
        m.x[(size_t)i * nmax + col] = rhs;
      }
      cd = ncd;
      cs = ncs;
      xc = nx;
    }
  }
  if (fabs(cd) < pivmin) cd = cd >= 0 ? pivmin : -pivmin;
  // back substitution, rows n-1 down to 0, in batches
  double y1 = xc / cd, y2 = 0.0;
  double ss = y1 * y1;
  if (st) m.x[(size_t)(n - 1) * nmax + col] = y1;
  for (int32_t i0 = n - 2; i0 >= 0; i0 -= kCB) {
    double r[kCB], a0[kCB], a1[kCB], a2[kCB];
#pragma unroll
    for (int q = 0; q < kCB; ++q) {
      const int32_t i = i0 - q;
      const bool ok = i >= 0;
      const size_t o = (size_t)(ok ? i : 0) * nmax + col;
      r[q] = ok ? m.x[o] : 0.0;
      a0[q] = ok ? m.u0[o] : 1.0;
      a1[q] = ok ? m.u1[o] : 0.0;
      a2[q] = ok ? m.u2[o] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < kCB; ++q) {
      const int32_t i = i0 - q;
      if (i < 0) break;
      const double y = (r[q] - a1[q] * y1 - a2[q] * y2) * a0[q];
      if (st) m.x[(size_t)i * nmax + col] = y;
      ss += y * y;
      y2 = y1;
      y1 = y;
    }
  }
  return sqrt(ss);
}

// Work list of phase 2: (colour, first member, members) of every cluster of close shifts (runs
// cut every kMaxCluster members) that holds a member phase 1 did not finish; one thread per shift,
// the order of the list does not matter (every item writes only its own columns)
__global__ void k_cl_items(int32_t kd, int32_t nmax, const int32_t* __restrict__ nblk,
                           const float* __restrict__ lam32, const double* __restrict__ tnorm, double rel_cluster,
                           const int32_t* __restrict__ flag, int32_t* __restrict__ count, int4* __restrict__ items) {
  const int32_t c = blockIdx.y;
  const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t n = nblk[c] * kd;
  if (k >= n) return;
  const float* l32 = lam32 + (size_t)c * nmax;
  const double tol = rel_cluster * tnorm[c];
  int32_t s = k;
  while (s > 0 && (double)l32[s] - (double)l32[s - 1] <= tol) --s;
  if ((k - s) % kMaxCluster != 0) return;  // not the first member of a cluster
  int32_t k1 = k;
  while (k1 + 1 < n && (double)l32[k1 + 1] - (double)l32[k1] <= tol && k1 + 1 - k < kMaxCluster) ++k1;
  bool any = false;
  for (int32_t kk = k; kk <= k1; ++kk) any = any || flag[(size_t)c * nmax + kk] != 0;
  if (!any) return;  // phase 1 finished every member
  items[atomicAdd(count, 1)] = make_int4(c, k, k1 - k + 1, 0);
}

// one warp per work item of k_cl_items (warps past the list's length return)
__global__ void __launch_bounds__(256) k_inviter_cl(int32_t kd, int32_t nmax, const int32_t* __restrict__ nblk,
                                                    const double* __restrict__ dd, const double* __restrict__ ee,
                                                    const float* __restrict__ lam32,
                                                    const double* __restrict__ tnorm, double rel_cluster,
                                                    double* __restrict__ U, double* __restrict__ F,
                                                    double* __restrict__ lam, int32_t* __restrict__ status,
                                                    const int32_t* __restrict__ gid, const int32_t* __restrict__ count,
                                                    const int4* __restrict__ items) {
  __shared__ double sC[8][kMaxCluster][kMaxCluster + 1];
  __shared__ double sV[8][kMaxCluster][kMaxCluster + 1];
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int32_t item = blockIdx.x * (blockDim.x >> 5) + warp;
  if (item >= *count) return;  // uniform over the warp
  const int4 it4 = items[item];
  const int32_t c = it4.x, k0 = it4.y, kc = it4.z, k1 = k0 + kc - 1;
  const uint64_t cseed = gid ? (uint64_t)gid[c] : (uint64_t)c;
  const int32_t n = nblk[c] * kd;
  const float* l32 = lam32 + (size_t)c * nmax;
  double* u = U + (size_t)c * nmax * nmax;
  ClusterCols m;
  m.d = dd + (size_t)c * nmax;
  m.e = ee + (size_t)c * nmax;
  m.u0 = F + (size_t)c * 5 * nmax * nmax;
  m.u1 = m.u0 + (size_t)nmax * nmax;
  m.u2 = m.u1 + (size_t)nmax * nmax;
  m.x = m.u2 + (size_t)nmax * nmax;
  m.n = n;
  m.nmax = nmax;
  const double tn = tnorm[c];
  const double pivmin = 2.2e-16 * tn;
  const double res_tol = kResTol * tn;
  int32_t failed = 0;
  {
    {
      const bool act = lane < kc;
      const int32_t col = k0 + (act ? lane : 0);  // idle lanes shadow member 0 and store nothing
      const double g_lo = k0 > 0 ? (double)l32[k0] - (double)l32[k0 - 1] : tn;
      const double g_hi = k1 + 1 < n ? (double)l32[k1 + 1] - (double)l32[k1] : tn;
      const double win_lo = (double)l32[k0] - 0.25 * g_lo - 2e-6 * tn;
      const double win_hi = (double)l32[k1] + 0.25 * g_hi + 2e-6 * tn;
      double lamj = 0.0;
      bool ok_all = false;
      for (int attempt = 0; attempt < 3 && !ok_all; ++attempt) {
        // start vectors (norm folded into the first solve's right-hand side)
        double nrm = 0.0;
        for (int32_t i0 = 0; i0 < n; i0 += kCB) {
#pragma unroll
          for (int q = 0; q < kCB; ++q) {
            const int32_t i = i0 + q;
            if (i < n) {
              const double x = hash_unit(cseed * 1000003ull + (uint64_t)col + 7919ull * attempt, (uint64_t)i);
              if (act) m.x[(size_t)i * nmax + col] = x;
              nrm += x * x;
            }
          }
        }
        double scl = 1.0 / sqrt(nrm);
        double sigma = (double)l32[col];
        for (int it = 0; it < 8; ++it) {
          const double growth = cl_solve(m, col, sigma, scl, pivmin, act);
          // modified Gram-Schmidt in member order; pass s subtracts the projection on member s-1
          // (coefficient from pass s-1) and takes the inner products with member s
          double cprev = 0.0, nrm2 = 1.0;
          for (int32_t s = 0; s < kc; ++s) {
            double dj = 0.0;
            for (int32_t i0 = 0; i0 < n; i0 += kCB) {
              double v[kCB];
#pragma unroll
              for (int q = 0; q < kCB; ++q) v[q] = (i0 + q < n) ? m.x[(size_t)(i0 + q) * nmax + col] : 0.0;
#pragma unroll
              for (int q = 0; q < kCB; ++q) {
                if (s > 0) {
                  const double xp = __shfl_sync(FULL, v[q], s - 1);
                  if (lane >= s) v[q] = fma(-cprev, xp, v[q]);
                }
                const double xs = __shfl_sync(FULL, v[q], s);
                dj = fma(xs, v[q], dj);
              }
              if (s > 0 && act && lane >= s) {
#pragma unroll
                for (int q = 0; q < kCB; ++q)
                  if (i0 + q < n) m.x[(size_t)(i0 + q) * nmax + col] = v[q];
              }
            }
            const double ds = __shfl_sync(FULL, dj, s);
            if (lane == s) nrm2 = ds;
            cprev = lane > s ? dj / ds : 0.0;
          }
          // normalise and take the Rayleigh quotient x^T T x
          const double r = 1.0 / sqrt(nrm2);
          double rq = 0.0, prev = 0.0;
          for (int32_t i0 = 0; i0 < n; i0 += kCB) {
            double v[kCB], dv[kCB], ev[kCB];
#pragma unroll
            for (int q = 0; q < kCB; ++q) {
              const int32_t i = i0 + q;
              v[q] = i < n ? m.x[(size_t)i * nmax + col] * r : 0.0;
              dv[q] = i < n ? m.d[i] : 0.0;
              ev[q] = (i > 0 && i < n) ? m.e[i - 1] : 0.0;
            }
#pragma unroll
            for (int q = 0; q < kCB; ++q) {
              rq += v[q] * (dv[q] * v[q] + 2.0 * ev[q] * prev);
              prev = v[q];
              if (act && i0 + q < n) m.x[(size_t)(i0 + q) * nmax + col] = v[q];
            }
          }
          scl = 1.0;
          if (it >= 1) sigma = rq;
          const bool conv = it >= 2 && growth * res_tol > 1.0;
          if (__all_sync(FULL, !act || conv)) break;
        }
        lamj = sigma;
        if (kc > 1) {
          // Rayleigh-Ritz inside the cluster: C = X^T T X, column j accumulated by lane j
          double cc[kMaxCluster];
#pragma unroll
          for (int a = 0; a < kMaxCluster; ++a) cc[a] = 0.0;
          double xprev = 0.0;
          double xcur = m.x[col];
          for (int32_t i0 = 0; i0 < n; i0 += kCB) {
            double xnx[kCB], dv[kCB], elo[kCB], ehi[kCB];
#pragma unroll
            for (int q = 0; q < kCB; ++q) {
              const int32_t i = i0 + q;
              xnx[q] = (i + 1 < n) ? m.x[(size_t)(i + 1) * nmax + col] : 0.0;
              dv[q] = i < n ? m.d[i] : 0.0;
              elo[q] = (i > 0 && i < n) ? m.e[i - 1] : 0.0;
              ehi[q] = (i + 1 < n) ? m.e[i] : 0.0;
            }
#pragma unroll
            for (int q = 0; q < kCB; ++q) {
              const double tx = dv[q] * xcur + elo[q] * xprev + ehi[q] * xnx[q];
#pragma unroll
              for (int a = 0; a < kMaxCluster; ++a) {
                const double xa = __shfl_sync(FULL, xcur, a);
                if (a < kc) cc[a] = fma(xa, tx, cc[a]);
              }
              xprev = xcur;
              xcur = xnx[q];
            }
          }
          if (act)
#pragma unroll
            for (int a = 0; a < kMaxCluster; ++a)
              if (a < kc) sC[warp][a][lane] = cc[a];
          __syncwarp();
          if (lane == 0) {
            double (*C)[kMaxCluster + 1] = sC[warp];
            double (*V)[kMaxCluster + 1] = sV[warp];
            for (int32_t a = 0; a < kc; ++a)
              for (int32_t q = 0; q < kc; ++q) V[a][q] = a == q ? 1.0 : 0.0;
            for (int32_t a = 0; a < kc; ++a)
              for (int32_t q = a + 1; q < kc; ++q) {
                const double t = 0.5 * (C[a][q] + C[q][a]);
                C[a][q] = t;
                C[q][a] = t;
              }
            for (int sweep = 0; sweep < 30; ++sweep) {  // cyclic Jacobi
              double off = 0.0, on = 0.0;
              for (int32_t a = 0; a < kc; ++a)
                for (int32_t q = 0; q < kc; ++q) (a == q ? on : off) += C[a][q] * C[a][q];
              if (off <= 1e-32 * on || off == 0.0) break;
              for (int32_t a = 0; a < kc; ++a)
                for (int32_t q = a + 1; q < kc; ++q) {
                  if (C[a][q] == 0.0) continue;
                  const double theta = (C[q][q] - C[a][a]) / (2.0 * C[a][q]);
                  const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                  const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
                  for (int32_t r2 = 0; r2 < kc; ++r2) {
                    const double ca = C[r2][a], cb = C[r2][q];
                    C[r2][a] = cs * ca - sn * cb;
                    C[r2][q] = sn * ca + cs * cb;
                  }
                  for (int32_t r2 = 0; r2 < kc; ++r2) {
                    const double ca = C[a][r2], cb = C[q][r2];
                    C[a][r2] = cs * ca - sn * cb;
                    C[q][r2] = sn * ca + cs * cb;
                  }
                  for (int32_t r2 = 0; r2 < kc; ++r2) {
                    const double va = V[r2][a], vb = V[r2][q];
                    V[r2][a] = cs * va - sn * vb;
                    V[r2][q] = sn * va + cs * vb;
                  }
                }
            }
          }
          __syncwarp();
          lamj = act ? sC[warp][lane][lane] : 0.0;
        }
        ok_all = __all_sync(FULL, !act || (lamj >= win_lo && lamj <= win_hi));
        if (!ok_all && attempt < 2) continue;
        // write the eigenvectors: X (rotated by V inside a cluster) into U
        double vcol[kMaxCluster];
#pragma unroll
        for (int a = 0; a < kMaxCluster; ++a) vcol[a] = (kc > 1 && act && a < kc) ? sV[warp][a][lane] : 0.0;
        for (int32_t i0 = 0; i0 < n; i0 += kCB) {
          double v[kCB];
#pragma unroll
          for (int q = 0; q < kCB; ++q) v[q] = (i0 + q < n) ? m.x[(size_t)(i0 + q) * nmax + col] : 0.0;
#pragma unroll
          for (int q = 0; q < kCB; ++q) {
            double o = v[q];
            if (kc > 1) {
              o = 0.0;
#pragma unroll
              for (int a = 0; a < kMaxCluster; ++a) {
                const double xa = __shfl_sync(FULL, v[q], a);
                if (a < kc) o = fma(xa, vcol[a], o);
              }
            }
            if (act && i0 + q < n) u[(size_t)(i0 + q) * nmax + col] = o;
          }
        }
        if (act) lam[(size_t)c * nmax + col] = lamj;
        if (!ok_all) failed = 1;
        __syncwarp();
      }
    }
  }
  if (failed) atomicOr(&status[c], 1);  // an eigenvalue outside its window after every attempt
}

// Y[k][col] = sum_i U[i][k] X[i][col], w[k] = ||Y[k]||^2 (one thread per k)
__global__ void k_ritz_y(int32_t kd, int32_t b, int32_t nmax, const int32_t* __restrict__ nblk,
                         const double* __restrict__ U, const double* __restrict__ X, double* __restrict__ Y,
                         double* __restrict__ wgt) {
  extern __shared__ double shx[];
  const int32_t c = blockIdx.y;
  const int32_t n = nblk[c] * kd;
  const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  const double* u = U + (size_t)c * nmax * nmax;
  const double* x = X + (size_t)c * nmax * b;
  double acc[CSS_MAX_B];
#pragma unroll
  for (int a = 0; a < CSS_MAX_B; ++a) acc[a] = 0.0;
  const int32_t CH = 64;
  for (int32_t i0 = 0; i0 < n; i0 += CH) {
    const int32_t ie = min(n, i0 + CH);
    __syncthreads();
    for (int32_t t = threadIdx.x; t < (ie - i0) * b; t += blockDim.x) shx[t] = x[(size_t)i0 * b + t];
    __syncthreads();
    if (k < n)
      for (int32_t i = i0; i < ie; ++i) {
        const double uk = u[(size_t)i * nmax + k];
#pragma unroll
        for (int a = 0; a < CSS_MAX_B; ++a)
          if (a < b) acc[a] = fma(uk, shx[(i - i0) * b + a], acc[a]);
      }
  }
  if (k < n) {
    double w = 0.0;
#pragma unroll
    for (int a = 0; a < CSS_MAX_B; ++a)
      if (a < b) {
        Y[((size_t)c * nmax + k) * b + a] = acc[a];
        w = fma(acc[a], acc[a], w);
      }
    wgt[(size_t)c * nmax + k] = w;
  } else if (k < nmax) {
    wgt[(size_t)c * nmax + k] = 0.0;
  }
}

// Zt[i][col] = sum_k U[i][k] g(lam_k) Y[k][col] (one thread per row i).  fn bit 1: g = x^(-1/2)
// (inverse square root of an overlap, positive Ritz values; NaN otherwise) instead of the Fermi
// function; bit 0: g multiplied by x (the energy-weighted density matrix, T_c Z_c).
__global__ void k_zt(int32_t kd, int32_t b, int32_t nmax, const int32_t* __restrict__ nblk,
                     const int32_t* __restrict__ sys_of_colour, const double* __restrict__ mu,
                     const double* __restrict__ kT, const double* __restrict__ U, const double* __restrict__ lam,
                     const double* __restrict__ Y, double* __restrict__ Z, int fn) {
  extern __shared__ double shy[];
  const int32_t c = blockIdx.y;
  const int32_t n = nblk[c] * kd;
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const double* u = U + (size_t)c * nmax * nmax;
  const int32_t s = sys_of_colour[c];
  const double m_ = mu[s], t_ = kT[s];
  double acc[CSS_MAX_B];
#pragma unroll
  for (int a = 0; a < CSS_MAX_B; ++a) acc[a] = 0.0;
  const int32_t CH = 64;
  for (int32_t k0 = 0; k0 < n; k0 += CH) {
    const int32_t ke = min(n, k0 + CH);
    __syncthreads();
    for (int32_t t = threadIdx.x; t < (ke - k0) * b; t += blockDim.x) {
      const int32_t kk = k0 + t / b;
      const double l = lam[(size_t)c * nmax + kk];
      double fw = (fn & 2) ? (l > 0.0 ? 1.0 / sqrt(l) : __longlong_as_double(0x7ff8000000000000ll))
                           : css_fermi_dirac(l, m_, t_);
      if (fn & 1) fw *= l;
      shy[t] = fw * Y[((size_t)c * nmax) * b + (size_t)k0 * b + t];
    }
    __syncthreads();
    if (i < n)
      for (int32_t kk = k0; kk < ke; ++kk) {
        const double uk = u[(size_t)i * nmax + kk];
#pragma unroll
        for (int a = 0; a < CSS_MAX_B; ++a)
          if (a < b) acc[a] = fma(uk, shy[(kk - k0) * b + a], acc[a]);
      }
  }
  if (i < nmax) {
#pragma unroll
    for (int a = 0; a < CSS_MAX_B; ++a)
      if (a < b) Z[((size_t)c * nmax + i) * b + a] = (i < n) ? acc[a] : 0.0;
  }
}

// diagnostics: copy the FP32 shifts over the eigenvalues
__global__ void k_shifts_out(int32_t nmax, const float* __restrict__ lam32, double* __restrict__ lam) {
  for (int32_t k = threadIdx.x; k < nmax; k += blockDim.x)
    lam[(size_t)blockIdx.x * nmax + k] = (double)lam32[(size_t)blockIdx.x * nmax + k];
}

}  // namespace

css_status css_eigen_ritz(css_ctx* ctx, const EigArgs& a, cudaStream_t st) {
  const int32_t nc = a.n_col, b = a.b, nmax = a.m * b, ldb = 2 * b + 1;
  k_band_build<<<nc, 256, 0, st>>>(b, a.m, nmax, ldb, a.Ablk, a.Bblk, a.nblk, a.AB);
  CSS_LAUNCHED(ctx);
  CSS_CU(ctx, cudaMemsetAsync(a.status, 0, sizeof(int32_t) * nc, st));
  k_band_to_tri<<<nc, 1024, 0, st>>>(b, nmax, ldb, a.rcap, a.nblk, a.AB, a.RV, a.RT, a.RR0, a.sweep_off, a.d, a.e,
                                     a.status);
  CSS_LAUNCHED(ctx);
  if (a.B0)
    k_x0_b0<<<nc, 256, 0, st>>>(b, nmax, a.B0, a.X0);
  else
    k_x0<<<nc, 256, 0, st>>>(b, nmax, a.cnt, a.X0);
  CSS_LAUNCHED(ctx);
  k_apply_refl<true><<<nc, 1024, 0, st>>>(b, b, nmax, a.rcap, a.nblk, a.RV, a.RT, a.RR0, a.sweep_off, a.X0);
  CSS_LAUNCHED(ctx);
  const size_t sh = 2 * (size_t)nmax * sizeof(float);
  if (sh > 48 * 1024) CSS_CU(ctx, cudaFuncSetAttribute(k_bisect32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
  k_bisect32<<<nc, 256, sh, st>>>(b, nmax, a.nblk, a.d, a.e, a.lam32, a.tnorm);
  CSS_LAUNCHED(ctx);
  k_inviter_p1<<<dim3((unsigned)css_ceil_div(nmax, 128), (unsigned)nc), 128, 0, st>>>(
      b, nmax, a.nblk, a.d, a.e, a.lam32, a.tnorm, 1e-4, a.U, a.F, a.lam, a.flag, a.gid);
  CSS_LAUNCHED(ctx);
  // phase 2 on a compact list: one warp per flagged cluster of any colour
  int32_t* cl_count;
  int4* cl_items;
  CSS_TRY(css_ws(ctx, "e_cl_count", 256, (void**)&cl_count));
  CSS_TRY(css_ws(ctx, "e_cl_items", (size_t)nc * nmax * sizeof(int4), (void**)&cl_items));
  CSS_CU(ctx, cudaMemsetAsync(cl_count, 0, sizeof(int32_t), st));
  k_cl_items<<<dim3((unsigned)css_ceil_div(nmax, 128), (unsigned)nc), 128, 0, st>>>(b, nmax, a.nblk, a.lam32, a.tnorm,
                                                                                   1e-4, a.flag, cl_count, cl_items);
  CSS_LAUNCHED(ctx);
  k_inviter_cl<<<(unsigned)css_ceil_div((int64_t)nc * nmax, 8), 256, 0, st>>>(
      b, nmax, a.nblk, a.d, a.e, a.lam32, a.tnorm, 1e-4, a.U, a.F, a.lam, a.status, a.gid, cl_count, cl_items);
  CSS_LAUNCHED(ctx);
  if (ctx->debug_eig == 1) {
    k_shifts_out<<<nc, 256, 0, st>>>(nmax, a.lam32, a.lam);
    CSS_LAUNCHED(ctx);
  }
  dim3 g((unsigned)css_ceil_div(nmax, 128), (unsigned)nc);
  k_ritz_y<<<g, 128, 64 * b * sizeof(double), st>>>(b, b, nmax, a.nblk, a.U, a.X0, a.Y, a.wgt);
  CSS_LAUNCHED(ctx);
  return CSS_OK;
}

css_status css_eigen_z(css_ctx* ctx, const EigArgs& a, const int32_t* sys_of_colour, const double* mu,
                       const double* kT, double* Z, cudaStream_t st, int fn) {
  const int32_t nc = a.n_col, b = a.b, nmax = a.m * b;
  dim3 g((unsigned)css_ceil_div(nmax, 128), (unsigned)nc);
  k_zt<<<g, 128, 64 * b * sizeof(double), st>>>(b, b, nmax, a.nblk, sys_of_colour, mu, kT, a.U, a.lam, a.Y, Z,
                                                 fn);
  CSS_LAUNCHED(ctx);
  k_apply_refl<false><<<nc, 1024, 0, st>>>(b, b, nmax, a.rcap, a.nblk, a.RV, a.RT, a.RR0, a.sweep_off, Z);
  CSS_LAUNCHED(ctx);
  return CSS_OK;
}

css_status css_eigen_project(css_ctx* ctx, const EigArgs& a, double* V, double* YV, double* scratch, cudaStream_t st) {
  const int32_t nc = a.n_col, b = a.b, nmax = a.m * b;
  k_apply_refl<true><<<nc, 1024, 0, st>>>(b, b, nmax, a.rcap, a.nblk, a.RV, a.RT, a.RR0, a.sweep_off, V);
  CSS_LAUNCHED(ctx);
  dim3 g((unsigned)css_ceil_div(nmax, 128), (unsigned)nc);
  k_ritz_y<<<g, 128, 64 * b * sizeof(double), st>>>(b, b, nmax, a.nblk, a.U, V, YV, scratch);
  CSS_LAUNCHED(ctx);
  return CSS_OK;
}
