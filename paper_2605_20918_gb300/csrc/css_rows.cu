// Row passes of one FP32 block-Lanczos step for block widths 17..24 (paper: the three-term
// recurrence and block QR of the block-Lanczos paragraph after Eq. 4).  Each pass streams the
// N x w Krylov blocks once and applies, per colour c, a small b x b matrix and/or accumulates a
// b x b Gram matrix:
//   S1    W0 = W - Q_{j-1} B_{j-1}^T (not stored);  Kq = Q_j^T W0,  Kp = Q_{j-1}^T W0
//   S3    W1 = W - Q_j Kq - Q_{j-1} (B_{j-1}^T + Kp), stored over W;  Gram W1^T W1
//   TRIG  Gram of W1 M (M = R0^-1 or R0^-1 R1^-1 of the shifted CholeskyQR3), not stored
//   TRI   Q_{j+1} = W1 M (M = R0^-1 R1^-1 R2^-1), stored
// so a step reads the three N x w blocks twice and W1 three more times and writes two blocks
// (11 passes; the CholeskyQR intermediates W1 R^-1 are recomputed, not stored).
//
// Thread (colour c of the CTA's group, column k) holds column k of the colour's b x b matrix
// in registers and row k of its Gram accumulator.  Rows are staged in shared memory with the
// colour's columns padded to 24 (cp.async, a four-stage ring of 8-row sub-chunks), so a thread
// reads the b values of a row of its colour with six 16-byte broadcast loads: four FMAs per
// shared-memory load for the products and for the Grams.  Gram sums are taken in FP32 over 32
// rows and added into an unevaluated hi + lo pair (TwoSum), widened to FP64 once per CTA; the
// per-CTA partials are summed in FP64 in a fixed order (k_reduce), so every run is bitwise
// reproducible.
#include "css_lanczos.cuh"

namespace {

constexpr int RP_KP = 24;      // padded colour width
constexpr int RP_RS = 8;       // rows per sub-chunk
constexpr int RP_NST = 4;      // cp.async ring depth (sub-chunks)
constexpr int RP_RCH = 1024;   // rows per CTA (the chunking of the Gram partials)
constexpr int RP_GRAM_RS = 32; // rows per FP32 Gram sum before the compensated update

enum { RP_S1 = 0, RP_S3 = 1, RP_TRIG = 2, RP_TRI = 3 };

struct RpArgs {
  int64_t N;
  int32_t b, ws, ncb, cb0, first;
  const float* Q;   // Q_j            (S1, S3)
  const float* Qp;  // Q_{j-1}        (S1, S3; unused when first)
  const float* W;   // W or W1        (all)
  float* OUT;       // S3: W1 (may be W), TRI: Q_{j+1}
  const double* M1;     // S1: B_{j-1} [cb0 + lc] (used transposed); S3: Kq [lc]; TRIG/TRI: M [lc]
  const double* Bprev;  // S3: B_{j-1} [cb0 + lc]
  const double* Kp;     // S3: Kp [lc]
  double* part1;        // Gram partials [chunk][lc][b][b]: S1 Kq, S3 / TRIG the Gram
  double* part2;        // S1 Kp
  int reorth;
};

// arrays staged per sub-chunk: S1 Q, Qp, W; S3 Q, Qp, W; TRIG / TRI W
// colours per CTA: 8 per thread set in S1 (two Grams, 384 threads), 10 in S3 (two matrix
// columns and a Gram per thread need more registers: 240 threads), 16 in the single-matrix passes
template <int MODE>
struct RpCfg {
  static constexpr int NSET = MODE == RP_S1 ? 2 : 1;  // S1: one thread set per Gram
  static constexpr int CG = MODE == RP_S1 ? 8 : MODE == RP_S3 ? 10 : 16;
  static constexpr int THREADS = NSET * CG * RP_KP;
  static constexpr int NA = (MODE == RP_S1 || MODE == RP_S3) ? 3 : 1;
  static constexpr int PITCH = CG * RP_KP;            // floats per staged row
  static constexpr int STAGE = NA * RP_RS * PITCH;    // floats per stage
  static constexpr bool GRAM = MODE != RP_TRI;
  static constexpr size_t SMEM = sizeof(float) * ((size_t)RP_NST * STAGE + 2 * RP_RS * PITCH);
};

__device__ __forceinline__ void cp4(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// sum_l x[l] m[l] over the 24 padded columns of a staged row (six broadcast 16-byte loads),
// in four interleaved partial sums (short dependency chains), combined in a fixed order
__device__ __forceinline__ float row_dot(const float* x, const float (&m)[RP_KP]) {
  float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
#pragma unroll
  for (int q = 0; q < RP_KP / 4; ++q) {
    const float4 v = *reinterpret_cast<const float4*>(x + 4 * q);
    s0 = fmaf(v.x, m[4 * q], s0);
    s1 = fmaf(v.y, m[4 * q + 1], s1);
    s2 = fmaf(v.z, m[4 * q + 2], s2);
    s3 = fmaf(v.w, m[4 * q + 3], s3);
  }
  return (s0 + s1) + (s2 + s3);
}
__device__ __forceinline__ void row_axpy(const float* y, float a, float (&g)[RP_KP]) {
#pragma unroll
  for (int q = 0; q < RP_KP / 4; ++q) {
    const float4 v = *reinterpret_cast<const float4*>(y + 4 * q);
    g[4 * q] = fmaf(a, v.x, g[4 * q]);
    g[4 * q + 1] = fmaf(a, v.y, g[4 * q + 1]);
    g[4 * q + 2] = fmaf(a, v.z, g[4 * q + 2]);
    g[4 * q + 3] = fmaf(a, v.w, g[4 * q + 3]);
  }
}
// Knuth's TwoSum of the FP32 chunk sums into (hi, lo)
__device__ __forceinline__ void gram_flush(float (&g)[RP_KP], float (&hi)[RP_KP], float (&lo)[RP_KP]) {
#pragma unroll
  for (int l = 0; l < RP_KP; ++l) {
    const float x = g[l];
    const float t = __fadd_rn(hi[l], x);
    const float z = __fsub_rn(t, hi[l]);
    lo[l] = __fadd_rn(lo[l], __fadd_rn(__fsub_rn(hi[l], __fsub_rn(t, z)), __fsub_rn(x, z)));
    hi[l] = t;
    g[l] = 0.0f;
  }
}

template <int MODE>
__global__ void __launch_bounds__(RpCfg<MODE>::THREADS, 1) k_rowpass(const RpArgs a) {
  using C = RpCfg<MODE>;
  extern __shared__ __align__(16) float rsm[];
  float* stage = rsm;                          // [NST][NA][RS][PITCH]
  float* sO = rsm + (size_t)RP_NST * C::STAGE;  // [2][RS][PITCH]
  const int tid = threadIdx.x;
  const int set = tid / (C::CG * RP_KP), t2 = tid - set * (C::CG * RP_KP);
  const int cl = t2 / RP_KP, k = t2 - cl * RP_KP;
  const int32_t lc = blockIdx.y * C::CG + cl;
  const bool valid = lc < a.ncb && k < a.b;
  const size_t col = valid ? (size_t)lc * a.b + k : 0;
  const int soff = cl * RP_KP + k;  // this thread's element in a staged row
  const int64_t rbeg = (int64_t)blockIdx.x * RP_RCH, rend = min(a.N, rbeg + RP_RCH);
  const int nsub = (int)((rend - rbeg + RP_RS - 1) / RP_RS);
  const bool first = a.first != 0;
  // this thread's column of the colour's matrices (zero beyond b and for idle threads)
  float m1[RP_KP], m2[RP_KP];
#pragma unroll
  for (int l = 0; l < RP_KP; ++l) {
    float x = 0.0f, y = 0.0f;
    if (valid && l < a.b) {
      const size_t bb = (size_t)a.b * a.b;
      if (MODE == RP_S1) {
        x = first ? 0.0f : (float)a.M1[(size_t)(a.cb0 + lc) * bb + (size_t)k * a.b + l];  // B^T[l][k]
      } else if (MODE == RP_S3) {
        x = (float)a.M1[(size_t)lc * bb + (size_t)l * a.b + k];
        if (!first)
          y = (float)(a.Bprev[(size_t)(a.cb0 + lc) * bb + (size_t)k * a.b + l] +
                      (a.Kp ? a.Kp[(size_t)lc * bb + (size_t)l * a.b + k] : 0.0));
      } else {
        x = (float)a.M1[(size_t)lc * bb + (size_t)l * a.b + k];
      }
    }
    m1[l] = x;
    m2[l] = y;
  }
  float g[RP_KP], hi[RP_KP], lo[RP_KP];
#pragma unroll
  for (int l = 0; l < RP_KP; ++l) g[l] = hi[l] = lo[l] = 0.0f;

  // each thread copies its own element of every staged row (rows past the end: zero)
  auto issue = [&](int sc) {
    if (sc < nsub) {
      float* st = stage + (size_t)(sc % RP_NST) * C::STAGE;
      const int64_t r0 = rbeg + (int64_t)sc * RP_RS;
      const float* src[3] = {C::NA == 3 ? a.Q : a.W, a.Qp, a.W};
#pragma unroll
      for (int ar = 0; ar < C::NA; ++ar) {
        const bool need = !(ar == 1 && first) && set == 0;  // one copy per element (set 0)
#pragma unroll
        for (int r = 0; r < RP_RS; ++r) {
          const bool in = valid && need && r0 + r < rend;
          float* d = st + ((size_t)ar * RP_RS + r) * C::PITCH + soff;
          if (set == 0) cp4(d, src[ar] + (size_t)(in ? r0 + r : 0) * a.ws + col, in);
        }
      }
    }
    cp_commit();
  };
  for (int s = 0; s < RP_NST - 1; ++s) issue(s);

  for (int sc = 0; sc < nsub; ++sc) {
    cp_wait<RP_NST - 2>();
    __syncthreads();  // sub-chunk sc is staged; every thread is done with sub-chunk sc - 1
    issue(sc + RP_NST - 1);
    const float* st = stage + (size_t)(sc % RP_NST) * C::STAGE;
    float* so = sO + (size_t)(sc & 1) * RP_RS * C::PITCH;
    const int64_t r0 = rbeg + (int64_t)sc * RP_RS;
    const float* rowbase = st + cl * RP_KP;
    if (MODE == RP_S1) {
      // W0 = W - Q_{j-1} B^T: each thread set takes half of the rows
      constexpr int H = RP_RS / C::NSET;
#pragma unroll
      for (int rr = 0; rr < H; ++rr) {
        const int r = set * H + rr;
        float o = st[((size_t)2 * RP_RS + r) * C::PITCH + soff];
        if (!first) o = o - row_dot(rowbase + ((size_t)RP_RS + r) * C::PITCH, m1);
        so[r * C::PITCH + soff] = o;
      }
    } else if (MODE == RP_S3) {
#pragma unroll
      for (int r = 0; r < RP_RS; ++r) {
        float o = st[((size_t)2 * RP_RS + r) * C::PITCH + soff] - row_dot(rowbase + (size_t)r * C::PITCH, m1);
        if (!first) o = o - row_dot(rowbase + ((size_t)RP_RS + r) * C::PITCH, m2);
        so[r * C::PITCH + soff] = o;
        if (valid && r0 + r < rend) a.OUT[(size_t)(r0 + r) * a.ws + col] = o;
      }
    } else {
#pragma unroll
      for (int r = 0; r < RP_RS; ++r) {
        const float o = row_dot(rowbase + (size_t)r * C::PITCH, m1);
        if (MODE == RP_TRIG) so[r * C::PITCH + soff] = o;
        if (MODE == RP_TRI && valid && r0 + r < rend) a.OUT[(size_t)(r0 + r) * a.ws + col] = o;
      }
    }
    if (C::GRAM) {
      __syncthreads();  // the products of this sub-chunk are in sO
      // S1: Gram row k of Q_j^T W0 (set 0) or Q_{j-1}^T W0 (set 1); S3 / TRIG: of W1^T W1
      const bool active = MODE != RP_S1 || set == 0 || (a.reorth && !first);
#pragma unroll
      for (int r = 0; r < RP_RS; ++r) {
        float x;
        if (MODE == RP_S1) x = st[((size_t)(set == 0 ? 0 : 1) * RP_RS + r) * C::PITCH + soff];
        else x = so[r * C::PITCH + soff];
        if (active) row_axpy(so + r * C::PITCH + cl * RP_KP, x, g);
      }
      if (((sc + 1) * RP_RS) % RP_GRAM_RS == 0 || sc + 1 == nsub) gram_flush(g, hi, lo);
    }
  }
  cp_wait<0>();
  if (C::GRAM && valid) {
    double* part = (MODE == RP_S1 && set == 1) ? a.part2 : a.part1;
    if (MODE != RP_S1 || set == 0 || (a.reorth && !first)) {
      double* o = part + (((size_t)blockIdx.x * a.ncb + lc) * a.b + k) * a.b;
#pragma unroll
      for (int l = 0; l < RP_KP; ++l)
        if (l < a.b) o[l] = (double)hi[l] + (double)lo[l];
    }
  }
}

// C[lc] = A[lc] B[lc] for b x b FP64 matrices (products of the CholeskyQR factors' inverses)
__global__ void k_small_mm(int32_t ncb, int32_t b, const double* __restrict__ A, const double* __restrict__ B,
                           double* __restrict__ Cm) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t bb = (int64_t)b * b;
  if (t >= (int64_t)ncb * bb) return;
  const int64_t lc = t / bb;
  const int32_t e = (int32_t)(t - lc * bb), i = e / b, j = e - i * b;
  const double* a = A + lc * bb;
  const double* bm = B + lc * bb;
  double s = 0.0;
  for (int32_t l = 0; l < b; ++l) s = fma(a[i * b + l], bm[l * b + j], s);
  Cm[t] = s;
}

}  // namespace

bool css_rowpass_supported(bool fp32, int32_t b) { return fp32 && b > 16 && b <= RP_KP; }

int32_t css_rowpass_chunks(int64_t N) { return (int32_t)css_ceil_div(N, RP_RCH); }

template <int MODE>
static css_status launch_rp(css_ctx* ctx, const RpArgs& a, cudaStream_t st) {
  using C = RpCfg<MODE>;
  CSS_CU(ctx, cudaFuncSetAttribute(k_rowpass<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
  const dim3 grid((unsigned)css_ceil_div(a.N, RP_RCH), (unsigned)css_ceil_div(a.ncb, C::CG));
  k_rowpass<MODE><<<grid, C::THREADS, C::SMEM, st>>>(a);
  CSS_LAUNCHED(ctx);
  return CSS_OK;
}

// One FP32 Lanczos step after H V (W = H Q_j in a.W): the three-term update, A_j, the local
// reorthogonalisation and the shifted CholeskyQR3 of the new block, with the small FP64 factor
// work done by the callbacks of css_lanczos.cu.  See the header comment for the passes.
css_status css_rowpass(css_ctx* ctx, int mode, int64_t N, int32_t b, int32_t ws, int32_t ncb, int32_t cb0, int first,
                       int reorth, const float* Q, const float* Qp, const float* W, float* OUT, const double* M1,
                       const double* Bprev, const double* Kp, double* part1, double* part2, cudaStream_t st) {
  RpArgs a;
  a.N = N;
  a.b = b;
  a.ws = ws;
  a.ncb = ncb;
  a.cb0 = cb0;
  a.first = first;
  a.reorth = reorth;
  a.Q = Q;
  a.Qp = Qp;
  a.W = W;
  a.OUT = OUT;
  a.M1 = M1;
  a.Bprev = Bprev;
  a.Kp = Kp;
  a.part1 = part1;
  a.part2 = part2;
  switch (mode) {
    case RP_S1: return launch_rp<RP_S1>(ctx, a, st);
    case RP_S3: return launch_rp<RP_S3>(ctx, a, st);
    case RP_TRIG: return launch_rp<RP_TRIG>(ctx, a, st);
    default: return launch_rp<RP_TRI>(ctx, a, st);
  }
}

css_status css_small_mm(css_ctx* ctx, int32_t ncb, int32_t b, const double* A, const double* B, double* Cm,
                        cudaStream_t st) {
  const int64_t n = (int64_t)ncb * b * b;
  k_small_mm<<<(unsigned)css_ceil_div(n, 256), 256, 0, st>>>(ncb, b, A, B, Cm);
  CSS_LAUNCHED(ctx);
  return CSS_OK;
}
