// FP32 H * V for the block widths of the two molecular bases (b = 6, minimal; b = 23, DZP-like):
// W = H V for the BSR matrix H and the Krylov blocks V of every colour of a batch (paper: the
// SpMMs that make up the whole cost of the method, paragraph after Eq. 10).
//
// The padded kernel of css_lanczos.cu multiplies BM x BM blocks (BM = 8 for b = 6, 24 for
// b = 23: 78% and 9% more FMAs than the blocks hold) and stages V through shared memory behind
// two CTA barriers per neighbour block.  This one
//  * pairs adjacent ROWS of W_I in the packed FMA fma.rn.f32x2: a thread owns CPT = 4 consecutive
//    columns and all b rows of W_I for them, each 64-bit accumulator two rows (2i, 2i + 1) of one
//    column; H enters as the natural pair {H_p[2i][k], H_p[2i+1][k]} of its transposed block
//    (Ht[p][k][r] = H_p[r][k], r padded to an even count RA, stored once per call) and V as the
//    duplicated pair {v, v} formed in registers, so a k costs (RA / 2) CPT packed FMAs and RA / 4
//    broadcast 16-byte shared loads (RA / 2 eight-byte ones when RA is not a multiple of 4);
//  * reads each thread's own 16 bytes of the b rows of V_J straight from L2 into registers,
//    DEPTH rows ahead of their use: V needs neither shared memory nor a barrier;
//  * keeps only the H blocks in shared memory, in a ring of NS stages that one thread fills with
//    bulk copies (cp.async.bulk) completing on mbarriers.  The warps of a CTA wait on a stage's
//    "full" barrier and release it on its "empty" barrier; only the copying thread waits for the
//    other warps, one stage behind.
// Each output is the same sum in the same order as in the padded kernel (neighbours in CSR
// order, k ascending, then the low FP32 part of the diagonal block), every term the same IEEE
// FMA, so both kernels give bitwise equal W.  Every wait is bounded: on time-out the CTA sets the
// error flag, waits for its own copies in flight, writes zeros to its part of W and returns.
#include <algorithm>

#include "css_lanczos.cuh"
#include "css_pipe.cuh"

namespace {

using namespace css_pipe;

constexpr int SD_NS = 4;     // H stages
constexpr int SD_DEPTH = 4;  // rows of V in flight per thread

template <int B, int NW>
struct SdCfg {
  static constexpr int RA = B + (B & 1);  // rows of a stored block (even)
  static constexpr int RP = RA / 2;       // row pairs
  static constexpr int HF = B * RA;       // floats per block
  static constexpr int HB = HF * 4;       // bytes per block, a multiple of 16 for b = 6 and 23
  static constexpr int NT = NW * 32;
  static constexpr int CPT = 4;           // columns per thread
  static constexpr int CW = 32 * CPT;     // columns per warp
  static constexpr int CT = NW * CW;      // columns per CTA
  static constexpr size_t smem = (size_t)SD_NS * HB + 2 * SD_NS * sizeof(uint64_t) + 16;
  static_assert(B >= SD_DEPTH && HB % 16 == 0, "shape");
};

struct SdArgs {
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const float* Ht;    // [nnzb][B][RA] transposed blocks
  const float* Hlot;  // [n_brow][B][RA] low parts of the diagonal blocks, or null
  const float* V;
  float* W;
  int32_t ws, w, jbase;
  int32_t empty_extra;  // 0; a test sets k > 0 so that the ring's waits run out
  int* err;
};

__device__ __forceinline__ float4 v_load(const float* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ unsigned long long dup2(float x) {
  unsigned long long d;
  asm("mov.b64 %0, {%1, %1};" : "=l"(d) : "f"(x));
  return d;
}
__device__ __forceinline__ void fma2(unsigned long long& d, unsigned long long h, unsigned long long v) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(h), "l"(v));
}
// grid (n_brow, column tiles of CT); rows without blocks (and no low part) give W_I = 0
template <int B, int NW, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) k_spmm_dup(SdArgs a) {
  using C = SdCfg<B, NW>;
  constexpr int RP = C::RP, CPT = C::CPT;
  extern __shared__ __align__(128) unsigned char smem[];
  float* ring = reinterpret_cast<float*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + SD_NS * C::HB);
  uint64_t* empty = full + SD_NS;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + SD_NS);
  const int32_t I = blockIdx.x;
  const int32_t tile0 = blockIdx.y * C::CT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int live = min(NW, (a.w - tile0 + C::CW - 1) / C::CW);  // warps with a column below w
  const int32_t p0 = a.row_ptr[I], nnz = a.row_ptr[I + 1] - p0;
  const int32_t nsteps = nnz + (a.Hlot ? 1 : 0);
  if (threadIdx.x == 0) {
    for (int s = 0; s < SD_NS; ++s) {
      bar_init(&full[s], 1);
      bar_init(&empty[s], (uint32_t)(live + a.empty_extra));
    }
    // after a time-out anywhere in this call the remaining CTAs return at once (the call fails)
    *abort_flag = *(volatile int*)a.err ? 1 : 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp >= live) return;  // no barrier below involves these warps
  const int32_t col = tile0 + (warp * 32 + lane) * CPT;
  float* Wr = a.W + (size_t)I * B * a.ws + col;
  // a failed call leaves zeros (finite values) in W for the rest of the pass
  auto zero_w = [&]() {
    if (col < a.w)
      for (int r = 0; r < B; ++r)
        for (int u = 0; u < CPT && col + u < a.w; ++u) Wr[(size_t)r * a.ws + u] = 0.0f;
  };
  if (*abort_flag) {
    zero_w();
    return;
  }

  const bool producer = warp == 0 && lane == 0;
  auto issue = [&](int32_t q) {
    const int s = q % SD_NS;
    const float* src = q < nnz ? a.Ht + (size_t)(p0 + q) * C::HF : a.Hlot + (size_t)I * C::HF;
    bar_expect(&full[s], C::HB);
    bulk_g2s(ring + (size_t)s * C::HF, src, C::HB, &full[s]);
  };
  int32_t issued = 0;
  if (producer)
    for (; issued < nsteps && issued < SD_NS - 1; ++issued) issue(issued);

  const float* Vc = a.V + (col < a.w ? col : 0);  // lanes past w read column 0 and store nothing
  auto jof = [&](int32_t q) -> int32_t { return q < nnz ? a.col_idx[p0 + q] - a.jbase : I; };
  auto vrow = [&](int32_t J, int k) { return v_load(Vc + ((size_t)J * B + k) * a.ws); };

  // acc[i][u]: rows 2i (low half) and 2i + 1 (high half) of column col + u
  unsigned long long acc[RP][CPT];
#pragma unroll
  for (int i = 0; i < RP; ++i)
#pragma unroll
    for (int u = 0; u < CPT; ++u) acc[i][u] = 0ull;
  bool ok = true;
  int32_t q = 0;
  if (nsteps > 0) {
    float4 vr[B];
    float4 vn[SD_DEPTH];
    int32_t Jc = jof(0);
#pragma unroll
    for (int k = 0; k < SD_DEPTH; ++k) vr[k] = vrow(Jc, k);
    for (; q < nsteps; ++q) {
      const int s = q % SD_NS;
      const bool more = q + 1 < nsteps;
      const int32_t Jn = more ? jof(q + 1) : Jc;
      bool good = true;
      if (producer && issued < nsteps) {
        // the stage of step `issued` was last read by step issued - NS (= q - 1)
        if (issued >= SD_NS)
          good = bar_wait(&empty[issued % SD_NS], (uint32_t)((issued / SD_NS - 1) & 1), abort_flag, a.err);
        if (good) {
          issue(issued);
          ++issued;
        }
      }
      if (good) good = bar_wait(&full[s], (uint32_t)((q / SD_NS) & 1), abort_flag, a.err);
      if (!__all_sync(0xffffffffu, good)) {
        ok = false;
        break;
      }
      const float* hs = ring + (size_t)s * C::HF;
#pragma unroll
      for (int k = 0; k < B; ++k) {
        if (k + SD_DEPTH < B)
          vr[k + SD_DEPTH] = vrow(Jc, k + SD_DEPTH);
        else if (more)
          vn[k + SD_DEPTH - B] = vrow(Jn, k + SD_DEPTH - B);
        const unsigned long long v2[CPT] = {dup2(vr[k].x), dup2(vr[k].y), dup2(vr[k].z), dup2(vr[k].w)};
        const float* hk = hs + k * C::RA;
        if constexpr (RP % 2 == 0) {
#pragma unroll
          for (int i = 0; i < RP; i += 2) {
            const ulonglong2 h = *reinterpret_cast<const ulonglong2*>(hk + 2 * i);
#pragma unroll
            for (int u = 0; u < CPT; ++u) {
              fma2(acc[i][u], h.x, v2[u]);
              fma2(acc[i + 1][u], h.y, v2[u]);
            }
          }
        } else {
#pragma unroll
          for (int i = 0; i < RP; ++i) {
            const unsigned long long h = *reinterpret_cast<const unsigned long long*>(hk + 2 * i);
#pragma unroll
            for (int u = 0; u < CPT; ++u) fma2(acc[i][u], h, v2[u]);
          }
        }
      }
      __syncwarp();
      if (lane == 0) bar_arrive(&empty[s]);
#pragma unroll
      for (int k = 0; k < SD_DEPTH; ++k) vr[k] = vn[k];
      Jc = Jn;
    }
  }
  if (!ok) {
    // bulk copies issued and not yet waited for are steps [q, issued): let them land first
    if (producer)
      for (int32_t n = q; n < issued; ++n) bar_drain(&full[n % SD_NS], (uint32_t)((n / SD_NS) & 1));
    zero_w();
    return;
  }
  if (col >= a.w) return;
  const bool whole = col + CPT <= a.w;
  auto half = [](unsigned long long x, int h) { return __uint_as_float((unsigned)(h ? (x >> 32) : (x & 0xffffffffull))); };
#pragma unroll
  for (int r = 0; r < B; ++r) {
    const int i = r >> 1, h = r & 1;
    if (whole) {
      *reinterpret_cast<float4*>(Wr + (size_t)r * a.ws) =
          make_float4(half(acc[i][0], h), half(acc[i][1], h), half(acc[i][2], h), half(acc[i][3], h));
    } else {
#pragma unroll
      for (int u = 0; u < CPT; ++u)
        if (col + u < a.w) Wr[(size_t)r * a.ws + u] = half(acc[i][u], h);
    }
  }
}

// Ht[p][k][r] = H_p[r][k] in FP32 (round to nearest) for r, k < b, zero for the pad row r = b of
// an odd b.  LO: block p is the diagonal block of row p, and the value the low FP32 part
// fl32(h - fl32(h)) (zero for a row without a diagonal block).
template <bool LO>
__global__ void k_hdup(int64_t nblocks, int32_t b, int32_t RA, const double* __restrict__ H,
                       const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                       float* __restrict__ Ht) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)b * RA;
  if (e >= nblocks * per) return;
  const int64_t p = e / per;
  const int32_t rem = (int32_t)(e - p * per), k = rem / RA, r = rem - k * RA;
  float v = 0.0f;
  if (r < b) {
    int64_t src = p;
    if (LO) {
      int32_t q = row_ptr[p];
      while (q < row_ptr[p + 1] && col_idx[q] != (int32_t)p) ++q;
      src = q < row_ptr[p + 1] ? q : -1;
    }
    if (src >= 0) {
      const double h = H[(size_t)src * b * b + (size_t)r * b + k];
      v = LO ? (float)(h - (double)(float)h) : (float)h;
    }
  }
  Ht[e] = v;
}

template <int B, int NW, int MINB>
css_status launch_dup(css_ctx* ctx, const LzArgs& a, const float* V, float* W, int* err, cudaStream_t st) {
  using C = SdCfg<B, NW>;
  auto kern = k_spmm_dup<B, NW, MINB>;
  static_assert(C::smem <= 48 * 1024, "static shared-memory limit");
  SdArgs s;
  s.row_ptr = a.row_ptr;
  s.col_idx = a.col_idx;
  s.Ht = (const float*)a.Hdup;
  s.Hlot = (const float*)a.Hlo_dup;
  s.V = V;
  s.W = W;
  s.ws = a.ws;
  s.w = a.w;
  s.jbase = a.row0;
  s.empty_extra = ctx->test_spmm_empty_extra;
  s.err = err;
  const dim3 grid((unsigned)a.n_brow, (unsigned)css_ceil_div(a.w, C::CT));
  kern<<<grid, C::NT, C::smem, st>>>(s);
  CSS_LAUNCHED(ctx);
  return CSS_OK;
}

// ---------------------------------------------------------------- FP64-accurate H * V in FP32
// W = H V for FP64 V and W with the products on the FP32 FMA pipe (precision CSS_FP64_SPLIT).
// Every value x is the unevaluated pair x_hi + x_lo of FP32 numbers (x_hi = fl32(x),
// x_lo = fl32(x - x_hi): 48 significand bits).  One term h v is taken as the rounded product
// p = h_hi v_hi, its exact error e = fma(h_hi, v_hi, -p) (Dekker's product through the FMA) and
// the cross terms h_hi v_lo + h_lo v_hi (h_lo v_lo, 2^-48 of the term, is dropped); p is added to
// the running sum S_hi by Knuth's TwoSum, whose error and the small terms go to S_lo.  The output
// is (double) S_hi + (double) S_lo.  Relative error per term about 2^-47, against 2^-53 in FP64.
// The kernel is the row-pair kernel above with FP64 data: a thread owns 2 columns and all b rows
// of W_I, each 64-bit S_hi / S_lo register holds rows 2i and 2i + 1 of one column, H's hi and lo
// parts arrive as natural row pairs from the shared-memory ring, and V as {hi, lo} pairs split
// once per launch (k_vsplit).
constexpr uint64_t kSignPair = 0x8000000080000000ull;

template <int B, int NW>
struct DfCfg {
  static constexpr int RA = B + (B & 1);  // rows of a stored block (even)
  static constexpr int RP = RA / 2;       // row pairs
  static constexpr int HF = B * RA;       // floats per part (hi, lo) of a block
  static constexpr int HB = 2 * HF * 4;   // bytes per block, a multiple of 16 for b = 6 and 23
  static constexpr int NT = NW * 32;
  static constexpr int CPT = 2;           // columns per thread
  static constexpr int CW = 32 * CPT;     // columns per warp
  static constexpr int CT = NW * CW;      // columns per CTA
  static constexpr size_t smem = (size_t)SD_NS * HB + 2 * SD_NS * sizeof(uint64_t) + 16;
  static_assert(B >= SD_DEPTH && HB % 16 == 0, "shape");
};

struct DfArgs {
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const float* Hs;  // [nnzb][2][B][RA]: transposed hi part, then lo part
  const float* Vs;  // [N][ws][2]: {hi, lo} of every entry of V
  double* W;
  int32_t ws, w, jbase;
  int32_t empty_extra;
  int* err;
};

__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long fmaq2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// (sh, sl) += (h_hi + h_lo)(v_hi + v_lo), both lanes of the pair
__device__ __forceinline__ void df_term(unsigned long long& sh, unsigned long long& sl, unsigned long long hh,
                                        unsigned long long hl, unsigned long long vh, unsigned long long vl) {
  const unsigned long long p = mul2(hh, vh);
  unsigned long long c = fmaq2(hh, vh, p ^ kSignPair);  // h_hi v_hi - p, exact
  c = fmaq2(hl, vh, c);
  c = fmaq2(hh, vl, c);
  const unsigned long long s = add2(sh, p);  // TwoSum(sh, p) = s + err exactly
  const unsigned long long bv = sub2(s, sh);
  const unsigned long long err = add2(sub2(sh, sub2(s, bv)), sub2(p, bv));
  sl = add2(sl, add2(err, c));
  sh = s;
}

// grid (n_brow, column tiles of CT); rows without blocks give W_I = 0
template <int B, int NW, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) k_spmm_df(DfArgs a) {
  using C = DfCfg<B, NW>;
  constexpr int RP = C::RP, CPT = C::CPT;
  extern __shared__ __align__(128) unsigned char smem[];
  float* ring = reinterpret_cast<float*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + SD_NS * C::HB);
  uint64_t* empty = full + SD_NS;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + SD_NS);
  const int32_t I = blockIdx.x;
  const int32_t tile0 = blockIdx.y * C::CT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int live = min(NW, (a.w - tile0 + C::CW - 1) / C::CW);  // warps with a column below w
  const int32_t p0 = a.row_ptr[I], nsteps = a.row_ptr[I + 1] - p0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < SD_NS; ++s) {
      bar_init(&full[s], 1);
      bar_init(&empty[s], (uint32_t)(live + a.empty_extra));
    }
    *abort_flag = *(volatile int*)a.err ? 1 : 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp >= live) return;  // no barrier below involves these warps
  const int32_t col = tile0 + (warp * 32 + lane) * CPT;
  double* Wr = a.W + (size_t)I * B * a.ws + col;
  auto zero_w = [&]() {
    if (col < a.w)
      for (int r = 0; r < B; ++r)
        for (int u = 0; u < CPT && col + u < a.w; ++u) Wr[(size_t)r * a.ws + u] = 0.0;
  };
  if (*abort_flag) {
    zero_w();
    return;
  }
  const bool producer = warp == 0 && lane == 0;
  auto issue = [&](int32_t q) {
    const int s = q % SD_NS;
    bar_expect(&full[s], C::HB);
    bulk_g2s(ring + (size_t)s * 2 * C::HF, a.Hs + (size_t)(p0 + q) * 2 * C::HF, C::HB, &full[s]);
  };
  int32_t issued = 0;
  if (producer)
    for (; issued < nsteps && issued < SD_NS - 1; ++issued) issue(issued);

  // {hi, lo} of this thread's two columns of a row of V (lanes past w read column 0, store nothing)
  const float* Vc = a.Vs + 2 * (size_t)(col < a.w ? col : 0);
  auto vrow = [&](int32_t J, int k) {
    return __ldcg(reinterpret_cast<const float4*>(Vc + 2 * ((size_t)J * B + k) * a.ws));
  };
  unsigned long long sh[RP][CPT], sl[RP][CPT];
#pragma unroll
  for (int i = 0; i < RP; ++i)
#pragma unroll
    for (int u = 0; u < CPT; ++u) sh[i][u] = sl[i][u] = 0ull;
  bool ok = true;
  int32_t q = 0;
  if (nsteps > 0) {
    // the k loop is not unrolled (an unrolled block step is ≈ 7,000 instructions, past the
    // instruction cache); V rows arrive three ahead of use through the registers v0, v1, v2,
    // across the end of a block into the next neighbour's first rows
    int32_t Jc = a.col_idx[p0] - a.jbase;
    float4 v0 = vrow(Jc, 0), v1 = vrow(Jc, 1), v2 = vrow(Jc, 2);
    for (; q < nsteps; ++q) {
      const int s = q % SD_NS;
      const bool more = q + 1 < nsteps;
      const int32_t Jn = more ? a.col_idx[p0 + q + 1] - a.jbase : Jc;
      bool good = true;
      if (producer && issued < nsteps) {
        if (issued >= SD_NS)
          good = bar_wait(&empty[issued % SD_NS], (uint32_t)((issued / SD_NS - 1) & 1), abort_flag, a.err);
        if (good) {
          issue(issued);
          ++issued;
        }
      }
      if (good) good = bar_wait(&full[s], (uint32_t)((q / SD_NS) & 1), abort_flag, a.err);
      if (!__all_sync(0xffffffffu, good)) {
        ok = false;
        break;
      }
      const float* hs = ring + (size_t)s * 2 * C::HF;
#pragma unroll 1
      for (int k = 0; k < B; ++k) {
        const int t = k + 3;  // the row this iteration prefetches
        float4 v3 = v2;       // past the last block: a copy, never used
        if (t < B)
          v3 = vrow(Jc, t);
        else if (more)
          v3 = vrow(Jn, t - B);
        const unsigned long long vh[CPT] = {dup2(v0.x), dup2(v0.z)};
        const unsigned long long vl[CPT] = {dup2(v0.y), dup2(v0.w)};
        const float* hk = hs + k * C::RA;
        const float* lk = hk + C::HF;
        if constexpr (RP % 2 == 0) {
#pragma unroll
          for (int i = 0; i < RP; i += 2) {
            const ulonglong2 h = *reinterpret_cast<const ulonglong2*>(hk + 2 * i);
            const ulonglong2 l = *reinterpret_cast<const ulonglong2*>(lk + 2 * i);
#pragma unroll
            for (int u = 0; u < CPT; ++u) {
              df_term(sh[i][u], sl[i][u], h.x, l.x, vh[u], vl[u]);
              df_term(sh[i + 1][u], sl[i + 1][u], h.y, l.y, vh[u], vl[u]);
            }
          }
        } else {
#pragma unroll
          for (int i = 0; i < RP; ++i) {
            const unsigned long long h = *reinterpret_cast<const unsigned long long*>(hk + 2 * i);
            const unsigned long long l = *reinterpret_cast<const unsigned long long*>(lk + 2 * i);
#pragma unroll
            for (int u = 0; u < CPT; ++u) df_term(sh[i][u], sl[i][u], h, l, vh[u], vl[u]);
          }
        }
        v0 = v1;
        v1 = v2;
        v2 = v3;
      }
      __syncwarp();
      if (lane == 0) bar_arrive(&empty[s]);
      Jc = Jn;
    }
  }
  if (!ok) {
    if (producer)
      for (int32_t n = q; n < issued; ++n) bar_drain(&full[n % SD_NS], (uint32_t)((n / SD_NS) & 1));
    zero_w();
    return;
  }
  if (col >= a.w) return;
  auto half = [](unsigned long long x, int h) { return __uint_as_float((unsigned)(h ? (x >> 32) : (x & 0xffffffffull))); };
#pragma unroll
  for (int r = 0; r < B; ++r) {
    const int i = r >> 1, h = r & 1;
    const double w0 = (double)half(sh[i][0], h) + (double)half(sl[i][0], h);
    const double w1 = (double)half(sh[i][1], h) + (double)half(sl[i][1], h);
    if (col + CPT <= a.w) {
      *reinterpret_cast<double2*>(Wr + (size_t)r * a.ws) = make_double2(w0, w1);
    } else {
      Wr[(size_t)r * a.ws] = w0;  // col < w here; col + 1 >= w
    }
  }
}

// Hs[p][0][k][r] = fl32(H_p[r][k]), Hs[p][1][k][r] = fl32(H_p[r][k] - fl32(H_p[r][k])); the pad
// row r = b of an odd b is zero
__global__ void k_hsplit(int64_t nblocks, int32_t b, int32_t RA, const double* __restrict__ H, float* __restrict__ Hs) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)b * RA;
  if (e >= nblocks * per) return;
  const int64_t p = e / per;
  const int32_t rem = (int32_t)(e - p * per), k = rem / RA, r = rem - k * RA;
  float hi = 0.0f, lo = 0.0f;
  if (r < b) {
    const double h = H[(size_t)p * b * b + (size_t)r * b + k];
    hi = (float)h;
    lo = (float)(h - (double)hi);
  }
  Hs[(size_t)p * 2 * per + rem] = hi;
  Hs[(size_t)p * 2 * per + per + rem] = lo;
}

// Vs[e] = {fl32(V[e]), fl32(V[e] - fl32(V[e]))} for the n entries of V
__global__ void k_vsplit(int64_t n, const double* __restrict__ V, float2* __restrict__ Vs) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const double v = V[e];
  const float hi = (float)v;
  Vs[e] = make_float2(hi, (float)(v - (double)hi));
}

template <int B, int NW, int MINB>
css_status launch_df(css_ctx* ctx, const LzArgs& a, const float* Vs, double* W, int* err, cudaStream_t st) {
  using C = DfCfg<B, NW>;
  static_assert(C::smem <= 48 * 1024, "static shared-memory limit");
  DfArgs s;
  s.row_ptr = a.row_ptr;
  s.col_idx = a.col_idx;
  s.Hs = (const float*)a.Hsplit;
  s.Vs = Vs;
  s.W = W;
  s.ws = a.ws;
  s.w = a.w;
  s.jbase = a.row0;
  s.empty_extra = ctx->test_spmm_empty_extra;
  s.err = err;
  const dim3 grid((unsigned)a.n_brow, (unsigned)css_ceil_div(a.w, C::CT));
  k_spmm_df<B, NW, MINB><<<grid, C::NT, C::smem, st>>>(s);
  CSS_LAUNCHED(ctx);
  return CSS_OK;
}

}  // namespace

bool css_spmm_dup_supported(bool fp32, int32_t b) { return fp32 && (b == 6 || b == 23); }

int css_spmm_dup_variants() { return 4; }

css_status css_spmm_dup_prepare(css_ctx* ctx, int32_t b, int32_t n_brow, int32_t nnzb, const int32_t* row_ptr,
                                const int32_t* col_idx, const double* H, const void** Hd, const void** Hlod,
                                cudaStream_t st) {
  if (!css_spmm_dup_supported(true, b)) return css_set_arg_error(ctx, "H*V: no exact-width kernel for this b");
  const int32_t RA = b + (b & 1);
  const int64_t per = (int64_t)b * RA;
  float *h, *l;
  CSS_TRY(css_ws(ctx, "h_dup", (size_t)std::max<int64_t>(nnzb, 1) * per * 4, (void**)&h));
  CSS_TRY(css_ws(ctx, "h_lodup", (size_t)std::max<int32_t>(n_brow, 1) * per * 4, (void**)&l));
  constexpr int T = 256;
  if (nnzb > 0) {
    k_hdup<false><<<(unsigned)css_ceil_div((int64_t)nnzb * per, T), T, 0, st>>>(nnzb, b, RA, H, row_ptr, col_idx, h);
    CSS_LAUNCHED(ctx);
  }
  if (n_brow > 0) {
    k_hdup<true><<<(unsigned)css_ceil_div((int64_t)n_brow * per, T), T, 0, st>>>(n_brow, b, RA, H, row_ptr, col_idx,
                                                                                 l);
    CSS_LAUNCHED(ctx);
  }
  int* err;  // the time-out flag starts clear for this call
  CSS_TRY(css_ws(ctx, "dup_err", 256, (void**)&err));
  CSS_CU(ctx, cudaMemsetAsync(err, 0, sizeof(int), st));
  *Hd = h;
  *Hlod = l;
  return CSS_OK;
}

// launch variants (columns per thread, warps per CTA, CTAs per SM the registers are sized for);
// every variant sums each output in the same order
css_status css_spmm_dup(css_ctx* ctx, const LzArgs& a, const float* V, float* W, int v, cudaStream_t st) {
  if (a.n_brow == 0 || a.w == 0) return CSS_OK;
  if (((uintptr_t)V & 15) || ((uintptr_t)W & 15) || (a.ws & 7))
    return css_set_arg_error(ctx, "H*V: V and W must be 16-byte aligned with a row stride of 8 floats");
  int* err;
  CSS_TRY(css_ws(ctx, "dup_err", 256, (void**)&err));
  if (a.b == 23) {
    switch (v) {
      case 0: return launch_dup<23, 4, 3>(ctx, a, V, W, err, st);
      case 1: return launch_dup<23, 2, 6>(ctx, a, V, W, err, st);
      case 2: return launch_dup<23, 4, 2>(ctx, a, V, W, err, st);
      default: return launch_dup<23, 8, 1>(ctx, a, V, W, err, st);
    }
  }
  if (a.b == 6) {
    switch (v) {
      case 0: return launch_dup<6, 2, 8>(ctx, a, V, W, err, st);
      case 1: return launch_dup<6, 4, 4>(ctx, a, V, W, err, st);
      case 2: return launch_dup<6, 8, 2>(ctx, a, V, W, err, st);
      default: return launch_dup<6, 1, 16>(ctx, a, V, W, err, st);
    }
  }
  return css_set_arg_error(ctx, "H*V: no exact-width kernel for this b");
}

// CSS_ERR_TIMEOUT when a wait of the exact-width H * V ran out since the last check (the flag is
// cleared); synchronises the stream
css_status css_spmm_dup_check(css_ctx* ctx, cudaStream_t st) {
  int* err;
  CSS_TRY(css_ws(ctx, "dup_err", 256, (void**)&err));
  int* h;
  CSS_TRY(css_pinned(ctx, 64, (void**)&h));
  CSS_CU(ctx, cudaMemcpyAsync(h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CSS_CU(ctx, cudaMemsetAsync(err, 0, sizeof(int), st));
  CSS_CU(ctx, cudaStreamSynchronize(st));
  if (*h) {
    ctx->last_error = "H*V: a bounded wait on the shared-memory ring of H blocks timed out";
    return CSS_ERR_TIMEOUT;
  }
  return CSS_OK;
}

// ------------------------------------------------------------ FP64-accurate H * V in FP32 pairs
bool css_spmm_split_supported(int32_t b) { return b == 6 || b == 23; }

int css_spmm_split_variants() { return 4; }

css_status css_spmm_split_prepare(css_ctx* ctx, int32_t b, int32_t nnzb, const double* H, const void** Hs,
                                  cudaStream_t st) {
  if (!css_spmm_split_supported(b)) return css_set_arg_error(ctx, "H*V: no split-FP64 kernel for this b");
  const int32_t RA = b + (b & 1);
  const int64_t per = (int64_t)b * RA;
  float* h;
  CSS_TRY(css_ws(ctx, "h_split", (size_t)std::max<int64_t>(nnzb, 1) * 2 * per * 4, (void**)&h));
  constexpr int T = 256;
  if (nnzb > 0) {
    k_hsplit<<<(unsigned)css_ceil_div((int64_t)nnzb * per, T), T, 0, st>>>(nnzb, b, RA, H, h);
    CSS_LAUNCHED(ctx);
  }
  int* err;  // the time-out flag starts clear for this call (shared with the exact-width kernel)
  CSS_TRY(css_ws(ctx, "dup_err", 256, (void**)&err));
  CSS_CU(ctx, cudaMemsetAsync(err, 0, sizeof(int), st));
  *Hs = h;
  return CSS_OK;
}

// V (FP64, N x ws) is split into {hi, lo} pairs in the context's workspace, then W = H V; launch
// variants as for the exact-width kernel (warps per CTA, CTAs per SM), every one summing each
// output in the same order
css_status css_spmm_split(css_ctx* ctx, const LzArgs& a, const double* V, double* W, int v, cudaStream_t st) {
  if (a.n_brow == 0 || a.w == 0) return CSS_OK;
  if (((uintptr_t)V & 15) || ((uintptr_t)W & 15) || (a.ws & 7))
    return css_set_arg_error(ctx, "H*V: V and W must be 16-byte aligned with a row stride of 8 values");
  const int64_t n = (int64_t)a.n_brow * a.b * a.ws;
  float2* vs;
  CSS_TRY(css_ws(ctx, "v_split", (size_t)n * sizeof(float2), (void**)&vs));
  k_vsplit<<<(unsigned)css_ceil_div(n, 256), 256, 0, st>>>(n, V, vs);
  CSS_LAUNCHED(ctx);
  int* err;
  CSS_TRY(css_ws(ctx, "dup_err", 256, (void**)&err));
  const float* Vs = reinterpret_cast<const float*>(vs);
  if (a.b == 23) {
    switch (v) {
      case 0: return launch_df<23, 4, 3>(ctx, a, Vs, W, err, st);
      case 1: return launch_df<23, 2, 6>(ctx, a, Vs, W, err, st);
      case 2: return launch_df<23, 4, 2>(ctx, a, Vs, W, err, st);
      default: return launch_df<23, 8, 1>(ctx, a, Vs, W, err, st);
    }
  }
  if (a.b == 6) {
    switch (v) {
      case 0: return launch_df<6, 2, 8>(ctx, a, Vs, W, err, st);
      case 1: return launch_df<6, 4, 4>(ctx, a, Vs, W, err, st);
      case 2: return launch_df<6, 8, 2>(ctx, a, Vs, W, err, st);
      default: return launch_df<6, 1, 16>(ctx, a, Vs, W, err, st);
    }
  }
  return css_set_arg_error(ctx, "H*V: no split-FP64 kernel for this b");
}
