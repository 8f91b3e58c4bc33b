// H * V on the fifth-generation tensor cores (tcgen05) for the FP32 (mixed-precision) mode and
// block widths 17..24: W = H V for the BSR matrix H and the Krylov blocks V of every colour of a
// batch (paper: the SpMMs that make up the whole cost of the method, paragraph after Eq. 10).
//
// FP32 accuracy from TF32 products (split-operand "3xTF32"): every operand x is written as
// x1 + x2 (+ x3) with TF32 parts xi = rna_tf32(x - x1 - ... - x_{i-1}).  A coupling block
// H_IJ (|H_IJ| <~ 1 eV) takes h1 v1 + h1 v2 + h2 v1, whose error is ~2^-22 |H_IJ| |v|; the
// diagonal block (on-site energies up to ~30 eV) takes three parts of both operands and
// h1 v1 + h1 v2 + h2 v1 + h1 v3 + h2 v2 + h3 v1, so its error stays below the FP32 rounding of
// the sum itself.  The products accumulate in FP32 in tensor memory.
//
// Work item = (group of G consecutive block rows, 256 consecutive columns of V = two M = 128
// tiles).  The CTA walks the union of the G rows' neighbour lists (a schedule built once per
// pass): for each neighbour J, V_J (BK rows x 256 columns) is read ONCE by a TMA tensor copy and
// serves every row of the group that couples to J, so V is read from L2 about |union| / (G *
// row length) as often as a one-row-per-CTA kernel reads it.  Per J:
//   producer (one thread)   TMA: V_J box -> shared stage; bulk copies: the TF32 parts of H_IJ
//                           (smem matrix layout, prepared once per call) for the group's rows
//   converters (256 thr.)   one column each: V_J -> v1, v2, v3 (registers) -> tensor memory
//                           (tcgen05.st), which is operand A of the MMAs
//   MMA issuer (one thread) tcgen05.mma kind::tf32, M = 128 (columns of V), N = 32 (rows of
//                           W_I, b <= 24 used), K = 8 per instruction: D_I^T += V_J^T H_IJ^T
// and at the end of an item the converters read D (tcgen05.ld) and write W.  Stages are
// double-buffered in tensor memory and four-deep in shared memory, chained by mbarriers; every
// wait is bounded (on time-out the CTA records an error flag, drains its own copies and MMAs,
// frees its tensor memory and returns).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "css_lanczos.cuh"
#include "css_pipe.cuh"

namespace {

using namespace css_pipe;

constexpr int TC_BK = 24;         // K per block: b <= 24, padded to 3 steps of 8
constexpr int TC_BN = 32;         // N of the MMA (rows of W_I; b <= 24 of them are kept)
constexpr int TC_G = 3;           // block rows per work item
constexpr int TC_TILE = 128;      // columns per M tile
constexpr int TC_COLS = 2 * TC_TILE;  // columns per work item
constexpr int TC_NS = 4;          // shared-memory stages
constexpr int TC_CONV = 256;      // converter / epilogue threads (8 warps)
constexpr int TC_THREADS = TC_CONV + 64;  // + producer warp + MMA warp
constexpr int TC_SL = TC_BK * TC_BK * 4;  // bytes of one TF32 part of a block (2304)
constexpr int TC_VST = TC_BK * TC_COLS * 4;                  // V stage (24576)
constexpr int TC_HST = TC_G * 2 * TC_SL + TC_SL + 1024;      // H stage: G x (h1,h2), diag h3, slack
constexpr int TC_BAR = 256;                                  // barriers and flags
constexpr int TC_SCHED_MAX = 384;                            // schedule entries of an item held in smem
constexpr int TC_META = TC_NS * 16 + TC_SCHED_MAX * 16;      // stage headers + the item's schedule
constexpr size_t TC_SMEM = (size_t)TC_NS * (TC_VST + TC_HST) + TC_BAR + TC_META + 1024;  // + alignment
// tensor memory columns: D[g][tile] (32 each), then A[slot][tile][part] (24 each)
constexpr int TC_DCOL = TC_G * 2 * TC_BN;  // 192
constexpr int TC_ACOL(int slot, int tile, int part) { return TC_DCOL + ((slot * 2 + tile) * 3 + part) * TC_BK; }
static_assert(TC_ACOL(1, 1, 2) + TC_BK <= 512, "tensor memory budget");
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
                              ((uint32_t)(128 >> 4) << 24);  // F32 += TF32 x TF32, K-major, M=128, N=32

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ void tma_v(void* dst, const CUtensorMap* map, int x, int y, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          su32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(su32(b))
      : "memory");
}
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_st8(uint32_t addr, const uint32_t (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(addr), "r"(v[0]),
               "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t addr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(addr));
}
// shared-memory matrix descriptor, no swizzle, K-major: core matrices of 8 rows x 16 bytes,
// LBO = 128 B between the two core matrices of a K step, SBO = (BK / 4) * 128 B between 8-row
// groups; bits 46..48 hold the fixed value 0b001
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  constexpr uint64_t LBO = 128, SBO = (TC_BK / 4) * 128;
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((LBO >> 4) << 16) | ((SBO >> 4) << 32) | (1ull << 46);
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint32_t a, uint64_t bdesc, bool acc) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p; }" ::"r"(d),
      "r"(a), "l"(bdesc), "r"(TC_IDESC), "r"((uint32_t)acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
               : "memory");
}

// offset (in floats) of element (n, k) of a block in the smem matrix layout above
__host__ __device__ __forceinline__ int tc_off(int n, int k) {
  return (n >> 3) * (TC_BK / 4) * 32 + (k >> 2) * 32 + (n & 7) * 4 + (k & 3);
}

// TF32 parts of H in the smem matrix layout: Htc[p][part][BK*BK] (part 0, 1) for every block
// (element (n, k) = H_p[n][k], zero padded), Hd3[I][BK*BK] the third part of row I's diagonal
// block (zero for a row without one)
__global__ void k_tc_hprep(int64_t nnzb, int32_t n_brow, int32_t b, const double* __restrict__ H,
                           const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                           float* __restrict__ Htc, float* __restrict__ Hd3) {
  constexpr int E = TC_BK * TC_BK;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nnzb * E) {
    const int64_t p = t / E;
    const int e = (int)(t - p * E), n = e / TC_BK, k = e - n * TC_BK;
    const double h = (n < b && k < b) ? H[(size_t)p * b * b + (size_t)n * b + k] : 0.0;
    const float h1 = __uint_as_float(tf32_rna((float)h));
    const float h2 = __uint_as_float(tf32_rna((float)(h - (double)h1)));
    Htc[(size_t)p * 2 * E + tc_off(n, k)] = h1;
    Htc[(size_t)p * 2 * E + E + tc_off(n, k)] = h2;
  }
  if (t < (int64_t)n_brow * E) {
    const int32_t I = (int32_t)(t / E);
    const int e = (int)(t - (int64_t)I * E), n = e / TC_BK, k = e - n * TC_BK;
    int32_t q = row_ptr[I];
    while (q < row_ptr[I + 1] && col_idx[q] != I) ++q;
    double h = 0.0;
    if (q < row_ptr[I + 1] && n < b && k < b) h = H[(size_t)q * b * b + (size_t)n * b + k];
    const float h1 = __uint_as_float(tf32_rna((float)h));
    const double r1 = h - (double)h1;
    const float h2 = __uint_as_float(tf32_rna((float)r1));
    Hd3[(size_t)I * E + tc_off(n, k)] = __uint_as_float(tf32_rna((float)(r1 - (double)h2)));
  }
}

// Schedule of one pass: group gi = rows [gi G, gi G + G) of the system; entry e of the group
// is a neighbour J of some row of the group (the union of their sorted column lists) with, per
// row slot, the global block index of (row, J) or -1.  The couplings (J outside the group) come
// first in increasing J and the group's own molecules last: the tensor cores add each product
// into the FP32 accumulator with truncation, which errs by up to an ulp of the running sum, so
// the large on-site terms are added last, onto a sum that is still small.
__global__ void k_tc_sched(int32_t n_brow, int32_t row0, const int32_t* __restrict__ row_ptr,
                           const int32_t* __restrict__ col_idx, int32_t cap, int32_t* __restrict__ cnt,
                           int32_t* __restrict__ sJ, int32_t* __restrict__ sp) {
  const int32_t gi = blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t ngr = (n_brow + TC_G - 1) / TC_G;
  if (gi >= ngr) return;
  int32_t pos[TC_G], end[TC_G];
  for (int g = 0; g < TC_G; ++g) {
    const int32_t I = gi * TC_G + g;
    pos[g] = I < n_brow ? row_ptr[I] : 0;
    end[g] = I < n_brow ? row_ptr[I + 1] : 0;
  }
  int32_t start[TC_G];
  for (int g = 0; g < TC_G; ++g) start[g] = pos[g];
  const int32_t lo = gi * TC_G, hi = gi * TC_G + TC_G;
  int32_t e = 0;
  for (int own = 0; own < 2; ++own) {  // pass 0: J outside [lo, hi); pass 1: J inside
    for (int g = 0; g < TC_G; ++g) pos[g] = start[g];
    while (e < cap) {
      int32_t J = INT32_MAX;
      for (int g = 0; g < TC_G; ++g)
        if (pos[g] < end[g]) J = min(J, col_idx[pos[g]] - row0);
      if (J == INT32_MAX) break;
      const bool inside = J >= lo && J < hi;
      if (inside == (own == 1)) sJ[(size_t)gi * cap + e] = J;
      for (int g = 0; g < TC_G; ++g) {
        int32_t p = -1;
        if (pos[g] < end[g] && col_idx[pos[g]] - row0 == J) p = pos[g]++;
        if (inside == (own == 1)) sp[((size_t)gi * cap + e) * TC_G + g] = p;
      }
      if (inside == (own == 1)) ++e;
    }
  }
  cnt[gi] = e;
}

struct TcArgs {
  int32_t n_brow, b, ws, w, n_groups, n_tp, cap, row0;
  const float* Htc;
  const float* Hd3;
  const int32_t* cnt;
  const int32_t* sJ;
  const int32_t* sp;
  float* W;
  int* err;
};

__global__ void __launch_bounds__(TC_THREADS, 1) k_hv_tc(const __grid_constant__ CUtensorMap vmap, const TcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* sV = reinterpret_cast<float*>(smem);                                   // [NS][BK][256]
  unsigned char* sH = smem + (size_t)TC_NS * TC_VST;                            // [NS][HST]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)TC_NS * (TC_VST + TC_HST));
  uint64_t* full = bars;                 // [NS] TMA -> converters, MMA
  uint64_t* empty = bars + TC_NS;        // [NS] MMA commit -> producer
  uint64_t* aready = bars + 2 * TC_NS;   // [2] converters -> MMA
  uint64_t* afree = aready + 2;          // [2] MMA commit -> converters
  uint64_t* dfull = afree + 2;           // MMA commit -> epilogue
  uint64_t* dfree = dfull + 1;           // epilogue -> MMA
  uint64_t* tdone = dfree + 1;           // MMA commit at tear-down
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tdone + 1);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tdone + 2);
  // per stage: J and the G block indices of its entry (written by the producer before it arms
  // the stage's barrier); the producer's copy of the running item's schedule
  int32_t* hdr = reinterpret_cast<int32_t*>(smem + (size_t)TC_NS * (TC_VST + TC_HST) + TC_BAR);
  int32_t* sched = hdr + TC_NS * 4;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 9) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(su32(tslot)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < TC_NS; ++s) {
      bar_init(&full[s], 1);
      bar_init(&empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      bar_init(&aready[s], TC_CONV);
      bar_init(&afree[s], 1);
    }
    bar_init(dfull, 1);
    bar_init(dfree, TC_CONV);
    bar_init(tdone, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm = *tslot;
  const int32_t n_items = a.n_groups * a.n_tp;

  if (warp == 8) {
    // ------------------------------------------------------------ producer
    uint32_t q = 0;
    for (int32_t item = blockIdx.x; item < n_items && !*abort_flag; item += gridDim.x) {
      const int32_t gi = item / a.n_tp, tp = item - gi * a.n_tp;
      const int32_t ne = a.cnt[gi];
      // the warp copies the item's schedule to shared memory (off the per-entry critical path)
      for (int32_t i = lane; i < ne; i += 32) {
        const size_t ent = (size_t)gi * a.cap + i;
        sched[i * 4] = a.sJ[ent];
        for (int g = 0; g < TC_G; ++g) sched[i * 4 + 1 + g] = a.sp[ent * TC_G + g];
      }
      __syncwarp();
      if (lane == 0) {
        for (int32_t e = 0; e < ne; ++e, ++q) {
          const uint32_t s = q % TC_NS, use = q / TC_NS;
          if (!bar_wait(&empty[s], (use & 1) ^ 1, abort_flag, a.err)) break;
          const int32_t J = sched[e * 4];
          const int32_t drow = J - gi * TC_G;  // row slot whose diagonal block this is
          uint32_t bytes = TC_VST + ((drow >= 0 && drow < TC_G) ? TC_SL : 0);
          int32_t p[TC_G];
          hdr[s * 4] = J;
          for (int g = 0; g < TC_G; ++g) {
            p[g] = sched[e * 4 + 1 + g];
            hdr[s * 4 + 1 + g] = p[g];
            if (p[g] >= 0) bytes += 2 * TC_SL;
          }
          bar_expect(&full[s], bytes);  // releases the header stores with the arrival
          tma_v(sV + (size_t)s * TC_BK * TC_COLS, &vmap, tp * TC_COLS, J * a.b, &full[s]);
          unsigned char* hs = sH + (size_t)s * TC_HST;
          for (int g = 0; g < TC_G; ++g)
            if (p[g] >= 0) bulk_g2s(hs + g * 2 * TC_SL, a.Htc + (size_t)p[g] * 2 * (TC_SL / 4), 2 * TC_SL, &full[s]);
          if (drow >= 0 && drow < TC_G)
            bulk_g2s(hs + TC_G * 2 * TC_SL, a.Hd3 + (size_t)(a.row0 + J) * (TC_SL / 4), TC_SL, &full[s]);
        }
      }
      __syncwarp();  // the schedule buffer is reused by the next item
    }
    if (lane == 0) {  // tear-down: the copies of the last stages may still be in flight
      const uint32_t q0 = q > TC_NS ? q - TC_NS : 0;
      for (uint32_t r = q0; r < q; ++r) bar_drain(&full[r % TC_NS], (r / TC_NS) & 1);
    }
  } else if (warp == 9) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t q = 0, it = 0;
      bool issued = false;
      for (int32_t item = blockIdx.x; item < n_items && !*abort_flag; item += gridDim.x, ++it) {
        const int32_t gi = item / a.n_tp, tp = item - gi * a.n_tp;
        const int32_t ne = a.cnt[gi];
        const int ntile = (a.w - tp * TC_COLS > TC_TILE) ? 2 : 1;
        if (!bar_wait(dfree, (it & 1) ^ 1, abort_flag, a.err)) break;
        tc_fence_after();
        uint32_t written = 0;  // bit g*2+t: D[g][t] holds this item's partial sum
        bool ok = true;
        for (int32_t e = 0; e < ne; ++e, ++q) {
          const uint32_t s = q % TC_NS, use = q / TC_NS, slot = q & 1, ause = q >> 1;
          if (!bar_wait(&full[s], use & 1, abort_flag, a.err) || !bar_wait(&aready[slot], ause & 1, abort_flag, a.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const int32_t J = hdr[s * 4];
          const uint32_t hbase = su32(sH + (size_t)s * TC_HST);
          for (int g = 0; g < TC_G; ++g) {
            if (hdr[s * 4 + 1 + g] < 0) continue;
            const bool diag = J == gi * TC_G + g;
            for (int t = 0; t < ntile; ++t) {
              const uint32_t d = tm + (uint32_t)((g * 2 + t) * TC_BN);
              for (int kk = 0; kk < TC_BK / 8; ++kk) {
                const uint32_t h1 = hbase + g * 2 * TC_SL + kk * 256, h2 = h1 + TC_SL;
                const uint32_t av = tm + (uint32_t)TC_ACOL(slot, t, 0) + kk * 8;
                bool acc = (written >> (g * 2 + t)) & 1;
                mma_tf32(d, av, smem_desc(h1), acc);  // h1 v1
                mma_tf32(d, av + TC_BK, smem_desc(h1), true);      // h1 v2
                mma_tf32(d, av, smem_desc(h2), true);              // h2 v1
                if (diag) {
                  const uint32_t h3 = hbase + TC_G * 2 * TC_SL + kk * 256;
                  mma_tf32(d, av + 2 * TC_BK, smem_desc(h1), true);  // h1 v3
                  mma_tf32(d, av + TC_BK, smem_desc(h2), true);      // h2 v2
                  mma_tf32(d, av, smem_desc(h3), true);              // h3 v1
                }
                written |= 1u << (g * 2 + t);
              }
            }
          }
          issued = true;
          mma_commit(&empty[s]);
          mma_commit(&afree[slot]);
        }
        if (!ok) break;
        mma_commit(dfull);
      }
      if (issued) {  // tear-down: every MMA of this CTA has finished before the memory is freed
        mma_commit(tdone);
        bar_drain(tdone, 0);
      }
    }
  } else {
    // ------------------------------------------------- converters and epilogue
    const int tile = tid >> 7, m = tid & 127;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    uint32_t q = 0, it = 0;
    for (int32_t item = blockIdx.x; item < n_items && !*abort_flag; item += gridDim.x, ++it) {
      const int32_t gi = item / a.n_tp, tp = item - gi * a.n_tp;
      const int32_t ne = a.cnt[gi];
      const bool live = a.w - tp * TC_COLS > tile * TC_TILE;  // the tile has columns (warp-uniform)
      bool ok = true;
      for (int32_t e = 0; e < ne; ++e, ++q) {
        const uint32_t s = q % TC_NS, use = q / TC_NS, slot = q & 1, ause = q >> 1;
        // every lane waits (bounded), then the warp decides together, so that no lane is left
        // behind in a warp-collective instruction
        bool w_ok = bar_wait(&full[s], use & 1, abort_flag, a.err);
        w_ok = bar_wait(&afree[slot], (ause & 1) ^ 1, abort_flag, a.err) && w_ok;
        if (!__all_sync(0xffffffffu, w_ok)) {
          ok = false;
          break;
        }
        tc_fence_after();
        if (live) {
          const int32_t J = hdr[s * 4];
          const bool diag = J >= gi * TC_G && J < gi * TC_G + TC_G;  // warp-uniform
          const float* v = sV + (size_t)s * TC_BK * TC_COLS + tid;
          const uint32_t acol = tm + lane_base + (uint32_t)TC_ACOL(slot, tile, 0);
#pragma unroll
          for (int c = 0; c < TC_BK / 8; ++c) {
            uint32_t x1[8], x2[8], x3[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const float x = v[(c * 8 + i) * TC_COLS];
              x1[i] = tf32_rna(x);
              const float r = x - __uint_as_float(x1[i]);  // exact
              x2[i] = tf32_rna(r);
              x3[i] = tf32_rna(r - __uint_as_float(x2[i]));  // exact difference
            }
            tmem_st8(acol + c * 8, x1);
            tmem_st8(acol + TC_BK + c * 8, x2);
            if (diag) tmem_st8(acol + 2 * TC_BK + c * 8, x3);
          }
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        tc_fence_before();
        bar_arrive(&aready[slot]);
      }
      if (!ok) break;
      // epilogue: D[g][tile] -> W rows of the group
      if (!__all_sync(0xffffffffu, bar_wait(dfull, it & 1, abort_flag, a.err))) break;
      tc_fence_after();
      if (live) {
        const int32_t col = tp * TC_COLS + tile * TC_TILE + m;
        for (int g = 0; g < TC_G; ++g) {
          const int32_t I = gi * TC_G + g;
          if (I >= a.n_brow) break;
          uint32_t r[32];
          tmem_ld32(tm + lane_base + (uint32_t)((g * 2 + tile) * TC_BN), r);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (col < a.w) {
            float* out = a.W + (size_t)I * a.b * a.ws + col;
#pragma unroll
            for (int k = 0; k < TC_BK; ++k)
              if (k < a.b) out[(size_t)k * a.ws] = __uint_as_float(r[k]);
          }
        }
      }
      tc_fence_before();
      bar_arrive(dfree);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 9) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tm) : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

}  // namespace

bool css_hv_tc_supported(bool fp32, int32_t b, int32_t max_row_blocks) {
  return fp32 && b > 16 && b <= TC_BK && TC_G * max_row_blocks <= TC_SCHED_MAX;
}

css_status css_hv_tc_prepare(css_ctx* ctx, int32_t b, int32_t n_brow, int32_t nnzb, const int32_t* row_ptr,
                             const int32_t* col_idx, const double* H, const void** Htc, const void** Hd3,
                             cudaStream_t st) {
  constexpr int E = TC_BK * TC_BK;
  float *h, *d;
  CSS_TRY(css_ws(ctx, "tc_h", (size_t)nnzb * 2 * E * sizeof(float), (void**)&h));
  CSS_TRY(css_ws(ctx, "tc_hd3", (size_t)n_brow * E * sizeof(float), (void**)&d));
  const int64_t n = std::max((int64_t)nnzb, (int64_t)n_brow) * E;
  k_tc_hprep<<<(unsigned)css_ceil_div(n, 256), 256, 0, st>>>(nnzb, n_brow, b, H, row_ptr, col_idx, h, d);
  CSS_LAUNCHED(ctx);
  int* err;  // the time-out flag starts clear for this call
  CSS_TRY(css_ws(ctx, "tc_err", 256, (void**)&err));
  CSS_CU(ctx, cudaMemsetAsync(err, 0, sizeof(int), st));
  *Htc = h;
  *Hd3 = d;
  return CSS_OK;
}

css_status css_hv_tc_schedule(css_ctx* ctx, LzArgs& a, cudaStream_t st) {
  const int32_t ngr = (int32_t)css_ceil_div(a.n_brow, TC_G);
  const int32_t cap = TC_G * std::max(a.max_row_blocks, 1);
  int32_t *cnt, *sJ, *sp;
  CSS_TRY(css_ws(ctx, "tc_cnt", sizeof(int32_t) * ngr, (void**)&cnt));
  CSS_TRY(css_ws(ctx, "tc_sJ", sizeof(int32_t) * (size_t)ngr * cap, (void**)&sJ));
  CSS_TRY(css_ws(ctx, "tc_sp", sizeof(int32_t) * (size_t)ngr * cap * TC_G, (void**)&sp));
  k_tc_sched<<<(unsigned)css_ceil_div(ngr, 128), 128, 0, st>>>(a.n_brow, a.row0, a.row_ptr, a.col_idx, cap, cnt, sJ,
                                                                sp);
  CSS_LAUNCHED(ctx);
  a.tc_cnt = cnt;
  a.tc_sJ = sJ;
  a.tc_sp = sp;
  a.tc_cap = cap;
  a.tc_groups = ngr;
  return CSS_OK;
}

css_status css_hv_tc(css_ctx* ctx, const LzArgs& a, const float* V, float* W, cudaStream_t st) {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  });
  if (!g_encode) return css_set_arg_error(ctx, "H*V: cuTensorMapEncodeTiled is not available");
  if (((uintptr_t)V & 15) || (a.ws & 3)) return css_set_arg_error(ctx, "H*V: V must be 16-byte aligned");
  CUtensorMap map;
  const cuuint64_t gdim[2] = {(cuuint64_t)a.ws, (cuuint64_t)a.n_brow * a.b};
  const cuuint64_t gstride[1] = {(cuuint64_t)a.ws * sizeof(float)};
  const cuuint32_t box[2] = {TC_COLS, TC_BK};
  const cuuint32_t es[2] = {1, 1};
  const CUresult cr = g_encode(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)V, gdim, gstride, box, es,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return css_set_arg_error(ctx, "H*V: cuTensorMapEncodeTiled failed");
  int* err;
  CSS_TRY(css_ws(ctx, "tc_err", 256, (void**)&err));
  TcArgs t;
  t.n_brow = a.n_brow;
  t.b = a.b;
  t.ws = a.ws;
  t.w = a.w;
  t.n_groups = a.tc_groups;
  t.n_tp = (int32_t)css_ceil_div(a.w, TC_COLS);
  t.cap = a.tc_cap;
  t.row0 = a.row0;
  t.Htc = (const float*)a.tc_H;
  t.Hd3 = (const float*)a.tc_Hd3;
  t.cnt = a.tc_cnt;
  t.sJ = a.tc_sJ;
  t.sp = a.tc_sp;
  t.W = W;
  t.err = err;
  CSS_CU(ctx, cudaFuncSetAttribute(k_hv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
  const int64_t n_items = (int64_t)t.n_groups * t.n_tp;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ctx->n_sm, n_items));
  k_hv_tc<<<grid, TC_THREADS, TC_SMEM, st>>>(map, t);
  CSS_LAUNCHED(ctx);
  return CSS_OK;
}

// CSS_ERR_TIMEOUT when a wait of the tensor-core H * V ran out since the last check (the flag is
// cleared); synchronises the stream
css_status css_hv_tc_check(css_ctx* ctx, cudaStream_t st) {
  int* err;
  CSS_TRY(css_ws(ctx, "tc_err", 256, (void**)&err));
  int* h;
  CSS_TRY(css_pinned(ctx, 64, (void**)&h));
  CSS_CU(ctx, cudaMemcpyAsync(h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CSS_CU(ctx, cudaMemsetAsync(err, 0, sizeof(int), st));
  CSS_CU(ctx, cudaStreamSynchronize(st));
  if (*h) {
    ctx->last_error = "H*V (tensor cores): a bounded wait between pipeline stages timed out";
    return CSS_ERR_TIMEOUT;
  }
  return CSS_OK;
}
