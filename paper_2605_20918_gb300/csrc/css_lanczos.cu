// Block-Lanczos on CSS probe blocks, all colours of a batch at once (paper: paragraph after
// Eq. 4, Golub-Underwood block-Lanczos; SpMM-only cost noted after Eq. 10).
//
// Krylov blocks of a batch of colours live side by side as the columns of one N x w matrix
// (row-major, row stride ws, w = b * colours): colour c of the batch owns columns
// [c b, c b + b).  One step j is
//     W = H Q_j                                       (k_spmm: every H block times all w columns)
//     W0 = W - Q_{j-1} B_{j-1}^T;  A_j = sym(Q_j^T W0)                     (k_s1)
//     W1 = W0 - Q_j (Q_j^T W0) - Q_{j-1} (Q_{j-1}^T W0)  (local reorthogonalisation; k_s3)
//     W1 = Q_{j+1} B_j by shifted CholeskyQR3: R = chol(W^T W [+ shift]), W R^-1, three times
//                                                      (k_chol, k_tri)
// Small per-colour matrices (A_j, B_j, Grams, Cholesky factors) are FP64; the per-row-chunk
// partial products are combined in FP64 in a fixed order, so every run is bitwise
// reproducible (a second pass regenerates the same basis).
#include "css_lanczos.cuh"

namespace {

// ------------------------------------------------------------------------ H * V
// H is kept as transposed, zero-padded BM x BM blocks: Ht[p][k][a] = H_p[a][k] (a, k < b), 0
// elsewhere (k_hpad, once per build), so a block is one contiguous run of 16-byte chunks and a
// column k of H_p is BM contiguous values.
//
// One CTA per (block row I, tile of 128*TC columns); blockIdx.x runs over I so the CTAs in
// flight share one column tile and the V rows they gather stay in L2.  Thread t owns TC
// contiguous columns (one 16-, 8- or 4-byte chunk per row) and all BM rows of W_I for them.
// The neighbours J of row I are walked through a two-stage shared-memory ring filled by
// cp.async: while step q is multiplied, the copies of step q+1 (the H block, and each
// thread's own chunk of the b rows of V_J, rows >= b and columns >= w zero-filled) are in
// flight.  In FP32 mode a last virtual step adds the low FP32 parts of the diagonal block
// times V_I.
template <typename T, int BM, int TC, int NT_>
struct SpmmCfg {
  static constexpr int NT = NT_;                 // threads
  static constexpr int CT = NT * TC;             // columns per tile
  static constexpr int CH = TC * sizeof(T);      // bytes of a thread's chunk of a row
  static constexpr int HB = BM * BM * (int)sizeof(T);  // bytes of one padded block
  static constexpr size_t stage = (size_t)BM * CT * sizeof(T) + HB;
  static constexpr size_t smem = 2 * stage;
};

template <int CH>
__device__ __forceinline__ void cp_async_chunk(void* dst, const void* src, int bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (CH == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(bytes) : "memory");
  else if constexpr (CH == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(bytes) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename T, int BM, int TC, int NT>
__global__ void __launch_bounds__(NT) k_spmm(int32_t b, const int32_t* __restrict__ row_ptr,
                                              const int32_t* __restrict__ col_idx, const T* __restrict__ Ht,
                                              const T* __restrict__ V, T* __restrict__ W, int32_t ws, int32_t w,
                                              const T* __restrict__ Hlo_t, int32_t jbase) {
  using C = SpmmCfg<T, BM, TC, NT>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int32_t I = blockIdx.x;
  const int32_t t = threadIdx.x;
  const int32_t col = blockIdx.y * C::CT + TC * t;  // first of this thread's columns
  const int32_t p0 = row_ptr[I], p1 = row_ptr[I + 1];
  const int32_t nsteps = (p1 - p0) + (Hlo_t ? 1 : 0);
  // bytes of this thread's chunk that lie inside the matrix (0 beyond the last column)
  const int cbytes = col >= w ? 0 : (w - col >= TC ? C::CH : (w - col) * (int)sizeof(T));
  const bool warp_live = blockIdx.y * C::CT + TC * 32 * (t >> 5) < w;  // some column of the warp
  auto stage_v = [&](int s) { return reinterpret_cast<T*>(smem_raw + s * C::stage); };
  auto stage_h = [&](int s) { return reinterpret_cast<T*>(smem_raw + s * C::stage + (size_t)BM * C::CT * sizeof(T)); };
  auto issue = [&](int32_t q, int32_t J, int s) {
    const bool lo = q == p1 - p0;  // the diagonal low-part step
    const unsigned char* hsrc =
        reinterpret_cast<const unsigned char*>(lo ? Hlo_t + (size_t)I * BM * BM : Ht + (size_t)(p0 + q) * BM * BM);
    unsigned char* hdst = reinterpret_cast<unsigned char*>(stage_h(s));
    for (int32_t o = t * 16; o < C::HB; o += C::NT * 16) cp_async_chunk<16>(hdst + o, hsrc + o, 16);
    T* vd = stage_v(s) + TC * t;
    const T* vsrc = V + (size_t)J * b * ws + (col < w ? col : 0);
#pragma unroll
    for (int k = 0; k < BM; ++k)
      cp_async_chunk<C::CH>(vd + (size_t)k * C::CT, vsrc + (size_t)(k < b ? k : 0) * ws, k < b ? cbytes : 0);
    cp_async_commit();
  };
  // FP32: accumulators packed in pairs of adjacent rows (a, a+1) and updated with the packed
  // FMA fma.rn.f32x2 (two IEEE round-to-nearest FMAs per instruction, element by element the
  // same arithmetic as two scalar FMAs): the H pair comes from one 8-byte shared load, the V
  // value is packed into both halves once per k.  FP64: one scalar FMA per element.
  constexpr bool PACK = sizeof(T) == 4;
  constexpr int AP = PACK ? BM / 2 : 1;
  unsigned long long acc2[AP][TC];
  T acc[PACK ? 1 : BM][TC];
#pragma unroll
  for (int a = 0; a < AP; ++a)
#pragma unroll
    for (int u = 0; u < TC; ++u) acc2[a][u] = 0ull;
#pragma unroll
  for (int a = 0; a < (PACK ? 1 : BM); ++a)
#pragma unroll
    for (int u = 0; u < TC; ++u) acc[a][u] = T(0);
  if (nsteps > 0) {
    int32_t Jn = p0 < p1 ? col_idx[p0] - jbase : I;
    issue(0, Jn, 0);
    Jn = (1 < p1 - p0) ? col_idx[p0 + 1] - jbase : I;
    for (int32_t q = 0; q < nsteps; ++q) {
      const int s = q & 1;
      if (q + 1 < nsteps) {
        issue(q + 1, Jn, s ^ 1);
        Jn = (q + 2 < p1 - p0) ? col_idx[p0 + q + 2] - jbase : I;  // its latency overlaps the multiply
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();  // the H block of step q (copied by every thread) is visible
      if (warp_live) {
        const T* hs = stage_h(s);
        const T* vs = stage_v(s) + TC * t;
        if constexpr (PACK) {
#pragma unroll 4
          for (int k = 0; k < BM; ++k) {
            unsigned long long vv[TC];
#pragma unroll
            for (int u = 0; u < TC; ++u) {
              const float x = (float)vs[(size_t)k * C::CT + u];
              asm("mov.b64 %0, {%1, %1};" : "=l"(vv[u]) : "f"(x));
            }
            const unsigned long long* hp = reinterpret_cast<const unsigned long long*>(hs + k * BM);
#pragma unroll
            for (int a = 0; a < AP; ++a) {
              const unsigned long long h2 = hp[a];
#pragma unroll
              for (int u = 0; u < TC; ++u) asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc2[a][u]) : "l"(h2), "l"(vv[u]));
            }
          }
        } else {
#pragma unroll 4
          for (int k = 0; k < BM; ++k) {
            T v[TC];
#pragma unroll
            for (int u = 0; u < TC; ++u) v[u] = vs[(size_t)k * C::CT + u];
#pragma unroll
            for (int a = 0; a < BM; ++a) {
              const T h = hs[k * BM + a];
#pragma unroll
              for (int u = 0; u < TC; ++u) acc[a][u] = fma(h, v[u], acc[a][u]);
            }
          }
        }
      }
      __syncthreads();  // stage s is free for step q + 2
    }
  }
  if (col >= w) return;
  T* Wr = W + (size_t)I * b * ws + col;
  auto out = [&](int a, int u) -> T {
    if constexpr (PACK) {
      const unsigned long long x = acc2[a >> 1][u];
      return (T)__uint_as_float((unsigned)((a & 1) ? (x >> 32) : (x & 0xffffffffull)));
    } else {
      return acc[a][u];
    }
  };
#pragma unroll
  for (int a = 0; a < BM; ++a) {
    if (a >= b) break;
    if (cbytes == C::CH) {
      if constexpr (C::CH == 16 && sizeof(T) == 4) {
        *reinterpret_cast<float4*>(Wr + (size_t)a * ws) = make_float4(out(a, 0), out(a, 1), out(a, 2), out(a, 3));
      } else if constexpr (C::CH == 16) {
        *reinterpret_cast<double2*>(Wr + (size_t)a * ws) = make_double2(out(a, 0), out(a, 1));
      } else {
#pragma unroll
        for (int u = 0; u < TC; ++u) Wr[(size_t)a * ws + u] = out(a, u);
      }
    } else {
#pragma unroll
      for (int u = 0; u < TC; ++u)
        if (col + u < w) Wr[(size_t)a * ws + u] = out(a, u);
    }
  }
}

// Ht[p][k][a] = H_p[a][k] for a, k < b, zero padding to BM x BM; the source is FP64 [p][b][b].
// LO: only the blocks p = diag[I] (the diagonal block of row I), and the FP32 remainder
// fl32(h - fl32(h)) of each entry.
template <typename T, bool LO>
__global__ void k_hpad(int64_t nblocks, int32_t b, int32_t BM, const double* __restrict__ H,
                       const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                       T* __restrict__ Ht) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t bb = (int64_t)BM * BM;
  if (e >= nblocks * bb) return;
  const int64_t p = e / bb;
  const int32_t r = (int32_t)(e - p * bb), k = r / BM, a = r - k * BM;
  T v = T(0);
  if (a < b && k < b) {
    int64_t src = p;
    if (LO) {  // the row's diagonal block; a row without one has no low part
      int32_t q = row_ptr[p];
      while (q < row_ptr[p + 1] && col_idx[q] != (int32_t)p) ++q;
      src = q < row_ptr[p + 1] ? q : -1;
    }
    if (src >= 0) {
      const double h = H[(size_t)src * b * b + (size_t)a * b + k];
      v = LO ? (T)(h - (double)(float)h) : (T)h;
    }
  }
  Ht[e] = v;
}

// --------------------------------------------------------------- row-chunk kernels
// CTA = (chunk of RCHK rows, group of G colours).  The chunk is walked in tiles of RTL rows;
// a tile of each array is staged in shared memory as [RTL][G*BP] (b padded to BP, the
// padding kept at zero), so the global reads of a row are G*b contiguous values.  Every
// small product (block update, Gram) is register-tiled in 4 x 4 blocks.  Per-tile Gram sums
// are taken in the vector precision; FP32 tiles are added into an unevaluated hi + lo pair
// of floats (error-free TwoSum, so the running sum carries about 44 bits), FP64 tiles into
// doubles.  The pair is widened to FP64 once per CTA: no FP64 arithmetic in the row loop.
constexpr int RW = 256;      // threads of a Gram half (see the launch sizes below)
constexpr int RCHK = 1024;   // rows per CTA

// colours of a staged tile sit CS = BP + 4 values apart: for BP = 24 the seven colours of a
// group start in seven different shared-memory banks
template <int BP>
struct ColStride {
  static constexpr int CS = BP + 4;
  // per-colour small matrices [G][BP][BP] sit MS = BP*BP + BP values apart: MS = BP (mod 32), so
  // the 16-byte loads of a quarter warp that spans two colours fall in distinct banks
  static constexpr int MS = BP * BP + BP;
};

// Tiles, Gram partials and ring depths of the row kernels.  The Gram sums of GRP consecutive rows
// are taken in the vector precision and then added into the running sum (FP32: the compensated
// hi + lo pair; FP64: doubles).  The kernels that stage three arrays per tile (k_s1, k_s3) walk
// tiles of RTL3 rows through NS3 stages, k_tri tiles of RTL1 rows through NS1 stages (row_pipeline:
// two stages run the barrier-separated schedule, three or more the overlapped one).  The depths
// are the fastest measured: FP32 with b = 23 (BP = 24) two stages of 32-row tiles, FP32 with
// b <= 16 three, FP64 three (k_s1, k_s3) and four (k_tri) stages of 16-row tiles.  None of them
// changes a result: every sum keeps its order.
template <typename T, int BP>
struct RowTile {
  static constexpr bool f32 = sizeof(T) == 4;
  static constexpr int GRP = f32 ? 32 : 16;
  static constexpr int RTL3 = f32 ? 32 : 16;
  static constexpr int NS3 = f32 && BP >= 24 ? 2 : 3;
  static constexpr int RTL1 = f32 ? 32 : 16;
  static constexpr int NS1 = f32 ? (BP >= 24 ? 2 : 3) : 4;
};
constexpr size_t kRowSmemMax = 227 * 1024;  // opt-in dynamic shared memory of one CTA

template <int BP>
__host__ __device__ constexpr int group_cap() {
  return RW / ((BP / 4) * (BP / 4));
}

// colours per CTA for block width b (runtime) padded to BP: at most group_cap (one Gram thread
// per 4 x 4 block), at most 192 contiguous columns per row, and small enough that the NS3-stage
// ring of three tiles plus two per-colour matrices fits in one CTA's shared memory
template <typename T, int BP>
__host__ __device__ inline int colours_per_cta(int b) {
  int g = group_cap<BP>();
  if (g > 192 / b) g = 192 / b;
  constexpr size_t row_bytes = (size_t)RowTile<T, BP>::RTL3 * sizeof(T);
  while (g > 1 && (size_t)RowTile<T, BP>::NS3 * 3 * row_bytes * (g * (BP + 4) + 4) +
                          2 * (size_t)g * (BP * BP + BP) * sizeof(T) >
                      kRowSmemMax)
    --g;
  return g < 1 ? 1 : g;
}

// A symmetric Gram has CB (CB + 1) / 2 blocks per colour.  Where twice that many threads are
// no more than max(GRP / 4, CB) CB per colour, two threads share a block, the first summing the
// first half of every GRP-row group and the second the second half (gram_store adds the two sums
// in FP64, in that order).
template <typename T, int BP>
__host__ __device__ constexpr bool sym_split() {
  constexpr int CB = BP / 4, a = (RowTile<T, BP>::GRP / 4) * CB, g = CB * CB;
  return CB * (CB + 1) <= (a > g ? a : g);
}

// threads of a k_s3 / k_tri launch (tiles of RTL rows): one per 4 x 4 output block of a tile
// (every block in one round), one per Gram block, two per block of a split symmetric Gram; whole
// warps
template <typename T, int BP, int RTL>
__host__ __device__ inline int row_threads(int b) {
  constexpr int CB = BP / 4;
  const int G = colours_per_cta<T, BP>(b);
  const int items = (RTL / 4) * G * CB, gram = G * CB * CB;
  int t = items > gram ? items : gram;
  if (sym_split<T, BP>() && G * CB * (CB + 1) > t) t = G * CB * (CB + 1);
  return (t + 31) / 32 * 32;
}

template <typename T, int BP>
struct RowCtx {
  int32_t b, ws, G, gcount, pitch, cg0;  // cg0 = first colour of the group within the batch
  int32_t my_col, my_smem;  // this thread's column of the group (width <= blockDim) and its tile offset
  // issue the asynchronous copy of one tile of RTL rows (rows >= nr are zero-filled); the copies
  // hold no registers, so every row of the tile is in flight at once.  The caller commits the
  // group and waits for it (cp_async_commit / cp_async_wait).
  template <int RTL>
  __device__ __forceinline__ void load(T* dst, const T* src, int64_t r0, int32_t nr) const {
    if (my_col < 0) return;
    const T* s = src + (size_t)r0 * ws + (size_t)cg0 * b + my_col;
#pragma unroll 4
    for (int32_t r = 0; r < RTL; ++r)
      cp_async_chunk<sizeof(T)>(dst + r * pitch + my_smem, s + (size_t)(r < nr ? r : 0) * ws,
                                r < nr ? (int)sizeof(T) : 0);
  }
  __device__ __forceinline__ void store(T* dst, const T* src, int64_t r0, int32_t nr) const {
    if (my_col < 0) return;
    T* d = dst + (size_t)r0 * ws + (size_t)cg0 * b + my_col;
#pragma unroll 4
    for (int32_t r = 0; r < nr; ++r) d[(size_t)r * ws] = src[r * pitch + my_smem];
  }
  // zero a whole tile (padding columns and missing rows stay zero afterwards)
  __device__ __forceinline__ void zero(T* t, int32_t rows) const {
    for (int32_t e = threadIdx.x; e < rows * pitch; e += blockDim.x) t[e] = T(0);
  }
  // small per-colour matrices [G][BP][BP] from global FP64 [colour][b][b] (optionally transposed)
  __device__ __forceinline__ void load_mat(T* dst, const double* src, int32_t colour0, bool trans) const {
    constexpr int MS = ColStride<BP>::MS;
    for (int32_t e = threadIdx.x; e < G * MS; e += blockDim.x) {
      const int32_t g = e / MS, rem = e - g * MS, l = rem / BP, k = rem - l * BP;
      T v = T(0);
      if (g < gcount && l < b && k < b)
        v = (T)src[(size_t)(colour0 + g) * b * b + (trans ? k * b + l : l * b + k)];
      dst[e] = v;
    }
  }
};

// OUT[r][g][k] (+)= sum_l X[r][g][l] M[g][l][k] over 4x4 output blocks.  SUB: OUT -= X M.
// TWO: a second product X2 M2 in the same pass (OUT -= X M + X2 M2)
template <typename T, int BP, bool SUB, bool TWO>
__device__ __forceinline__ void tile_mul(const RowCtx<T, BP>& c, const T* X, const T* M, T* OUT, int32_t rtl,
                                         const T* X2, const T* M2) {
  constexpr int CS = ColStride<BP>::CS;
  constexpr int CB = BP / 4;
  const int32_t nblk = (rtl / 4) * c.G * CB;
  if constexpr (sizeof(T) == 4) {
    // FP32: the four columns of a row in two packed pairs, fma.rn.f32x2 against the row's x
    // duplicated into both halves: element by element the same IEEE FMAs in the same order as
    // the scalar loop below (4-column blocks start on 16-byte boundaries: CS, BP, pitch and MS
    // are multiples of 4)
    for (int32_t t = threadIdx.x; t < nblk; t += blockDim.x) {
      const int32_t rb = t / (c.G * CB), rem = t - rb * c.G * CB, g = rem / CB, cb = rem - g * CB;
      const int32_t r0 = rb * 4, col = g * CS + cb * 4;
      unsigned long long acc[4][2];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (SUB) {
          const ulonglong2 o = *reinterpret_cast<const ulonglong2*>(OUT + (r0 + i) * c.pitch + col);
          acc[i][0] = o.x;
          acc[i][1] = o.y;
        } else {
          acc[i][0] = acc[i][1] = 0ull;
        }
      }
      auto accumulate = [&](const T* Xs, const T* Ms) {
        const T* xm = Xs + g * CS;
        const T* mm = Ms + (size_t)g * ColStride<BP>::MS + cb * 4;
        for (int32_t l = 0; l < c.b; ++l) {
          const ulonglong2 m = *reinterpret_cast<const ulonglong2*>(mm + l * BP);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float x = SUB ? -(float)xm[(r0 + i) * c.pitch + l] : (float)xm[(r0 + i) * c.pitch + l];
            unsigned long long xx;
            asm("mov.b64 %0, {%1, %1};" : "=l"(xx) : "f"(x));
            asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc[i][0]) : "l"(xx), "l"(m.x));
            asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc[i][1]) : "l"(xx), "l"(m.y));
          }
        }
      };
      accumulate(X, M);
      if (TWO) accumulate(X2, M2);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        *reinterpret_cast<ulonglong2*>(OUT + (r0 + i) * c.pitch + col) = make_ulonglong2(acc[i][0], acc[i][1]);
    }
    return;
  }
  for (int32_t t = threadIdx.x; t < nblk; t += blockDim.x) {
    const int32_t rb = t / (c.G * CB), rem = t - rb * c.G * CB, g = rem / CB, cb = rem - g * CB;
    const int32_t r0 = rb * 4, col = g * CS + cb * 4;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = SUB ? OUT[(r0 + i) * c.pitch + col + j] : T(0);
    const T* xm = X + g * CS;
    const T* mm = M + (size_t)g * ColStride<BP>::MS + cb * 4;
    for (int32_t l = 0; l < c.b; ++l) {
      T x[4], m[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) x[i] = xm[(r0 + i) * c.pitch + l];
#pragma unroll
      for (int j = 0; j < 4; ++j) m[j] = mm[l * BP + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = SUB ? fma(-x[i], m[j], acc[i][j]) : fma(x[i], m[j], acc[i][j]);
    }
    if (TWO) {
      const T* xm2 = X2 + g * CS;
      const T* mm2 = M2 + (size_t)g * ColStride<BP>::MS + cb * 4;
      for (int32_t l = 0; l < c.b; ++l) {
        T x[4], m[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) x[i] = xm2[(r0 + i) * c.pitch + l];
#pragma unroll
        for (int j = 0; j < 4; ++j) m[j] = mm2[l * BP + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = SUB ? fma(-x[i], m[j], acc[i][j]) : fma(x[i], m[j], acc[i][j]);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) OUT[(r0 + i) * c.pitch + col + j] = acc[i][j];
  }
}

// running sum of 16 Gram entries: doubles for FP64 vectors, hi + lo float pairs for FP32
template <typename T>
struct GramAcc {
  double s[16];
  __device__ __forceinline__ GramAcc() {
#pragma unroll
    for (int i = 0; i < 16; ++i) s[i] = 0.0;
  }
  __device__ __forceinline__ void add(int i, double x) { s[i] += x; }
  __device__ __forceinline__ double get(int i) const { return s[i]; }
};
template <>
struct GramAcc<float> {
  float hi[16], lo[16];
  __device__ __forceinline__ GramAcc() {
#pragma unroll
    for (int i = 0; i < 16; ++i) hi[i] = lo[i] = 0.0f;
  }
  // Knuth's TwoSum: hi + x = t + err exactly; err is collected in lo
  __device__ __forceinline__ void add(int i, float x) {
    const float t = __fadd_rn(hi[i], x);
    const float z = __fsub_rn(t, hi[i]);
    const float err = __fadd_rn(__fsub_rn(hi[i], __fsub_rn(t, z)), __fsub_rn(x, z));
    lo[i] = __fadd_rn(lo[i], err);
    hi[i] = t;
  }
  __device__ __forceinline__ double get(int i) const { return (double)hi[i] + (double)lo[i]; }
};

// Gram block of thread t: (g, bi, bj) over all CB x CB blocks, or with SYM (X = Y, a symmetric
// Gram) over the CB (CB + 1) / 2 blocks with bi <= bj only
template <int CB, bool SYM>
__device__ __forceinline__ bool gram_block(int32_t t, int32_t G, int32_t& g, int32_t& bi, int32_t& bj) {
  constexpr int NB = SYM ? CB * (CB + 1) / 2 : CB * CB;
  if (t >= G * NB) return false;
  g = t / NB;
  int32_t q = t - g * NB;
  if (!SYM) {
    bi = q / CB;
    bj = q - bi * CB;
    return true;
  }
  bi = 0;
  while (q >= CB - bi) {  // row bi holds the blocks bj = bi .. CB-1
    q -= CB - bi;
    ++bi;
  }
  bj = bi + q;
  return true;
}

// One thread's Gram block: (g, bi, bj) and, for a split symmetric Gram, its half of every
// GRP-row group (0 or 1); inactive threads hold none.
struct GramRole {
  bool active;
  int32_t t, g, bi, bj, half;  // t: index of the block among the CTA's Gram blocks
};

template <typename T, int BP, bool SYM>
__device__ __forceinline__ GramRole gram_role(int32_t G, int32_t t) {
  constexpr int CB = BP / 4;
  GramRole r;
  r.half = 0;
  if (SYM && sym_split<T, BP>()) {
    const int32_t nbt = G * (CB * (CB + 1) / 2);
    r.half = t / nbt;
    if (r.half >= 2) {
      r.active = false;
      r.t = r.g = r.bi = r.bj = 0;
      return r;
    }
    t -= r.half * nbt;
  }
  r.t = t;
  r.active = gram_block<CB, SYM>(t, G, r.g, r.bi, r.bj);
  return r;
}

// The running Gram partial of one 4 x 4 block over the rows since its last flush, in the vector
// precision: FP32 as packed pairs (columns j, j + 1 of row i in one 64-bit register, summed with
// fma.rn.f32x2: element by element the IEEE FMAs of a scalar loop), FP64 as plain values.
template <typename T>
struct GramPart {
  T a[4][4];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) a[i][j] = T(0);
  }
  // a[i][j] += sum over n rows of x[r][i] y[r][j] (x, y: the block's first column, row stride p)
  __device__ __forceinline__ void rows(const T* x, const T* y, int32_t p, int32_t n) {
    for (int32_t r = 0; r < n; ++r) {
      T xv[4], yv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        xv[i] = x[r * p + i];
        yv[i] = y[r * p + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) a[i][j] = fma(xv[i], yv[j], a[i][j]);
    }
  }
  __device__ __forceinline__ void flush(GramAcc<T>& acc) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc.add(i * 4 + j, a[i][j]);
    zero();
  }
};
template <>
struct GramPart<float> {
  unsigned long long a2[4][2];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < 4; ++i) a2[i][0] = a2[i][1] = 0ull;
  }
  __device__ __forceinline__ void rows(const float* x, const float* y, int32_t p, int32_t n) {
    for (int32_t r = 0; r < n; ++r) {
      const float4 xq = *reinterpret_cast<const float4*>(x + r * p);
      const ulonglong2 yq = *reinterpret_cast<const ulonglong2*>(y + r * p);
      const float xv[4] = {xq.x, xq.y, xq.z, xq.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        unsigned long long xx;
        asm("mov.b64 %0, {%1, %1};" : "=l"(xx) : "f"(xv[i]));
        asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(a2[i][0]) : "l"(xx), "l"(yq.x));
        asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(a2[i][1]) : "l"(xx), "l"(yq.y));
      }
    }
  }
  __device__ __forceinline__ void flush(GramAcc<float>& acc) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const unsigned long long q = a2[i][j >> 1];
        acc.add(i * 4 + j, __uint_as_float((unsigned)((j & 1) ? (q >> 32) : (q & 0xffffffffull))));
      }
    zero();
  }
};

// Gram rows of tile i (0-based within the CTA's chunk; `last`: the chunk's last tile) for this
// thread's block: part += X^T Y over the tile's rows (its half of them for a split Gram), then
// into acc at the end of each GRP-row group (of each half-group when split).  Rows past the
// end of the matrix are zero in the tile and add nothing.
template <typename T, int BP, bool SYM, int RTL>
__device__ __forceinline__ void gram_tile(const RowCtx<T, BP>& c, const GramRole& role, const T* X, const T* Y,
                                          int32_t i, bool last, GramPart<T>& part, GramAcc<T>& acc) {
  constexpr int CS = ColStride<BP>::CS;
  constexpr int GRP = RowTile<T, BP>::GRP, SEG = GRP / 2;
  static_assert(GRP % RTL == 0 && (RTL <= SEG || RTL == GRP), "tiles must tile the Gram groups");
  if (!role.active) return;
  const int32_t pos = (i * RTL) % GRP;  // offset of the tile in its GRP-row group
  int32_t lo = 0, n = RTL;
  bool flush = pos + RTL == GRP || last;
  if (SYM && sym_split<T, BP>()) {
    if constexpr (RTL <= SEG) {  // the tile lies in one half of its group
      if (pos / SEG != role.half) return;
      flush = (pos + RTL) % SEG == 0 || last;
    } else {  // the thread's half of the tile
      lo = role.half * SEG;
      n = SEG;
    }
  }
  const T* xp = X + lo * c.pitch + role.g * CS + role.bi * 4;
  const T* yp = Y + lo * c.pitch + role.g * CS + role.bj * 4;
  if constexpr (RTL == GRP) {  // every tile closes its group: the partial lives in this call only
    GramPart<T> local;
    local.zero();
    local.rows(xp, yp, c.pitch, n);
    local.flush(acc);
  } else {
    part.rows(xp, yp, c.pitch, n);
    if (flush) part.flush(acc);
  }
}

// every thread of the CTA calls this (a split Gram synchronises the CTA once; `scratch`: 16
// doubles per Gram block of shared memory no longer in use)
template <typename T, int BP, bool SYM = false>
__device__ __forceinline__ void gram_store(const RowCtx<T, BP>& c, const GramRole& role, const GramAcc<T>& acc,
                                           double* part, double* scratch = nullptr) {
  constexpr bool split = SYM && sym_split<T, BP>();
  const int32_t t = role.t;
  if (split) {
    if (role.active && role.half == 1)
#pragma unroll
      for (int i = 0; i < 16; ++i) scratch[t * 16 + i] = acc.get(i);
    __syncthreads();
    if (role.half != 0) return;
  }
  if (!role.active || role.g >= c.gcount) return;
  double* o = part + (size_t)(c.cg0 + role.g) * c.b * c.b;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int32_t k = role.bi * 4 + i, l = role.bj * 4 + j;
      if (k < c.b && l < c.b) {
        const double v = split ? acc.get(i * 4 + j) + scratch[t * 16 + i * 4 + j] : acc.get(i * 4 + j);
        o[k * c.b + l] = v;
        if (SYM && role.bi != role.bj) o[l * c.b + k] = v;  // the mirrored block of a symmetric Gram
      }
    }
}

template <typename T, int BP>
__device__ __forceinline__ RowCtx<T, BP> make_ctx(int32_t b, int32_t ws, int32_t ncb) {
  constexpr int CS = ColStride<BP>::CS;
  RowCtx<T, BP> c;
  c.b = b;
  c.ws = ws;
  c.G = colours_per_cta<T, BP>(b);
  c.cg0 = blockIdx.y * c.G;
  c.gcount = min(c.G, ncb - c.cg0);
  c.pitch = c.G * CS + 4;
  const int32_t t = threadIdx.x;
  if (t < c.gcount * b) {
    c.my_col = t;
    c.my_smem = (t / b) * CS + (t % b);
  } else {
    c.my_col = -1;
    c.my_smem = 0;
  }
  return c;
}

// The row kernels below walk their chunk of RCHK rows in tiles of RTL rows through an NS-stage
// shared-memory ring filled by cp.async.  Padding columns of a stage are zeroed once and never
// written by a copy; rows past the end of the matrix are zero-filled by the copies themselves.
template <typename T, int BP>
struct RowRing {
  T* base;
  int32_t tile, na;  // elements per tile, arrays per stage
  __device__ __forceinline__ T* at(int s, int a) const { return base + ((size_t)s * na + a) * tile; }
};

// Tiles of this CTA's chunk.  fn_issue(stage, tile, r0, nr) issues (does not commit) the copies
// of a tile, fn_mul(stage, tile, r0, nr) is its first phase (a block product in place in its
// stage), fn_fin(stage, tile, r0, nr, last) its second (stores and Gram sums of that product).
// Two stages: the barrier-separated schedule, per tile wait, barrier, first phase, barrier, second
// phase, with the next tile's copies in flight.  NS >= 3 stages: one barrier per tile; the copies
// run NS - 2 tiles ahead, and in the iteration of tile i the CTA works on two tiles at once, the
// first phase of tile i + 1 and the second phase of tile i (different stages, so no barrier
// separates them).
template <int NS, typename Issue, typename Mul, typename Fin>
__device__ __forceinline__ void row_pipeline(int64_t N, int32_t rtl, Issue fn_issue, Mul fn_mul, Fin fn_fin) {
  static_assert(NS >= 2, "the ring needs a stage in flight besides the one being worked on");
  const int64_t rbeg = (int64_t)blockIdx.x * RCHK, rend = min(N, rbeg + RCHK);
  if (rbeg >= rend) return;
  const int32_t ntile = (int32_t)((rend - rbeg + rtl - 1) / rtl);
  auto r0_of = [&](int32_t i) { return rbeg + (int64_t)i * rtl; };
  auto nr_of = [&](int32_t i) { return (int32_t)min((int64_t)rtl, rend - r0_of(i)); };
  if constexpr (NS == 2) {
    fn_issue(0, 0, r0_of(0), nr_of(0));
    cp_async_commit();
#pragma unroll 1
    for (int32_t it = 0; it < ntile; ++it) {
      const int s = it & 1;
      if (it + 1 < ntile) {
        fn_issue(s ^ 1, it + 1, r0_of(it + 1), nr_of(it + 1));
        cp_async_commit();
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();  // tile it is in shared memory for every thread
      fn_mul(s, it, r0_of(it), nr_of(it));
      __syncthreads();
      fn_fin(s, it, r0_of(it), nr_of(it), it + 1 == ntile);
      __syncthreads();  // stage s is free for tile it + 2
    }
    return;
  } else {
#pragma unroll 1
    for (int32_t i = 0; i < NS - 1; ++i) {  // one commit group per tile (empty past the end)
      if (i < ntile) fn_issue(i, i, r0_of(i), nr_of(i));
      cp_async_commit();
    }
    cp_async_wait<NS - 2>();  // this thread's copies of tile 0
    __syncthreads();
    fn_mul(0, 0, r0_of(0), nr_of(0));
#pragma unroll 1
    for (int32_t it = 0; it < ntile; ++it) {
      cp_async_wait<NS - 3>();  // this thread's copies of tile it + 1
      // every thread's copies of tile it + 1 and products of tile it are done, and tile it - 1
      // (finished in the previous iteration) has left its stage
      __syncthreads();
      const int32_t nx = it + NS - 1;
      if (nx < ntile) fn_issue(nx % NS, nx, r0_of(nx), nr_of(nx));
      cp_async_commit();
      if (it + 1 < ntile) fn_mul((it + 1) % NS, it + 1, r0_of(it + 1), nr_of(it + 1));
      fn_fin(it % NS, it, r0_of(it), nr_of(it), it + 1 == ntile);
    }
    __syncthreads();  // the stages are free (gram_store may reuse them as scratch)
  }
}

// S1: W = H Q_j arrives in W.  W0 = W - Q_{j-1} B_{j-1}^T (skipped at the first step), stored;
// partials Kq = Q_j^T W0 and Kp = Q_{j-1}^T W0 (REORTH).
// With REORTH the CTA has 2*RW threads: the first RW accumulate Kq, the second RW Kp.
template <typename T, int BP, bool REORTH>
__global__ void __launch_bounds__(REORTH ? 2 * RW : RW, 1)
    k_s1(int64_t N, int32_t b, int32_t ws, int32_t ncb, int32_t cb0, const T* __restrict__ Qp,
         const T* __restrict__ Q, T* __restrict__ W, const double* __restrict__ Bprev, int first,
         double* __restrict__ partKq, double* __restrict__ partKp) {
  constexpr int RTL = RowTile<T, BP>::RTL3, NS = RowTile<T, BP>::NS3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const RowCtx<T, BP> c = make_ctx<T, BP>(b, ws, ncb);
  const bool usep = REORTH || !first;
  RowRing<T, BP> ring{reinterpret_cast<T*>(smem_raw), RTL * c.pitch, 3};  // Q, Q_{j-1}, W
  T* sB = ring.at(NS, 0);                                                   // [G][BP][BP] B_{j-1}^T
  GramAcc<T> acc;                                   // Kq (first RW threads) or Kp (second RW)
  GramPart<T> gp;
  gp.zero();
  const bool second = REORTH && threadIdx.x >= RW;
  const GramRole role = gram_role<T, BP, false>(c.G, threadIdx.x - (second ? RW : 0));
  if (!first) c.load_mat(sB, Bprev, cb0 + c.cg0, true);
  c.zero(ring.at(0, 0), 3 * NS * RTL);
  __syncthreads();
  row_pipeline<NS>(
      N, RTL,
      [&](int s, int32_t, int64_t r0, int32_t nr) {
        c.template load<RTL>(ring.at(s, 0), Q, r0, nr);
        c.template load<RTL>(ring.at(s, 2), W, r0, nr);
        if (usep) c.template load<RTL>(ring.at(s, 1), Qp, r0, nr);
      },
      [&](int s, int32_t, int64_t, int32_t) {
        if (!first) tile_mul<T, BP, true, false>(c, ring.at(s, 1), sB, ring.at(s, 2), RTL, nullptr, nullptr);
      },
      [&](int s, int32_t i, int64_t r0, int32_t nr, bool last) {
        if (!first) c.store(W, ring.at(s, 2), r0, nr);
        gram_tile<T, BP, false, RTL>(c, role, ring.at(s, second ? 1 : 0), ring.at(s, 2), i, last, gp, acc);
      });
  const size_t o = (size_t)blockIdx.x * ncb;
  gram_store<T, BP>(c, role, acc, (second ? partKp : partKq) + o * b * b);
}

// S3: W1 = W0 - Q_j M1 (- Q_{j-1} M2), stored; partial Gram W1^T W1
template <typename T, int BP, bool REORTH>
__global__ void __launch_bounds__(2 * RW, 1)
    k_s3(int64_t N, int32_t b, int32_t ws, int32_t ncb, const T* __restrict__ Q, const T* __restrict__ Qp,
         T* __restrict__ W, const double* __restrict__ M1, const double* __restrict__ M2,
         double* __restrict__ partG) {
  constexpr int RTL = RowTile<T, BP>::RTL3, NS = RowTile<T, BP>::NS3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const RowCtx<T, BP> c = make_ctx<T, BP>(b, ws, ncb);
  RowRing<T, BP> ring{reinterpret_cast<T*>(smem_raw), RTL * c.pitch, 3};  // Q, Q_{j-1}, W
  T* sM1 = ring.at(NS, 0);
  T* sM2 = sM1 + c.G * ColStride<BP>::MS;
  GramAcc<T> acc;
  GramPart<T> gp;
  gp.zero();
  const GramRole role = gram_role<T, BP, true>(c.G, threadIdx.x);
  c.load_mat(sM1, M1, c.cg0, false);
  if (REORTH) c.load_mat(sM2, M2, c.cg0, false);
  c.zero(ring.at(0, 0), 3 * NS * RTL);
  __syncthreads();
  row_pipeline<NS>(
      N, RTL,
      [&](int s, int32_t, int64_t r0, int32_t nr) {
        c.template load<RTL>(ring.at(s, 0), Q, r0, nr);
        c.template load<RTL>(ring.at(s, 2), W, r0, nr);
        if (REORTH) c.template load<RTL>(ring.at(s, 1), Qp, r0, nr);
      },
      [&](int s, int32_t, int64_t, int32_t) {
        tile_mul<T, BP, true, REORTH>(c, ring.at(s, 0), sM1, ring.at(s, 2), RTL, ring.at(s, 1), sM2);
      },
      [&](int s, int32_t i, int64_t r0, int32_t nr, bool last) {
        c.store(W, ring.at(s, 2), r0, nr);
        gram_tile<T, BP, true, RTL>(c, role, ring.at(s, 2), ring.at(s, 2), i, last, gp, acc);
      });
  gram_store<T, BP, true>(c, role, acc, partG + (size_t)blockIdx.x * ncb * b * b,
                          reinterpret_cast<double*>(smem_raw));
}

// OUT = W R^-1 (R^-1 upper triangular per colour); partial Gram of OUT when GRAM.  OUT may be W.
// With three or more stages the products of consecutive tiles alternate between two output tiles.
// need3 (optional): the per-colour flags of k_chol<1>.  The second CholeskyQR pass (OUT2 set)
// writes the columns of a colour whose flag is clear to OUT2 (Q_{j+1}) instead of OUT; the third
// pass (OUT2 null) writes only the columns of colours whose flag is set, and a CTA none of whose
// colours needs it returns at once.
template <typename T, int BP, bool GRAM>
__global__ void __launch_bounds__(384, 2)
    k_tri(int64_t N, int32_t b, int32_t ws, int32_t ncb, const T* __restrict__ W, T* OUT,
          const double* __restrict__ Rinv, double* __restrict__ partG, const int32_t* __restrict__ need3,
          T* OUT2) {
  constexpr int RTL = RowTile<T, BP>::RTL1, NS = RowTile<T, BP>::NS1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const RowCtx<T, BP> c = make_ctx<T, BP>(b, ws, ncb);
  bool store_mine = true;  // this thread's column is stored (to OUT)
  if (need3) {
    if (!OUT2) {
      bool any = false;
      for (int32_t g = 0; g < c.gcount; ++g) any = any || need3[c.cg0 + g] != 0;
      if (!any) return;  // uniform over the CTA
    }
    if (c.my_col >= 0) {
      const bool n3 = need3[c.cg0 + c.my_col / b] != 0;
      if (OUT2 && !n3) OUT = OUT2;
      if (!OUT2 && !n3) store_mine = false;
    }
  }
  constexpr int NO = NS == 2 ? 1 : 2;  // output tiles (the overlapped schedule alternates two)
  RowRing<T, BP> ring{reinterpret_cast<T*>(smem_raw), RTL * c.pitch, 1};  // W
  T* sO = ring.at(NS, 0);
  T* sR = sO + NO * RTL * c.pitch;
  GramAcc<T> acc;
  GramPart<T> gp;
  gp.zero();
  const GramRole role = gram_role<T, BP, true>(c.G, threadIdx.x);
  c.load_mat(sR, Rinv, c.cg0, false);
  c.zero(ring.at(0, 0), (NS + NO) * RTL);
  __syncthreads();
  row_pipeline<NS>(
      N, RTL,
      [&](int s, int32_t, int64_t r0, int32_t nr) { c.template load<RTL>(ring.at(s, 0), W, r0, nr); },
      [&](int s, int32_t i, int64_t, int32_t) {
        tile_mul<T, BP, false, false>(c, ring.at(s, 0), sR, sO + (i & (NO - 1)) * RTL * c.pitch, RTL, nullptr, nullptr);
      },
      [&](int, int32_t i, int64_t r0, int32_t nr, bool last) {
        const T* o = sO + (i & (NO - 1)) * RTL * c.pitch;
        if (store_mine) c.store(OUT, o, r0, nr);
        if (GRAM) gram_tile<T, BP, true, RTL>(c, role, o, o, i, last, gp, acc);
      });
  if (GRAM)
    gram_store<T, BP, true>(c, role, acc, partG + (size_t)blockIdx.x * ncb * b * b,
                            reinterpret_cast<double*>(smem_raw));
}

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
// ||H Q_j||_F^2 per colour for the breakdown test.  H Q_j = Q_{j-1} B_{j-1}^T + Q_j A_j + W1
// with orthonormal blocks orthogonal to W1 (the residual after the projections), so its
// square norm is ||B_{j-1}||^2 + ||A_j||^2 + trace(W1^T W1) (no B term at the first step).
__global__ void k_hnorm(int32_t ncb, int32_t b, int32_t cb0, int32_t j, const double* __restrict__ Araw,
                        const double* __restrict__ Bprev, const double* __restrict__ G, double* __restrict__ hq2) {
  const int32_t lc = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (lc >= ncb) return;
  const int32_t bb = b * b;
  const double* a = Araw + (size_t)lc * bb;
  const double* bp = Bprev + (size_t)(cb0 + lc) * bb;
  const double* g = G + (size_t)lc * bb;
  double s = 0.0;
  for (int32_t e = lane; e < bb; e += 32) {
    s += a[e] * a[e];
    if (j > 0) s += bp[e] * bp[e];
  }
  if (lane < b) s += g[lane * b + lane];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) hq2[lc] = s;
}

// need3 (optional, one flag per colour of the pass): MODE 1 sets a colour's flag when the Gram
// of its W R0^-1 is not within kQr2Dev of the identity (max entry), clears it otherwise; MODE 2
// with the flag clear takes R2 = I, so that B_j = R1 R0 (that colour's third CholeskyQR pass is
// then skipped: its second pass has written Q_{j+1}).  Each colour decides on its own Gram, so
// its result does not depend on the other colours of the pass.
constexpr double kQr2Dev = 1e-2;
template <int MODE>
__global__ void k_chol(int32_t ncb, int32_t b, int32_t cb0, int32_t m, int32_t j, const double* __restrict__ G,
                       const double* __restrict__ hq2, double tau, double shift_rel, double* __restrict__ R,
                       double* __restrict__ Rinv, double* __restrict__ Rprod, double* __restrict__ Bblk,
                       int32_t* __restrict__ done, int32_t* __restrict__ nblk, int32_t* __restrict__ need3) {
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
  const bool two_pass = MODE == 2 && need3 && need3[lc] == 0;
  if (MODE == 1 && need3) {
    double dev = broken ? 1.0 : 0.0;
    if (lane < b && !broken)
      for (int32_t i = 0; i < b; ++i) dev = fmax(dev, fabs(g[i * b + lane] - (i == lane ? 1.0 : 0.0)));
    for (int o = 16; o > 0; o >>= 1) dev = fmax(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    if (lane == 0) need3[lc] = dev <= kQr2Dev ? 0 : 1;
  }
  if (two_pass) {
    if (lane < b)
      for (int32_t i = 0; i < b; ++i) r[i][lane] = i == lane ? 1.0 : 0.0;
  } else if (!broken) {
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

// M[lc] = I_b for the colours of the batch
__global__ void k_eye(int32_t ncb, int32_t b, double* __restrict__ M) {
  const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncb * b * b) return;
  const int32_t e = t % (b * b);
  M[t] = (e / b == e % b) ? 1.0 : 0.0;
}

// hq2[lc] = trace of the Gram G[lc] = ||W_c||_F^2 (breakdown scale of a start block)
__global__ void k_gtrace(int32_t ncb, int32_t b, const double* __restrict__ G, double* __restrict__ hq2) {
  const int32_t lc = blockIdx.x * blockDim.x + threadIdx.x;
  if (lc >= ncb) return;
  double s = 0.0;
  for (int32_t k = 0; k < b; ++k) s += G[((size_t)lc * b + k) * b + k];
  hq2[lc] = s;
}

// Vc[cb0 + lc][j b + k][l] = P[lc][k][l]
__global__ void k_store_v(int32_t ncb, int32_t b, int32_t cb0, int32_t nmax, int32_t j, const double* __restrict__ P,
                          double* __restrict__ Vc) {
  const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncb * b * b) return;
  const int32_t lc = t / (b * b), e = t % (b * b), k = e / b, l = e % b;
  Vc[((size_t)(cb0 + lc) * nmax + (size_t)j * b + k) * b + l] = P[t];
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

// Sampled rows of Q_j: Qs[p][j][a][k] = Q_j[(I_p, a), c_p block, k] for the batch's pairs, one
// warp per pair (its b x b block is one contiguous run of Qs)
template <typename T>
__global__ void k_scatter(int64_t p_begin, int64_t p_end, int32_t b, int32_t ws, int32_t cb0, int32_t m, int32_t j,
                          const int32_t* __restrict__ pair_I, const int32_t* __restrict__ pair_c,
                          const T* __restrict__ Q, T* __restrict__ Qs, int32_t ibase) {
  const int64_t p = p_begin + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (p >= p_end) return;
  const int32_t bb = b * b;
  const int32_t I = pair_I[p] - ibase, c = pair_c[p] - cb0;
  const T* q = Q + (size_t)I * b * ws + (size_t)c * b;
  T* o = Qs + ((size_t)p * m + j) * bb;
  for (int32_t e = lane; e < bb; e += 32) {
    const int32_t a = e / b, k = e - a * b;
    o[e] = q[(size_t)a * ws + k];
  }
}

// Second pass, every row: Y[r][c b + k] += sum_l Q_j[r][lc b + l] Z_c[j b + l][k] for the
// batch's colours (lc = c - cb0), one CTA per row r
template <typename T>
__global__ void k_accum_full(int32_t b, int32_t ws, int32_t ncb, int32_t cb0, int32_t ldz, int32_t j,
                             const int32_t* __restrict__ nblk, const T* __restrict__ Q,
                             const double* __restrict__ Z, T* __restrict__ Y, int32_t ldy) {
  const int64_t r = blockIdx.x;
  const T* q = Q + (size_t)r * ws;
  for (int32_t col = threadIdx.x; col < ncb * b; col += blockDim.x) {
    const int32_t lc = col / b, k = col - lc * b, cg = cb0 + lc;
    if (j >= nblk[cg]) continue;
    const double* z = Z + ((size_t)cg * ldz + (size_t)j * b) * b + k;
    double s = 0.0;
    for (int32_t l = 0; l < b; ++l) s = fma((double)q[(size_t)lc * b + l], z[(size_t)l * b], s);
    T* y = Y + (size_t)r * ldy + (size_t)cg * b + k;
    *y = (T)((double)*y + s);
  }
}

// Second pass: X[p][a][kk] += sum_l Q_j[(I_p, a), c_p block, l] Z_c[j b + l][kk] (FP64)
template <typename T>
__global__ void k_accum_x(int64_t p_begin, int64_t p_end, int32_t b, int32_t ws, int32_t cb0, int32_t ldz,
                          int32_t j, const int32_t* __restrict__ pair_I, const int32_t* __restrict__ pair_c,
                          const int32_t* __restrict__ nblk, const T* __restrict__ Q, const double* __restrict__ Z,
                          double* __restrict__ X, int32_t ibase) {
  const int32_t bb = b * b;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t p = p_begin + t / bb;
  if (p >= p_end) return;
  int32_t e = (int32_t)(t % bb), a = e / b, kk = e % b;
  int32_t I = pair_I[p] - ibase, cg = pair_c[p], c = cg - cb0;
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

template <typename T, int BM, int TC, int NT>
css_status launch_spmm_t(css_ctx* ctx, const LzArgs& a, const T* V, T* W, cudaStream_t st) {
  using C = SpmmCfg<T, BM, TC, NT>;
  auto kern = k_spmm<T, BM, TC, NT>;
  CSS_TRY(smem_optin(ctx, kern, C::smem));
  dim3 grid((unsigned)a.n_brow, (unsigned)css_ceil_div(a.w, C::CT));
  kern<<<grid, C::NT, C::smem, st>>>(a.b, a.row_ptr, a.col_idx, (const T*)a.Hval, V, W, a.ws, a.w,
                                     (const T*)a.Hlo_diag, a.row0);
  CSS_LAUNCHED(ctx);
  return CSS_OK;
}

// launch variants (columns per thread, threads per CTA); every variant sums each output in the
// same order, so the choice changes the speed only, never the result
constexpr int kSpmmVariants = 5;

template <typename T, int BM>
css_status launch_spmm_bm(css_ctx* ctx, const LzArgs& a, const T* V, T* W, int v, cudaStream_t st) {
  constexpr int TCW = (sizeof(T) == 4 && BM < 32) ? 4 : (sizeof(T) == 4 || BM < 32) ? 2 : 1;  // widest
  constexpr int TCN = TCW > 1 ? TCW / 2 : 1;
  if (v == 0) return launch_spmm_t<T, BM, TCW, 128>(ctx, a, V, W, st);
  if (v == 1) return launch_spmm_t<T, BM, TCN, 256>(ctx, a, V, W, st);
  if (v == 2) return launch_spmm_t<T, BM, TCN, 128>(ctx, a, V, W, st);
  if (v == 3) return launch_spmm_t<T, BM, TCW, 64>(ctx, a, V, W, st);  // more, smaller CTAs per SM
  return launch_spmm_t<T, BM, TCW, 96>(ctx, a, V, W, st);
}

template <typename T>
css_status launch_spmm_v(css_ctx* ctx, const LzArgs& a, const T* V, T* W, int v, cudaStream_t st) {
  switch (css_spmm_bm(a.b)) {
    case 8: return launch_spmm_bm<T, 8>(ctx, a, V, W, v, st);
    case 12: return launch_spmm_bm<T, 12>(ctx, a, V, W, v, st);
    case 16: return launch_spmm_bm<T, 16>(ctx, a, V, W, v, st);
    case 24: return launch_spmm_bm<T, 24>(ctx, a, V, W, v, st);
    default: return launch_spmm_bm<T, 32>(ctx, a, V, W, v, st);
  }
}

// W = H V with the variant tuned for this shape: the first time a shape is seen, every variant
// runs once untimed (first-launch costs) and once timed on the call's own data (each writes the
// same W), and the fastest is kept.  Shapes: precision, b, columns in buckets of 256, rows.
// With tune_only the call only makes sure the shape's variant is chosen (tuning it on V and W
// when it is new) and launches nothing else, so that a later pass can be captured in a graph.
template <typename T>
css_status launch_spmm(css_ctx* ctx, const LzArgs& a, const T* V, T* W, cudaStream_t st, bool tune_only = false) {
  bool dup = false;
  if constexpr (sizeof(T) == 4) {
    if (a.use_tc) return tune_only ? CSS_OK : css_hv_tc(ctx, a, V, W, st);
    dup = a.Hdup != nullptr;
  } else {
    dup = a.Hsplit != nullptr;
  }
  // the exact-width kernel (FP32) or the split-FP64 one (css_spmm.cu) when H was prepared for
  // it, else the padded one
  auto run = [&](int v) -> css_status {
    if constexpr (sizeof(T) == 4) {
      if (dup) return css_spmm_dup(ctx, a, V, W, v, st);
    } else {
      if (dup) return css_spmm_split(ctx, a, V, W, v, st);
    }
    return launch_spmm_v<T>(ctx, a, V, W, v, st);
  };
  const int nv = dup ? (sizeof(T) == 4 ? css_spmm_dup_variants() : css_spmm_split_variants()) : kSpmmVariants;
  const uint64_t key = ((uint64_t)sizeof(T) << 60) ^ ((uint64_t)dup << 59) ^ ((uint64_t)a.b << 48) ^
                       ((uint64_t)(a.w / 256) << 24) ^ (uint64_t)(a.n_brow >= (1 << 24) ? (1 << 24) - 1 : a.n_brow);
  if (!dup && ctx->spmm_variant >= 0) return tune_only ? CSS_OK : run(ctx->spmm_variant);
  if (dup && ctx->spmm_dup_variant >= 0) return tune_only ? CSS_OK : run(ctx->spmm_dup_variant);
  for (const auto& kv : ctx->spmm_tune)
    if (kv.first == key) return tune_only ? CSS_OK : run(kv.second);
  css_events ev;
  CSS_CU(ctx, ev.create((size_t)nv + 1));
  css_status rc = CSS_OK;
  for (int v = 0; v < nv && rc == CSS_OK; ++v) rc = run(v);
  if (rc == CSS_OK) CSS_CU(ctx, cudaEventRecord(ev[0], st));
  for (int v = 0; v < nv && rc == CSS_OK; ++v) {
    rc = run(v);
    if (rc == CSS_OK) rc = cudaEventRecord(ev[v + 1], st) == cudaSuccess ? CSS_OK : CSS_ERR_CUDA;
  }
  int best = 0;
  if (rc == CSS_OK && cudaEventSynchronize(ev[nv]) == cudaSuccess) {
    float tbest = 0.0f;
    for (int v = 0; v < nv; ++v) {
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, ev[v], ev[v + 1]);
      if (v == 0 || ms < tbest) {
        tbest = ms;
        best = v;
      }
    }
    ctx->spmm_tune.emplace_back(key, best);
  }
  return rc;
}

template <typename T, int BP>
css_status run_pass_bp(css_ctx* ctx, const LzArgs& a_in, cudaStream_t st) {
  LzArgs a = a_in;
  if (a.use_tc) CSS_TRY(css_hv_tc_schedule(ctx, a, st));
  const int32_t b = a.b, bb = b * b, ncb = a.ncb, m = a.m;
  const int64_t N = (int64_t)a.n_brow * b;
  const int32_t nch = (int32_t)css_ceil_div(N, RCHK);
  const int32_t G = colours_per_cta<T, BP>(b);
  const int32_t ngr = (int32_t)css_ceil_div(ncb, G);
  const bool reorth = (a.flags & CSS_REORTH_LOCAL) != 0;
  T* Qp = (T*)a.Q0;
  T* Qc = (T*)a.Q1;
  T* W = (T*)a.W;
  const size_t vec_bytes = (size_t)N * a.ws * sizeof(T);
  const dim3 rgrid((unsigned)nch, (unsigned)ngr);
  constexpr int RTL3 = RowTile<T, BP>::RTL3, NS3 = RowTile<T, BP>::NS3, RTL1 = RowTile<T, BP>::RTL1, NS1 = RowTile<T, BP>::NS1;
  const size_t pitch_bytes = (size_t)(G * (BP + 4) + 4) * sizeof(T);
  const size_t mat = (size_t)G * ColStride<BP>::MS * sizeof(T);
  const size_t sm_s1 = 3 * NS3 * RTL3 * pitch_bytes + mat;
  const size_t sm_s3 = 3 * NS3 * RTL3 * pitch_bytes + 2 * mat;
  const size_t sm_tri = (NS1 + (NS1 == 2 ? 1 : 2)) * RTL1 * pitch_bytes + mat;
  const int th3 = row_threads<T, BP, RTL3>(b), th1 = row_threads<T, BP, RTL1>(b);
  double* partKq = a.part;
  double* partKp = a.part + (size_t)nch * ncb * bb;
  double* sA = a.small;                          // [2][ncb][bb]: raw, symmetrised
  double* sH = a.small + 2 * (size_t)ncb * bb;   // [ncb]
  double* sG = sH + ncb;                         // [ncb][bb]
  double* sR1 = sG + (size_t)ncb * bb;
  double* sR1i = sR1 + (size_t)ncb * bb;
  double* sR2 = sR1i + (size_t)ncb * bb;
  double* sR2i = sR2 + (size_t)ncb * bb;
  double* sC1 = sR2i + (size_t)ncb * bb;
  double* sKp = sC1 + (size_t)ncb * bb;
  double* sV = sKp + (size_t)ncb * bb;  // Q_j^T u of the running step (the tenth small matrix)
  double* sRi10 = sV + (size_t)ncb * bb;     // R0^-1 R1^-1 (FP32 row passes)
  double* sRi210 = sRi10 + (size_t)ncb * bb;  // R0^-1 R1^-1 R2^-1
  // per colour: "a third CholeskyQR pass is needed" in the running step (after the matrices)
  int32_t* need3 = reinterpret_cast<int32_t*>(sRi210 + (size_t)ncb * bb);
  // FP32, 16 < b <= 24, env CSS_ROWS_STREAM=1: the streaming row passes of css_rows.cu
  constexpr bool kF32 = sizeof(T) == 4;
  const bool rp = kF32 && BP == 24 && css_rowpass_supported(true, b) && ctx->rows_stream;
  const unsigned rblocks_bb = (unsigned)css_ceil_div((int64_t)ncb * bb, 256);
  const int64_t pb = a.pair_off_h[a.cb0], pe = a.pair_off_h[a.cb0 + ncb];
  const unsigned sblocks = (unsigned)css_ceil_div((pe - pb) * bb, 256);
  auto s1 = reorth ? k_s1<T, BP, true> : k_s1<T, BP, false>;
  auto s3 = reorth ? k_s3<T, BP, true> : k_s3<T, BP, false>;
  CSS_TRY(smem_optin(ctx, s1, sm_s1));
  CSS_TRY(smem_optin(ctx, s3, sm_s3));
  CSS_TRY(smem_optin(ctx, k_tri<T, BP, true>, sm_tri));
  CSS_TRY(smem_optin(ctx, k_tri<T, BP, false>, sm_tri));
  if (a.ucol) CSS_TRY(smem_optin(ctx, k_s1<T, BP, false>, sm_s1));
  CSS_CU(ctx, cudaMemsetAsync(Qp, 0, vec_bytes, st));
  CSS_CU(ctx, cudaMemsetAsync(Qc, 0, vec_bytes, st));
  if (a.start) {
    // Q_1 B_0 = start by the shifted CholeskyQR3 of the steps below: the start block is copied
    // into W (times the identity) with its Gram, and B_0 is the product of the three factors
    k_eye<<<rblocks_bb, 256, 0, st>>>(ncb, b, sR1i);
    CSS_LAUNCHED(ctx);
    k_tri<T, BP, true><<<rgrid, th1, sm_tri, st>>>(N, b, a.ws, ncb, (const T*)a.start, W, sR1i,
                                                                     partKq, nullptr, nullptr);
    CSS_LAUNCHED(ctx);
    k_reduce<<<rblocks_bb, 256, 0, st>>>(nch, ncb, bb, partKq, sG);
    CSS_LAUNCHED(ctx);
    k_gtrace<<<(unsigned)css_ceil_div(ncb, 128), 128, 0, st>>>(ncb, b, sG, sH);
    CSS_LAUNCHED(ctx);
    const unsigned gb = (unsigned)css_ceil_div(ncb, 4);
    k_chol<0><<<gb, 128, 0, st>>>(ncb, b, a.cb0, 1, 0, sG, sH, a.tau, a.shift_rel, sR1, sR1i, sC1, a.B0, a.done,
                                  a.nblk, nullptr);
    CSS_LAUNCHED(ctx);
    CSS_CU(ctx, cudaMemcpyAsync(sC1, sR1, sizeof(double) * ncb * bb, cudaMemcpyDeviceToDevice, st));
    k_tri<T, BP, true><<<rgrid, th1, sm_tri, st>>>(N, b, a.ws, ncb, W, W, sR1i, partKq, nullptr, nullptr);
    CSS_LAUNCHED(ctx);
    k_reduce<<<rblocks_bb, 256, 0, st>>>(nch, ncb, bb, partKq, sG);
    CSS_LAUNCHED(ctx);
    k_chol<1><<<gb, 128, 0, st>>>(ncb, b, a.cb0, 1, 0, sG, sH, a.tau, 0.0, sR1, sR1i, sC1, a.B0, a.done, a.nblk,
                                  nullptr);
    CSS_LAUNCHED(ctx);
    k_tri<T, BP, true><<<rgrid, th1, sm_tri, st>>>(N, b, a.ws, ncb, W, W, sR1i, partKq, nullptr, nullptr);
    CSS_LAUNCHED(ctx);
    k_reduce<<<rblocks_bb, 256, 0, st>>>(nch, ncb, bb, partKq, sG);
    CSS_LAUNCHED(ctx);
    k_chol<2><<<gb, 128, 0, st>>>(ncb, b, a.cb0, 1, 0, sG, sH, a.tau, 0.0, sR2, sR2i, sC1, a.B0, a.done, a.nblk,
                                  nullptr);
    CSS_LAUNCHED(ctx);
    k_tri<T, BP, false><<<rgrid, th1, sm_tri, st>>>(N, b, a.ws, ncb, W, Qc, sR2i, nullptr, nullptr, nullptr);
    CSS_LAUNCHED(ctx);
  } else {
    k_init_q1<T><<<(unsigned)css_ceil_div(N, 256), 256, 0, st>>>(a.n_brow, b, a.ws, a.cb0, ncb, a.colour, a.sign,
                                                                  a.inv_sqrt_cnt, Qc);
    CSS_LAUNCHED(ctx);
  }
  // Vc[c][j] = Q_j^T u (the u block is only read: the first-step form of the three-term kernel)
  auto project_u = [&](const T* Qj, int32_t j) -> css_status {
    if (!a.ucol) return CSS_OK;
    k_s1<T, BP, false><<<rgrid, RW, sm_s1, st>>>(N, b, a.ws, ncb, a.cb0, nullptr, Qj, (T*)a.ucol, nullptr, 1,
                                                  partKq, nullptr);
    CSS_LAUNCHED(ctx);
    k_reduce<<<rblocks_bb, 256, 0, st>>>(nch, ncb, bb, partKq, sV);
    CSS_LAUNCHED(ctx);
    k_store_v<<<rblocks_bb, 256, 0, st>>>(ncb, b, a.cb0, m * b, j, sV, a.Vc);
    CSS_LAUNCHED(ctx);
    return CSS_OK;
  };
  auto sampled = [&](const T* Qj, int32_t j) -> css_status {
    if (a.mode == 2 && a.Yfull) {
      k_accum_full<T><<<(unsigned)((int64_t)a.n_brow * b), 128, 0, st>>>(b, a.ws, a.ncb, a.cb0, a.ldz, j, a.nblk,
                                                                         Qj, a.Z, (T*)a.Yfull, a.ldy);
      CSS_LAUNCHED(ctx);
    }
    if (pe <= pb) return CSS_OK;
    if (a.mode == 1) {
      k_scatter<T><<<(unsigned)css_ceil_div((pe - pb) * 32, 256), 256, 0, st>>>(pb, pe, b, a.ws, a.cb0, m, j,
                                                                                a.pair_I, a.pair_c, Qj, (T*)a.Qs,
                                                                                a.row0);
    } else if (a.mode == 2) {
      k_accum_x<T><<<sblocks, 256, 0, st>>>(pb, pe, b, a.ws, a.cb0, a.ldz, j, a.pair_I, a.pair_c, a.nblk, Qj, a.Z,
                                            a.X, a.row0);
    } else {
      return CSS_OK;
    }
    CSS_LAUNCHED(ctx);
    return CSS_OK;
  };
  auto chol = [&](int mode, int32_t j, double* R, double* Ri, double shift, int32_t* n3) -> css_status {
    const unsigned gb = (unsigned)css_ceil_div(ncb, 4);
    if (mode == 0)
      k_chol<0><<<gb, 128, 0, st>>>(ncb, b, a.cb0, m, j, sG, sH, a.tau, shift, R, Ri, sC1, a.Bblk, a.done, a.nblk,
                                    n3);
    else if (mode == 1)
      k_chol<1><<<gb, 128, 0, st>>>(ncb, b, a.cb0, m, j, sG, sH, a.tau, 0.0, R, Ri, sC1, a.Bblk, a.done, a.nblk, n3);
    else
      k_chol<2><<<gb, 128, 0, st>>>(ncb, b, a.cb0, m, j, sG, sH, a.tau, 0.0, R, Ri, sC1, a.Bblk, a.done, a.nblk, n3);
    CSS_LAUNCHED(ctx);
    return CSS_OK;
  };
  CSS_TRY(sampled(Qc, 0));
  CSS_TRY(project_u(Qc, 0));
  // timing events: inside a stream capture they are recorded as external event nodes of the graph
  // (real records each time the graph runs); that flag is refused outside a capture
  unsigned ev_flags = cudaEventRecordDefault;
  if (a.ev_spmm) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CSS_CU(ctx, cudaStreamIsCapturing(st, &cap));
    if (cap == cudaStreamCaptureStatusActive) ev_flags = cudaEventRecordExternal;
  }
  for (int32_t j = 0; j < m; ++j) {
    if (a.ev_spmm) CSS_CU(ctx, cudaEventRecordWithFlags(a.ev_spmm[2 * j], st, ev_flags));
    CSS_TRY(launch_spmm<T>(ctx, a, Qc, W, st));
    if (a.ev_spmm) CSS_CU(ctx, cudaEventRecordWithFlags(a.ev_spmm[2 * j + 1], st, ev_flags));
    if (rp) {
      const int first = j == 0 ? 1 : 0, ro = reorth ? 1 : 0;
      const float *q = (const float*)Qc, *qp = (const float*)Qp;
      float* wv = (float*)W;
      // Kq = Q_j^T W0, Kp = Q_{j-1}^T W0 with W0 = W - Q_{j-1} B_{j-1}^T
      CSS_TRY(css_rowpass(ctx, 0, N, b, a.ws, ncb, a.cb0, first, ro, q, qp, wv, nullptr, a.Bblk_prev, nullptr, nullptr,
                          partKq, partKp, st));
      k_reduce<<<rblocks_bb, 256, 0, st>>>(nch, ncb, bb, partKq, sA);
      CSS_LAUNCHED(ctx);
      if (reorth && !first) {
        k_reduce<<<rblocks_bb, 256, 0, st>>>(nch, ncb, bb, partKp, sKp);
        CSS_LAUNCHED(ctx);
      }
      k_store_A<<<rblocks_bb, 256, 0, st>>>(ncb, b, a.cb0, m, j, sA, a.Ablk);
      CSS_LAUNCHED(ctx);
      if (j + 1 == m) break;
      // W1 = W - Q_j Kq - Q_{j-1} (B_{j-1}^T + Kp) over W, and its Gram
      CSS_TRY(css_rowpass(ctx, 1, N, b, a.ws, ncb, a.cb0, first, ro, q, qp, wv, wv, sA, a.Bblk_prev,
                          (reorth && !first) ? sKp : nullptr, partKq, nullptr, st));
      k_reduce<<<rblocks_bb, 256, 0, st>>>(nch, ncb, bb, partKq, sG);
      CSS_LAUNCHED(ctx);
      k_hnorm<<<(unsigned)css_ceil_div(ncb, 8), 256, 0, st>>>(ncb, b, a.cb0, j, sA, a.Bblk_prev, sG, sH);
      CSS_LAUNCHED(ctx);
      // shifted CholeskyQR3 on W1 without storing the intermediates: the Grams of W1 R0^-1 and
      // W1 R0^-1 R1^-1 are taken from W1 itself, and Q_{j+1} = W1 R0^-1 R1^-1 R2^-1
      CSS_TRY(chol(0, j, sR1, sR1i, a.shift_rel, rp ? nullptr : need3));
      CSS_CU(ctx, cudaMemcpyAsync(sC1, sR1, sizeof(double) * ncb * bb, cudaMemcpyDeviceToDevice, st));
      CSS_TRY(css_rowpass(ctx, 2, N, b, a.ws, ncb, a.cb0, first, ro, nullptr, nullptr, wv, nullptr, sR1i, nullptr,
                          nullptr, partKq, nullptr, st));
      k_reduce<<<rblocks_bb, 256, 0, st>>>(nch, ncb, bb, partKq, sG);
      CSS_LAUNCHED(ctx);
      CSS_TRY(chol(1, j, sR2, sR2i, 0.0, nullptr));
      CSS_TRY(css_small_mm(ctx, ncb, b, sR1i, sR2i, sRi10, st));
      CSS_TRY(css_rowpass(ctx, 2, N, b, a.ws, ncb, a.cb0, first, ro, nullptr, nullptr, wv, nullptr, sRi10, nullptr,
                          nullptr, partKq, nullptr, st));
      k_reduce<<<rblocks_bb, 256, 0, st>>>(nch, ncb, bb, partKq, sG);
      CSS_LAUNCHED(ctx);
      CSS_TRY(chol(2, j, sR1, sR1i, 0.0, nullptr));
      CSS_TRY(css_small_mm(ctx, ncb, b, sRi10, sR1i, sRi210, st));
      CSS_TRY(css_rowpass(ctx, 3, N, b, a.ws, ncb, a.cb0, first, ro, nullptr, nullptr, wv, (float*)Qp, sRi210, nullptr,
                          nullptr, nullptr, nullptr, st));
      CSS_TRY(sampled(Qp, j + 1));
      CSS_TRY(project_u(Qp, j + 1));
      CSS_CU(ctx, cudaMemcpy2DAsync(a.Bblk_prev + (size_t)a.cb0 * bb, bb * sizeof(double),
                                    a.Bblk + ((size_t)a.cb0 * m + j) * bb, (size_t)m * bb * sizeof(double),
                                    bb * sizeof(double), ncb, cudaMemcpyDeviceToDevice, st));
      T* t = Qp;
      Qp = Qc;
      Qc = t;
      continue;
    }
    // three-term update and the projections onto Q_j (and Q_{j-1})
    s1<<<rgrid, reorth ? 2 * RW : RW, sm_s1, st>>>(N, b, a.ws, ncb, a.cb0, Qp, Qc, W, a.Bblk_prev, j == 0 ? 1 : 0,
                                                   partKq, partKp);
    CSS_LAUNCHED(ctx);
    k_reduce<<<rblocks_bb, 256, 0, st>>>(nch, ncb, bb, partKq, sA);
    CSS_LAUNCHED(ctx);
    if (reorth) {
      k_reduce<<<rblocks_bb, 256, 0, st>>>(nch, ncb, bb, partKp, sKp);
      CSS_LAUNCHED(ctx);
    }
    k_store_A<<<rblocks_bb, 256, 0, st>>>(ncb, b, a.cb0, m, j, sA, a.Ablk);
    CSS_LAUNCHED(ctx);
    if (j + 1 == m) break;
    // W1 = W0 - Q_j Kq (- Q_{j-1} Kp) and its Gram
    s3<<<rgrid, th3, sm_s3, st>>>(N, b, a.ws, ncb, Qc, Qp, W, sA, sKp, partKq);
    CSS_LAUNCHED(ctx);
    // shifted CholeskyQR3 of W: R0 from G + sI, then two plain CholeskyQR passes; the third is
    // skipped (need3 clear) when the second pass's input W R0^-1 already has a Gram within
    // kQr2Dev of the identity for every colour: one CholeskyQR pass of so well-conditioned a
    // block gives orthonormal columns to the working precision, as the third pass would
    k_reduce<<<rblocks_bb, 256, 0, st>>>(nch, ncb, bb, partKq, sG);
    CSS_LAUNCHED(ctx);
    k_hnorm<<<(unsigned)css_ceil_div(ncb, 8), 256, 0, st>>>(ncb, b, a.cb0, j, sA, a.Bblk_prev, sG, sH);
    CSS_LAUNCHED(ctx);
    CSS_TRY(chol(0, j, sR1, sR1i, a.shift_rel, rp ? nullptr : need3));
    CSS_CU(ctx, cudaMemcpyAsync(sC1, sR1, sizeof(double) * ncb * bb, cudaMemcpyDeviceToDevice, st));
    k_tri<T, BP, true><<<rgrid, th1, sm_tri, st>>>(N, b, a.ws, ncb, W, W, sR1i, partKq, nullptr, nullptr);
    CSS_LAUNCHED(ctx);
    k_reduce<<<rblocks_bb, 256, 0, st>>>(nch, ncb, bb, partKq, sG);
    CSS_LAUNCHED(ctx);
    CSS_TRY(chol(1, j, sR1, sR1i, 0.0, need3));
    k_tri<T, BP, true><<<rgrid, th1, sm_tri, st>>>(N, b, a.ws, ncb, W, W, sR1i, partKq, need3, Qp);
    CSS_LAUNCHED(ctx);
    k_reduce<<<rblocks_bb, 256, 0, st>>>(nch, ncb, bb, partKq, sG);
    CSS_LAUNCHED(ctx);
    CSS_TRY(chol(2, j, sR2, sR2i, 0.0, need3));
    // Q_{j+1} = W R2^-1 overwrites Q_{j-1} (done by the second pass when two passes sufficed)
    k_tri<T, BP, false><<<rgrid, th1, sm_tri, st>>>(N, b, a.ws, ncb, W, Qp, sR2i, nullptr, need3, nullptr);
    CSS_LAUNCHED(ctx);
    CSS_TRY(sampled(Qp, j + 1));
    CSS_TRY(project_u(Qp, j + 1));
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

template <typename T>
css_status run_pass(css_ctx* ctx, const LzArgs& a, cudaStream_t st) {
  if (a.b <= 8) return run_pass_bp<T, 8>(ctx, a, st);
  if (a.b <= 16) return run_pass_bp<T, 16>(ctx, a, st);
  if (a.b <= 24) return run_pass_bp<T, 24>(ctx, a, st);
  return run_pass_bp<T, 32>(ctx, a, st);
}

}  // namespace

// Bblk_prev is indexed by global colour; the three-term kernel reads [cb0 + lc]
css_status css_lanczos_tune(css_ctx* ctx, const LzArgs& a, cudaStream_t st) {
  if (a.use_tc) {  // sizes the schedule's workspace before any capture
    LzArgs t = a;
    return css_hv_tc_schedule(ctx, t, st);
  }
  if (a.fp32) return launch_spmm<float>(ctx, a, (const float*)a.Q1, (float*)a.W, st, true);
  return launch_spmm<double>(ctx, a, (const double*)a.Q1, (double*)a.W, st, true);
}

css_status css_lanczos_pass(css_ctx* ctx, const LzArgs& a, cudaStream_t st) {
  if (a.fp32) return run_pass<float>(ctx, a, st);
  return run_pass<double>(ctx, a, st);
}

css_status css_spmm(css_ctx* ctx, const LzArgs& a, const void* V, void* W, cudaStream_t st) {
  if (a.fp32) return launch_spmm<float>(ctx, a, (const float*)V, (float*)W, st);
  return launch_spmm<double>(ctx, a, (const double*)V, (double*)W, st);
}

size_t css_lanczos_part_doubles(int64_t N, int32_t b, int32_t ncb) {
  const int64_t nch = css_ceil_div(N, RCHK);
  return (size_t)nch * ncb * b * b * 2 + (size_t)nch * ncb + 64;
}

// twelve per-colour b x b matrices, the breakdown scales and the colours' CholeskyQR flags
size_t css_lanczos_small_doubles(int32_t b, int32_t ncb) {
  return (size_t)ncb * b * b * 12 + ncb + (ncb + 1) / 2 + 64;
}

int32_t css_spmm_bm(int32_t b) { return b <= 8 ? 8 : b <= 12 ? 12 : b <= 16 ? 16 : b <= 24 ? 24 : 32; }

css_status css_spmm_prepare_as(css_ctx* ctx, const char* tag, bool fp32, int32_t b, int32_t n_brow, int32_t nnzb,
                               const int32_t* row_ptr, const int32_t* col_idx, const double* H, const void** Hpad,
                               const void** Hlo_pad, cudaStream_t st) {
  const int32_t BM = css_spmm_bm(b);
  const int64_t bb = (int64_t)BM * BM;
  constexpr int T = 256;
  char n1[64], n2[64];
  snprintf(n1, sizeof(n1), "%s_pad%d", tag, fp32 ? 32 : 64);
  snprintf(n2, sizeof(n2), "%s_lopad32", tag);
  if (fp32) {
    float *hp, *lp;
    CSS_TRY(css_ws(ctx, n1, (size_t)nnzb * bb * sizeof(float), (void**)&hp));
    CSS_TRY(css_ws(ctx, n2, (size_t)n_brow * bb * sizeof(float), (void**)&lp));
    k_hpad<float, false><<<(unsigned)css_ceil_div((int64_t)nnzb * bb, T), T, 0, st>>>(nnzb, b, BM, H, row_ptr,
                                                                                       col_idx, hp);
    CSS_LAUNCHED(ctx);
    k_hpad<float, true><<<(unsigned)css_ceil_div((int64_t)n_brow * bb, T), T, 0, st>>>(n_brow, b, BM, H, row_ptr,
                                                                                       col_idx, lp);
    CSS_LAUNCHED(ctx);
    *Hpad = hp;
    *Hlo_pad = lp;
  } else {
    double* hp;
    CSS_TRY(css_ws(ctx, n1, (size_t)nnzb * bb * sizeof(double), (void**)&hp));
    k_hpad<double, false><<<(unsigned)css_ceil_div((int64_t)nnzb * bb, T), T, 0, st>>>(nnzb, b, BM, H, row_ptr,
                                                                                        col_idx, hp);
    CSS_LAUNCHED(ctx);
    *Hpad = hp;
    *Hlo_pad = nullptr;
  }
  return CSS_OK;
}

css_status css_probe_block(css_ctx* ctx, bool fp32, int32_t n_brow, int32_t b, int32_t ws, int32_t cb0, int32_t ncb,
                           const int32_t* colour, const int8_t* sign, const double* scale, void* out,
                           cudaStream_t st) {
  const int64_t N = (int64_t)n_brow * b;
  CSS_CU(ctx, cudaMemsetAsync(out, 0, (size_t)N * ws * (fp32 ? sizeof(float) : sizeof(double)), st));
  if (fp32)
    k_init_q1<float><<<(unsigned)css_ceil_div(N, 256), 256, 0, st>>>(n_brow, b, ws, cb0, ncb, colour, sign, scale,
                                                                      (float*)out);
  else
    k_init_q1<double><<<(unsigned)css_ceil_div(N, 256), 256, 0, st>>>(n_brow, b, ws, cb0, ncb, colour, sign, scale,
                                                                       (double*)out);
  CSS_LAUNCHED(ctx);
  return CSS_OK;
}

css_status css_spmm_prepare(css_ctx* ctx, bool fp32, int32_t b, int32_t n_brow, int32_t nnzb,
                            const int32_t* row_ptr, const int32_t* col_idx, const double* H, const void** Hpad,
                            const void** Hlo_pad, cudaStream_t st) {
  const int32_t BM = css_spmm_bm(b);
  const int64_t bb = (int64_t)BM * BM;
  constexpr int T = 256;
  if (fp32) {
    float *hp, *lp;
    CSS_TRY(css_ws(ctx, "h_pad32", (size_t)nnzb * bb * sizeof(float), (void**)&hp));
    CSS_TRY(css_ws(ctx, "h_lopad32", (size_t)n_brow * bb * sizeof(float), (void**)&lp));
    k_hpad<float, false><<<(unsigned)css_ceil_div((int64_t)nnzb * bb, T), T, 0, st>>>(nnzb, b, BM, H, row_ptr,
                                                                                       col_idx, hp);
    CSS_LAUNCHED(ctx);
    k_hpad<float, true><<<(unsigned)css_ceil_div((int64_t)n_brow * bb, T), T, 0, st>>>(n_brow, b, BM, H, row_ptr,
                                                                                       col_idx, lp);
    CSS_LAUNCHED(ctx);
    *Hpad = hp;
    *Hlo_pad = lp;
  } else {
    double* hp;
    CSS_TRY(css_ws(ctx, "h_pad64", (size_t)nnzb * bb * sizeof(double), (void**)&hp));
    k_hpad<double, false><<<(unsigned)css_ceil_div((int64_t)nnzb * bb, T), T, 0, st>>>(nnzb, b, BM, H, row_ptr,
                                                                                        col_idx, hp);
    CSS_LAUNCHED(ctx);
    *Hpad = hp;
    *Hlo_pad = nullptr;
  }
  return CSS_OK;
}
