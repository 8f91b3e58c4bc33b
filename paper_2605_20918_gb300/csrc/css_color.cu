// Colour graph (cell list, exact int64 fixed-point distances), Jones-Plassmann colouring and
// CSS probe signs.  Paper: CSS construction paragraph after Eq. 2 (greedy multicolouring,
// Welsh-Powell order) and Fig. 1(b,c).
//
// Jones-Plassmann with the priority (degree desc, SplitMix64(seed, id) desc, id asc) colours a
// vertex in the first round in which all of its higher-priority neighbours are coloured, and
// gives it the smallest colour none of them uses.  That is exactly the sequential greedy
// colouring in priority order, so the result is bit-identical to it.
#include "css_internal.cuh"

namespace {

constexpr int64_t kFix = 1048576;  // 2^20 per Angstrom

struct __align__(32) q4 {
  long long x, y, z, w;
};

__device__ __forceinline__ int64_t min_image(int64_t d, int64_t Lq) {
  int64_t r = d % Lq;
  if (r > Lq / 2) r -= Lq;
  if (r < -(Lq / 2)) r += Lq;
  return r;
}

__device__ __forceinline__ bool higher(int32_t du, uint64_t ku, int32_t u, int32_t dv, uint64_t kv, int32_t v) {
  if (du != dv) return du > dv;
  if (ku != kv) return ku > kv;
  return u < v;
}

__global__ void k_quantise(int32_t n, const double* __restrict__ xyz, int64_t Lq, int32_t nc, q4* __restrict__ q,
                           int32_t* __restrict__ cell) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t a = __double2ll_rn(xyz[3 * (int64_t)i] * (double)kFix);
  int64_t b = __double2ll_rn(xyz[3 * (int64_t)i + 1] * (double)kFix);
  int64_t c = __double2ll_rn(xyz[3 * (int64_t)i + 2] * (double)kFix);
  q[i] = q4{a, b, c, 0};
  if (nc >= 3) {
    int64_t w[3] = {a % Lq, b % Lq, c % Lq};
    int32_t ci[3];
    for (int d = 0; d < 3; ++d) {
      if (w[d] < 0) w[d] += Lq;
      int64_t t = (w[d] * nc) / Lq;
      ci[d] = (int32_t)(t >= nc ? nc - 1 : t);
    }
    cell[i] = (ci[0] * nc + ci[1]) * nc + ci[2];
  } else {
    cell[i] = 0;
  }
}

__global__ void k_cell_count(int32_t n, const int32_t* __restrict__ cell, int32_t* __restrict__ cnt) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&cnt[cell[i]], 1);
}

__global__ void k_cell_fill(int32_t n, const int32_t* __restrict__ cell, const int32_t* __restrict__ start,
                            int32_t* __restrict__ fillpos, int32_t* __restrict__ members) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    int32_t c = cell[i];
    int32_t p = atomicAdd(&fillpos[c], 1);
    members[start[c] + p] = i;
  }
}

// insertion-sort each cell's members by id (the fill order above is arbitrary)
__global__ void k_cell_sort(int32_t ncells, const int32_t* __restrict__ start, int32_t* __restrict__ members) {
  int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  int32_t s = start[c], e = start[c + 1];
  for (int32_t i = s + 1; i < e; ++i) {
    int32_t v = members[i];
    int32_t j = i - 1;
    while (j >= s && members[j] > v) {
      members[j + 1] = members[j];
      --j;
    }
    members[j + 1] = v;
  }
}

// pass 0: count neighbours, pass 1: write them.  Candidates come from the 27 cells around
// the molecule (or from all molecules when the box holds fewer than 3 cells per edge).
template <int PASS>
__global__ void k_neighbours(int32_t n, const q4* __restrict__ q, const int32_t* __restrict__ cell, int32_t nc,
                             const int32_t* __restrict__ cstart, const int32_t* __restrict__ members, int64_t Lq,
                             int64_t R2, int32_t* __restrict__ deg, const int32_t* __restrict__ adj_ptr,
                             int32_t* __restrict__ adj) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  q4 qi = q[i];
  int32_t count = 0;
  int32_t out = PASS ? adj_ptr[i] : 0;
  auto test = [&](int32_t j) {
    if (j == i) return;
    q4 qj = q[j];
    int64_t dx = min_image(qi.x - qj.x, Lq), dy = min_image(qi.y - qj.y, Lq), dz = min_image(qi.z - qj.z, Lq);
    if (dx * dx + dy * dy + dz * dz < R2) {
      if (PASS) adj[out + count] = j;
      ++count;
    }
  };
  if (nc < 3) {
    for (int32_t j = 0; j < n; ++j) test(j);
  } else {
    int32_t c = cell[i];
    int32_t cx = c / (nc * nc), cy = (c / nc) % nc, cz = c % nc;
    for (int dx = -1; dx <= 1; ++dx)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dz = -1; dz <= 1; ++dz) {
          int32_t x = (cx + dx + nc) % nc, y = (cy + dy + nc) % nc, z = (cz + dz + nc) % nc;
          int32_t cc = (x * nc + y) * nc + z;
          for (int32_t k = cstart[cc]; k < cstart[cc + 1]; ++k) test(members[k]);
        }
  }
  if (!PASS) deg[i] = count;
}

// ---------------------------------------------------------------- exclusive scan
__global__ void k_scan_block(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t n,
                             int32_t* __restrict__ block_sums) {
  __shared__ int32_t s[1024];
  int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
  int32_t v = i < n ? in[i] : 0;
  s[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    int32_t t = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = s[threadIdx.x] - v;
  if (threadIdx.x == 1023 && block_sums) block_sums[blockIdx.x] = s[1023];
}

__global__ void k_scan_add(int32_t* __restrict__ out, int64_t n, const int32_t* __restrict__ offs) {
  int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
  if (i < n) out[i] += offs[blockIdx.x];
}

}  // namespace

// exclusive scan of n int32 values into out[0..n) and out[n] = total (out has n+1 slots)
css_status css_scan_i32(css_ctx* ctx, const int32_t* in, int32_t* out, int64_t n, cudaStream_t st, int depth = 0) {
  if (n <= 0) {
    CSS_CU(ctx, cudaMemsetAsync(out, 0, sizeof(int32_t), st));
    return CSS_OK;
  }
  int64_t nb = css_ceil_div(n, 1024);
  if (nb == 1) {  // one block: its total is the grand total
    k_scan_block<<<1, 1024, 0, st>>>(in, out, n, out + n);
    CSS_LAUNCHED(ctx);
    return CSS_OK;
  }
  char name[32];
  snprintf(name, sizeof(name), "scan_sums_%d", depth);
  int32_t* sums = nullptr;
  CSS_TRY(css_ws(ctx, name, sizeof(int32_t) * (nb + 1), (void**)&sums));
  k_scan_block<<<(unsigned)nb, 1024, 0, st>>>(in, out, n, sums);
  CSS_LAUNCHED(ctx);
  char name2[32];
  snprintf(name2, sizeof(name2), "scan_offs_%d", depth);
  int32_t* offs = nullptr;
  CSS_TRY(css_ws(ctx, name2, sizeof(int32_t) * (nb + 1), (void**)&offs));
  CSS_TRY(css_scan_i32(ctx, sums, offs, nb, st, depth + 1));
  k_scan_add<<<(unsigned)nb, 1024, 0, st>>>(out, n, offs);
  CSS_LAUNCHED(ctx);
  // total = offs[nb]
  CSS_CU(ctx, cudaMemcpyAsync(out + n, offs + nb, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  return CSS_OK;
}

namespace {

// ---------------------------------------------------------------- Jones-Plassmann
__global__ void k_jp_init(int32_t n, const int32_t* __restrict__ adj_ptr, uint64_t seed, int32_t* __restrict__ deg,
                          uint64_t* __restrict__ key, int32_t* __restrict__ colour) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  deg[i] = adj_ptr[i + 1] - adj_ptr[i];
  key[i] = css_splitmix64(seed, (uint64_t)i);
  colour[i] = -1;
}

// One Jones-Plassmann round, one warp per uncoloured vertex v (lanes walk v's neighbours): v is
// ready when every higher-priority neighbour is coloured (a colour, once set, never changes);
// then it takes the smallest colour none of them uses, searched 256 colours at a time with the
// lanes' bit masks OR-reduced over the warp.  Vertices not ready count into *remaining.
__global__ void k_jp_round(int32_t n, const int32_t* __restrict__ adj_ptr, const int32_t* __restrict__ adj,
                           const int32_t* __restrict__ deg, const uint64_t* __restrict__ key, int32_t* colour,
                           int32_t* __restrict__ remaining) {
  const int32_t v = (int32_t)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (v >= n) return;
  if (__ldcg(&colour[v]) >= 0) return;  // whole warp
  const int32_t dv = deg[v];
  const uint64_t kv = key[v];
  const int32_t s = adj_ptr[v], e = adj_ptr[v + 1];
  bool blocked = false;
  for (int32_t k = s + lane; k < e; k += 32) {
    const int32_t u = adj[k];
    if (higher(deg[u], key[u], u, dv, kv, v) && __ldcg(&colour[u]) < 0) blocked = true;
  }
  if (__any_sync(0xffffffffu, blocked)) {
    if (lane == 0) atomicAdd(remaining, 1);
    return;
  }
  for (int32_t base = 0;; base += 256) {
    uint64_t w[4] = {0, 0, 0, 0};
    for (int32_t k = s + lane; k < e; k += 32) {
      const int32_t u = adj[k];
      if (!higher(deg[u], key[u], u, dv, kv, v)) continue;
      const int32_t c = __ldcg(&colour[u]) - base;
      if (c < 0 || c >= 256) continue;
      w[c >> 6] |= 1ull << (c & 63);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      for (int o = 16; o > 0; o >>= 1) w[q] |= __shfl_xor_sync(0xffffffffu, w[q], o);
    int32_t off = -1;
    if (~w[0]) off = __ffsll((long long)~w[0]) - 1;
    else if (~w[1]) off = 64 + __ffsll((long long)~w[1]) - 1;
    else if (~w[2]) off = 128 + __ffsll((long long)~w[2]) - 1;
    else if (~w[3]) off = 192 + __ffsll((long long)~w[3]) - 1;
    if (off >= 0) {
      if (lane == 0) colour[v] = base + off;
      return;
    }
  }
}

// An explicit graph must have adj_ptr[0] = 0, non-decreasing adj_ptr and every neighbour in
// [0, n): vertex i checks its own row and sets *bad otherwise (its entries are then not read)
__global__ void k_graph_check(int32_t n, const int32_t* __restrict__ adj_ptr, const int32_t* __restrict__ adj,
                              int32_t* __restrict__ bad) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t s = adj_ptr[i], e = adj_ptr[i + 1];
  if ((i == 0 && s != 0) || e < s) {
    atomicOr(bad, 1);
    return;
  }
  for (int32_t k = s; k < e; ++k) {
    const int32_t u = adj[k];
    if (u < 0 || u >= n) {
      atomicOr(bad, 1);
      return;
    }
  }
}

__global__ void k_max_colour(int32_t n, const int32_t* __restrict__ colour, int32_t* __restrict__ maxc) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  int32_t c = i < n ? colour[i] : -1;
  for (int o = 16; o > 0; o >>= 1) c = max(c, __shfl_xor_sync(0xffffffffu, c, o));
  if ((threadIdx.x & 31) == 0) atomicMax(maxc, c);
}

__global__ void k_probe_signs(int64_t count, uint64_t seed, int ones, int8_t* __restrict__ sign) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  sign[i] = ones ? (int8_t)1 : ((css_splitmix64(seed, (uint64_t)i) & 1ull) ? (int8_t)-1 : (int8_t)1);
}

// Molecule centres in fixed point, binned into a periodic grid of cells at least r_col wide
// (about one molecule per cell; any coarser grid is also correct), members of each cell
// sorted by id.  nc = 1 (one cell) when the box holds fewer than 3 cells per edge.
struct CellList {
  q4* q;
  int32_t *cell, *cstart, *members;
  int32_t nc;
  int64_t Lq, R2;
};

css_status build_cells(css_ctx* ctx, int32_t n, const double* xyz, double box, double r_col, CellList* cl,
                       cudaStream_t st) {
  const int T = 256;
  const unsigned nbk = (unsigned)css_ceil_div(n, T);
  const int64_t Lq = llrint(box * (double)kFix);
  const int64_t Rq = llrint(r_col * (double)kFix);
  int64_t nc64 = Rq > 0 ? Lq / Rq : 1024;
  int64_t nc_cap = (int64_t)cbrt((double)n) + 1;
  if (nc64 > nc_cap) nc64 = nc_cap;
  if (nc64 > 1024) nc64 = 1024;
  const int32_t nc = nc64 < 3 ? 1 : (int32_t)nc64;
  const int32_t ncells = nc >= 3 ? nc * nc * nc : 1;
  int32_t *ccnt, *cfill;
  CSS_TRY(css_ws(ctx, "col_q", sizeof(q4) * n, (void**)&cl->q));
  CSS_TRY(css_ws(ctx, "col_cell", sizeof(int32_t) * n, (void**)&cl->cell));
  CSS_TRY(css_ws(ctx, "col_ccnt", sizeof(int32_t) * (ncells + 1), (void**)&ccnt));
  CSS_TRY(css_ws(ctx, "col_cstart", sizeof(int32_t) * (ncells + 1), (void**)&cl->cstart));
  CSS_TRY(css_ws(ctx, "col_cfill", sizeof(int32_t) * (ncells + 1), (void**)&cfill));
  CSS_TRY(css_ws(ctx, "col_members", sizeof(int32_t) * n, (void**)&cl->members));
  k_quantise<<<nbk, T, 0, st>>>(n, xyz, Lq, nc, cl->q, cl->cell);
  CSS_LAUNCHED(ctx);
  CSS_CU(ctx, cudaMemsetAsync(ccnt, 0, sizeof(int32_t) * (ncells + 1), st));
  CSS_CU(ctx, cudaMemsetAsync(cfill, 0, sizeof(int32_t) * (ncells + 1), st));
  k_cell_count<<<nbk, T, 0, st>>>(n, cl->cell, ccnt);
  CSS_LAUNCHED(ctx);
  CSS_TRY(css_scan_i32(ctx, ccnt, cl->cstart, ncells, st));
  k_cell_fill<<<nbk, T, 0, st>>>(n, cl->cell, cl->cstart, cfill, cl->members);
  CSS_LAUNCHED(ctx);
  k_cell_sort<<<(unsigned)css_ceil_div(ncells, T), T, 0, st>>>(ncells, cl->cstart, cl->members);
  CSS_LAUNCHED(ctx);
  cl->nc = nc;
  cl->Lq = Lq;
  cl->R2 = Rq * Rq;
  return CSS_OK;
}

// Same-coloured pairs {i, j}, i < j, closer than r_col: thread i walks the 27 cells around
// molecule i (or all molecules when there is one cell).  Colours outside [0, n_colours) set
// *bad.  Per-warp sums are added into *count.
__global__ void k_conflicts(int32_t n, const q4* __restrict__ q, const int32_t* __restrict__ cell, int32_t nc,
                            const int32_t* __restrict__ cstart, const int32_t* __restrict__ members, int64_t Lq,
                            int64_t R2, const int32_t* __restrict__ colour, int32_t n_colours,
                            unsigned long long* __restrict__ count, int32_t* __restrict__ bad) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long k = 0;
  if (i < n) {
    const int32_t ci = colour[i];
    if (ci < 0 || ci >= n_colours) atomicOr(bad, 1);
    const q4 qi = q[i];
    auto test = [&](int32_t j) {
      if (j <= i || colour[j] != ci) return;
      const q4 qj = q[j];
      const int64_t dx = min_image(qi.x - qj.x, Lq), dy = min_image(qi.y - qj.y, Lq),
                    dz = min_image(qi.z - qj.z, Lq);
      if (dx * dx + dy * dy + dz * dz < R2) ++k;
    };
    if (nc < 3) {
      for (int32_t j = i + 1; j < n; ++j) test(j);
    } else {
      const int32_t c = cell[i];
      const int32_t cx = c / (nc * nc), cy = (c / nc) % nc, cz = c % nc;
      for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dz = -1; dz <= 1; ++dz) {
            const int32_t x = (cx + dx + nc) % nc, y = (cy + dy + nc) % nc, z = (cz + dz + nc) % nc;
            const int32_t cc = (x * nc + y) * nc + z;
            for (int32_t p = cstart[cc]; p < cstart[cc + 1]; ++p) test(members[p]);
          }
    }
  }
  for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
  if ((threadIdx.x & 31) == 0 && k) atomicAdd(count, k);
}

// conflicts of a colouring on a geometry (blocking); *bad = 1 when a colour is out of range
css_status count_conflicts(css_ctx* ctx, const css_geom* geom, double r_col, const int32_t* colour,
                           int32_t n_colours, int64_t* count, int32_t* bad, cudaStream_t st) {
  const int32_t n = geom->n_mol;
  CellList cl;
  CSS_TRY(build_cells(ctx, n, geom->xyz, geom->box, r_col, &cl, st));
  unsigned long long* dcount;
  int32_t* dbad;
  CSS_TRY(css_ws(ctx, "chk_count", 2 * sizeof(unsigned long long), (void**)&dcount));
  dbad = (int32_t*)(dcount + 1);
  CSS_CU(ctx, cudaMemsetAsync(dcount, 0, 2 * sizeof(unsigned long long), st));
  k_conflicts<<<(unsigned)css_ceil_div(n, 256), 256, 0, st>>>(n, cl.q, cl.cell, cl.nc, cl.cstart, cl.members, cl.Lq,
                                                               cl.R2, colour, n_colours, dcount, dbad);
  CSS_LAUNCHED(ctx);
  unsigned long long* h;
  CSS_TRY(css_pinned(ctx, 64, (void**)&h));
  CSS_CU(ctx, cudaMemcpyAsync(h, dcount, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  CSS_CU(ctx, cudaStreamSynchronize(st));
  *count = (int64_t)h[0];
  *bad = *(const int32_t*)(h + 1) != 0 ? 1 : 0;
  return CSS_OK;
}

css_status check_geom(css_ctx* ctx, const css_geom* geom, double r_col, const char* what) {
  if (geom->n_mol < 1 || !(geom->box > 0.0) || geom->box > 1000.0 || !(r_col >= 0.0) || r_col > 1000.0)
    return css_set_arg_error(ctx, what);
  return CSS_OK;
}

}  // namespace

// Colour either a geometry (xyz != nullptr) or an explicit CSR graph.
css_status css_color_impl(css_ctx* ctx, int32_t n, const double* xyz, double box, double r_col, uint64_t seed,
                          const int32_t* adj_ptr_in, const int32_t* adj_in, int32_t* colour, int32_t* n_colours,
                          cudaStream_t st) {
  const int T = 256;
  const unsigned nbk = (unsigned)css_ceil_div(n, T);
  const int32_t* adj_ptr = adj_ptr_in;
  const int32_t* adj = adj_in;
  int32_t* hbuf = nullptr;
  CSS_TRY(css_pinned(ctx, 64, (void**)&hbuf));
  if (xyz) {
    CellList cl;
    CSS_TRY(build_cells(ctx, n, xyz, box, r_col, &cl, st));
    int32_t *deg, *ptr;
    CSS_TRY(css_ws(ctx, "col_deg", sizeof(int32_t) * (n + 1), (void**)&deg));
    CSS_TRY(css_ws(ctx, "col_adjptr", sizeof(int32_t) * (n + 1), (void**)&ptr));
    k_neighbours<0><<<nbk, T, 0, st>>>(n, cl.q, cl.cell, cl.nc, cl.cstart, cl.members, cl.Lq, cl.R2, deg, nullptr,
                                       nullptr);
    CSS_LAUNCHED(ctx);
    CSS_TRY(css_scan_i32(ctx, deg, ptr, n, st));
    CSS_CU(ctx, cudaMemcpyAsync(hbuf, ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CSS_CU(ctx, cudaStreamSynchronize(st));
    int64_t nadj = hbuf[0];
    int32_t* a;
    CSS_TRY(css_ws(ctx, "col_adj", sizeof(int32_t) * (nadj > 0 ? nadj : 1), (void**)&a));
    k_neighbours<1><<<nbk, T, 0, st>>>(n, cl.q, cl.cell, cl.nc, cl.cstart, cl.members, cl.Lq, cl.R2, nullptr, ptr,
                                       a);
    CSS_LAUNCHED(ctx);
    adj_ptr = ptr;
    adj = a;
  }
  int32_t* deg;
  uint64_t* key;
  int32_t* counters;
  CSS_TRY(css_ws(ctx, "jp_deg", sizeof(int32_t) * n, (void**)&deg));
  CSS_TRY(css_ws(ctx, "jp_key", sizeof(uint64_t) * n, (void**)&key));
  CSS_TRY(css_ws(ctx, "jp_counters", sizeof(int32_t) * 64, (void**)&counters));
  if (!xyz) {  // a caller's graph: refuse a malformed pattern before any round reads through it
    CSS_CU(ctx, cudaMemsetAsync(counters + 40, 0, sizeof(int32_t), st));
    k_graph_check<<<nbk, T, 0, st>>>(n, adj_ptr, adj, counters + 40);
    CSS_LAUNCHED(ctx);
    CSS_CU(ctx, cudaMemcpyAsync(hbuf, counters + 40, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CSS_CU(ctx, cudaStreamSynchronize(st));
    if (hbuf[0] != 0)
      return css_set_arg_error(ctx, "css_color_graph: adj_ptr not non-decreasing from 0 or a neighbour outside [0, n)");
  }
  k_jp_init<<<nbk, T, 0, st>>>(n, adj_ptr, seed, deg, key, colour);
  CSS_LAUNCHED(ctx);
  // rounds, checked in groups; every round colours at least the highest-priority uncoloured
  // vertex, so n rounds always suffice
  const int group = 8;
  int64_t rounds = 0;
  for (;;) {
    CSS_CU(ctx, cudaMemsetAsync(counters, 0, sizeof(int32_t) * group, st));
    for (int r = 0; r < group; ++r) {
      k_jp_round<<<(unsigned)css_ceil_div((int64_t)n * 32, T), T, 0, st>>>(n, adj_ptr, adj, deg, key, colour,
                                                                           counters + r);
      CSS_LAUNCHED(ctx);
    }
    rounds += group;
    CSS_CU(ctx, cudaMemcpyAsync(hbuf, counters + group - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CSS_CU(ctx, cudaStreamSynchronize(st));
    if (hbuf[0] == 0) break;
    if (rounds > (int64_t)n + group) return css_set_arg_error(ctx, "colouring did not finish (inconsistent graph)");
  }
  CSS_CU(ctx, cudaMemsetAsync(counters + 32, 0xff, sizeof(int32_t), st));
  k_max_colour<<<nbk, T, 0, st>>>(n, colour, counters + 32);
  CSS_LAUNCHED(ctx);
  CSS_CU(ctx, cudaMemcpyAsync(hbuf, counters + 32, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CSS_CU(ctx, cudaStreamSynchronize(st));
  *n_colours = hbuf[0] + 1;
  return CSS_OK;
}

extern "C" {

css_status css_color(css_ctx* ctx, const css_geom* geom, double r_col, uint64_t seed, int32_t* colour,
                     int32_t* n_colours, void* stream) {
  if (!ctx || !geom || !geom->xyz || !colour || !n_colours) return css_set_arg_error(ctx, "css_color: null pointer");
  if (geom->n_mol < 1 || !(geom->box > 0.0) || geom->box > 1000.0 || !(r_col >= 0.0) || r_col > 1000.0)
    return css_set_arg_error(ctx, "css_color: n_mol < 1, box not in (0, 1000] or r_col not in [0, 1000]");
  CSS_CU(ctx, cudaSetDevice(ctx->device));
  return css_color_impl(ctx, geom->n_mol, geom->xyz, geom->box, r_col, seed, nullptr, nullptr, colour, n_colours,
                        (cudaStream_t)stream);
}

css_status css_color_graph(css_ctx* ctx, int32_t n, const int32_t* adj_ptr, const int32_t* adj, uint64_t seed,
                           int32_t* colour, int32_t* n_colours, void* stream) {
  if (!ctx || !adj_ptr || !colour || !n_colours || n < 1) return css_set_arg_error(ctx, "css_color_graph: bad argument");
  CSS_CU(ctx, cudaSetDevice(ctx->device));
  return css_color_impl(ctx, n, nullptr, 0.0, 0.0, seed, adj_ptr, adj, colour, n_colours, (cudaStream_t)stream);
}

css_status css_color_check(css_ctx* ctx, const css_geom* geom, double r_col, const int32_t* colour,
                           int32_t n_colours, int64_t* n_conflicts, void* stream) {
  if (!ctx || !geom || !geom->xyz || !colour || !n_conflicts) return css_set_arg_error(ctx, "css_color_check: null pointer");
  CSS_TRY(check_geom(ctx, geom, r_col, "css_color_check: n_mol < 1, box not in (0, 1000] or r_col not in [0, 1000]"));
  if (n_colours < 1) return css_set_arg_error(ctx, "css_color_check: n_colours < 1");
  CSS_CU(ctx, cudaSetDevice(ctx->device));
  int64_t k = 0;
  int32_t bad = 0;
  CSS_TRY(count_conflicts(ctx, geom, r_col, colour, n_colours, &k, &bad, (cudaStream_t)stream));
  if (bad) return css_set_arg_error(ctx, "css_color_check: colour outside [0, n_colours)");
  *n_conflicts = k;
  return CSS_OK;
}

css_status css_color_update(css_ctx* ctx, const css_geom* geom, double r_col, double skin, uint64_t seed,
                            int32_t* colour, int32_t* n_colours, int32_t* recoloured, void* stream) {
  if (!ctx || !geom || !geom->xyz || !colour || !n_colours) return css_set_arg_error(ctx, "css_color_update: null pointer");
  if (!(skin >= 0.0)) return css_set_arg_error(ctx, "css_color_update: skin < 0");
  CSS_TRY(check_geom(ctx, geom, r_col + skin,
                     "css_color_update: n_mol < 1, box not in (0, 1000] or r_col + skin not in [0, 1000]"));
  CSS_CU(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (*n_colours >= 1) {
    int64_t k = 0;
    int32_t bad = 0;
    CSS_TRY(count_conflicts(ctx, geom, r_col, colour, *n_colours, &k, &bad, st));
    if (k == 0 && !bad) {
      if (recoloured) *recoloured = 0;
      return CSS_OK;
    }
  }
  int32_t nc = 0;
  CSS_TRY(css_color_impl(ctx, geom->n_mol, geom->xyz, geom->box, r_col + skin, seed, nullptr, nullptr, colour, &nc,
                         st));
  *n_colours = nc;
  if (recoloured) *recoloured = 1;
  return CSS_OK;
}

css_status css_probes(css_ctx* ctx, const int32_t* colour, int32_t n_mol, int32_t b, uint64_t sign_seed,
                      uint32_t flags, int8_t* sign, void* stream) {
  (void)colour;
  if (!ctx || !sign || n_mol < 1 || b < 1 || b > CSS_MAX_B) return css_set_arg_error(ctx, "css_probes: bad argument");
  CSS_CU(ctx, cudaSetDevice(ctx->device));
  int64_t count = (int64_t)n_mol * b;
  k_probe_signs<<<(unsigned)css_ceil_div(count, 256), 256, 0, (cudaStream_t)stream>>>(
      count, sign_seed, (flags & CSS_SIGNS_ONES) ? 1 : 0, sign);
  CSS_LAUNCHED(ctx);
  return CSS_OK;
}

}  // extern "C"
