// Approximate KNN by inverted lists (the large-n variant of Section 7's KNN
// construction, which the paper runs with Faiss IVFPQ for n >= 100k): the
// unit rows are partitioned by spherical k-means into nlist cells, every row
// probes its nprobe nearest cells, and the exact cosine is computed only
// against the rows of the probed cells.
//
//   1. centroids: nlist rows of U spread over the row range (seeded), then
//      `iters` rounds of spherical k-means on a strided subset of the rows
//      (assignment by the tcgen05 contraction against the centroid matrix,
//      centroid = normalised sum of its members, summed in row order);
//   2. every row's nprobe nearest centroids (the same contraction);
//   3. rows sorted by their own (nearest) cell, then by their second-nearest
//      cell, then in row order;
//   4. per 128-row query block of the sorted rows: the union of the key
//      tiles (256 sorted rows) that hold a cell probed by one of its rows;
//   5. the tcgen05 contraction of every block against its key tiles only,
//      keeping two 16-entry candidate lists per row (the exact path's kernel
//      in tile-list mode);
//   6. exact FP32 cosines of the 32 candidates, the K best by (cosine desc,
//      index asc), mapped back to the original row order.
// Every step is deterministic: no floating-point atomics, fixed summation
// orders.  With nprobe = nlist every row sweeps every key tile and the lists
// are the exact path's candidate lists.
#include <algorithm>

#include "common.cuh"

namespace ancka {

namespace {

constexpr int kIvfChunk = 4096;  // rows per chunk of the counting sort
constexpr int kTileRows = 256;   // key rows per tile of the contraction
constexpr int kBlockRows = 128;  // query rows per block of the contraction

inline unsigned grid_for(int64_t n, int b) { return (unsigned)ceil_div(n > 0 ? n : 1, b); }

__device__ __forceinline__ uint64_t splitmix64_ivf(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// centroid c = unit row of a row drawn from the c-th of nlist equal slices of
// the row range (distinct rows); padding centroids stay zero
__global__ void k_ivf_init_centroids(const __nv_bfloat16* __restrict__ xb, int dp, int64_t n, int nlist,
                                     uint64_t seed, __nv_bfloat16* __restrict__ C) {
  const int c = blockIdx.x;
  if (c >= nlist) return;
  const int64_t lo = (int64_t)c * n / nlist, hi = (int64_t)(c + 1) * n / nlist;
  const int64_t row = lo + (int64_t)(splitmix64_ivf(seed * 0x100000001ull + (uint64_t)c) % (uint64_t)(hi - lo));
  for (int f = threadIdx.x; f < dp; f += blockDim.x) C[(int64_t)c * dp + f] = xb[row * dp + f];
}

// the m best of a row's two sorted 16-entry lists (score desc, index asc)
__global__ void k_ivf_top(const float* __restrict__ cand_val, const int32_t* __restrict__ cand_idx,
                          const int32_t* __restrict__ rows, int64_t n_rows, int m, int32_t* __restrict__ out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_rows) return;
  const int64_t i = rows ? rows[q] : q;
  const float* v = cand_val + i * kCandC;
  const int32_t* x = cand_idx + i * kCandC;
  int a = 0, b = kCandC / 2;
  for (int e = 0; e < m; ++e) {
    bool take_a;
    if (a >= kCandC / 2 || x[a] < 0) take_a = false;
    else if (b >= kCandC || x[b] < 0) take_a = true;
    else take_a = v[a] > v[b] || (v[a] == v[b] && x[a] < x[b]);
    int32_t pick;
    if (take_a) pick = x[a++];
    else if (b < kCandC && x[b] >= 0) pick = x[b++];
    else pick = -1;
    out[q * m + e] = pick;
  }
}

// counting sort of a sequence of rows (seq, or the rows in order) by a key
// per row (cell), stable: per-chunk histograms ...
__global__ void k_ivf_hist(const int32_t* __restrict__ cell, const int32_t* __restrict__ seq, int64_t n, int nlist,
                           int32_t* __restrict__ hist) {
  const int64_t ch = blockIdx.x;
  const int64_t r0 = ch * kIvfChunk, r1 = min(n, r0 + kIvfChunk);
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x)
    atomicAdd(&hist[ch * nlist + max(0, cell[seq ? seq[r] : r])], 1);
}

// ... per cell, the chunks' offsets inside the cell and the cell's size ...
__global__ void k_ivf_cell_scan(int32_t* __restrict__ hist, int64_t nchunks, int nlist,
                                int64_t* __restrict__ cell_size) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nlist) return;
  int64_t run = 0;
  for (int64_t ch = 0; ch < nchunks; ++ch) {
    const int32_t c = hist[ch * nlist + l];
    hist[ch * nlist + l] = (int32_t)run;
    run += c;
  }
  cell_size[l] = run;
}

// ... exclusive scan of the cell sizes (one CTA, fixed order) ...
__global__ void k_ivf_exscan(const int64_t* __restrict__ in, int count, int64_t* __restrict__ out) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x, per = (count + blockDim.x - 1) / blockDim.x;
  const int a = t * per, b = min(count, a + per);
  int64_t s = 0;
  for (int e = a; e < b; ++e) s += in[e];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int64_t run = 0;
    for (int u = 0; u < (int)blockDim.x; ++u) {
      const int64_t v = part[u];
      part[u] = run;
      run += v;
    }
    out[count] = run;
  }
  __syncthreads();
  int64_t run = part[t];
  for (int e = a; e < b; ++e) {
    out[e] = run;
    run += in[e];
  }
}

// ... and the placement: a chunk's rows in sequence order (one thread per chunk)
__global__ void k_ivf_place(const int32_t* __restrict__ cell, const int32_t* __restrict__ seq, int64_t n, int nlist,
                            int32_t* __restrict__ hist, const int64_t* __restrict__ cell_off,
                            int32_t* __restrict__ order) {
  const int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t r0 = ch * kIvfChunk;
  if (r0 >= n) return;
  const int64_t r1 = min(n, r0 + kIvfChunk);
  // the chunk's running position per cell lives in global scratch: the
  // offsets table row of this chunk is advanced in place (each chunk owns it)
  int32_t* pos = hist + ch * nlist;
  for (int64_t r = r0; r < r1; ++r) {
    const int32_t row = seq ? seq[r] : (int32_t)r;
    const int l = max(0, cell[row]);  // a row with no finite score (NaN input) joins cell 0
    order[cell_off[l] + pos[l]++] = row;
  }
}

// centroid = normalised sum of its members' unit rows (one warp per cell,
// members in row order, FP32); an empty cell keeps its centroid
__global__ void k_ivf_update(const __nv_bfloat16* __restrict__ xb, int dp, const int32_t* __restrict__ order,
                             const int64_t* __restrict__ cell_off, int nlist, __nv_bfloat16* __restrict__ C) {
  const int l = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (l >= nlist) return;
  const int64_t a = cell_off[l], b = cell_off[l + 1];
  if (a == b) return;
  float acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0.f;
  for (int64_t p = a; p < b; ++p) {
    const __nv_bfloat16* row = xb + (int64_t)order[p] * dp;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int f = lane + 32 * q;
      if (f < dp) acc[q] += __bfloat162float(row[f]);
    }
  }
  float ss = 0.f;
#pragma unroll
  for (int q = 0; q < 16; ++q) ss = fmaf(acc[q], acc[q], ss);
  for (int off = 16; off >= 1; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
  const float inv = ss > 0.f ? rsqrtf(ss) : 0.f;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int f = lane + 32 * q;
    if (f < dp) C[(int64_t)l * dp + f] = __float2bfloat16(acc[q] * inv);
  }
}

// Key tiles of a query block: the tiles holding a row of a cell probed by one
// of the block's rows, as a bitmap over the tiles in shared memory; pass 0
// counts them, pass 1 writes them in increasing order.
__global__ void __launch_bounds__(kBlockRows)
k_ivf_block_tiles(const int32_t* __restrict__ probes, int nprobe, int64_t n, const int64_t* __restrict__ cell_off,
                  int n_tiles, int pass, int64_t* __restrict__ blk_cnt,
                  const int64_t* __restrict__ blk_ptr, int32_t* __restrict__ blk_tiles) {
  extern __shared__ uint32_t bits[];
  __shared__ int64_t wsum[kBlockRows / 32];
  const int words = (n_tiles + 31) / 32;
  for (int e = threadIdx.x; e < words; e += blockDim.x) bits[e] = 0u;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * kBlockRows + threadIdx.x;  // sorted row
  if (i < n) {
    // the block's own rows' tiles, so that every row sees its own cell
    const int own = (int)(i / kTileRows);
    atomicOr(&bits[own >> 5], 1u << (own & 31));
    for (int e = 0; e < nprobe; ++e) {
      const int l = probes[i * nprobe + e];
      if (l < 0) continue;
      const int64_t a = cell_off[l], b = cell_off[l + 1];
      if (a == b) continue;
      for (int64_t t = a / kTileRows; t <= (b - 1) / kTileRows; ++t) atomicOr(&bits[t >> 5], 1u << (t & 31));
    }
  }
  __syncthreads();
  // per thread a contiguous run of words: count, then (pass 1) write in order
  const int per = (words + blockDim.x - 1) / blockDim.x;
  const int w0 = threadIdx.x * per, w1 = min(words, w0 + per);
  int64_t c = 0;
  for (int w = w0; w < w1; ++w) c += __popc(bits[w]);
  // block-wide exclusive scan of c (fixed order)
  int64_t x = c;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  for (int off = 1; off < 32; off <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) wsum[wp] = x;
  __syncthreads();
  int64_t before = x - c;
  for (int q = 0; q < wp; ++q) before += wsum[q];
  int64_t total = 0;
  for (int q = 0; q < kBlockRows / 32; ++q) total += wsum[q];
  if (pass == 0) {
    if (threadIdx.x == 0) blk_cnt[blockIdx.x] = total;
    return;
  }
  int32_t* out = blk_tiles + blk_ptr[blockIdx.x] + before;
  for (int w = w0; w < w1; ++w) {
    uint32_t m = bits[w];
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      *out++ = w * 32 + b;
    }
  }
}

// probes of every sorted row
__global__ void k_ivf_permute_probes(const int32_t* __restrict__ order, const int32_t* __restrict__ probes, int64_t n,
                                     int nprobe, int32_t* __restrict__ out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * nprobe) return;
  const int64_t p = q / nprobe;
  out[q] = probes[(int64_t)order[p] * nprobe + (q % nprobe)];
}

// Cosines of a row's 32 candidates (one warp per sorted row, one lane per
// candidate: a compensated FP32 dot product of the original rows scaled by
// the FP64 norms, rounded once to FP32), sorted by (cosine desc, original
// index asc); the K best go to the row's original position with original
// indices.
__global__ void k_ivf_rerank(const float* __restrict__ X, int d, const double* __restrict__ nrm2,
                             const int32_t* __restrict__ order, int64_t n, const float* __restrict__ cand_val,
                             const int32_t* __restrict__ cand_idx, int K, int32_t* __restrict__ out_idx,
                             float* __restrict__ out_sim) {
  const int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (p >= n) return;
  const int64_t i = order[p];
  const int32_t jc = cand_idx[p * kCandC + lane];
  const int64_t j = jc >= 0 ? (int64_t)order[jc] : -1;
  float s = -INFINITY;
  if (j >= 0) {
    const float* xi = X + i * d;
    const float* xj = X + j * d;
    // compensated dot product (Ogita, Rump and Oishi's Dot2: TwoProduct by
    // FMA, TwoSum of the running sum), ~2^-44 relative before the division
    float hi = 0.f, lo = 0.f;
    for (int f = 0; f < d; ++f) {
      const float pr = xi[f] * xj[f];
      const float pe = fmaf(xi[f], xj[f], -pr);
      const float t = hi + pr;
      const float z = t - hi;
      lo += (hi - (t - z)) + (pr - z) + pe;
      hi = t;
    }
    const double ni = nrm2[i], nj = nrm2[j];
    s = (ni > 0.0 && nj > 0.0) ? (float)(((double)hi + (double)lo) / sqrt(ni * nj)) : 0.f;
  }
  // bitonic sort of 32 (score desc, index asc) pairs across the warp
  int64_t key_j = j >= 0 ? j : INT64_MAX;
  for (int size = 2; size <= 32; size <<= 1) {
    for (int stride = size >> 1; stride >= 1; stride >>= 1) {
      const float os = __shfl_xor_sync(0xffffffffu, s, stride);
      const int64_t oj = __shfl_xor_sync(0xffffffffu, key_j, stride);
      const bool up = ((lane & size) == 0);           // this pair sorts "better first"
      const bool lower = (lane & stride) == 0;
      const bool mine_better = s > os || (s == os && key_j < oj);
      const bool keep_mine = (lower == up) ? mine_better : !mine_better;
      if (!keep_mine) {
        s = os;
        key_j = oj;
      }
    }
  }
  if (lane < K) {
    out_idx[i * K + lane] = key_j == INT64_MAX ? -1 : (int32_t)key_j;
    out_sim[i * K + lane] = s;
  }
}

// training subset: rows floor(t n / n_train)
__global__ void k_strided_rows(int64_t n, int64_t n_train, int32_t* __restrict__ rows) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n_train) rows[t] = (int32_t)(t * n / n_train);
}

// order holds positions into the subset: map them to rows
__global__ void k_ivf_map_order(const int32_t* __restrict__ rows, int64_t count, int32_t* __restrict__ order) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count && rows) order[t] = rows[order[t]];
}

// a row's e-th nearest cell (0 if missing)
__global__ void k_ivf_nth(const int32_t* __restrict__ probes, int nprobe, int64_t n, int e, int32_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = max(0, probes[i * nprobe + e]);
}

// a row's own cell = its nearest centroid (the first probe)
__global__ void k_ivf_first(const int32_t* __restrict__ probes, int nprobe, int64_t n, int32_t* __restrict__ cell) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) cell[i] = max(0, probes[i * nprobe]);
}

// BF16 rows in the order given (zero rows past n)
__global__ void k_gather_rows_bf16(const __nv_bfloat16* __restrict__ x, int dp, const int32_t* __restrict__ order,
                                   int64_t n, int64_t n_pad, __nv_bfloat16* __restrict__ out) {
  const int64_t p = blockIdx.x;
  if (p >= n_pad) return;
  const uint4* src = p < n ? reinterpret_cast<const uint4*>(x + (int64_t)order[p] * dp) : nullptr;
  uint4* dst = reinterpret_cast<uint4*>(out + p * dp);
  for (int c = threadIdx.x; c < dp / 8; c += blockDim.x) dst[c] = src ? src[c] : make_uint4(0, 0, 0, 0);
}

// exclusive scan of count int64 values into count + 1 (one CTA, fixed order)
ancka_status exclusive_scan_i64(Workspace&, const int64_t* in, int64_t* out, int64_t count, cudaStream_t s) {
  k_ivf_exscan<<<1, 1024, 0, s>>>(in, (int)count, out);
  ANCKA_LAUNCHED();
  return ANCKA_OK;
}

// the rows (of seq, or all in order) sorted by cell, stable: order[position]
// = row, and the cells' offsets (nlist + 1)
ancka_status sort_by_cell(Workspace& ws, const int32_t* cell, const int32_t* seq, int64_t n, int nlist, int32_t* order,
                          int64_t* cell_off, cudaStream_t s) {
  const int64_t nchunks = ceil_div(n, kIvfChunk);
  int32_t* hist;
  int64_t* size;
  ANCKA_TRY(ws.zeros(&hist, (size_t)nchunks * nlist));
  ANCKA_TRY(ws.alloc(&size, (size_t)nlist));
  k_ivf_hist<<<(unsigned)nchunks, 256, 0, s>>>(cell, seq, n, nlist, hist);
  ANCKA_LAUNCHED();
  k_ivf_cell_scan<<<grid_for(nlist, 128), 128, 0, s>>>(hist, nchunks, nlist, size);
  ANCKA_LAUNCHED();
  k_ivf_exscan<<<1, 1024, 0, s>>>(size, nlist, cell_off);
  ANCKA_LAUNCHED();
  k_ivf_place<<<grid_for(nchunks, 64), 64, 0, s>>>(cell, seq, n, nlist, hist, cell_off, order);
  ANCKA_LAUNCHED();
  return ANCKA_OK;
}

}  // namespace

int ivf_max_tiles() { return 1 << 16; }

ancka_status knn_ivf(Workspace& ws, const float* X, int64_t n, int32_t d, int32_t K, int32_t nlist, int32_t nprobe,
                     int32_t iters, uint64_t seed, int32_t* out_idx, float* out_sim, int32_t** zero_row,
                     IvfStats* stats, cudaStream_t s) {
  PrepOut pr;
  ANCKA_TRY(prep_rows(ws, X, n, d, ANCKA_PREC_BF16, &pr, s));
  if (zero_row) *zero_row = pr.zero_row;
  const int dp = pr.dp;
  int32_t* terr;
  ANCKA_TRY(ws.zeros(&terr, 1));
  float* cv;
  int32_t* ci;
  ANCKA_TRY(ws.alloc(&cv, (size_t)n * kCandC));
  ANCKA_TRY(ws.alloc(&ci, (size_t)n * kCandC));
  // 1. centroids (zero padding rows up to the key tile height)
  const int64_t nl_pad = round_up(nlist, kTileRows);
  __nv_bfloat16* C;
  ANCKA_TRY(ws.zeros(&C, (size_t)nl_pad * dp));
  k_ivf_init_centroids<<<(unsigned)nlist, 128, 0, s>>>(pr.xb, dp, n, nlist, seed, C);
  ANCKA_LAUNCHED();
  const int64_t n_train = std::min<int64_t>(n, (int64_t)64 * nlist);
  int32_t* train_rows;
  int32_t* cell;
  int32_t* order;
  int64_t* cell_off;
  ANCKA_TRY(ws.alloc(&train_rows, (size_t)n_train));
  ANCKA_TRY(ws.alloc(&cell, (size_t)n));
  ANCKA_TRY(ws.alloc(&order, (size_t)n));
  ANCKA_TRY(ws.alloc(&cell_off, (size_t)nlist + 1));
  k_strided_rows<<<grid_for(n_train, 256), 256, 0, s>>>(n, n_train, train_rows);
  ANCKA_LAUNCHED();
  for (int it = 0; it < iters; ++it) {
    ANCKA_TRY(knn_lists_bf16(ws, pr.xb, pr.n_pad, n_train < n ? train_rows : nullptr, n_train, C, nlist, nl_pad, dp, d,
                             nullptr, nullptr, 0, true, cv, ci, terr, s));
    k_ivf_top<<<grid_for(n_train, 256), 256, 0, s>>>(cv, ci, n_train < n ? train_rows : nullptr, n_train, 1, cell);
    ANCKA_LAUNCHED();
    ANCKA_TRY(sort_by_cell(ws, cell, nullptr, n_train, nlist, order, cell_off, s));
    k_ivf_map_order<<<grid_for(n_train, 256), 256, 0, s>>>(n_train < n ? train_rows : nullptr, n_train, order);
    ANCKA_LAUNCHED();
    k_ivf_update<<<grid_for((int64_t)nlist * 32, 256), 256, 0, s>>>(pr.xb, dp, order, cell_off, nlist, C);
    ANCKA_LAUNCHED();
  }
  // 2. every row's nprobe nearest cells; its own cell is the first
  int32_t* probes;
  ANCKA_TRY(ws.alloc(&probes, (size_t)n * nprobe));
  ANCKA_TRY(knn_lists_bf16(ws, pr.xb, pr.n_pad, nullptr, n, C, nlist, nl_pad, dp, d, nullptr, nullptr, 0, true, cv, ci,
                           terr, s));
  k_ivf_top<<<grid_for(n, 256), 256, 0, s>>>(cv, ci, nullptr, n, nprobe, probes);
  ANCKA_LAUNCHED();
  k_ivf_first<<<grid_for(n, 256), 256, 0, s>>>(probes, nprobe, n, cell);
  ANCKA_LAUNCHED();
  // 3. rows sorted by (own cell, second-nearest cell, row): rows of a block
  // then share more of their probed cells (two stable passes, minor key first)
  {
    int32_t *second, *order1;
    int64_t* off1;
    ANCKA_TRY(ws.alloc(&second, (size_t)n));
    ANCKA_TRY(ws.alloc(&order1, (size_t)n));
    ANCKA_TRY(ws.alloc(&off1, (size_t)nlist + 1));
    k_ivf_nth<<<grid_for(n, 256), 256, 0, s>>>(probes, nprobe, n, nprobe > 1 ? 1 : 0, second);
    ANCKA_LAUNCHED();
    ANCKA_TRY(sort_by_cell(ws, second, nullptr, n, nlist, order1, off1, s));
    ANCKA_TRY(sort_by_cell(ws, cell, order1, n, nlist, order, cell_off, s));
  }
  __nv_bfloat16* xs;
  ANCKA_TRY(ws.alloc(&xs, (size_t)pr.n_pad * dp));
  k_gather_rows_bf16<<<(unsigned)pr.n_pad, 64, 0, s>>>(pr.xb, dp, order, n, pr.n_pad, xs);
  ANCKA_LAUNCHED();
  int32_t* sprobes;
  ANCKA_TRY(ws.alloc(&sprobes, (size_t)n * nprobe));
  k_ivf_permute_probes<<<grid_for(n * nprobe, 256), 256, 0, s>>>(order, probes, n, nprobe, sprobes);
  ANCKA_LAUNCHED();
  // 4. key tiles of every query block
  const int64_t qblocks = ceil_div(n, kBlockRows);
  const int n_tiles = (int)ceil_div(pr.n_pad, kTileRows);
  if (n_tiles > ivf_max_tiles()) {
    set_error("inverted-list KNN: n = %lld exceeds %d key tiles", (long long)n, ivf_max_tiles());
    return ANCKA_ERR_UNSUPPORTED;
  }
  int64_t *blk_cnt, *blk_ptr;
  ANCKA_TRY(ws.alloc(&blk_cnt, (size_t)qblocks));
  ANCKA_TRY(ws.alloc(&blk_ptr, (size_t)qblocks + 1));
  const size_t bm = (size_t)((n_tiles + 31) / 32) * sizeof(uint32_t);
  if (bm > 48 * 1024)
    ANCKA_CUDA(cudaFuncSetAttribute(k_ivf_block_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bm));
  k_ivf_block_tiles<<<(unsigned)qblocks, kBlockRows, bm, s>>>(sprobes, nprobe, n, cell_off, n_tiles, 0, blk_cnt,
                                                              nullptr, nullptr);
  ANCKA_LAUNCHED();
  ANCKA_TRY(exclusive_scan_i64(ws, blk_cnt, blk_ptr, qblocks, s));
  int64_t work = 0;
  ANCKA_CUDA(cudaMemcpyAsync(&work, blk_ptr + qblocks, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  ANCKA_CUDA(cudaStreamSynchronize(s));
  int32_t* blk_tiles;
  ANCKA_TRY(ws.alloc(&blk_tiles, (size_t)std::max<int64_t>(work, 1)));
  k_ivf_block_tiles<<<(unsigned)qblocks, kBlockRows, bm, s>>>(sprobes, nprobe, n, cell_off, n_tiles, 1, blk_cnt,
                                                              blk_ptr, blk_tiles);
  ANCKA_LAUNCHED();
  // 5. the contraction of every block against its tiles (sorted row ids)
  ANCKA_TRY(knn_lists_bf16(ws, xs, pr.n_pad, nullptr, n, xs, n, pr.n_pad, dp, d, blk_ptr, blk_tiles, work, false, cv,
                           ci, terr, s));
  // 6. exact cosines of the candidates, back to the original order
  k_ivf_rerank<<<grid_for(n * 32, 256), 256, 0, s>>>(X, d, pr.nrm2, order, n, cv, ci, K, out_idx, out_sim);
  ANCKA_LAUNCHED();
  int32_t he = 0;
  ANCKA_CUDA(cudaMemcpyAsync(&he, terr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  ANCKA_CUDA(cudaStreamSynchronize(s));
  if (he) {
    set_error("inverted-list KNN: a contraction pipeline wait expired (role %d)", he);
    return ANCKA_ERR_TIMEOUT;
  }
  if (stats) {
    stats->key_tiles = work;
    stats->full_tiles = qblocks * (int64_t)n_tiles;
  }
  return ANCKA_OK;
}

}  // namespace ancka
