// Device sort, scan and de-duplication used by the walk build (the sorted,
// de-duplicated (row, column) pairs of the binary adjacency behind Eqs. rw-ag,
// rw-hg, rw-mg and the KNN graph of Eq. AK) and by InitBCM's degree order
// (Alg. 4 lines 3-5).  All three are exact integer work, deterministic and
// stream-ordered.
//
//   radix_sort_u64  least-significant-digit radix sort, 8 bits per pass over
//                   [0, end_bit); each pass is a digit histogram per 4096-key
//                   tile, an exclusive scan of the (digit, tile) table, and a
//                   stable scatter that ranks a tile's keys in index order
//                   (warp match on the digit, then per-digit warp prefixes).
//   exclusive_scan  tile sums, a recursive scan of the sums, a tile add.
//   unique_u64      first-of-run flags, a scan, a compaction.
#include "common.cuh"

namespace ancka {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;  // 4096 keys or values per CTA
constexpr int kWarps = kThreads / 32;

inline unsigned blocks_for(int64_t count) { return (unsigned)ceil_div(count > 0 ? count : 1, kTile); }

// digit counts of one tile: hist[digit * tiles + tile]
__global__ void __launch_bounds__(kThreads) k_rs_hist(const uint64_t* __restrict__ keys, int64_t count, int shift,
                                                      int64_t tiles, int64_t* __restrict__ hist) {
  __shared__ uint32_t h[256];
  const int t = threadIdx.x;
  h[t] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kTile;
  const unsigned lane_lt = (1u << (t & 31)) - 1u;
  unsigned dg[kItems];  // all loads in flight before the first vote
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int64_t i = base + r * kThreads + t;
    dg[r] = i < count ? (unsigned)(keys[i] >> shift) & 255u : 256u;
  }
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const unsigned peers = __match_any_sync(0xffffffffu, dg[r]);
    if (dg[r] < 256u && (peers & lane_lt) == 0) atomicAdd(&h[dg[r]], (uint32_t)__popc(peers));
  }
  __syncthreads();
  hist[(int64_t)t * tiles + blockIdx.x] = h[t];
}

// stable scatter of one tile: keys keep their index order within a digit.
// Warp w ranks the 512 consecutive keys [w 512, (w + 1) 512) of the tile in
// 16 rounds of 32 (a match on the digit, the group's leader advancing the
// warp's counter for that digit); one block-wide prefix over the warps'
// counters then places warp w's keys of a digit after those of warps < w.
__global__ void __launch_bounds__(kThreads) k_rs_scatter(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                                         int64_t count, int shift, int64_t tiles,
                                                         const int64_t* __restrict__ off) {
  __shared__ int64_t run[256];
  __shared__ uint32_t wc[kWarps][256];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const unsigned lane_lt = (1u << lane) - 1u;
  run[t] = off[(int64_t)t * tiles + blockIdx.x];
#pragma unroll
  for (int w = 0; w < kWarps; ++w) wc[w][t] = 0;
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)warp * (32 * kItems) + lane;
  uint64_t keys[kItems];  // all loads in flight before the first rank
#pragma unroll
  for (int r = 0; r < kItems; ++r) keys[r] = base + 32 * r < count ? in[base + 32 * r] : 0ull;
  __syncthreads();
  uint32_t rank[kItems];
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const bool valid = base + 32 * r < count;
    const unsigned d = valid ? (unsigned)(keys[r] >> shift) & 255u : 256u;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int leader = __ffs(peers) - 1;
    uint32_t before = 0;
    if (valid && lane == leader) {
      before = wc[warp][d];
      wc[warp][d] = before + (uint32_t)__popc(peers);
    }
    before = __shfl_sync(0xffffffffu, before, leader);
    rank[r] = before + (uint32_t)__popc(peers & lane_lt);
    __syncwarp();
  }
  __syncthreads();
  // thread t owns digit t: counts of the warps before each warp
  uint32_t acc = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const uint32_t c = wc[w][t];
    wc[w][t] = acc;
    acc += c;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    if (base + 32 * r < count) {
      const unsigned d = (unsigned)(keys[r] >> shift) & 255u;
      out[run[d] + wc[warp][d] + rank[r]] = keys[r];
    }
  }
}

// exclusive scan of one tile (16 consecutive values per thread) + tile total
__global__ void __launch_bounds__(kThreads) k_scan_tile(const int64_t* __restrict__ in, int64_t* __restrict__ out,
                                                        int64_t count, int64_t* __restrict__ sums) {
  __shared__ int64_t wsum[kWarps];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t i0 = (int64_t)blockIdx.x * kTile + (int64_t)t * kItems;
  int64_t v[kItems];
  int64_t tot = 0;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    v[j] = i0 + j < count ? in[i0 + j] : 0;
    tot += v[j];
  }
  int64_t inc = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  int64_t before = inc - tot;
  int64_t block_tot = 0;
  for (int w = 0; w < kWarps; ++w) {
    if (w < warp) before += wsum[w];
    block_tot += wsum[w];
  }
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    if (i0 + j < count) out[i0 + j] = before;
    before += v[j];
  }
  if (t == 0 && sums) sums[blockIdx.x] = block_tot;
}

__global__ void k_scan_add(int64_t* __restrict__ out, int64_t count, const int64_t* __restrict__ tile_off) {
  const int64_t tile = blockIdx.x;
  if (tile == 0) return;
  const int64_t add = tile_off[tile];
  const int64_t base = tile * kTile;
  for (int j = threadIdx.x; j < kTile; j += blockDim.x)
    if (base + j < count) out[base + j] += add;
}

// flags[i] = 1 where a run of equal keys starts; flags[count] = 0
__global__ void k_run_starts(const uint64_t* __restrict__ in, int64_t count, int64_t* __restrict__ flags) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) flags[i] = (i == 0 || in[i] != in[i - 1]) ? 1 : 0;
  if (i == count) flags[i] = 0;
}

__global__ void k_compact_runs(const uint64_t* __restrict__ in, int64_t count, const int64_t* __restrict__ pos,
                               uint64_t* __restrict__ out, int64_t* __restrict__ count_dev) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count && (i == 0 || in[i] != in[i - 1])) out[pos[i]] = in[i];
  if (i == count) *count_dev = pos[count];
}

}  // namespace

ancka_status exclusive_scan(Workspace& ws, const int64_t* in, int64_t* out, int64_t count, cudaStream_t s) {
  if (count <= 0) return ANCKA_OK;
  const unsigned tiles = blocks_for(count);
  int64_t* sums = nullptr;
  if (tiles > 1) ANCKA_TRY(ws.alloc(&sums, (size_t)tiles));
  k_scan_tile<<<tiles, kThreads, 0, s>>>(in, out, count, sums);
  ANCKA_LAUNCHED();
  if (tiles > 1) {
    int64_t* tile_off;
    ANCKA_TRY(ws.alloc(&tile_off, (size_t)tiles));
    ANCKA_TRY(exclusive_scan(ws, sums, tile_off, tiles, s));
    k_scan_add<<<tiles, kThreads, 0, s>>>(out, count, tile_off);
    ANCKA_LAUNCHED();
  }
  return ANCKA_OK;
}

ancka_status radix_sort_u64(Workspace& ws, const uint64_t* in, uint64_t* out, int64_t count, int end_bit,
                            cudaStream_t s) {
  if (count <= 0) return ANCKA_OK;
  if (end_bit < 1) end_bit = 1;
  if (end_bit > 64) end_bit = 64;
  const int passes = (end_bit + 7) / 8;
  const int64_t tiles = blocks_for(count);
  uint64_t* tmp = nullptr;
  if (passes > 1) ANCKA_TRY(ws.alloc(&tmp, (size_t)count));
  int64_t *hist, *off;
  ANCKA_TRY(ws.alloc(&hist, (size_t)tiles * 256));
  ANCKA_TRY(ws.alloc(&off, (size_t)tiles * 256));
  const uint64_t* src = in;
  for (int p = 0; p < passes; ++p) {
    uint64_t* dst = ((passes - 1 - p) % 2 == 0) ? out : tmp;  // the last pass lands in out
    k_rs_hist<<<(unsigned)tiles, kThreads, 0, s>>>(src, count, 8 * p, tiles, hist);
    ANCKA_LAUNCHED();
    ANCKA_TRY(exclusive_scan(ws, hist, off, tiles * 256, s));
    k_rs_scatter<<<(unsigned)tiles, kThreads, 0, s>>>(src, dst, count, 8 * p, tiles, off);
    ANCKA_LAUNCHED();
    src = dst;
  }
  return ANCKA_OK;
}

ancka_status unique_u64(Workspace& ws, const uint64_t* in, uint64_t* out, int64_t* count_dev, int64_t count,
                        cudaStream_t s) {
  if (count <= 0) {
    ANCKA_CUDA(cudaMemsetAsync(count_dev, 0, sizeof(int64_t), s));
    return ANCKA_OK;
  }
  int64_t *flags, *pos;
  ANCKA_TRY(ws.alloc(&flags, (size_t)count + 1));
  ANCKA_TRY(ws.alloc(&pos, (size_t)count + 1));
  const unsigned g = (unsigned)ceil_div(count + 1, 256);
  k_run_starts<<<g, 256, 0, s>>>(in, count, flags);
  ANCKA_LAUNCHED();
  ANCKA_TRY(exclusive_scan(ws, flags, pos, count + 1, s));
  k_compact_runs<<<g, 256, 0, s>>>(in, count, pos, out, count_dev);
  ANCKA_LAUNCHED();
  return ANCKA_OK;
}

}  // namespace ancka
