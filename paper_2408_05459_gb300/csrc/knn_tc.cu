// tcgen05 BF16 / FP8-e4m3 candidate search for the cosine KNN of Section 3.1.
//
// Persistent CTAs (one per SM) share the (128-row query block, 256-row key
// tile) pairs in equal contiguous runs (stream-K), so no wave tail is left
// idle.  In each CTA:
//   warp 0     TMA producer: the current query block A (128 x dp, 128-byte
//              swizzle) when the run enters it, then key tiles B (256 rows x
//              128 bytes of features per stage: 64 BF16 or 128 FP8) through
//              an nstages-deep ring (mbarrier full/empty);
//   warp 1     MMA issuer: allocates 512 TMEM columns, issues
//              tcgen05.mma.cta_group::1.kind::f16 (BF16, K=16) or
//              kind::f8f6f4 (E4M3, K=32) with M=128, N=256 into two
//              ping-pong FP32 accumulators, commits stage releases,
//              accumulator-ready signals and the release of A at the end of
//              each query block;
//   warps 2-9  epilogue: two warps per TMEM lane quarter, each owning half of
//              every tile's 256 columns; tcgen05.ld (32x32b) of the thread's
//              accumulator row (TMEM lane = query row), threshold test and
//              insert into a register-resident list of its 16 best scores.
//              Row i thus leaves two 16-entry lists (one per column half),
//              kCandC = 32 candidates in total; a query block split between
//              two CTAs leaves partial lists that k_merge_lists combines.
// The MMA of tile t+1 overlaps the epilogue of tile t.  n x n scores never
// leave the SM.  Every mbarrier wait is bounded: on expiry the kernel records
// an error code, stops all roles, drains its own copies and MMAs (bounded),
// frees TMEM and returns.
#include <algorithm>
#include <atomic>

#include "tc_common.cuh"

namespace ancka {

namespace {

constexpr int kTM = 128;                 // query rows per CTA = TMEM lanes
constexpr int kTN = 256;                 // key rows per tile = accumulator columns
constexpr int kLists = 2;                // lists per row = column slices of every tile
constexpr int kEpiWarps = 4 * kLists;    // one warp per (TMEM lane quarter, column slice)
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kListC = kCandC / kLists;  // entries of each list
constexpr int kSliceN = kTN / kLists;    // columns of a tile per slice
constexpr int kABytes = kTM * kTKB;      // 16 KB per 128-byte block of A
constexpr int kBBytes = kTN * kTKB;      // 32 KB per stage of B
constexpr int kMmaPerStage = 4;          // 32 bytes of K per MMA: 16 BF16 or 32 FP8
constexpr int kMaxStages = 8;
constexpr int kMaxSmem = 232448;         // 227 KB opt-in dynamic shared memory
constexpr uint32_t kTmemCols = 512;      // two 256-column FP32 accumulators

// instruction descriptors: D = F32 (bits 4-5 = 1), both operands K-major,
// N >> 3 at bits 17-22, M >> 4 at bits 24-28; kind::f16 with A = B = BF16
// (format 1 at bits 7-9 and 10-12); kind::f8f6f4 with A = B = E4M3 (format 0)
constexpr uint32_t kIdescBF16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                                ((uint32_t)(kTM >> 4) << 24);
constexpr uint32_t kIdescE4M3 = (1u << 4) | ((uint32_t)(kTN >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);

struct __align__(8) Bars {
  uint64_t full[kMaxStages];
  uint64_t empty[kMaxStages];
  uint64_t a_full;
  uint64_t a_empty;
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
  int rot[2];  // key rotation of the current and the previous segment (written by the producer)
};

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          tmem_d),
      "l"(da), "l"(db), "r"(kIdescBF16), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void umma_e4m3(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(
          tmem_d),
      "l"(da), "l"(db), "r"(kIdescE4M3), "r"(accum)
      : "memory");
}
// Row lists are kept sorted in descending score order, lv[0] >= ... >=
// lv[C-1], so the threshold is lv[C-1] and an insert is C independent
// select pairs (two levels deep) instead of a C-long minimum scan.  A score
// equal to an entry goes after it: among equal scores the earlier key stays.
template <int C>
__device__ __forceinline__ void sorted_insert(float (&lv)[C], int32_t (&li)[C], float s, int32_t j) {
#pragma unroll
  for (int c = C - 1; c >= 1; --c) {
    const bool at_or_before = s > lv[c];
    const bool before_prev = s > lv[c - 1];
    lv[c] = at_or_before ? (before_prev ? lv[c - 1] : s) : lv[c];
    li[c] = at_or_before ? (before_prev ? li[c - 1] : j) : li[c];
  }
  if (s > lv[0]) {
    lv[0] = s;
    li[0] = j;
  }
}

// r[e] for a lane-dependent e in 0..31: a five-level select tree
__device__ __forceinline__ float pick32(const uint32_t (&r)[32], int e) {
  float v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float((e & 16) ? r[q + 16] : r[q]);
#pragma unroll
  for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
    for (int q = 0; q < w; ++q) v[q] = (e & w) ? v[q + w] : v[q];
  return v[0];
}

// Fold one 32-key chunk (scores in r, keys j0..j0+31, mx = their maximum
// from the TMEM load) into the row's list.
template <int C>
__device__ __forceinline__ void fold_chunk(const uint32_t (&r)[32], float mx, int64_t j0, int64_t n, int64_t i,
                                           float (&lv)[C], int32_t (&li)[C]) {
  // skip the chunk when no lane of the warp has a key above its threshold
  const float thr0 = lv[C - 1];
  if (!__any_sync(0xffffffffu, mx > thr0)) return;
  // pass mask against the threshold at chunk start (it only rises, so the
  // mask is a superset); padding keys and the row itself removed
  uint32_t pm = 0;
#pragma unroll
  for (int e = 0; e < 32; ++e) pm |= (__uint_as_float(r[e]) > thr0 ? 1u : 0u) << e;
  if (j0 + 32 > n) pm &= (j0 >= n) ? 0u : ((1u << (uint32_t)(n - j0)) - 1u);
  if (i >= j0 && i < j0 + 32) pm &= ~(1u << (uint32_t)(i - j0));
  // one insert per passing key; lanes without keys idle
  while (__any_sync(0xffffffffu, pm != 0)) {
    if (pm) {
      const int e = __ffs(pm) - 1;
      pm &= pm - 1;
      const float val = pick32(r, e);
      if (val > lv[C - 1]) sorted_insert<C>(lv, li, val, (int32_t)(j0 + e));
    }
  }
}

// Collect mode: append every key whose score reaches the row's fixed
// threshold t to the row's buffer (cap entries; the counter keeps counting
// past cap so the caller can see an overflow).
__device__ __forceinline__ void collect_chunk(const uint32_t (&r)[32], float mx, int64_t j0, int64_t n, int64_t i,
                                              float t, int64_t ra, int32_t* __restrict__ cnt,
                                              int32_t* __restrict__ buf, int cap) {
  if (!__any_sync(0xffffffffu, mx >= t)) return;
  uint32_t pm = 0;
#pragma unroll
  for (int e = 0; e < 32; ++e) pm |= (__uint_as_float(r[e]) >= t ? 1u : 0u) << e;
  if (j0 + 32 > n) pm &= (j0 >= n) ? 0u : ((1u << (uint32_t)(n - j0)) - 1u);
  if (i >= j0 && i < j0 + 32) pm &= ~(1u << (uint32_t)(i - j0));
  while (pm) {
    const int e = __ffs(pm) - 1;
    pm &= pm - 1;
    const int pos = atomicAdd(&cnt[ra], 1);
    if (pos < cap) buf[ra * (int64_t)cap + pos] = (int32_t)(j0 + e);
  }
}

struct CollectArgs {
  const int32_t* a_rows;  // global row of each compact query row (null: A holds rows 0..n-1)
  int64_t n_a;            // compact query rows (0: as many as keys)
  const float* thr;       // collect mode: per compact row threshold
  int32_t* cnt;           // collect mode: per compact row counter
  int32_t* buf;           // collect mode: n_a x cap keys
  int cap;
  // tile-list mode (null: every block sweeps every key tile): query block qb
  // sweeps the key tiles blk_tiles[blk_ptr[qb] .. blk_ptr[qb + 1])
  const int64_t* blk_ptr = nullptr;
  const int32_t* blk_tiles = nullptr;
  int64_t blk_work = 0;   // blk_ptr[qblocks]
  int no_self = 0;        // the keys are another set (no row excludes "itself")
};

// The segment of query block qb that a run [w, w_end) covers from w:
// positions [t0, t1) of the block's len key tiles.
struct Seg {
  int64_t qb;
  int t0, t1, len;
  int64_t base;  // tile-list mode: offset of the block's tiles
};
__device__ __forceinline__ Seg segment_at(int64_t w, int64_t w_end, int n_tiles, int64_t qblocks,
                                          const CollectArgs& ca) {
  Seg sg;
  if (ca.blk_ptr) {
    int64_t lo = 0, hi = qblocks;  // the last qb with blk_ptr[qb] <= w
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (ca.blk_ptr[mid] <= w) lo = mid; else hi = mid;
    }
    sg.qb = lo;
    sg.base = ca.blk_ptr[lo];
    sg.len = (int)(ca.blk_ptr[lo + 1] - sg.base);
  } else {
    sg.qb = w / n_tiles;
    sg.base = sg.qb * n_tiles;
    sg.len = n_tiles;
  }
  sg.t0 = (int)(w - sg.base);
  sg.t1 = (int)(w_end - w < (int64_t)(sg.len - sg.t0) ? sg.t0 + (w_end - w) : sg.len);
  return sg;
}

// Work split (stream-K): the (query block, key tile) pairs, numbered
// qb * n_tiles + t, are cut into gridDim.x equal contiguous ranges, one per
// persistent CTA.  A CTA's range is a sequence of segments, one per query
// block it touches; only its first and its last segment can miss part of a
// block's key tiles.  Such a partial segment leaves its lists in slot 0
// (first segment) or 1 (last) of the CTA's partial area, and k_merge_lists
// combines the pieces of every split block.
__device__ __forceinline__ int64_t range_begin(int64_t c, int64_t work, int64_t ctas) { return c * work / ctas; }

// Position t of query block qb sweeps key tile (t + key_rotation(qb)) mod
// n_tiles.  The rotation puts the block's first tile at the time its owner
// CTA (the one whose run holds position 0) reaches it, modulo n_tiles, so at
// any moment the CTAs read the same key tile and each tile comes from DRAM
// about once per sweep (only a run's first, split segment is out of step).
__device__ __forceinline__ int key_rotation(int64_t qb, int n_tiles, int64_t work, int64_t ctas) {
  const int64_t x0 = qb * n_tiles;
  const int64_t c0 = ((x0 + 1) * ctas + work - 1) / work - 1;
  const int64_t lag = x0 - range_begin(c0, work, ctas);  // owner's time at position 0
  return (int)(lag % n_tiles);
}

// kCollect: collect mode (keys above a per-row threshold) instead of list
// mode (two 16-entry lists per row); kE4M3: FP8 operands.  out_scale (list
// mode, may be null) multiplies the scores written out.
// key_stride > 1: only every key_stride-th key tile is swept (the sampled
// pass of the symmetric contraction).  k_last: MMAs issued for the last
// 128-byte block of features (those past the last one holding a feature of
// X are zero padding and are skipped).
template <bool kCollect, bool kE4M3>
__global__ void __launch_bounds__(kThreads, 1)
k_knn_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int64_t n,
         int64_t n_pad, int64_t qblocks, int kb_count, int k_last, int nstages, int key_stride,
         float* __restrict__ cand_val,
         int32_t* __restrict__ cand_idx, const float* __restrict__ out_scale, float* __restrict__ part_val,
         int32_t* __restrict__ part_idx, CollectArgs ca, unsigned long long* __restrict__ tick,
         int* __restrict__ err) {
  constexpr int kTK = kE4M3 ? 128 : 64;  // features per stage
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = sA + kb_count * kABytes;
  Bars* bars = reinterpret_cast<Bars*>(sB + nstages * kBBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_tiles = (int)ceil_div(ceil_div(n_pad, kTN), key_stride);
  const int64_t work = ca.blk_ptr ? ca.blk_work : qblocks * n_tiles;
  const int64_t w_begin = range_begin(blockIdx.x, work, gridDim.x);
  const int64_t w_end = range_begin((int64_t)blockIdx.x + 1, work, gridDim.x);
  volatile int* abort = &bars->abort;

  if (threadIdx.x == 0) {
    for (int s = 0; s < nstages; ++s) {
      mbar_init(&bars->full[s], 1);
      mbar_init(&bars->empty[s], 1);
    }
    mbar_init(&bars->a_full, 1);
    mbar_init(&bars->a_empty, 1);
    mbar_init(&bars->tfull[0], 1);
    mbar_init(&bars->tfull[1], 1);
    mbar_init(&bars->tempty[0], kEpiWarps);
    mbar_init(&bars->tempty[1], kEpiWarps);
    mbar_init(&bars->drain, 1);
    bars->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&bars->tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      bool pending[kMaxStages];
      uint32_t pend_par[kMaxStages];
      for (int s = 0; s < kMaxStages; ++s) pending[s] = false;
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int seg = 0;
      uint32_t tiles_issued = 0;
      for (int64_t w = w_begin; w < w_end && ok; ++seg) {
        const Seg sg = segment_at(w, w_end, n_tiles, qblocks, ca);
        const int64_t qb = sg.qb;
        const int t0 = sg.t0, t1 = sg.t1;
        int rot = ca.blk_ptr ? 0 : key_rotation(qb, n_tiles, work, gridDim.x);
        w += t1 - t0;
        // the previous block of A stays in use until its last MMA completes
        if (seg > 0 && !mbar_wait(&bars->a_empty, (uint32_t)((seg - 1) & 1), abort, err, 6)) {
          ok = false;
          break;
        }
        // A block this CTA sweeps whole starts at the key tile the CTAs are
        // reading now (tiles issued by all CTAs / CTAs), so that CTAs whose
        // rates drift apart re-align at every block and keep sharing the key
        // tiles in L2; a split block keeps the static rotation both of its
        // CTAs can compute.
        if (tick && !ca.blk_ptr && t0 == 0 && t1 == n_tiles)
          rot = (int)((*reinterpret_cast<volatile unsigned long long*>(tick) / gridDim.x) % (uint64_t)n_tiles);
        bars->rot[seg & 1] = rot;
        __threadfence_block();
        mbar_expect_tx(&bars->a_full, (uint32_t)(kb_count * kABytes));
        for (int kb = 0; kb < kb_count; ++kb)
          tma_load_2d(smem_u32(sA + kb * kABytes), &tmA, kb * kTK, (int)(qb * kTM), &bars->a_full);
        for (int t = t0; t < t1 && ok; ++t) {
          for (int kb = 0; kb < kb_count; ++kb) {
            if (!mbar_wait(&bars->empty[stage], phase ^ 1, abort, err, 1)) {
              ok = false;
              break;
            }
            pending[stage] = false;
            mbar_expect_tx(&bars->full[stage], (uint32_t)kBBytes);
            const int kt = ca.blk_ptr ? ca.blk_tiles[sg.base + t]
                                      : (t + rot < n_tiles ? t + rot : t + rot - n_tiles) * key_stride;
            tma_load_2d(smem_u32(sB + stage * kBBytes), &tmB, kb * kTK, kt * kTN, &bars->full[stage]);
            pending[stage] = true;
            pend_par[stage] = phase;
            if (++stage == nstages) {
              stage = 0;
              phase ^= 1;
            }
          }
          if (tick && ((++tiles_issued) & 15) == 0) atomicAdd(tick, 16ull);
        }
      }
      if (!ok) {  // drain this warp's copies still in flight (bounded)
        if (seg > 0) mbar_wait(&bars->a_full, (uint32_t)((seg - 1) & 1), nullptr, nullptr, 0);
        for (int s = 0; s < nstages; ++s)
          if (pending[s]) mbar_wait(&bars->full[s], pend_par[s], nullptr, nullptr, 0);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      int stage = 0;
      uint32_t phase = 0;
      bool issued = false;
      int64_t g = 0;  // accumulator tiles so far (ping-pong over two)
      int seg = 0;
      for (int64_t w = w_begin; w < w_end && ok; ++seg) {
        const Seg sg = segment_at(w, w_end, n_tiles, qblocks, ca);
        const int t0 = sg.t0, t1 = sg.t1;
        w += t1 - t0;
        if (!mbar_wait(&bars->a_full, (uint32_t)(seg & 1), abort, err, 2)) {
          ok = false;
          break;
        }
        for (int t = t0; t < t1; ++t, ++g) {
          const int b = (int)(g & 1);
          const uint32_t use = (uint32_t)(g >> 1);
          if (!mbar_wait(&bars->tempty[b], (use & 1) ^ 1, abort, err, 3)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(b * kTN);
          for (int kb = 0; kb < kb_count; ++kb) {
            if (!mbar_wait(&bars->full[stage], phase, abort, err, 4)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA + kb * kABytes);
            const uint32_t b0 = smem_u32(sB + stage * kBBytes);
            const int kmax = kb == kb_count - 1 ? k_last : kMmaPerStage;
#pragma unroll
            for (int kk = 0; kk < kMmaPerStage; ++kk) {
              if (kk >= kmax) break;
              if constexpr (kE4M3)
                umma_e4m3(d, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), (kb | kk) != 0 ? 1u : 0u);
              else
                umma_bf16(d, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), (kb | kk) != 0 ? 1u : 0u);
            }
            issued = true;
            umma_commit(&bars->empty[stage]);
            if (++stage == nstages) {
              stage = 0;
              phase ^= 1;
            }
          }
          if (!ok) break;
          umma_commit(&bars->tfull[b]);
        }
        if (ok) umma_commit(&bars->a_empty);  // A may be replaced once these MMAs complete
      }
      if (!ok && issued) {  // wait for this thread's MMAs before TMEM is freed (bounded)
        umma_commit(&bars->drain);
        mbar_wait(&bars->drain, 0, nullptr, nullptr, 0);
      }
    }
  } else {
    const int ew = warp - 2;   // epilogue warp 0..7
    const int q = warp & 3;    // TMEM lane quarter this warp may access
    const int h = ew >> 2;     // column slice of every tile
    const int r = q * 32 + lane;
    constexpr int C = kListC;
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
    const float sc = (!kCollect && out_scale) ? *out_scale : 1.f;
    int64_t g = 0;
    int seg = 0;
    bool ok = true;
    for (int64_t w = w_begin; w < w_end && ok; ++seg) {
      const Seg sg = segment_at(w, w_end, n_tiles, qblocks, ca);
      const int64_t qb = sg.qb;
      const int t0 = sg.t0, t1 = sg.t1;
      int rot = 0;
      w += t1 - t0;
      // A row ra is query row ra, or compact row ra -> global row a_rows[ra]
      const int64_t ra = qb * kTM + r;
      const bool row_ok = ra < (ca.n_a > 0 ? ca.n_a : n);
      const int64_t i = ca.a_rows ? (row_ok ? (int64_t)ca.a_rows[ra] : -1) : ra;
      const int64_t i_self = ca.no_self ? -1 : i;  // the key index this row excludes
      const float t_row = kCollect && row_ok ? ca.thr[ra] : INFINITY;
      float lv[C];
      int32_t li[C];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        lv[c] = -INFINITY;
        li[c] = -1;
      }
      for (int t = t0; t < t1; ++t, ++g) {
        const int b = (int)(g & 1);
        const uint32_t use = (uint32_t)(g >> 1);
        const bool got = mbar_wait(&bars->tfull[b], use & 1, abort, err, 5);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        tc_fence_after();
        // the producer wrote the segment's rotation before loading its block
        // of A, which the first accumulator of the segment waited for
        if (t == t0) rot = *reinterpret_cast<volatile int*>(&bars->rot[seg & 1]);
        const int kt = ca.blk_ptr ? ca.blk_tiles[sg.base + t]
                                  : (t + rot < n_tiles ? t + rot : t + rot - n_tiles) * key_stride;
        const int64_t jb = (int64_t)kt * kTN + h * kSliceN;
        const uint32_t tb = lane_base + (uint32_t)(b * kTN + h * kSliceN);
        // the hardware's maximum over each 32-column load settles most
        // chunks with one compare and one vote
#pragma unroll 1
        for (int c = 0; c < kSliceN / 32; ++c) {
          uint32_t rv[32];
          float mx;
          tmem_ld32_max_issue(tb + (uint32_t)(c * 32), rv, mx);
          tmem_wait();
          pin(rv);
          pin1(mx);
          if constexpr (kCollect) {
            collect_chunk(rv, mx, jb + c * 32, n, i_self, t_row, ra, ca.cnt, ca.buf, ca.cap);
          } else {
            fold_chunk<C>(rv, mx, jb + c * 32, n, i_self, lv, li);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars->tempty[b]);
      }
      if (!kCollect && ok) {
        float* ov;
        int32_t* oi;
        if (t0 == 0 && t1 == sg.len) {  // whole block: final lists
          if (!row_ok) continue;
          ov = cand_val + i * kCandC;
          oi = cand_idx + i * kCandC;
        } else {
          const int64_t slot = ((int64_t)blockIdx.x * 2 + (seg == 0 ? 0 : 1)) * kTM + r;
          ov = part_val + slot * kCandC;
          oi = part_idx + slot * kCandC;
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
          ov[h * C + c] = lv[c] * sc;
          oi[h * C + c] = li[c];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// Lists of the query blocks split between runs: per row and column half, the
// 16 best of the pieces' lists (each piece holds the best of its own key
// tiles, so the result is the best of the whole half).  One CTA of kTM
// threads per query block; blocks that one run covered return at once.
// Block qb's work items are [x0, x1) = [qb n_tiles, (qb + 1) n_tiles), or
// [blk_ptr[qb], blk_ptr[qb + 1]) in tile-list mode (a block with no tiles
// gets empty lists).
__global__ void __launch_bounds__(kTM) k_merge_lists(int n_tiles, int64_t work, int64_t ctas,
                                                     const int64_t* __restrict__ blk_ptr,
                                                     const float* __restrict__ part_val,
                                                     const int32_t* __restrict__ part_idx,
                                                     const int32_t* __restrict__ a_rows, int64_t n_rows,
                                                     float* __restrict__ cand_val, int32_t* __restrict__ cand_idx) {
  const int64_t qb = blockIdx.x;
  const int64_t x0 = blk_ptr ? blk_ptr[qb] : qb * n_tiles;
  const int64_t x1 = blk_ptr ? blk_ptr[qb + 1] : x0 + n_tiles;
  const int r = threadIdx.x;
  const int64_t ra = qb * kTM + r;
  if (ra >= n_rows) return;
  const int64_t i = a_rows ? (int64_t)a_rows[ra] : ra;
  constexpr int C = kListC;
  if (x0 == x1) {
    for (int e = 0; e < kCandC; ++e) {
      cand_val[i * kCandC + e] = -INFINITY;
      cand_idx[i * kCandC + e] = -1;
    }
    return;
  }
  const int64_t c0 = ((x0 + 1) * ctas + work - 1) / work - 1;  // the CTA whose range holds x0
  if (range_begin(c0 + 1, work, ctas) >= x1) return;
  for (int h = 0; h < kLists; ++h) {
    float lv[C];
    int32_t li[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      lv[c] = -INFINITY;
      li[c] = -1;
    }
    for (int64_t cc = c0; cc < ctas; ++cc) {
      const int64_t b = range_begin(cc, work, ctas);
      if (b >= x1) break;
      const int64_t slot = (cc * 2 + (b >= x0 ? 0 : 1)) * kTM + r;  // run cc starts inside the block: its first segment
      for (int e = 0; e < C; ++e) {
        const int32_t j = part_idx[slot * kCandC + h * C + e];
        const float v = part_val[slot * kCandC + h * C + e];
        if (j >= 0 && v > lv[C - 1]) sorted_insert<C>(lv, li, v, j);
      }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      cand_val[i * kCandC + h * C + c] = lv[c];
      cand_idx[i * kCandC + h * C + c] = li[c];
    }
  }
}

// pipeline depth and dynamic shared memory for kb_count blocks of A
ancka_status tc_smem(int kb_count, int* nstages, size_t* smem) {
  const size_t fixed = 1024 + (size_t)kb_count * kABytes + sizeof(Bars);
  int ns = (int)((kMaxSmem - fixed) / kBBytes);
  if (ns > kMaxStages) ns = kMaxStages;
  if (ns < 2) {
    set_error("tensor-core contraction: not enough shared memory for two stages");
    return ANCKA_ERR_UNSUPPORTED;
  }
  // at least ~120 KB so that one CTA owns an SM and its 512 TMEM columns
  size_t sm = fixed + (size_t)ns * kBBytes;
  if (sm < 120 * 1024) sm = 120 * 1024;
  *nstages = ns;
  *smem = sm;
  return ANCKA_OK;
}

// ---------------------------------------------------------------------------
// Symmetric contraction (the scores are symmetric: s_ij = s_ji).
//
// Only the pairs j > i are multiplied: the tiles (query block qb, key tile t)
// with t >= qb / 2, in stream-K runs as above.  Every row-half (the keys of
// one column half of the 256-key tiles, the halves of the two lists) has a
// threshold L, the 16th-best score of that row-half over every 8th key tile
// (the list kernel with key_stride 8): at least 16 keys of the full half
// score >= L.  A tile's score s_ij is appended to row i's buffer when s_ij >=
// L_i (row path, half = the key's column half) and to row j's buffer when
// s_ij >= L_j (column path, half = (i mod 256) / 128 = qb & 1, the same for
// the whole CTA); a per-32-key minimum of the column thresholds skips most
// chunks.  k_sym_select then takes each row-half's 16 best, which are the
// lists of a full sweep: a key left out scored below L or below the 16th
// collected score.  A row whose buffer overflowed gets empty lists, which
// the certificate sends to the exact fallback.
// ---------------------------------------------------------------------------
constexpr int kSymStride = 8;  // key tiles of the sampled pass

// first work item of query block qb: sum over q < qb of (n_tiles - q / 2)
__device__ __forceinline__ int64_t sym_start(int64_t qb, int64_t n_tiles) {
  const int64_t a = qb >> 1;
  const int64_t s = (qb & 1) ? a * a : a * (a - 1);
  return qb * n_tiles - s;
}

// the query block holding work item w (binary search over qb)
__device__ __forceinline__ int64_t sym_block(int64_t w, int64_t qblocks, int64_t n_tiles) {
  int64_t lo = 0, hi = qblocks - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (sym_start(mid, n_tiles) <= w) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// The contraction stages (row-half, key, score) entries: each epilogue warp
// reserves blocks of kSymBlock entries with one atomic and fills them without
// waiting on atomics (unused tails are marked -1); k_sym_scatter then appends
// the entries to per-row-half buffers.
constexpr int kSymBlock = 256;

struct SymArgs {
  const float* L;      // 2 x lstride thresholds (half-major); lstride = 256 x key tiles
  const float* Lmin;   // 2 x (lstride / 32) minima over 32 consecutive rows
  int32_t* st_slot;    // staging: row * 2 + half, -1 unused
  int32_t* st_key;
  float* st_val;
  unsigned long long* st_count;  // entries reserved (may exceed st_cap: overflow)
  int64_t st_cap;
};

__device__ __forceinline__ void sym_stage(const SymArgs& sa, int64_t pos, int32_t slot, int32_t key, float v) {
  if (pos < sa.st_cap) {
    sa.st_slot[pos] = slot;
    sa.st_key[pos] = key;
    sa.st_val[pos] = v;
  }
}

__global__ void __launch_bounds__(kThreads, 1)
k_knn_sym(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int64_t n,
          int64_t n_pad, int64_t qblocks, int kb_count, int nstages, SymArgs sa, int* __restrict__ err) {
  constexpr int kTK = 64;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = sA + kb_count * kABytes;
  Bars* bars = reinterpret_cast<Bars*>(sB + nstages * kBBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n_tiles = ceil_div(n_pad, kTN);
  const int64_t work = sym_start(qblocks, n_tiles);
  const int64_t w_begin = range_begin(blockIdx.x, work, gridDim.x);
  const int64_t w_end = range_begin((int64_t)blockIdx.x + 1, work, gridDim.x);
  volatile int* abort = &bars->abort;
  if (threadIdx.x == 0) {
    for (int s = 0; s < nstages; ++s) {
      mbar_init(&bars->full[s], 1);
      mbar_init(&bars->empty[s], 1);
    }
    mbar_init(&bars->a_full, 1);
    mbar_init(&bars->a_empty, 1);
    mbar_init(&bars->tfull[0], 1);
    mbar_init(&bars->tfull[1], 1);
    mbar_init(&bars->tempty[0], kEpiWarps);
    mbar_init(&bars->tempty[1], kEpiWarps);
    mbar_init(&bars->drain, 1);
    bars->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&bars->tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;
  // segment of a run: (qb, t0, t1) with t in [qb / 2, n_tiles)
  auto segment = [&](int64_t w, int64_t& qb, int64_t& t0, int64_t& t1) {
    qb = sym_block(w, qblocks, n_tiles);
    t0 = (qb >> 1) + (w - sym_start(qb, n_tiles));
    t1 = w_end - w < n_tiles - t0 ? t0 + (w_end - w) : n_tiles;
  };

  if (warp == 0) {
    if (lane == 0) {
      bool pending[kMaxStages];
      uint32_t pend_par[kMaxStages];
      for (int s = 0; s < kMaxStages; ++s) pending[s] = false;
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int seg = 0;
      for (int64_t w = w_begin; w < w_end && ok; ++seg) {
        int64_t qb, t0, t1;
        segment(w, qb, t0, t1);
        w += t1 - t0;
        if (seg > 0 && !mbar_wait(&bars->a_empty, (uint32_t)((seg - 1) & 1), abort, err, 6)) {
          ok = false;
          break;
        }
        mbar_expect_tx(&bars->a_full, (uint32_t)(kb_count * kABytes));
        for (int kb = 0; kb < kb_count; ++kb)
          tma_load_2d(smem_u32(sA + kb * kABytes), &tmA, kb * kTK, (int)(qb * kTM), &bars->a_full);
        for (int64_t t = t0; t < t1 && ok; ++t) {
          for (int kb = 0; kb < kb_count; ++kb) {
            if (!mbar_wait(&bars->empty[stage], phase ^ 1, abort, err, 1)) {
              ok = false;
              break;
            }
            pending[stage] = false;
            mbar_expect_tx(&bars->full[stage], (uint32_t)kBBytes);
            tma_load_2d(smem_u32(sB + stage * kBBytes), &tmB, kb * kTK, (int)(t * kTN), &bars->full[stage]);
            pending[stage] = true;
            pend_par[stage] = phase;
            if (++stage == nstages) {
              stage = 0;
              phase ^= 1;
            }
          }
        }
      }
      if (!ok) {
        if (seg > 0) mbar_wait(&bars->a_full, (uint32_t)((seg - 1) & 1), nullptr, nullptr, 0);
        for (int s = 0; s < nstages; ++s)
          if (pending[s]) mbar_wait(&bars->full[s], pend_par[s], nullptr, nullptr, 0);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      int stage = 0;
      uint32_t phase = 0;
      bool issued = false;
      int64_t g = 0;
      int seg = 0;
      for (int64_t w = w_begin; w < w_end && ok; ++seg) {
        int64_t qb, t0, t1;
        segment(w, qb, t0, t1);
        w += t1 - t0;
        if (!mbar_wait(&bars->a_full, (uint32_t)(seg & 1), abort, err, 2)) {
          ok = false;
          break;
        }
        for (int64_t t = t0; t < t1; ++t, ++g) {
          const int b = (int)(g & 1);
          const uint32_t use = (uint32_t)(g >> 1);
          if (!mbar_wait(&bars->tempty[b], (use & 1) ^ 1, abort, err, 3)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(b * kTN);
          for (int kb = 0; kb < kb_count; ++kb) {
            if (!mbar_wait(&bars->full[stage], phase, abort, err, 4)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA + kb * kABytes);
            const uint32_t b0 = smem_u32(sB + stage * kBBytes);
#pragma unroll
            for (int kk = 0; kk < kMmaPerStage; ++kk)
              umma_bf16(d, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), (kb | kk) != 0 ? 1u : 0u);
            issued = true;
            umma_commit(&bars->empty[stage]);
            if (++stage == nstages) {
              stage = 0;
              phase ^= 1;
            }
          }
          if (!ok) break;
          umma_commit(&bars->tfull[b]);
        }
        if (ok) umma_commit(&bars->a_empty);
      }
      if (!ok && issued) {
        umma_commit(&bars->drain);
        mbar_wait(&bars->drain, 0, nullptr, nullptr, 0);
      }
    }
  } else {
    const int ew = warp - 2;
    const int q = warp & 3;
    const int h = ew >> 2;  // column half of the tile = the row path's list half
    const int r = q * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
    int64_t g = 0;
    bool ok = true;
    int64_t blk_base = 0;  // the warp's staging block (uniform over the warp)
    int blk_cap = 0, blk_used = 0;
    for (int64_t w = w_begin; w < w_end && ok;) {
      int64_t qb, t0, t1;
      segment(w, qb, t0, t1);
      w += t1 - t0;
      const int64_t i = qb * kTM + r;
      const int64_t lstride = n_tiles * kTN;
      const float Lrow = i < n ? sa.L[(int64_t)h * lstride + i] : INFINITY;
      const int hc = (int)(qb & 1);  // the column path's list half
      const float* Lc = sa.L + (int64_t)hc * lstride;
      const float* Lm = sa.Lmin + (int64_t)hc * (lstride / 32);
      for (int64_t t = t0; t < t1; ++t, ++g) {
        const int b = (int)(g & 1);
        const uint32_t use = (uint32_t)(g >> 1);
        const int64_t jb = t * kTN + h * kSliceN;
        // the tile's column thresholds (lane: keys jb + 4 lane .. + 3) and
        // per-chunk minima, loaded before the wait so that their latency hides
        const float4 lcol = *reinterpret_cast<const float4*>(Lc + jb + 4 * lane);
        const float4 lmin4 = *reinterpret_cast<const float4*>(Lm + (jb >> 5));
        const bool got = mbar_wait(&bars->tfull[b], use & 1, abort, err, 5);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t tb = lane_base + (uint32_t)(b * kTN + h * kSliceN);
#pragma unroll 1
        for (int c = 0; c < kSliceN / 32; ++c) {
          uint32_t rv[32];
          tmem_ld32_issue(tb + (uint32_t)(c * 32), rv);
          tmem_wait();
          pin(rv);
          const int64_t j0 = jb + c * 32;
          // keys j0 + e with i < j < n
          const int64_t lo = i + 1 - j0, hi = n - j0;
          const int e0 = lo < 0 ? 0 : (lo > 32 ? 32 : (int)lo);
          const int e1 = hi < 0 ? 0 : (hi > 32 ? 32 : (int)hi);
          uint32_t vm = 0;
          if (e1 > e0) vm = (e1 - e0 == 32 ? 0xffffffffu : ((1u << (e1 - e0)) - 1u)) << e0;
          float m[16];
#pragma unroll
          for (int u = 0; u < 16; ++u) m[u] = fmaxf(__uint_as_float(rv[u]), __uint_as_float(rv[u + 16]));
#pragma unroll
          for (int u2 = 8; u2 >= 1; u2 >>= 1)
#pragma unroll
            for (int u = 0; u < u2; ++u) m[u] = fmaxf(m[u], m[u + u2]);
          const float mx = vm ? m[0] : -INFINITY;
          uint32_t pr = 0, pc = 0;
          if (__any_sync(0xffffffffu, mx >= Lrow)) {  // row path
#pragma unroll
            for (int e = 0; e < 32; ++e) pr |= (__uint_as_float(rv[e]) >= Lrow ? 1u : 0u) << e;
            pr &= vm;
          }
          const float lmin = c == 0 ? lmin4.x : c == 1 ? lmin4.y : c == 2 ? lmin4.z : lmin4.w;
          if (__any_sync(0xffffffffu, mx >= lmin)) {  // column path
#pragma unroll
            for (int e4 = 0; e4 < 8; ++e4) {  // chunk c's thresholds sit in lanes 8c .. 8c + 7
              const int src = c * 8 + e4;
              const float t0v = __shfl_sync(0xffffffffu, lcol.x, src);
              const float t1v = __shfl_sync(0xffffffffu, lcol.y, src);
              const float t2v = __shfl_sync(0xffffffffu, lcol.z, src);
              const float t3v = __shfl_sync(0xffffffffu, lcol.w, src);
              pc |= (__uint_as_float(rv[4 * e4]) >= t0v ? 1u : 0u) << (4 * e4);
              pc |= (__uint_as_float(rv[4 * e4 + 1]) >= t1v ? 1u : 0u) << (4 * e4 + 1);
              pc |= (__uint_as_float(rv[4 * e4 + 2]) >= t2v ? 1u : 0u) << (4 * e4 + 2);
              pc |= (__uint_as_float(rv[4 * e4 + 3]) >= t3v ? 1u : 0u) << (4 * e4 + 3);
            }
            pc &= vm;
          }
          // the warp's entries: one exclusive prefix, one block reservation when needed
          const int cl = __popc(pr) + __popc(pc);
          int incl = cl;
#pragma unroll
          for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
          }
          const int ctot = __shfl_sync(0xffffffffu, incl, 31);
          if (ctot > 0) {
            if (blk_used + ctot > blk_cap) {
              for (int e = blk_used + lane; e < blk_cap; e += 32) sym_stage(sa, blk_base + e, -1, -1, 0.f);
              const int nblk = (ctot + kSymBlock - 1) / kSymBlock;
              unsigned long long b = 0;
              if (lane == 0) b = atomicAdd(sa.st_count, (unsigned long long)nblk * kSymBlock);
              blk_base = (int64_t)__shfl_sync(0xffffffffu, b, 0);
              blk_cap = nblk * kSymBlock;
              blk_used = 0;
            }
            int64_t pos = blk_base + blk_used + (incl - cl);
            while (pr) {
              const int e = __ffs(pr) - 1;
              pr &= pr - 1;
              sym_stage(sa, pos++, (int32_t)(i * 2 + h), (int32_t)(j0 + e), pick32(rv, e));
            }
            while (pc) {
              const int e = __ffs(pc) - 1;
              pc &= pc - 1;
              sym_stage(sa, pos++, (int32_t)((j0 + e) * 2 + hc), (int32_t)i, pick32(rv, e));
            }
            blk_used += ctot;
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars->tempty[b]);
      }
    }
    for (int e = blk_used + lane; e < blk_cap; e += 32) sym_stage(sa, blk_base + e, -1, -1, 0.f);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// the staged entries into per-row-half buffers (cnt counts past cap); a
// staging overflow marks every row (overflow flag), so that all go to the
// exact fallback
__global__ void k_sym_scatter(const int32_t* __restrict__ st_slot, const int32_t* __restrict__ st_key,
                              const float* __restrict__ st_val, const unsigned long long* __restrict__ st_count,
                              int64_t st_cap, int32_t* __restrict__ cnt, float* __restrict__ bufv,
                              int32_t* __restrict__ bufi, int cap, int32_t* __restrict__ overflow) {
  const unsigned long long tot = *st_count;
  if (tot > (unsigned long long)st_cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *overflow = 1;
    return;
  }
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)tot;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t slot = st_slot[q];
    if (slot < 0) continue;
    const int pos = atomicAdd(&cnt[slot], 1);
    if (pos < cap) {
      bufv[(int64_t)slot * cap + pos] = st_val[q];
      bufi[(int64_t)slot * cap + pos] = st_key[q];
    }
  }
}

// thresholds from the sampled lists: L[h][i] = the 16th score of row i's
// half-h list (sorted descending), -inf if that list is not full; rows >= n
// +inf; Lmin[h][g] = min over rows 32g .. 32g + 31 (lstride a multiple of 256)
__global__ void k_sym_thresholds(const float* __restrict__ cand_val, const int32_t* __restrict__ cand_idx,
                                 int64_t n, int64_t lstride, float* __restrict__ L, float* __restrict__ Lmin) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= lstride) return;
  const int64_t n_pad = lstride;
  for (int h = 0; h < 2; ++h) {
    float v = INFINITY;
    if (i < n) {
      const int64_t last = i * kCandC + h * kListC + (kListC - 1);
      v = cand_idx[last] >= 0 ? cand_val[last] : -INFINITY;
    }
    L[(int64_t)h * n_pad + i] = v;
    float mn = v;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, off));
    if ((threadIdx.x & 31) == 0) Lmin[(int64_t)h * (n_pad / 32) + (i >> 5)] = mn;
  }
}

// each row's two lists: the 16 best collected entries per half, sorted
// descending; a row with an overflowing half gets two empty lists (sent to
// the exact fallback by the certificate)
__global__ void k_sym_select(const int32_t* __restrict__ cnt, const float* __restrict__ bufv,
                             const int32_t* __restrict__ bufi, int cap, int64_t n,
                             const int32_t* __restrict__ overflow, float* __restrict__ cand_val,
                             int32_t* __restrict__ cand_idx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool over = *overflow || cnt[i * 2] > cap || cnt[i * 2 + 1] > cap;
  constexpr int C = kListC;
  for (int h = 0; h < 2; ++h) {
    float lv[C];
    int32_t li[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      lv[c] = -INFINITY;
      li[c] = -1;
    }
    if (!over) {
      const int64_t slot = i * 2 + h;
      const int c_n = cnt[slot];
      for (int e = 0; e < c_n; ++e) {
        const float v = bufv[slot * cap + e];
        if (v > lv[C - 1]) sorted_insert<C>(lv, li, v, bufi[slot * cap + e]);
      }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      cand_val[i * kCandC + h * C + c] = lv[c];
      cand_idx[i * kCandC + h * C + c] = li[c];
    }
  }
}

__global__ void k_gather_rows(const uint8_t* __restrict__ x, int row_bytes, const int32_t* __restrict__ rows,
                              int64_t n_a, int64_t n_a_pad, uint8_t* __restrict__ out) {
  const int64_t r = blockIdx.x;
  if (r >= n_a_pad) return;
  const uint4* src = r < n_a ? reinterpret_cast<const uint4*>(x + (int64_t)rows[r] * row_bytes) : nullptr;
  uint4* dst = reinterpret_cast<uint4*>(out + r * row_bytes);
  for (int c = threadIdx.x; c < row_bytes / 16; c += blockDim.x) dst[c] = src ? src[c] : make_uint4(0, 0, 0, 0);
}

// One persistent CTA per SM (at most one per work item); list mode adds the
// partial-list area and the merge of split query blocks.
template <bool kCollect, bool kE4M3>
ancka_status launch_tc(Workspace& ws, const CUtensorMap& ta, const CUtensorMap& tb, int64_t n, int64_t n_pad,
                       int64_t n_rows, int kb_count, int d, float* cand_val, int32_t* cand_idx,
                       const float* out_scale, const CollectArgs& ca, int32_t* err, cudaStream_t s,
                       int key_stride = 1) {
  // MMAs over the last 128-byte feature block: K = 16 features (BF16) or 32
  // (E4M3) each; the padding past d is zero and needs none
  const int per_kb = kE4M3 ? 128 : 64, per_mma = kE4M3 ? 32 : 16;
  const int rem = d - per_kb * (kb_count - 1);
  const int k_last = (rem >= 1 && rem <= per_kb) ? (int)ceil_div(rem, per_mma) : kMmaPerStage;
  int nstages;
  size_t smem;
  ANCKA_TRY(tc_smem(kb_count, &nstages, &smem));
  int sms = 152, dev = 0;
  ANCKA_CUDA(cudaGetDevice(&dev));
  ANCKA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t qblocks = ceil_div(n_rows, kTM);
  const int n_tiles = (int)ceil_div(ceil_div(n_pad, kTN), key_stride);
  const int64_t work = ca.blk_ptr ? ca.blk_work : qblocks * n_tiles;
  const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(sms, work));
  float* part_val = nullptr;
  int32_t* part_idx = nullptr;
  if (!kCollect) {
    ANCKA_TRY(ws.alloc(&part_val, (size_t)ctas * 2 * kTM * kCandC));
    ANCKA_TRY(ws.alloc(&part_idx, (size_t)ctas * 2 * kTM * kCandC));
  }
  unsigned long long* tick = nullptr;  // tiles issued by all CTAs (re-aligns whole blocks' key order)
  // (not for tile lists or foreign keys, whose callers want the same lists
  // on every call: a key order that moves with timing resolves exact score
  // ties differently)
  if (key_stride == 1 && !ca.blk_ptr && !ca.no_self) ANCKA_TRY(ws.zeros(&tick, 1));
  ANCKA_CUDA(cudaFuncSetAttribute(k_knn_tc<kCollect, kE4M3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_knn_tc<kCollect, kE4M3><<<(unsigned)ctas, kThreads, smem, s>>>(ta, tb, n, n_pad, qblocks, kb_count, k_last,
                                                                   nstages, key_stride, cand_val, cand_idx,
                                                                   out_scale, part_val, part_idx, ca, tick, err);
  ANCKA_LAUNCHED();
  if (!kCollect) {
    k_merge_lists<<<(unsigned)qblocks, kTM, 0, s>>>(n_tiles, work, ctas, ca.blk_ptr, part_val, part_idx, ca.a_rows,
                                                    n_rows, cand_val, cand_idx);
    ANCKA_LAUNCHED();
  }
  return ANCKA_OK;
}

int64_t sym_start_host(int64_t qb, int64_t n_tiles) {
  const int64_t a = qb >> 1;
  return qb * n_tiles - ((qb & 1) ? a * a : a * (a - 1));
}

// off by default: on the measured workloads the symmetric form is slower than
// the full sweep (its fixed thresholds admit ~8x more candidates than the
// full sweep's running ones, so its epilogue does about twice the work per
// tile over half the tiles)
std::atomic<int64_t> g_sym_min_rows{INT64_MAX};

// BF16 lists by the symmetric contraction (sampled thresholds, the j > i
// tiles with both paths, selection)
ancka_status knn_candidates_bf16_sym(Workspace& ws, const PrepOut& pr, int64_t n, const CUtensorMap& ta,
                                     const CUtensorMap& tb, int kb_count, float* cand_val, int32_t* cand_idx,
                                     int32_t* err, cudaStream_t s) {
  // 1. sampled lists: every kSymStride-th key tile
  float* sv;
  int32_t* si;
  ANCKA_TRY(ws.alloc(&sv, (size_t)n * kCandC));
  ANCKA_TRY(ws.alloc(&si, (size_t)n * kCandC));
  CollectArgs none{};
  const ancka_status st = launch_tc<false, false>(ws, ta, tb, n, pr.n_pad, n, kb_count, pr.d, sv, si, nullptr, none,
                                                  err, s, kSymStride);
  if (st != ANCKA_OK) return st;
  // 2. thresholds
  const int64_t n_tiles = ceil_div(pr.n_pad, kTN);
  const int64_t lstride = n_tiles * kTN;
  float *L, *Lmin;
  ANCKA_TRY(ws.alloc(&L, (size_t)2 * lstride));
  ANCKA_TRY(ws.alloc(&Lmin, (size_t)2 * (lstride / 32)));
  k_sym_thresholds<<<(unsigned)(lstride / 256), 256, 0, s>>>(sv, si, n, lstride, L, Lmin);
  ANCKA_LAUNCHED();
  // 3. the j > i tiles, both paths
  constexpr int kCap = 320;  // ~16 x kSymStride entries expected per row-half
  SymArgs sa{L, Lmin, nullptr, nullptr, nullptr, nullptr, 0};
  sa.st_cap = n * 2 * 16 * kSymStride * 5 / 2 + (int64_t)8 * kThreads / 32 * kSymBlock * 152;
  ANCKA_TRY(ws.alloc(&sa.st_slot, (size_t)sa.st_cap));
  ANCKA_TRY(ws.alloc(&sa.st_key, (size_t)sa.st_cap));
  ANCKA_TRY(ws.alloc(&sa.st_val, (size_t)sa.st_cap));
  ANCKA_TRY(ws.zeros(&sa.st_count, 1));
  int32_t *cnt, *bufi, *overflow;
  float* bufv;
  ANCKA_TRY(ws.zeros(&cnt, (size_t)n * 2));
  ANCKA_TRY(ws.alloc(&bufv, (size_t)n * 2 * kCap));
  ANCKA_TRY(ws.alloc(&bufi, (size_t)n * 2 * kCap));
  ANCKA_TRY(ws.zeros(&overflow, 1));
  int nstages;
  size_t smem;
  ANCKA_TRY(tc_smem(kb_count, &nstages, &smem));
  int sms = 152, dev = 0;
  ANCKA_CUDA(cudaGetDevice(&dev));
  ANCKA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t qblocks = ceil_div(n, kTM);
  const int64_t work = sym_start_host(qblocks, n_tiles);
  const int64_t ctas = std::min<int64_t>(sms, work);
  ANCKA_CUDA(cudaFuncSetAttribute(k_knn_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_knn_sym<<<(unsigned)ctas, kThreads, smem, s>>>(ta, tb, n, pr.n_pad, qblocks, kb_count, nstages, sa, err);
  ANCKA_LAUNCHED();
  // 4. staged entries into the row-half buffers, then the two lists of every row
  k_sym_scatter<<<(unsigned)(4 * sms), 256, 0, s>>>(sa.st_slot, sa.st_key, sa.st_val, sa.st_count, sa.st_cap, cnt,
                                                   bufv, bufi, kCap, overflow);
  ANCKA_LAUNCHED();
  k_sym_select<<<(unsigned)ceil_div(n, 128), 128, 0, s>>>(cnt, bufv, bufi, kCap, n, overflow, cand_val, cand_idx);
  ANCKA_LAUNCHED();
  return ANCKA_OK;
}

}  // namespace

bool knn_tc_available() { return true; }

int knn_tc_max_dp() { return 512; }

ancka_status knn_candidates_bf16(Workspace& ws, const PrepOut& pr, int64_t n, float* cand_val, int32_t* cand_idx,
                                 int32_t* err, cudaStream_t s) {
  const int kb_count = pr.dp / 64;
  if (pr.dp % 64 != 0 || kb_count < 1 || pr.dp > knn_tc_max_dp()) {
    set_error("BF16 contraction supports up to %d features (got %d)", knn_tc_max_dp(), pr.dp);
    return ANCKA_ERR_UNSUPPORTED;
  }
  CUtensorMap ta, tb;
  ANCKA_TRY(make_map(&ta, pr.xb, pr.dp, pr.n_pad, kTM, 2));
  ANCKA_TRY(make_map(&tb, pr.xb, pr.dp, pr.n_pad, kTN, 2));
  if (n >= g_sym_min_rows.load(std::memory_order_relaxed))
    return knn_candidates_bf16_sym(ws, pr, n, ta, tb, kb_count, cand_val, cand_idx, err, s);
  CollectArgs none{};
  return launch_tc<false, false>(ws, ta, tb, n, pr.n_pad, n, kb_count, pr.d, cand_val, cand_idx, nullptr, none, err,
                                 s);
}

void knn_set_symmetric_min_rows(int64_t n_min) { g_sym_min_rows.store(n_min, std::memory_order_relaxed); }

ancka_status knn_candidates_fp8(Workspace& ws, const PrepOut& pr, int64_t n, float* cand_val, int32_t* cand_idx,
                                int32_t* err, cudaStream_t s) {
  const int kb_count = pr.dp8 / 128;
  if (!pr.x8 || pr.dp8 % 128 != 0 || kb_count < 1 || pr.dp8 > knn_tc_max_dp_fp8()) {
    set_error("FP8 contraction supports up to %d features (got %d)", knn_tc_max_dp_fp8(), pr.dp8);
    return ANCKA_ERR_UNSUPPORTED;
  }
  CUtensorMap ta, tb;
  ANCKA_TRY(make_map(&ta, pr.x8, pr.dp8, pr.n_pad, kTM, 1));
  ANCKA_TRY(make_map(&tb, pr.x8, pr.dp8, pr.n_pad, kTN, 1));
  CollectArgs none{};
  return launch_tc<false, true>(ws, ta, tb, n, pr.n_pad, n, kb_count, pr.d, cand_val, cand_idx, pr.inv_s2, none, err,
                                s);
}

int knn_tc_max_dp_fp8() { return 1024; }

// BF16 lists for the n_a rows listed in rows (written at their global rows)
ancka_status knn_list_gathered_bf16(Workspace& ws, const PrepOut& pr, int64_t n, const int32_t* rows, int64_t n_a,
                                    float* cand_val, int32_t* cand_idx, int32_t* err, cudaStream_t s) {
  const int kb_count = pr.dp / 64;
  const int64_t n_a_pad = round_up(n_a, kTM);
  __nv_bfloat16* af;
  ANCKA_TRY(ws.alloc(&af, (size_t)n_a_pad * pr.dp));
  k_gather_rows<<<(unsigned)n_a_pad, 64, 0, s>>>(reinterpret_cast<const uint8_t*>(pr.xb), pr.dp * 2, rows, n_a,
                                                 n_a_pad, reinterpret_cast<uint8_t*>(af));
  ANCKA_LAUNCHED();
  CUtensorMap ta, tb;
  ANCKA_TRY(make_map(&ta, af, pr.dp, n_a_pad, kTM, 2));
  ANCKA_TRY(make_map(&tb, pr.xb, pr.dp, pr.n_pad, kTN, 2));
  CollectArgs ca{rows, n_a, nullptr, nullptr, nullptr, 0};
  return launch_tc<false, false>(ws, ta, tb, n, pr.n_pad, n_a, kb_count, pr.d, cand_val, cand_idx, nullptr, ca, err,
                                 s);
}

ancka_status knn_lists_bf16(Workspace& ws, const __nv_bfloat16* a, int64_t a_rows_total, const int32_t* rows,
                           int64_t n_rows, const __nv_bfloat16* keys, int64_t n_keys, int64_t keys_pad, int dp, int d,
                           const int64_t* blk_ptr, const int32_t* blk_tiles, int64_t blk_work, bool no_self,
                           float* cand_val, int32_t* cand_idx, int32_t* err, cudaStream_t s) {
  const int kb_count = dp / 64;
  if (dp % 64 != 0 || kb_count < 1 || dp > knn_tc_max_dp()) {
    set_error("BF16 contraction supports up to %d features (got %d)", knn_tc_max_dp(), dp);
    return ANCKA_ERR_UNSUPPORTED;
  }
  CUtensorMap ta, tb;
  if (rows) {
    const int64_t n_a_pad = round_up(n_rows, kTM);
    __nv_bfloat16* af;
    ANCKA_TRY(ws.alloc(&af, (size_t)n_a_pad * dp));
    k_gather_rows<<<(unsigned)n_a_pad, 64, 0, s>>>(reinterpret_cast<const uint8_t*>(a), dp * 2, rows, n_rows,
                                                   n_a_pad, reinterpret_cast<uint8_t*>(af));
    ANCKA_LAUNCHED();
    ANCKA_TRY(make_map(&ta, af, dp, n_a_pad, kTM, 2));
  } else {
    ANCKA_TRY(make_map(&ta, a, dp, round_up(a_rows_total, kTM), kTM, 2));
  }
  ANCKA_TRY(make_map(&tb, keys, dp, keys_pad, kTN, 2));
  CollectArgs ca{rows, n_rows, nullptr, nullptr, nullptr, 0};
  ca.blk_ptr = blk_ptr;
  ca.blk_tiles = blk_tiles;
  ca.blk_work = blk_work;
  ca.no_self = no_self ? 1 : 0;
  return launch_tc<false, false>(ws, ta, tb, n_keys, keys_pad, n_rows, kb_count, d, cand_val, cand_idx, nullptr, ca,
                                 err, s);
}

ancka_status knn_collect_bf16(Workspace& ws, const PrepOut& pr, int64_t n, const int32_t* rows, int64_t n_a,
                              const float* thr, int32_t* cnt, int32_t* buf, int cap, int32_t* err, cudaStream_t s) {
  const int kb_count = pr.dp / 64;
  const int64_t n_a_pad = round_up(n_a, kTM);
  __nv_bfloat16* af;
  ANCKA_TRY(ws.alloc(&af, (size_t)n_a_pad * pr.dp));
  k_gather_rows<<<(unsigned)n_a_pad, 64, 0, s>>>(reinterpret_cast<const uint8_t*>(pr.xb), pr.dp * 2, rows, n_a,
                                                 n_a_pad, reinterpret_cast<uint8_t*>(af));
  ANCKA_LAUNCHED();
  CUtensorMap ta, tb;
  ANCKA_TRY(make_map(&ta, af, pr.dp, n_a_pad, kTM, 2));
  ANCKA_TRY(make_map(&tb, pr.xb, pr.dp, pr.n_pad, kTN, 2));
  CollectArgs ca{rows, n_a, thr, cnt, buf, cap};
  return launch_tc<true, false>(ws, ta, tb, n, pr.n_pad, n_a, kb_count, pr.d, nullptr, nullptr, nullptr, ca, err, s);
}

}  // namespace ancka
