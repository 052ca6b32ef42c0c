// tcgen05 BF16 / FP8-e4m3 candidate search for the cosine KNN of Section 3.1.
//
// One CTA per 128 query rows sweeps every 256-row key tile:
//   warp 0     TMA producer: the CTA's query block A (128 x dp, 128-byte
//              swizzle) once, then key tiles B (256 rows x 128 bytes of
//              features per stage: 64 BF16 or 128 FP8) through an
//              nstages-deep ring (mbarrier full/empty);
//   warp 1     MMA issuer: allocates 512 TMEM columns, issues
//              tcgen05.mma.cta_group::1.kind::f16 (BF16, K=16) or
//              kind::f8f6f4 (E4M3, K=32) with M=128, N=256 into two
//              ping-pong FP32 accumulators, commits stage releases and
//              accumulator-ready signals;
//   warps 2-9  epilogue: two warps per TMEM lane quarter, each owning half of
//              every tile's 256 columns; tcgen05.ld (32x32b) of the thread's
//              accumulator row (TMEM lane = query row), threshold test and
//              insert into a register-resident list of its 16 best scores.
//              Row i thus leaves two 16-entry lists (one per column half),
//              kCandC = 32 candidates in total.
// The MMA of tile t+1 overlaps the epilogue of tile t.  n x n scores never
// leave the SM.  Every mbarrier wait is bounded: on expiry the kernel records
// an error code, stops all roles, drains its own copies and MMAs (bounded),
// frees TMEM and returns.
#include <algorithm>

#include "tc_common.cuh"

namespace ancka {

namespace {

constexpr int kTM = 128;                 // query rows per CTA = TMEM lanes
constexpr int kTN = 256;                 // key rows per tile = accumulator columns
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kListC = kCandC / 2;     // per-thread list (two per row)
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
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
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
// Fold one 32-key chunk (scores in r, keys j0..j0+31) into the row's list.
template <int C>
__device__ __forceinline__ void fold_chunk(const uint32_t (&r)[32], int64_t j0, int64_t n, int64_t i,
                                           float (&lv)[C], int32_t (&li)[C], float& thr, int& mp) {
  // skip the chunk when no lane of the warp has a key above its threshold
  float mx = __uint_as_float(r[0]);
#pragma unroll
  for (int e = 1; e < 32; ++e) mx = fmaxf(mx, __uint_as_float(r[e]));
  if (!__any_sync(0xffffffffu, mx > thr)) return;
  // pass mask against the threshold at chunk start (it only rises, so the
  // mask is a superset); padding keys and the row itself removed
  uint32_t pm = 0;
#pragma unroll
  for (int e = 0; e < 32; ++e) pm |= (__uint_as_float(r[e]) > thr ? 1u : 0u) << e;
  if (j0 + 32 > n) pm &= (j0 >= n) ? 0u : ((1u << (uint32_t)(n - j0)) - 1u);
  if (i >= j0 && i < j0 + 32) pm &= ~(1u << (uint32_t)(i - j0));
  // one insert per passing key; lanes without keys idle
  while (__any_sync(0xffffffffu, pm != 0)) {
    if (pm) {
      const int e = __ffs(pm) - 1;
      pm &= pm - 1;
      float val = __uint_as_float(r[0]);
#pragma unroll
      for (int q = 1; q < 32; ++q)
        if (e == q) val = __uint_as_float(r[q]);
      if (val > thr) list_insert<C>(lv, li, thr, mp, val, (int32_t)(j0 + e));
    }
  }
}

// Collect mode: append every key whose score reaches the row's fixed
// threshold t to the row's buffer (cap entries; the counter keeps counting
// past cap so the caller can see an overflow).
__device__ __forceinline__ void collect_chunk(const uint32_t (&r)[32], int64_t j0, int64_t n, int64_t i, float t,
                                              int64_t ra, int32_t* __restrict__ cnt, int32_t* __restrict__ buf,
                                              int cap) {
  float mx = __uint_as_float(r[0]);
#pragma unroll
  for (int e = 1; e < 32; ++e) mx = fmaxf(mx, __uint_as_float(r[e]));
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
  int64_t n_a;            // compact query rows
  const float* thr;       // collect mode: per compact row threshold
  int32_t* cnt;           // collect mode: per compact row counter
  int32_t* buf;           // collect mode: n_a x cap keys
  int cap;
};

// kCollect: collect mode (keys above a per-row threshold) instead of list
// mode (two 16-entry lists per row); kE4M3: FP8 operands.  out_scale (list
// mode, may be null) multiplies the scores written out.
template <bool kCollect, bool kE4M3>
__global__ void __launch_bounds__(kThreads, 1)
k_knn_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int64_t n,
         int64_t n_pad, int kb_count, int nstages, int tps, float* __restrict__ cand_val,
         int32_t* __restrict__ cand_idx, const float* __restrict__ out_scale, CollectArgs ca,
         int* __restrict__ err) {
  constexpr int kTK = kE4M3 ? 128 : 64;  // features per stage
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = sA + kb_count * kABytes;
  Bars* bars = reinterpret_cast<Bars*>(sB + nstages * kBBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ib = (int64_t)blockIdx.x * kTM;
  // this CTA's key tiles: [t_begin, t_begin + ntiles) (collect mode splits
  // the sweep over blockIdx.y; list mode sweeps all keys)
  const int all_tiles = (int)ceil_div(n_pad, kTN);
  const int t_begin = (int)blockIdx.y * tps;
  const int ntiles = max(0, min(all_tiles, t_begin + tps) - t_begin);
  volatile int* abort = &bars->abort;

  if (threadIdx.x == 0) {
    for (int s = 0; s < nstages; ++s) {
      mbar_init(&bars->full[s], 1);
      mbar_init(&bars->empty[s], 1);
    }
    mbar_init(&bars->a_full, 1);
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
      mbar_expect_tx(&bars->a_full, (uint32_t)(kb_count * kABytes));
      for (int kb = 0; kb < kb_count; ++kb)
        tma_load_2d(smem_u32(sA + kb * kABytes), &tmA, kb * kTK, (int)ib, &bars->a_full);
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int t = 0; t < ntiles && ok; ++t) {
        for (int kb = 0; kb < kb_count; ++kb) {
          if (!mbar_wait(&bars->empty[stage], phase ^ 1, abort, err, 1)) {
            ok = false;
            break;
          }
          pending[stage] = false;
          mbar_expect_tx(&bars->full[stage], (uint32_t)kBBytes);
          tma_load_2d(smem_u32(sB + stage * kBBytes), &tmB, kb * kTK, (t_begin + t) * kTN, &bars->full[stage]);
          pending[stage] = true;
          pend_par[stage] = phase;
          if (++stage == nstages) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      if (!ok) {  // drain this warp's copies still in flight (bounded)
        mbar_wait(&bars->a_full, 0, nullptr, nullptr, 0);
        for (int s = 0; s < nstages; ++s)
          if (pending[s]) mbar_wait(&bars->full[s], pend_par[s], nullptr, nullptr, 0);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = mbar_wait(&bars->a_full, 0, abort, err, 2);
      int stage = 0;
      uint32_t phase = 0;
      bool issued = false;
      for (int t = 0; t < ntiles && ok; ++t) {
        const int b = t & 1;
        const uint32_t use = (uint32_t)(t >> 1);
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
          for (int kk = 0; kk < kMmaPerStage; ++kk) {
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
      if (!ok && issued) {  // wait for this thread's MMAs before TMEM is freed (bounded)
        umma_commit(&bars->drain);
        mbar_wait(&bars->drain, 0, nullptr, nullptr, 0);
      }
    }
  } else {
    const int ew = warp - 2;   // epilogue warp 0..7
    const int q = warp & 3;    // TMEM lane quarter this warp may access
    const int h = ew >> 2;     // column half of every tile
    const int r = q * 32 + lane;
    // A row ra is query row ra, or compact row ra -> global row a_rows[ra]
    const int64_t ra = ib + r;
    const bool row_ok = ca.a_rows ? (ra < ca.n_a) : (ra < n);
    const int64_t i = ca.a_rows ? (row_ok ? (int64_t)ca.a_rows[ra] : -1) : ra;
    const float t_row = kCollect && row_ok ? ca.thr[ra] : INFINITY;
    constexpr int C = kListC;
    float lv[C];
    int32_t li[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      lv[c] = -INFINITY;
      li[c] = -1;
    }
    float thr = -INFINITY;
    int mp = 0;
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
    for (int t = 0; t < ntiles; ++t) {
      const int b = t & 1;
      const uint32_t use = (uint32_t)(t >> 1);
      bool ok = mbar_wait(&bars->tfull[b], use & 1, abort, err, 5);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      const int64_t jb = (int64_t)(t_begin + t) * kTN + h * (kTN / 2);
      const uint32_t tb = lane_base + (uint32_t)(b * kTN + h * (kTN / 2));
#pragma unroll 1
      for (int c = 0; c < kTN / 64; ++c) {
        uint32_t rv[32];
        tmem_ld32_issue(tb + (uint32_t)(c * 32), rv);
        tmem_wait();
        pin(rv);
        if constexpr (kCollect) {
          collect_chunk(rv, jb + c * 32, n, i, t_row, ra, ca.cnt, ca.buf, ca.cap);
        } else {
          fold_chunk<C>(rv, jb + c * 32, n, i, lv, li, thr, mp);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars->tempty[b]);
    }
    if (!kCollect && row_ok) {
      const float sc = out_scale ? *out_scale : 1.f;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        cand_val[i * kCandC + h * C + c] = lv[c] * sc;
        cand_idx[i * kCandC + h * C + c] = li[c];
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

__global__ void k_gather_rows(const uint8_t* __restrict__ x, int row_bytes, const int32_t* __restrict__ rows,
                              int64_t n_a, int64_t n_a_pad, uint8_t* __restrict__ out) {
  const int64_t r = blockIdx.x;
  if (r >= n_a_pad) return;
  const uint4* src = r < n_a ? reinterpret_cast<const uint4*>(x + (int64_t)rows[r] * row_bytes) : nullptr;
  uint4* dst = reinterpret_cast<uint4*>(out + r * row_bytes);
  for (int c = threadIdx.x; c < row_bytes / 16; c += blockDim.x) dst[c] = src ? src[c] : make_uint4(0, 0, 0, 0);
}

}  // namespace

bool knn_tc_available() { return true; }

int knn_tc_max_dp() { return 512; }

ancka_status knn_candidates_bf16(const PrepOut& pr, int64_t n, float* cand_val, int32_t* cand_idx, int32_t* err,
                                 cudaStream_t s) {
  const int kb_count = pr.dp / 64;
  if (pr.dp % 64 != 0 || kb_count < 1 || pr.dp > knn_tc_max_dp()) {
    set_error("BF16 contraction supports up to %d features (got %d)", knn_tc_max_dp(), pr.dp);
    return ANCKA_ERR_UNSUPPORTED;
  }
  int nstages;
  size_t smem;
  ANCKA_TRY(tc_smem(kb_count, &nstages, &smem));
  CUtensorMap ta, tb;
  ANCKA_TRY(make_map(&ta, pr.xb, pr.dp, pr.n_pad, kTM, 2));
  ANCKA_TRY(make_map(&tb, pr.xb, pr.dp, pr.n_pad, kTN, 2));
  ANCKA_CUDA(cudaFuncSetAttribute(k_knn_tc<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  CollectArgs none{};
  const int all_tiles = (int)ceil_div(pr.n_pad, kTN);
  k_knn_tc<false, false><<<(unsigned)(pr.n_pad / kTM), kThreads, smem, s>>>(
      ta, tb, n, pr.n_pad, kb_count, nstages, all_tiles, cand_val, cand_idx, nullptr, none, err);
  ANCKA_LAUNCHED();
  return ANCKA_OK;
}

ancka_status knn_candidates_fp8(const PrepOut& pr, int64_t n, float* cand_val, int32_t* cand_idx, int32_t* err,
                                cudaStream_t s) {
  const int kb_count = pr.dp8 / 128;
  if (!pr.x8 || pr.dp8 % 128 != 0 || kb_count < 1 || pr.dp8 > knn_tc_max_dp_fp8()) {
    set_error("FP8 contraction supports up to %d features (got %d)", knn_tc_max_dp_fp8(), pr.dp8);
    return ANCKA_ERR_UNSUPPORTED;
  }
  int nstages;
  size_t smem;
  ANCKA_TRY(tc_smem(kb_count, &nstages, &smem));
  CUtensorMap ta, tb;
  ANCKA_TRY(make_map(&ta, pr.x8, pr.dp8, pr.n_pad, kTM, 1));
  ANCKA_TRY(make_map(&tb, pr.x8, pr.dp8, pr.n_pad, kTN, 1));
  ANCKA_CUDA(cudaFuncSetAttribute(k_knn_tc<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  CollectArgs none{};
  const int all_tiles = (int)ceil_div(pr.n_pad, kTN);
  k_knn_tc<false, true><<<(unsigned)(pr.n_pad / kTM), kThreads, smem, s>>>(
      ta, tb, n, pr.n_pad, kb_count, nstages, all_tiles, cand_val, cand_idx, pr.inv_s2, none, err);
  ANCKA_LAUNCHED();
  return ANCKA_OK;
}

int knn_tc_max_dp_fp8() { return 1024; }

// BF16 lists for the n_a rows listed in rows (written at their global rows)
ancka_status knn_list_gathered_bf16(Workspace& ws, const PrepOut& pr, int64_t n, const int32_t* rows, int64_t n_a,
                                    float* cand_val, int32_t* cand_idx, int32_t* err, cudaStream_t s) {
  const int kb_count = pr.dp / 64;
  int nstages;
  size_t smem;
  ANCKA_TRY(tc_smem(kb_count, &nstages, &smem));
  const int64_t n_a_pad = round_up(n_a, kTM);
  __nv_bfloat16* af;
  ANCKA_TRY(ws.alloc(&af, (size_t)n_a_pad * pr.dp));
  k_gather_rows<<<(unsigned)n_a_pad, 64, 0, s>>>(reinterpret_cast<const uint8_t*>(pr.xb), pr.dp * 2, rows, n_a,
                                                 n_a_pad, reinterpret_cast<uint8_t*>(af));
  ANCKA_LAUNCHED();
  CUtensorMap ta, tb;
  ANCKA_TRY(make_map(&ta, af, pr.dp, n_a_pad, kTM, 2));
  ANCKA_TRY(make_map(&tb, pr.xb, pr.dp, pr.n_pad, kTN, 2));
  ANCKA_CUDA(cudaFuncSetAttribute(k_knn_tc<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  CollectArgs ca{rows, n_a, nullptr, nullptr, nullptr, 0};
  const int all_tiles = (int)ceil_div(pr.n_pad, kTN);
  k_knn_tc<false, false><<<(unsigned)(n_a_pad / kTM), kThreads, smem, s>>>(
      ta, tb, n, pr.n_pad, kb_count, nstages, all_tiles, cand_val, cand_idx, nullptr, ca, err);
  ANCKA_LAUNCHED();
  return ANCKA_OK;
}

ancka_status knn_collect_bf16(Workspace& ws, const PrepOut& pr, int64_t n, const int32_t* rows, int64_t n_a,
                              const float* thr, int32_t* cnt, int32_t* buf, int cap, int32_t* err, cudaStream_t s) {
  const int kb_count = pr.dp / 64;
  int nstages;
  size_t smem;
  ANCKA_TRY(tc_smem(kb_count, &nstages, &smem));
  const int64_t n_a_pad = round_up(n_a, kTM);
  __nv_bfloat16* af;
  ANCKA_TRY(ws.alloc(&af, (size_t)n_a_pad * pr.dp));
  k_gather_rows<<<(unsigned)n_a_pad, 64, 0, s>>>(reinterpret_cast<const uint8_t*>(pr.xb), pr.dp * 2, rows, n_a,
                                                 n_a_pad, reinterpret_cast<uint8_t*>(af));
  ANCKA_LAUNCHED();
  CUtensorMap ta, tb;
  ANCKA_TRY(make_map(&ta, af, pr.dp, n_a_pad, kTM, 2));
  ANCKA_TRY(make_map(&tb, pr.xb, pr.dp, pr.n_pad, kTN, 2));
  ANCKA_CUDA(cudaFuncSetAttribute(k_knn_tc<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  CollectArgs ca{rows, n_a, thr, cnt, buf, cap};
  // split the key sweep so that about two waves of CTAs run
  int sms = 152, dev = 0;
  ANCKA_CUDA(cudaGetDevice(&dev));
  ANCKA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int all_tiles = (int)ceil_div(pr.n_pad, kTN);
  const int64_t qblocks = n_a_pad / kTM;
  int splits = (int)std::max<int64_t>(1, std::min<int64_t>(all_tiles, (2 * sms) / std::max<int64_t>(1, qblocks)));
  const int tps = (int)ceil_div(all_tiles, splits);
  splits = (int)ceil_div(all_tiles, tps);
  k_knn_tc<true, false><<<dim3((unsigned)qblocks, (unsigned)splits), kThreads, smem, s>>>(
      ta, tb, n, pr.n_pad, kb_count, nstages, tps, nullptr, nullptr, nullptr, ca, err);
  ANCKA_LAUNCHED();
  return ANCKA_OK;
}

}  // namespace ancka
