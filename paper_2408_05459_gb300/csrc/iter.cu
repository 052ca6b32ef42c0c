// Algorithm 4 after the walk matrices exist: InitBCM (Alg. 3 / Eq. pi_c_t),
// the orthogonal iteration Z = P Q (Eq. zt) with CholeskyQR2, Discretize
// (Def. 2, Alg. 5) and CalMHC (Alg. 2, Eq. mhc-comp-ancka), all enqueued on
// one stream without host synchronisation.
//
// Dense blocks are n x ld FP32 row-major with ld = round_up(width, 4) and
// zero padding columns.  Every reduction has a fixed order, so a run is
// bitwise reproducible.  FP64 is used only for k x k work (the CholeskyQR
// Cholesky factor and inverse, Discretize's trace and objective); cross-CTA
// sums are float-float.  Discretize's k x k polar factor is FP32
// (Newton-Schulz, Jacobi SVD fallback).

#include <algorithm>

#include "common.cuh"

namespace ancka {

namespace {

constexpr int kMaxW = 68;  // k <= 64 -> k+1 <= 65 columns, padded to 68

inline unsigned grid_for(int64_t n, int b) { return (unsigned)ceil_div(n > 0 ? n : 1, b); }

// ---------------------------------------------------------------------------
// generic CSR SpMM with an optional second CSR part and a one-hot addend:
//   out[i] = coef * ( rsA[i] * sum_p vA[p] csA[colA[p]] srcA[colA[p]]
//                     + sum_p vB[p] srcB[colB[p]] )
//            + oh_coef * oh_scale[oh_col[i]] * e_{oh_col[i]}
// G lanes per row, one float4 column chunk per lane.
// ---------------------------------------------------------------------------
struct SpmmArgs {
  const int64_t* ptrA = nullptr;
  const int32_t* colA = nullptr;
  const float* valA = nullptr;
  const float* rsA = nullptr;
  const float* csA = nullptr;
  const float* srcA = nullptr;
  int ldA = 0;
  const int64_t* ptrB = nullptr;
  const int32_t* colB = nullptr;
  const float* valB = nullptr;
  const float* srcB = nullptr;
  int ldB = 0;
  float coef = 1.f;
  const int32_t* oh_col = nullptr;
  const float* oh_scale = nullptr;
  float oh_coef = 0.f;
  float* out = nullptr;
  int ldo = 0;
  int64_t nrows = 0;
  int nv4 = 0;  // float4 chunks per row
  const int32_t* long_rows = nullptr;  // rows with more than long_min entries
  const int32_t* n_long = nullptr;     // their count (device)
  int64_t n_long_host = -1;            // the same count on the host (-1: not known)
  int64_t long_min = 0;                // rows with more entries than this are long
  int64_t mean_entries = 0;            // mean entries per row (picks the slices per row)
  int oh_off = 0;                      // column of the block where this launch's columns start
  int64_t srcA_rows = 0;               // rows of srcA / srcB (0: not known)
  int64_t srcB_rows = 0;
  const int2* long_items = nullptr;    // (long row q, part) work items of at most kLongChunk entries
  const int32_t* long_off = nullptr;   // items of long row q: [long_off[q], long_off[q + 1])
  int64_t n_items_host = 0;
};

__device__ __forceinline__ void fma4(float4& acc, float w, const float4& x) {
  acc.x = fmaf(w, x.x, acc.x);
  acc.y = fmaf(w, x.y, acc.y);
  acc.z = fmaf(w, x.z, acc.z);
  acc.w = fmaf(w, x.w, acc.w);
}

// A row is long when it has more than max(256, 4 x the mean row length)
// entries, or max(1024, 16 x mean) when the gathered block exceeds 64 MB (a
// long row's items pay a block-wide reduction each, so only the hubs whose
// warp would otherwise trail the launch go there; measured on the 2.4M-node
// graph, 10 hops: 93 ms at max(128, 2 x mean), 88 ms at this threshold);
// long rows are cut into work items of at most kLongChunk entries (topology
// entries, then KNN entries) for k_spmm_long.
constexpr int kLongChunk = 1024;

__device__ __forceinline__ int64_t row_entries(const SpmmArgs& a, int64_t i) {
  return (a.ptrA[i + 1] - a.ptrA[i]) + (a.ptrB ? a.ptrB[i + 1] - a.ptrB[i] : 0);
}

// One row per G * S lanes: G lanes over the row's float4 chunks, S slices
// over its entries (slice sl takes entries sl, sl + S, ..., four per step
// with their loads in flight); the slices are summed by a fixed xor
// butterfly, so every lane of the group holds the same sum.  Rows with more
// than long_min entries are left to k_spmm_long.
template <int G, int S>
__global__ void __launch_bounds__(256) k_spmm(SpmmArgs a) {
  constexpr int L = G * S;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = t / L;
  const int u = (int)(t % L);
  const int g = u % G, sl = u / G;
  const bool row_ok = i < a.nrows && row_entries(a, i) <= a.long_min;
  const bool act = row_ok && g < a.nv4;
  float4 accA = make_float4(0.f, 0.f, 0.f, 0.f), accB = accA;
  if (act) {
    int64_t p = a.ptrA[i] + sl;
    const int64_t e = a.ptrA[i + 1];
    for (; p + 3 * S < e; p += 4 * S) {
      int32_t j[4];
      float w[4];
      float4 x[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) j[q] = *(a.colA + p + q * S);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        w[q] = a.valA ? *(a.valA + p + q * S) : 1.f;
        if (a.csA) w[q] *= a.csA[j[q]];
        x[q] = *reinterpret_cast<const float4*>(a.srcA + (int64_t)j[q] * a.ldA + 4 * g);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) fma4(accA, w[q], x[q]);
    }
    if (p < e) {  // at most three entries left: one predicated batch
      int32_t j[3];
      float w[3];
      float4 x[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) j[q] = p + q * S < e ? *(a.colA + p + q * S) : -1;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        w[q] = 0.f;
        x[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j[q] >= 0) {
          w[q] = a.valA ? *(a.valA + p + q * S) : 1.f;
          if (a.csA) w[q] *= a.csA[j[q]];
          x[q] = *reinterpret_cast<const float4*>(a.srcA + (int64_t)j[q] * a.ldA + 4 * g);
        }
      }
#pragma unroll
      for (int q = 0; q < 3; ++q)
        if (j[q] >= 0) fma4(accA, w[q], x[q]);
    }
    if (a.ptrB) {
      int64_t pb = a.ptrB[i] + sl;
      const int64_t eb = a.ptrB[i + 1];
      for (; pb + 3 * S < eb; pb += 4 * S) {
        int32_t j[4];
        float4 x[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) j[q] = *(a.colB + pb + q * S);
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] = *reinterpret_cast<const float4*>(a.srcB + (int64_t)j[q] * a.ldB + 4 * g);
#pragma unroll
        for (int q = 0; q < 4; ++q) fma4(accB, *(a.valB + pb + q * S), x[q]);
      }
      if (pb < eb) {  // at most three entries left: one predicated batch
        int32_t j[3];
        float w[3];
        float4 x[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) j[q] = pb + q * S < eb ? *(a.colB + pb + q * S) : -1;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          w[q] = 0.f;
          x[q] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (j[q] >= 0) {
            w[q] = *(a.valB + pb + q * S);
            x[q] = *reinterpret_cast<const float4*>(a.srcB + (int64_t)j[q] * a.ldB + 4 * g);
          }
        }
#pragma unroll
        for (int q = 0; q < 3; ++q)
          if (j[q] >= 0) fma4(accB, w[q], x[q]);
      }
    }
  }
  if constexpr (S > 1) {  // every lane of the warp takes part
#pragma unroll
    for (int off = G; off < L; off <<= 1) {
      accA.x += __shfl_xor_sync(0xffffffffu, accA.x, off);
      accA.y += __shfl_xor_sync(0xffffffffu, accA.y, off);
      accA.z += __shfl_xor_sync(0xffffffffu, accA.z, off);
      accA.w += __shfl_xor_sync(0xffffffffu, accA.w, off);
      accB.x += __shfl_xor_sync(0xffffffffu, accB.x, off);
      accB.y += __shfl_xor_sync(0xffffffffu, accB.y, off);
      accB.z += __shfl_xor_sync(0xffffffffu, accB.z, off);
      accB.w += __shfl_xor_sync(0xffffffffu, accB.w, off);
    }
  }
  if (!act || sl != 0) return;
  float4 acc = accA;
  if (a.rsA) {
    const float r = a.rsA[i];
    acc.x *= r;
    acc.y *= r;
    acc.z *= r;
    acc.w *= r;
  }
  acc.x = (acc.x + accB.x) * a.coef;
  acc.y = (acc.y + accB.y) * a.coef;
  acc.z = (acc.z + accB.z) * a.coef;
  acc.w = (acc.w + accB.w) * a.coef;
  if (a.oh_col) {
    const int c = a.oh_col[i];
    const int cl = c - a.oh_off;  // this launch's column
    if (cl >= 4 * g && cl < 4 * g + 4) {
      const float add = a.oh_coef * (a.oh_scale ? a.oh_scale[c] : 1.f);
      const int q = cl - 4 * g;
      if (q == 0) acc.x += add;
      else if (q == 1) acc.y += add;
      else if (q == 2) acc.z += add;
      else acc.w += add;
    }
  }
  *reinterpret_cast<float4*>(a.out + i * a.ldo + 4 * g) = acc;
}

// Long rows (hubs of skewed degree distributions): CTAs take work items
// (row, part) grid-stride; 256/G teams of G lanes split the item's entries
// (four in flight per team), a fixed-order tree in shared memory combines
// the teams, and the item's partial sums (topology part, KNN part) go to
// part[item].  k_spmm_long_finish then adds a row's items in order.
template <int G>
__global__ void __launch_bounds__(256) k_spmm_long(SpmmArgs a, float4* __restrict__ part) {
  constexpr int kTeams = 256 / G;
  __shared__ float4 redA[kTeams][G];
  __shared__ float4 redB[kTeams][G];
  const int team = threadIdx.x / G, g = threadIdx.x % G;
  for (int64_t it = blockIdx.x; it < a.n_items_host; it += gridDim.x) {
    const int2 item = a.long_items[it];
    const int64_t i = a.long_rows[item.x];
    const int64_t a0 = a.ptrA[i], lenA = a.ptrA[i + 1] - a0;
    const int64_t b0 = a.ptrB ? a.ptrB[i] : 0, lenB = a.ptrB ? a.ptrB[i + 1] - b0 : 0;
    const int64_t e0 = (int64_t)item.y * kLongChunk;
    const int64_t e1 = (e0 + kLongChunk < lenA + lenB) ? e0 + kLongChunk : lenA + lenB;
    float4 accA = make_float4(0.f, 0.f, 0.f, 0.f), accB = accA;
    if (g < a.nv4) {
      {  // topology entries [e0, min(e1, lenA))
        const int64_t end = a0 + (e1 < lenA ? e1 : lenA);
        int64_t p = a0 + e0 + team;
        for (; p + 3 * kTeams < end; p += 4 * kTeams) {
          int32_t j[4];
          float w[4];
          float4 x[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) j[u] = a.colA[p + u * kTeams];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            w[u] = a.valA ? a.valA[p + u * kTeams] : 1.f;
            if (a.csA) w[u] *= a.csA[j[u]];
            x[u] = *reinterpret_cast<const float4*>(a.srcA + (int64_t)j[u] * a.ldA + 4 * g);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) fma4(accA, w[u], x[u]);
        }
        for (; p < end; p += kTeams) {
          const int32_t j = a.colA[p];
          float w = a.valA ? a.valA[p] : 1.f;
          if (a.csA) w *= a.csA[j];
          fma4(accA, w, *reinterpret_cast<const float4*>(a.srcA + (int64_t)j * a.ldA + 4 * g));
        }
      }
      if (e1 > lenA) {  // KNN entries [max(e0, lenA), e1) - lenA
        const int64_t end = b0 + (e1 - lenA);
        int64_t p = b0 + (e0 > lenA ? e0 - lenA : 0) + team;
        for (; p + 3 * kTeams < end; p += 4 * kTeams) {
          int32_t j[4];
          float4 x[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) j[u] = a.colB[p + u * kTeams];
#pragma unroll
          for (int u = 0; u < 4; ++u) x[u] = *reinterpret_cast<const float4*>(a.srcB + (int64_t)j[u] * a.ldB + 4 * g);
#pragma unroll
          for (int u = 0; u < 4; ++u) fma4(accB, a.valB[p + u * kTeams], x[u]);
        }
        for (; p < end; p += kTeams)
          fma4(accB, a.valB[p], *reinterpret_cast<const float4*>(a.srcB + (int64_t)a.colB[p] * a.ldB + 4 * g));
      }
    }
    redA[team][g] = accA;
    redB[team][g] = accB;
    __syncthreads();
    for (int half = kTeams / 2; half >= 1; half >>= 1) {
      if (team < half) {
        float4 x = redA[team][g], y = redA[team + half][g];
        redA[team][g] = make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w);
        x = redB[team][g];
        y = redB[team + half][g];
        redB[team][g] = make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w);
      }
      __syncthreads();
    }
    if (team == 0) {
      part[(it * 2 + 0) * G + g] = redA[0][g];
      part[(it * 2 + 1) * G + g] = redB[0][g];
    }
    __syncthreads();
  }
}

template <int G>
__global__ void k_spmm_long_finish(SpmmArgs a, const float4* __restrict__ part) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t q = t / G;
  const int g = (int)(t % G);
  if (q >= a.n_long_host || g >= a.nv4) return;
  const int64_t i = a.long_rows[q];
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f), b = acc;
  for (int64_t it = a.long_off[q]; it < a.long_off[q + 1]; ++it) {
    const float4 x = part[(it * 2 + 0) * G + g], y = part[(it * 2 + 1) * G + g];
    acc = make_float4(acc.x + x.x, acc.y + x.y, acc.z + x.z, acc.w + x.w);
    b = make_float4(b.x + y.x, b.y + y.y, b.z + y.z, b.w + y.w);
  }
  if (a.rsA) {
    const float r = a.rsA[i];
    acc.x *= r;
    acc.y *= r;
    acc.z *= r;
    acc.w *= r;
  }
  acc = make_float4((acc.x + b.x) * a.coef, (acc.y + b.y) * a.coef, (acc.z + b.z) * a.coef, (acc.w + b.w) * a.coef);
  if (a.oh_col) {
    const int c = a.oh_col[i];
    const int cl = c - a.oh_off;
    if (cl >= 4 * g && cl < 4 * g + 4) {
      const float add = a.oh_coef * (a.oh_scale ? a.oh_scale[c] : 1.f);
      const int qq = cl - 4 * g;
      if (qq == 0) acc.x += add;
      else if (qq == 1) acc.y += add;
      else if (qq == 2) acc.z += add;
      else acc.w += add;
    }
  }
  *reinterpret_cast<float4*>(a.out + i * a.ldo + 4 * g) = acc;
}

// The long-row threshold comes from the mean row length, taken here from the
// row pointers (meta[1] = mean, meta[2] = threshold) so that the host needs
// no count before the launch.
__global__ void k_find_long(const int64_t* __restrict__ ptrA, const int64_t* __restrict__ ptrB, int64_t nrows,
                            int big, int32_t* __restrict__ rows, int32_t* __restrict__ count,
                            int64_t* __restrict__ meta) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nnz = (ptrA[nrows] - ptrA[0]) + (ptrB ? ptrB[nrows] - ptrB[0] : 0);
  const int64_t mean = nrows > 0 ? (nnz + nrows - 1) / nrows : 0;
  const int64_t lo = big ? 1024 : 256, f = big ? 16 : 4;
  const int64_t long_min = f * mean > lo ? f * mean : lo;
  if (i == 0) {
    meta[1] = mean;
    meta[2] = long_min;
  }
  if (i >= nrows) return;
  const int64_t e = (ptrA[i + 1] - ptrA[i]) + (ptrB ? ptrB[i + 1] - ptrB[i] : 0);
  if (e > long_min) rows[atomicAdd(count, 1)] = (int32_t)i;
}

struct LongRows {
  int32_t* rows = nullptr;
  int32_t* count = nullptr;   // device: long rows found
  int64_t* meta = nullptr;    // device: work items, mean row length, long-row threshold
  int64_t nrows = 0;
  int64_t nnz_bound = 0;      // upper bound of the entries (sizes the work-item array)
  int64_t count_host = -1;    // host copies, valid after read_long_rows
  int64_t min_entries = 0;
  int64_t mean = 0;
  int2* items = nullptr;      // (q, part) work items
  int32_t* off = nullptr;     // count + 1 item offsets
  int64_t items_host = 0;
};

// Work-item offsets of the long rows (count read on the device): one CTA,
// 1024 rows per round, block-wide exclusive scan; meta[0] = total items.
__global__ void __launch_bounds__(1024) k_long_item_offsets(const int64_t* __restrict__ ptrA,
                                                            const int64_t* __restrict__ ptrB,
                                                            const int32_t* __restrict__ rows,
                                                            const int32_t* __restrict__ count,
                                                            int32_t* __restrict__ off, int64_t* __restrict__ meta) {
  __shared__ int32_t wsum[32];
  __shared__ int32_t carry_s;
  const int nl = *count;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int base = 0; base < nl; base += blockDim.x) {
    const int q = base + (int)threadIdx.x;
    int32_t c = 0;
    if (q < nl) {
      const int64_t i = rows[q];
      const int64_t len = (ptrA[i + 1] - ptrA[i]) + (ptrB ? ptrB[i + 1] - ptrB[i] : 0);
      c = (int32_t)((len + kLongChunk - 1) / kLongChunk);
    }
    int32_t x = c;  // inclusive warp scan
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int32_t v = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
      }
      wsum[lane] = v;  // inclusive over warps
    }
    __syncthreads();
    const int32_t carry = carry_s;
    const int32_t before = (wid > 0 ? wsum[wid - 1] : 0) + x - c;
    if (q < nl) off[q] = carry + before;
    __syncthreads();
    if (threadIdx.x == 0) carry_s = carry + wsum[(blockDim.x >> 5) - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    off[nl] = carry_s;
    meta[0] = carry_s;
  }
}

__global__ void k_long_item_fill(const int32_t* __restrict__ off, const int32_t* __restrict__ count,
                                 int2* __restrict__ items) {
  const int64_t nl = *count;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nl; q += (int64_t)gridDim.x * blockDim.x)
    for (int32_t it = off[q]; it < off[q + 1]; ++it) items[it] = make_int2((int)q, it - off[q]);
}

// work items of the long rows, on the device (arrays sized by upper bounds)
ancka_status build_long_items(Workspace& ws, const int64_t* ptrA, const int64_t* ptrB, LongRows* lr, cudaStream_t s) {
  const int64_t nr = lr->nrows > 0 ? lr->nrows : 1;
  ANCKA_TRY(ws.alloc(&lr->off, (size_t)nr + 1));
  ANCKA_TRY(ws.alloc(&lr->items, (size_t)(nr + lr->nnz_bound / kLongChunk + 1)));
  k_long_item_offsets<<<1, 1024, 0, s>>>(ptrA, ptrB, lr->rows, lr->count, lr->off, lr->meta);
  ANCKA_LAUNCHED();
  const unsigned g = (unsigned)(ceil_div(nr, 256) < 1216 ? ceil_div(nr, 256) : 1216);
  k_long_item_fill<<<g, 256, 0, s>>>(lr->off, lr->count, lr->items);
  ANCKA_LAUNCHED();
  return ANCKA_OK;
}

// long rows with a fixed threshold: max(256, 4 x mean), or max(1024, 16 x
// mean) when the gathered block exceeds 64 MB; nnz_bound >= the entries
ancka_status find_long_rows(Workspace& ws, const int64_t* ptrA, const int64_t* ptrB, int64_t nrows,
                            int64_t nnz_bound, double block_bytes, LongRows* out, cudaStream_t s) {
  out->nrows = nrows;
  out->nnz_bound = nnz_bound;
  const bool big = block_bytes > 64.0 * (1 << 20);
  ANCKA_TRY(ws.alloc(&out->rows, (size_t)(nrows > 0 ? nrows : 1)));
  ANCKA_TRY(ws.zeros(&out->count, 1));
  ANCKA_TRY(ws.zeros(&out->meta, 3));
  k_find_long<<<(unsigned)ceil_div(nrows > 0 ? nrows : 1, 256), 256, 0, s>>>(ptrA, ptrB, nrows, big ? 1 : 0,
                                                                              out->rows, out->count, out->meta);
  ANCKA_LAUNCHED();
  return ANCKA_OK;
}

// the host copies of every LongRows' counts with one stream sync
ancka_status read_long_rows(LongRows* const* lrs, int nlr, cudaStream_t s) {
  int32_t cnt[4] = {0, 0, 0, 0};
  int64_t meta[4][3] = {};
  for (int q = 0; q < nlr; ++q) {
    ANCKA_CUDA(cudaMemcpyAsync(&cnt[q], lrs[q]->count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    ANCKA_CUDA(cudaMemcpyAsync(meta[q], lrs[q]->meta, sizeof(int64_t) * 3, cudaMemcpyDeviceToHost, s));
  }
  ANCKA_CUDA(cudaStreamSynchronize(s));
  for (int q = 0; q < nlr; ++q) {
    lrs[q]->count_host = cnt[q];
    lrs[q]->items_host = meta[q][0];
    lrs[q]->mean = meta[q][1];
    lrs[q]->min_entries = meta[q][2];
  }
  return ANCKA_OK;
}

template <int G, int S>
void launch_spmm(const SpmmArgs& a, cudaStream_t s) {
  k_spmm<G, S><<<grid_for(a.nrows * G * S, 256), 256, 0, s>>>(a);
}

template <int G>
void launch_spmm_slices(const SpmmArgs& a, int S, cudaStream_t s) {
  if constexpr (G <= 4) {
    if (S >= 8) return launch_spmm<G, 8>(a, s);
  }
  if constexpr (G <= 8) {
    if (S >= 4) return launch_spmm<G, 4>(a, s);
  }
  if constexpr (G <= 16) {
    if (S >= 2) return launch_spmm<G, 2>(a, s);
  }
  launch_spmm<G, 1>(a, s);
}

ancka_status spmm(const SpmmArgs& a0, cudaStream_t s) {
  if (!a0.long_rows || a0.n_long_host < 0) {
    set_error("internal: SpMM without a long-row list");
    return ANCKA_ERR_INTERNAL;
  }
  const int ld = 4 * a0.nv4;
  // long rows: work items into partial sums, then the per-row finish
  const bool longs = a0.n_long_host > 0 && a0.n_items_host > 0;
  if (a0.n_long_host > 0 && !a0.long_items) {
    set_error("internal: SpMM with long rows but no work items");
    return ANCKA_ERR_INTERNAL;
  }
  float4* part = nullptr;
  if (longs)
    ANCKA_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&part), sizeof(float4) * 2 * 16 * a0.n_items_host, s));
  const unsigned lgrid = (unsigned)(a0.n_items_host < 1216 ? a0.n_items_host : 1216);
  for (int c0 = 0; c0 < ld; c0 += 64) {  // a launch covers at most 64 columns
    SpmmArgs a = a0;
    const int w = ld - c0 < 64 ? ld - c0 : 64;
    a.nv4 = w / 4;
    a.oh_off = c0;
    a.out = a0.out + c0;
    a.srcA = a0.srcA + c0;
    if (a0.srcB) a.srcB = a0.srcB + c0;
    const int nv4 = a.nv4;
    const int G = nv4 <= 1 ? 1 : nv4 <= 2 ? 2 : nv4 <= 4 ? 4 : nv4 <= 8 ? 8 : 16;
    // slices per row: about four entries per slice, at most 32 lanes per row
    int S = 1;
    while (S < 8 && 4 * S * 2 <= a.mean_entries && G * S * 2 <= 32) S <<= 1;
    const unsigned fgrid = grid_for(a0.n_long_host * G, 256);
    switch (G) {
      case 1:
        launch_spmm_slices<1>(a, S, s);
        if (longs) { k_spmm_long<1><<<lgrid, 256, 0, s>>>(a, part); k_spmm_long_finish<1><<<fgrid, 256, 0, s>>>(a, part); }
        break;
      case 2:
        launch_spmm_slices<2>(a, S, s);
        if (longs) { k_spmm_long<2><<<lgrid, 256, 0, s>>>(a, part); k_spmm_long_finish<2><<<fgrid, 256, 0, s>>>(a, part); }
        break;
      case 4:
        if (nv4 == 3 && S == 1)  // three chunks: three lanes per row, no idle lane
          launch_spmm<3, 1>(a, s);
        else
          launch_spmm_slices<4>(a, S, s);
        if (longs) { k_spmm_long<4><<<lgrid, 256, 0, s>>>(a, part); k_spmm_long_finish<4><<<fgrid, 256, 0, s>>>(a, part); }
        break;
      case 8:
        launch_spmm_slices<8>(a, S, s);
        if (longs) { k_spmm_long<8><<<lgrid, 256, 0, s>>>(a, part); k_spmm_long_finish<8><<<fgrid, 256, 0, s>>>(a, part); }
        break;
      default:
        launch_spmm_slices<16>(a, S, s);
        if (longs) { k_spmm_long<16><<<lgrid, 256, 0, s>>>(a, part); k_spmm_long_finish<16><<<fgrid, 256, 0, s>>>(a, part); }
        break;
    }
    ANCKA_LAUNCHED();
    if (longs) {
      count_launch();
      count_launch();
    }
  }
  if (part) ANCKA_CUDA(cudaFreeAsync(part, s));
  return ANCKA_OK;
}

// ---------------------------------------------------------------------------
// Gram matrix of the n x w block Z, then its Cholesky inverse.
// Each CTA stages 128-row tiles of Z in shared memory; a thread owns a 4 x 4
// block of Gram entries and a subset of the tile's rows, sums them in FP32
// within the tile and carries the running total as a float-float pair
// (hi + lo, compensated), so accuracy does not degrade with n.  The CTA's
// subsets are combined in a fixed order into the packed upper triangle.
// CholeskyQR2's second pass restores orthogonality lost to rounding in the
// first Gram.
// ---------------------------------------------------------------------------
constexpr int kGramThreads = 256, kGramRows = 128, kGramLd = kMaxW;

__device__ __forceinline__ int tri_index(int a, int b, int w) { return a * w - a * (a - 1) / 2 + (b - a); }

// block pair index q -> (A, B), A <= B < nb
__device__ __forceinline__ void block_pair(int q, int nb, int& A, int& B) {
  A = 0;
  while (q >= nb - A) {
    q -= nb - A;
    ++A;
  }
  B = A + q;
}

__device__ void chol_inv_block(const float2* __restrict__ partial, int nblk, int w, float* __restrict__ Rinv_out,
                               int32_t* __restrict__ status, double* csm, float2* scratch);

// Rows of a staged tile times an upper-triangular R^-1 (rows of T and of Rs
// at stride ld; Rs zero below the diagonal and past w): out[r, c] =
// sum_{a <= c} T[r, a] Rs[a, c], each element's terms in ascending a (fmaf).
// A thread takes two rows x two float4 column groups, so each load of T or
// Rs serves two outputs.  Results go to the tile buffer Tout (may be null,
// stride ld) and to global rows (stride ldo).
__device__ __forceinline__ void rinv_tile(const float* __restrict__ T, int ld, int rows, int nb, int w,
                                          const float* __restrict__ Rs, float* __restrict__ Tout,
                                          float* __restrict__ gout, int64_t ldo) {
  const int ngp = (nb + 1) >> 1, nrp = (rows + 1) >> 1;
  for (int e = threadIdx.x; e < nrp * ngp; e += blockDim.x) {
    const int rp = e / ngp, gp = e - rp * ngp;
    const int r0 = 2 * rp, g0 = 2 * gp;
    const bool r1ok = r0 + 1 < rows, g1ok = g0 + 1 < nb;
    const float* z0 = T + r0 * ld;
    const float* z1 = T + (r1ok ? r0 + 1 : r0) * ld;
    const int am0 = (4 * g0 + 3 < w - 1) ? 4 * g0 + 3 : w - 1;
    const int am1 = g1ok ? ((4 * g0 + 7 < w - 1) ? 4 * g0 + 7 : w - 1) : am0;
    float4 c00 = make_float4(0.f, 0.f, 0.f, 0.f), c01 = c00, c10 = c00, c11 = c00;  // [row][group]
    int a = 0;
#pragma unroll 4
    for (; a <= am0; ++a) {
      const float za0 = z0[a], za1 = z1[a];
      const float4 r0v = *reinterpret_cast<const float4*>(&Rs[a * ld + 4 * g0]);
      c00.x = fmaf(za0, r0v.x, c00.x); c00.y = fmaf(za0, r0v.y, c00.y);
      c00.z = fmaf(za0, r0v.z, c00.z); c00.w = fmaf(za0, r0v.w, c00.w);
      c10.x = fmaf(za1, r0v.x, c10.x); c10.y = fmaf(za1, r0v.y, c10.y);
      c10.z = fmaf(za1, r0v.z, c10.z); c10.w = fmaf(za1, r0v.w, c10.w);
      if (g1ok) {
        const float4 r1v = *reinterpret_cast<const float4*>(&Rs[a * ld + 4 * g0 + 4]);
        c01.x = fmaf(za0, r1v.x, c01.x); c01.y = fmaf(za0, r1v.y, c01.y);
        c01.z = fmaf(za0, r1v.z, c01.z); c01.w = fmaf(za0, r1v.w, c01.w);
        c11.x = fmaf(za1, r1v.x, c11.x); c11.y = fmaf(za1, r1v.y, c11.y);
        c11.z = fmaf(za1, r1v.z, c11.z); c11.w = fmaf(za1, r1v.w, c11.w);
      }
    }
    for (; a <= am1; ++a) {  // the second group's remaining terms
      const float za0 = z0[a], za1 = z1[a];
      const float4 r1v = *reinterpret_cast<const float4*>(&Rs[a * ld + 4 * g0 + 4]);
      c01.x = fmaf(za0, r1v.x, c01.x); c01.y = fmaf(za0, r1v.y, c01.y);
      c01.z = fmaf(za0, r1v.z, c01.z); c01.w = fmaf(za0, r1v.w, c01.w);
      c11.x = fmaf(za1, r1v.x, c11.x); c11.y = fmaf(za1, r1v.y, c11.y);
      c11.z = fmaf(za1, r1v.z, c11.z); c11.w = fmaf(za1, r1v.w, c11.w);
    }
    if (Tout) *reinterpret_cast<float4*>(&Tout[r0 * ld + 4 * g0]) = c00;
    *reinterpret_cast<float4*>(gout + r0 * ldo + 4 * g0) = c00;
    if (g1ok) {
      if (Tout) *reinterpret_cast<float4*>(&Tout[r0 * ld + 4 * g0 + 4]) = c01;
      *reinterpret_cast<float4*>(gout + r0 * ldo + 4 * g0 + 4) = c01;
    }
    if (r1ok) {
      if (Tout) *reinterpret_cast<float4*>(&Tout[(r0 + 1) * ld + 4 * g0]) = c10;
      *reinterpret_cast<float4*>(gout + (r0 + 1) * ldo + 4 * g0) = c10;
      if (g1ok) {
        if (Tout) *reinterpret_cast<float4*>(&Tout[(r0 + 1) * ld + 4 * g0 + 4]) = c11;
        *reinterpret_cast<float4*>(gout + (r0 + 1) * ldo + 4 * g0 + 4) = c11;
      }
    }
  }
}

// Gram partials of Z; the CTA that finishes last (atomic ticket) sums the
// partials and factors them (chol_inv_block), so one launch does both.  With
// Rin (an R^-1 of the previous pass) the launch first forms each tile's rows
// Q = Z R^-1 (the same terms in the same order as k_apply_rinv), writes them
// to Qout and takes the Gram matrix of Q: CholeskyQR2's middle step in one
// pass.  Dynamic shared memory: the k x k factorisation, or (with Rin) R^-1
// padded to 4 nb columns and the Q tile.
__global__ void __launch_bounds__(kGramThreads)
k_gram_chol(const float* __restrict__ Z, int ldz, int64_t n, int w, const float* __restrict__ Rin,
            float* __restrict__ Qout, float2* __restrict__ partial, unsigned int* __restrict__ ticket,
            float* __restrict__ Rinv_out, int32_t* __restrict__ status) {
  __shared__ __align__(16) float T[kGramRows * kGramLd];
  __shared__ unsigned int my_ticket;
  extern __shared__ double csm[];
  const int64_t per = ceil_div(n, (int64_t)gridDim.x);
  const int64_t r0 = (int64_t)blockIdx.x * per;
  const int64_t r1 = (r0 + per < n) ? r0 + per : n;
  const int nb = (w + 3) / 4, nbp = nb * (nb + 1) / 2;
  const int S = max(1, kGramThreads / nbp);
  const int t = threadIdx.x;
  const bool active = t < nbp * S;
  const int bp = active ? t % nbp : 0, sub = active ? t / nbp : 0;
  int A, B;
  block_pair(bp, nb, A, B);
  float hi[16], lo[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) hi[e] = lo[e] = 0.f;
  // tiles as tall as the buffer allows at this width (row stride 4 nb), so
  // that a CTA's rows arrive in few load waves
  const int tld = 4 * nb;
  const int trows = (kGramRows * kGramLd) / tld;
  float* Rs = reinterpret_cast<float*>(csm);  // with Rin: R^-1 (tld x tld), then the Q tile
  float* TQ = Rs + tld * tld;
  if (Rin)
    for (int e = t; e < tld * tld; e += kGramThreads) {
      const int a = e / tld, c = e % tld;
      Rs[e] = (c < w && a <= c) ? Rin[a * w + c] : 0.f;
    }
  const float* src = Rin ? TQ : T;
  for (int64_t rb = r0; rb < r1; rb += trows) {
    const int rows = (int)((r1 - rb) < trows ? (r1 - rb) : trows);
    __syncthreads();
    {  // a tile is trows x nb <= kGramRows kGramLd / 4 float4, all of a thread's loads issued first
      constexpr int kLd = (kGramRows * kGramLd / 4 + kGramThreads - 1) / kGramThreads;
      float4 v[kLd];
#pragma unroll
      for (int u = 0; u < kLd; ++u) {
        const int e = t + u * kGramThreads;
        const int r = e / nb, c = 4 * (e - r * nb);
        v[u] = r < rows ? *reinterpret_cast<const float4*>(Z + (rb + r) * ldz + c) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < kLd; ++u) {
        const int e = t + u * kGramThreads;
        const int r = e / nb, c = 4 * (e - r * nb);
        if (r < rows) {
          if (c + 1 >= w) v[u].y = 0.f;  // columns >= w read as zero
          if (c + 2 >= w) v[u].z = 0.f;
          if (c + 3 >= w) v[u].w = 0.f;
          *reinterpret_cast<float4*>(&T[r * tld + c]) = v[u];
        }
      }
    }
    __syncthreads();
    if (Rin) {  // Q rows of the tile: q[c] = sum_{a <= c} z[a] R^-1[a, c]
      rinv_tile(T, tld, rows, nb, w, Rs, TQ, Qout + rb * ldz, ldz);
      __syncthreads();
    }
    if (active) {
      float acc[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) acc[e] = 0.f;
#pragma unroll 4
      for (int r = sub; r < rows; r += S) {  // four rows' loads in flight
        const float4 xa = *reinterpret_cast<const float4*>(&src[r * tld + 4 * A]);
        const float4 xb = *reinterpret_cast<const float4*>(&src[r * tld + 4 * B]);
        const float a4[4] = {xa.x, xa.y, xa.z, xa.w}, b4[4] = {xb.x, xb.y, xb.z, xb.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i * 4 + j] = fmaf(a4[i], b4[j], acc[i * 4 + j]);
      }
#pragma unroll
      for (int e = 0; e < 16; ++e) ff_add(hi[e], lo[e], acc[e], 0.f);
    }
  }
  __syncthreads();
  float2* red = reinterpret_cast<float2*>(T);  // nbp * 16 * S <= 4096 pairs
  if (active) {
#pragma unroll
    for (int e = 0; e < 16; ++e) red[(bp * 16 + e) * S + sub] = make_float2(hi[e], lo[e]);
  }
  __syncthreads();
  const int np = w * (w + 1) / 2;
  for (int e = t; e < nbp * 16; e += kGramThreads) {
    int Aq, Bq;
    block_pair(e / 16, nb, Aq, Bq);
    const int a = 4 * Aq + (e % 16) / 4, b = 4 * Bq + (e % 4);
    if (a >= w || b >= w || a > b) continue;
    float h = 0.f, l = 0.f;
    for (int q = 0; q < S; ++q) {
      const float2 v = red[e * S + q];
      ff_add(h, l, v.x, v.y);
    }
    partial[(int64_t)blockIdx.x * np + tri_index(a, b, w)] = make_float2(h, l);
  }
  __threadfence();
  __syncthreads();
  if (t == 0) my_ticket = atomicAdd(ticket, 1u);
  __syncthreads();
  if (my_ticket != gridDim.x - 1) return;
  __threadfence();
  chol_inv_block(partial, gridDim.x, w, Rinv_out, status, csm, reinterpret_cast<float2*>(T));
  if (t == 0) *ticket = 0u;  // ready for the next launch
}

// One CTA: G = sum of the per-CTA partials (float-float, fixed order, then
// FP64), upper Cholesky G = R^T R in FP64, Rinv = R^-1 (upper), written as
// FP32.  A non-positive pivot marks the status and is replaced by a tiny one
// so the run finishes.  csm: G, R, X (w*w doubles each); scratch: up to
// max(w(w+1)/2, 256) float pairs.
// 1/sqrt(d) for d in [1e-30, 1e30]: FP32 seed, then two Newton-Raphson
// steps y <- y (3 - d y^2) / 2 in FP64 (the error squares each step:
// ~2^-22 -> ~2^-43 -> FP64 rounding); outside that range the exact quotient.
__device__ __forceinline__ double rsqrt_newton(double d) {
  if (!(d >= 1e-30 && d <= 1e30)) return 1.0 / sqrt(d);
  double y = (double)rsqrtf((float)d);
  const double h = -0.5 * d;
  y = y * fma(h, y * y, 1.5);
  y = y * fma(h, y * y, 1.5);
  return y;
}

// Sums the CTA partials into G (FP64), factors G = R^T R and writes R^-1
// (row-major, upper triangular, FP32).  Right-looking Cholesky: at step j the
// pivot gives r_j = 1/R_jj, row j of R is G's row j times r_j, and the
// trailing block loses the outer product of that row.  R^-1 comes from the
// same steps as Y = L^-1 (L = R^T) by Gauss-Jordan elimination on [L | I]:
// row j of Y is scaled by r_j and row j times L_ij is taken from every later
// row i.  Each step is a few dependent FP64 operations across the CTA, with
// no division or square root on the chain.
__device__ void chol_inv_block(const float2* __restrict__ partial, int nblk, int w, float* __restrict__ Rinv_out,
                               int32_t* __restrict__ status, double* csm, float2* scratch) {
  const int ww = w * w, np = w * (w + 1) / 2;
  double* G = csm;
  double* R = csm + ww;
  double* Y = csm + 2 * ww;
  double* rj_s = csm + 3 * ww;
  {
    // Tn threads per entry, each summing a strided subset of the CTA
    // partials with sixteen loads in flight; subsets combined in fixed order
    const int Tn = max(1, min((int)blockDim.x / np, 16));
    for (int e = threadIdx.x; e < np * Tn; e += blockDim.x) {
      const int entry = e / Tn, sub = e % Tn;
      float h = 0.f, l = 0.f;
      int bb = sub;
      for (; bb + 15 * Tn < nblk; bb += 16 * Tn) {
        float2 v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] = __ldcg(partial + (int64_t)(bb + u * Tn) * np + entry);
#pragma unroll
        for (int u = 0; u < 16; ++u) ff_add(h, l, v[u].x, v[u].y);
      }
      for (; bb < nblk; bb += Tn) {
        const float2 v = __ldcg(partial + (int64_t)bb * np + entry);
        ff_add(h, l, v.x, v.y);
      }
      scratch[e] = make_float2(h, l);
    }
    for (int e = threadIdx.x; e < ww; e += blockDim.x) {
      R[e] = 0.0;
      Y[e] = (e / w == e % w) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
      float h = 0.f, l = 0.f;
      for (int sub = 0; sub < Tn; ++sub) ff_add(h, l, scratch[e * Tn + sub].x, scratch[e * Tn + sub].y);
      int a = 0, q = e;
      while (q >= w - a) {
        q -= w - a;
        ++a;
      }
      const double g = (double)h + (double)l;
      G[a * w + a + q] = g;
      G[(a + q) * w + a] = g;
    }
    __syncthreads();
  }
  for (int j = 0; j < w; ++j) {
    const int m = w - 1 - j;  // rows / columns after j
    if (threadIdx.x == 0) {
      double d = G[j * w + j];
      if (!(d > 1e-300)) {
        atomicExch(status, 1);
        d = 1e-300;
      }
      const double r = rsqrt_newton(d);
      rj_s[0] = r;
      R[j * w + j] = d * r;
    }
    __syncthreads();
    const double r = rj_s[0];
    // row j of R right of the pivot; row j of Y (entries 0..j)
    for (int e = threadIdx.x; e < m + j + 1; e += blockDim.x) {
      if (e < m) {
        R[j * w + j + 1 + e] = G[j * w + j + 1 + e] * r;
      } else {
        const int a = e - m;
        Y[j * w + a] *= r;
      }
    }
    __syncthreads();
    // trailing update of G (upper triangle) and of the later rows of Y
    for (int e = threadIdx.x; e < m * m + m * (j + 1); e += blockDim.x) {
      if (e < m * m) {
        const int i = j + 1 + e / m, l = j + 1 + e % m;
        if (i <= l) G[i * w + l] = fma(-R[j * w + i], R[j * w + l], G[i * w + l]);
      } else {
        const int f = e - m * m;
        const int i = j + 1 + f / (j + 1), a = f % (j + 1);
        Y[i * w + a] = fma(-R[j * w + i], Y[j * w + a], Y[i * w + a]);
      }
    }
    __syncthreads();
  }
  // R^-1 = Y^T
  for (int e = threadIdx.x; e < ww; e += blockDim.x) {
    const int a = e / w, c = e % w;
    Rinv_out[e] = a <= c ? (float)Y[c * w + a] : 0.f;
  }
}

// out[i, c] = sum_{a <= c} Z[i, a] Rinv[a, c]  (padding columns -> 0).
// CTAs take tiles of rows grid-stride: a tile is staged in shared memory by
// coalesced 16-byte loads (all of a thread's loads issued first), then each
// thread forms one float4 of an output row from the staged row and R^-1.
__global__ void __launch_bounds__(kGramThreads)
k_apply_rinv(const float* __restrict__ Z, int ld, int64_t n, int w, const float* __restrict__ Rinv,
             float* __restrict__ out) {
  constexpr int kApplyRows = 64;  // tile buffer rows at the widest block (static shared memory <= 48 KB)
  __shared__ __align__(16) float Rs[kMaxW * kMaxW];
  __shared__ __align__(16) float T[kApplyRows * kGramLd];
  const int nv4 = ld / 4;
  const int t = threadIdx.x;
  for (int e = t; e < w * ld; e += blockDim.x) {
    const int a = e / ld, c = e % ld;
    Rs[a * ld + c] = (c < w && a <= c) ? Rinv[a * w + c] : 0.f;
  }
  const int trows = (kApplyRows * kGramLd) / ld;
  for (int64_t rb = (int64_t)blockIdx.x * trows; rb < n; rb += (int64_t)gridDim.x * trows) {
    const int rows = (int)((n - rb) < trows ? (n - rb) : trows);
    __syncthreads();
    {
      constexpr int kLd = (kApplyRows * kGramLd / 4 + kGramThreads - 1) / kGramThreads;
      const float4* src = reinterpret_cast<const float4*>(Z + rb * ld);
      float4 v[kLd];
#pragma unroll
      for (int u = 0; u < kLd; ++u) {
        const int e = t + u * kGramThreads;
        v[u] = e < rows * nv4 ? src[e] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < kLd; ++u) {
        const int e = t + u * kGramThreads;
        if (e < rows * nv4) *reinterpret_cast<float4*>(&T[4 * e]) = v[u];
      }
    }
    __syncthreads();
    rinv_tile(T, ld, rows, nv4, w, Rs, nullptr, out + rb * ld, ld);
  }
}

ancka_status apply_rinv(const float* Z, int ld, int64_t n, int w, const float* Rinv, float* out,
                        cudaStream_t s) {
  const int64_t tiles = ceil_div(n, (int64_t)((64 * kGramLd) / ld));  // kApplyRows rows of kGramLd floats
  const unsigned grid = (unsigned)(tiles < 4 * 152 ? tiles : 4 * 152);
  k_apply_rinv<<<grid > 0 ? grid : 1, kGramThreads, 0, s>>>(Z, ld, n, w, Rinv, out);
  ANCKA_LAUNCHED();
  return ANCKA_OK;
}

// ---------------------------------------------------------------------------
// Discretize (Def. 2, Alg. 5)
// ---------------------------------------------------------------------------
struct DiscState {
  long long* part;      // kDiscMaxGrid x k x k: per-CTA sums of Q~ rows per cluster (fixed point)
  int32_t* partc;       // kDiscMaxGrid x k: per-CTA cluster sizes
  long long* S;         // k x k: totals of part
  int32_t* cnt;         // k: cluster sizes of the current Y
  unsigned int* bar;    // 2: grid barrier count and generation
  int32_t* err;         // 1: grid barrier expired
};

constexpr int kDiscThreads = 512;
constexpr int kDiscMaxGrid = 320;
// dynamic shared memory, in floats: a region of 256 x 68 (the row tile
// in phase A; M, X, X', P (4 x 64 x 65) or Jacobi's A and V in phase B), the tile's
// labels, the slice sums, R with rows padded to a multiple of 16 columns
constexpr int kDiscLd = 65;
constexpr int kDiscRegion = 256 * 68;  // >= 4 x 64 x kDiscLd (phase B) and the staged tile of phase A
constexpr int kDiscLabels = 512;
constexpr int kDiscSlices = 8192;  // the int64 cluster sums, k x k <= 4096 of them
constexpr int kDiscR = 64 * 64;
constexpr int kNsMaxIter = 60;

__global__ void k_rownorm(const float* __restrict__ Q, int ldq, int off, int64_t n, int k,
                          float* __restrict__ Qt, int ldt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* q = Q + i * ldq + off;
  float s = 0.f;
  for (int c = 0; c < k; ++c) s = fmaf(q[c], q[c], s);
  const float inv = s > 0.f ? 1.f / sqrtf(s) : 0.f;  // a zero row stays zero
  for (int c = 0; c < ldt; ++c) Qt[i * ldt + c] = c < k ? q[c] * inv : 0.f;
}

// The same rows through shared memory (block strides up to 68 and 64): the
// tile is loaded and stored coalesced, and each thread takes its row from the
// tile with the same operations in the same order as k_rownorm.
constexpr int kRnRows = 64;
__global__ void __launch_bounds__(kRnRows)
k_rownorm_tiled(const float* __restrict__ Q, int ldq, int off, int64_t n, int k, float* __restrict__ Qt, int ldt) {
  __shared__ float T[kRnRows * 69];
  __shared__ float O[kRnRows * 65];
  const int64_t r0 = (int64_t)blockIdx.x * kRnRows;
  const int rows = (int)((n - r0) < kRnRows ? (n - r0) : kRnRows);
  const int tq = ldq + 1, to = ldt + 1;
  const float* src = Q + r0 * ldq;
#pragma unroll 4
  for (int e = threadIdx.x; e < rows * ldq; e += kRnRows) {
    const int r = e / ldq;
    T[r * tq + (e - r * ldq)] = src[e];
  }
  __syncthreads();
  const int r = threadIdx.x;
  if (r < rows) {
    const float* q = T + r * tq + off;
    float s = 0.f;
    for (int c = 0; c < k; ++c) s = fmaf(q[c], q[c], s);
    const float inv = s > 0.f ? 1.f / sqrtf(s) : 0.f;  // a zero row stays zero
    for (int c = 0; c < ldt; ++c) O[r * to + c] = c < k ? q[c] * inv : 0.f;
  }
  __syncthreads();
  float* dst = Qt + r0 * ldt;
#pragma unroll 4
  for (int e = threadIdx.x; e < rows * ldt; e += kRnRows) {
    const int rr = e / ldt;
    dst[e] = O[rr * to + (e - rr * ldt)];
  }
}

// row-normalised copy: tiled for the library's own blocks, a thread per row
// for a caller's block of any stride
void rownorm(const float* Q, int ldq, int off, int64_t n, int k, float* Qt, int ldt, cudaStream_t s) {
  if (ldq <= 68 && ldt <= 64)
    k_rownorm_tiled<<<(unsigned)ceil_div(n > 0 ? n : 1, (int64_t)kRnRows), kRnRows, 0, s>>>(Q, ldq, off, n, k, Qt, ldt);
  else
    k_rownorm<<<(unsigned)ceil_div(n > 0 ? n : 1, (int64_t)256), 256, 0, s>>>(Q, ldq, off, n, k, Qt, ldt);
}

__global__ void k_disc_init(unsigned int* bar, int32_t* err) {
  if (threadIdx.x == 0) {
    bar[0] = 0;
    bar[1] = 0;
    *err = 0;
  }
}

// Software grid barrier for a cooperative launch (all CTAs co-resident).
// Bounded: on expiry it records the error and returns false.
__device__ bool grid_barrier(unsigned int* bar, int32_t* err) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = bar + 1;
    const unsigned int g = *gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(bar, 1u) + 1u;
    int ok = 1;
    if (arrived == gridDim.x) {
      bar[0] = 0;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        if (clock64() - t0 > 4000000000LL || *(volatile int32_t*)err) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// One-sided Jacobi SVD (Hestenes) of the k x k matrix A in FP32, stored by
// columns (column stride lda, kp = k rounded up to even columns, a padding
// column is zero); V (kp x kp, by columns) accumulates the rotations, so
// A V = U Sigma on return.  Round-robin pair schedule, one warp per pair,
// lanes over rows (consecutive addresses).  Returns the number of sweeps.
__device__ int jacobi_svd_f32(float* A, float* V, int k, int kp, int lda, int* rotated) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // rotation threshold on |a_p . a_q| / (|a_p| |a_q|): above the rounding
  // level of a k-term FP32 dot product, so the sweeps end
  const float tol = fmaxf(1e-6f, 2.f * (float)k * 5.9604645e-8f);
  for (int e = threadIdx.x; e < kp * lda; e += blockDim.x) V[e] = (e / lda == e % lda) ? 1.f : 0.f;
  __syncthreads();
  int sweep = 0;
  for (; sweep < 60; ++sweep) {
    if (threadIdx.x == 0) *rotated = 0;
    __syncthreads();
    for (int r = 0; r < kp - 1; ++r) {
      for (int pr = wp; pr < kp / 2; pr += nw) {
        int p, q;
        if (pr == 0) {
          p = kp - 1;
          q = r;
        } else {
          p = (r + pr) % (kp - 1);
          q = (r - pr + kp - 1) % (kp - 1);
        }
        float* ap = A + p * lda;
        float* aq = A + q * lda;
        float al = 0.f, be = 0.f, ga = 0.f;
        for (int row = lane; row < k; row += 32) {
          const float x = ap[row], y = aq[row];
          al = fmaf(x, x, al);
          be = fmaf(y, y, be);
          ga = fmaf(x, y, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (al > 0.f && be > 0.f && fabsf(ga) > tol * sqrtf(al * be)) {
          const float zeta = (be - al) / (2.f * ga);
          const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
          const float cs = rsqrtf(1.f + t * t), sn = cs * t;
          for (int row = lane; row < k; row += 32) {
            const float x = ap[row], y = aq[row];
            ap[row] = cs * x - sn * y;
            aq[row] = sn * x + cs * y;
          }
          float* vp = V + p * lda;
          float* vq = V + q * lda;
          for (int row = lane; row < kp; row += 32) {
            const float x = vp[row], y = vq[row];
            vp[row] = cs * x - sn * y;
            vq[row] = sn * x + cs * y;
          }
          if (lane == 0) *rotated = 1;
        }
        __syncwarp();
      }
      __syncthreads();
    }
    if (!*rotated) break;
    __syncthreads();
  }
  return sweep;
}

// R = V U^T from M = U Omega V^T by Jacobi (M row-major in M, stride
// kDiscLd), with U completed to an orthonormal basis where Omega has zero
// entries (empty clusters).  A, V, u: scratch.  R goes to Rs (stride ldr).
// Returns the number of sweeps.
__device__ int polar_jacobi(const float* M, int k, float* A, float* V, float* u, float* Rs, int ldr, int* rotated) {
  __shared__ float sig[64];
  const int kp = (k + 1) & ~1;
  for (int e = threadIdx.x; e < kp * kDiscLd; e += blockDim.x) {
    const int c = e / kDiscLd, l = e % kDiscLd;
    A[e] = (c < k && l < k) ? M[l * kDiscLd + c] : 0.f;
  }
  __syncthreads();
  const int sweeps = jacobi_svd_f32(A, V, k, kp, kDiscLd, rotated);
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    float t = 0.f;
    for (int row = 0; row < k; ++row) t = fmaf(A[c * kDiscLd + row], A[c * kDiscLd + row], t);
    sig[c] = sqrtf(t);
  }
  __syncthreads();
  float smax = 0.f;
  for (int c = 0; c < k; ++c) smax = fmaxf(smax, sig[c]);
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int c = e / k, row = e % k;
    const float sc = sig[c];
    A[c * kDiscLd + row] = (sc > 1e-6f * smax && sc > 0.f) ? A[c * kDiscLd + row] / sc : 0.f;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // rank-deficient M: complete U to an orthonormal basis (Gram-Schmidt of
    // unit vectors, twice, against the columns already set)
    for (int c = 0; c < k; ++c) {
      if (sig[c] > 1e-6f * smax && sig[c] > 0.f) continue;
      for (int cand = 0; cand < k; ++cand) {
        for (int row = 0; row < k; ++row) u[row] = (row == cand) ? 1.f : 0.f;
        for (int rep = 0; rep < 2; ++rep)
          for (int o = 0; o < k; ++o) {
            if (o == c) continue;
            float dot = 0.f;
            for (int row = 0; row < k; ++row) dot = fmaf(A[o * kDiscLd + row], u[row], dot);
            for (int row = 0; row < k; ++row) u[row] -= dot * A[o * kDiscLd + row];
          }
        float nn = 0.f;
        for (int row = 0; row < k; ++row) nn = fmaf(u[row], u[row], nn);
        if (nn > 0.25f) {
          nn = rsqrtf(nn);
          for (int row = 0; row < k; ++row) A[c * kDiscLd + row] = u[row] * nn;
          break;
        }
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k * ldr; e += blockDim.x) {  // R[a][b] = sum_j V[a][j] U[b][j]
    const int a = e / ldr, b = e % ldr;
    float t = 0.f;
    if (b < k)
      for (int j = 0; j < k; ++j) t = fmaf(V[j * kDiscLd + a], A[j * kDiscLd + b], t);
    Rs[e] = t;
  }
  __syncthreads();
  return sweeps;
}

// barrier of the first n threads of the CTA (all of them: __syncthreads)
__device__ __forceinline__ void ns_sync(int nthr) {
  if (nthr == (int)blockDim.x)
    __syncthreads();
  else
    asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory");
}

// R = polar(M)^T by the Newton-Schulz iteration X <- X (3I - X^T X) / 2 from
// X = M / s, s >= ||M||_2 (min of the Frobenius norm and sqrt(||M||_1
// ||M||_inf)); every singular value of X then lies in (0, 1] and converges to
// 1, so X -> U V^T for M = U Omega V^T.  Stops once max |X^T X - I| < tol
// (after one more step).  Returns false (R untouched) if M is zero or the
// iteration has not converged after kNsMaxIter steps.  KM >= k bounds the
// terms of each k x k product so that they are unrolled (terms past k
// predicated off) and their shared-memory loads overlap; the largest
// deviation of each step is left per warp and read back after the barrier.
template <int KM>
__device__ bool polar_newton_schulz(const float* M, int k, float* X, float* Xn, float* P, float* Rs, int ldr) {
  __shared__ float rsum[64], csum[64], f2s[64];
  __shared__ float wdl[2][kDiscThreads / 32];
  __shared__ float scale_s;
  __shared__ int conv_s;
  const int kk = k * k;
  if (threadIdx.x < k) {  // row / column absolute sums and squared row norms
    float rs = 0.f, cs = 0.f, f2 = 0.f;
    for (int c = 0; c < k; ++c) {
      const float x = M[threadIdx.x * kDiscLd + c];
      rs += fabsf(x);
      cs += fabsf(M[c * kDiscLd + threadIdx.x]);
      f2 = fmaf(x, x, f2);
    }
    rsum[threadIdx.x] = rs;
    csum[threadIdx.x] = cs;
    f2s[threadIdx.x] = f2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float n1 = 0.f, ninf = 0.f, fro2 = 0.f;
    for (int l = 0; l < k; ++l) {
      ninf = fmaxf(ninf, rsum[l]);
      n1 = fmaxf(n1, csum[l]);
      fro2 += f2s[l];
    }
    const float s = fminf(sqrtf(fro2), sqrtf(n1 * ninf));
    scale_s = (s > 0.f && isfinite(s)) ? 1.f / s : 0.f;
  }
  __syncthreads();
  const float inv = scale_s;
  if (inv == 0.f) return false;
  const float tol = 1e-6f + 8.f * (float)k * 5.9604645e-8f;
  for (int e = threadIdx.x; e < kk; e += blockDim.x) {
    const int r = e / k, c = e % k;
    X[r * kDiscLd + c] = M[r * kDiscLd + c] * inv;
  }
  __syncthreads();
  // small matrices run on the first 128 threads behind named barrier 1 (the
  // other warps wait at the closing __syncthreads); larger ones on the CTA
  const int nthr = kk <= 128 ? 128 : (int)blockDim.x;
  const int nw = nthr >> 5;
  if ((int)threadIdx.x < nthr) {
    bool conv = false;
    for (int t = 0; t < kNsMaxIter; ++t) {
      float dl = 0.f;
      for (int e = threadIdx.x; e < kk; e += nthr) {  // P = X^T X
        const int a = e / k, b = e % k;
        float p = 0.f;
#pragma unroll
        for (int r = 0; r < KM; ++r)
          if (r < k) p = fmaf(X[r * kDiscLd + a], X[r * kDiscLd + b], p);
        P[a * kDiscLd + b] = p;
        const float dv = fabsf(p - (a == b ? 1.f : 0.f));
        dl = (dv == dv) ? fmaxf(dl, dv) : INFINITY;  // a NaN never converges
      }
      for (int off = 16; off >= 1; off >>= 1) dl = fmaxf(dl, __shfl_xor_sync(0xffffffffu, dl, off));
      if ((threadIdx.x & 31) == 0) wdl[t & 1][threadIdx.x >> 5] = dl;
      ns_sync(nthr);
      for (int e = threadIdx.x; e < kk; e += nthr) {  // X' = 1.5 X - 0.5 X P
        const int r = e / k, b = e % k;
        float s = 0.f;
#pragma unroll
        for (int a = 0; a < KM; ++a)
          if (a < k) s = fmaf(X[r * kDiscLd + a], P[a * kDiscLd + b], s);
        Xn[r * kDiscLd + b] = fmaf(-0.5f, s, 1.5f * X[r * kDiscLd + b]);
      }
      ns_sync(nthr);
      float* tmp = X;
      X = Xn;
      Xn = tmp;
      float dmax = 0.f;
#pragma unroll
      for (int q = 0; q < kDiscThreads / 32; ++q) dmax = fmaxf(dmax, q < nw ? wdl[t & 1][q] : 0.f);
      if (dmax < tol) {
        conv = true;
        break;
      }
    }
    if (conv)
      for (int e = threadIdx.x; e < k * ldr; e += nthr) {  // R = X^T
        const int a = e / ldr, b = e % ldr;
        Rs[e] = b < k ? X[b * kDiscLd + a] : 0.f;
      }
    if (threadIdx.x == 0) conv_s = conv ? 1 : 0;
  }
  __syncthreads();
  return conv_s != 0;
}

// Fixed-point scale of the cluster sums in Discretize: |q| <= 1 for a
// row-normalised Q~, so n < 2^31 rows of 2^31-scaled entries cannot overflow
// an int64, and integer sums are exact in any order (the totals do not
// depend on how the rows are split between CTAs).  Rounding each entry costs
// at most 2^-32, far below FP32's resolution of M.
constexpr float kDiscFix = 2147483648.0f;
constexpr double kDiscFixInv = 1.0 / 2147483648.0;

// Y = argmax(Q~ R) for the rows of one staged tile, a register-blocked
// product.  The tile is staged row-major (row stride kDiscLds, 16-byte
// aligned); lane (row group g, column group cg) of warp w computes rows
// 16 w + g + 4 i (i = 0..3) x columns cg CPC .. cg CPC + CPC - 1 (CPC =
// ldr / 8: eight lanes span the padded columns of R), four features a at a
// time: four 16-byte loads of Q~ and 4 CPC / 2 8-byte loads of R feed
// 16 CPC FMAs.  Per lane the columns are visited in ascending order with
// strict ">", and across the eight lanes the lower column wins equal
// scores: ties go to the lowest column.  Features past k are zero in Q~
// and rows past k of R are zero.
constexpr int kDiscTR = 256;  // rows per tile
constexpr int kDiscLds = 68;  // row stride of the staged tile: 64 features + 4 (bank offset 4 rows apart)
template <int CPC>
__device__ __forceinline__ void disc_argmax_tile(const float* __restrict__ tile, int rows, const float* __restrict__ Rs,
                                                 int ldr, int k4, int k, int64_t tb, int32_t* __restrict__ labels,
                                                 int32_t* __restrict__ labt) {
  const int lane = threadIdx.x & 31, cg = lane & 7;
  const int rbase = 16 * (threadIdx.x >> 5) + (lane >> 3);  // rows rbase + 4 i
  const int c0 = cg * CPC;
  float acc[4][CPC];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < CPC; ++j) acc[i][j] = 0.f;
  for (int a = 0; a < k4; a += 4) {
    float4 q[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) q[i] = *reinterpret_cast<const float4*>(tile + (rbase + 4 * i) * kDiscLds + a);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      float rv[CPC];
#pragma unroll
      for (int j = 0; j < CPC; j += 2) {
        const float2 t = *reinterpret_cast<const float2*>(Rs + (a + u) * ldr + c0 + j);
        rv[j] = t.x;
        rv[j + 1] = t.y;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float x = u == 0 ? q[i].x : u == 1 ? q[i].y : u == 2 ? q[i].z : q[i].w;
#pragma unroll
        for (int j = 0; j < CPC; ++j) acc[i][j] = fmaf(x, rv[j], acc[i][j]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float best = -INFINITY;
    int bc = 0x7fffffff;
#pragma unroll
    for (int j = 0; j < CPC; ++j)
      if (c0 + j < k && acc[i][j] > best) {
        best = acc[i][j];
        bc = c0 + j;
      }
#pragma unroll
    for (int off = 1; off <= 4; off <<= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, off);
      const int oc = __shfl_xor_sync(0xffffffffu, bc, off);
      if (ob > best || (ob == best && oc < bc)) {
        best = ob;
        bc = oc;
      }
    }
    const int r = rbase + 4 * i;
    if (cg == 0 && r < rows) {
      if (bc == 0x7fffffff) bc = 0;  // a NaN row
      labels[tb + r] = bc;
      labt[r] = bc;
    }
  }
}

// Discretize (Def. 2, Alg. 5) as one persistent cooperative kernel.  Per
// iteration:
//  A. every CTA takes a contiguous row range in tiles staged in shared
//     memory (the next tile prefetched to L2), sets Y = argmax(Q~ R) (ties
//     to the lowest column), orders the tile's rows by cluster (stable) and
//     adds each cluster's rows (FP32, in order) to its sums in fixed point
//     (exact int64), with its cluster sizes;
//  R. after a grid barrier the CTAs total the per-CTA sums, one warp per
//     entry (exact int64);
//  B. after a second barrier every CTA forms M = Y~^T Q~ (the totals over
//     the cluster sizes), takes R = V U^T for M = U Omega V^T (Newton-Schulz,
//     or Jacobi for rank-deficient M) and obj = n - 2 tr(Omega), and stops
//     once |obj - obj_prev| <= 4 eps max(1, |obj|).  All CTAs compute the
//     same R and the same decision from the same totals.
__global__ void __launch_bounds__(kDiscThreads, 2)  // <= 64 registers: half an SM's file, room for the hops' blocks
k_discretize(const float* __restrict__ Qt, int ldt, int64_t n, int k, int max_iter, int32_t* __restrict__ labels,
             DiscState st, int32_t* __restrict__ iters_out, int32_t* __restrict__ flags) {
  extern __shared__ __align__(16) float dsm_f[];
  __shared__ int32_t hist[64];
  __shared__ int32_t cnt_s[64];
  __shared__ double trl[64];
  __shared__ int rotated;
  __shared__ int done_s;
  const int tid = threadIdx.x;
  const int kk = k * k;
  const int ldr = (k + 15) & ~15;
  constexpr int TR = kDiscTR;
  static_assert(2 * TR <= kDiscLabels, "tile labels and order");
  static_assert(kDiscThreads * 4 == TR * 8, "four rows x eight column lanes per tile row group");
  static_assert(TR * kDiscLds <= kDiscRegion && 4 * 64 * kDiscLd <= kDiscRegion, "staged tile, phase B");
  __shared__ int32_t wcnt[TR / 32][64];
  __shared__ int32_t seg0[64], segn[64];
  float* region = dsm_f;
  int32_t* labt = reinterpret_cast<int32_t*>(dsm_f + kDiscRegion);
  int32_t* ordt = labt + TR;
  unsigned long long* sMi = reinterpret_cast<unsigned long long*>(dsm_f + kDiscRegion + kDiscLabels);
  float* Rs = dsm_f + kDiscRegion + kDiscLabels + kDiscSlices;
  const int64_t per = ceil_div(n, (int64_t)gridDim.x);
  const int64_t r0 = (int64_t)blockIdx.x * per;
  const int64_t r1 = (r0 + per < n) ? r0 + per : n;
  const int nv4 = ldt / 4;
  const int cpc = ldr >> 3;  // columns per lane in the argmax: 2, 4, 6 or 8
  const int wid = tid >> 5, lane = tid & 31;
  // R = I; rows k .. ldt - 1 stay zero (the argmax reads R four rows at a time)
  for (int e = tid; e < ldt * ldr; e += blockDim.x) Rs[e] = (e / ldr == e % ldr && e / ldr < k) ? 1.f : 0.f;
  double obj_prev = 0.0;
  for (int it = 0; it < max_iter; ++it) {
    // ---------------- phase A ----------------------------------------------
    for (int e = tid; e < 64; e += blockDim.x) hist[e] = 0;
    for (int e = tid; e < kk; e += blockDim.x) sMi[e] = 0ull;
    __syncthreads();
    for (int64_t tb = r0; tb < r1; tb += TR) {
      const int rows = (int)((r1 - tb) < TR ? (r1 - tb) : TR);
      {  // row-major, coalesced: float4 j of row r; all of a thread's loads
         // (at most 8: nv4 <= 16) are issued first; rows past the range are zero
        constexpr int kLd = kDiscTR * 16 / kDiscThreads;
        const float4* src = reinterpret_cast<const float4*>(Qt + tb * ldt);
        float4 v[kLd];
#pragma unroll
        for (int u = 0; u < kLd; ++u) {
          const int e = tid + u * kDiscThreads;
          const int r = e / nv4;
          v[u] = (r < rows) ? src[e] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kLd; ++u) {
          const int e = tid + u * kDiscThreads;
          const int r = e / nv4, j = e - r * nv4;
          if (r < TR) *reinterpret_cast<float4*>(region + r * kDiscLds + 4 * j) = v[u];
        }
      }
      for (int e = tid; e < (TR / 32) * 64; e += blockDim.x) (&wcnt[0][0])[e] = 0;
      {  // the next tile of this CTA's rows towards L2 while this one is scored
        const int64_t nb = tb + TR;
        const int64_t nrows = nb < r1 ? ((r1 - nb) < TR ? (r1 - nb) : TR) : 0;
        const int64_t lines = (nrows * ldt * 4 + 127) / 128;
        if (tid < lines) {
          const char* pf = reinterpret_cast<const char*>(Qt + nb * ldt) + 128 * tid;
          asm volatile("prefetch.global.L2 [%0];" ::"l"(pf));
        }
      }
      __syncthreads();
      if (cpc <= 2) disc_argmax_tile<2>(region, rows, Rs, ldr, ldt, k, tb, labels, labt);
      else if (cpc == 4) disc_argmax_tile<4>(region, rows, Rs, ldr, ldt, k, tb, labels, labt);
      else if (cpc == 6) disc_argmax_tile<6>(region, rows, Rs, ldr, ldt, k, tb, labels, labt);
      else disc_argmax_tile<8>(region, rows, Rs, ldr, ldt, k, tb, labels, labt);
      __syncthreads();
      // the tile's rows in a stable order by cluster: warp ranks (a match on
      // the label), per-cluster prefixes over the warps, cluster offsets
      int lr = 64, rk = 0;
      if (tid < TR) {
        const bool v = tid < rows;
        lr = v ? labt[tid] : 64;
        const unsigned peers = __match_any_sync(0xffffffffu, lr);
        rk = __popc(peers & ((1u << lane) - 1u));
        if (v && rk == 0) wcnt[wid][lr] = __popc(peers);
      }
      __syncthreads();
      if (wid == 0) {  // lane owns clusters lane and lane + 32: prefixes over the warps, then a scan
        int tot[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int l = lane + 32 * h;
          int acc = 0;
          if (l < k) {
#pragma unroll
            for (int w = 0; w < TR / 32; ++w) {
              const int c = wcnt[w][l];
              wcnt[w][l] = acc;
              acc += c;
            }
            segn[l] = acc;
            hist[l] += acc;
          }
          tot[h] = acc;
        }
        int base = 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          int inc = tot[h];
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
          }
          if (lane + 32 * h < k) seg0[lane + 32 * h] = base + inc - tot[h];
          base += __shfl_sync(0xffffffffu, inc, 31);
        }
      }
      __syncthreads();
      if (tid < rows) ordt[seg0[lr] + wcnt[wid][lr] + rk] = tid;
      __syncthreads();
      // cluster sums: thread e owns entry (l, c) = (e / k, e % k) of the k x k
      // sums for the whole call; a tile adds its rows of cluster l in order
      // (FP32), then the tile's sum in fixed point (exact int64)
      for (int e = tid; e < kk; e += blockDim.x) {
        const int l = e / k, c = e - l * k;
        const int b = seg0[l], m = segn[l];
        if (m == 0) continue;
        const float* col = region + c;
        float s4[4] = {0.f, 0.f, 0.f, 0.f};  // four interleaved partial sums, combined in a fixed order
        int q = 0;
        for (; q + 4 <= m; q += 4) {
          const int i0 = ordt[b + q], i1 = ordt[b + q + 1], i2 = ordt[b + q + 2], i3 = ordt[b + q + 3];
          s4[0] += col[i0 * kDiscLds];
          s4[1] += col[i1 * kDiscLds];
          s4[2] += col[i2 * kDiscLds];
          s4[3] += col[i3 * kDiscLds];
        }
        for (; q < m; ++q) s4[q & 3] += col[ordt[b + q] * kDiscLds];
        const float sum = (s4[0] + s4[1]) + (s4[2] + s4[3]);
        sMi[e] += (unsigned long long)__float2ll_rn(sum * kDiscFix);
      }
      __syncthreads();
    }
    for (int e = tid; e < kk; e += blockDim.x) st.part[(int64_t)blockIdx.x * kk + e] = (long long)sMi[e];
    for (int e = tid; e < k; e += blockDim.x) st.partc[(int64_t)blockIdx.x * k + e] = hist[e];
    if (!grid_barrier(st.bar, st.err)) return;
    // ---------------- phase R: totals, one warp per entry ------------------
    {
      const int nw = blockDim.x >> 5, wid = tid >> 5, lane = tid & 31;
      for (int e = blockIdx.x * nw + wid; e < kk + k; e += gridDim.x * nw) {
        if (e < kk) {
          long long t = 0;
          for (int b = lane; b < (int)gridDim.x; b += 32) t += __ldcg(st.part + (int64_t)b * kk + e);
          for (int off = 16; off >= 1; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
          if (lane == 0) st.S[e] = t;
        } else {
          int c = 0;
          for (int b = lane; b < (int)gridDim.x; b += 32) c += __ldcg(st.partc + (int64_t)b * k + (e - kk));
          for (int off = 16; off >= 1; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
          if (lane == 0) st.cnt[e - kk] = c;
        }
      }
    }
    if (!grid_barrier(st.bar, st.err)) return;
    // ---------------- phase B: every CTA, same result ----------------------
    float* M = region;
    for (int e = tid; e < k; e += blockDim.x) cnt_s[e] = __ldcg(st.cnt + e);
    __syncthreads();
    for (int e = tid; e < kk; e += blockDim.x) {
      const int l = e / k, c = e % k;
      const long long v = __ldcg(st.S + e);
      const int cl = cnt_s[l];
      M[l * kDiscLd + c] = cl > 0 ? (float)((double)v * kDiscFixInv / (double)cl) : 0.f;
    }
    __syncthreads();
    bool empty = false;
    for (int c = 0; c < k; ++c) empty |= cnt_s[c] == 0;
    int sweeps = 0;
    bool ok = false;
    if (!empty) {
      float* X0 = region + kDiscLd * 64;
      float* X1 = region + 2 * kDiscLd * 64;
      float* P0 = region + 3 * kDiscLd * 64;
      ok = k <= 16   ? polar_newton_schulz<16>(M, k, X0, X1, P0, Rs, ldr)
           : k <= 32 ? polar_newton_schulz<32>(M, k, X0, X1, P0, Rs, ldr)
           : k <= 48 ? polar_newton_schulz<48>(M, k, X0, X1, P0, Rs, ldr)
                     : polar_newton_schulz<64>(M, k, X0, X1, P0, Rs, ldr);
    }
    if (!ok)
      sweeps = polar_jacobi(M, k, region + kDiscLd * 64, region + 2 * kDiscLd * 64, region + 3 * kDiscLd * 64, Rs,
                            ldr, &rotated);
    // tr(Omega) = tr(M R), rows in FP64, summed in order
    for (int l = tid; l < k; l += blockDim.x) {
      double t = 0.0;
      for (int c = 0; c < k; ++c) t += (double)M[l * kDiscLd + c] * (double)Rs[c * ldr + l];
      trl[l] = t;
    }
    __syncthreads();
    if (tid == 0) {
      double tr = 0.0;
      for (int l = 0; l < k; ++l) tr += trl[l];
      const double obj = (double)n - 2.0 * tr;
      int dn = 0;
      if (it > 0 && fabs(obj - obj_prev) <= 4.0 * 2.220446049250313e-16 * fmax(1.0, fabs(obj))) dn = 1;
      if (it + 1 >= max_iter) dn = 1;
      obj_prev = obj;
      done_s = dn;
      if (blockIdx.x == 0) {
        if (iters_out) *iters_out = it + 1;
        if (flags) {
          if (empty) atomicOr(flags, 1);
          if (sweeps >= 60) atomicOr(flags, 2);
        }
      }
    }
    __syncthreads();
    if (done_s) break;
  }
}

// Diagnostic: R = V U^T for one k x k matrix M = U Omega V^T (row-major,
// stride k) by the routines of k_discretize's phase B -- Newton-Schulz, or
// the Jacobi SVD when a row of M is zero (an empty cluster) or the iteration
// does not settle.  One CTA; method = 0 (Newton-Schulz) or 1 (Jacobi).
__global__ void __launch_bounds__(kDiscThreads) k_polar_diag(const float* __restrict__ Min, int k,
                                                             float* __restrict__ Rout, int32_t* __restrict__ method) {
  extern __shared__ __align__(16) float dsm_f[];
  __shared__ int rotated;
  __shared__ int zero_row;
  const int ldr = (k + 15) & ~15;
  float* M = dsm_f;
  float* X0 = M + kDiscLd * 64;
  float* X1 = M + 2 * kDiscLd * 64;
  float* P0 = M + 3 * kDiscLd * 64;
  float* Rs = M + 4 * kDiscLd * 64;
  if (threadIdx.x == 0) zero_row = 0;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) M[(e / k) * kDiscLd + e % k] = Min[e];
  for (int e = threadIdx.x; e < k * ldr; e += blockDim.x) Rs[e] = (e / ldr == e % ldr) ? 1.f : 0.f;
  __syncthreads();
  for (int l = threadIdx.x; l < k; l += blockDim.x) {
    bool z = true;
    for (int c = 0; c < k; ++c) z &= M[l * kDiscLd + c] == 0.f;
    if (z) atomicOr(&zero_row, 1);
  }
  __syncthreads();
  bool ok = false;
  if (!zero_row)
    ok = k <= 16   ? polar_newton_schulz<16>(M, k, X0, X1, P0, Rs, ldr)
         : k <= 32 ? polar_newton_schulz<32>(M, k, X0, X1, P0, Rs, ldr)
         : k <= 48 ? polar_newton_schulz<48>(M, k, X0, X1, P0, Rs, ldr)
                   : polar_newton_schulz<64>(M, k, X0, X1, P0, Rs, ldr);
  if (!ok) polar_jacobi(M, k, X0, X1, P0, Rs, ldr, &rotated);
  __syncthreads();
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) Rout[e] = Rs[(e / k) * ldr + e % k];
  if (threadIdx.x == 0) *method = ok ? 0 : 1;
}

// ---------------------------------------------------------------------------
// labels -> counts, 1/sqrt(count), one-hot fills, trace, keep-best
// ---------------------------------------------------------------------------
__global__ void k_count_labels(const int32_t* __restrict__ labels, int64_t n, int k, int32_t* __restrict__ cnt) {
  __shared__ int32_t hist[64];
  for (int e = threadIdx.x; e < 64; e += blockDim.x) hist[e] = 0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&hist[labels[i]], 1);
  __syncthreads();
  for (int e = threadIdx.x; e < k; e += blockDim.x)
    if (hist[e]) atomicAdd(&cnt[e], hist[e]);
}

__global__ void k_inv_sqrt_counts(const int32_t* __restrict__ cnt, int k, float* __restrict__ inv) {
  const int c = threadIdx.x;
  if (c < k) inv[c] = cnt[c] > 0 ? (float)(1.0 / sqrt((double)cnt[c])) : 0.f;
}

// splitmix64 (Steele, Lea, Flood 2014): one output for state x
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Q^(0) = [n^-1/2 1 | h(Y^(0))] (col_off = 1) or F^(0) = alpha h(Y) (col_off = 0).
// [n^-1/2 1 | h(Y)] has rank k only (1 = sum_c sqrt|C_c| h(Y)_c, and an empty
// cluster gives a zero column), so the QR would be undefined: the column of
// the highest-index non-empty cluster and of every empty cluster c becomes
// the sign vector +-n^-1/2 from the top bit of splitmix64(64 i + c), which
// keeps span(h(Y)) and gives Q^(0) full rank.
__global__ void k_fill_onehot(const int32_t* __restrict__ labels, const float* __restrict__ inv,
                              const int32_t* __restrict__ cnt, int k, int64_t n, int ld, int col_off,
                              float first_col, float scale, float* __restrict__ out,
                              const int32_t* __restrict__ names = nullptr) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * ld) return;
  const int64_t i = t / ld;
  const int c = (int)(t % ld);
  float v = 0.f;
  if (col_off == 1 && c == 0) v = first_col;
  const int y = labels[i];
  if (c == y + col_off) v = scale * inv[y];
  if (col_off == 1 && c >= 1 && c <= k) {
    int last = 0;
    for (int q = 0; q < k; ++q)
      if (cnt[q] > 0) last = q;
    if (cnt[c - 1] == 0 || c - 1 == last)
      v = (splitmix64((uint64_t)(names ? names[i] : i) * 64u + (uint64_t)(c - 1)) >> 63) ? -first_col : first_col;
  }
  out[t] = v;
}

// per-CTA partial of tr(Yh^T F) = sum_i inv[y_i] F[i, y_i]
__global__ void k_trace_partial(const float* __restrict__ F, int ld, const int32_t* __restrict__ labels,
                                const float* __restrict__ inv, int64_t n, double* __restrict__ partial) {
  __shared__ double ws[8];
  double s = 0.0;
  const int64_t per = ceil_div(n, (int64_t)gridDim.x);
  const int64_t r0 = (int64_t)blockIdx.x * per;
  const int64_t r1 = (r0 + per < n) ? r0 + per : n;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    const int y = labels[i];
    s += (double)inv[y] * (double)F[i * ld + y];
  }
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    partial[blockIdx.x] = t;
  }
}

// phi = 1 - tr / k; keep-best decision (strictly lower phi wins)
__global__ void k_phi_decide(const double* __restrict__ partial, int nblk, int k, double* __restrict__ phi_slot,
                             double* __restrict__ phi_best, int32_t* __restrict__ take,
                             int32_t* __restrict__ taken_slot, int first) {
  if (threadIdx.x != 0) return;
  double t = 0.0;
  for (int b = 0; b < nblk; ++b) t += partial[b];
  const double phi = 1.0 - t / (double)k;
  *phi_slot = phi;
  int tk = first ? 1 : (phi < *phi_best ? 1 : 0);
  if (tk) *phi_best = phi;
  *take = tk;
  if (taken_slot) *taken_slot = first ? 0 : tk;
}

__global__ void k_copy_if(const int32_t* __restrict__ take, const int32_t* __restrict__ src,
                          int32_t* __restrict__ dst, int64_t n) {
  if (!*take) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i];
}

// row argmax (InitBCM g(v) of Eq. argmaxlabel), ties to the lowest column
__global__ void k_argmax_rows(const float* __restrict__ P, int ld, int64_t n, int k, int32_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* p = P + i * ld;
  float b = p[0];
  int bc = 0;
  for (int c = 1; c < k; ++c)
    if (p[c] > b) {
      b = p[c];
      bc = c;
    }
  out[i] = bc;
}

// V_c: keys (UINT32_MAX - degree, id) sorted ascending; the first k ids,
// re-sorted by id, become the centres (reading R7)
__global__ void k_degree_keys(const int32_t* __restrict__ deg, int64_t n, uint64_t* __restrict__ keys) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) keys[i] = ((uint64_t)(0xffffffffu - (uint32_t)deg[i]) << 32) | (uint32_t)i;
}

__global__ void k_seed_setup(const uint64_t* __restrict__ sorted, int k, int32_t* __restrict__ seedcol) {
  if (threadIdx.x != 0) return;
  int32_t ids[64];
  for (int r = 0; r < k; ++r) ids[r] = (int32_t)(sorted[r] & 0xffffffffull);
  for (int a = 1; a < k; ++a) {
    int32_t v = ids[a];
    int b = a - 1;
    while (b >= 0 && ids[b] > v) {
      ids[b + 1] = ids[b];
      --b;
    }
    ids[b + 1] = v;
  }
  for (int r = 0; r < k; ++r) seedcol[ids[r]] = r;
}

__global__ void k_fill_seed(const int32_t* __restrict__ seedcol, int64_t n, int ld, float alpha,
                            float* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * ld) return;
  const int64_t i = t / ld;
  const int c = (int)(t % ld);
  out[t] = (seedcol[i] == c) ? alpha : 0.f;
}

// ---------------------------------------------------------------------------
// host-side helpers
// ---------------------------------------------------------------------------
struct Ctx {
  const Walk& w;
  int64_t n;
  int k, ld, ldk;
  float alpha;
  float* E;       // hypergraph edge buffer (m x max(ld, ldk))
  cudaStream_t s;
  LongRows lr_walk;   // (topo, knn): Eq. zt node side
  LongRows lr_edges;  // (edges): hypergraph hyperedge side
  LongRows lr_topo;   // (topo): InitBCM node side
};

// Z = P Q (Eq. zt); with oh_labels: Z = coef P Q + oh_coef h(Y)
ancka_status apply_walk(const Ctx& c, const float* Q, int ld, float* Z, float coef,
                        const int32_t* oh_labels, const float* oh_inv, float oh_coef) {
  const Walk& w = c.w;
  SpmmArgs a;
  a.nv4 = ld / 4;
  a.nrows = c.n;
  a.ldo = ld;
  a.out = Z;
  a.coef = coef;
  a.oh_col = oh_labels;
  a.oh_scale = oh_inv;
  a.oh_coef = oh_coef;
  a.ptrB = w.knn.ptr;
  a.colB = w.knn.col;
  a.valB = w.knn.val;
  a.srcB = Q;
  a.ldB = ld;
  if (w.kind == ANCKA_HYPERGRAPH) {
    SpmmArgs e;
    e.ptrA = w.edges.ptr;
    e.colA = w.edges.col;
    e.rsA = w.inv_size;
    e.srcA = Q;
    e.srcA_rows = c.n;
    e.ldA = ld;
    e.out = c.E;
    e.ldo = ld;
    e.nrows = w.m;
    e.nv4 = ld / 4;
    e.long_rows = c.lr_edges.rows;
    e.n_long = c.lr_edges.count;
    e.n_long_host = c.lr_edges.count_host;

    e.long_items = c.lr_edges.items;

    e.long_off = c.lr_edges.off;

    e.n_items_host = c.lr_edges.items_host;
    e.long_min = c.lr_edges.min_entries;
    e.mean_entries = c.lr_edges.mean;
    ANCKA_TRY(spmm(e, c.s));
    a.ptrA = w.topo.ptr;
    a.colA = w.topo.col;
    a.rsA = w.rs_topo;
    a.srcA = c.E;
    a.srcA_rows = w.m;
    a.ldA = ld;
  } else {
    a.ptrA = w.topo.ptr;
    a.colA = w.topo.col;
    a.valA = w.row_uniform ? nullptr : w.topo.val;  // one layer: 1/delta_i is inside rs_topo
    a.rsA = w.rs_topo;
    a.srcA = Q;
    a.srcA_rows = c.n;
    a.ldA = ld;
  }
  a.srcB_rows = c.n;
  a.long_rows = c.lr_walk.rows;
  a.n_long = c.lr_walk.count;
  a.n_long_host = c.lr_walk.count_host;

  a.long_items = c.lr_walk.items;

  a.long_off = c.lr_walk.off;

  a.n_items_host = c.lr_walk.items_host;
  a.long_min = c.lr_walk.min_entries;
  a.mean_entries = c.lr_walk.mean;
  return spmm(a, c.s);
}

// Pi^T <- (1 - alpha) P_N^T Pi^T + alpha Z_0^T  (one InitBCM hop)
}  // namespace

// out = P_N U for an n x ld block U (Eqs. rw-hg, rw-ag, rw-mg: the topology
// walk alone, no KNN part), in column chunks of at most 64 (the SpMM's
// widest row); ld a multiple of 4, U and out 16-byte aligned.
ancka_status apply_topology(Workspace& ws, const Walk& w, const float* U, int ld, float* out, cudaStream_t s) {
  const bool hyper = w.kind == ANCKA_HYPERGRAPH;
  LongRows lt, le;
  const double ub = (double)(hyper ? w.m : w.n) * (ld < 64 ? ld : 64) * 4.0;
  ANCKA_TRY(find_long_rows(ws, w.topo.ptr, nullptr, w.n, w.topo.nnz, ub, &lt, s));
  float* E = nullptr;
  if (hyper) {
    ANCKA_TRY(find_long_rows(ws, w.edges.ptr, nullptr, w.m, w.edges.nnz, (double)w.n * (ld < 64 ? ld : 64) * 4.0,
                             &le, s));
    ANCKA_TRY(ws.alloc(&E, (size_t)w.m * ld));
  }
  ANCKA_TRY(build_long_items(ws, w.topo.ptr, nullptr, &lt, s));
  if (hyper) ANCKA_TRY(build_long_items(ws, w.edges.ptr, nullptr, &le, s));
  LongRows* lrs[2] = {&lt, &le};
  ANCKA_TRY(read_long_rows(lrs, hyper ? 2 : 1, s));
  for (int c0 = 0; c0 < ld; c0 += 64) {
    const int cw = ld - c0 < 64 ? ld - c0 : 64;
    SpmmArgs a;
    a.nrows = w.n;
    a.nv4 = cw / 4;
    a.out = out + c0;
    a.ldo = ld;
    a.ptrA = w.topo.ptr;
    a.colA = w.topo.col;
    a.ldA = ld;
    a.long_rows = lt.rows;
    a.n_long = lt.count;
    a.n_long_host = lt.count_host;

    a.long_items = lt.items;

    a.long_off = lt.off;

    a.n_items_host = lt.items_host;
    a.long_min = lt.min_entries;
    a.mean_entries = lt.mean;
    if (hyper) {
      SpmmArgs e;  // E = D_E^-1 H U, then P_N U = D_V^-1 H^T E
      e.nrows = w.m;
      e.nv4 = cw / 4;
      e.ptrA = w.edges.ptr;
      e.colA = w.edges.col;
      e.rsA = w.inv_size;
      e.srcA = U + c0;
      e.srcA_rows = w.n;
      e.ldA = ld;
      e.out = E + c0;
      e.ldo = ld;
      e.long_rows = le.rows;
      e.n_long = le.count;
      e.n_long_host = le.count_host;

      e.long_items = le.items;

      e.long_off = le.off;

      e.n_items_host = le.items_host;
      e.long_min = le.min_entries;
      e.mean_entries = le.mean;
      ANCKA_TRY(spmm(e, s));
      a.rsA = w.inv_deg;
      a.srcA = E + c0;
      a.srcA_rows = w.m;
    } else {
      if (w.row_uniform)
        a.rsA = w.inv_deg;
      else
        a.valA = w.topo.val;
      a.srcA = U + c0;
      a.srcA_rows = w.n;
    }
    ANCKA_TRY(spmm(a, s));
  }
  return ANCKA_OK;
}

namespace {

ancka_status initbcm_hop(const Ctx& c, const float* Pi, float* out, const int32_t* seedcol) {
  const Walk& w = c.w;
  SpmmArgs a;
  a.nv4 = c.ldk / 4;
  a.nrows = c.n;
  a.ldo = c.ldk;
  a.out = out;
  a.coef = 1.f - c.alpha;
  a.oh_col = seedcol;
  a.oh_coef = c.alpha;
  if (w.kind == ANCKA_HYPERGRAPH) {
    SpmmArgs e;  // y_e = sum_{v in e} Pi[v] / delta_v
    e.ptrA = w.edges.ptr;
    e.colA = w.edges.col;
    e.csA = w.inv_deg;
    e.srcA = Pi;
    e.srcA_rows = c.n;
    e.ldA = c.ldk;
    e.out = c.E;
    e.ldo = c.ldk;
    e.nrows = w.m;
    e.nv4 = c.ldk / 4;
    e.long_rows = c.lr_edges.rows;
    e.n_long = c.lr_edges.count;
    e.n_long_host = c.lr_edges.count_host;

    e.long_items = c.lr_edges.items;

    e.long_off = c.lr_edges.off;

    e.n_items_host = c.lr_edges.items_host;
    e.long_min = c.lr_edges.min_entries;
    e.mean_entries = c.lr_edges.mean;
    ANCKA_TRY(spmm(e, c.s));
    a.ptrA = w.topo.ptr;  // sum_{e ni i} y_e / |e|
    a.colA = w.topo.col;
    a.csA = w.inv_size;
    a.srcA = c.E;
    a.srcA_rows = w.m;
    a.ldA = c.ldk;
  } else {
    a.ptrA = w.topo.ptr;
    a.colA = w.topo.col;
    if (w.row_uniform)
      a.csA = w.inv_deg;  // P_N^T entry (i, j) = 1/delta_j
    else
      a.valA = w.topo.valT;
    a.srcA = Pi;
    a.srcA_rows = c.n;
    a.ldA = c.ldk;
  }
  a.long_rows = c.lr_topo.rows;
  a.n_long = c.lr_topo.count;
  a.n_long_host = c.lr_topo.count_host;

  a.long_items = c.lr_topo.items;

  a.long_off = c.lr_topo.off;

  a.n_items_host = c.lr_topo.items_host;
  a.long_min = c.lr_topo.min_entries;
  a.mean_entries = c.lr_topo.mean;
  return spmm(a, c.s);
}

struct Scratch {
  int32_t* cnt;        // k
  float* inv;          // k
  float* Fa;
  float* Fb;           // n x ldk
  double* tpart;       // trace partials
  int tblk;
  int32_t* take;       // 1
};

// CalMHC(Y) (Alg. 2): phi into phi_slot, keep-best into best_labels
// The first CalMHC hop, Z = coef P F0 + oh_coef h(Y) with F0 = f0 h(Y)
// (h(Y)[j, c] = inv[c] for c = y_j, else 0), of a graph or multiplex walk:
// row i of P F0 is f0 inv[c] times the sum of P[i, j] over the j with
// y_j = c, so the hop gathers 4-byte labels instead of rows of F0.  A warp
// per row takes 32 entries a round; the lanes holding the same label add
// their weights in lane order (every lane walks the 32 lanes), the lowest of
// them adds the sum to the row's per-cluster total (rounds in order), first
// for the topology part (scaled by the row scale), then for the KNN part.
__global__ void __launch_bounds__(256)
k_walk_onehot(const int64_t* __restrict__ ptrA, const int32_t* __restrict__ colA, const float* __restrict__ valA,
              const float* __restrict__ rsA, const int64_t* __restrict__ ptrB, const int32_t* __restrict__ colB,
              const float* __restrict__ valB, const int32_t* __restrict__ labels, const float* __restrict__ inv,
              int k, int ld, float f0, float coef, float oh_coef, int64_t n, int64_t long_min,
              float* __restrict__ out) {
  __shared__ float acc[8][2][64];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t i = (int64_t)blockIdx.x * 8 + w; i < n; i += (int64_t)gridDim.x * 8) {
    if (long_min > 0 && (ptrA[i + 1] - ptrA[i]) + (ptrB ? ptrB[i + 1] - ptrB[i] : 0) > long_min)
      continue;  // a long row: k_walk_onehot_long
    for (int c = lane; c < 64; c += 32) acc[w][0][c] = acc[w][1][c] = 0.f;
    __syncwarp();
#pragma unroll 1
    for (int part = 0; part < 2; ++part) {
      const int64_t* ptr = part == 0 ? ptrA : ptrB;
      const int32_t* col = part == 0 ? colA : colB;
      const float* val = part == 0 ? valA : valB;
      if (!ptr) continue;
      const int64_t b = ptr[i], e = ptr[i + 1];
      for (int64_t p0 = b; p0 < e; p0 += 32) {
        const int64_t p = p0 + lane;
        int l = 64;
        float wv = 0.f;
        if (p < e) {
          l = labels[col[p]];
          wv = val ? val[p] : 1.f;
        }
        float sum = 0.f;
        bool first = true;  // no lower lane holds this label
#pragma unroll
        for (int src = 0; src < 32; ++src) {
          const int ls = __shfl_sync(0xffffffffu, l, src);
          const float vs = __shfl_sync(0xffffffffu, wv, src);
          if (ls == l) {
            sum += vs;
            if (src < lane) first = false;
          }
        }
        if (l < 64 && first) acc[w][part][l] += sum;
        __syncwarp();
      }
    }
    const int yi = labels[i];
    const float rs = rsA ? rsA[i] : 1.f;
    for (int c = lane; c < ld; c += 32) {
      float z = 0.f;
      if (c < k) {
        z = coef * (f0 * inv[c] * (acc[w][0][c] * rs + acc[w][1][c]));
        if (c == yi) z += oh_coef * inv[c];
      }
      out[i * ld + c] = z;
    }
    __syncwarp();
  }
}

// The same hop for the long rows (more than long_min entries): a CTA per
// row, warp w taking the rounds w, w + 8, ... of each part; the warps'
// per-cluster totals are added in warp order.
__global__ void __launch_bounds__(256)
k_walk_onehot_long(const int32_t* __restrict__ rows, const int64_t* __restrict__ ptrA,
                   const int32_t* __restrict__ colA, const float* __restrict__ valA, const float* __restrict__ rsA,
                   const int64_t* __restrict__ ptrB, const int32_t* __restrict__ colB,
                   const float* __restrict__ valB, const int32_t* __restrict__ labels, const float* __restrict__ inv,
                   int k, int ld, float f0, float coef, float oh_coef, float* __restrict__ out) {
  __shared__ float acc[8][2][64];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t i = rows[blockIdx.x];
  for (int c = lane; c < 64; c += 32) acc[w][0][c] = acc[w][1][c] = 0.f;
  __syncwarp();
#pragma unroll 1
  for (int part = 0; part < 2; ++part) {
    const int64_t* ptr = part == 0 ? ptrA : ptrB;
    const int32_t* col = part == 0 ? colA : colB;
    const float* val = part == 0 ? valA : valB;
    if (!ptr) continue;
    const int64_t b = ptr[i], e = ptr[i + 1];
    for (int64_t p0 = b + 32 * w; p0 < e; p0 += 32 * 8) {
      const int64_t p = p0 + lane;
      int l = 64;
      float wv = 0.f;
      if (p < e) {
        l = labels[col[p]];
        wv = val ? val[p] : 1.f;
      }
      float sum = 0.f;
      bool first = true;
#pragma unroll
      for (int src = 0; src < 32; ++src) {
        const int ls = __shfl_sync(0xffffffffu, l, src);
        const float vs = __shfl_sync(0xffffffffu, wv, src);
        if (ls == l) {
          sum += vs;
          if (src < lane) first = false;
        }
      }
      if (l < 64 && first) acc[w][part][l] += sum;
      __syncwarp();
    }
  }
  __syncthreads();
  const int yi = labels[i];
  const float rs = rsA ? rsA[i] : 1.f;
  for (int c = threadIdx.x; c < ld; c += blockDim.x) {
    float z = 0.f;
    if (c < k) {
      float a0 = 0.f, a1 = 0.f;
      for (int q = 0; q < 8; ++q) {
        a0 += acc[q][0][c];
        a1 += acc[q][1][c];
      }
      z = coef * (f0 * inv[c] * (a0 * rs + a1));
      if (c == yi) z += oh_coef * inv[c];
    }
    out[i * ld + c] = z;
  }
}

// The first orthogonal-iteration hop Z = P Q^(0) of a graph or multiplex
// walk when Q^(0) comes from labels (Alg. 4 line 12 with reading R13):
// column 0 of Q^(0) is n^-1/2, column 1 + c is inv[c] on the rows labelled c
// -- or, for a dependent column (the highest-index non-empty cluster and every
// empty one), the sign vector +-n^-1/2 from the top bit of
// splitmix64(64 name_j + c).  Row i of P Q^(0) needs, per part (topology,
// then KNN): the total of P[i, j], the per-label totals and, per dependent
// column, the signed total -- 4-byte gathers instead of rows of Q^(0).  The
// label totals as in k_walk_onehot; the row and signed totals by a fixed
// xor butterfly per round, added round by round.
struct Q0Cols {
  int ndep;
  int8_t depidx[64];   // index among the dependent columns, or -1
  int32_t dep[64];     // the dependent columns
};

__device__ void q0_columns(const int32_t* __restrict__ cnt, int k, Q0Cols& qc) {
  if (threadIdx.x == 0) {
    int last = 0;
    for (int c = 0; c < k; ++c)
      if (cnt[c] > 0) last = c;
    int nd = 0;
    for (int c = 0; c < k; ++c) {
      if (cnt[c] == 0 || c == last) {
        qc.depidx[c] = (int8_t)nd;
        qc.dep[nd++] = c;
      } else {
        qc.depidx[c] = -1;
      }
    }
    qc.ndep = nd;
  }
  __syncthreads();
}

__device__ __forceinline__ float q0_sign(int64_t name, int c) {
  return (splitmix64((uint64_t)name * 64u + (uint64_t)c) >> 63) ? -1.f : 1.f;
}

// one round of 32 entries [p0, p0 + 32) of row part `part` for warp slot w
__device__ __forceinline__ void q0_round(int64_t p0, int64_t e, const int32_t* __restrict__ col,
                                         const float* __restrict__ val, const int32_t* __restrict__ labels,
                                         const int32_t* __restrict__ names, const Q0Cols& qc,
                                         float (&acc)[64], float (&sgn)[64], float& tot) {
  const int lane = threadIdx.x & 31;
  const int64_t p = p0 + lane;
  int l = 64;
  float wv = 0.f;
  int64_t j = 0;
  if (p < e) {
    j = col[p];
    l = labels[j];
    wv = val ? val[p] : 1.f;
  }
  float sum = 0.f;
  bool first = true;
#pragma unroll
  for (int src = 0; src < 32; ++src) {
    const int ls = __shfl_sync(0xffffffffu, l, src);
    const float vs = __shfl_sync(0xffffffffu, wv, src);
    if (ls == l) {
      sum += vs;
      if (src < lane) first = false;
    }
  }
  if (l < 64 && first) acc[l] += sum;
  float t = wv;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  tot += t;
  const int64_t name = names ? (int64_t)names[j] : j;
  for (int d = 0; d < qc.ndep; ++d) {
    float sv = p < e ? wv * q0_sign(name, qc.dep[d]) : 0.f;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, off);
    if (lane == 0) sgn[d] += sv;
  }
  __syncwarp();
}

__device__ __forceinline__ void q0_write_row(int64_t i, int k, int ld, float c0, float rs, const float* __restrict__ inv,
                                             const Q0Cols& qc, const float* A0, const float* A1, const float* S0,
                                             const float* S1, float T0, float T1, float* __restrict__ out) {
  for (int col = threadIdx.x & 31; col < ld; col += 32) {
    float z = 0.f;
    if (col == 0) {
      z = c0 * (T0 * rs + T1);
    } else if (col <= k) {
      const int c = col - 1, d = qc.depidx[c];
      z = d >= 0 ? c0 * (S0[d] * rs + S1[d]) : inv[c] * (A0[c] * rs + A1[c]);
    }
    out[i * ld + col] = z;
  }
}

__global__ void __launch_bounds__(256)
k_walk_q0(const int64_t* __restrict__ ptrA, const int32_t* __restrict__ colA, const float* __restrict__ valA,
          const float* __restrict__ rsA, const int64_t* __restrict__ ptrB, const int32_t* __restrict__ colB,
          const float* __restrict__ valB, const int32_t* __restrict__ labels, const float* __restrict__ inv,
          const int32_t* __restrict__ cnt, const int32_t* __restrict__ names, int k, int ld, float c0, int64_t n,
          int64_t long_min, float* __restrict__ out) {
  __shared__ Q0Cols qc;
  __shared__ float acc[8][2][64], sgn[8][2][64];
  q0_columns(cnt, k, qc);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t i = (int64_t)blockIdx.x * 8 + w; i < n; i += (int64_t)gridDim.x * 8) {
    if (long_min > 0 && (ptrA[i + 1] - ptrA[i]) + (ptrB ? ptrB[i + 1] - ptrB[i] : 0) > long_min)
      continue;  // a long row: k_walk_q0_long
    for (int c = lane; c < 64; c += 32) acc[w][0][c] = acc[w][1][c] = sgn[w][0][c] = sgn[w][1][c] = 0.f;
    __syncwarp();
    float tot[2] = {0.f, 0.f};
#pragma unroll 1
    for (int part = 0; part < 2; ++part) {
      const int64_t* ptr = part == 0 ? ptrA : ptrB;
      if (!ptr) continue;
      const int64_t e = ptr[i + 1];
      for (int64_t p0 = ptr[i]; p0 < e; p0 += 32)
        q0_round(p0, e, part == 0 ? colA : colB, part == 0 ? valA : valB, labels, names, qc, acc[w][part],
                 sgn[w][part], tot[part]);
    }
    q0_write_row(i, k, ld, c0, rsA ? rsA[i] : 1.f, inv, qc, acc[w][0], acc[w][1], sgn[w][0], sgn[w][1], tot[0],
                 tot[1], out);
    __syncwarp();
  }
}

// the long rows: a CTA per row, warp w taking rounds w, w + 8, ...; the
// warps' totals added in warp order
__global__ void __launch_bounds__(256)
k_walk_q0_long(const int32_t* __restrict__ rows, const int64_t* __restrict__ ptrA, const int32_t* __restrict__ colA,
               const float* __restrict__ valA, const float* __restrict__ rsA, const int64_t* __restrict__ ptrB,
               const int32_t* __restrict__ colB, const float* __restrict__ valB, const int32_t* __restrict__ labels,
               const float* __restrict__ inv, const int32_t* __restrict__ cnt, const int32_t* __restrict__ names,
               int k, int ld, float c0, float* __restrict__ out) {
  __shared__ Q0Cols qc;
  __shared__ float acc[8][2][64], sgn[8][2][64], tots[8][2];
  __shared__ float A[2][64], S[2][64], T[2];
  q0_columns(cnt, k, qc);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t i = rows[blockIdx.x];
  for (int c = lane; c < 64; c += 32) acc[w][0][c] = acc[w][1][c] = sgn[w][0][c] = sgn[w][1][c] = 0.f;
  __syncwarp();
  float tot[2] = {0.f, 0.f};
#pragma unroll 1
  for (int part = 0; part < 2; ++part) {
    const int64_t* ptr = part == 0 ? ptrA : ptrB;
    if (!ptr) continue;
    const int64_t e = ptr[i + 1];
    for (int64_t p0 = ptr[i] + 32 * w; p0 < e; p0 += 32 * 8)
      q0_round(p0, e, part == 0 ? colA : colB, part == 0 ? valA : valB, labels, names, qc, acc[w][part],
               sgn[w][part], tot[part]);
  }
  if (lane == 0) {
    tots[w][0] = tot[0];
    tots[w][1] = tot[1];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 2 * 64; e += blockDim.x) {
    const int part = e >> 6, c = e & 63;
    float a = 0.f, sg = 0.f;
    for (int q = 0; q < 8; ++q) {
      a += acc[q][part][c];
      sg += sgn[q][part][c];
    }
    A[part][c] = a;
    S[part][c] = sg;
  }
  if (threadIdx.x < 2) {
    float t = 0.f;
    for (int q = 0; q < 8; ++q) t += tots[q][threadIdx.x];
    T[threadIdx.x] = t;
  }
  __syncthreads();
  if (w == 0) q0_write_row(i, k, ld, c0, rsA ? rsA[i] : 1.f, inv, qc, A[0], A[1], S[0], S[1], T[0], T[1], out);
}

ancka_status cal_mhc(const Ctx& c, Scratch& sc, const int32_t* labels, int gamma, double* phi_slot,
                     double* phi_best, int32_t* taken_slot, int32_t* best_labels, bool first) {
  cudaStream_t s = c.s;
  ANCKA_CUDA(cudaMemsetAsync(sc.cnt, 0, sizeof(int32_t) * c.k, s));
  k_count_labels<<<grid_for(c.n, 1024) < 304 ? grid_for(c.n, 1024) : 304, 256, 0, s>>>(labels, c.n, c.k, sc.cnt);
  ANCKA_LAUNCHED();
  k_inv_sqrt_counts<<<1, 64, 0, s>>>(sc.cnt, c.k, sc.inv);
  ANCKA_LAUNCHED();
  float* cur = sc.Fa;
  float* nxt = sc.Fb;
  // graphs and multiplex graphs: the first hop from F0 = alpha h(Y) gathers labels
  const bool onehot_hop = c.w.kind != ANCKA_HYPERGRAPH && gamma > 0;
  if (!onehot_hop || gamma == 0) {
    k_fill_onehot<<<grid_for(c.n * c.ldk, 256), 256, 0, s>>>(labels, sc.inv, sc.cnt, c.k, c.n, c.ldk, 0, 0.f,
                                                             c.alpha, sc.Fa);
    ANCKA_LAUNCHED();
  }
  for (int l = 0; l < gamma; ++l) {  // F <- (1 - alpha) P F + alpha h(Y)
    if (l == 0 && onehot_hop) {
      const int64_t blocks = ceil_div(c.n, (int64_t)8);
      const Walk& w = c.w;
      const LongRows& lr = c.lr_walk;  // the walk's long rows (found before the iteration)
      const bool longs = lr.rows && lr.count_host > 0;
      k_walk_onehot<<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, s>>>(
          w.topo.ptr, w.topo.col, w.row_uniform ? nullptr : w.topo.val, w.rs_topo, w.knn.ptr, w.knn.col, w.knn.val,
          labels, sc.inv, c.k, c.ldk, c.alpha, 1.f - c.alpha, c.alpha, c.n, longs ? lr.min_entries : 0, nxt);
      ANCKA_LAUNCHED();
      if (longs) {
        k_walk_onehot_long<<<(unsigned)lr.count_host, 256, 0, s>>>(
            lr.rows, w.topo.ptr, w.topo.col, w.row_uniform ? nullptr : w.topo.val, w.rs_topo, w.knn.ptr, w.knn.col,
            w.knn.val, labels, sc.inv, c.k, c.ldk, c.alpha, 1.f - c.alpha, c.alpha, nxt);
        ANCKA_LAUNCHED();
      }
      float* t = cur;
      cur = nxt;
      nxt = t;
      continue;
    }
    ANCKA_TRY(apply_walk(c, cur, c.ldk, nxt, 1.f - c.alpha, labels, sc.inv, c.alpha));
    float* t = cur;
    cur = nxt;
    nxt = t;
  }
  k_trace_partial<<<sc.tblk, 256, 0, s>>>(cur, c.ldk, labels, sc.inv, c.n, sc.tpart);
  ANCKA_LAUNCHED();
  k_phi_decide<<<1, 32, 0, s>>>(sc.tpart, sc.tblk, c.k, phi_slot, phi_best, sc.take, taken_slot, first ? 1 : 0);
  ANCKA_LAUNCHED();
  k_copy_if<<<grid_for(c.n, 256), 256, 0, s>>>(sc.take, labels, best_labels, c.n);
  ANCKA_LAUNCHED();
  return ANCKA_OK;
}

// [n^-1/2 1 | W | 0-padding] (reading W6)
__global__ void k_warm_block(const float* __restrict__ W, int ldw, int64_t n, int k, int ld, float c0,
                             float* __restrict__ Q) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * ld) return;
  const int64_t i = t / ld;
  const int c = (int)(t % ld);
  Q[t] = c == 0 ? c0 : (c <= k ? W[i * ldw + c - 1] : 0.f);
}

// per-block partial sums of (A - B)^2 over the first w columns
__global__ void k_diff_norm2(const float* __restrict__ A, const float* __restrict__ B, int64_t n, int w, int ld,
                             float* __restrict__ partial) {
  __shared__ float red[32];
  float acc = 0.f;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * w; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / w;
    const int c = (int)(t % w);
    const float d = A[i * ld + c] - B[i * ld + c];
    acc = fmaf(d, d, acc);
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    partial[blockIdx.x] = t;
  }
}

ancka_status make_disc_state(Workspace& ws, int64_t n, int k, DiscState* st) {
  (void)n;
  ANCKA_TRY(ws.alloc(&st->part, (size_t)kDiscMaxGrid * k * k));
  ANCKA_TRY(ws.alloc(&st->partc, (size_t)kDiscMaxGrid * k));
  ANCKA_TRY(ws.alloc(&st->S, (size_t)k * k));
  ANCKA_TRY(ws.alloc(&st->cnt, (size_t)k));
  ANCKA_TRY(ws.alloc(&st->bar, 2));
  ANCKA_TRY(ws.alloc(&st->err, 1));
  return ANCKA_OK;
}

size_t disc_smem_bytes() { return (size_t)(kDiscRegion + kDiscLabels + kDiscSlices + kDiscR) * sizeof(float); }

// Launch Discretize on a row-normalised block (one cooperative launch).
// half_grid: at most half the SMs, for a Discretize that shares the GPU with
// other work (the rows per CTA, and so the FP32 partial sums, follow the grid)
ancka_status run_discretize(const DiscState& st, const float* Qt, int ldt, int64_t n, int k, int max_iter,
                            int32_t* labels, int32_t* iters_out, int32_t* flags, cudaStream_t s,
                            bool half_grid = false) {
  k_disc_init<<<1, 32, 0, s>>>(st.bar, st.err);
  ANCKA_LAUNCHED();
  const size_t smem = disc_smem_bytes();
  static int max_grids[kMaxDevices] = {};
  int& max_grid = max_grids[device_slot()];
  if (max_grid == 0) {
    ANCKA_CUDA(cudaFuncSetAttribute(k_discretize, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0, occ = 0;
    ANCKA_CUDA(cudaGetDevice(&dev));
    ANCKA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    ANCKA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_discretize, kDiscThreads, smem));
    max_grid = sms * (occ > 2 ? 2 : occ);
    if (max_grid > kDiscMaxGrid) max_grid = kDiscMaxGrid;
    if (max_grid < 1) {
      set_error("Discretize kernel cannot be resident");
      return ANCKA_ERR_UNSUPPORTED;
    }
  }
  int grid = (int)ceil_div(n, 512);
  const int cap = half_grid ? (max_grid + 1) / 2 : max_grid;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  DiscState stc = st;
  void* args[] = {(void*)&Qt, (void*)&ldt, (void*)&n, (void*)&k, (void*)&max_iter, (void*)&labels,
                  (void*)&stc, (void*)&iters_out, (void*)&flags};
  ANCKA_CUDA(cudaLaunchCooperativeKernel((const void*)k_discretize, dim3(grid), dim3(kDiscThreads), args, smem, s));
  ANCKA_LAUNCHED();
  return ANCKA_OK;
}

// CholeskyQR2 (diag(R) > 0) of the n x w block Z (result in Z, Q is scratch): Gram +
// factor of Z; Q = Z R1^-1 with the Gram + factor of Q in one pass; Z = Q
// R2^-1.  Rinv holds two w x w matrices.
ancka_status cholqr2(Workspace& ws, const Ctx& c, float* Z, float* Q, int w, float2* gpart, int gblk,
                     unsigned int* ticket, float* Rinv, int32_t* status) {
  cudaStream_t s = c.s;
  const int tld = 4 * ((w + 3) / 4);
  const size_t chol_bytes = (size_t)(3 * w * w + 1) * sizeof(double);
  const size_t fused_bytes = (size_t)(tld * tld + kGramRows * kGramLd) * sizeof(float);
  static bool configured[kMaxDevices] = {};
  if (!configured[device_slot()]) {
    ANCKA_CUDA(cudaFuncSetAttribute(k_gram_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (3 * 65 * 65 + 1) * 8));
    configured[device_slot()] = true;
  }
  float* R1 = Rinv;
  float* R2 = Rinv + (size_t)w * w;
  k_gram_chol<<<gblk, kGramThreads, chol_bytes, s>>>(Z, c.ld, c.n, w, nullptr, nullptr, gpart, ticket, R1, status);
  ANCKA_LAUNCHED();
  k_gram_chol<<<gblk, kGramThreads, chol_bytes > fused_bytes ? chol_bytes : fused_bytes, s>>>(
      Z, c.ld, c.n, w, R1, Q, gpart, ticket, R2, status);
  ANCKA_LAUNCHED();
  ANCKA_TRY(apply_rinv(Q, c.ld, c.n, w, R2, Z, s));
  (void)ws;
  return ANCKA_OK;
}

struct PhaseTimer {
  IterTrace* tr;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  int phase;
  PhaseTimer(IterTrace* t, cudaStream_t st, int ph) : tr(t), s(st), phase(ph) {
    if (tr && tr->events) {
      a = pooled_event();
      cudaEventRecord(a, s);
    }
  }
  ~PhaseTimer() {
    if (tr && tr->events) {
      cudaEvent_t b = pooled_event();
      cudaEventRecord(b, s);
      tr->events->push_back(a);
      tr->events->push_back(b);
      tr->phases->push_back(phase);
    }
  }
};

// the keep-best chain's stream (one per device and host thread), at the
// highest priority: its work ends the call
ancka_status side_stream(cudaStream_t* out) {
  static thread_local cudaStream_t streams[kMaxDevices] = {};
  cudaStream_t& ds = streams[device_slot()];
  if (!ds) {
    int lo = 0, hi = 0;
    ANCKA_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    ANCKA_CUDA(cudaStreamCreateWithPriority(&ds, cudaStreamNonBlocking, hi));
  }
  *out = ds;
  return ANCKA_OK;
}

// on every exit: the call's stream waits for the side stream's work (which
// uses the call's workspace) before anything is released
struct SideJoin {
  cudaStream_t s = nullptr, ds = nullptr;
  cudaEvent_t ev = nullptr;
  bool active = false;
  ~SideJoin() {
    if (active) {
      cudaEventRecord(ev, ds);
      cudaStreamWaitEvent(s, ev, 0);
    }
    if (ev) release_event(ev);
  }
};

}  // namespace

// InitBCM (Alg. 4 lines 3-11) on its own: the k highest-degree nodes (ties by
// index) seed one column each, T_i hops of the topology walk, then the
// argmax of each row gives Y^(0).  It reads only the topology part of the walk
// (no attributes, no KNN part), with its own scratch, so it may run on a
// stream of its own while the KNN is computed.
ancka_status initbcm_labels(Workspace& ws, const Walk& w, const IterCfg& cfg, int32_t* y0, cudaStream_t s) {
  const int64_t n = w.n;
  const int k = cfg.k;
  const int ld = (int)round_up(k + 1, 4);
  const int ldk = (int)round_up(k, 4);
  const bool hyper = w.kind == ANCKA_HYPERGRAPH;
  float* E = nullptr;
  if (hyper) ANCKA_TRY(ws.alloc(&E, (size_t)(w.m > 0 ? w.m : 1) * ldk));
  Ctx c{w, n, k, ld, ldk, cfg.alpha, E, s, {}, {}, {}};
  // the same long-row classes as the iteration's (block sizes at width ld)
  const double qbytes = (double)n * ld * 4.0, ebytes = (double)w.m * ld * 4.0;
  ANCKA_TRY(find_long_rows(ws, w.topo.ptr, nullptr, n, w.topo.nnz, hyper ? ebytes : qbytes, &c.lr_topo, s));
  if (hyper) ANCKA_TRY(find_long_rows(ws, w.edges.ptr, nullptr, w.m, w.edges.nnz, qbytes, &c.lr_edges, s));
  ANCKA_TRY(build_long_items(ws, w.topo.ptr, nullptr, &c.lr_topo, s));
  if (hyper) ANCKA_TRY(build_long_items(ws, w.edges.ptr, nullptr, &c.lr_edges, s));
  {
    LongRows* lrs[2] = {&c.lr_topo, &c.lr_edges};
    ANCKA_TRY(read_long_rows(lrs, hyper ? 2 : 1, s));
  }
  float *Fa, *Fb;
  ANCKA_TRY(ws.alloc(&Fa, (size_t)n * ldk));
  ANCKA_TRY(ws.alloc(&Fb, (size_t)n * ldk));
  uint64_t *keys, *skeys;
  int32_t* seedcol;
  ANCKA_TRY(ws.alloc(&keys, (size_t)n));
  ANCKA_TRY(ws.alloc(&skeys, (size_t)n));
  ANCKA_TRY(ws.alloc(&seedcol, (size_t)n));
  ANCKA_CUDA(cudaMemsetAsync(seedcol, 0xff, sizeof(int32_t) * n, s));
  k_degree_keys<<<grid_for(n, 256), 256, 0, s>>>(w.degree, n, keys);
  ANCKA_LAUNCHED();
  ANCKA_TRY(radix_sort_u64(ws, keys, skeys, n, 64, s));
  k_seed_setup<<<1, 32, 0, s>>>(skeys, k, seedcol);
  ANCKA_LAUNCHED();
  k_fill_seed<<<grid_for(n * ldk, 256), 256, 0, s>>>(seedcol, n, ldk, cfg.alpha, Fa);
  ANCKA_LAUNCHED();
  float* cur = Fa;
  float* nxt = Fb;
  for (int t2 = 0; t2 < cfg.T_i; ++t2) {
    ANCKA_TRY(initbcm_hop(c, cur, nxt, seedcol));
    float* tt = cur;
    cur = nxt;
    nxt = tt;
  }
  k_argmax_rows<<<grid_for(n, 256), 256, 0, s>>>(cur, ldk, n, k, y0);
  ANCKA_LAUNCHED();
  return ANCKA_OK;
}

namespace {

// ---- degree order of the nodes (locality of the walk products) ----
// Algorithm 4 is equivariant under a renaming of the nodes, except for
// InitBCM's tie-break by index, which is therefore taken on the caller's
// names.  Renaming the nodes by descending degree puts the rows of Q that
// most entries gather (the hubs) next to each other, so more of the gathers
// hit L2.

// new row r holds old row order[r]; pos is the inverse
__global__ void k_order_maps(const uint64_t* __restrict__ sorted, int64_t n, int32_t* __restrict__ order,
                             int32_t* __restrict__ pos) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int32_t o = (int32_t)(sorted[r] & 0xffffffffull);
  order[r] = o;
  pos[o] = (int32_t)r;
}

// entries of new row r (and len[n] = 0, for the scan into row pointers)
__global__ void k_permuted_lens(const int64_t* __restrict__ ptr, const int32_t* __restrict__ order, int64_t n,
                                int64_t* __restrict__ len) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) len[r] = ptr[order[r] + 1] - ptr[order[r]];
  if (r == n) len[r] = 0;
}

constexpr int kPermPerLane = 16;  // entries per lane of k_permute_csr

// the renamed CSR: entry q of new row r is entry q - nptr[r] of old row
// order[r] (the row's entry order is kept), its column renamed by pos.  A
// warp covers 32 x kPermPerLane consecutive entries (lane-interleaved, so
// the copies coalesce); each lane finds its first row by binary search and
// then walks forward.
__global__ void k_permute_csr(const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                              const float* __restrict__ val, const float* __restrict__ valT,
                              const int32_t* __restrict__ order, const int32_t* __restrict__ pos, int64_t n,
                              const int64_t* __restrict__ nptr, int32_t* __restrict__ ncol,
                              float* __restrict__ nval, float* __restrict__ nvalT) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t total = nptr[n];
  const int64_t q0 = warp * 32 * kPermPerLane + lane;
  if (q0 >= total) return;
  int64_t lo = 0, hi = n - 1;  // last row r with nptr[r] <= q0
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (nptr[mid] <= q0) lo = mid;
    else hi = mid - 1;
  }
  int64_t r = lo;
  for (int j = 0; j < kPermPerLane; ++j) {
    const int64_t q = q0 + 32 * j;
    if (q >= total) break;
    while (nptr[r + 1] <= q) ++r;
    const int64_t src = ptr[order[r]] + (q - nptr[r]);
    ncol[q] = pos[col[src]];
    if (nval) nval[q] = val[src];
    if (nvalT) nvalT[q] = valT[src];
  }
}

template <class T>
__global__ void k_gather_vec(const T* __restrict__ in, const int32_t* __restrict__ order, int64_t n,
                             T* __restrict__ out) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) out[r] = in[order[r]];
}

template <class T>
__global__ void k_scatter_vec(const T* __restrict__ in, const int32_t* __restrict__ order, int64_t n,
                              T* __restrict__ out) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) out[order[r]] = in[r];
}

// out row r = in row order[r] (gather) or out row order[r] = in row r
template <bool Gather>
__global__ void k_permute_rows(const float* __restrict__ in, int ldi, const int32_t* __restrict__ order, int64_t n,
                               int width, float* __restrict__ out, int ldo) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * width) return;
  const int64_t r = t / width;
  const int c = (int)(t % width);
  if (Gather) out[r * ldo + c] = in[(int64_t)order[r] * ldi + c];
  else out[(int64_t)order[r] * ldo + c] = in[r * ldi + c];
}

ancka_status permute_csr(Workspace& ws, const Csr& a, int64_t n, const int32_t* order, const int32_t* pos, Csr* b,
                         cudaStream_t s) {
  *b = a;
  int64_t* len;
  ANCKA_TRY(ws.alloc(&len, (size_t)n + 1));
  ANCKA_TRY(ws.alloc(&b->ptr, (size_t)n + 1));
  k_permuted_lens<<<grid_for(n + 1, 256), 256, 0, s>>>(a.ptr, order, n, len);
  ANCKA_LAUNCHED();
  ANCKA_TRY(exclusive_scan(ws, len, b->ptr, n + 1, s));
  // nnz may be an upper bound (the KNN part): the kernel stops at ptr[n]
  ANCKA_TRY(ws.alloc(&b->col, (size_t)a.nnz));
  b->val = b->valT = nullptr;
  if (a.val) ANCKA_TRY(ws.alloc(&b->val, (size_t)a.nnz));
  if (a.valT) ANCKA_TRY(ws.alloc(&b->valT, (size_t)a.nnz));
  const int64_t warps = ceil_div(a.nnz, 32 * kPermPerLane);
  k_permute_csr<<<grid_for(warps * 32, 256), 256, 0, s>>>(a.ptr, a.col, a.val, a.valT, order, pos, n, b->ptr,
                                                          b->col, b->val, b->valT);
  ANCKA_LAUNCHED();
  return ANCKA_OK;
}

template <class T>
ancka_status gather_vec(Workspace& ws, const T* in, const int32_t* order, int64_t n, T** out, cudaStream_t s) {
  *out = nullptr;
  if (!in) return ANCKA_OK;
  T* o;
  ANCKA_TRY(ws.alloc(&o, (size_t)n));
  k_gather_vec<T><<<grid_for(n, 256), 256, 0, s>>>(in, order, n, o);
  ANCKA_LAUNCHED();
  *out = o;
  return ANCKA_OK;
}

// the walk with its nodes renamed: graphs and multiplex graphs only
ancka_status permute_walk(Workspace& ws, const Walk& w, const int32_t* order, const int32_t* pos, Walk* v,
                          cudaStream_t s) {
  const int64_t n = w.n;
  *v = w;
  ANCKA_TRY(permute_csr(ws, w.topo, n, order, pos, &v->topo, s));
  ANCKA_TRY(permute_csr(ws, w.knn, n, order, pos, &v->knn, s));
  ANCKA_TRY(gather_vec(ws, w.rs_topo, order, n, &v->rs_topo, s));
  ANCKA_TRY(gather_vec(ws, w.inv_deg, order, n, &v->inv_deg, s));
  ANCKA_TRY(gather_vec(ws, w.degree, order, n, &v->degree, s));
  ANCKA_TRY(gather_vec(ws, w.beta, order, n, &v->beta, s));
  return ANCKA_OK;
}

}  // namespace

// phases: 2 = init, 3 = iteration, 4 = discretize, 5 = mhc, 6 = the walk products inside 3
static ancka_status run_ancka_rows(Workspace& ws, const Walk& w, const IterCfg& cfg, const int32_t* init_labels,
                                   const float* warm_W, int ldw, int32_t* labels_out, float* Q_out,
                                   int32_t* init_out, IterTrace* tr, cudaStream_t s) {
  const int64_t n = w.n;
  const int k = cfg.k;
  const int wq = k + 1;
  const int ld = (int)round_up(wq, 4);
  const int ldk = (int)round_up(k, 4);
  float *Qa, *Qb, *Qt, *E = nullptr, *Rinv;
  ANCKA_TRY(ws.alloc(&Qa, (size_t)n * ld));
  ANCKA_TRY(ws.alloc(&Qb, (size_t)n * ld));
  ANCKA_TRY(ws.alloc(&Qt, (size_t)n * ldk));
  ANCKA_TRY(ws.alloc(&Rinv, (size_t)2 * wq * wq));
  if (w.kind == ANCKA_HYPERGRAPH) ANCKA_TRY(ws.alloc(&E, (size_t)(w.m > 0 ? w.m : 1) * (ld > ldk ? ld : ldk)));
  Ctx c{w, n, k, ld, ldk, cfg.alpha, E, s, {}, {}, {}};
  const double qbytes = (double)n * ld * 4.0, ebytes = (double)w.m * ld * 4.0;
  // the KNN part's nnz is an upper bound (its exact count stays on the device)
  ANCKA_TRY(find_long_rows(ws, w.topo.ptr, w.knn.ptr, n, w.topo.nnz + w.knn.nnz,
                           w.kind == ANCKA_HYPERGRAPH ? ebytes : qbytes, &c.lr_walk, s));
  if (w.kind == ANCKA_HYPERGRAPH)
    ANCKA_TRY(find_long_rows(ws, w.edges.ptr, nullptr, w.m, w.edges.nnz, qbytes, &c.lr_edges, s));
  ANCKA_TRY(build_long_items(ws, w.topo.ptr, w.knn.ptr, &c.lr_walk, s));
  if (w.kind == ANCKA_HYPERGRAPH) ANCKA_TRY(build_long_items(ws, w.edges.ptr, nullptr, &c.lr_edges, s));
  {
    LongRows* lrs[2] = {&c.lr_walk, &c.lr_edges};
    ANCKA_TRY(read_long_rows(lrs, w.kind == ANCKA_HYPERGRAPH ? 2 : 1, s));
  }
  Scratch sc;
  ANCKA_TRY(ws.alloc(&sc.cnt, 64));
  ANCKA_TRY(ws.alloc(&sc.inv, 64));
  ANCKA_TRY(ws.alloc(&sc.Fa, (size_t)n * ldk));
  ANCKA_TRY(ws.alloc(&sc.Fb, (size_t)n * ldk));
  sc.tblk = (int)(ceil_div(n, 4096) < 304 ? ceil_div(n, 4096) : 304);
  ANCKA_TRY(ws.alloc(&sc.tpart, (size_t)sc.tblk));
  ANCKA_TRY(ws.alloc(&sc.take, 1));
  const int gblk = (int)(ceil_div(n, 512) < 2 * 152 ? ceil_div(n, 512) : 2 * 152);  // two CTAs per SM
  float2* gpart;
  unsigned int* gticket;
  ANCKA_TRY(ws.alloc(&gpart, (size_t)gblk * wq * (wq + 1) / 2));
  ANCKA_TRY(ws.zeros(&gticket, 1));
  int32_t *y0, *yt, *ybest, *chol_status;
  ANCKA_TRY(ws.alloc(&y0, (size_t)n));
  ANCKA_TRY(ws.alloc(&yt, (size_t)n));
  ANCKA_TRY(ws.alloc(&ybest, (size_t)n));
  ANCKA_TRY(ws.zeros(&chol_status, 1));
  DiscState st;
  ANCKA_TRY(make_disc_state(ws, n, k, &st));
  // Fixed schedule: the keep-best chain (CalMHC of Y^(0), then Discretize and
  // CalMHC at each check point) reads Q^(t) but feeds nothing back into the
  // hops, so it runs on a second stream beside them, in its own order, with
  // its own edge buffer and two row-normalised snapshots of Q (alternating
  // between check points).  Paper mode decides whether to go on from phi, so
  // there the chain stays on the call's stream.
  const bool side = !cfg.early_stop;
  cudaStream_t ds = s;
  if (side) ANCKA_TRY(side_stream(&ds));
  Ctx cd = c;
  cd.s = ds;
  float* Qt2[2] = {Qt, Qt};
  if (side) {
    ANCKA_TRY(ws.alloc(&Qt2[1], (size_t)n * ldk));
    if (w.kind == ANCKA_HYPERGRAPH) ANCKA_TRY(ws.alloc(&cd.E, (size_t)(w.m > 0 ? w.m : 1) * (ld > ldk ? ld : ldk)));
  }

  // ---- InitBCM (Alg. 4 lines 3-11) ----
  {
    PhaseTimer pt(tr, s, 2);
    if (init_labels) {
      ANCKA_CUDA(cudaMemcpyAsync(y0, init_labels, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    } else {
      ANCKA_TRY(initbcm_labels(ws, w, cfg, y0, s));
    }
    // Q^(0) = [n^-1/2 1 | h(Y^(0))]
    ANCKA_CUDA(cudaMemsetAsync(sc.cnt, 0, sizeof(int32_t) * k, s));
    k_count_labels<<<grid_for(n, 1024) < 304 ? grid_for(n, 1024) : 304, 256, 0, s>>>(y0, n, k, sc.cnt);
    ANCKA_LAUNCHED();
    k_inv_sqrt_counts<<<1, 64, 0, s>>>(sc.cnt, k, sc.inv);
    ANCKA_LAUNCHED();
    k_fill_onehot<<<grid_for(n * ld, 256), 256, 0, s>>>(y0, sc.inv, sc.cnt, k, n, ld, 1,
                                                        (float)(1.0 / sqrt((double)n)), 1.f, Qa, w.names);
    ANCKA_LAUNCHED();
  }
  tr->warm_used = 0;
  if (warm_W) {  // phi(Y^(0)) (reading R8), compared with the warm start's below
    PhaseTimer pt(tr, s, 5);
    ANCKA_TRY(cal_mhc(c, sc, y0, cfg.gamma, tr->phi_dev + 0, tr->phi_best_dev, nullptr, ybest, true));
  }
  if (warm_W) {
    // learned warm start: Q_w = QR([n^-1/2 1 | W]) and Y_w = Discretize(Q_w[:, 1:]);
    // it replaces InitBCM's start only if Phi(Y_w) <= Phi(Y^(0)) (reading W6)
    PhaseTimer pt(tr, s, 2);
    float* Qs;
    double* phw;
    int32_t *yw, *ywb, *wstatus;
    ANCKA_TRY(ws.alloc(&Qs, (size_t)n * ld));
    ANCKA_TRY(ws.alloc(&phw, 2));
    ANCKA_TRY(ws.alloc(&yw, (size_t)n));
    ANCKA_TRY(ws.alloc(&ywb, (size_t)n));
    ANCKA_TRY(ws.zeros(&wstatus, 1));
    k_warm_block<<<grid_for(n * ld, 256), 256, 0, s>>>(warm_W, ldw, n, k, ld, (float)(1.0 / sqrt((double)n)), Qb);
    ANCKA_LAUNCHED();
    ANCKA_TRY(cholqr2(ws, c, Qb, Qs, wq, gpart, gblk, gticket, Rinv, wstatus));  // result in Qb
    rownorm(Qb, ld, 1, n, k, Qt, ldk, s);
    ANCKA_LAUNCHED();
    ANCKA_TRY(run_discretize(st, Qt, ldk, n, k, cfg.disc_max_iter, yw, nullptr, tr->flags_dev, s));
    ANCKA_TRY(cal_mhc(c, sc, yw, cfg.gamma, phw, phw + 1, nullptr, ywb, true));
    double h[2] = {0.0, 0.0};
    int32_t hs = 0, de = 0;
    ANCKA_CUDA(cudaMemcpyAsync(&h[0], phw, sizeof(double), cudaMemcpyDeviceToHost, s));
    ANCKA_CUDA(cudaMemcpyAsync(&h[1], tr->phi_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    ANCKA_CUDA(cudaMemcpyAsync(&hs, wstatus, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    ANCKA_CUDA(cudaMemcpyAsync(&de, st.err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    ANCKA_CUDA(cudaStreamSynchronize(s));
    if (de) {
      set_error("Discretize: a grid barrier wait expired");
      return ANCKA_ERR_TIMEOUT;
    }
    if (hs == 0 && h[0] <= h[1]) {
      ANCKA_CUDA(cudaMemcpyAsync(Qa, Qb, sizeof(float) * n * ld, cudaMemcpyDeviceToDevice, s));
      ANCKA_CUDA(cudaMemcpyAsync(y0, yw, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
      ANCKA_CUDA(cudaMemcpyAsync(ybest, yw, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
      ANCKA_CUDA(cudaMemcpyAsync(tr->phi_dev, phw, sizeof(double), cudaMemcpyDeviceToDevice, s));
      ANCKA_CUDA(cudaMemcpyAsync(tr->phi_best_dev, phw, sizeof(double), cudaMemcpyDeviceToDevice, s));
      tr->warm_used = 1;
    }
  }
  if (init_out) ANCKA_CUDA(cudaMemcpyAsync(init_out, y0, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  // the first hop from the labels (graphs, multiplex graphs, Q^(0) from InitBCM
  // or given labels): its own copies of the cluster sizes and 1/sqrt(size),
  // since the keep-best chain recomputes the scratch ones beside the hops
  const bool q0_labels = w.kind != ANCKA_HYPERGRAPH && !tr->warm_used;
  int32_t* q0cnt = nullptr;
  float* q0inv = nullptr;
  if (q0_labels) {
    ANCKA_TRY(ws.alloc(&q0cnt, 64));
    ANCKA_TRY(ws.alloc(&q0inv, 64));
    ANCKA_CUDA(cudaMemcpyAsync(q0cnt, sc.cnt, sizeof(int32_t) * k, cudaMemcpyDeviceToDevice, s));
    ANCKA_CUDA(cudaMemcpyAsync(q0inv, sc.inv, sizeof(float) * k, cudaMemcpyDeviceToDevice, s));
  }
  // fork: everything above (Y^(0), Q^(0), the scratch) is ready on s here
  SideJoin sj;
  cudaEvent_t q_ev = nullptr, disc_done[2] = {nullptr, nullptr};
  bool qt_used[2] = {false, false};
  struct Events {
    cudaEvent_t* e[3];
    ~Events() {
      for (cudaEvent_t* p : e)
        if (*p) release_event(*p);
    }
  } evs{{&q_ev, &disc_done[0], &disc_done[1]}};
  if (side) {
    sj.s = s;
    sj.ds = ds;
    sj.ev = pooled_event();
    q_ev = pooled_event();
    disc_done[0] = pooled_event();
    disc_done[1] = pooled_event();
    ANCKA_CUDA(cudaEventRecord(q_ev, s));
    ANCKA_CUDA(cudaStreamWaitEvent(ds, q_ev, 0));
    sj.active = true;
  }
  if (!warm_W) {  // phi(Y^(0)) (reading R8)
    PhaseTimer pt(tr, ds, 5);
    ANCKA_TRY(cal_mhc(cd, sc, y0, cfg.gamma, tr->phi_dev + 0, tr->phi_best_dev, nullptr, ybest, true));
  }
  // paper mode (Eq. tcond-1 / tcond-2): Q(t-1) kept at the check points
  float* Qprev = nullptr;
  float* dq_part = nullptr;
  constexpr int kDqBlocks = 256;
  double phi_hist[3] = {0.0, 0.0, 0.0};
  int n_hist = 0;
  double *phi_spare = nullptr;
  int32_t *di_spare = nullptr, *tk_spare = nullptr;
  ANCKA_TRY(ws.alloc(&phi_spare, 1));
  ANCKA_TRY(ws.alloc(&di_spare, 1));
  ANCKA_TRY(ws.alloc(&tk_spare, 1));
  if (cfg.early_stop) {
    ANCKA_TRY(ws.alloc(&Qprev, (size_t)n * ld));
    ANCKA_TRY(ws.alloc(&dq_part, kDqBlocks));
    ANCKA_CUDA(cudaMemcpyAsync(&phi_hist[0], tr->phi_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    ANCKA_CUDA(cudaStreamSynchronize(s));
    n_hist = 1;
  }
  int slot = 1;
  float* Q = Qa;
  float* Z = Qb;
  int t_run = 0;
  for (int t = 1; t <= cfg.T; ++t) {
    const bool check = t % cfg.tau == 0 || t == cfg.T;
    {
      PhaseTimer pt(tr, s, 3);
      {
        PhaseTimer pw(tr, s, 6);
        if (t == 1 && q0_labels) {  // Z = P Q^(0) from the labels
          const int64_t blocks = ceil_div(n, (int64_t)8);
          const LongRows& lr = c.lr_walk;
          const bool longs = lr.rows && lr.count_host > 0;
          const float c0 = (float)(1.0 / sqrt((double)n));
          k_walk_q0<<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, s>>>(
              w.topo.ptr, w.topo.col, w.row_uniform ? nullptr : w.topo.val, w.rs_topo, w.knn.ptr, w.knn.col,
              w.knn.val, y0, q0inv, q0cnt, w.names, k, ld, c0, n, longs ? lr.min_entries : 0, Z);
          ANCKA_LAUNCHED();
          if (longs) {
            k_walk_q0_long<<<(unsigned)lr.count_host, 256, 0, s>>>(
                lr.rows, w.topo.ptr, w.topo.col, w.row_uniform ? nullptr : w.topo.val, w.rs_topo, w.knn.ptr,
                w.knn.col, w.knn.val, y0, q0inv, q0cnt, w.names, k, ld, c0, Z);
            ANCKA_LAUNCHED();
          }
        } else {
          ANCKA_TRY(apply_walk(c, Q, ld, Z, 1.f, nullptr, nullptr, 0.f));  // Z = P Q
        }
      }
      if (Qprev && check)  // Q(t-1); CholeskyQR2 below uses Q as scratch
        ANCKA_CUDA(cudaMemcpyAsync(Qprev, Q, sizeof(float) * n * ld, cudaMemcpyDeviceToDevice, s));
      ANCKA_TRY(cholqr2(ws, c, Z, Q, wq, gpart, gblk, gticket, Rinv, chol_status));  // result in Z
      float* tt = Q;
      Q = Z;
      Z = tt;
    }
    t_run = t;
    if (check) {
      // trace slots beyond ANCKA_MAX_TRACE are not recorded
      const bool rec = slot < ANCKA_MAX_TRACE;
      double* phi_slot = rec ? tr->phi_dev + slot : phi_spare;
      const int b = side ? slot & 1 : 0;
      if (side && qt_used[b]) ANCKA_CUDA(cudaStreamWaitEvent(s, disc_done[b], 0));  // its last reader is done
      rownorm(Q, ld, 1, n, k, Qt2[b], ldk, s);  // the snapshot of Q^(t)
      ANCKA_LAUNCHED();
      if (side) {
        ANCKA_CUDA(cudaEventRecord(q_ev, s));
        ANCKA_CUDA(cudaStreamWaitEvent(ds, q_ev, 0));
      }
      {
        PhaseTimer pt(tr, ds, 4);
        // beside the hops on half the SMs; the last one runs alone, on all
        ANCKA_TRY(run_discretize(st, Qt2[b], ldk, n, k, cfg.disc_max_iter, yt,
                                 rec ? tr->disc_iters_dev + slot : di_spare, tr->flags_dev, ds, side && t < cfg.T));
      }
      if (side) {
        ANCKA_CUDA(cudaEventRecord(disc_done[b], ds));
        qt_used[b] = true;
      }
      {
        PhaseTimer pt(tr, ds, 5);
        ANCKA_TRY(cal_mhc(cd, sc, yt, cfg.gamma, phi_slot, tr->phi_best_dev, rec ? tr->taken_dev + slot : tk_spare,
                          ybest, false));
      }
      ++slot;
      if (cfg.early_stop) {
        k_diff_norm2<<<kDqBlocks, 256, 0, s>>>(Q, Qprev, n, wq, ld, dq_part);
        ANCKA_LAUNCHED();
        float hp[kDqBlocks];
        double ph = 0.0;
        ANCKA_CUDA(cudaMemcpyAsync(hp, dq_part, sizeof(hp), cudaMemcpyDeviceToHost, s));
        ANCKA_CUDA(cudaMemcpyAsync(&ph, phi_slot, sizeof(double), cudaMemcpyDeviceToHost, s));
        ANCKA_CUDA(cudaStreamSynchronize(s));
        double dq = 0.0;
        for (int b = 0; b < kDqBlocks; ++b) dq += hp[b];
        dq = std::sqrt(dq);
        if (n_hist == 3) {
          phi_hist[0] = phi_hist[1];
          phi_hist[1] = phi_hist[2];
          n_hist = 2;
        }
        phi_hist[n_hist++] = ph;
        const bool conv = dq < (double)cfg.eps_Q;                                                    // Eq. tcond-1
        const bool rising = n_hist == 3 && phi_hist[0] < phi_hist[1] && phi_hist[1] < phi_hist[2];  // Eq. tcond-2
        if (conv || rising) break;
      }
    }
  }
  tr->n_phi = slot < ANCKA_MAX_TRACE ? slot : ANCKA_MAX_TRACE;
  tr->iters_run = t_run;
  if (sj.active) {  // join: ybest, the trace and the Discretize flags are final on s after this
    ANCKA_CUDA(cudaEventRecord(sj.ev, ds));
    ANCKA_CUDA(cudaStreamWaitEvent(s, sj.ev, 0));
    sj.active = false;
  }
  ANCKA_CUDA(cudaMemcpyAsync(labels_out, ybest, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  if (Q_out) ANCKA_CUDA(cudaMemcpy2DAsync(Q_out, sizeof(float) * wq, Q, sizeof(float) * ld, sizeof(float) * wq, n,
                                         cudaMemcpyDeviceToDevice, s));
  // a singular Gram matrix is reported (numeric failure of CholeskyQR)
  int32_t cs = 0, de = 0;
  ANCKA_CUDA(cudaMemcpyAsync(&cs, chol_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  ANCKA_CUDA(cudaMemcpyAsync(&de, st.err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  ANCKA_CUDA(cudaStreamSynchronize(s));
  if (de) {
    set_error("Discretize: a grid barrier wait expired");
    return ANCKA_ERR_TIMEOUT;
  }
  if (cs) {
    set_error("CholeskyQR: Gram matrix of Z is not positive definite (rank-deficient block)");
    return ANCKA_ERR_NUMERIC;
  }
  return ANCKA_OK;
}

bool degree_order_applies(const Walk& w, const IterCfg& cfg) {
  if (w.kind == ANCKA_HYPERGRAPH || cfg.node_order == 1 || w.n < 2) return false;
  if (cfg.node_order == 2) return true;
  return (double)w.n * round_up(cfg.k + 1, 4) * 4.0 > kDegreeOrderMinBytes;
}

ancka_status run_ancka(Workspace& ws, const Walk& w, const IterCfg& cfg, const int32_t* init_labels,
                       const float* warm_W, int ldw, int32_t* labels_out, float* Q_out, int32_t* init_out,
                       IterTrace* tr, cudaStream_t s) {
  if (!degree_order_applies(w, cfg))
    return run_ancka_rows(ws, w, cfg, init_labels, warm_W, ldw, labels_out, Q_out, init_out, tr, s);
  const int64_t n = w.n;
  const int k = cfg.k;
  const int wq = k + 1;
  int32_t *y0 = nullptr, *order, *pos;
  {
    PhaseTimer pt(tr, s, 2);
    if (!init_labels) {  // InitBCM breaks degree ties by the caller's node index
      ANCKA_TRY(ws.alloc(&y0, (size_t)n));
      ANCKA_TRY(initbcm_labels(ws, w, cfg, y0, s));
      init_labels = y0;
    }
  }
  Walk v;
  int32_t *y_in, *lab, *init_v = nullptr;
  float *W_v = nullptr, *Q_v = nullptr;
  {
    PhaseTimer pt(tr, s, 1);
    uint64_t *keys, *skeys;
    ANCKA_TRY(ws.alloc(&keys, (size_t)n));
    ANCKA_TRY(ws.alloc(&skeys, (size_t)n));
    ANCKA_TRY(ws.alloc(&order, (size_t)n));
    ANCKA_TRY(ws.alloc(&pos, (size_t)n));
    k_degree_keys<<<grid_for(n, 256), 256, 0, s>>>(w.degree, n, keys);
    ANCKA_LAUNCHED();
    ANCKA_TRY(radix_sort_u64(ws, keys, skeys, n, 64, s));
    k_order_maps<<<grid_for(n, 256), 256, 0, s>>>(skeys, n, order, pos);
    ANCKA_LAUNCHED();
    ANCKA_TRY(permute_walk(ws, w, order, pos, &v, s));
    v.names = order;  // R13's sign vectors follow the caller's node index
    ANCKA_TRY(ws.alloc(&y_in, (size_t)n));
    ANCKA_TRY(ws.alloc(&lab, (size_t)n));
    if (init_out) ANCKA_TRY(ws.alloc(&init_v, (size_t)n));
    k_gather_vec<int32_t><<<grid_for(n, 256), 256, 0, s>>>(init_labels, order, n, y_in);
    ANCKA_LAUNCHED();
    if (warm_W) {
      ANCKA_TRY(ws.alloc(&W_v, (size_t)n * ldw));
      k_permute_rows<true><<<grid_for(n * k, 256), 256, 0, s>>>(warm_W, ldw, order, n, k, W_v, ldw);
      ANCKA_LAUNCHED();
    }
    if (Q_out) ANCKA_TRY(ws.alloc(&Q_v, (size_t)n * wq));
  }
  const ancka_status st = run_ancka_rows(ws, v, cfg, y_in, W_v, ldw, lab, Q_v, init_v, tr, s);
  if (st != ANCKA_OK && st != ANCKA_ERR_NUMERIC) return st;
  PhaseTimer pt(tr, s, 1);
  k_scatter_vec<int32_t><<<grid_for(n, 256), 256, 0, s>>>(lab, order, n, labels_out);
  ANCKA_LAUNCHED();
  if (init_out) {
    k_scatter_vec<int32_t><<<grid_for(n, 256), 256, 0, s>>>(init_v, order, n, init_out);
    ANCKA_LAUNCHED();
  }
  if (Q_out) {
    k_permute_rows<false><<<grid_for(n * wq, 256), 256, 0, s>>>(Q_v, wq, order, n, wq, Q_out, wq);
    ANCKA_LAUNCHED();
  }
  return st;
}

ancka_status discretize(Workspace& ws, const float* Qk, int64_t n, int32_t k, int32_t ldq, int32_t max_iter,
                        int32_t* labels, int32_t* iters_dev, int32_t* flags_dev, int32_t** err_dev,
                        cudaStream_t s) {
  const int ldk = (int)round_up(k, 4);
  float* Qt;
  ANCKA_TRY(ws.alloc(&Qt, (size_t)n * ldk));
  rownorm(Qk, ldq, 0, n, k, Qt, ldk, s);
  ANCKA_LAUNCHED();
  DiscState st;
  ANCKA_TRY(make_disc_state(ws, n, k, &st));
  *err_dev = st.err;
  return run_discretize(st, Qt, ldk, n, k, max_iter, labels, iters_dev, flags_dev, s);
}

}  // namespace ancka

namespace ancka {

namespace {
inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
}  // namespace

// The polar factor of one k x k matrix by Discretize's device routines.
ancka_status polar_factor(const float* M, int32_t k, float* R, int32_t* method_dev, cudaStream_t s) {
  const size_t smem = (size_t)(4 * kDiscLd * 64 + 64 * 64) * sizeof(float);
  ANCKA_CUDA(cudaFuncSetAttribute(k_polar_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_polar_diag<<<1, kDiscThreads, smem, s>>>(M, k, R, method_dev);
  ANCKA_LAUNCHED();
  return ANCKA_OK;
}

// Bytes of caller-provided scratch Discretize needs for an n x k block.
size_t discretize_scratch_bytes(int64_t n, int32_t k) {
  const size_t ldk = (size_t)round_up(k, 4);
  return align256((size_t)n * ldk * sizeof(float)) + align256((size_t)kDiscMaxGrid * k * k * sizeof(long long)) +
         align256((size_t)kDiscMaxGrid * k * sizeof(int32_t)) + align256((size_t)k * k * sizeof(long long)) +
         align256((size_t)k * sizeof(int32_t)) + 256;
}

// Discretize on a caller-provided scratch block of at least
// discretize_scratch_bytes(n, k) bytes (256-byte aligned); the per-call state
// is reset by a kernel and a memset, nothing is allocated.  *iters_dev and
// *err_dev point into the scratch afterwards.
ancka_status discretize_scratch(void* scratch, size_t bytes, const float* Qk, int64_t n, int32_t k, int32_t ldq,
                                int32_t max_iter, int32_t* labels, int32_t** iters_dev, int32_t** err_dev,
                                cudaStream_t s) {
  if (bytes < discretize_scratch_bytes(n, k)) {
    set_error("Discretize scratch too small");
    return ANCKA_ERR_INVALID_ARG;
  }
  const int ldk = (int)round_up(k, 4);
  char* p = static_cast<char*>(scratch);
  float* Qt = reinterpret_cast<float*>(p);
  p += align256((size_t)n * ldk * sizeof(float));
  DiscState st;
  st.part = reinterpret_cast<long long*>(p);
  p += align256((size_t)kDiscMaxGrid * k * k * sizeof(long long));
  st.partc = reinterpret_cast<int32_t*>(p);
  p += align256((size_t)kDiscMaxGrid * k * sizeof(int32_t));
  st.S = reinterpret_cast<long long*>(p);
  p += align256((size_t)k * k * sizeof(long long));
  st.cnt = reinterpret_cast<int32_t*>(p);
  p += align256((size_t)k * sizeof(int32_t));
  st.bar = reinterpret_cast<unsigned int*>(p);
  st.err = reinterpret_cast<int32_t*>(p + 8);
  int32_t* it = reinterpret_cast<int32_t*>(p + 12);
  ANCKA_CUDA(cudaMemsetAsync(it, 0, sizeof(int32_t), s));
  rownorm(Qk, ldq, 0, n, k, Qt, ldk, s);
  ANCKA_LAUNCHED();
  ANCKA_TRY(run_discretize(st, Qt, ldk, n, k, max_iter, labels, it, nullptr, s));
  *iters_dev = it;
  *err_dev = st.err;
  return ANCKA_OK;
}

}  // namespace ancka
