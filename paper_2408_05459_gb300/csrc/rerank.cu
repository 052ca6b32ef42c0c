// Exact KNN lists from low-precision candidates (Section 3.1, reading R2).
//
// Row i comes out of the contraction with kCandC approximate scores s^_ij:
// one list of its 32 best (CUDA-core kernel) or two lists of the 16 best of
// each half of the key columns (tensor-core kernel).  thr_i = the largest
// minimum over the full lists bounds every key not kept.  With the per-pair
// error bound
//     |cos_ij - s^_ij| <= m_ij = e_i (1 + e_j) + e_j + acc (1 + e_i)(1 + e_j)
// (e = quantisation bound of the row copies, acc = accumulation bound of the
// contraction) the K-th largest lower bound lb_i = K-th max (s^ - m) is a
// lower bound of the true K-th similarity.  Candidates with s^ + m < lb and
// every non-candidate (s^ <= thr_i) when thr_i + m_max < lb cannot be in the
// list.  The remaining candidates are re-scored with a compensated (Dot2)
// dot product of the raw FP32 rows (over row i's nonzero positions alone when
// it is sparse), scaled by the inverse norms in float-float, and sorted by
// (cosine desc, index asc).  A row that fails the certificate goes to the
// collect pass, and one that overflows it to the exhaustive kernels (FP64
// cosines there).
#include "common.cuh"

namespace ancka {

namespace {

constexpr int kWarps = 8;

struct Key {
  double v;
  int32_t j;
};

__device__ __forceinline__ bool before(double a, int32_t ia, double b, int32_t ib) {
  return a > b || (a == b && ia < ib);
}

// order-preserving map of a double to an unsigned key (larger value ->
// larger key; -0 is never produced by cos_from)
__device__ __forceinline__ unsigned long long dkey(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_value(unsigned long long k) {
  return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

// order-preserving map of a float to 32 bits
__device__ __forceinline__ uint32_t fkey(float v) {
  const uint32_t b = __float_as_uint(v);
  return (b >> 31) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_value(uint32_t k) { return __uint_as_float((k >> 31) ? (k & 0x7fffffffu) : ~k); }

// key of a normalised float-float value hi + lo (|lo| <= ulp(hi) / 2): by hi,
// then by lo
__device__ __forceinline__ unsigned long long ffkey(float hi, float lo) {
  return ((unsigned long long)fkey(hi) << 32) | fkey(lo);
}

// bitonic sort of one (key, index) pair per lane: lane 0 ends with the first
// element of the (key desc, index asc) order
__device__ __forceinline__ void warp_sort_key(unsigned long long& key, int32_t& j) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int s = k >> 1; s > 0; s >>= 1) {
      const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, s);
      const int32_t oj = __shfl_xor_sync(0xffffffffu, j, s);
      const bool lower = (lane & s) == 0;
      const bool dir = (lane & k) == 0;
      const bool self_first = key > ok || (key == ok && j < oj);
      const bool take = (lower == dir) ? !self_first : self_first;
      if (take) {
        key = ok;
        j = oj;
      }
    }
  }
}

// the same order on FP64 values, through integer keys (the FP64 pipe is
// narrow on this part)
__device__ __forceinline__ void warp_sort(double& v, int32_t& j) {
  unsigned long long key = dkey(v);
  warp_sort_key(key, j);
  v = dkey_value(key);
}

// Dot2 dot product of rows i and j with a warp: (s, c) with s + c the
// compensated result, the same in every lane (fixed-order merge)
__device__ __forceinline__ void dot2_rows(const float* __restrict__ xi, const float* __restrict__ xj, int d, float& s,
                                          float& c) {
  const int lane = threadIdx.x & 31;
  s = 0.f;
  c = 0.f;
  // eight strided loads per lane in flight before the compensated steps;
  // padding contributes exact zeros, which leave (s, c) unchanged
  for (int t0 = lane; t0 < d; t0 += 32 * 8) {
    float a[8], b[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = t0 + 32 * u;
      a[u] = t < d ? xi[t] : 0.f;
      b[u] = t < d ? xj[t] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) dot2_step(s, c, a[u], b[u]);
  }
  dot2_warp_reduce(s, c);
}

// cosine from the compensated dot product and the rows' inverse norms
// (0 for a zero row), evaluated in double; +0 for a zero result
__device__ __forceinline__ double cos_from(float s, float c, double ri, double rj) {
  return ((double)s + (double)c) * ri * rj + 0.0;
}

// (ah + al)(bh + bl) as a normalised float-float pair (TwoProd by FMA, the
// cross terms added to the error, then a fast TwoSum)
__device__ __forceinline__ void ff_mul(float ah, float al, float bh, float bl, float& ph, float& pl) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  ph = p + e;
  pl = e - (ph - p);
}

// the same cosine in float-float on the FP32 pipe: the Dot2 pair times the
// inverse norms (float-float pairs); +0 for a zero result.  Its error is
// that of the Dot2 sum (~2^-44 relative), as in the FP64 form.
__device__ __forceinline__ void cos_ff(float s, float c, float2 ri, float2 rj, float& h, float& l) {
  float sh, sl;
  two_sum(s, c, sh, sl);
  float th, tl;
  ff_mul(sh, sl, ri.x, ri.y, th, tl);
  ff_mul(th, tl, rj.x, rj.y, h, l);
  h = h + 0.f;
}

// Per-lane Dot2 partials of row i with up to four rows j[u] (j[u] < 0:
// skipped) for dot2_reduce4: the loads of all four rows are issued before the
// Dot2 steps, and each sees the same per-lane order as dot2_rows.
__device__ __forceinline__ void dot2_rows4(const float* __restrict__ X, const float* __restrict__ xi, int d,
                                           const int32_t (&j)[4], float (&s)[4], float (&c)[4]) {
  const int lane = threadIdx.x & 31;
  const float* xj[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    xj[u] = X + (int64_t)(j[u] >= 0 ? j[u] : 0) * d;
    s[u] = 0.f;
    c[u] = 0.f;
  }
  for (int t0 = lane; t0 < d; t0 += 32 * 4) {
    float a[4], b[4][4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int t = t0 + 32 * v;
      a[v] = t < d ? xi[t] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int t = t0 + 32 * v;
        b[u][v] = (t < d && j[u] >= 0) ? xj[u][t] : 0.f;
      }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) dot2_step(s[u], c[u], a[v], b[u][v]);
  }
}

// (s, c) += (s2, c2) with the lower lane's partial first, as in
// dot2_warp_reduce (`upper`: this lane has the level's bit set)
__device__ __forceinline__ void dot2_merge_lanes(float& s, float& c, float s2, float c2, bool upper) {
  if (upper) {
    const float ts = s, tc = c;
    s = s2;
    c = c2;
    s2 = ts;
    c2 = tc;
  }
  dot2_merge(s, c, s2, c2);
}

// The butterfly of dot2_warp_reduce applied to four partials at once, each
// of the first two levels keeping half of them (a reduce-scatter): after it
// lane L holds the full sum of partial 2*bit4(L) + bit3(L), with every merge
// taking the same operands in the same order as the one-partial butterfly,
// so the bits are the same.  14 shuffles instead of 40.
__device__ __forceinline__ void dot2_reduce4(const float (&s)[4], const float (&c)[4], float& rs, float& rc) {
  const int lane = threadIdx.x & 31;
  const bool h16 = lane & 16, h8 = lane & 8;
  // level 16: keep {0,1} (bit clear) or {2,3}; send the other pair
  float ks0 = h16 ? s[2] : s[0], kc0 = h16 ? c[2] : c[0];
  float ks1 = h16 ? s[3] : s[1], kc1 = h16 ? c[3] : c[1];
  {
    const float o0 = __shfl_xor_sync(0xffffffffu, h16 ? s[0] : s[2], 16);
    const float p0 = __shfl_xor_sync(0xffffffffu, h16 ? c[0] : c[2], 16);
    const float o1 = __shfl_xor_sync(0xffffffffu, h16 ? s[1] : s[3], 16);
    const float p1 = __shfl_xor_sync(0xffffffffu, h16 ? c[1] : c[3], 16);
    dot2_merge_lanes(ks0, kc0, o0, p0, h16);
    dot2_merge_lanes(ks1, kc1, o1, p1, h16);
  }
  // level 8: keep the first (bit clear) or second of the pair
  rs = h8 ? ks1 : ks0;
  rc = h8 ? kc1 : kc0;
  {
    const float o = __shfl_xor_sync(0xffffffffu, h8 ? ks0 : ks1, 8);
    const float p = __shfl_xor_sync(0xffffffffu, h8 ? kc0 : kc1, 8);
    dot2_merge_lanes(rs, rc, o, p, h8);
  }
#pragma unroll
  for (int off = 4; off >= 1; off >>= 1) {
    const float o = __shfl_xor_sync(0xffffffffu, rs, off);
    const float p = __shfl_xor_sync(0xffffffffu, rc, off);
    dot2_merge_lanes(rs, rc, o, p, (lane & off) != 0);
  }
}

// the lane of the same octet position that holds partial u after dot2_reduce4
__device__ __forceinline__ int dot2_reduce4_src(int u, int lane) { return ((u >> 1) << 4) | ((u & 1) << 3) | (lane & 7); }

// Sparse row i: each lane keeps the positions t of its strided share
// (t = lane + 32m) where x_i[t] != 0, in increasing order.  A zero x_i[t]
// makes the Dot2 step (s, c) += x_i[t] x_j[t] an exact no-op (for finite
// x_j[t]), so stepping over only these positions gives the dense loop's
// values; only x_j at these positions is read.
constexpr int kSpLane = 4;  // positions kept per lane; a row with more uses the dense loop
struct SparseRow {
  int t[kSpLane];
  float a[kSpLane];
  int cnt;   // this lane's nonzeros (may exceed kSpLane)
  int cmax;  // the largest count over the warp
};

__device__ __forceinline__ void sparse_row(const float* __restrict__ xi, int d, SparseRow& r) {
  const int lane = threadIdx.x & 31;
  r.cnt = 0;
#pragma unroll
  for (int q = 0; q < kSpLane; ++q) {
    r.t[q] = 0;
    r.a[q] = 0.f;
  }
  for (int t0 = lane; t0 < d; t0 += 32 * 8) {
    float x[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const int t = t0 + 32 * v;
      x[v] = t < d ? xi[t] : 0.f;
    }
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      if (x[v] != 0.f) {
#pragma unroll
        for (int q = 0; q < kSpLane; ++q)
          if (r.cnt == q) {
            r.t[q] = t0 + 32 * v;
            r.a[q] = x[v];
          }
        ++r.cnt;
      }
    }
  }
  r.cmax = __reduce_max_sync(0xffffffffu, (unsigned)r.cnt);
}

// Dot2 partials of row i (sparse form, r.cmax <= kSpLane) with up to four
// rows j[u] (j[u] < 0: skipped); the gathers of all four are issued first
__device__ __forceinline__ void dot2_sparse4(const float* __restrict__ X, int d, const SparseRow& r,
                                             const int32_t (&j)[4], float (&s)[4], float (&c)[4]) {
  float b[4][kSpLane];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const float* xj = X + (int64_t)(j[u] >= 0 ? j[u] : 0) * d;
    s[u] = 0.f;
    c[u] = 0.f;
#pragma unroll
    for (int q = 0; q < kSpLane; ++q) b[u][q] = (q < r.cnt && j[u] >= 0) ? xj[r.t[q]] : 0.f;
  }
#pragma unroll
  for (int q = 0; q < kSpLane; ++q) {
    if (q < r.cmax) {  // warp-uniform
#pragma unroll
      for (int u = 0; u < 4; ++u) dot2_step(s[u], c[u], r.a[q], b[u][q]);
    }
  }
}

__global__ void k_inv_norms(const double* __restrict__ nrm2, int64_t n, double* __restrict__ rinv,
                            float2* __restrict__ rinv2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double r = nrm2[i] > 0.0 ? 1.0 / sqrt(nrm2[i]) : 0.0;
  rinv[i] = r;
  const float h = (float)r;
  rinv2[i] = make_float2(h, (float)(r - (double)h));
}

__global__ void __launch_bounds__(kWarps * 32, 3)
k_rerank(const float* __restrict__ X, const int32_t* __restrict__ rows_in, int64_t n_rows, int d, int K,
         const float* __restrict__ err,
         const float* __restrict__ err_max_p, float acc_coef, const float2* __restrict__ rinv2,
         const float* __restrict__ cand_val, const int32_t* __restrict__ cand_idx, int lists,
         int32_t* __restrict__ out_idx, float* __restrict__ out_sim, int32_t* __restrict__ fb_rows,
         float* __restrict__ fb_thr, int32_t* __restrict__ fb_count, unsigned long long* __restrict__ n_cand,
         const int32_t* __restrict__ list_err) {
  if (list_err && *list_err) return;  // the list pass failed: its lists are not valid (uniform over the grid)
  __shared__ unsigned int block_cand;
  if (threadIdx.x == 0) block_cand = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (w < n_rows) {
    const int64_t i = rows_in ? (int64_t)rows_in[w] : w;  // all rows, or the listed ones
    float v = cand_val[i * kCandC + lane];
    int32_t j = cand_idx[i * kCandC + lane];
    const bool valid = j >= 0;
    const unsigned vmask = __ballot_sync(0xffffffffu, valid);
    const int nvalid = __popc(vmask);
    const float ei = err[i], emax = *err_max_p;
    const float ej = valid ? err[j] : 0.f;
    const float2 rj2 = valid ? rinv2[j] : make_float2(0.f, 0.f);  // used by this lane if j is re-scored
    // row i's nonzeros, read while the candidate loads are in flight
    const float* xi = X + i * (int64_t)d;
    SparseRow sp;
    sparse_row(xi, d, sp);
    const float m = ei * (1.f + ej) + ej + acc_coef * (1.f + ei) * (1.f + ej);
    const float lower = valid ? v - m : -INFINITY;
    const float upper = valid ? v + m : -INFINITY;
    // K-th largest lower bound (ties by lane)
    int rank = 0;
    for (int t = 0; t < 32; ++t) {
      float o = __shfl_sync(0xffffffffu, lower, t);
      rank += (o > lower) || (o == lower && t < lane);
    }
    const unsigned kmask = __ballot_sync(0xffffffffu, rank == K - 1);
    const float lb = __shfl_sync(0xffffffffu, lower, __ffs(kmask) - 1);
    bool ok = nvalid >= K;
    const float mmax = ei * (1.f + emax) + emax + acc_coef * (1.f + ei) * (1.f + emax);
    // The candidates come as `lists` lists of 32/lists lanes, each the best
    // scores of its own share of the keys.  A full list bounds the keys of its
    // share that it did not keep by its minimum; a list that is not full kept
    // every key of its share.
    {
      const int per = 32 / lists;
      float gmin = valid ? v : INFINITY;
      for (int off = per / 2; off >= 1; off >>= 1) gmin = fminf(gmin, __shfl_xor_sync(0xffffffffu, gmin, off));
      const unsigned gmask = per == 32 ? 0xffffffffu : (((1u << per) - 1u) << ((lane / per) * per));
      const bool gfull = __popc(vmask & gmask) == per;
      float U = gfull ? gmin : -INFINITY;
      for (int off = per; off < 32; off <<= 1) U = fmaxf(U, __shfl_xor_sync(0xffffffffu, U, off));
      if (__any_sync(0xffffffffu, gfull)) {
        // strict: every outside node's cosine is < lb <= the true K-th value
        ok = ok && (U + mmax < lb);
      }
    }
    if (!ok) {
      // a key j can be in the list only if s^_ij >= lb - m_ij >= lb - mmax
      if (lane == 0) {
        const int pos = atomicAdd(fb_count, 1);
        fb_rows[pos] = (int32_t)i;
        if (fb_thr) fb_thr[pos] = nvalid >= K ? lb - mmax : -INFINITY;
      }
    } else {
      const bool inR = valid && upper >= lb;
      unsigned rmask = __ballot_sync(0xffffffffu, inR);
      if (lane == 0) atomicAdd(&block_cand, (unsigned)__popc(rmask));
      const float2 ri = rinv2[i];
      unsigned long long myk = 0;  // below every cosine's key
      int32_t myj = INT32_MAX;
      const bool sparse = sp.cmax <= kSpLane && sp.cmax < (d + 31) / 32;  // warp-uniform
      while (rmask) {  // four candidates per pass
        int tl[4];
        int32_t jt[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          tl[u] = rmask ? __ffs(rmask) - 1 : -1;
          if (rmask) rmask &= rmask - 1;
          jt[u] = __shfl_sync(0xffffffffu, j, tl[u] >= 0 ? tl[u] : 0);
          if (tl[u] < 0) jt[u] = -1;
        }
        float ds[4], dc[4];
        if (sparse)
          dot2_sparse4(X, d, sp, jt, ds, dc);
        else
          dot2_rows4(X, xi, d, jt, ds, dc);
        float rs, rc;
        dot2_reduce4(ds, dc, rs, rc);
        // each lane owns at most one of the four candidates (its own j); fetch its sum
        int own = -1;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (lane == tl[u]) own = u;
        const int src = own >= 0 ? dot2_reduce4_src(own, lane) : lane;
        rs = __shfl_sync(0xffffffffu, rs, src);
        rc = __shfl_sync(0xffffffffu, rc, src);
        if (own >= 0) {  // the owner lane alone evaluates its cosine
          float h, l;
          cos_ff(rs, rc, ri, rj2, h, l);
          myk = ffkey(h, l);
          myj = j;
        }
      }
      warp_sort_key(myk, myj);
      if (lane < K) {
        out_idx[i * K + lane] = myj;
        out_sim[i * K + lane] = fkey_value((uint32_t)(myk >> 32));
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && n_cand) atomicAdd(n_cand, (unsigned long long)block_cand);
}

// Exhaustive exact list for the flagged rows (or every row when K exceeds
// what the candidate list can certify).  One CTA per row; each warp keeps a
// sorted top-K of its own strided share of the keys in shared memory, and
// thread 0 merges the warp lists.
constexpr int kExWarps = 8;
constexpr int kMaxK = 64;
constexpr int kSlices = 64;           // key slices per flagged row
constexpr int kSlicedMaxRows = 1024;  // flagged rows handled by the sliced kernels

__global__ void __launch_bounds__(kExWarps * 32)
k_knn_exhaustive(const float* __restrict__ X, int64_t n, int d, int K, const double* __restrict__ rinv,
                 const int32_t* __restrict__ rows, const int32_t* __restrict__ row_count,
                 int64_t all_rows, int32_t* __restrict__ out_idx, float* __restrict__ out_sim) {
  __shared__ double lv[kExWarps][kMaxK];
  __shared__ int32_t li[kExWarps][kMaxK];
  __shared__ int head[kExWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t count = rows ? (int64_t)*row_count : all_rows;
  if (rows && count <= kSlicedMaxRows) return;  // few rows: the sliced kernels take them
  for (int64_t r = blockIdx.x; r < count; r += gridDim.x) {
    const int64_t i = rows ? rows[r] : r;
    for (int t = threadIdx.x; t < kExWarps * kMaxK; t += blockDim.x) {
      lv[t / kMaxK][t % kMaxK] = -INFINITY;
      li[t / kMaxK][t % kMaxK] = INT32_MAX;
    }
    __syncthreads();
    const float* xi = X + i * (int64_t)d;
    const double ri = rinv[i];
    for (int64_t j = w; j < n; j += kExWarps) {
      if (j == i) continue;
      float ds, dc;
      dot2_rows(xi, X + j * (int64_t)d, d, ds, dc);
      if (lane == 0) {
        const double cs = cos_from(ds, dc, ri, rinv[j]);
        if (before(cs, (int32_t)j, lv[w][K - 1], li[w][K - 1])) {
          int p = K - 1;
          while (p > 0 && before(cs, (int32_t)j, lv[w][p - 1], li[w][p - 1])) {
            lv[w][p] = lv[w][p - 1];
            li[w][p] = li[w][p - 1];
            --p;
          }
          lv[w][p] = cs;
          li[w][p] = (int32_t)j;
        }
      }
      __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int q = 0; q < kExWarps; ++q) head[q] = 0;
      for (int o = 0; o < K; ++o) {
        int best = -1;
        for (int q = 0; q < kExWarps; ++q) {
          if (head[q] >= K) continue;
          if (best < 0 || before(lv[q][head[q]], li[q][head[q]], lv[best][head[best]], li[best][head[best]]))
            best = q;
        }
        out_idx[i * K + o] = li[best][head[best]];
        out_sim[i * K + o] = (float)lv[best][head[best]];
        ++head[best];
      }
    }
    __syncthreads();
  }
}

// Exact re-rank of the keys collected for flagged rows (every key whose
// low-precision score reached the row's threshold): batches of 32 exact
// cosines are sorted and merged into a running (value desc, index asc) top-32.
// A row whose buffer overflowed (or holds fewer than K keys) goes to the
// exhaustive kernels.
__global__ void __launch_bounds__(kWarps * 32)
k_rerank_collected(const float* __restrict__ X, int d, int K, const double* __restrict__ rinv,
                   const int32_t* __restrict__ rows, const int32_t* __restrict__ n_rows_p,
                   const int32_t* __restrict__ cnt, const int32_t* __restrict__ buf, int cap,
                   int32_t* __restrict__ out_idx, float* __restrict__ out_sim, int32_t* __restrict__ ov_rows,
                   int32_t* __restrict__ ov_count, const int32_t* __restrict__ collect_err) {
  if (*collect_err) return;  // the collect pass failed: its buffers are not valid
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (r >= *n_rows_p) return;
  const int64_t i = rows[r];
  const int c = cnt[r];
  if (c > cap || c < K) {
    if (lane == 0) ov_rows[atomicAdd(ov_count, 1)] = (int32_t)i;
    return;
  }
  const float* xi = X + i * (int64_t)d;
  const double ri = rinv[i];
  double tv = -INFINITY;
  int32_t tj = INT32_MAX;
  for (int q0 = 0; q0 < c; q0 += 32) {
    const int32_t mine = (q0 + lane < c) ? buf[r * (int64_t)cap + q0 + lane] : -1;
    double nv = -INFINITY;
    int32_t nj = INT32_MAX;
    const int nb = min(32, c - q0);
    for (int t = 0; t < nb; ++t) {
      const int32_t jt = __shfl_sync(0xffffffffu, mine, t);
      float ds, dc;
      dot2_rows(xi, X + (int64_t)jt * d, d, ds, dc);
      if (lane == t) {
        nv = cos_from(ds, dc, ri, rinv[jt]);
        nj = jt;
      }
    }
    warp_sort(nv, nj);
    // best of the running list and the reversed new batch (a bitonic sequence)
    const double rv = __shfl_sync(0xffffffffu, nv, 31 - lane);
    const int32_t rj = __shfl_sync(0xffffffffu, nj, 31 - lane);
    if (before(rv, rj, tv, tj)) {
      tv = rv;
      tj = rj;
    }
    warp_sort(tv, tj);
  }
  if (lane < K) {
    out_idx[i * K + lane] = tj;
    out_sim[i * K + lane] = (float)tv;
  }
}

// Few flagged rows: each row is split into kSlices key slices handled by
// separate CTAs (the whole GPU streams X once per row instead of one SM);
// every CTA writes the exact top-K of its slice, k_exh_merge combines them.
__global__ void __launch_bounds__(kExWarps * 32)
k_exh_sliced(const float* __restrict__ X, int64_t n, int d, int K, const double* __restrict__ rinv,
             const int32_t* __restrict__ rows, const int32_t* __restrict__ row_count, double* __restrict__ pv,
             int32_t* __restrict__ pi) {
  __shared__ double lv[kExWarps][kMaxK];
  __shared__ int32_t li[kExWarps][kMaxK];
  __shared__ int head[kExWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t count = *row_count;
  if (count > kSlicedMaxRows) return;
  for (int64_t item = blockIdx.x; item < count * kSlices; item += gridDim.x) {
    const int64_t r = item / kSlices;
    const int sl = (int)(item % kSlices);
    const int64_t i = rows[r];
    const int64_t j0 = n * sl / kSlices, j1 = n * (sl + 1) / kSlices;
    for (int t = threadIdx.x; t < kExWarps * kMaxK; t += blockDim.x) {
      lv[t / kMaxK][t % kMaxK] = -INFINITY;
      li[t / kMaxK][t % kMaxK] = INT32_MAX;
    }
    __syncthreads();
    const float* xi = X + i * (int64_t)d;
    const double ri = rinv[i];
    for (int64_t j = j0 + w; j < j1; j += kExWarps) {
      if (j == i) continue;
      float ds, dc;
      dot2_rows(xi, X + j * (int64_t)d, d, ds, dc);
      if (lane == 0) {
        const double cs = cos_from(ds, dc, ri, rinv[j]);
        if (before(cs, (int32_t)j, lv[w][K - 1], li[w][K - 1])) {
          int p = K - 1;
          while (p > 0 && before(cs, (int32_t)j, lv[w][p - 1], li[w][p - 1])) {
            lv[w][p] = lv[w][p - 1];
            li[w][p] = li[w][p - 1];
            --p;
          }
          lv[w][p] = cs;
          li[w][p] = (int32_t)j;
        }
      }
      __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int q = 0; q < kExWarps; ++q) head[q] = 0;
      for (int o = 0; o < K; ++o) {
        int best = 0;
        for (int q = 1; q < kExWarps; ++q)
          if (before(lv[q][head[q]], li[q][head[q]], lv[best][head[best]], li[best][head[best]])) best = q;
        pv[(r * kSlices + sl) * K + o] = lv[best][head[best]];
        pi[(r * kSlices + sl) * K + o] = li[best][head[best]];
        if (head[best] < K - 1) ++head[best];
        else { lv[best][head[best]] = -INFINITY; li[best][head[best]] = INT32_MAX; }
      }
    }
    __syncthreads();
  }
}

__global__ void k_exh_merge(const int32_t* __restrict__ rows, const int32_t* __restrict__ row_count, int K,
                            const double* __restrict__ pv, const int32_t* __restrict__ pi,
                            int32_t* __restrict__ out_idx, float* __restrict__ out_sim) {
  const int64_t count = *row_count;
  if (count > kSlicedMaxRows) return;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < count; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = rows[r];
    int head[kSlices];
    for (int q = 0; q < kSlices; ++q) head[q] = 0;
    const double* v = pv + r * kSlices * K;
    const int32_t* x = pi + r * kSlices * K;
    for (int o = 0; o < K; ++o) {
      int best = -1;
      for (int q = 0; q < kSlices; ++q) {
        if (head[q] >= K) continue;
        if (best < 0 || before(v[q * K + head[q]], x[q * K + head[q]], v[best * K + head[best]], x[best * K + head[best]]))
          best = q;
      }
      out_idx[i * K + o] = x[best * K + head[best]];
      out_sim[i * K + o] = (float)v[best * K + head[best]];
      ++head[best];
    }
  }
}

}  // namespace

ancka_status knn_rerank(Workspace& ws, const float* X, int64_t n, int32_t d, int32_t K,
                        const PrepOut& pr, int list_prec, float acc_coef, float acc_bf16, float* cand_val,
                        int32_t* cand_idx, int lists, int collect_prec, const int32_t* list_err, int32_t* out_idx,
                        float* out_sim, int64_t* n_candidates, int64_t* n_fallback, int64_t* n_exhaustive,
                        bool want_counts, cudaStream_t s) {
  int32_t *fb_rows, *fb_count;
  unsigned long long* ncand;
  double* rinv;
  float2* rinv2;
  ANCKA_TRY(ws.alloc(&rinv, (size_t)n));
  ANCKA_TRY(ws.alloc(&rinv2, (size_t)n));
  k_inv_norms<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(pr.nrm2, n, rinv, rinv2);
  ANCKA_LAUNCHED();
  ANCKA_TRY(ws.alloc(&fb_rows, (size_t)n));
  ANCKA_TRY(ws.zeros(&fb_count, 1));
  ANCKA_TRY(ws.zeros(&ncand, 1));
  const int32_t* collect_err = nullptr;  // read back with the counts at the end
  const int32_t* ex_count_dev = nullptr;
  const bool use_candidates = cand_val != nullptr;
  if (use_candidates) {
    const bool fp8 = list_prec == ANCKA_PREC_FP8;
    float* fb_thr = nullptr;
    if (collect_prec == ANCKA_PREC_BF16 && !fp8) ANCKA_TRY(ws.alloc(&fb_thr, (size_t)n));
    k_rerank<<<(unsigned)ceil_div(n, kWarps), kWarps * 32, 0, s>>>(
        X, nullptr, n, d, K, fp8 ? pr.err8 : pr.err, fp8 ? pr.err8_max : pr.err_max, acc_coef, rinv2, cand_val,
        cand_idx, lists, out_idx, out_sim, fb_rows, fb_thr, fb_count, ncand, list_err);
    ANCKA_LAUNCHED();
    int32_t* cl_rows = fb_rows;   // rows for the collect pass, their count and thresholds
    int32_t* cl_count = fb_count;
    float* cl_thr = fb_thr;
    if (fp8) {
      // rows the FP8 lists could not certify: BF16 lists for those rows, then
      // the BF16 certificate; what it cannot settle goes to the collect pass
      int32_t nf8 = 0, le = 0;
      ANCKA_CUDA(cudaMemcpyAsync(&nf8, fb_count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      if (list_err) ANCKA_CUDA(cudaMemcpyAsync(&le, list_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      ANCKA_CUDA(cudaStreamSynchronize(s));
      if (le) {
        set_error("tensor-core contraction: a pipeline wait expired (role %d)", le);
        return ANCKA_ERR_TIMEOUT;
      }
      list_err = nullptr;  // checked
      ANCKA_TRY(ws.alloc(&cl_rows, (size_t)(nf8 > 0 ? nf8 : 1)));
      ANCKA_TRY(ws.zeros(&cl_count, 1));
      ANCKA_TRY(ws.alloc(&cl_thr, (size_t)(nf8 > 0 ? nf8 : 1)));
      if (nf8 > 0) {
        int32_t* terr;
        ANCKA_TRY(ws.zeros(&terr, 1));
        ANCKA_TRY(knn_list_gathered_bf16(ws, pr, n, fb_rows, nf8, cand_val, cand_idx, terr, s));
        k_rerank<<<(unsigned)ceil_div(nf8, kWarps), kWarps * 32, 0, s>>>(
            X, fb_rows, nf8, d, K, pr.err, pr.err_max, acc_bf16, rinv2, cand_val, cand_idx, 2, out_idx, out_sim,
            cl_rows, cl_thr, cl_count, ncand, terr);
        ANCKA_LAUNCHED();
        list_err = terr;  // reported with the next read
      }
    }
    int32_t* ex_rows = cl_rows;
    int32_t* ex_count = cl_count;
    if (collect_prec == ANCKA_PREC_BF16) {
      // flagged rows: collect every key above the row's certified threshold
      // with the tensor-core contraction, then re-rank those exactly
      int32_t nf = 0, le = 0;
      ANCKA_CUDA(cudaMemcpyAsync(&nf, cl_count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      if (list_err) ANCKA_CUDA(cudaMemcpyAsync(&le, list_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      ANCKA_CUDA(cudaStreamSynchronize(s));
      if (le) {
        set_error("tensor-core list pass: a pipeline wait expired (role %d)", le);
        return ANCKA_ERR_TIMEOUT;
      }
      list_err = nullptr;  // checked
      ANCKA_TRY(ws.zeros(&ex_count, 1));
      ANCKA_TRY(ws.alloc(&ex_rows, (size_t)(nf > 0 ? nf : 1)));
      if (nf > 0) {
        constexpr int kCap = 2048;
        int32_t *cnt, *buf, *terr;
        ANCKA_TRY(ws.zeros(&cnt, (size_t)nf));
        ANCKA_TRY(ws.alloc(&buf, (size_t)nf * kCap));
        ANCKA_TRY(ws.zeros(&terr, 1));
        ANCKA_TRY(knn_collect_bf16(ws, pr, n, cl_rows, nf, cl_thr, cnt, buf, kCap, terr, s));
        k_rerank_collected<<<(unsigned)ceil_div(nf, kWarps), kWarps * 32, 0, s>>>(
            X, d, K, rinv, cl_rows, cl_count, cnt, buf, kCap, out_idx, out_sim, ex_rows, ex_count, terr);
        ANCKA_LAUNCHED();
        collect_err = terr;  // reported with the final read
      }
    }
    // rows left: sliced over the whole GPU when few, one CTA per row when many
    double* pv;
    int32_t* pi;
    ANCKA_TRY(ws.alloc(&pv, (size_t)kSlicedMaxRows * kSlices * K));
    ANCKA_TRY(ws.alloc(&pi, (size_t)kSlicedMaxRows * kSlices * K));
    k_exh_sliced<<<1216, kExWarps * 32, 0, s>>>(X, n, d, K, rinv, ex_rows, ex_count, pv, pi);
    ANCKA_LAUNCHED();
    k_exh_merge<<<8, 128, 0, s>>>(ex_rows, ex_count, K, pv, pi, out_idx, out_sim);
    ANCKA_LAUNCHED();
    k_knn_exhaustive<<<304, kExWarps * 32, 0, s>>>(X, n, d, K, rinv, ex_rows, ex_count, 0, out_idx,
                                                   out_sim);
    ANCKA_LAUNCHED();
    ex_count_dev = ex_count;
  } else {
    const unsigned g = (unsigned)(n < 4096 ? n : 4096);
    k_knn_exhaustive<<<g, kExWarps * 32, 0, s>>>(X, n, d, K, rinv, nullptr, nullptr, n, out_idx,
                                                 out_sim);
    ANCKA_LAUNCHED();
    if (n_exhaustive) *n_exhaustive = n;
  }
  // one host read for the counts and the error flags not read yet
  if (want_counts || collect_err || list_err) {
    int32_t fb = 0, ex = 0, ce = 0, le = 0;
    unsigned long long nc = 0;
    ANCKA_CUDA(cudaMemcpyAsync(&fb, fb_count, sizeof(fb), cudaMemcpyDeviceToHost, s));
    ANCKA_CUDA(cudaMemcpyAsync(&nc, ncand, sizeof(nc), cudaMemcpyDeviceToHost, s));
    if (ex_count_dev) ANCKA_CUDA(cudaMemcpyAsync(&ex, ex_count_dev, sizeof(ex), cudaMemcpyDeviceToHost, s));
    if (collect_err) ANCKA_CUDA(cudaMemcpyAsync(&ce, collect_err, sizeof(ce), cudaMemcpyDeviceToHost, s));
    if (list_err) ANCKA_CUDA(cudaMemcpyAsync(&le, list_err, sizeof(le), cudaMemcpyDeviceToHost, s));
    ANCKA_CUDA(cudaStreamSynchronize(s));
    if (le) {
      set_error("tensor-core list pass: a pipeline wait expired (role %d)", le);
      return ANCKA_ERR_TIMEOUT;
    }
    if (ce) {
      set_error("tensor-core collect pass: a pipeline wait expired (role %d)", ce);
      return ANCKA_ERR_TIMEOUT;
    }
    if (want_counts) {
      *n_fallback = use_candidates ? fb : n;
      *n_candidates = (int64_t)nc;
      if (ex_count_dev && n_exhaustive) *n_exhaustive = ex;
    }
  }
  return ANCKA_OK;
}

}  // namespace ancka
