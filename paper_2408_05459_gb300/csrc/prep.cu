// Row preparation for the KNN contraction (Alg. 6 lines 1-2: normalise rows).
//
// One warp per row: ||x||^2 with a compensated (Dot2) sum, the unit row in
// FP32 or BF16 (zero-padded to the tile width), and an upper bound of the
// copy's distance to the exact unit vector x/||x||:
//     err_i >= || copy_i - x_i/||x_i|| ||_2 .
// The bound feeds the candidate certificate of the re-rank: for unit rows
// |cos_ij - copy_i . copy_j| <= err_i (1 + err_j) + err_j + (accumulation).
#include <cuda_fp8.h>

#include "common.cuh"

namespace ancka {

namespace {

constexpr int kPrepWarps = 8;

// slack covering the FP32 rounding of the unit row itself: the computed
// u = x * (1/||x||) is within 4 unit roundoffs of x/||x|| per element, i.e.
// ||u - x/||x|||| <= 2^-22; twice that is used.
constexpr float kUnitSlack = 4.8e-7f;

// the FP32 sum of dp squares (fmaf, in any order) is within a factor
// 1 + (dp + 1) 2^-24 of the exact sum; its square root within half that
__device__ __forceinline__ float norm_slack(int dp) { return 1.f + (float)(dp + 2) * 5.9604645e-8f; }

// Warps take rows grid-stride; the largest bound and the largest |u| are
// kept per warp, combined per CTA in shared memory and published with one
// atomicMax per CTA (one per row serialised on a single address: 2.4 ms for
// 2.4e6 rows).
__global__ void __launch_bounds__(kPrepWarps * 32)
k_prep_rows(const float* __restrict__ X, int64_t n, int32_t d, int32_t dp, int prec,
            float* __restrict__ xu32, __nv_bfloat16* __restrict__ xb, float* __restrict__ err,
            double* __restrict__ nrm2, int32_t* __restrict__ zero_row,
            unsigned int* __restrict__ err_max_bits, unsigned int* __restrict__ umax_bits, int64_t n_pad) {
  __shared__ unsigned int wmax[kPrepWarps][2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // this warp's largest bound and |u| as float bits (non-negative floats, and
  // a NaN above them all, order as unsigned integers, as atomicMax sees them)
  unsigned int emax = 0u, umax = 0u;
  for (int64_t row = (int64_t)blockIdx.x * kPrepWarps + wid; row < n_pad; row += (int64_t)gridDim.x * kPrepWarps) {
    if (row >= n) {  // padding rows of the copy are zero
      for (int c = lane; c < dp; c += 32) {
        if (xu32) xu32[row * dp + c] = 0.f;
        if (xb) xb[row * dp + c] = __float2bfloat16_rn(0.f);
      }
      continue;
    }
    const float* x = X + row * (int64_t)d;
    float s = 0.f, cc = 0.f;
    bool any = false;
    for (int c = lane; c < d; c += 32) {
      float v = x[c];
      any |= (v != 0.f);
      dot2_step(s, cc, v, v);
    }
    dot2_warp_reduce(s, cc);
    any = __any_sync(0xffffffffu, any);
    double n2 = (double)s + (double)cc;
    // 1/||x|| in FP64 on one lane (GB300's FP64 pipe is narrow), then broadcast
    float inv = 0.f;
    if (lane == 0) inv = any ? (float)(1.0 / sqrt(n2)) : 0.f;
    inv = __shfl_sync(0xffffffffu, inv, 0);
    float e2 = 0.f, um = 0.f;
    for (int c = lane; c < dp; c += 32) {
      float u = c < d ? x[c] * inv : 0.f;
      um = fmaxf(um, fabsf(u));
      if (prec == ANCKA_PREC_BF16) {
        __nv_bfloat16 b = __float2bfloat16_rn(u);
        xb[row * dp + c] = b;
        float dq = __bfloat162float(b) - u;
        e2 = fmaf(dq, dq, e2);
      } else {
        xu32[row * dp + c] = u;
      }
    }
    e2 = warp_sum(e2);
    for (int off = 16; off >= 1; off >>= 1) um = fmaxf(um, __shfl_xor_sync(0xffffffffu, um, off));
    const float e = any ? sqrtf(e2) * norm_slack(dp) + kUnitSlack : 0.f;
    if (lane == 0) {
      err[row] = e;
      nrm2[row] = n2;
      zero_row[row] = any ? 0 : 1;
    }
    emax = max(emax, __float_as_uint(e));
    umax = max(umax, __float_as_uint(um));
  }
  if (lane == 0) {
    wmax[wid][0] = emax;
    wmax[wid][1] = umax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int a = 0u, b = 0u;
    for (int w = 0; w < kPrepWarps; ++w) {
      a = max(a, wmax[w][0]);
      b = max(b, wmax[w][1]);
    }
    atomicMax(err_max_bits, a);
    if (umax_bits) atomicMax(umax_bits, b);
  }
}

// the power-of-two scale of the FP8 copy: the largest S with S * max|u| <= 448
// (E4M3's largest finite value); S = 1 for an all-zero input
__device__ __forceinline__ float fp8_scale(const unsigned int* umax_bits) {
  const float um = __uint_as_float(*umax_bits);
  if (!(um > 0.f)) return 1.f;
  return ldexpf(1.f, (int)floorf(log2f(448.f / um)));
}

// E4M3 copy of S * unit rows (round to nearest even, saturating) and the
// exact distance bound err8_i >= || q_i / S - u_i ||, one warp per row.  The
// unit row u is formed as in k_prep_rows (same norm, same reciprocal).
__global__ void __launch_bounds__(kPrepWarps * 32)
k_prep_fp8(const float* __restrict__ X, int64_t n, int32_t d, int32_t dp8, const double* __restrict__ nrm2,
           const int32_t* __restrict__ zero_row, const unsigned int* __restrict__ umax_bits,
           uint8_t* __restrict__ x8, float* __restrict__ err8, unsigned int* __restrict__ err8_max_bits,
           float* __restrict__ inv_s2, int64_t n_pad) {
  __shared__ unsigned int wmax[kPrepWarps];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const float S = fp8_scale(umax_bits);
  if (blockIdx.x == 0 && threadIdx.x == 0) *inv_s2 = 1.f / (S * S);  // exact: a power of two
  const float invS = 1.f / S;
  unsigned int emax = 0u;  // bits of this warp's largest bound (see k_prep_rows)
  for (int64_t row = (int64_t)blockIdx.x * kPrepWarps + wid; row < n_pad; row += (int64_t)gridDim.x * kPrepWarps) {
    if (row >= n) {
      for (int c = lane; c < dp8; c += 32) x8[row * dp8 + c] = 0;
      continue;
    }
    const float* x = X + row * (int64_t)d;
    const bool zero = zero_row[row] != 0;
    float inv = 0.f;  // FP64 on one lane, then broadcast (as in k_prep_rows)
    if (lane == 0) inv = zero ? 0.f : (float)(1.0 / sqrt(nrm2[row]));
    inv = __shfl_sync(0xffffffffu, inv, 0);
    float e2 = 0.f;
    for (int c = lane; c < dp8; c += 32) {
      const float u = c < d ? x[c] * inv : 0.f;
      const __nv_fp8_e4m3 q(u * S);
      x8[row * dp8 + c] = q.__x;
      const float dq = (float)q * invS - u;  // exact: q / S is exact and within a factor 2 of u (or 0)
      e2 = fmaf(dq, dq, e2);
    }
    e2 = warp_sum(e2);
    const float e = zero ? 0.f : sqrtf(e2) * norm_slack(dp8) + kUnitSlack;
    if (lane == 0) err8[row] = e;
    emax = max(emax, __float_as_uint(e));
  }
  if (lane == 0) wmax[wid] = emax;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int a = 0u;
    for (int w = 0; w < kPrepWarps; ++w) a = max(a, wmax[w]);
    atomicMax(err8_max_bits, a);
  }
}

}  // namespace

ancka_status prep_rows(Workspace& ws, const float* X, int64_t n, int32_t d, int prec, PrepOut* out,
                       cudaStream_t s) {
  PrepOut o{};
  // BF16 tiles consume 64 features (128 bytes) per pipeline stage; the FP32
  // SIMT tiles consume 8.  Rows are padded to the 128-row tile height.
  const bool tc = prec == ANCKA_PREC_BF16 || prec == ANCKA_PREC_FP8;
  o.d = d;
  o.dp = (int32_t)(tc ? round_up(d, 64) : round_up(d, 8));
  o.n_pad = round_up(n, 128);
  if (tc) {
    ANCKA_TRY(ws.alloc(&o.xb, (size_t)o.n_pad * o.dp));
  } else {
    ANCKA_TRY(ws.alloc(&o.xu32, (size_t)o.n_pad * o.dp));
  }
  ANCKA_TRY(ws.alloc(&o.err, (size_t)n));
  ANCKA_TRY(ws.alloc(&o.nrm2, (size_t)n));
  ANCKA_TRY(ws.alloc(&o.zero_row, (size_t)n));
  ANCKA_TRY(ws.zeros(&o.err_max, 1));
  unsigned int* umax = nullptr;
  if (prec == ANCKA_PREC_FP8) ANCKA_TRY(ws.zeros(&umax, 1));
  const int64_t row_blocks = ceil_div(o.n_pad, kPrepWarps);
  dim3 grid_rows((unsigned)(row_blocks < 152 * 16 ? row_blocks : 152 * 16));
  k_prep_rows<<<grid_rows, kPrepWarps * 32, 0, s>>>(X, n, d, o.dp, tc ? ANCKA_PREC_BF16 : ANCKA_PREC_FP32, o.xu32, o.xb,
                                               o.err, o.nrm2, o.zero_row,
                                               reinterpret_cast<unsigned int*>(o.err_max), umax, o.n_pad);
  ANCKA_LAUNCHED();
  if (prec == ANCKA_PREC_FP8) {
    o.dp8 = (int32_t)round_up(d, 128);
    ANCKA_TRY(ws.alloc(&o.x8, (size_t)o.n_pad * o.dp8));
    ANCKA_TRY(ws.alloc(&o.err8, (size_t)n));
    ANCKA_TRY(ws.zeros(&o.err8_max, 1));
    ANCKA_TRY(ws.alloc(&o.inv_s2, 1));
    k_prep_fp8<<<grid_rows, kPrepWarps * 32, 0, s>>>(X, n, d, o.dp8, o.nrm2, o.zero_row, umax, o.x8, o.err8,
                                                reinterpret_cast<unsigned int*>(o.err8_max), o.inv_s2, o.n_pad);
    ANCKA_LAUNCHED();
  }
  *out = o;
  return ANCKA_OK;
}

}  // namespace ancka
