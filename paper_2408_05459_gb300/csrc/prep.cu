// Row preparation for the KNN contraction (Alg. 6 lines 1-2: normalise rows).
//
// One warp per row: ||x||^2 with a compensated (Dot2) sum, the unit row in
// FP32 or BF16 (zero-padded to the tile width), and an upper bound of the
// copy's distance to the exact unit vector x/||x||:
//     err_i >= || copy_i - x_i/||x_i|| ||_2 .
// The bound feeds the candidate certificate of the re-rank: for unit rows
// |cos_ij - copy_i . copy_j| <= err_i (1 + err_j) + err_j + (accumulation).
#include "common.cuh"

namespace ancka {

namespace {

constexpr int kPrepWarps = 8;

// slack covering the FP32 rounding of the unit row itself: the computed
// u = x * (1/||x||) is within 4 unit roundoffs of x/||x|| per element, i.e.
// ||u - x/||x|||| <= 2^-22; twice that is used.
constexpr float kUnitSlack = 4.8e-7f;

__global__ void __launch_bounds__(kPrepWarps * 32)
k_prep_rows(const float* __restrict__ X, int64_t n, int32_t d, int32_t dp, int prec,
            float* __restrict__ xu32, __nv_bfloat16* __restrict__ xb, float* __restrict__ err,
            double* __restrict__ nrm2, int32_t* __restrict__ zero_row,
            unsigned int* __restrict__ err_max_bits, int64_t n_pad) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * kPrepWarps + (threadIdx.x >> 5);
  if (row >= n_pad) return;
  if (row >= n) {  // padding rows of the copy are zero
    for (int c = lane; c < dp; c += 32) {
      if (xu32) xu32[row * dp + c] = 0.f;
      if (xb) xb[row * dp + c] = __float2bfloat16_rn(0.f);
    }
    return;
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
  float inv = any ? (float)(1.0 / sqrt(n2)) : 0.f;
  float e2 = 0.f;
  for (int c = lane; c < dp; c += 32) {
    float u = c < d ? x[c] * inv : 0.f;
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
  if (lane == 0) {
    float e = any ? sqrtf(e2) * (1.f + 1e-6f) + kUnitSlack : 0.f;
    err[row] = e;
    nrm2[row] = n2;
    zero_row[row] = any ? 0 : 1;
    atomicMax(err_max_bits, __float_as_uint(e));  // non-negative floats order as uints
  }
}

}  // namespace

ancka_status prep_rows(Workspace& ws, const float* X, int64_t n, int32_t d, int prec, PrepOut* out,
                       cudaStream_t s) {
  PrepOut o{};
  // BF16 tiles consume 64 features (128 bytes) per pipeline stage; the FP32
  // SIMT tiles consume 8.  Rows are padded to the 128-row tile height.
  o.dp = (int32_t)(prec == ANCKA_PREC_BF16 ? round_up(d, 64) : round_up(d, 8));
  o.n_pad = round_up(n, 128);
  if (prec == ANCKA_PREC_BF16) {
    ANCKA_TRY(ws.alloc(&o.xb, (size_t)o.n_pad * o.dp));
  } else {
    ANCKA_TRY(ws.alloc(&o.xu32, (size_t)o.n_pad * o.dp));
  }
  ANCKA_TRY(ws.alloc(&o.err, (size_t)n));
  ANCKA_TRY(ws.alloc(&o.nrm2, (size_t)n));
  ANCKA_TRY(ws.alloc(&o.zero_row, (size_t)n));
  ANCKA_TRY(ws.zeros(&o.err_max, 1));
  dim3 grid((unsigned)ceil_div(o.n_pad, kPrepWarps));
  k_prep_rows<<<grid, kPrepWarps * 32, 0, s>>>(X, n, d, o.dp, prec, o.xu32, o.xb, o.err, o.nrm2,
                                               o.zero_row, reinterpret_cast<unsigned int*>(o.err_max),
                                               o.n_pad);
  ANCKA_LAUNCHED();
  *out = o;
  return ANCKA_OK;
}

}  // namespace ancka
