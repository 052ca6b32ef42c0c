// Learned warm start (an addition to the paper's method: an MLP predicts the
// initial n x k block instead of InitBCM).
//
//   features   A = [U | P_N U], U the unit rows of X (a zero row stays zero),
//              P_N the topology walk (Eqs. rw-hg, rw-ag, rw-mg), BF16, row
//              length kp = round_up(2d, 64), zero-padded;
//   forward    Z1 = A W1 + b1 on the tensor cores (tcgen05, BF16 operands,
//              FP32 accumulation), H = GELU(Z1), W = H W2 + b2 (CUDA cores);
//   loss       L = k - tr(G^-1 M^T M) + lam ||G/n - I||_F^2 with G = W^T W and
//              M = Q_t^T W (Q_t the target's k orthonormal columns): it
//              depends on W only through span(W) and its scale; dL/dW =
//              W C1 + Q_t C2 with C1 = 2 S + (4 lam / n)(G/n - I),
//              C2 = -2 M G^-1, S = G^-1 M^T M G^-1;
//   backward   dW2 = H^T dW, db2 = 1^T dW, dZ1 = (dW W2^T) * GELU'(Z1),
//              db1 = 1^T dZ1, dW1 = A^T dZ1 on the tensor cores (A^T and dZ1
//              in BF16, split over the node range);
//   update     Adam with FP32 master weights; W1^T refreshed in BF16.
// Reductions over nodes use float-float partial sums in a fixed order.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace ancka {

namespace {

constexpr int kHidden = 256;

__global__ void k_unit_rows(const float* __restrict__ X, int64_t n, int d, int ld, float* __restrict__ U) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= n) return;
  const float* x = X + i * d;
  float s = 0.f;
  for (int c = lane; c < d; c += 32) s = fmaf(x[c], x[c], s);
  s = warp_sum(s);
  const float inv = s > 0.f ? 1.f / sqrtf(s) : 0.f;
  for (int c = lane; c < ld; c += 32) U[i * ld + c] = c < d ? x[c] * inv : 0.f;
}

// A[i, :] = [U_i | PU_i | 0] in BF16 (n x kp); At = A^T (kp x n_pad, zero for
// i >= n) when requested
__global__ void k_pack_features(const float* __restrict__ U, const float* __restrict__ PU, int64_t n, int d, int ld,
                                int kp, __nv_bfloat16* __restrict__ A) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * kp) return;
  const int64_t i = t / kp;
  const int c = (int)(t % kp);
  const float v = c < d ? U[i * ld + c] : (c < 2 * d ? PU[i * ld + c - d] : 0.f);
  A[t] = __float2bfloat16_rn(v);
}

// 32 x 32 tile transpose of a BF16 matrix (rows x cols) into (cols x rows_pad)
__global__ void k_transpose_bf16(const __nv_bfloat16* __restrict__ A, int64_t rows, int cols, int64_t rows_pad,
                                 __nv_bfloat16* __restrict__ At) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int64_t r = r0 + q;
    const int c = c0 + threadIdx.x;
    tile[q][threadIdx.x] = (r < rows && c < cols) ? A[r * cols + c] : __float2bfloat16_rn(0.f);
  }
  __syncthreads();
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int c = c0 + q;
    const int64_t r = r0 + threadIdx.x;
    if (c < cols && r < rows_pad) At[(int64_t)c * rows_pad + r] = tile[threadIdx.x][q];
  }
}

// W = H W2 + b2, one warp per row (fixed-order butterfly per output)
__global__ void k_mlp_out(const float* __restrict__ H, int64_t n, const float* __restrict__ W2,
                          const float* __restrict__ b2, int k, float* __restrict__ W, int ldw) {
  extern __shared__ float w2s[];  // kHidden x k
  for (int e = threadIdx.x; e < kHidden * k; e += blockDim.x) w2s[e] = W2[e];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= n) return;
  float h[kHidden / 32];
#pragma unroll
  for (int j = 0; j < kHidden / 32; ++j) h[j] = H[i * kHidden + lane + 32 * j];
  for (int c = 0; c < k; ++c) {
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < kHidden / 32; ++j) acc = fmaf(h[j], w2s[(lane + 32 * j) * k + c], acc);
    acc = warp_sum(acc);
    if (lane == 0) W[i * ldw + c] = acc + b2[c];
  }
}

// (hi, lo) += (bh, bl): float-float addition
__device__ __forceinline__ void ffa(float& hi, float& lo, float bh, float bl) {
  float s, e;
  two_sum(hi, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(lo, bl));
  hi = __fadd_rn(s, e);
  lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// partial[blk][a][b] = sum over the CTA's rows of X[r, a] Y[r, b] (X null:
// ones, p = 1), FP32 within 32-row tiles, float-float across tiles.  Thread a
// owns row a of the result, columns in chunks of 16.
constexpr int kXtyRows = 32;
__global__ void __launch_bounds__(256)
k_xty_partial(const float* __restrict__ X, int ldx, const float* __restrict__ Y, int ldy, int64_t n, int p, int q,
              float2* __restrict__ partial) {
  extern __shared__ float xs[];  // kXtyRows x (p + q)
  float* ys = xs + kXtyRows * p;
  const int64_t per = ceil_div(n, (int64_t)gridDim.x);
  const int64_t r0 = (int64_t)blockIdx.x * per;
  const int64_t r1 = (r0 + per < n) ? r0 + per : n;
  const int a = threadIdx.x;
  for (int b0 = 0; b0 < q; b0 += 16) {
    float hi[16], lo[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) hi[e] = lo[e] = 0.f;
    for (int64_t rb = r0; rb < r1; rb += kXtyRows) {
      const int rows = (int)((r1 - rb) < kXtyRows ? (r1 - rb) : kXtyRows);
      __syncthreads();
      for (int e = threadIdx.x; e < kXtyRows * p; e += blockDim.x) {
        const int r = e / p, c = e % p;
        xs[e] = r < rows ? (X ? X[(rb + r) * ldx + c] : 1.f) : 0.f;
      }
      for (int e = threadIdx.x; e < kXtyRows * q; e += blockDim.x) {
        const int r = e / q, c = e % q;
        ys[e] = r < rows ? Y[(rb + r) * ldy + c] : 0.f;
      }
      __syncthreads();
      if (a < p) {
        float acc[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[e] = 0.f;
        for (int r = 0; r < rows; ++r) {
          const float xa = xs[r * p + a];
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (b0 + e < q) acc[e] = fmaf(xa, ys[r * q + b0 + e], acc[e]);
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) ffa(hi[e], lo[e], acc[e], 0.f);
      }
    }
    if (a < p)
      for (int e = 0; e < 16 && b0 + e < q; ++e)
        partial[((int64_t)blockIdx.x * p + a) * q + b0 + e] = make_float2(hi[e], lo[e]);
  }
}

// out[a][b] = sum over blocks (in order) of the partials, as double
__global__ void k_xty_reduce(const float2* __restrict__ partial, int nblk, int p, int q, double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p * q) return;
  float hi = 0.f, lo = 0.f;
  for (int b = 0; b < nblk; ++b) {
    const float2 v = partial[(int64_t)b * p * q + t];
    ffa(hi, lo, v.x, v.y);
  }
  out[t] = (double)hi + (double)lo;
}

int xty_blocks(int64_t n) { return (int)std::min<int64_t>(304, std::max<int64_t>(1, ceil_div(n, 256))); }

ancka_status xty(Workspace& ws, const float* X, int ldx, const float* Y, int ldy, int64_t n, int p, int q,
                 double* out, cudaStream_t s) {
  const int nb = xty_blocks(n);
  float2* part;
  ANCKA_TRY(ws.alloc(&part, (size_t)nb * p * q));
  const size_t smem = (size_t)kXtyRows * (p + q) * sizeof(float);
  ANCKA_CUDA(cudaFuncSetAttribute(k_xty_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_xty_partial<<<nb, 256, smem, s>>>(X, ldx, Y, ldy, n, p, q, part);
  ANCKA_LAUNCHED();
  k_xty_reduce<<<(unsigned)ceil_div(p * q, 128), 128, 0, s>>>(part, nb, p, q, out);
  ANCKA_LAUNCHED();
  return ANCKA_OK;
}

// One CTA, FP64: from G = W^T W and M = Q_t^T W (k x k), the loss and the
// coefficient matrices of dL/dW = W C1 + Q_t C2.  G^-1 by Cholesky; a
// non-positive pivot sets *status.
__global__ void k_warm_coeffs(const double* __restrict__ G, const double* __restrict__ M, int k, double n, double lam,
                              float* __restrict__ C1, float* __restrict__ C2, double* __restrict__ loss,
                              int32_t* __restrict__ status) {
  extern __shared__ double sm[];
  double* R = sm;               // k x k Cholesky factor (upper)
  double* Gi = R + k * k;       // G^-1
  double* T1 = Gi + k * k;      // M^T M
  double* T2 = T1 + k * k;      // G^-1 M^T M
  double* Sm = T2 + k * k;      // S
  const int kk = k * k;
  for (int e = threadIdx.x; e < kk; e += blockDim.x) R[e] = 0.0;
  __syncthreads();
  for (int j = 0; j < k; ++j) {  // G = R^T R
    if (threadIdx.x == 0) {
      double dgn = G[j * k + j];
      for (int m = 0; m < j; ++m) dgn -= R[m * k + j] * R[m * k + j];
      if (!(dgn > 0.0)) {
        *status = 1;
        dgn = 1e-300;
      }
      R[j * k + j] = sqrt(dgn);
    }
    __syncthreads();
    for (int c = j + 1 + threadIdx.x; c < k; c += blockDim.x) {
      double v = G[j * k + c];
      for (int m = 0; m < j; ++m) v -= R[m * k + j] * R[m * k + c];
      R[j * k + c] = v / R[j * k + j];
    }
    __syncthreads();
  }
  // G^-1 = R^-1 R^-T: column c of R^-1 by back substitution (thread c), then Gi
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    for (int i = k - 1; i >= 0; --i) {  // X = R^-1 stored in T2 (column c)
      double v = (i == c) ? 1.0 : 0.0;
      for (int m = i + 1; m < k; ++m) v -= R[i * k + m] * T2[m * k + c];
      T2[i * k + c] = v / R[i * k + i];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kk; e += blockDim.x) {
    const int a = e / k, b = e % k;
    double v = 0.0;
    for (int m = 0; m < k; ++m) v += T2[a * k + m] * T2[b * k + m];
    Gi[e] = v;
    double w = 0.0;
    for (int m = 0; m < k; ++m) w += M[m * k + a] * M[m * k + b];
    T1[e] = w;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kk; e += blockDim.x) {
    const int a = e / k, b = e % k;
    double v = 0.0;
    for (int m = 0; m < k; ++m) v += Gi[a * k + m] * T1[m * k + b];
    T2[e] = v;  // G^-1 M^T M
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kk; e += blockDim.x) {
    const int a = e / k, b = e % k;
    double v = 0.0, u = 0.0;
    for (int m = 0; m < k; ++m) {
      v += T2[a * k + m] * Gi[m * k + b];   // S = G^-1 M^T M G^-1
      u += M[a * k + m] * Gi[m * k + b];    // M G^-1
    }
    Sm[e] = v;
    const double pen = G[e] / n - (a == b ? 1.0 : 0.0);
    C1[e] = (float)(2.0 * v + 4.0 * lam / n * pen);
    C2[e] = (float)(-2.0 * u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, pen = 0.0;
    for (int a = 0; a < k; ++a) tr += T2[a * k + a];
    for (int e = 0; e < kk; ++e) {
      const double v = G[e] / n - ((e / k) == (e % k) ? 1.0 : 0.0);
      pen += v * v;
    }
    *loss = (double)k - tr + lam * pen;
  }
}

// dW[i, c] = sum_a W[i, a] C1[a, c] + Qt[i, a] C2[a, c]
__global__ void k_grad_w(const float* __restrict__ W, int ldw, const float* __restrict__ Qt, int ldq, int64_t n, int k,
                         const float* __restrict__ C1, const float* __restrict__ C2, float* __restrict__ dW) {
  extern __shared__ float cs[];  // C1, C2
  for (int e = threadIdx.x; e < 2 * k * k; e += blockDim.x) cs[e] = e < k * k ? C1[e] : C2[e - k * k];
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  const int64_t i = t / k;
  const int c = (int)(t % k);
  float acc = 0.f;
  for (int a = 0; a < k; ++a) {
    acc = fmaf(W[i * ldw + a], cs[a * k + c], acc);
    acc = fmaf(Qt[i * ldq + a], cs[k * k + a * k + c], acc);
  }
  dW[i * ldw + c] = acc;
}

__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.3989422804014327f * expf(-0.5f * z * z);
}

// dZ1 = (dW W2^T) * GELU'(Z1) in tiles of 32 rows (a CTA takes tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...), thread j = hidden unit; written
// transposed in BF16 (dZ1t: kHidden x n_pad) and summed per CTA for db1
// (float-float partials)
constexpr int kDzRows = 32;
__global__ void __launch_bounds__(kHidden)
k_dz1(const float* __restrict__ dW, int ldw, const float* __restrict__ Z1, const float* __restrict__ W2, int k,
      int64_t n, int64_t n_pad, __nv_bfloat16* __restrict__ dZ1t, float2* __restrict__ db1_part) {
  __shared__ float dws[kDzRows][64];
  __shared__ __nv_bfloat16 tile[kHidden][kDzRows + 2];
  const int j = threadIdx.x;
  float w2[64];
#pragma unroll
  for (int c = 0; c < 64; ++c) w2[c] = c < k ? W2[j * k + c] : 0.f;
  float hi = 0.f, lo = 0.f;
  const int64_t ntiles = ceil_div(n_pad, (int64_t)kDzRows);
  for (int64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
    const int64_t r0 = tl * kDzRows;
    __syncthreads();
    for (int e = threadIdx.x; e < kDzRows * k; e += blockDim.x) {
      const int r = e / k, c = e % k;
      dws[r][c] = (r0 + r < n) ? dW[(r0 + r) * ldw + c] : 0.f;
    }
    __syncthreads();
    for (int r = 0; r < kDzRows; ++r) {
      float dz = 0.f;
      if (r0 + r < n) {
        float dh = 0.f;
#pragma unroll
        for (int c = 0; c < 64; ++c)
          if (c < k) dh = fmaf(dws[r][c], w2[c], dh);
        dz = dh * gelu_grad_f(Z1[(r0 + r) * kHidden + j]);
      }
      ffa(hi, lo, dz, 0.f);
      tile[j][r] = __float2bfloat16_rn(dz);
    }
    __syncthreads();
    // row jj of dZ1t: 32 consecutive nodes
    for (int e = threadIdx.x; e < kHidden * kDzRows; e += blockDim.x) {
      const int jj = e / kDzRows, r = e % kDzRows;
      if (r0 + r < n_pad) dZ1t[(int64_t)jj * n_pad + r0 + r] = tile[jj][r];
    }
  }
  db1_part[(int64_t)blockIdx.x * kHidden + j] = make_float2(hi, lo);
}

__global__ void k_reduce_f2(const float2* __restrict__ part, int nblk, int m, float* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m) return;
  float hi = 0.f, lo = 0.f;
  for (int b = 0; b < nblk; ++b) {
    const float2 v = part[(int64_t)b * m + t];
    ffa(hi, lo, v.x, v.y);
  }
  out[t] = hi + lo;
}

__global__ void k_d2f(const double* __restrict__ a, int64_t m, float* __restrict__ b) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m) b[t] = (float)a[t];
}

// Adam (bias-corrected): p -= lr * (m / c1) / (sqrt(v / c2) + eps), for
// m rows x cols of g with row stride ldg (p, m, v contiguous)
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, int64_t rows, int cols, int ldg,
                       float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2, float c1, float c2,
                       float eps) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * cols) return;
  const float gv = g[(t / cols) * ldg + (t % cols)];
  const float mv = b1 * m[t] + (1.f - b1) * gv;
  const float vv = b2 * v[t] + (1.f - b2) * gv * gv;
  m[t] = mv;
  v[t] = vv;
  p[t] -= lr * (mv / c1) / (sqrtf(vv / c2) + eps);
}

// W1^T in BF16 (kHidden x kp) from W1 (d_in x kHidden FP32), zero-padded
__global__ void k_w1t(const float* __restrict__ W1, int d_in, int kp, __nv_bfloat16* __restrict__ W1t) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)kHidden * kp) return;
  const int j = (int)(t / kp), c = (int)(t % kp);
  W1t[t] = __float2bfloat16_rn(c < d_in ? W1[(int64_t)c * kHidden + j] : 0.f);
}

}  // namespace

int warm_kp(int d) { return (int)round_up(2 * (int64_t)d, 64); }

// A (round_up(n, 128) x kp BF16, rows >= n zero) and, if At is not null, At
// (round_up(kp, 128) x n_pad BF16, n_pad = round_up(n, 64), zero outside
// kp x n) for a topology and its attributes
ancka_status warm_features(Workspace& ws, const Walk& w, const float* X, int d, __nv_bfloat16* A,
                           __nv_bfloat16* At, cudaStream_t s) {
  const int64_t n = w.n;
  const int ld = (int)round_up(d, 4);
  const int kp = warm_kp(d);
  ANCKA_CUDA(cudaMemsetAsync(A, 0, sizeof(__nv_bfloat16) * round_up(n, 128) * kp, s));
  if (At) ANCKA_CUDA(cudaMemsetAsync(At, 0, sizeof(__nv_bfloat16) * round_up(kp, 128) * round_up(n, 64), s));
  float *U, *PU;
  ANCKA_TRY(ws.alloc(&U, (size_t)n * ld));
  ANCKA_TRY(ws.alloc(&PU, (size_t)n * ld));
  k_unit_rows<<<(unsigned)ceil_div(n * 32, 256), 256, 0, s>>>(X, n, d, ld, U);
  ANCKA_LAUNCHED();
  ANCKA_TRY(apply_topology(ws, w, U, ld, PU, s));
  k_pack_features<<<(unsigned)ceil_div(n * kp, 256), 256, 0, s>>>(U, PU, n, d, ld, kp, A);
  ANCKA_LAUNCHED();
  if (At) {
    const int64_t n_pad = round_up(n, 64);
    dim3 grid((unsigned)ceil_div(n_pad, 32), (unsigned)ceil_div(kp, 32));
    k_transpose_bf16<<<grid, dim3(32, 8), 0, s>>>(A, n, kp, n_pad, At);
    ANCKA_LAUNCHED();
  }
  return ANCKA_OK;
}

// W = GELU(A W1 + b1) W2 + b2 (n x k, row stride ldw); Z1 and H (n x 256)
// are kept for a backward pass when the caller passes them
ancka_status warm_forward(Workspace& ws, const __nv_bfloat16* A, int64_t n, int kp, const __nv_bfloat16* W1t,
                          const float* b1, const float* W2, const float* b2, int k, float* W, int ldw, float* Z1,
                          float* H, int32_t* err, cudaStream_t s) {
  if (!Z1) ANCKA_TRY(ws.alloc(&Z1, (size_t)n * kHidden));
  if (!H) ANCKA_TRY(ws.alloc(&H, (size_t)n * kHidden));
  ANCKA_TRY(gemm_bias_gelu(A, n, kp, W1t, b1, Z1, H, kHidden, err, s));
  const size_t smem = (size_t)kHidden * k * sizeof(float);
  ANCKA_CUDA(cudaFuncSetAttribute(k_mlp_out, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_mlp_out<<<(unsigned)ceil_div(n * 32, 256), 256, smem, s>>>(H, n, W2, b2, k, W, ldw);
  ANCKA_LAUNCHED();
  return ANCKA_OK;
}

ancka_status warm_refresh_w1t(const float* W1, int d_in, int kp, __nv_bfloat16* W1t, cudaStream_t s) {
  k_w1t<<<(unsigned)ceil_div((int64_t)kHidden * kp, 256), 256, 0, s>>>(W1, d_in, kp, W1t);
  ANCKA_LAUNCHED();
  return ANCKA_OK;
}

// One training step on one graph: forward, loss, backward and Adam.  The
// model tensors (FP32) and their Adam moments are updated in place; *loss_dev
// receives the loss before the update.
ancka_status warm_train_step(Workspace& ws, const WarmStepArgs& a, cudaStream_t s) {
  const int64_t n = a.n;
  const int k = a.k;
  const int ldw = (int)round_up(k, 4);
  float *W, *Z1, *H, *dW, *C1, *C2, *dW2, *db2, *db1, *dW1;
  double *G, *M, *dW2d, *db2d;
  __nv_bfloat16* dZ1t;
  ANCKA_TRY(ws.alloc(&W, (size_t)n * ldw));
  ANCKA_TRY(ws.alloc(&Z1, (size_t)n * kHidden));
  ANCKA_TRY(ws.alloc(&H, (size_t)n * kHidden));
  ANCKA_TRY(ws.alloc(&dW, (size_t)n * ldw));
  ANCKA_TRY(ws.alloc(&C1, (size_t)k * k));
  ANCKA_TRY(ws.alloc(&C2, (size_t)k * k));
  ANCKA_TRY(ws.alloc(&G, (size_t)k * k));
  ANCKA_TRY(ws.alloc(&M, (size_t)k * k));
  ANCKA_TRY(ws.alloc(&dW2d, (size_t)kHidden * k));
  ANCKA_TRY(ws.alloc(&db2d, (size_t)k));
  ANCKA_TRY(ws.alloc(&dW2, (size_t)kHidden * k));
  ANCKA_TRY(ws.alloc(&db2, (size_t)k));
  ANCKA_TRY(ws.alloc(&db1, (size_t)kHidden));
  ANCKA_TRY(ws.alloc(&dW1, (size_t)round_up(a.kp, 128) * kHidden));
  const int64_t n_pad = round_up(n, 64);
  ANCKA_TRY(ws.alloc(&dZ1t, (size_t)kHidden * n_pad));
  // forward
  ANCKA_TRY(warm_forward(ws, a.A, n, a.kp, a.W1t, a.b1, a.W2, a.b2, k, W, ldw, Z1, H, a.err, s));
  // loss and dL/dW
  ANCKA_TRY(xty(ws, W, ldw, W, ldw, n, k, k, G, s));
  ANCKA_TRY(xty(ws, a.Qt, a.ldq, W, ldw, n, k, k, M, s));
  const size_t csm = (size_t)5 * k * k * sizeof(double);
  ANCKA_CUDA(cudaFuncSetAttribute(k_warm_coeffs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm));
  k_warm_coeffs<<<1, 128, csm, s>>>(G, M, k, (double)n, (double)a.lam, C1, C2, a.loss_dev, a.status);
  ANCKA_LAUNCHED();
  k_grad_w<<<(unsigned)ceil_div(n * k, 256), 256, (size_t)2 * k * k * sizeof(float), s>>>(W, ldw, a.Qt, a.ldq, n, k,
                                                                                           C1, C2, dW);
  ANCKA_LAUNCHED();
  // backward
  ANCKA_TRY(xty(ws, H, kHidden, dW, ldw, n, kHidden, k, dW2d, s));
  ANCKA_TRY(xty(ws, nullptr, 0, dW, ldw, n, 1, k, db2d, s));
  k_d2f<<<(unsigned)ceil_div((int64_t)kHidden * k, 256), 256, 0, s>>>(dW2d, (int64_t)kHidden * k, dW2);
  ANCKA_LAUNCHED();
  k_d2f<<<1, 64, 0, s>>>(db2d, k, db2);
  ANCKA_LAUNCHED();
  const int nb = (int)std::min<int64_t>(304, ceil_div(n_pad, (int64_t)kDzRows));
  float2* db1p;
  ANCKA_TRY(ws.alloc(&db1p, (size_t)nb * kHidden));
  k_dz1<<<nb, kHidden, 0, s>>>(dW, ldw, Z1, a.W2, k, n, n_pad, dZ1t, db1p);
  ANCKA_LAUNCHED();
  k_reduce_f2<<<1, kHidden, 0, s>>>(db1p, nb, kHidden, db1);
  ANCKA_LAUNCHED();
  ANCKA_TRY(gemm_at_b(ws, a.At, a.kp, n_pad, dZ1t, dW1, a.err, s));
  if (a.grads) {  // gradients out (tests)
    ANCKA_CUDA(cudaMemcpyAsync(a.grads->W1, dW1, sizeof(float) * a.d_in * kHidden, cudaMemcpyDeviceToDevice, s));
    ANCKA_CUDA(cudaMemcpyAsync(a.grads->b1, db1, sizeof(float) * kHidden, cudaMemcpyDeviceToDevice, s));
    ANCKA_CUDA(cudaMemcpyAsync(a.grads->W2, dW2, sizeof(float) * kHidden * k, cudaMemcpyDeviceToDevice, s));
    ANCKA_CUDA(cudaMemcpyAsync(a.grads->b2, db2, sizeof(float) * k, cudaMemcpyDeviceToDevice, s));
  }
  // Adam
  const double c1 = 1.0 - std::pow(0.9, (double)a.t), c2 = 1.0 - std::pow(0.999, (double)a.t);
  struct T {
    float* p;
    const float* g;
    int64_t rows;
    int cols;
    float* m;
    float* v;
  } ts[4] = {{a.W1, dW1, a.d_in, kHidden, a.mW1, a.vW1},
             {a.b1, db1, 1, kHidden, a.mb1, a.vb1},
             {a.W2, dW2, kHidden, k, a.mW2, a.vW2},
             {a.b2, db2, 1, k, a.mb2, a.vb2}};
  for (const T& q : ts) {
    k_adam<<<(unsigned)ceil_div(q.rows * q.cols, 256), 256, 0, s>>>(q.p, q.g, q.rows, q.cols, q.cols, q.m, q.v,
                                                                      a.lr, 0.9f, 0.999f, (float)c1, (float)c2, 1e-8f);
    ANCKA_LAUNCHED();
  }
  return warm_refresh_w1t(a.W1, a.d_in, a.kp, a.W1t, s);
}

}  // namespace ancka
