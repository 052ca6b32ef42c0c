// Plain FP32 (CUDA-core) candidate search for the cosine KNN of Section 3.1.
//
// Each CTA owns 128 query rows and sweeps every 128-row key block: a
// register-tiled SGEMM (8x8 outputs per thread, k-chunks of 8 double-buffered
// in shared memory) produces the 128x128 score tile u_i . u_j of the unit
// rows, the tile goes to shared memory, and thread r < 128 folds row r of it
// into its register-resident list of the kCandC best (score, index) pairs.
// Keys arrive in increasing index order and a score must beat the current
// worst strictly, so among equal scores the lower index is kept.
// n x n scores are never written to global memory.
#include "common.cuh"

namespace ancka {

namespace {

constexpr int kBM = 128, kBN = 128, kBK = 8, kThreads = 256;
constexpr int kSPad = kBN + 1;  // conflict-free row reads of the score tile

__global__ void __launch_bounds__(kThreads, 1)
k_knn_simt(const float* __restrict__ Xu, int64_t n, int64_t n_pad, int dp,
           float* __restrict__ cand_val, int32_t* __restrict__ cand_idx) {
  __shared__ __align__(16) float As[2][kBK][kBM];
  __shared__ __align__(16) float Bs[2][kBK][kBN];
  extern __shared__ float S[];  // kBM x kSPad

  const int tid = threadIdx.x;
  const int64_t ib = (int64_t)blockIdx.x * kBM;
  const int ty = tid >> 4, tx = tid & 15;
  const int lr = tid >> 1, lc = (tid & 1) * 4;  // loader: row, 4-wide column chunk
  const int64_t my_row = ib + tid;              // scanning threads: tid < 128

  constexpr int C = kCandC;
  float lv[C];
  int32_t li[C];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    lv[c] = -INFINITY;
    li[c] = -1;
  }
  float thr = -INFINITY;
  int mp = 0;

  const float* Arow = Xu + (ib + lr) * (int64_t)dp + lc;
  for (int64_t jb = 0; jb < n_pad; jb += kBN) {
    const float* Brow = Xu + (jb + lr) * (int64_t)dp + lc;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    float4 ra = *reinterpret_cast<const float4*>(Arow);
    float4 rb = *reinterpret_cast<const float4*>(Brow);
    As[0][lc + 0][lr] = ra.x;
    As[0][lc + 1][lr] = ra.y;
    As[0][lc + 2][lr] = ra.z;
    As[0][lc + 3][lr] = ra.w;
    Bs[0][lc + 0][lr] = rb.x;
    Bs[0][lc + 1][lr] = rb.y;
    Bs[0][lc + 2][lr] = rb.z;
    Bs[0][lc + 3][lr] = rb.w;
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < dp; k0 += kBK) {
      const bool more = k0 + kBK < dp;
      if (more) {
        ra = *reinterpret_cast<const float4*>(Arow + k0 + kBK);
        rb = *reinterpret_cast<const float4*>(Brow + k0 + kBK);
      }
#pragma unroll
      for (int kk = 0; kk < kBK; ++kk) {
        float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
        float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
        float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
        float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
        const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
      }
      if (more) {
        const int nb = buf ^ 1;
        As[nb][lc + 0][lr] = ra.x;
        As[nb][lc + 1][lr] = ra.y;
        As[nb][lc + 2][lr] = ra.z;
        As[nb][lc + 3][lr] = ra.w;
        Bs[nb][lc + 0][lr] = rb.x;
        Bs[nb][lc + 1][lr] = rb.y;
        Bs[nb][lc + 2][lr] = rb.z;
        Bs[nb][lc + 3][lr] = rb.w;
      }
      __syncthreads();
      buf ^= 1;
    }
    // score tile -> shared memory
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = (j < 4) ? tx * 4 + j : 64 + tx * 4 + (j - 4);
        S[r * kSPad + c] = acc[i][j];
      }
    }
    __syncthreads();
    if (tid < kBM && my_row < n) {
      const int64_t jend = (jb + kBN < n) ? jb + kBN : n;
      const float* srow = S + tid * kSPad;
      for (int64_t j = jb; j < jend; ++j) {
        const float s = srow[j - jb];
        if (s > thr && j != my_row) list_insert<C>(lv, li, thr, mp, s, (int32_t)j);
      }
    }
    // the next block's first smem writes (As/Bs) do not touch S; the S
    // writes come after that block's k-loop barriers.
  }
  if (tid < kBM && my_row < n) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      cand_val[my_row * kCandC + c] = lv[c];
      cand_idx[my_row * kCandC + c] = li[c];
    }
  }
}

}  // namespace

ancka_status knn_candidates_fp32(const PrepOut& pr, int64_t n, float* cand_val, int32_t* cand_idx,
                                 cudaStream_t s) {
  const size_t smem = (size_t)kBM * kSPad * sizeof(float);
  static bool configured[kMaxDevices] = {};
  if (!configured[device_slot()]) {
    ANCKA_CUDA(cudaFuncSetAttribute(k_knn_simt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured[device_slot()] = true;
  }
  dim3 grid((unsigned)(pr.n_pad / kBM));
  k_knn_simt<<<grid, kThreads, smem, s>>>(pr.xu32, n, pr.n_pad, pr.dp, cand_val, cand_idx);
  ANCKA_LAUNCHED();
  return ANCKA_OK;
}

}  // namespace ancka
