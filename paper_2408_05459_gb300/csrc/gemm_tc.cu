// tcgen05 BF16 GEMM C = A B^T for the warm-start MLP (both operands K-major,
// FP32 accumulation in TMEM).  One CTA computes a 128 x 256 tile of C:
//   warp 0     TMA producer: per stage a 128 x 64 block of A and a 256 x 64
//              block of B (128-byte swizzle) through a 4-deep mbarrier ring;
//   warp 1     MMA issuer: 256 TMEM columns, tcgen05.mma.cta_group::1.kind::f16
//              (M = 128, N = 256, K = 16), four per stage;
//   warps 2-9  epilogue: two per TMEM lane quarter, 128 columns each.
// The K range can be split over gridDim.z (each split writes its own FP32
// partial tile, summed afterwards in a fixed order).  Every wait is bounded;
// on expiry the kernel records an error code, drains its own copies / MMAs,
// frees TMEM and returns.
#include <algorithm>

#include "tc_common.cuh"

namespace ancka {

namespace {

constexpr int gM = 128, gN = 256, gK = 64;
constexpr int gEpiWarps = 8;
constexpr int gThreads = 64 + 32 * gEpiWarps;
constexpr int gABytes = gM * kTKB;  // 16 KB
constexpr int gBBytes = gN * kTKB;  // 32 KB
constexpr int gStages = 4;
constexpr uint32_t gTmemCols = 256;
// kind::f16, D = F32, A = B = BF16, K-major, N >> 3 at 17, M >> 4 at 24
constexpr uint32_t gIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(gN >> 3) << 17) |
                            ((uint32_t)(gM >> 4) << 24);

struct __align__(8) GBars {
  uint64_t full[gStages];
  uint64_t empty[gStages];
  uint64_t done;
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
};

__device__ __forceinline__ void umma_bf16_g(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          tmem_d),
      "l"(da), "l"(db), "r"(gIdesc), "r"(accum)
      : "memory");
}

enum { kEpiBiasGelu = 0, kEpiPartial = 1 };

struct GemmOut {
  int64_t m_real;     // rows of C that exist
  const float* bias;  // bias-GELU: gN
  float* Z;           // bias-GELU: pre-activation A B^T + bias (ld = ldz)
  float* H;           // bias-GELU: GELU(Z) (ld = ldz)
  int ldz;
  float* P;           // partial: gridDim.z x m_pad x gN
  int64_t m_pad;
};

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }

template <int kEpi>
__global__ void __launch_bounds__(gThreads, 1)
k_gemm_tn(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int k_stages,
          int stages_per_split, GemmOut o, int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = sA + gStages * gABytes;
  GBars* bars = reinterpret_cast<GBars*>(sB + gStages * gBBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = (int64_t)blockIdx.x * gM;
  const int ks0 = (int)blockIdx.z * stages_per_split;
  const int nks = max(0, min(k_stages, ks0 + stages_per_split) - ks0);
  volatile int* abort = &bars->abort;

  if (threadIdx.x == 0) {
    for (int s = 0; s < gStages; ++s) {
      mbar_init(&bars->full[s], 1);
      mbar_init(&bars->empty[s], 1);
    }
    mbar_init(&bars->done, 1);
    mbar_init(&bars->drain, 1);
    bars->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&bars->tmem_base)),
                 "r"(gTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      bool pending[gStages];
      uint32_t pend_par[gStages];
      for (int s = 0; s < gStages; ++s) pending[s] = false;
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int ks = 0; ks < nks; ++ks) {
        if (!mbar_wait(&bars->empty[stage], phase ^ 1, abort, err, 11)) {
          ok = false;
          break;
        }
        mbar_expect_tx(&bars->full[stage], (uint32_t)(gABytes + gBBytes));
        tma_load_2d(smem_u32(sA + stage * gABytes), &tmA, (ks0 + ks) * gK, (int)m0, &bars->full[stage]);
        tma_load_2d(smem_u32(sB + stage * gBBytes), &tmB, (ks0 + ks) * gK, 0, &bars->full[stage]);
        pending[stage] = true;
        pend_par[stage] = phase;
        if (++stage == gStages) {
          stage = 0;
          phase ^= 1;
        }
      }
      if (!ok)  // drain this warp's copies still in flight (bounded)
        for (int s = 0; s < gStages; ++s)
          if (pending[s]) mbar_wait(&bars->full[s], pend_par[s], nullptr, nullptr, 0);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true, issued = false;
      for (int ks = 0; ks < nks; ++ks) {
        if (!mbar_wait(&bars->full[stage], phase, abort, err, 12)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a0 = smem_u32(sA + stage * gABytes);
        const uint32_t b0 = smem_u32(sB + stage * gBBytes);
#pragma unroll
        for (int kk = 0; kk < gK / 16; ++kk)
          umma_bf16_g(tmem, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), (ks | kk) != 0 ? 1u : 0u);
        issued = true;
        umma_commit(&bars->empty[stage]);
        if (++stage == gStages) {
          stage = 0;
          phase ^= 1;
        }
      }
      if (ok && issued) umma_commit(&bars->done);
      if (!ok && issued) {  // wait for this thread's MMAs before TMEM is freed (bounded)
        umma_commit(&bars->drain);
        mbar_wait(&bars->drain, 0, nullptr, nullptr, 0);
      }
    }
  } else {
    const int q = warp & 3;          // TMEM lane quarter this warp may access
    const int h = (warp - 2) >> 2;   // column half
    const int r = q * 32 + lane;
    const int64_t row = m0 + r;
    bool ok = true;
    if (nks > 0) {
      ok = mbar_wait(&bars->done, 0, abort, err, 13);
      ok = __all_sync(0xffffffffu, ok);
      tc_fence_after();
    }
    if (ok) {
      const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * 128);
#pragma unroll 1
      for (int c = 0; c < 4; ++c) {
        uint32_t rv[32];
        if (nks > 0) {
          tmem_ld32_issue(tb + (uint32_t)(c * 32), rv);
          tmem_wait();
          pin(rv);
        } else {
#pragma unroll
          for (int e = 0; e < 32; ++e) rv[e] = 0u;  // empty K range: C = 0
        }
        const int col0 = h * 128 + c * 32;
        if constexpr (kEpi == kEpiBiasGelu) {
          if (row < o.m_real) {
            float* zr = o.Z + row * o.ldz + col0;
            float* hr = o.H + row * o.ldz + col0;
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              const float z = __uint_as_float(rv[e]) + o.bias[col0 + e];
              zr[e] = z;
              hr[e] = gelu_f(z);
            }
          }
        } else {
          float* pr = o.P + ((int64_t)blockIdx.z * o.m_pad + row) * gN + col0;
#pragma unroll
          for (int e = 0; e < 32; ++e) pr[e] = __uint_as_float(rv[e]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(gTmemCols) : "memory");
  }
}

// C[i, j] = sum over splits of P[s, i, j] in split order (i < m_real)
__global__ void k_sum_splits(const float* __restrict__ P, int splits, int64_t m_pad, int64_t m_real,
                             float* __restrict__ C) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m_real * gN) return;
  float acc = 0.f;
  for (int s = 0; s < splits; ++s) acc += P[(int64_t)s * m_pad * gN + t];
  C[t] = acc;
}

size_t gemm_smem() { return 1024 + (size_t)gStages * (gABytes + gBBytes) + sizeof(GBars); }

}  // namespace

// Z = A W^T + bias and H = GELU(Z) (m x 256, FP32, ld ldz) for A (m x k_pad
// BF16, K-major, k_pad a multiple of 64, allocated with round_up(m, 128)
// rows, the extra rows zero) and Wt (256 x k_pad BF16).
ancka_status gemm_bias_gelu(const __nv_bfloat16* A, int64_t m, int64_t k_pad, const __nv_bfloat16* Wt,
                            const float* bias, float* Z, float* H, int ldz, int32_t* err, cudaStream_t s) {
  if (k_pad % gK != 0 || k_pad < gK) {
    set_error("internal: GEMM K must be a positive multiple of %d", gK);
    return ANCKA_ERR_INTERNAL;
  }
  CUtensorMap ta, tb;
  ANCKA_TRY(make_map(&ta, A, k_pad, round_up(m, (int64_t)gM), gM, 2));
  ANCKA_TRY(make_map(&tb, Wt, k_pad, gN, gN, 2));
  const size_t smem = gemm_smem();
  ANCKA_CUDA(cudaFuncSetAttribute(k_gemm_tn<kEpiBiasGelu>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  GemmOut o{};
  o.m_real = m;
  o.bias = bias;
  o.Z = Z;
  o.H = H;
  o.ldz = ldz;
  const int ks = (int)(k_pad / gK);
  k_gemm_tn<kEpiBiasGelu><<<dim3((unsigned)ceil_div(m, gM), 1, 1), gThreads, smem, s>>>(ta, tb, ks, ks, o, err);
  ANCKA_LAUNCHED();
  return ANCKA_OK;
}

// C = At B (m x 256, FP32) for At (m x k_pad BF16, K-major: the transpose of
// the k_pad x m left factor, allocated with round_up(m, 128) rows, the extra
// rows zero) and Bt (256 x k_pad BF16): the K range (k_pad,
// a multiple of 64, typically the node count) is split over about two waves
// of CTAs and the partial tiles summed in split order.
ancka_status gemm_at_b(Workspace& ws, const __nv_bfloat16* At, int64_t m, int64_t k_pad, const __nv_bfloat16* Bt,
                       float* C, int32_t* err, cudaStream_t s) {
  if (k_pad % gK != 0 || k_pad < gK) {
    set_error("internal: GEMM K must be a positive multiple of %d", gK);
    return ANCKA_ERR_INTERNAL;
  }
  CUtensorMap ta, tb;
  ANCKA_TRY(make_map(&ta, At, k_pad, round_up(m, (int64_t)gM), gM, 2));
  ANCKA_TRY(make_map(&tb, Bt, k_pad, gN, gN, 2));
  const size_t smem = gemm_smem();
  ANCKA_CUDA(cudaFuncSetAttribute(k_gemm_tn<kEpiPartial>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, sms = 152;
  ANCKA_CUDA(cudaGetDevice(&dev));
  ANCKA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t mt = ceil_div(m, gM);
  const int ks = (int)(k_pad / gK);
  int splits = (int)std::max<int64_t>(1, std::min<int64_t>(ks, (2 * sms) / std::max<int64_t>(1, mt)));
  const int sps = (int)ceil_div(ks, splits);
  splits = (int)ceil_div(ks, sps);
  GemmOut o{};
  o.m_pad = mt * gM;
  ANCKA_TRY(ws.alloc(&o.P, (size_t)splits * o.m_pad * gN));
  k_gemm_tn<kEpiPartial><<<dim3((unsigned)mt, 1, (unsigned)splits), gThreads, smem, s>>>(ta, tb, ks, sps, o, err);
  ANCKA_LAUNCHED();
  k_sum_splits<<<(unsigned)ceil_div(m * gN, 256), 256, 0, s>>>(o.P, splits, o.m_pad, m, C);
  ANCKA_LAUNCHED();
  return ANCKA_OK;
}

}  // namespace ancka
