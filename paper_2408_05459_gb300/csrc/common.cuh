// Shared device helpers and internal host interfaces of the ANCKA library.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../../include/ancka.h"

namespace ancka {

// ---------------------------------------------------------------------------
// error plumbing (host)
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);
ancka_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define ANCKA_CUDA(x)                                                        \
  do {                                                                       \
    cudaError_t e_ = (x);                                                    \
    if (e_ != cudaSuccess) return ::ancka::cuda_fail(e_, #x, __FILE__, __LINE__); \
  } while (0)

void count_launch();
// timing events for the diagnostics (ancka_info): a per-thread pool, so an
// instrumented call creates no events once the pool is warm
cudaEvent_t pooled_event();
void release_event(cudaEvent_t e);
// the current device's ordinal, clamped to [0, kMaxDevices) (the per-device
// caches: streams, pooled events, kernel attributes)
constexpr int kMaxDevices = 64;
int device_slot();
#define ANCKA_LAUNCHED()            \
  do {                              \
    ::ancka::count_launch();        \
    ANCKA_CUDA(cudaGetLastError()); \
  } while (0)

#define ANCKA_TRY(x)                               \
  do {                                             \
    ancka_status s_ = (x);                         \
    if (s_ != ANCKA_OK) return s_;                 \
  } while (0)

// Stream-ordered workspace: every buffer is allocated with cudaMallocAsync on
// the call's stream and released (stream-ordered) when the object dies.
class Workspace {
 public:
  explicit Workspace(cudaStream_t s) : s_(s) {}
  ~Workspace() { release(); }
  template <class T>
  ancka_status alloc(T** p, size_t count) {
    void* q = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(&q, bytes, s_);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMallocAsync(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
      return ANCKA_ERR_OOM;
    }
    ptrs_.push_back(q);
    *p = static_cast<T*>(q);
    return ANCKA_OK;
  }
  template <class T>
  ancka_status zeros(T** p, size_t count) {
    ANCKA_TRY(alloc(p, count));
    ANCKA_CUDA(cudaMemsetAsync(*p, 0, (count ? count : 1) * sizeof(T), s_));
    return ANCKA_OK;
  }
  void release() {
    for (void* q : ptrs_) cudaFreeAsync(q, s_);
    ptrs_.clear();
  }
  cudaStream_t stream() const { return s_; }

 private:
  cudaStream_t s_;
  std::vector<void*> ptrs_;
};

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// ---------------------------------------------------------------------------
// error-free transformations (Ogita, Rump, Oishi 2005, "Accurate sum and dot
// product"): the _rn intrinsics are never contracted into FMAs, which keeps
// TwoSum / TwoProd exact.
// ---------------------------------------------------------------------------
struct DW {  // unevaluated sum hi + lo
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// (hi, lo) += (bh, bl): float-float addition (TwoSum, then renormalise)
__device__ __forceinline__ void ff_add(float& hi, float& lo, float bh, float bl) {
  float s, e;
  two_sum(hi, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(lo, bl));
  hi = __fadd_rn(s, e);
  lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// Dot2 accumulation step: (s, c) += x * y
__device__ __forceinline__ void dot2_step(float& s, float& c, float x, float y) {
  float p = __fmul_rn(x, y);
  float ep = __fmaf_rn(x, y, -p);
  float t, es;
  two_sum(s, p, t, es);
  s = t;
  c = __fadd_rn(c, __fadd_rn(es, ep));
}

// combine two Dot2 partials (s1,c1) + (s2,c2)
__device__ __forceinline__ void dot2_merge(float& s, float& c, float s2, float c2) {
  float t, e;
  two_sum(s, s2, t, e);
  s = t;
  c = __fadd_rn(__fadd_rn(c, c2), e);
}

// fixed-order butterfly reduction of a Dot2 partial across a full warp
__device__ __forceinline__ void dot2_warp_reduce(float& s, float& c) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    float s2 = __shfl_xor_sync(0xffffffffu, s, off);
    float c2 = __shfl_xor_sync(0xffffffffu, c, off);
    // order the operands by lane so both partners compute the same value
    int lane = threadIdx.x & 31;
    if (lane & off) {
      float ts = s, tc = c;
      s = s2; c = c2; s2 = ts; c2 = tc;
    }
    dot2_merge(s, c, s2, c2);
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Insert (s, j) into an unsorted register list of C scores whose minimum is
// thr at slot mp (caller checked s > thr); recompute the minimum.  Fully
// unrolled so the list stays in registers.
template <int C>
__device__ __forceinline__ void list_insert(float (&lv)[C], int32_t (&li)[C], float& thr, int& mp, float s,
                                            int32_t j) {
#pragma unroll
  for (int c = 0; c < C; ++c)
    if (c == mp) {
      lv[c] = s;
      li[c] = j;
    }
  thr = lv[0];
  mp = 0;
#pragma unroll
  for (int c = 1; c < C; ++c)
    if (lv[c] < thr) {
      thr = lv[c];
      mp = c;
    }
}

// ---------------------------------------------------------------------------
// internal host interfaces (one translation unit each)
// ---------------------------------------------------------------------------

// prep.cu: unit rows, low-precision copy, per-row quantisation error
struct PrepOut {
  int32_t d;           // feature dimension of X (unpadded)
  int32_t dp;          // padded feature dimension of the copy
  int64_t n_pad;       // padded row count of the copy
  float* xu32;         // FP32 unit rows (n_pad x dp) or null
  __nv_bfloat16* xb;   // BF16 unit rows (n_pad x dp) or null
  float* err;          // n: upper bound of || copy_i - x_i/||x_i|| ||_2
  double* nrm2;        // n: ||x_i||^2 (compensated)
  int32_t* zero_row;   // n: 1 if x_i == 0
  float* err_max;      // 1: max_i err_i
  // FP8 mode (besides the BF16 copy above): E4M3 copy of S * unit rows, one
  // power-of-two scale S for all rows, so q_i . q_j / S^2 approximates the
  // cosine; err8 bounds || q_i / S - x_i/||x_i|| ||_2
  int32_t dp8;            // padded feature dimension (multiple of 128)
  uint8_t* x8;            // n_pad x dp8 E4M3 codes, or null
  float* err8;            // n
  float* err8_max;        // 1
  float* inv_s2;          // 1: 1 / S^2
};
ancka_status prep_rows(Workspace& ws, const float* X, int64_t n, int32_t d, int prec, PrepOut* out,
                       cudaStream_t s);

// knn_simt.cu / knn_tc.cu: candidate top-C lists from the low-precision scores
constexpr int kCandC = 32;  // candidates kept per row
ancka_status knn_candidates_fp32(const PrepOut& pr, int64_t n, float* cand_val, int32_t* cand_idx,
                                 cudaStream_t s);
ancka_status knn_candidates_bf16(Workspace& ws, const PrepOut& pr, int64_t n, float* cand_val, int32_t* cand_idx,
                                 int32_t* err, cudaStream_t s);
// FP8 (E4M3) list pass: scores written in cosine units (times 1/S^2)
ancka_status knn_candidates_fp8(Workspace& ws, const PrepOut& pr, int64_t n, float* cand_val, int32_t* cand_idx,
                                int32_t* err, cudaStream_t s);
int knn_tc_max_dp_fp8();
// ivf.cu: approximate KNN by inverted lists (spherical k-means cells, nprobe
// nearest cells per row, exact cosines of the candidates found there)
struct IvfStats {
  int64_t key_tiles = 0;   // (query block, key tile) pairs multiplied
  int64_t full_tiles = 0;  // the same for the exact sweep
};
ancka_status knn_ivf(Workspace& ws, const float* X, int64_t n, int32_t d, int32_t K, int32_t nlist, int32_t nprobe,
                     int32_t iters, uint64_t seed, int32_t* out_idx, float* out_sim, int32_t** zero_row,
                     IvfStats* stats, cudaStream_t s);
int ivf_max_tiles();
// sort.cu: keys sorted ascending on bits [0, end_bit) (in is left as it was;
// in != out); out[i] = in[0] + ... + in[i-1] for i < count; the distinct
// values of sorted keys, their count written to *count_dev
ancka_status radix_sort_u64(Workspace& ws, const uint64_t* in, uint64_t* out, int64_t count, int end_bit,
                            cudaStream_t s);
ancka_status exclusive_scan(Workspace& ws, const int64_t* in, int64_t* out, int64_t count, cudaStream_t s);
ancka_status unique_u64(Workspace& ws, const uint64_t* in, uint64_t* out, int64_t* count_dev, int64_t count,
                        cudaStream_t s);
// Two 16-entry candidate lists per query row of the BF16 matrix a (rows
// 0..n_rows-1, or the rows listed in `rows`, written at their own row index)
// against the keys (n_keys rows of keys, keys_pad rows addressable, zero
// padded); optional key-tile lists per 128-row query block (blk_ptr /
// blk_tiles, blk_work = blk_ptr[blocks]); no_self: the keys are another set.
ancka_status knn_lists_bf16(Workspace& ws, const __nv_bfloat16* a, int64_t a_rows_total, const int32_t* rows,
                           int64_t n_rows, const __nv_bfloat16* keys, int64_t n_keys, int64_t keys_pad, int dp, int d,
                           const int64_t* blk_ptr, const int32_t* blk_tiles, int64_t blk_work, bool no_self,
                           float* cand_val, int32_t* cand_idx, int32_t* err, cudaStream_t s);
// BF16 list pass for the n_a rows listed in rows; lists written at their global rows
ancka_status knn_list_gathered_bf16(Workspace& ws, const PrepOut& pr, int64_t n, const int32_t* rows, int64_t n_a,
                                    float* cand_val, int32_t* cand_idx, int32_t* err, cudaStream_t s);
bool knn_tc_available();
int knn_tc_max_dp();
// BF16 lists of n >= n_min rows come from the symmetric contraction
void knn_set_symmetric_min_rows(int64_t n_min);
// collect pass: for the n_a query rows listed in `rows`, every key j != row
// with a BF16 score >= thr[r] is appended to buf[r * cap ..] (cnt[r] counts,
// also past cap)
ancka_status knn_collect_bf16(Workspace& ws, const PrepOut& pr, int64_t n, const int32_t* rows, int64_t n_a,
                              const float* thr, int32_t* cnt, int32_t* buf, int cap, int32_t* err, cudaStream_t s);

// rerank.cu: certified exact re-rank + exhaustive fallback
// list_prec: precision of the candidate lists (FP32, BF16 or FP8; acc_coef
// is its accumulation bound); lists: 1 (one 32-list per row) or 2 (two
// 16-lists).  FP8: rows the FP8 lists cannot certify get BF16 lists
// (acc_bf16) and a second certificate.  collect_prec == ANCKA_PREC_BF16 sends
// rows still uncertified through the tensor-core collect pass.  list_err
// (device, may be null): the error flag of the pass that wrote the lists; the
// re-rank skips its work when it is set, and the call reports it with its
// first host read (ANCKA_ERR_TIMEOUT), so the list pass needs no sync of its own.
ancka_status knn_rerank(Workspace& ws, const float* X, int64_t n, int32_t d, int32_t K,
                        const PrepOut& pr, int list_prec, float acc_coef, float acc_bf16, float* cand_val,
                        int32_t* cand_idx, int lists, int collect_prec, const int32_t* list_err, int32_t* out_idx,
                        float* out_sim, int64_t* n_candidates, int64_t* n_fallback, int64_t* n_exhaustive,
                        bool want_counts, cudaStream_t s);

// graph.cu: walk structures
struct Csr {
  int64_t nrows = 0, nnz = 0;
  int64_t* ptr = nullptr;
  int32_t* col = nullptr;
  float* val = nullptr;    // P_N (or KNN) values, may be null
  float* valT = nullptr;   // P_N^T values on the same pattern (graph/multiplex)
};
struct Walk {
  int kind = 0;
  int64_t n = 0, m = 0;
  Csr topo;         // graph/multiplex: merged layers; hypergraph: node -> hyperedges (H^T)
  Csr edges;        // hypergraph: hyperedge -> nodes (H)
  Csr knn;          // KNN part with values beta_i A_K[i,j] / D_K[i]
  float* rs_topo = nullptr;     // n: (1 - beta_i) [/ delta_i for hypergraphs and one-layer graphs]
  float* inv_deg = nullptr;     // hypergraph, one-layer graph: n, 1/delta_v (0 if delta = 0)
  bool row_uniform = false;     // one-layer graph: P_N = D^-1 A, so topo.val / valT are not
                                // stored (row scale inv_deg[i], column scale inv_deg[j])
  float* inv_size = nullptr;    // hypergraph: m, 1/|e|
  int32_t* degree = nullptr;    // n: delta(v) used for V_c
  float* beta = nullptr;        // n: beta_i
  const int32_t* names = nullptr;  // n: the caller's index of each row when the nodes are renamed, else null
};
ancka_status build_topology(Workspace& ws, const ancka_topology& t, Walk* w, cudaStream_t s);
ancka_status build_knn_part(Workspace& ws, int64_t n, int32_t K, const int32_t* idx, const float* sim,
                            const int32_t* zero_row, float beta, Walk* w, cudaStream_t s);

// iter.cu: the orthogonal iteration and its helpers
struct IterCfg {
  int32_t k, T, gamma, T_i, tau, disc_max_iter;
  float alpha;
  int32_t early_stop;  // Eq. tcond-1 / tcond-2 checks (paper mode)
  float eps_Q;         // Eq. tcond-1 threshold
  int32_t node_order = 0;  // 0: degree order when the block exceeds kDegreeOrderMinBytes, 1: as given, 2: degree order
};
// graphs whose n x (k+1) FP32 block is larger than this are iterated with the
// nodes renamed by descending degree (the gathers of the walk products then
// hit L2 more often); smaller blocks stay in L2 as they are
constexpr double kDegreeOrderMinBytes = 64.0 * 1024 * 1024;
struct IterTrace {
  double* phi_dev;         // device [ANCKA_MAX_TRACE]
  int32_t* disc_iters_dev; // device [ANCKA_MAX_TRACE]
  int32_t* taken_dev;      // device [ANCKA_MAX_TRACE]
  int32_t* flags_dev;      // device [1]
  double* phi_best_dev;    // device [1]
  int n_phi;
  int iters_run;           // orthogonal iterations executed
  int warm_used;           // 1 if the learned warm start replaced InitBCM's
  std::vector<cudaEvent_t>* events;  // (phase, start, stop) triples
  std::vector<int>* phases;
};
// InitBCM's Y^(0) from the topology part of the walk alone (no attributes, no
// KNN part): may run on its own stream while the KNN is computed
ancka_status initbcm_labels(Workspace& ws, const Walk& w, const IterCfg& cfg, int32_t* y0, cudaStream_t s);
// warm_W: n x k block predicted by the warm-start MLP (row stride ldw), or null
ancka_status run_ancka(Workspace& ws, const Walk& w, const IterCfg& c, const int32_t* init_labels,
                       const float* warm_W, int ldw, int32_t* labels_out, float* Q_out, int32_t* init_out,
                       IterTrace* tr, cudaStream_t s);
// out = P_N U (topology walk only) for an n x ld block (ld a multiple of 4)
ancka_status apply_topology(Workspace& ws, const Walk& w, const float* U, int ld, float* out, cudaStream_t s);

// warm.cu: learned warm start (MLP d_in -> 256 -> k)
int warm_kp(int d);  // padded feature width of [U | P_N U]: round_up(2d, 64)
ancka_status warm_features(Workspace& ws, const Walk& w, const float* X, int d, __nv_bfloat16* A,
                           __nv_bfloat16* At, cudaStream_t s);
ancka_status warm_forward(Workspace& ws, const __nv_bfloat16* A, int64_t n, int kp, const __nv_bfloat16* W1t,
                          const float* b1, const float* W2, const float* b2, int k, float* W, int ldw, float* Z1,
                          float* H, int32_t* err, cudaStream_t s);
ancka_status warm_refresh_w1t(const float* W1, int d_in, int kp, __nv_bfloat16* W1t, cudaStream_t s);
struct WarmGrads {
  float* W1;  // d_in x 256
  float* b1;  // 256
  float* W2;  // 256 x k
  float* b2;  // k
};
struct WarmStepArgs {
  int64_t n;
  int k, d_in, kp;
  const __nv_bfloat16* A;   // n x kp
  const __nv_bfloat16* At;  // kp x round_up(n, 64)
  const float* Qt;          // n x k target (row stride ldq)
  int ldq;
  float *W1, *b1, *W2, *b2;  // FP32 master weights (updated)
  __nv_bfloat16* W1t;        // 256 x kp BF16 copy of W1^T (refreshed)
  float *mW1, *vW1, *mb1, *vb1, *mW2, *vW2, *mb2, *vb2;  // Adam moments
  float lr, lam;
  int t;                     // Adam step (1-based)
  double* loss_dev;          // loss before the update
  int32_t* status;           // singular W^T W
  int32_t* err;              // tensor-core wait expired
  const WarmGrads* grads;    // optional: raw gradients out
};
ancka_status warm_train_step(Workspace& ws, const WarmStepArgs& a, cudaStream_t s);

// gemm_tc.cu: tcgen05 BF16 GEMMs of the warm-start MLP (N = 256 columns)
ancka_status gemm_bias_gelu(const __nv_bfloat16* A, int64_t m, int64_t k_pad, const __nv_bfloat16* Wt,
                            const float* bias, float* Z, float* H, int ldz, int32_t* err, cudaStream_t s);
ancka_status gemm_at_b(Workspace& ws, const __nv_bfloat16* At, int64_t m, int64_t k_pad, const __nv_bfloat16* Bt,
                       float* C, int32_t* err, cudaStream_t s);
ancka_status discretize(Workspace& ws, const float* Qk, int64_t n, int32_t k, int32_t ldq,
                        int32_t max_iter, int32_t* labels, int32_t* iters_dev, int32_t* flags_dev,
                        int32_t** err_dev, cudaStream_t s);
size_t discretize_scratch_bytes(int64_t n, int32_t k);
ancka_status polar_factor(const float* M, int32_t k, float* R, int32_t* method_dev, cudaStream_t s);
ancka_status discretize_scratch(void* scratch, size_t bytes, const float* Qk, int64_t n, int32_t k, int32_t ldq,
                                int32_t max_iter, int32_t* labels, int32_t** iters_dev, int32_t** err_dev,
                                cudaStream_t s);

}  // namespace ancka
