// C ABI of the ANCKA hot path: validation, workspace, phase sequencing.
#include <atomic>
#include <cstdarg>
#include <cstring>
#include <mutex>

#include <cuda_fp8.h>

#include <cmath>
#include <vector>

#include <functional>

#include "common.cuh"

namespace ancka {

namespace {
thread_local char g_err[512] = "";
std::atomic<int64_t> g_launches{0};
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int device_slot() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    dev = 0;
  }
  return dev < 0 ? 0 : (dev < kMaxDevices ? dev : kMaxDevices - 1);
}

namespace {
// events belong to the device they were created on: one pool per device
struct EventPool {
  std::vector<cudaEvent_t> free[kMaxDevices];
  ~EventPool() {
    for (auto& v : free)
      for (cudaEvent_t e : v) cudaEventDestroy(e);
  }
};
thread_local EventPool g_event_pool;
}  // namespace

cudaEvent_t pooled_event() {
  auto& v = g_event_pool.free[device_slot()];
  if (!v.empty()) {
    cudaEvent_t e = v.back();
    v.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// the event goes back to the pool of the current device, which is the
// device it was taken on (a call does not switch devices)
void release_event(cudaEvent_t e) {
  if (e) g_event_pool.free[device_slot()].push_back(e);
}

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

ancka_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  return e == cudaErrorMemoryAllocation ? ANCKA_ERR_OOM : ANCKA_ERR_CUDA;
}

namespace {

#define ANCKA_REQUIRE(cond, ...)            \
  do {                                      \
    if (!(cond)) {                          \
      ::ancka::set_error(__VA_ARGS__);      \
      return ANCKA_ERR_INVALID_ARG;         \
    }                                       \
  } while (0)

ancka_status device_check() {
  // discard a non-sticky error left by an unrelated earlier runtime call, so
  // that the launch checks of this call only see this call's failures
  cudaGetLastError();
  int dev = 0;
  ANCKA_CUDA(cudaGetDevice(&dev));
  static std::mutex mu;
  static int checked[64] = {0};  // 0 unknown, 1 ok, 2 bad
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 64 && checked[dev] == 0) {
    int major = 0, minor = 0;
    ANCKA_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
    ANCKA_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
    checked[dev] = (major == 10 && minor == 3) ? 1 : 2;
    if (checked[dev] == 1) {
      // keep freed workspace in the stream-ordered pool between calls
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
      }
    }
  }
  if (dev >= 64 || checked[dev] != 1) {
    set_error("device %d is not a compute capability 10.3 (GB300) device", dev);
    return ANCKA_ERR_UNSUPPORTED;
  }
  return ANCKA_OK;
}

struct Timer {
  std::vector<cudaEvent_t> ev;
  std::vector<int> ph;
};

struct Phase {
  Timer* t;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  int phase;
  Phase(Timer* tt, cudaStream_t st, int p) : t(tt), s(st), phase(p) {
    if (t) {
      a = pooled_event();
      cudaEventRecord(a, s);
    }
  }
  ~Phase() {
    if (t) {
      cudaEvent_t b = pooled_event();
      cudaEventRecord(b, s);
      t->ev.push_back(a);
      t->ev.push_back(b);
      t->ph.push_back(phase);
    }
  }
};

void fill_times(Timer& t, ancka_info* info) {
  float acc[8] = {0};
  for (size_t q = 0; q < t.ph.size(); ++q) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.ev[2 * q], t.ev[2 * q + 1]) == cudaSuccess && t.ph[q] < 8) acc[t.ph[q]] += ms;
  }
  for (cudaEvent_t e : t.ev) release_event(e);
  t.ev.clear();
  cudaGetLastError();
  if (info) {
    info->ms_knn = acc[0];
    info->ms_build = acc[1];
    info->ms_init = acc[2];
    info->ms_iter = acc[3];
    info->ms_disc = acc[4];
    info->ms_mhc = acc[5];
    info->ms_spmm = acc[6];
  }
}

__global__ void k_zero_rows(const float* __restrict__ X, int64_t n, int d, int32_t* __restrict__ z) {
  const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  bool any = false;
  for (int c = lane; c < d; c += 32) any |= X[row * d + c] != 0.f;
  any = __any_sync(0xffffffffu, any);
  if (lane == 0) z[row] = any ? 0 : 1;
}

__global__ void k_check_knn(const int32_t* __restrict__ idx, int64_t n, int K, int32_t* __restrict__ bad) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * K) return;
  const int32_t j = idx[q];
  if (j < 0 || j >= n || j == (int32_t)(q / K)) atomicExch(bad, 1);
}

__global__ void k_check_labels(const int32_t* __restrict__ y, int64_t n, int k, int32_t* __restrict__ bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && (y[i] < 0 || y[i] >= k)) atomicExch(bad, 1);
}

ancka_status read_flag(const int32_t* dev, cudaStream_t s, int32_t* host) {
  ANCKA_CUDA(cudaMemcpyAsync(host, dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  ANCKA_CUDA(cudaStreamSynchronize(s));
  return ANCKA_OK;
}

ancka_status validate_knn_args(const float* X, int64_t n, int32_t d, int32_t K, int32_t prec) {
  ANCKA_REQUIRE(X != nullptr, "X is NULL");
  ANCKA_REQUIRE(n >= 2 && n < (int64_t(1) << 31) - 1, "n = %lld out of range [2, 2^31-1)", (long long)n);
  ANCKA_REQUIRE(d >= 1 && d <= 4096, "d = %d out of range [1, 4096]", d);
  ANCKA_REQUIRE(K >= 1 && K <= 64 && K < n, "K = %d must satisfy 1 <= K <= 64 and K < n", K);
  ANCKA_REQUIRE(prec == ANCKA_PREC_FP32 || prec == ANCKA_PREC_BF16 || prec == ANCKA_PREC_FP8,
                "unknown precision %d", prec);
  const bool tc = prec == ANCKA_PREC_BF16 || prec == ANCKA_PREC_FP8;
  if (tc && !knn_tc_available()) {
    set_error("tensor-core contraction is not available in this build");
    return ANCKA_ERR_UNSUPPORTED;
  }
  // FP8 keeps a BF16 copy for the rows its certificate leaves open
  if (tc && K <= kCandC / 2 - 4 && round_up(d, 64) > knn_tc_max_dp()) {
    set_error("tensor-core contraction keeps the query block in shared memory: d must be <= %d", knn_tc_max_dp());
    return ANCKA_ERR_UNSUPPORTED;
  }
  return ANCKA_OK;
}

int max_candidate_K(int prec) { return prec == ANCKA_PREC_FP32 ? kCandC / 2 : kCandC / 2 - 4; }

// accumulation bound of the tensor-core contraction: a few units in the last
// place of FP32 per MMA step (16 BF16 or 32 FP8 products), checked against
// exact products of the quantised rows in the tests
float tc_acc_bound(int dp, int k_per_mma, int ulp_log2) {
  return (float)((dp / k_per_mma + 2) * std::ldexp(1.0, ulp_log2));
}

// the KNN lists with every step on the device
// after_contraction (may be empty): called once the contraction kernel is
// enqueued, before the first host read (with device inputs the cluster call
// starts InitBCM on a second stream there, so that its kernels queue behind
// the contraction's)
ancka_status knn_impl(Workspace& ws, const float* X, int64_t n, int32_t d, int32_t K, int32_t prec,
                      int32_t* idx, float* sim, int32_t** zero_row, int64_t* ncand, int64_t* nfb,
                      int64_t* nex, bool counts, cudaStream_t s, cudaEvent_t* contract_ev = nullptr,
                      const std::function<ancka_status()>& after_contraction = {}) {
  PrepOut pr;
  ANCKA_TRY(prep_rows(ws, X, n, d, prec, &pr, s));
  if (zero_row) *zero_row = pr.zero_row;
  // the candidate lists certify K when a few slots of slack remain: one list
  // of 32 (CUDA-core contraction) or two of 16 (tensor-core contraction)
  if (K <= max_candidate_K(prec)) {
    float* cv;
    int32_t* ci;
    ANCKA_TRY(ws.alloc(&cv, (size_t)n * kCandC));
    ANCKA_TRY(ws.alloc(&ci, (size_t)n * kCandC));
    float acc;
    int32_t* terr = nullptr;  // contraction error flag, read back by the re-rank's first host read
    if (contract_ev) ANCKA_CUDA(cudaEventRecord(contract_ev[0], s));
    if (prec == ANCKA_PREC_BF16) {
      ANCKA_TRY(ws.zeros(&terr, 1));
      ANCKA_TRY(knn_candidates_bf16(ws, pr, n, cv, ci, terr, s));
      if (contract_ev) ANCKA_CUDA(cudaEventRecord(contract_ev[1], s));
      acc = tc_acc_bound(pr.dp, 16, -22);
    } else if (prec == ANCKA_PREC_FP8) {
      ANCKA_TRY(ws.zeros(&terr, 1));
      ANCKA_TRY(knn_candidates_fp8(ws, pr, n, cv, ci, terr, s));
      if (contract_ev) ANCKA_CUDA(cudaEventRecord(contract_ev[1], s));
      acc = tc_acc_bound(pr.dp8, 32, -18);
    } else {
      ANCKA_TRY(knn_candidates_fp32(pr, n, cv, ci, s));
      if (contract_ev) ANCKA_CUDA(cudaEventRecord(contract_ev[1], s));
      // sequential FMA accumulation over dp terms: gamma_dp with u = 2^-24
      const double g = pr.dp * 5.960464477539063e-08;
      acc = (float)(1.01 * g / (1.0 - g));
    }
    if (after_contraction) ANCKA_TRY(after_contraction());
    // the tensor-core kernel leaves two 16-entry lists per row (one per half
    // of the key columns), the CUDA-core kernel one 32-entry list
    ANCKA_TRY(knn_rerank(ws, X, n, d, K, pr, prec, acc, tc_acc_bound(pr.dp, 16, -22), cv, ci,
                         prec == ANCKA_PREC_FP32 ? 1 : 2, prec == ANCKA_PREC_FP32 ? prec : ANCKA_PREC_BF16, terr, idx,
                         sim, ncand, nfb, nex, counts, s));
    if (contract_ev) ANCKA_CUDA(cudaEventRecord(contract_ev[2], s));
  } else {
    if (after_contraction) ANCKA_TRY(after_contraction());
    ANCKA_TRY(knn_rerank(ws, X, n, d, K, pr, ANCKA_PREC_FP32, 0.f, 0.f, nullptr, nullptr, 1, ANCKA_PREC_FP32,
                         nullptr, idx, sim, ncand, nfb, nex, counts, s));
  }
  return ANCKA_OK;
}

constexpr int kIvfIters = 8;  // spherical k-means rounds of the inverted-list KNN

ancka_status validate_ivf_args(const float* X, int64_t n, int32_t d, int32_t K, int32_t nlist, int32_t nprobe) {
  ANCKA_REQUIRE(X != nullptr, "X is NULL");
  ANCKA_REQUIRE(n >= 2 && n < (int64_t(1) << 31) - 1, "n out of range");
  ANCKA_REQUIRE(d >= 1 && round_up(d, 64) <= knn_tc_max_dp(), "inverted-list KNN: d must be in [1, %d]",
                knn_tc_max_dp());
  ANCKA_REQUIRE(K >= 1 && K <= 16 && K < n, "inverted-list KNN: need 1 <= K <= 16 and K < n");
  ANCKA_REQUIRE(nlist >= 1 && nlist <= 8192 && nlist <= n, "inverted-list KNN: need 1 <= nlist <= min(n, 8192)");
  ANCKA_REQUIRE(nprobe >= 1 && nprobe <= 32 && nprobe <= nlist, "inverted-list KNN: need 1 <= nprobe <= min(32, nlist)");
  ANCKA_REQUIRE(ceil_div(round_up(n, 128), 256) <= ivf_max_tiles(), "inverted-list KNN: n too large");
  return ANCKA_OK;
}

ancka_status validate_topology(const ancka_topology* t) {
  ANCKA_REQUIRE(t != nullptr, "topology is NULL");
  ANCKA_REQUIRE(t->n >= 2 && t->n < (int64_t(1) << 31) - 1, "topology n out of range");
  if (t->kind == ANCKA_HYPERGRAPH) {
    ANCKA_REQUIRE(t->m >= 1 && t->m < (int64_t(1) << 31) - 1, "hypergraph needs 1 <= m < 2^31");
    ANCKA_REQUIRE(t->he_ptr && t->he_nodes, "hypergraph pointers are NULL");
  } else if (t->kind == ANCKA_GRAPH || t->kind == ANCKA_MULTIPLEX) {
    ANCKA_REQUIRE(t->L >= 1 && t->L <= 64, "layers L = %d out of range [1, 64]", t->L);
    ANCKA_REQUIRE(t->kind == ANCKA_MULTIPLEX || t->L == 1, "a graph has exactly one layer");
    ANCKA_REQUIRE(t->row_ptr && (t->col_idx || t->nnz == 0), "graph pointers are NULL");
  } else {
    ANCKA_REQUIRE(false, "unknown topology kind %d", t->kind);
  }
  return ANCKA_OK;
}

ancka_status validate_params(const ancka_params* p, int64_t n) {
  ANCKA_REQUIRE(p != nullptr, "params is NULL");
  ANCKA_REQUIRE(p->k >= 1 && p->k <= 64 && p->k <= n, "k = %d must satisfy 1 <= k <= min(64, n)", p->k);
  ANCKA_REQUIRE(p->alpha > 0.f && p->alpha <= 1.f, "alpha must lie in (0, 1]");
  ANCKA_REQUIRE(p->beta >= 0.f && p->beta <= 1.f, "beta must lie in [0, 1]");
  ANCKA_REQUIRE(p->T >= 1 && p->tau >= 1, "T and tau must be >= 1");
  ANCKA_REQUIRE(p->gamma >= 0 && p->T_i >= 0, "gamma and T_i must be >= 0");
  ANCKA_REQUIRE(p->disc_max_iter >= 1 && p->disc_max_iter <= 1000, "disc_max_iter out of range");
  ANCKA_REQUIRE(p->T <= 100000, "T must be <= 100000");
  ANCKA_REQUIRE(p->init == 0 || (p->init == 1 && p->init_labels) || (p->init == 2 && p->warm),
                "init must be 0, 1 with init_labels, or 2 with a warm model");
  ANCKA_REQUIRE(p->early_stop == 0 || (p->early_stop == 1 && p->eps_Q >= 0.f), "early_stop must be 0 or 1, eps_Q >= 0");
  ANCKA_REQUIRE(p->knn_nlist >= 0, "knn_nlist must be >= 0 (0: exact KNN)");
  ANCKA_REQUIRE(p->node_order >= 0 && p->node_order <= 2, "node_order = %d must be 0, 1 or 2", p->node_order);
  return ANCKA_OK;
}

ancka_status validate_warm(const ancka_warm_model* m, int32_t d, int32_t k) {
  ANCKA_REQUIRE(m != nullptr, "warm model is NULL");
  ANCKA_REQUIRE(m->W1 && m->b1 && m->W2 && m->b2, "warm model has NULL weights");
  ANCKA_REQUIRE(m->hidden == 256, "warm model: hidden must be 256 (got %d)", m->hidden);
  ANCKA_REQUIRE(m->d_in == 2 * d, "warm model: d_in = %d must be 2 d = %d", m->d_in, 2 * d);
  ANCKA_REQUIRE(m->k == k && k >= 1 && k <= 64, "warm model: k = %d must equal the clusters %d (<= 64)", m->k, k);
  return ANCKA_OK;
}

// W = MLP([U | P_N U]) for the walk's topology (n x k, row stride ldw)
ancka_status warm_predict_impl(Workspace& ws, const Walk& w, const float* X, int32_t d, const ancka_warm_model* m,
                               float* W, int ldw, cudaStream_t s) {
  const int64_t n = w.n;
  const int kp = warm_kp(d);
  __nv_bfloat16 *A, *W1t;
  int32_t* err;
  ANCKA_TRY(ws.alloc(&A, (size_t)round_up(n, 128) * kp));
  ANCKA_TRY(ws.alloc(&W1t, (size_t)256 * kp));
  ANCKA_TRY(ws.zeros(&err, 1));
  ANCKA_TRY(warm_features(ws, w, X, d, A, nullptr, s));
  ANCKA_TRY(warm_refresh_w1t(m->W1, m->d_in, kp, W1t, s));
  ANCKA_TRY(warm_forward(ws, A, n, kp, W1t, m->b1, m->W2, m->b2, m->k, W, ldw, nullptr, nullptr, err, s));
  int32_t he = 0;
  ANCKA_CUDA(cudaMemcpyAsync(&he, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  ANCKA_CUDA(cudaStreamSynchronize(s));
  if (he) {
    set_error("warm-start GEMM: a pipeline wait expired (role %d)", he);
    return ANCKA_ERR_TIMEOUT;
  }
  return ANCKA_OK;
}

// x_ready (may be null): an event after which X is valid on the device; the
// topology build, which does not read X, runs before the stream waits on it.
ancka_status cluster_impl(const ancka_topology* topo, const float* X, int32_t d, const int32_t* knn_idx_in,
                          const float* knn_sim_in, const ancka_params* p, int32_t* labels,
                          const ancka_outputs* out, ancka_info* info, cudaStream_t s,
                          cudaEvent_t x_ready = nullptr) {
  ANCKA_TRY(device_check());
  ANCKA_TRY(validate_topology(topo));
  const int64_t n = topo->n;
  ANCKA_TRY(validate_params(p, n));
  ANCKA_REQUIRE(labels != nullptr, "labels is NULL");
  if (!knn_idx_in && p->knn_nlist > 0) {
    ANCKA_TRY(validate_ivf_args(X, n, d, p->K, p->knn_nlist, p->knn_nprobe));
  } else if (!knn_idx_in) {
    ANCKA_TRY(validate_knn_args(X, n, d, p->K, p->knn_prec));
  } else {
    ANCKA_REQUIRE(X && knn_sim_in && d >= 1 && p->K >= 1 && p->K < n, "bad KNN inputs");
  }
  if (info) memset(info, 0, sizeof(*info));
  Timer timer;
  Timer* tp = info ? &timer : nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaEvent_t cev[3] = {nullptr, nullptr, nullptr};
  bool contract_timed = false;
  if (info) {
    t0 = pooled_event();
    t1 = pooled_event();
    cev[0] = pooled_event();
    cev[1] = pooled_event();
    cev[2] = pooled_event();
    cudaEventRecord(t0, s);
  }
  ancka_status st = ANCKA_OK;
  {
    Workspace ws(s);
    const int K = p->K;
    int32_t* idx = (out && out->knn_idx) ? out->knn_idx : nullptr;
    float* sim = (out && out->knn_sim) ? out->knn_sim : nullptr;
    int32_t* zero_row = nullptr;
    int64_t ncand = 0, nfb = 0, nex = 0;
    int32_t* bad = nullptr;
    st = ws.zeros(&bad, 1);
    Walk w;
    if (st == ANCKA_OK) {  // the topology part of the walk needs no attributes
      Phase ph(tp, s, 1);
      st = build_topology(ws, *topo, &w, s);
    }
    // InitBCM needs only the topology: with the default start it runs on a
    // second stream.  For host inputs it starts as soon as the topology is
    // built, while X is still being copied; otherwise it is launched right
    // after the contraction kernel, so that it never holds SMs the
    // contraction's persistent CTAs wait for, and overlaps the re-rank and
    // the build.  The call's stream waits for it before the iteration, and
    // on every exit before the workspace is released.
    static thread_local cudaStream_t init_streams[kMaxDevices] = {};
    cudaStream_t& is = init_streams[device_slot()];
    if (!is) ANCKA_CUDA(cudaStreamCreateWithFlags(&is, cudaStreamNonBlocking));
    struct InitJoin {
      cudaStream_t s;
      cudaEvent_t topo_ev = nullptr, done_ev = nullptr;
      bool launched = false;
      ~InitJoin() {
        if (launched) cudaStreamWaitEvent(s, done_ev, 0);
        if (topo_ev) release_event(topo_ev);
        if (done_ev) release_event(done_ev);
      }
    } ij{s};
    Workspace wsi(is);  // InitBCM's scratch, used and released on its stream
    int32_t* y0_async = nullptr;
    const IterCfg cfg{p->k,     p->T,          p->gamma, p->T_i,  p->tau,
                      p->disc_max_iter, p->alpha, p->early_stop, p->eps_Q, p->node_order};
    auto start_init = [&]() -> ancka_status {
      if (p->init == 1) return ANCKA_OK;  // labels given
      ANCKA_TRY(ws.alloc(&y0_async, (size_t)n));
      ij.topo_ev = pooled_event();
      ij.done_ev = pooled_event();
      ANCKA_CUDA(cudaEventRecord(ij.topo_ev, s));  // the walk's topology and y0_async are ready on s here
      ANCKA_CUDA(cudaStreamWaitEvent(is, ij.topo_ev, 0));
      {
        Phase ph(tp, is, 2);
        ANCKA_TRY(initbcm_labels(wsi, w, cfg, y0_async, is));
      }
      ANCKA_CUDA(cudaEventRecord(ij.done_ev, is));
      ij.launched = true;
      return ANCKA_OK;
    };
    const bool early_init = x_ready != nullptr;
    if (st == ANCKA_OK && early_init) st = start_init();
    if (st == ANCKA_OK && x_ready) ANCKA_CUDA(cudaStreamWaitEvent(s, x_ready, 0));
    if (st == ANCKA_OK && !knn_idx_in) {
      Phase ph(tp, s, 0);
      if (!idx) st = ws.alloc(&idx, (size_t)n * K);
      if (st == ANCKA_OK && !sim) st = ws.alloc(&sim, (size_t)n * K);
      if (st == ANCKA_OK && p->knn_nlist > 0) {
        IvfStats stats;
        st = knn_ivf(ws, X, n, d, K, p->knn_nlist, p->knn_nprobe, kIvfIters, 0x5eed, idx, sim, &zero_row, &stats,
                     s);
        if (st == ANCKA_OK && !early_init) st = start_init();
        if (info) {
          info->knn_tiles = stats.key_tiles;
          info->knn_full_tiles = stats.full_tiles;
        }
      } else if (st == ANCKA_OK) {
        st = knn_impl(ws, X, n, d, K, p->knn_prec, idx, sim, &zero_row, &ncand, &nfb, &nex, info != nullptr, s,
                      info && K <= max_candidate_K(p->knn_prec) ? cev : nullptr,
                      early_init ? std::function<ancka_status()>() : std::function<ancka_status()>(start_init));
        contract_timed = info && K <= max_candidate_K(p->knn_prec);
      }
    } else if (st == ANCKA_OK) {
      Phase ph(tp, s, 0);
      k_check_knn<<<(unsigned)ceil_div(n * K, 256), 256, 0, s>>>(knn_idx_in, n, K, bad);
      int32_t hb = 0;
      st = read_flag(bad, s, &hb);
      if (st == ANCKA_OK && hb) {
        set_error("KNN list entry out of range or equal to its own row");
        st = ANCKA_ERR_INVALID_ARG;
      }
      if (st == ANCKA_OK) st = ws.alloc(&zero_row, (size_t)n);
      if (st == ANCKA_OK) {
        k_zero_rows<<<(unsigned)ceil_div(n, 8), 256, 0, s>>>(X, n, d, zero_row);
        if (cudaGetLastError() != cudaSuccess) st = ANCKA_ERR_CUDA;
      }
      if (st == ANCKA_OK && out && out->knn_idx)
        cudaMemcpyAsync(out->knn_idx, knn_idx_in, sizeof(int32_t) * n * K, cudaMemcpyDeviceToDevice, s);
      if (st == ANCKA_OK && out && out->knn_sim)
        cudaMemcpyAsync(out->knn_sim, knn_sim_in, sizeof(float) * n * K, cudaMemcpyDeviceToDevice, s);
      idx = const_cast<int32_t*>(knn_idx_in);
      sim = const_cast<float*>(knn_sim_in);
    }
    if (st == ANCKA_OK && knn_idx_in && !early_init) st = start_init();  // no contraction to queue behind
    if (st == ANCKA_OK && p->init == 1) {
      k_check_labels<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(p->init_labels, n, p->k, bad);
      int32_t hb = 0;
      st = read_flag(bad, s, &hb);
      if (st == ANCKA_OK && hb) {
        set_error("init_labels entry outside [0, k)");
        st = ANCKA_ERR_INVALID_ARG;
      }
    }
    if (st == ANCKA_OK) {
      Phase ph(tp, s, 1);
      st = build_knn_part(ws, n, K, idx, sim, zero_row, p->beta, &w, s);
    }
    IterTrace tr{};
    if (st == ANCKA_OK) {
      st = ws.zeros(&tr.phi_dev, ANCKA_MAX_TRACE);
      if (st == ANCKA_OK) st = ws.zeros(&tr.disc_iters_dev, ANCKA_MAX_TRACE);
      if (st == ANCKA_OK) st = ws.zeros(&tr.taken_dev, ANCKA_MAX_TRACE);
      if (st == ANCKA_OK) st = ws.zeros(&tr.flags_dev, 1);
      if (st == ANCKA_OK) st = ws.zeros(&tr.phi_best_dev, 1);
    }
    float* warmW = nullptr;
    const int ldwarm = p->k;
    if (st == ANCKA_OK && p->init == 2) {
      Phase ph(tp, s, 2);
      st = validate_warm(p->warm, d, p->k);
      if (st == ANCKA_OK) st = ws.alloc(&warmW, (size_t)n * ldwarm);
      if (st == ANCKA_OK) st = warm_predict_impl(ws, w, X, d, p->warm, warmW, ldwarm, s);
    }
    if (st == ANCKA_OK) {
      tr.events = tp ? &timer.ev : nullptr;
      tr.phases = tp ? &timer.ph : nullptr;
      const int32_t* y_init = p->init == 1 ? p->init_labels : y0_async;
      if (y0_async && ij.launched) ANCKA_CUDA(cudaStreamWaitEvent(s, ij.done_ev, 0));
      st = run_ancka(ws, w, cfg, y_init, warmW, ldwarm, labels, out ? out->Q : nullptr,
                     out ? out->init_labels : nullptr, &tr, s);
    }
    if (info) cudaEventRecord(t1, s);
    if (info && (st == ANCKA_OK || st == ANCKA_ERR_NUMERIC)) {
      cudaMemcpyAsync(info->phi, tr.phi_dev, sizeof(double) * ANCKA_MAX_TRACE, cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(info->disc_iters, tr.disc_iters_dev, sizeof(int32_t) * ANCKA_MAX_TRACE,
                      cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(info->taken, tr.taken_dev, sizeof(int32_t) * ANCKA_MAX_TRACE, cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(&info->numeric_flags, tr.flags_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(&info->phi_best, tr.phi_best_dev, sizeof(double), cudaMemcpyDeviceToHost, s);
      cudaError_t e = cudaStreamSynchronize(s);
      if (e != cudaSuccess && st == ANCKA_OK) st = cuda_fail(e, "cudaStreamSynchronize", __FILE__, __LINE__);
      info->n_phi = tr.n_phi;
      info->iters_run = tr.iters_run;
      info->warm_used = tr.warm_used;
      info->knn_candidates = ncand;
      info->knn_fallback_rows = nfb;
      info->knn_exhaustive_rows = nex;
    }
  }  // workspace released (stream-ordered)
  if (info) {
    cudaStreamSynchronize(s);
    fill_times(timer, info);
    float tot = 0.f;
    if (cudaEventElapsedTime(&tot, t0, t1) == cudaSuccess) info->ms_total = tot;
    float mc = 0.f;
    if (contract_timed && st == ANCKA_OK && cudaEventElapsedTime(&mc, cev[0], cev[1]) == cudaSuccess)
      info->ms_contract = mc;
    if (contract_timed && st == ANCKA_OK && cudaEventElapsedTime(&mc, cev[1], cev[2]) == cudaSuccess)
      info->ms_rerank = mc;
    cudaGetLastError();  // an event of a failed call may never have been recorded
    release_event(t0);
    release_event(t1);
    release_event(cev[0]);
    release_event(cev[1]);
    release_event(cev[2]);
  }
  if (st == ANCKA_OK) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "kernel launch", __FILE__, __LINE__);
  }
  return st;
}

}  // namespace
}  // namespace ancka

using namespace ancka;

// quantised unit rows as the contraction multiplied them (diagnostics)
__global__ void k_copy_qrows(const __nv_bfloat16* __restrict__ xb, int dp, const uint8_t* __restrict__ x8, int dp8,
                             const float* __restrict__ inv_s2, int64_t n, int d, float* __restrict__ q) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * d) return;
  const int64_t row = t / d;
  const int c = (int)(t % d);
  if (x8) {
    __nv_fp8_e4m3 v;
    v.__x = x8[row * dp8 + c];
    q[t] = (float)v * sqrtf(*inv_s2);  // 1/S exactly: S^2 is an even power of two
  } else {
    q[t] = __bfloat162float(xb[row * dp + c]);
  }
}

extern "C" {

void ancka_params_default(ancka_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->k = 5;
  p->K = 10;
  p->alpha = 0.2f;
  p->beta = 0.5f;
  p->T = 10;
  p->gamma = 3;
  p->T_i = 25;
  p->tau = 5;
  p->disc_max_iter = 20;
  p->knn_prec = ANCKA_PREC_BF16;
  p->init = 0;
  p->init_labels = nullptr;
  p->early_stop = 0;
  p->eps_Q = 0.005f;
  p->warm = nullptr;
}

const char* ancka_status_str(ancka_status s) {
  switch (s) {
    case ANCKA_OK: return "ANCKA_OK";
    case ANCKA_ERR_INVALID_ARG: return "ANCKA_ERR_INVALID_ARG";
    case ANCKA_ERR_OOM: return "ANCKA_ERR_OOM";
    case ANCKA_ERR_CUDA: return "ANCKA_ERR_CUDA";
    case ANCKA_ERR_NUMERIC: return "ANCKA_ERR_NUMERIC";
    case ANCKA_ERR_TIMEOUT: return "ANCKA_ERR_TIMEOUT";
    case ANCKA_ERR_UNSUPPORTED: return "ANCKA_ERR_UNSUPPORTED";
    case ANCKA_ERR_INTERNAL: return "ANCKA_ERR_INTERNAL";
  }
  return "ANCKA_ERR_UNKNOWN";
}

const char* ancka_last_error(void) { return g_err; }

ancka_status ancka_device_check(void) { return device_check(); }

int64_t ancka_kernel_launches(void) { return g_launches.load(); }

void ancka_set_symmetric_knn_min_rows(int64_t n_min) { knn_set_symmetric_min_rows(n_min); }

ancka_status ancka_knn_ivf(const float* X, int64_t n, int32_t d, int32_t K, int32_t nlist, int32_t nprobe,
                           int32_t* out_idx, float* out_sim, ancka_info* info, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ANCKA_TRY(device_check());
  ANCKA_TRY(validate_ivf_args(X, n, d, K, nlist, nprobe));
  ANCKA_REQUIRE(out_idx && out_sim, "output pointers are NULL");
  if (info) memset(info, 0, sizeof(*info));
  cudaEvent_t a = nullptr, b = nullptr;
  if (info) {
    a = pooled_event();
    b = pooled_event();
    cudaEventRecord(a, s);
  }
  ancka_status st;
  IvfStats stats;
  {
    Workspace ws(s);
    st = knn_ivf(ws, X, n, d, K, nlist, nprobe, kIvfIters, 0x5eed, out_idx, out_sim, nullptr, &stats, s);
  }
  if (info) {
    cudaEventRecord(b, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess && st == ANCKA_OK) st = cuda_fail(e, "cudaStreamSynchronize", __FILE__, __LINE__);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    info->ms_knn = ms;
    info->ms_total = ms;
    info->knn_tiles = stats.key_tiles;
    info->knn_full_tiles = stats.full_tiles;
    release_event(a);
    release_event(b);
  }
  return st;
}

ancka_status ancka_knn(const float* X, int64_t n, int32_t d, int32_t K, int32_t prec, int32_t* out_idx,
                       float* out_sim, ancka_info* info, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ANCKA_TRY(device_check());
  ANCKA_TRY(validate_knn_args(X, n, d, K, prec));
  ANCKA_REQUIRE(out_idx && out_sim, "output pointers are NULL");
  if (info) memset(info, 0, sizeof(*info));
  cudaEvent_t a = nullptr, b = nullptr;
  if (info) {
    a = pooled_event();
    b = pooled_event();
    cudaEventRecord(a, s);
  }
  ancka_status st;
  int64_t nc = 0, nf = 0, ne = 0;
  cudaEvent_t cev[3] = {nullptr, nullptr, nullptr};
  const bool timed = info && K <= max_candidate_K(prec);
  if (timed) {
    cev[0] = pooled_event();
    cev[1] = pooled_event();
    cev[2] = pooled_event();
  }
  {
    Workspace ws(s);
    st = knn_impl(ws, X, n, d, K, prec, out_idx, out_sim, nullptr, &nc, &nf, &ne, info != nullptr, s,
                  timed ? cev : nullptr);
  }
  if (info) {
    cudaEventRecord(b, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess && st == ANCKA_OK) st = cuda_fail(e, "cudaStreamSynchronize", __FILE__, __LINE__);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    info->ms_knn = ms;
    info->ms_total = ms;
    info->knn_candidates = nc;
    info->knn_fallback_rows = nf;
    info->knn_exhaustive_rows = ne;
    if (timed) {
      float mc = 0.f;
      if (st == ANCKA_OK && cudaEventElapsedTime(&mc, cev[0], cev[1]) == cudaSuccess) info->ms_contract = mc;
      if (st == ANCKA_OK && cudaEventElapsedTime(&mc, cev[1], cev[2]) == cudaSuccess) info->ms_rerank = mc;
      cudaGetLastError();
      release_event(cev[0]);
      release_event(cev[1]);
      release_event(cev[2]);
    }
    release_event(a);
    release_event(b);
  }
  return st;
}

ancka_status ancka_knn_candidates(const float* X, int64_t n, int32_t d, int32_t prec, float* cand_val,
                                  int32_t* cand_idx, float* qrows, float* err, float* acc, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ANCKA_TRY(device_check());
  ANCKA_REQUIRE(prec == ANCKA_PREC_BF16 || prec == ANCKA_PREC_FP8, "precision must be BF16 or FP8");
  ANCKA_TRY(validate_knn_args(X, n, d, 1, prec));
  ANCKA_REQUIRE(cand_val && cand_idx, "output pointers are NULL");
  Workspace ws(s);
  PrepOut pr;
  ANCKA_TRY(prep_rows(ws, X, n, d, prec, &pr, s));
  int32_t* terr;
  ANCKA_TRY(ws.zeros(&terr, 1));
  if (prec == ANCKA_PREC_BF16) {
    ANCKA_TRY(knn_candidates_bf16(ws, pr, n, cand_val, cand_idx, terr, s));
  } else {
    ANCKA_TRY(knn_candidates_fp8(ws, pr, n, cand_val, cand_idx, terr, s));
  }
  if (qrows) {
    k_copy_qrows<<<(unsigned)ceil_div(n * d, 256), 256, 0, s>>>(pr.xb, pr.dp, prec == ANCKA_PREC_FP8 ? pr.x8 : nullptr,
                                                                pr.dp8, pr.inv_s2, n, d, qrows);
    ANCKA_LAUNCHED();
  }
  if (err)
    ANCKA_CUDA(cudaMemcpyAsync(err, prec == ANCKA_PREC_FP8 ? pr.err8 : pr.err, sizeof(float) * n,
                               cudaMemcpyDeviceToDevice, s));
  int32_t hterr = 0;
  ANCKA_CUDA(cudaMemcpyAsync(&hterr, terr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  ANCKA_CUDA(cudaStreamSynchronize(s));
  if (hterr) {
    set_error("tensor-core contraction: a pipeline wait expired (role %d)", hterr);
    return ANCKA_ERR_TIMEOUT;
  }
  if (acc) *acc = prec == ANCKA_PREC_FP8 ? tc_acc_bound(pr.dp8, 32, -18) : tc_acc_bound(pr.dp, 16, -22);
  return ANCKA_OK;
}

ancka_status ancka_cluster(const ancka_topology* topo, const float* X, int32_t d, const ancka_params* p,
                           int32_t* labels, const ancka_outputs* out, ancka_info* info, void* stream) {
  return cluster_impl(topo, X, d, nullptr, nullptr, p, labels, out, info, static_cast<cudaStream_t>(stream));
}

ancka_status ancka_cluster_with_knn(const ancka_topology* topo, const float* X, int32_t d,
                                    const int32_t* knn_idx, const float* knn_sim, const ancka_params* p,
                                    int32_t* labels, const ancka_outputs* out, ancka_info* info, void* stream) {
  if (!knn_idx || !knn_sim) {
    set_error("knn_idx / knn_sim are NULL");
    return ANCKA_ERR_INVALID_ARG;
  }
  return cluster_impl(topo, X, d, knn_idx, knn_sim, p, labels, out, info, static_cast<cudaStream_t>(stream));
}

ancka_status ancka_cluster_host(const ancka_topology* topo, const float* X, int32_t d, const ancka_params* p,
                                int32_t* labels, ancka_info* info, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ANCKA_TRY(device_check());
  ANCKA_TRY(validate_topology(topo));
  ANCKA_REQUIRE(X && labels, "X or labels is NULL");
  const int64_t n = topo->n;
  ANCKA_TRY(validate_params(p, n));
  ANCKA_REQUIRE(d >= 1 && d <= 4096, "d out of range");
  ancka_topology dt = *topo;
  ancka_status st = ANCKA_OK;
  // X (the large copy) goes on a second stream so that the topology build
  // overlaps it; the call's stream waits for it before the KNN
  static thread_local cudaStream_t copy_streams[kMaxDevices] = {};
  cudaStream_t& xs = copy_streams[device_slot()];
  if (!xs) ANCKA_CUDA(cudaStreamCreateWithFlags(&xs, cudaStreamNonBlocking));
  // on every exit: s waits for the copy before the workspace frees dX on s,
  // and the events go back to the pool
  struct CopyGuard {
    cudaStream_t s;
    cudaEvent_t alloc_ev, x_ev;
    bool recorded = false;
    ~CopyGuard() {
      if (recorded) cudaStreamWaitEvent(s, x_ev, 0);
      release_event(alloc_ev);
      release_event(x_ev);
    }
  };
  {
    Workspace ws(s);
    CopyGuard guard{s, pooled_event(), pooled_event()};
    cudaEvent_t alloc_ev = guard.alloc_ev, x_ev = guard.x_ev;
    if (topo->kind == ANCKA_HYPERGRAPH) {
      const int64_t m = topo->m;
      const int64_t nnz = topo->he_ptr[m];
      int64_t* hp;
      int32_t* hn;
      ANCKA_TRY(ws.alloc(&hp, (size_t)m + 1));
      ANCKA_TRY(ws.alloc(&hn, (size_t)(nnz > 0 ? nnz : 1)));
      ANCKA_CUDA(cudaMemcpyAsync(hp, topo->he_ptr, sizeof(int64_t) * (m + 1), cudaMemcpyHostToDevice, s));
      if (nnz > 0) ANCKA_CUDA(cudaMemcpyAsync(hn, topo->he_nodes, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s));
      dt.he_ptr = hp;
      dt.he_nodes = hn;
    } else {
      const int64_t np = (int64_t)topo->L * (n + 1);
      int64_t* rp;
      int32_t* ci;
      ANCKA_TRY(ws.alloc(&rp, (size_t)np));
      ANCKA_TRY(ws.alloc(&ci, (size_t)(topo->nnz > 0 ? topo->nnz : 1)));
      ANCKA_CUDA(cudaMemcpyAsync(rp, topo->row_ptr, sizeof(int64_t) * np, cudaMemcpyHostToDevice, s));
      if (topo->nnz > 0)
        ANCKA_CUDA(cudaMemcpyAsync(ci, topo->col_idx, sizeof(int32_t) * topo->nnz, cudaMemcpyHostToDevice, s));
      dt.row_ptr = rp;
      dt.col_idx = ci;
    }
    // X after the topology: copies on one engine run in issue order, and the
    // topology build should not wait behind the large copy
    float* dX;
    int32_t* dlab;
    ANCKA_TRY(ws.alloc(&dX, (size_t)n * d));
    ANCKA_TRY(ws.alloc(&dlab, (size_t)n));
    ANCKA_CUDA(cudaEventRecord(alloc_ev, s));  // the allocation is valid on xs after this point of s
    ANCKA_CUDA(cudaStreamWaitEvent(xs, alloc_ev, 0));
    ANCKA_CUDA(cudaMemcpyAsync(dX, X, sizeof(float) * n * d, cudaMemcpyHostToDevice, xs));
    ANCKA_CUDA(cudaEventRecord(x_ev, xs));
    guard.recorded = true;
    ancka_params dp = *p;
    int32_t* dinit = nullptr;
    if (p->init == 1) {
      ANCKA_TRY(ws.alloc(&dinit, (size_t)n));
      ANCKA_CUDA(cudaMemcpyAsync(dinit, p->init_labels, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
      dp.init_labels = dinit;
    }
    st = cluster_impl(&dt, dX, d, nullptr, nullptr, &dp, dlab, nullptr, info, s, x_ev);
    if (st == ANCKA_OK) ANCKA_CUDA(cudaMemcpyAsync(labels, dlab, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
  }
  ANCKA_CUDA(cudaStreamSynchronize(s));
  return st;
}

ancka_status ancka_discretize(const float* Qk, int64_t n, int32_t k, int32_t ldq, int32_t max_iter,
                              int32_t* labels, int32_t* iters, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ANCKA_TRY(device_check());
  ANCKA_REQUIRE(Qk && labels, "Qk or labels is NULL");
  ANCKA_REQUIRE(n >= 1 && n < (int64_t(1) << 31) - 1, "n out of range");
  ANCKA_REQUIRE(k >= 1 && k <= 64, "k = %d out of range [1, 64]", k);
  ANCKA_REQUIRE(ldq >= k, "ldq < k");
  ANCKA_REQUIRE(max_iter >= 1 && max_iter <= 1000, "max_iter out of range");
  ancka_status st;
  int32_t hit = 0;
  {
    Workspace ws(s);
    int32_t* it;
    int32_t* derr = nullptr;
    ANCKA_TRY(ws.zeros(&it, 1));
    st = discretize(ws, Qk, n, k, ldq, max_iter, labels, it, nullptr, &derr, s);
    if (st == ANCKA_OK) {
      int32_t he = 0;
      ANCKA_CUDA(cudaMemcpyAsync(&hit, it, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      ANCKA_CUDA(cudaMemcpyAsync(&he, derr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      ANCKA_CUDA(cudaStreamSynchronize(s));
      if (he) {
        set_error("Discretize: a grid barrier wait expired");
        st = ANCKA_ERR_TIMEOUT;
      }
      if (iters) *iters = hit;
    }
  }
  return st;
}

ancka_status ancka_polar_factor(const float* M, int32_t k, float* R, int32_t* method, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ANCKA_TRY(device_check());
  ANCKA_REQUIRE(M && R, "M or R is NULL");
  ANCKA_REQUIRE(k >= 1 && k <= 64, "k = %d out of range [1, 64]", k);
  Workspace ws(s);
  int32_t* md;
  ANCKA_TRY(ws.zeros(&md, 1));
  ANCKA_TRY(polar_factor(M, k, R, md, s));
  if (method) {
    ANCKA_CUDA(cudaMemcpyAsync(method, md, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    ANCKA_CUDA(cudaStreamSynchronize(s));
  }
  return ANCKA_OK;
}

ancka_status ancka_warm_predict(const ancka_topology* topo, const float* X, int32_t d, const ancka_warm_model* model,
                                float* W, void* stream) {
  using namespace ancka;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ANCKA_TRY(device_check());
  ANCKA_TRY(validate_topology(topo));
  ANCKA_REQUIRE(X && W && d >= 1 && d <= 4096, "bad X / W / d");
  ANCKA_REQUIRE(model != nullptr, "warm model is NULL");
  ANCKA_TRY(validate_warm(model, d, model->k));
  Workspace ws(s);
  Walk w;
  ANCKA_TRY(build_topology(ws, *topo, &w, s));
  return warm_predict_impl(ws, w, X, d, model, W, model->k, s);
}

namespace {
struct WarmBuffers {
  float *mW1, *vW1, *mb1, *vb1, *mW2, *vW2, *mb2, *vb2;
  __nv_bfloat16* W1t;
  double* loss;
  int32_t *status, *err;
};

ancka_status warm_buffers(ancka::Workspace& ws, int d_in, int kp, int k, int steps, WarmBuffers* b) {
  using namespace ancka;
  ANCKA_TRY(ws.zeros(&b->mW1, (size_t)d_in * 256));
  ANCKA_TRY(ws.zeros(&b->vW1, (size_t)d_in * 256));
  ANCKA_TRY(ws.zeros(&b->mb1, 256));
  ANCKA_TRY(ws.zeros(&b->vb1, 256));
  ANCKA_TRY(ws.zeros(&b->mW2, (size_t)256 * k));
  ANCKA_TRY(ws.zeros(&b->vW2, (size_t)256 * k));
  ANCKA_TRY(ws.zeros(&b->mb2, (size_t)k));
  ANCKA_TRY(ws.zeros(&b->vb2, (size_t)k));
  ANCKA_TRY(ws.alloc(&b->W1t, (size_t)256 * kp));
  ANCKA_TRY(ws.zeros(&b->loss, (size_t)(steps > 0 ? steps : 1)));
  ANCKA_TRY(ws.zeros(&b->status, 1));
  ANCKA_TRY(ws.zeros(&b->err, 1));
  return ANCKA_OK;
}

struct WarmGraphDev {
  int64_t n;
  __nv_bfloat16 *A, *At;
  const float* Qt;
};

ancka_status warm_graph_setup(ancka::Workspace& ws, const ancka_warm_graph& g, int d, int k, WarmGraphDev* o,
                              cudaStream_t s) {
  using namespace ancka;
  ANCKA_REQUIRE(g.topo && g.X && g.Qt, "warm graph with NULL topology, X or Qt");
  ANCKA_REQUIRE(g.d == d, "every warm graph must have d = %d", d);
  ANCKA_TRY(validate_topology(g.topo));
  ANCKA_REQUIRE(g.topo->n >= k + 1, "warm graph smaller than k + 1 nodes");
  Walk w;
  ANCKA_TRY(build_topology(ws, *g.topo, &w, s));
  const int kp = warm_kp(d);
  o->n = w.n;
  ANCKA_TRY(ws.alloc(&o->A, (size_t)round_up(w.n, 128) * kp));
  ANCKA_TRY(ws.alloc(&o->At, (size_t)round_up(kp, 128) * round_up(w.n, 64)));
  ANCKA_TRY(warm_features(ws, w, g.X, d, o->A, o->At, s));
  o->Qt = g.Qt;
  return ANCKA_OK;
}

ancka_status warm_step_args(const WarmGraphDev& g, const ancka_warm_model* m, int kp, const WarmBuffers& b, float lr,
                            float lam, int t, double* loss_dev, const ancka::WarmGrads* grads,
                            ancka::WarmStepArgs* a) {
  a->n = g.n;
  a->k = m->k;
  a->d_in = m->d_in;
  a->kp = kp;
  a->A = g.A;
  a->At = g.At;
  a->Qt = g.Qt;
  a->ldq = m->k;
  a->W1 = m->W1;
  a->b1 = m->b1;
  a->W2 = m->W2;
  a->b2 = m->b2;
  a->W1t = b.W1t;
  a->mW1 = b.mW1;
  a->vW1 = b.vW1;
  a->mb1 = b.mb1;
  a->vb1 = b.vb1;
  a->mW2 = b.mW2;
  a->vW2 = b.vW2;
  a->mb2 = b.mb2;
  a->vb2 = b.vb2;
  a->lr = lr;
  a->lam = lam;
  a->t = t;
  a->loss_dev = loss_dev;
  a->status = b.status;
  a->err = b.err;
  a->grads = grads;
  return ANCKA_OK;
}

ancka_status warm_check(const WarmBuffers& b, cudaStream_t s) {
  using namespace ancka;
  int32_t h[2] = {0, 0};
  ANCKA_CUDA(cudaMemcpyAsync(&h[0], b.err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  ANCKA_CUDA(cudaMemcpyAsync(&h[1], b.status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  ANCKA_CUDA(cudaStreamSynchronize(s));
  if (h[0]) {
    set_error("warm-start GEMM: a pipeline wait expired (role %d)", h[0]);
    return ANCKA_ERR_TIMEOUT;
  }
  if (h[1]) {
    set_error("warm start: W^T W is singular");
    return ANCKA_ERR_NUMERIC;
  }
  return ANCKA_OK;
}
}  // namespace

ancka_status ancka_warm_train(const ancka_warm_graph* graphs, int32_t n_graphs, int32_t epochs, float lr, float lam,
                              ancka_warm_model* model, float* losses, void* stream) {
  using namespace ancka;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ANCKA_TRY(device_check());
  ANCKA_REQUIRE(graphs && n_graphs >= 1 && epochs >= 1 && epochs <= 100000, "bad graphs / epochs");
  ANCKA_REQUIRE(lr >= 0.f && lam >= 0.f, "lr and lam must be >= 0");
  ANCKA_REQUIRE(model != nullptr, "warm model is NULL");
  const int d = graphs[0].d;
  ANCKA_TRY(validate_warm(model, d, model->k));
  const int kp = warm_kp(d);
  Workspace ws(s);
  std::vector<WarmGraphDev> gd((size_t)n_graphs);
  for (int g = 0; g < n_graphs; ++g) ANCKA_TRY(warm_graph_setup(ws, graphs[g], d, model->k, &gd[(size_t)g], s));
  const int steps = epochs * n_graphs;
  WarmBuffers b;
  ANCKA_TRY(warm_buffers(ws, model->d_in, kp, model->k, steps, &b));
  ANCKA_TRY(warm_refresh_w1t(model->W1, model->d_in, kp, b.W1t, s));
  for (int e = 0; e < epochs; ++e)
    for (int g = 0; g < n_graphs; ++g) {
      const int t = e * n_graphs + g;
      WarmStepArgs a;
      warm_step_args(gd[(size_t)g], model, kp, b, lr, lam, t + 1, b.loss + t, nullptr, &a);
      Workspace step_ws(s);  // the step's temporaries, released (stream-ordered) after it
      ANCKA_TRY(warm_train_step(step_ws, a, s));
    }
  ANCKA_TRY(warm_check(b, s));
  if (losses) {
    std::vector<double> h((size_t)steps);
    ANCKA_CUDA(cudaMemcpyAsync(h.data(), b.loss, sizeof(double) * steps, cudaMemcpyDeviceToHost, s));
    ANCKA_CUDA(cudaStreamSynchronize(s));
    for (int t = 0; t < steps; ++t) losses[t] = (float)h[(size_t)t];
  }
  return ANCKA_OK;
}

ancka_status ancka_warm_gradients(const ancka_warm_graph* graph, float lam, const ancka_warm_model* model,
                                  float* dW1, float* db1, float* dW2, float* db2, double* loss, void* stream) {
  using namespace ancka;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ANCKA_TRY(device_check());
  ANCKA_REQUIRE(graph && model && dW1 && db1 && dW2 && db2, "NULL argument");
  ANCKA_TRY(validate_warm(model, graph->d, model->k));
  const int kp = warm_kp(graph->d);
  Workspace ws(s);
  WarmGraphDev g;
  ANCKA_TRY(warm_graph_setup(ws, *graph, graph->d, model->k, &g, s));
  WarmBuffers b;
  ANCKA_TRY(warm_buffers(ws, model->d_in, kp, model->k, 1, &b));
  ANCKA_TRY(warm_refresh_w1t(model->W1, model->d_in, kp, b.W1t, s));
  // lr = 0: the step leaves the weights unchanged (its Adam moments are scratch)
  const WarmGrads gr{dW1, db1, dW2, db2};
  WarmStepArgs a;
  warm_step_args(g, model, kp, b, 0.f, lam, 1, b.loss, &gr, &a);
  ANCKA_TRY(warm_train_step(ws, a, s));
  ANCKA_TRY(warm_check(b, s));
  if (loss) {
    ANCKA_CUDA(cudaMemcpyAsync(loss, b.loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    ANCKA_CUDA(cudaStreamSynchronize(s));
  }
  return ANCKA_OK;
}

}  // extern "C"
