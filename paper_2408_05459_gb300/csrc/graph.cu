// Walk-matrix structures of Section 6.1 and the KNN graph of Eq. AK.
//
// Topology (built once per call, deterministic):
//   graph / multiplex  each layer's (row, col) pairs (plus reversed pairs for
//     directed input) are sorted and de-duplicated (skipped for undirected
//     input whose rows are already strictly increasing), giving the binary A_l of
//     Eq. rw-ag / rw-mg; the layers are then concatenated row by row into one
//     CSR whose values are P_N[i,j] = 1/(L deg_l(i)) and, on the same
//     pattern, P_N^T[i,j] = 1/(L deg_l(j)) (A_l is symmetric).
//   hypergraph  (e, v) pairs are sorted and de-duplicated into H (hyperedge
//     -> members) and H^T (node -> incident hyperedges) of Eq. rw-hg; the
//     diagonal scalings 1/|e| and 1/delta(v) are kept as vectors.
// KNN part: row i holds its K out-neighbours with A_K = 2f (mutual) or f,
// then the nodes that list i but are not listed by i (weight f), in source
// order; values are pre-scaled to beta_i A_K[i,j] / D_K[i] (Eq. p-mat-ancka).
#include "common.cuh"

namespace ancka {

namespace {

// Sort keys pack (row, col) as row << cb | col with cb = bits of the column
// range, so a sort covers only the bits in use (8 bits per radix pass).
__host__ __device__ __forceinline__ uint64_t col_mask(int cb) { return (uint64_t(1) << cb) - 1; }

int bits_for(int64_t n) {
  int b = 1;
  while ((int64_t(1) << b) < n) ++b;
  return b;
}

ancka_status check_bad(const int32_t* bad, cudaStream_t s, const char* fmt, int arg = 0) {
  int32_t h = 0;
  ANCKA_CUDA(cudaMemcpyAsync(&h, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  ANCKA_CUDA(cudaStreamSynchronize(s));
  if (h) {
    set_error(fmt, arg);
    return ANCKA_ERR_INVALID_ARG;
  }
  return ANCKA_OK;
}

ancka_status read_count(const int64_t* dev, int64_t* host, cudaStream_t s) {
  ANCKA_CUDA(cudaMemcpyAsync(host, dev, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  ANCKA_CUDA(cudaStreamSynchronize(s));
  return ANCKA_OK;
}

// --- kernels -----------------------------------------------------------------
// a row pointer must start at >= 0, never decrease, and end at <= limit
__global__ void k_check_ptr(const int64_t* __restrict__ ptr, int64_t rows, int64_t limit,
                            int32_t* __restrict__ bad) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > rows) return;
  if (i == 0 && ptr[0] < 0) atomicExch(bad, 1);
  if (i == rows && limit >= 0 && ptr[rows] > limit) atomicExch(bad, 1);
  if (i < rows && ptr[i] > ptr[i + 1]) atomicExch(bad, 1);
}

// Entry-parallel kernels: a warp covers 32 x kPerLane consecutive entries,
// lane-interleaved (so loads and stores coalesce); each lane finds the row of
// its first entry by binary search and walks forward.  Rows of any length
// (hubs of skewed degree distributions) cost the same per entry.
constexpr int kPerLane = 16;

// the last row r in [0, nrows) with ptr[r] <= p (the row holding entry p
// when ptr[0] <= p < ptr[nrows])
__device__ __forceinline__ int64_t row_of(const int64_t* __restrict__ ptr, int64_t nrows, int64_t p) {
  int64_t lo = 0, hi = nrows - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (ptr[mid] <= p) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// (row, col) keys of one layer (and the reversed pairs for directed input);
// *unsorted is set if some row's columns are not strictly increasing
__global__ void k_csr_to_keys(const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                              int64_t n, int directed, int cb, uint64_t* __restrict__ keys,
                              int32_t* __restrict__ bad, int32_t* __restrict__ unsorted) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t base = ptr[0], total = ptr[n] - base;
  const int64_t q0 = warp * 32 * kPerLane + lane;
  if (q0 >= total) return;
  int64_t i = row_of(ptr, n, base + q0);
  bool out_of_order = false;
  for (int t = 0; t < kPerLane; ++t) {
    const int64_t q = q0 + 32 * t;
    if (q >= total) break;
    const int64_t p = base + q;
    while (ptr[i + 1] <= p) ++i;
    int32_t j = col[p];
    if (p > ptr[i] && col[p - 1] >= j) out_of_order = true;
    if (j < 0 || j >= n) {
      atomicExch(bad, 1);
      j = 0;
    }
    keys[directed ? 2 * q : q] = ((uint64_t)i << cb) | (uint32_t)j;
    if (directed) keys[2 * q + 1] = ((uint64_t)j << cb) | (uint32_t)i;
  }
  if (out_of_order) *unsorted = 1;
}

__global__ void k_hyper_to_keys(const int64_t* __restrict__ he_ptr, const int32_t* __restrict__ nodes,
                                int64_t m, int64_t n, int cb, uint64_t* __restrict__ keys,
                                int32_t* __restrict__ bad) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  for (int64_t p = he_ptr[e]; p < he_ptr[e + 1]; ++p) {
    int32_t v = nodes[p];
    if (v < 0 || v >= n) {
      atomicExch(bad, 1);
      v = 0;
    }
    keys[p - he_ptr[0]] = ((uint64_t)e << cb) | (uint32_t)v;
  }
}

// counts per row (key >> cb); col = low cb bits
__global__ void k_keys_to_cols(const uint64_t* __restrict__ keys, int64_t cnt, int cb, int32_t* __restrict__ col) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < cnt) col[q] = (int32_t)(keys[q] & col_mask(cb));
}

// ptr[r] = the first key position whose row is >= r (r = 0..nrows)
__global__ void k_row_bounds(const uint64_t* __restrict__ keys, int64_t cnt, int cb, int64_t nrows,
                             int64_t* __restrict__ ptr) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r > nrows) return;
  int64_t lo = 0, hi = cnt;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)(keys[mid] >> cb) < r) lo = mid + 1;
    else hi = mid;
  }
  ptr[r] = lo;
}

__global__ void k_row_counts(const int64_t* __restrict__ ptr, int64_t nrows, int32_t* __restrict__ cnt) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nrows) cnt[r] = (int32_t)(ptr[r + 1] - ptr[r]);
}

// (row << cb_in | col) -> (col << cb_out | row); cb_out covers the old rows
__global__ void k_swap_halves(const uint64_t* __restrict__ in, const int64_t* __restrict__ cnt_dev, int cb_in,
                              int cb_out, uint64_t* __restrict__ out) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= *cnt_dev) return;
  uint64_t k = in[q];
  out[q] = ((k & col_mask(cb_in)) << cb_out) | (k >> cb_in);
}

__global__ void k_inv_count(const int32_t* __restrict__ c, float* __restrict__ inv, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) inv[i] = c[i] > 0 ? 1.f / (float)c[i] : 0.f;
}

// merged multiplex / graph CSR: row i = layer 0 row i, layer 1 row i, ...
// merged entry o of row i: the layers' rows in layer order
__global__ void k_merge_layers(int L, int64_t n, const int64_t* const* __restrict__ lptr,
                               const int32_t* const* __restrict__ lcol,
                               const int32_t* const* __restrict__ ldeg,
                               const int64_t* __restrict__ mptr, int32_t* __restrict__ mcol,
                               float* __restrict__ val, float* __restrict__ valT) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t total = mptr[n];
  const int64_t o0 = warp * 32 * kPerLane + lane;
  if (o0 >= total) return;
  const float invL = 1.f / (float)L;
  int64_t i = row_of(mptr, n, o0);
  for (int t = 0; t < kPerLane; ++t) {
    const int64_t o = o0 + 32 * t;
    if (o >= total) break;
    while (mptr[i + 1] <= o) ++i;
    int64_t d = o - mptr[i];
    int l = 0;
    for (; l < L - 1; ++l) {
      const int64_t len = lptr[l][i + 1] - lptr[l][i];
      if (d < len) break;
      d -= len;
    }
    const int32_t j = lcol[l][lptr[l][i] + d];
    mcol[o] = j;
    const int32_t* deg = ldeg[l];
    if (val) val[o] = deg[i] > 0 ? invL / (float)deg[i] : 0.f;
    if (valT) valT[o] = deg[j] > 0 ? invL / (float)deg[j] : 0.f;  // deg[j] >= 1 for a symmetric A_l
  }
}

__global__ void k_sum_deg(int L, int64_t n, const int32_t* const* __restrict__ ldeg,
                          int32_t* __restrict__ deg, int64_t* __restrict__ mlen) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t s = 0;
  for (int l = 0; l < L; ++l) s += ldeg[l][i];
  deg[i] = s;
  mlen[i] = s;
}

// --- KNN augmentation -------------------------------------------------------
__global__ void k_knn_mutual(const int32_t* __restrict__ idx, int64_t n, int K, int cb,
                             uint8_t* __restrict__ mutual, uint64_t* __restrict__ keys,
                             int32_t* __restrict__ in_cnt) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * K) return;
  int64_t i = q / K;
  int32_t j = idx[q];
  bool mu = false;
  for (int p = 0; p < K; ++p) mu |= (idx[(int64_t)j * K + p] == (int32_t)i);
  mutual[q] = mu ? 1 : 0;
  if (mu) {
    keys[q] = uint64_t(1) << (2 * cb);  // sorts after every real key
  } else {
    keys[q] = ((uint64_t)j << cb) | (uint32_t)i;
    atomicAdd(&in_cnt[j], 1);
  }
}

__global__ void k_knn_len(const int32_t* __restrict__ in_cnt, int64_t n, int K,
                          int64_t* __restrict__ len, int64_t* __restrict__ in_len) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  len[i] = K + in_cnt[i];
  in_len[i] = in_cnt[i];
}

// row i: K out-entries, then in-entries; A_K values, D_K, beta_i, P values.
// One warp per row: lanes take the entries round-robin, D_K is a fixed-order
// butterfly sum, and each lane rescales the entries it wrote.
__global__ void k_knn_fill(const int32_t* __restrict__ idx, const float* __restrict__ sim,
                           const uint8_t* __restrict__ mutual, const uint64_t* __restrict__ skeys,
                           const int64_t* __restrict__ in_start, const int32_t* __restrict__ in_cnt,
                           int64_t n, int K, const int64_t* __restrict__ ptr,
                           int32_t* __restrict__ col, float* __restrict__ val,
                           const int32_t* __restrict__ zero_row, const int32_t* __restrict__ degree,
                           float beta, int cb, float* __restrict__ beta_out) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= n) return;  // uniform over the warp
  const int64_t o = ptr[i];
  // D_K[i] as a float-float pair (compensated FP32; GB300's FP64 pipe is narrow)
  float Dh = 0.f, Dl = 0.f;
  for (int p = lane; p < K; p += 32) {
    const int64_t q = i * K + p;
    const float a = mutual[q] ? 2.f * sim[q] : sim[q];
    col[o + p] = idx[q];
    val[o + p] = a;
    ff_add(Dh, Dl, a, 0.f);
  }
  const int64_t b = in_start[i];
  const int32_t c = in_cnt[i];
  for (int32_t t = lane; t < c; t += 32) {
    const int32_t src = (int32_t)(skeys[b + t] & col_mask(cb));
    float f = 0.f;
    for (int p = 0; p < K; ++p)
      if (idx[(int64_t)src * K + p] == (int32_t)i) f = sim[(int64_t)src * K + p];
    col[o + K + t] = src;
    val[o + K + t] = f;
    ff_add(Dh, Dl, f, 0.f);
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {  // ff_add is symmetric: every lane ends equal
    const float oh = __shfl_xor_sync(0xffffffffu, Dh, off), ol = __shfl_xor_sync(0xffffffffu, Dl, off);
    ff_add(Dh, Dl, oh, ol);
  }
  // Eq. beta_i, then reading R3 (a non-positive KNN degree disables the KNN walk)
  float bi = zero_row[i] ? 0.f : (degree[i] == 0 ? 1.f : beta);
  if (!(Dh > 0.f)) bi = 0.f;
  if (lane == 0) beta_out[i] = bi;
  // bi / (Dh + Dl) with one correction step: q = bi / Dh, then q -= q * Dl / Dh
  float scale = 0.f;
  if (Dh > 0.f) {
    const float q0 = __fdiv_rn(bi, Dh);
    scale = fmaf(-q0, __fdiv_rn(Dl, Dh), q0);
  }
  for (int p = lane; p < K; p += 32) val[o + p] *= scale;
  for (int32_t t = lane; t < c; t += 32) val[o + K + t] *= scale;
}

__global__ void k_topo_rowscale(const float* __restrict__ beta, const float* __restrict__ inv_deg,
                                int64_t n, float* __restrict__ rs) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  rs[i] = (1.f - beta[i]) * (inv_deg ? inv_deg[i] : 1.f);
}

inline unsigned grid_for(int64_t n, int b) { return (unsigned)ceil_div(n > 0 ? n : 1, b); }

// sorted unique keys -> CSR over the high halves (rows 0..nrows-1)
ancka_status keys_to_csr(Workspace& ws, const uint64_t* ukeys, int64_t ucnt,
                         int64_t nrows, int cb, Csr* out, int32_t** rowcnt_out, cudaStream_t s) {
  int32_t* rowcnt;
  ANCKA_TRY(ws.alloc(&rowcnt, (size_t)nrows + 1));
  ANCKA_TRY(ws.alloc(&out->col, (size_t)ucnt));
  k_keys_to_cols<<<grid_for(ucnt, 256), 256, 0, s>>>(ukeys, ucnt, cb, out->col);
  ANCKA_LAUNCHED();
  ANCKA_TRY(ws.alloc(&out->ptr, (size_t)nrows + 1));
  k_row_bounds<<<grid_for(nrows + 1, 256), 256, 0, s>>>(ukeys, ucnt, cb, nrows, out->ptr);
  ANCKA_LAUNCHED();
  k_row_counts<<<grid_for(nrows, 256), 256, 0, s>>>(out->ptr, nrows, rowcnt);
  ANCKA_LAUNCHED();
  out->nrows = nrows;
  out->nnz = ucnt;
  *rowcnt_out = rowcnt;
  return ANCKA_OK;
}

}  // namespace

ancka_status build_topology(Workspace& ws, const ancka_topology& t, Walk* w, cudaStream_t s) {
  const int64_t n = t.n;
  w->kind = t.kind;
  w->n = n;
  int32_t* bad;
  ANCKA_TRY(ws.zeros(&bad, 1));
  const int nb = bits_for(n);
  if (t.kind == ANCKA_HYPERGRAPH) {
    const int64_t m = t.m;
    w->m = m;
    k_check_ptr<<<grid_for(m + 1, 256), 256, 0, s>>>(t.he_ptr, m, -1, bad);
    ANCKA_LAUNCHED();
    // the pointer check and the entry count in one host read
    int64_t nnz = 0, base = 0;
    int32_t hbad = 0;
    ANCKA_CUDA(cudaMemcpyAsync(&nnz, t.he_ptr + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    ANCKA_CUDA(cudaMemcpyAsync(&base, t.he_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    ANCKA_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    ANCKA_CUDA(cudaStreamSynchronize(s));
    if (hbad) {
      set_error("hyperedge pointer must be non-negative and non-decreasing");
      return ANCKA_ERR_INVALID_ARG;
    }
    nnz -= base;
    uint64_t *k0, *k1, *k2;
    ANCKA_TRY(ws.alloc(&k0, (size_t)nnz));
    ANCKA_TRY(ws.alloc(&k1, (size_t)nnz));
    ANCKA_TRY(ws.alloc(&k2, (size_t)nnz));
    // out-of-range node ids are replaced by 0 in the keys and reported with
    // the unique count below (one host read)
    k_hyper_to_keys<<<grid_for(m, 256), 256, 0, s>>>(t.he_ptr, t.he_nodes, m, n, nb, k0, bad);
    ANCKA_LAUNCHED();
    const int mb = bits_for(m);
    ANCKA_TRY(radix_sort_u64(ws, k0, k1, nnz, mb + nb, s));
    int64_t* ucnt_dev;
    ANCKA_TRY(ws.zeros(&ucnt_dev, 1));
    if (nnz > 0) ANCKA_TRY(unique_u64(ws, k1, k2, ucnt_dev, nnz, s));
    int64_t ucnt = 0;
    ANCKA_CUDA(cudaMemcpyAsync(&ucnt, ucnt_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    ANCKA_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    ANCKA_CUDA(cudaStreamSynchronize(s));
    if (hbad) {
      set_error("topology: node id out of range [0, n)");
      return ANCKA_ERR_INVALID_ARG;
    }
    int32_t* esize;
    ANCKA_TRY(keys_to_csr(ws, k2, ucnt, m, nb, &w->edges, &esize, s));
    // node -> hyperedge incidence
    k_swap_halves<<<grid_for(ucnt, 256), 256, 0, s>>>(k2, ucnt_dev, nb, mb, k0);
    ANCKA_LAUNCHED();
    ANCKA_TRY(radix_sort_u64(ws, k0, k1, ucnt, nb + mb, s));
    int32_t* vdeg;
    ANCKA_TRY(keys_to_csr(ws, k1, ucnt, n, mb, &w->topo, &vdeg, s));
    w->degree = vdeg;
    ANCKA_TRY(ws.alloc(&w->inv_size, (size_t)m));
    ANCKA_TRY(ws.alloc(&w->inv_deg, (size_t)n));
    k_inv_count<<<grid_for(m, 256), 256, 0, s>>>(esize, w->inv_size, m);
    ANCKA_LAUNCHED();
    k_inv_count<<<grid_for(n, 256), 256, 0, s>>>(vdeg, w->inv_deg, n);
    ANCKA_LAUNCHED();
  } else {
    const int L = t.L;
    std::vector<const int64_t*> lptr(L);
    std::vector<const int32_t*> lcol(L);
    std::vector<const int32_t*> ldeg(L);
    for (int l = 0; l < L; ++l) {
      const int64_t* rp = t.row_ptr + (int64_t)l * (n + 1);
      k_check_ptr<<<grid_for(n + 1, 256), 256, 0, s>>>(rp, n, t.nnz, bad);
      ANCKA_LAUNCHED();
      ANCKA_TRY(check_bad(bad, s, "row pointer of layer %d must be non-decreasing within [0, nnz]", l));
      int64_t b = 0, e = 0;
      ANCKA_CUDA(cudaMemcpyAsync(&b, rp, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      ANCKA_CUDA(cudaMemcpyAsync(&e, rp + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      ANCKA_CUDA(cudaStreamSynchronize(s));
      int64_t cnt = (e - b) * (t.directed ? 2 : 1);
      uint64_t *k0, *k1, *k2;
      ANCKA_TRY(ws.alloc(&k0, (size_t)cnt));
      ANCKA_TRY(ws.alloc(&k1, (size_t)cnt));
      ANCKA_TRY(ws.alloc(&k2, (size_t)cnt));
      int32_t* unsorted;
      ANCKA_TRY(ws.zeros(&unsorted, 1));
      k_csr_to_keys<<<grid_for(ceil_div(e - b, 32 * kPerLane) * 32, 256), 256, 0, s>>>(rp, t.col_idx, n, t.directed,
                                                                                      nb, k0, bad, unsorted);
      ANCKA_LAUNCHED();
      int32_t hu = 0;
      ANCKA_CUDA(cudaMemcpyAsync(&hu, unsorted, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      ANCKA_TRY(check_bad(bad, s, "topology: node id out of range [0, n)"));
      int64_t* ucnt_dev;
      ANCKA_TRY(ws.zeros(&ucnt_dev, 1));
      int64_t ucnt = 0;
      if (!t.directed && !hu) {  // rows already strictly increasing: the keys are sorted and unique
        k2 = k0;
        ucnt = cnt;
      } else {
        ANCKA_TRY(radix_sort_u64(ws, k0, k1, cnt, 2 * nb, s));
        if (cnt > 0) ANCKA_TRY(unique_u64(ws, k1, k2, ucnt_dev, cnt, s));
        ANCKA_TRY(read_count(ucnt_dev, &ucnt, s));
      }
      Csr lay;
      int32_t* deg;
      ANCKA_TRY(keys_to_csr(ws, k2, ucnt, n, nb, &lay, &deg, s));
      lptr[l] = lay.ptr;
      lcol[l] = lay.col;
      ldeg[l] = deg;
    }
    // merge layers
    const int64_t** dlptr;
    const int32_t** dlcol;
    const int32_t** dldeg;
    ANCKA_TRY(ws.alloc(&dlptr, (size_t)L));
    ANCKA_TRY(ws.alloc(&dlcol, (size_t)L));
    ANCKA_TRY(ws.alloc(&dldeg, (size_t)L));
    ANCKA_CUDA(cudaMemcpyAsync(dlptr, lptr.data(), L * sizeof(void*), cudaMemcpyHostToDevice, s));
    ANCKA_CUDA(cudaMemcpyAsync(dlcol, lcol.data(), L * sizeof(void*), cudaMemcpyHostToDevice, s));
    ANCKA_CUDA(cudaMemcpyAsync(dldeg, ldeg.data(), L * sizeof(void*), cudaMemcpyHostToDevice, s));
    int64_t* mlen;
    ANCKA_TRY(ws.alloc(&mlen, (size_t)n + 1));
    ANCKA_CUDA(cudaMemsetAsync(mlen + n, 0, sizeof(int64_t), s));
    ANCKA_TRY(ws.alloc(&w->degree, (size_t)n));
    k_sum_deg<<<grid_for(n, 256), 256, 0, s>>>(L, n, dldeg, w->degree, mlen);
    ANCKA_LAUNCHED();
    ANCKA_TRY(ws.alloc(&w->topo.ptr, (size_t)n + 1));
    ANCKA_TRY(exclusive_scan(ws, mlen, w->topo.ptr, n + 1, s));
    int64_t tot = 0;
    ANCKA_CUDA(cudaMemcpyAsync(&tot, w->topo.ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    ANCKA_CUDA(cudaStreamSynchronize(s));
    w->topo.nrows = n;
    w->topo.nnz = tot;
    ANCKA_TRY(ws.alloc(&w->topo.col, (size_t)tot));
    if (L == 1) {  // D^-1 A: a row scale and a column scale replace the per-entry values
      w->row_uniform = true;
      ANCKA_TRY(ws.alloc(&w->inv_deg, (size_t)n));
      k_inv_count<<<grid_for(n, 256), 256, 0, s>>>(w->degree, w->inv_deg, n);
      ANCKA_LAUNCHED();
    } else {
      ANCKA_TRY(ws.alloc(&w->topo.val, (size_t)tot));
      ANCKA_TRY(ws.alloc(&w->topo.valT, (size_t)tot));
    }
    k_merge_layers<<<grid_for(ceil_div(tot, 32 * kPerLane) * 32, 256), 256, 0, s>>>(L, n, dlptr, dlcol, dldeg, w->topo.ptr,
                                                    w->topo.col, w->topo.val, w->topo.valT);
    ANCKA_LAUNCHED();
  }
  return ANCKA_OK;
}

ancka_status build_knn_part(Workspace& ws, int64_t n, int32_t K, const int32_t* idx, const float* sim,
                            const int32_t* zero_row, float beta, Walk* w, cudaStream_t s) {
  const int64_t nk = n * K;
  uint8_t* mutual;
  uint64_t *keys, *skeys;
  int32_t* in_cnt;
  ANCKA_TRY(ws.alloc(&mutual, (size_t)nk));
  ANCKA_TRY(ws.alloc(&keys, (size_t)nk));
  ANCKA_TRY(ws.alloc(&skeys, (size_t)nk));
  ANCKA_TRY(ws.zeros(&in_cnt, (size_t)n));
  const int nb = bits_for(n);
  k_knn_mutual<<<grid_for(nk, 256), 256, 0, s>>>(idx, n, K, nb, mutual, keys, in_cnt);
  ANCKA_LAUNCHED();
  ANCKA_TRY(radix_sort_u64(ws, keys, skeys, nk, 2 * nb + 1, s));
  int64_t *len, *in_len, *in_start;
  ANCKA_TRY(ws.alloc(&len, (size_t)n + 1));
  ANCKA_TRY(ws.alloc(&in_len, (size_t)n + 1));
  ANCKA_TRY(ws.alloc(&in_start, (size_t)n + 1));
  ANCKA_CUDA(cudaMemsetAsync(len + n, 0, sizeof(int64_t), s));
  ANCKA_CUDA(cudaMemsetAsync(in_len + n, 0, sizeof(int64_t), s));
  k_knn_len<<<grid_for(n, 256), 256, 0, s>>>(in_cnt, n, K, len, in_len);
  ANCKA_LAUNCHED();
  Csr& c = w->knn;
  ANCKA_TRY(ws.alloc(&c.ptr, (size_t)n + 1));
  ANCKA_TRY(exclusive_scan(ws, len, c.ptr, n + 1, s));
  ANCKA_TRY(exclusive_scan(ws, in_len, in_start, n + 1, s));
  // a row holds its K out-neighbours and at most K in-neighbours per entry of
  // other lists, so n K + n K bounds the entries; the exact count (c.ptr[n])
  // stays on the device and nnz holds the bound
  const int64_t bound = 2 * nk;
  c.nrows = n;
  c.nnz = bound;
  ANCKA_TRY(ws.alloc(&c.col, (size_t)(bound > 0 ? bound : 1)));
  ANCKA_TRY(ws.alloc(&c.val, (size_t)(bound > 0 ? bound : 1)));
  ANCKA_TRY(ws.alloc(&w->beta, (size_t)n));
  k_knn_fill<<<grid_for(n * 32, 256), 256, 0, s>>>(idx, sim, mutual, skeys, in_start, in_cnt, n, K, c.ptr,
                                              c.col, c.val, zero_row, w->degree, beta, nb, w->beta);
  ANCKA_LAUNCHED();
  ANCKA_TRY(ws.alloc(&w->rs_topo, (size_t)n));
  k_topo_rowscale<<<grid_for(n, 256), 256, 0, s>>>(w->beta,
                                                   (w->kind == ANCKA_HYPERGRAPH || w->row_uniform) ? w->inv_deg
                                                                                                   : nullptr,
                                                   n, w->rs_topo);
  ANCKA_LAUNCHED();
  return ANCKA_OK;
}

}  // namespace ancka
