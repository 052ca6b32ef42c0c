/*
 * ancka.h -- C ABI of the GB300 (sm_103a) ANCKA hot path.
 *
 * ANCKA (attributed network clustering, arXiv 2408.05459) clusters the nodes
 * of an attributed graph, hypergraph or multiplex graph into k groups:
 *   1. KNN augmentation (Section 3.1, Eq. AK): for every node the K most
 *      cosine-similar other nodes by attributes, giving the KNN graph A_K and
 *      its walk matrix P_K = D_K^-1 A_K;
 *   2. the augmented walk P = (I - B) P_N + B P_K (Eq. p-mat-ancka) with P_N
 *      from Eq. rw-hg (hypergraph), rw-ag (graph) or rw-mg (multiplex) and
 *      B = diag(beta_i) (Eq. beta_i);
 *   3. Algorithm 4: InitBCM, T orthogonal iterations Z = P Q, QR, and every
 *      tau iterations Discretize (Def. 2, Alg. 5) + CalMHC (Alg. 2), keeping
 *      the labels with the lowest multi-hop conductance.
 *
 * Conventions for every entry point
 *   - Pointers are DEVICE pointers of the current CUDA device unless the
 *     function name ends in _host.  The caller owns every input and output
 *     buffer; the library allocates its own workspace with stream-ordered
 *     cudaMallocAsync on `stream` and frees it before returning.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *     Parts of a call with no data dependence on each other may run on the
 *     library's own streams (one set per device and host thread); each is
 *     joined back into `stream` before the outputs are written and before
 *     the workspace is released, so the outputs are ordered on `stream`.
 *   - Matrices are row-major and dense unless stated; int32 node ids.
 *   - Inputs are validated on the host before any launch; a bad argument
 *     returns ANCKA_ERR_INVALID_ARG and launches nothing.
 *   - When `info` is non-NULL the call synchronises `stream` before
 *     returning and fills it; with info == NULL the call only enqueues work.
 *   - No exceptions cross this interface; ancka_last_error() gives a
 *     human-readable message for the last failing call of this thread.
 *   - Requires a device of compute capability 10.3 (GB300); other devices
 *     give ANCKA_ERR_UNSUPPORTED.  There is no CPU fallback.
 */
#ifndef ANCKA_H_
#define ANCKA_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ANCKA_OK = 0,
  ANCKA_ERR_INVALID_ARG = 1,   /* argument out of range / inconsistent sizes */
  ANCKA_ERR_OOM = 2,           /* device workspace allocation failed */
  ANCKA_ERR_CUDA = 3,          /* a CUDA runtime call or kernel failed */
  ANCKA_ERR_NUMERIC = 4,       /* Cholesky of a singular Gram matrix (rank-deficient Z) */
  ANCKA_ERR_TIMEOUT = 5,       /* a bounded device-side wait expired */
  ANCKA_ERR_UNSUPPORTED = 6,   /* device is not sm_103 or option not available */
  ANCKA_ERR_INTERNAL = 7
} ancka_status;

/* Arithmetic of the KNN similarity contraction (step 1).  Every choice
 * returns the exact KNN lists of Section 3.1: candidates found in the low
 * precision are re-ranked with a compensated FP32 dot product and rows whose
 * candidate set cannot be certified are recomputed exhaustively. */
typedef enum {
  ANCKA_PREC_FP32 = 0,  /* CUDA-core FP32 contraction */
  ANCKA_PREC_BF16 = 1,  /* tcgen05 BF16 x BF16 -> FP32 (TMEM) contraction */
  ANCKA_PREC_FP8 = 2    /* tcgen05 FP8-E4M3 x E4M3 -> FP32 contraction (d <= 512); rows
                           it cannot certify are redone from BF16 candidates */
} ancka_prec;

typedef enum { ANCKA_GRAPH = 0, ANCKA_HYPERGRAPH = 1, ANCKA_MULTIPLEX = 2 } ancka_topo_kind;

/* Network topology N_O (Section 2).
 *   graph / multiplex: L adjacency layers in CSR form.  Layer l's row pointer
 *     is row_ptr + l*(n+1) (L*(n+1) int64 in total); its entries are
 *     col_idx[row_ptr[l*(n+1)+i] .. row_ptr[l*(n+1)+i+1]) with offsets into
 *     the single col_idx array (length nnz).  A graph has L = 1.  With
 *     directed = 0 each layer is read as an undirected adjacency (both
 *     directions present); with directed = 1 reversed edges are added
 *     (Eq. rw-ag).  Repeated entries count once (A is binary).
 *   hypergraph: m hyperedges, members of e at he_nodes[he_ptr[e] .. he_ptr[e+1])
 *     (nnz = he_ptr[m]); repeated members count once.
 * Node ids must lie in [0, n). */
typedef struct {
  int32_t kind;             /* ancka_topo_kind */
  int32_t L;                /* number of layers (graph: 1) */
  int64_t n;                /* number of nodes */
  const int64_t* row_ptr;   /* graph/multiplex: L*(n+1) */
  const int32_t* col_idx;   /* graph/multiplex: nnz */
  int64_t nnz;              /* graph/multiplex: length of col_idx */
  int32_t directed;         /* graph/multiplex: 1 = symmetrise */
  int32_t pad_;
  int64_t m;                /* hypergraph: number of hyperedges */
  const int64_t* he_ptr;    /* hypergraph: m+1 */
  const int32_t* he_nodes;  /* hypergraph: he_ptr[m] */
} ancka_topology;

/* Learned warm-start MLP (an addition to the paper's method; no counterpart
 * in the paper): W = GELU(A W1 + b1) W2 + b2 with A = [U | P_N U], U the unit
 * rows of X and P_N the topology walk of Eqs. rw-hg / rw-ag / rw-mg.  The
 * first layer runs on the tensor cores with BF16 operands and FP32
 * accumulation.  All pointers are device FP32, row-major, caller-owned. */
typedef struct {
  int32_t d_in;    /* 2 d (d = attribute columns) */
  int32_t hidden;  /* 256 (the only width this build supports) */
  int32_t k;       /* outputs: the number of clusters */
  int32_t pad_;
  float* W1;       /* d_in x hidden */
  float* b1;       /* hidden */
  float* W2;       /* hidden x k */
  float* b2;       /* k */
} ancka_warm_model;

/* Parameters of Algorithm 4 (defaults from the method's settings, Section 8.1). */
typedef struct {
  int32_t k;             /* clusters, 1 <= k <= 64 (default 5) */
  int32_t K;             /* KNN neighbours, 1 <= K <= 64, K < n (default 10) */
  float alpha;           /* walk stopping probability (0.2) */
  float beta;            /* KNN mixing weight of Eq. beta_i (0.5) */
  int32_t T;             /* orthogonal iterations T_a (10) */
  int32_t gamma;         /* CalMHC hops (3) */
  int32_t T_i;           /* InitBCM hops (25) */
  int32_t tau;           /* Discretize / CalMHC interval (5) */
  int32_t disc_max_iter; /* Discretize inner iterations (20) */
  int32_t knn_prec;      /* ancka_prec (ANCKA_PREC_BF16) */
  int32_t init;          /* 0 = InitBCM, 1 = labels in init_labels (device, n int32),
                            2 = learned warm start (warm), InitBCM as the fallback */
  int32_t pad_;
  const int32_t* init_labels;
  int32_t early_stop;    /* 1: stop by Eq. tcond-1 or Eq. tcond-2 at the Discretize
                            points (the paper's mode, T = T_a up to 1000); 0: run T (0) */
  float eps_Q;           /* Eq. tcond-1 threshold on ||Q(t) - Q(t-1)||_F (0.005) */
  const ancka_warm_model* warm;  /* init = 2: the MLP (device weights) */
  int32_t knn_nlist;     /* 0: exact KNN lists (default); > 0: approximate lists from
                            nlist inverted-list cells, as ancka_knn_ivf (BF16 only) */
  int32_t knn_nprobe;    /* cells probed per row when knn_nlist > 0 (1 <= nprobe <= min(32, nlist)) */
  int32_t node_order;    /* graphs and multiplex graphs: the order in which the iteration stores
                            the nodes (results are always in the caller's order).  0 (default):
                            descending degree when the n x (k+1) FP32 block exceeds 64 MiB,
                            else as given; 1: as given; 2: descending degree.  Algorithm 4 is
                            unchanged by the renaming (InitBCM's tie-break stays on the
                            caller's indices); only FP32 summation orders differ. */
} ancka_params;

/* Optional device outputs (any field may be NULL). */
typedef struct {
  float* Q;              /* n x (k+1) row-major: the final orthonormal block Q^(T) */
  int32_t* init_labels;  /* n: InitBCM labels Y^(0) */
  int32_t* knn_idx;      /* n x K: KNN lists */
  float* knn_sim;        /* n x K: their cosine similarities */
} ancka_outputs;

#define ANCKA_MAX_TRACE 64

/* Diagnostics filled when a non-NULL pointer is passed (the call then syncs). */
typedef struct {
  int64_t knn_candidates;      /* (row, candidate) pairs re-ranked exactly */
  int64_t knn_fallback_rows;   /* rows whose candidates could not be certified */
  int64_t knn_exhaustive_rows; /* of those, rows recomputed by an exhaustive exact scan */
  int32_t iters_run;           /* orthogonal iterations executed */
  int32_t n_phi;               /* entries of phi[] used: phi(Y0), then one per Discretize */
  double phi[ANCKA_MAX_TRACE];
  int32_t disc_iters[ANCKA_MAX_TRACE]; /* Discretize inner iterations per call */
  int32_t taken[ANCKA_MAX_TRACE];      /* 1 if that Discretize result became the kept Y */
  double phi_best;
  int32_t numeric_flags;       /* bit0: empty cluster seen in Discretize; bit1: SVD sweep limit hit */
  int32_t pad_;
  float ms_knn;                /* normalise + contraction + re-rank + fallback */
  float ms_build;              /* A_K, P_K, beta, P_N structures */
  float ms_init;               /* InitBCM + Q^(0) + phi(Y0) */
  float ms_iter;               /* SpMM + CholeskyQR2 over all iterations */
  float ms_disc;               /* all Discretize calls */
  float ms_mhc;                /* all CalMHC calls and the keep-best step */
  float ms_total;
  float ms_contract;           /* the candidate similarity contraction kernel alone */
  float ms_rerank;             /* exact re-rank, certificate and fallback after the contraction */
  float ms_spmm;               /* the T products Z = P Q of the orthogonal iteration (inside ms_iter) */
  int32_t warm_used;           /* init = 2: 1 if the warm start replaced InitBCM's (lower or equal Phi) */
  int32_t pad2_;
  int64_t knn_tiles;           /* approximate KNN: (query block, key tile) pairs multiplied */
  int64_t knn_full_tiles;      /* approximate KNN: the same for the exact sweep */
} ancka_info;

/* Fill *p with the defaults above. */
void ancka_params_default(ancka_params* p);

/* Static name of a status code. */
const char* ancka_status_str(ancka_status s);

/* Message of the last failing call on this host thread ("" if none). */
const char* ancka_last_error(void);

/* ANCKA_OK if the current device is an sm_103 part this library was built for. */
ancka_status ancka_device_check(void);

/* Number of this library's own CUDA kernels launched by the calling process
 * so far (a diagnostics counter; every kernel is the library's own, the sorts
 * and scans of the graph build included). */
int64_t ancka_kernel_launches(void);

/* Tuning (process-wide, thread-safe): BF16 KNN lists of inputs with at least
 * n_min rows come from the symmetric contraction, which multiplies only the
 * pairs j > i (Section 3.1: the cosine is symmetric) and pushes each score to
 * both rows through thresholds taken from a sampled pass; the lists, and so
 * ancka_knn's results, are the same as the full sweep's.  Smaller inputs use
 * the full sweep.  Default INT64_MAX (never: its appends still cost more than
 * the full sweep's list upkeep saves); n_min <= 1 selects the symmetric form
 * for every size.  FP32 and FP8 are not affected. */
void ancka_set_symmetric_knn_min_rows(int64_t n_min);

/* KNN lists of Section 3.1 (Eq. AK inputs).
 *   X        n x d FP32 attributes (device, row-major, any values; a zero row
 *            has similarity 0 to everything)
 *   out_idx  n x K int32: N_K(v_i) ordered by (cosine desc, index asc), i excluded
 *   out_sim  n x K FP32: the cosines, correctly rounded from a compensated
 *            (double-FP32) evaluation
 *   prec     ancka_prec of the candidate contraction: FP32 (CUDA cores), BF16
 *            or FP8-E4M3 (tensor cores, d <= 512).  The result is the same
 *            exact list for every precision; FP8 rows whose candidates cannot
 *            be certified are redone from BF16 candidates.
 * Requires 1 <= K <= 64, K < n, 1 <= d <= 4096, n < 2^31. */
ancka_status ancka_knn(const float* X, int64_t n, int32_t d, int32_t K, int32_t prec,
                       int32_t* out_idx, float* out_sim, ancka_info* info, void* stream);

/* Approximate KNN lists by inverted lists: the large-graph variant of the
 * paper's KNN construction (Section 7 builds the KNN graph with Faiss IVFPQ
 * when n >= 100k; here the codes are the BF16 unit rows themselves and the
 * final ranking is exact).  The unit rows are partitioned into nlist cells by
 * spherical k-means (8 rounds on min(n, 64 nlist) evenly spaced rows,
 * assignment by the tcgen05 BF16 contraction against the centroids, seeded
 * initial centroids), every row probes its nprobe nearest cells, the BF16
 * contraction scores it against the rows of the probed cells only (plus its
 * own 256-row key tile), and the 32 best candidates are re-ranked by their
 * exact FP32 cosine.  The lists are valid KNN lists (K distinct other rows,
 * ordered by cosine desc, index asc) but not necessarily the exact N_K: the
 * recall against ancka_knn is the quality measure.  Deterministic for fixed
 * inputs.
 *   X        n x d FP32 (device); d <= 512
 *   out_idx  n x K int32, out_sim n x K FP32 (device, caller-owned)
 *   info     may be NULL; fills ms_knn, knn_tiles and knn_full_tiles
 * Requires 1 <= K <= 16, K < n, 1 <= nlist <= min(n, 8192),
 * 1 <= nprobe <= min(32, nlist), n <= 16.7e6. */
ancka_status ancka_knn_ivf(const float* X, int64_t n, int32_t d, int32_t K, int32_t nlist, int32_t nprobe,
                           int32_t* out_idx, float* out_sim, ancka_info* info, void* stream);

/* Diagnostic, not part of the method: the candidate lists of the tensor-core
 * contraction before the exact re-rank, with the quantised copy and the error
 * model the certificate uses, so that the bounds can be checked against exact
 * arithmetic (Section 3.1 candidates; no counterpart in the paper).
 *   X         n x d FP32 (device); prec BF16 or FP8; d <= 512
 *   cand_val  n x 32 FP32 (device): row i's two 16-entry lists, entries
 *             [0, 16) for keys j with (j mod 256) < 128 and [16, 32) for the
 *             others; each list holds the 16 best low-precision scores of its
 *             keys (self excluded), in cosine units
 *   cand_idx  n x 32 int32 (device): their keys, -1 for an empty slot
 *   qrows     n x d FP32 (device) or NULL: the quantised unit rows q_i the
 *             contraction multiplied (FP8: codes divided by the scale)
 *   err       n FP32 (device) or NULL: e_i >= || q_i - x_i/||x_i|| ||_2
 *   acc       host, or NULL: the bound acc with
 *             |score_ij - q_i . q_j| <= acc ||q_i|| ||q_j||
 * All buffers are caller-owned. */
ancka_status ancka_knn_candidates(const float* X, int64_t n, int32_t d, int32_t prec, float* cand_val,
                                  int32_t* cand_idx, float* qrows, float* err, float* acc, void* stream);

/* Algorithm 4 end to end: labels[i] in [0, k) for every node.
 *   topo   topology with device pointers
 *   X      n x d FP32 attributes (device)
 *   labels n int32 output (device)
 *   out    optional extra outputs (device buffers), may be NULL */
ancka_status ancka_cluster(const ancka_topology* topo, const float* X, int32_t d,
                           const ancka_params* p, int32_t* labels, const ancka_outputs* out,
                           ancka_info* info, void* stream);

/* As ancka_cluster but with the KNN lists supplied (n x K int32 indices and
 * their FP32 cosines); X is still read for Eq. beta_i's zero-row test. */
ancka_status ancka_cluster_with_knn(const ancka_topology* topo, const float* X, int32_t d,
                                    const int32_t* knn_idx, const float* knn_sim,
                                    const ancka_params* p, int32_t* labels,
                                    const ancka_outputs* out, ancka_info* info, void* stream);

/* ancka_cluster on HOST buffers: topo, X and labels are host pointers (pinned
 * or pageable); the call copies inputs to the device, runs, copies labels
 * back and synchronises. `out` must be NULL. */
ancka_status ancka_cluster_host(const ancka_topology* topo, const float* X, int32_t d,
                                const ancka_params* p, int32_t* labels, ancka_info* info,
                                void* stream);

/* Discretize (Definition 2, Algorithm 5) of an n x k block.
 *   Qk      n x k FP32 with leading dimension ldq >= k (device)
 *   labels  n int32 output: the last Y of the alternation
 *   iters   host int32 out (may be NULL): inner iterations executed
 * R starts at I; stops when |obj - obj_prev| <= 4 eps max(1,|obj|) or after
 * max_iter iterations.  1 <= k <= 64.
 * Precision: M = Y~^T Q~ is summed in float-float (compensated FP32) and
 * rounded to FP32; the k x k polar factor R = V U^T is computed in FP32 by
 * the Newton-Schulz iteration (an FP32 one-sided Jacobi SVD when M is
 * rank-deficient or the iteration does not settle); tr(Omega) = tr(M R) and
 * obj are accumulated in FP64.  R feeds only the FP32 argmax of Q~ R, so no
 * part of the k x k work is carried out in FP64 arithmetic on GB300's narrow
 * FP64 pipe. */
ancka_status ancka_discretize(const float* Qk, int64_t n, int32_t k, int32_t ldq,
                              int32_t max_iter, int32_t* labels, int32_t* iters, void* stream);

/* Diagnostic: the k x k polar factor Discretize computes from
 * M = Y~^T Q~ (Alg. 5, Eq. svd-in-discr): R = V U^T for M = U Omega V^T,
 * by the same device routines (FP32 Newton-Schulz; FP32 Jacobi SVD when a
 * row of M is zero or the iteration does not settle), so that R can be
 * compared with an FP64 SVD.
 *   M       k x k FP32 row-major (device, caller-owned)
 *   R       k x k FP32 row-major output (device, caller-owned)
 *   method  host int32 out (may be NULL): 0 = Newton-Schulz, 1 = Jacobi;
 *           when non-NULL the call synchronises `stream`.
 * 1 <= k <= 64; ANCKA_ERR_INVALID_ARG otherwise. */
ancka_status ancka_polar_factor(const float* M, int32_t k, float* R, int32_t* method, void* stream);

/* Discretize exactly as ancka_discretize, but without allocating any device
 * memory (the paper has no counterpart: this serves callers that must not
 * allocate while they run -- code that reserves all memory at start-up,
 * programs whose device memory is owned by another allocator, loops that
 * avoid cudaMalloc/cudaFree because freeing synchronises the device).
 * Scratch comes from a fixed 32 MiB device array inside the library, held by
 * every GPU that loads it until exit; sizes needing more (about
 * n * round_up(k, 4) * 4 bytes plus small state) return
 * ANCKA_ERR_INVALID_ARG.  The first call on a device looks up that array's
 * device address (a runtime query, no allocation); make that first call
 * before any stream capture.  Every call waits for `stream` before it
 * returns, because it reads the inner-iteration count and an error flag back
 * to the host.  Calls share the array: calls that overlap on the GPU race.
 * Arguments as for ancka_discretize. */
ancka_status ancka_discretize_noalloc(const float* Qk, int64_t n, int32_t k, int32_t ldq,
                                      int32_t max_iter, int32_t* labels, int32_t* iters, void* stream);

/* Learned warm start: one training graph (device pointers).  The target is
 * ANCKA's own final block: Qt = columns 2..k+1 of Q^(T) (n x k, orthonormal
 * columns, row stride k), e.g. from ancka_cluster's outputs. */
typedef struct {
  const ancka_topology* topo;
  const float* X;   /* n x d attributes */
  const float* Qt;  /* n x k target block */
  int32_t d;
  int32_t pad_;
} ancka_warm_graph;

/* Trains the warm-start MLP in place: epochs x n_graphs full-graph steps (graph
 * order fixed) of Adam (lr; beta 0.9 / 0.999, eps 1e-8) on the loss
 *   L = k - tr(G^-1 M^T M) + lam ||G/n - I||_F^2,  G = W^T W, M = Qt^T W,
 * i.e. k - ||Qt^T orth(W)||_F^2 plus a scale penalty; it depends on W only
 * through span(W) and its scale.  model: initial weights in, trained weights
 * out (device FP32; d_in = 2d, hidden = 256, k as in the graphs).  losses:
 * host array of epochs * n_graphs values (the loss before each step), or
 * NULL.  Every graph needs the same d and k.  ANCKA_ERR_NUMERIC if some
 * W^T W is singular. */
ancka_status ancka_warm_train(const ancka_warm_graph* graphs, int32_t n_graphs, int32_t epochs, float lr, float lam,
                              ancka_warm_model* model, float* losses, void* stream);

/* W = MLP([U | P_N U]) (n x k, device, row stride k) for a topology and its
 * attributes. */
ancka_status ancka_warm_predict(const ancka_topology* topo, const float* X, int32_t d, const ancka_warm_model* model,
                                float* W, void* stream);

/* Diagnostic: the gradients of the training loss for one graph at the given
 * weights, without updating them (dW1 d_in x 256, db1 256, dW2 256 x k, db2 k,
 * device), and the loss (host, may be NULL). */
ancka_status ancka_warm_gradients(const ancka_warm_graph* graph, float lam, const ancka_warm_model* model,
                                  float* dW1, float* db1, float* dW2, float* db2, double* loss, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ANCKA_H_ */
