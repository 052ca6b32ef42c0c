"""FP64 CPU oracle for the ANCKA hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this module.  The CUDA
path never calls it and shares no code with it.

It restates, in plain numpy / scipy.sparse float64, what the paper defines:

* Section 3.1, Eq. (AK): cosine KNN augmentation graph A_K.
* Eq. (beta_i): per-node mixing weight beta_i.
* Eqs. (rw-hg), (rw-ag), (rw-mg): the topology walk matrix P_N; Eq.
  (p-mat-ancka): P = (I - B) P_N + B P_K.
* Algorithm 4 (ANCKA): InitBCM (Alg. 3, Eq. pi_c_t / argmaxlabel), the
  orthogonal iteration (Eq. ortho-iter / zt), Discretize (Def. 2, Eq. updateY,
  Eq. svd-in-discr, Alg. 5), CalMHC (Alg. 2, Eq. mhc-comp-ancka) and the
  keep-the-best rule.

Library routines serve as single steps (a dense or sparse matmul, a stable
sort, LAPACK QR / SVD); nothing is blocked, fused or reordered beyond what the
paper states.  Where the paper is silent the following readings are used
(each one is also listed in the design notes):

R1  cos(x, y) = 0 when either row is all-zero.
R2  K-nearest neighbours are ordered by (similarity desc, index asc); the node
    itself is excluded by index.
R3  a node whose KNN degree D_K[i] <= 0 gets a zero row in P_K and beta_i = 0.
R4  Q^(0) has k+1 columns; Discretize receives columns 2..k+1 of Q (the
    constant column is the known leading eigenvector).
R5  Discretize: R starts at I, max_iter = 20, the loop stops when
    |obj - obj_prev| <= 4 eps max(1, |obj|); Y~ divides each column of Y by its
    count (Alg. 5); a zero row of Q stays zero in the row-normalised Q~.
R6  argmax ties go to the lowest index (InitBCM, Discretize, labels).
R7  V_c: degree desc then id asc, k nodes, re-sorted by id; degree = number of
    neighbours (graph), incident hyperedges (hypergraph), summed over layers
    (multiplex).
R8  Phi(Y^(0)) is evaluated with CalMHC before the loop; a later Y replaces the
    kept one only if its Phi is strictly lower.
R9  fixed schedule: T iterations, Discretize + CalMHC when t mod tau == 0 and
    also at t == T; the early-termination tests (Eq. tcond-1/2) are used only
    when ``early_stop`` is set.
R10 QR: Householder (LAPACK) with the signs fixed so that diag(R) > 0.
R11 directed graph input is made symmetric and binary (A or A^T); repeated
    entries in an adjacency or a hyperedge count once; a node with no
    neighbours in a layer contributes a zero row for that layer.
R12 h(Y) = (Y^T Y)^{-1/2} Y with an empty cluster giving a zero column.
R13 Q^(0) = [n^{-1/2} 1 | h(Y^(0))] has rank k, not k+1: 1 = sum_c
    sqrt(|C_c|) h(Y)_c lies in the span of h(Y), and an empty cluster adds a
    zero column.  For the QR of Alg. 4 to be defined the dependent columns are
    replaced, keeping span(h(Y^(0))): the column of the highest-index
    non-empty cluster and the column of every empty cluster c become the sign
    vector s_i / sqrt(n), s_i = +1 or -1 from the top bit of
    splitmix64(64 i + c) (Steele, Lea, Flood 2014; Vigna's constants).

Learned warm start (an addition to the paper's method: an MLP predicts the
initial block instead of InitBCM; no counterpart in the paper):
W1  features A = [U | P_N U], U the unit rows of X (a zero row stays zero),
    P_N the topology walk of Eqs. (rw-hg), (rw-ag), (rw-mg) (no KNN part).
W2  MLP: W = GELU(A W1 + b1) W2 + b2 with GELU(z) = z Phi(z) (Phi the standard
    normal CDF, erf form).  The two large operands of the first layer (A and
    W1, and A^T and dZ1 in its weight gradient) are BF16 with FP32
    accumulation; ``bf16=True`` rounds exactly those operands (round to
    nearest even), everything else is FP64.
W3  loss L = k - tr(G^-1 M^T M) + lam ||G/n - I||_F^2 with G = W^T W and
    M = Q_t^T W for the target's k orthonormal columns Q_t; the first term is
    k - ||Q_t^T orth(W)||_F^2 for any orthonormal basis orth(W) of span(W)
    (CholeskyQR's included), so L depends on W only through its span and
    scale; dL/dW = -2 (Q_t M G^-1 - W S) + (4 lam / n) W (G/n - I) with
    S = G^-1 M^T M G^-1.
W4  Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected), one full-graph
    step per training graph in a fixed order, epochs repeated.
W5  the initial weights are inputs (drawn by the seeded input generators).
W6  the warm block is Q^(0) = QR([n^-1/2 1 | W]) with diag(R) > 0 and
    Y^(0) = Discretize(Q^(0)[:, 1:]); it replaces InitBCM's start only when
    Phi(Y^(0)) is not higher than InitBCM's (otherwise InitBCM is the fallback).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

F64 = np.float64
EPS = np.finfo(F64).eps

DEFAULTS = dict(k=5, K=10, alpha=0.2, beta=0.5, T=10, gamma=3, T_i=25, tau=5,
                disc_max_iter=20, eps_Q=0.005, early_stop=False)


# ----------------------------------------------------------------------------
# Section 3.1: cosine similarity and the KNN augmentation graph
# ----------------------------------------------------------------------------
def unit_rows(X):
    """Rows of X scaled to unit 2-norm; zero rows stay zero (reading R1)."""
    X = np.asarray(X, dtype=F64)
    nrm = np.sqrt(np.einsum("ij,ij->i", X, X))
    inv = np.zeros_like(nrm)
    nz = nrm > 0
    inv[nz] = 1.0 / nrm[nz]
    return X * inv[:, None]


def cosine(X, i, j):
    """f(v_i, v_j) = cos(X[i], X[j]) of Section 3.1 for one pair (reading R1)."""
    X = np.asarray(X, dtype=F64)
    a, b = X[i], X[j]
    na, nb = np.sqrt(a @ a), np.sqrt(b @ b)
    if na == 0 or nb == 0:
        return 0.0
    return float(a @ b) / (na * nb)


def knn_cosine(X, K, rows=None, chunk=256, extra=1):
    """N_K(v_i) of Section 3.1 for every (or every listed) row i.

    Returns ``idx`` (len(rows) x K, int64) and ``sim`` (len(rows) x (K+extra)):
    the similarities of the first K+extra entries of the (sim desc, index asc)
    order over V \\ {v_i} (readings R1, R2), so callers can see the gap
    between the K-th and (K+1)-th neighbour.
    """
    Xn = unit_rows(X)
    n = Xn.shape[0]
    if not 1 <= K <= n - 1:
        raise ValueError("need 1 <= K <= n-1")
    rows = np.arange(n) if rows is None else np.asarray(rows, np.int64)
    kk = min(K + extra, n - 1)
    idx = np.empty((rows.size, K), np.int64)
    sim = np.full((rows.size, K + extra), -np.inf)
    for s in range(0, rows.size, chunk):
        r = rows[s:s + chunk]
        S = Xn[r] @ Xn.T
        S[np.arange(r.size), r] = -np.inf  # v_i itself is not a candidate
        order = np.argsort(-S, axis=1, kind="stable")[:, :kk]
        idx[s:s + r.size] = order[:, :K]
        sim[s:s + r.size, :kk] = np.take_along_axis(S, order, axis=1)
    return idx, sim


def knn_adjacency(X, idx):
    """A_K of Eq. (AK) from the KNN lists.

    A_K[i,j] = 2 f(i,j) if i and j are in each other's list, f(i,j) if only one
    of them is, 0 otherwise.  f is evaluated once per unordered pair.
    """
    Xn = unit_rows(X)
    n, K = idx.shape
    src = np.repeat(np.arange(n, dtype=np.int64), K)
    dst = np.asarray(idx, np.int64).ravel()
    # membership count of the unordered pair {i, j}: 1 = one-sided, 2 = mutual
    lo, hi = np.minimum(src, dst), np.maximum(src, dst)
    key, count = np.unique(lo * n + hi, return_counts=True)
    a, b = key // n, key % n
    f = np.empty(a.size)
    for s in range(0, a.size, 1 << 18):       # pairs in chunks; each dot product is unchanged
        e = min(a.size, s + (1 << 18))
        f[s:e] = np.einsum("ij,ij->i", Xn[a[s:e]], Xn[b[s:e]])
    w = count * f
    A = sp.coo_matrix((np.concatenate([w, w]), (np.concatenate([a, b]), np.concatenate([b, a]))),
                      shape=(n, n)).tocsr()
    A.sum_duplicates()
    return A


def knn_transition(A_K):
    """P_K = D_K^{-1} A_K (Alg. 4 line 1); rows with D_K <= 0 become zero (R3)."""
    D = np.asarray(A_K.sum(axis=1)).ravel()
    inv = np.zeros_like(D)
    pos = D > 0
    inv[pos] = 1.0 / D[pos]
    return sp.diags(inv) @ A_K, D


# ----------------------------------------------------------------------------
# Section 6.1: the topology walk P_N
# ----------------------------------------------------------------------------
def adjacency_from_csr(n, row_ptr, col, directed=False):
    """Binary adjacency matrix A; a directed input is made symmetric (R11)."""
    row_ptr = np.asarray(row_ptr, np.int64)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    A = sp.coo_matrix((np.ones(rows.size), (rows, np.asarray(col, np.int64))), shape=(n, n)).tocsr()
    if directed:
        A = A + A.T
    A.data[:] = 1.0  # repeated entries count once (binary A)
    A.eliminate_zeros()
    return A


def incidence_from_csr(n, he_ptr, he_nodes):
    """Binary incidence H (m x n) with H[e, v] = 1 iff v in e (Section 2)."""
    he_ptr = np.asarray(he_ptr, np.int64)
    m = he_ptr.size - 1
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(he_ptr))
    H = sp.coo_matrix((np.ones(rows.size), (rows, np.asarray(he_nodes, np.int64))), shape=(m, n)).tocsr()
    H.data[:] = 1.0
    return H


def spmm_rows(M, Q, blocks=32):
    """M @ Q for a CSR matrix M and a dense Q, by row blocks in a thread pool:
    every row of the result is the same sum, in the same order, as in M @ Q
    (scipy releases the GIL inside the product)."""
    n = M.shape[0]
    if n < 100_000:
        return M @ Q
    from concurrent.futures import ThreadPoolExecutor
    b = np.linspace(0, n, blocks + 1).astype(np.int64)
    out = np.empty((n,) + Q.shape[1:], dtype=np.result_type(M.dtype, Q.dtype))
    def run(i):
        out[b[i]:b[i + 1]] = M[b[i]:b[i + 1]] @ Q
    with ThreadPoolExecutor(min(blocks, 16)) as ex:
        list(ex.map(run, range(blocks)))
    return out


def _inv_or_zero(v):
    out = np.zeros_like(v, dtype=F64)
    nz = v > 0
    out[nz] = 1.0 / v[nz]
    return out


class Topology:
    """P_N of Eqs. (rw-hg), (rw-ag), (rw-mg) kept in factored form.

    ``apply(Q)`` returns P_N Q and ``apply_T(Q)`` returns P_N^T Q, each as the
    paper orders the products (the hypergraph form never builds P_V P_E).
    ``degree`` is delta(v) (reading R7).
    """

    def __init__(self, topo: dict):
        self.kind = topo["kind"]
        n = self.n = int(topo["n"])
        if self.kind == "hypergraph":
            H = incidence_from_csr(n, topo["he_ptr"], topo["he_nodes"])
            dV = np.asarray(H.sum(axis=0)).ravel()   # delta(v): incident hyperedges
            dE = np.asarray(H.sum(axis=1)).ravel()   # |e|
            self.P_V = sp.diags(_inv_or_zero(dV)) @ H.T.tocsr()   # D_V^{-1} H^T
            self.P_E = sp.diags(_inv_or_zero(dE)) @ H              # D_E^{-1} H
            self.degree = dV
        elif self.kind in ("graph", "multiplex"):
            layers = topo["layers"]
            directed = bool(topo.get("directed", False))
            mats, deg = [], np.zeros(n)
            for row_ptr, col in layers:
                A = adjacency_from_csr(n, row_ptr, col, directed)
                d = np.asarray(A.sum(axis=1)).ravel()
                deg += d
                mats.append(sp.diags(_inv_or_zero(d)) @ A)        # D_l^{-1} A_l
            L = len(mats)
            PN = mats[0]
            for M in mats[1:]:
                PN = PN + M
            self.P_N = (PN * (1.0 / L)).tocsr() if L > 1 else PN.tocsr()
            self.degree = deg
        else:
            raise ValueError(self.kind)

    def apply(self, Q):
        if self.kind == "hypergraph":
            return spmm_rows(self.P_V, spmm_rows(self.P_E, Q))   # Eq. (zt): P_V (P_E Q)
        return spmm_rows(self.P_N, Q)

    def apply_T(self, Q):
        if self.kind == "hypergraph":
            return self.P_E.T @ (self.P_V.T @ Q)      # (Pi P_V) P_E, transposed
        return self.P_N.T @ Q

    def dense(self):
        if self.kind == "hypergraph":
            return (self.P_V @ self.P_E).toarray()
        return self.P_N.toarray()


def beta_vector(X, degree, beta, D_K):
    """beta_i of Eq. (beta_i) with reading R3 for a non-positive KNN degree."""
    X = np.asarray(X, F64)
    zero_row = ~np.any(X != 0, axis=1)
    b = np.full(X.shape[0], float(beta))
    b[degree == 0] = 1.0
    b[zero_row] = 0.0
    b[D_K <= 0] = 0.0
    return b


class WalkOperator:
    """P = (I - B) P_N + B P_K of Eq. (p-mat-ancka), applied as Eq. (zt)."""

    def __init__(self, topo: Topology, P_K, b):
        self.topo, self.P_K, self.b = topo, P_K, b

    def apply(self, Q):
        return (1.0 - self.b)[:, None] * self.topo.apply(Q) + self.b[:, None] * spmm_rows(self.P_K, Q)

    def dense(self):
        return (1.0 - self.b)[:, None] * self.topo.dense() + self.b[:, None] * self.P_K.toarray()


# ----------------------------------------------------------------------------
# Section 4: BCM matrices
# ----------------------------------------------------------------------------
def bcm(labels, k):
    """Binary cluster membership Y of Eq. (y)."""
    n = labels.size
    Y = np.zeros((n, k))
    Y[np.arange(n), labels] = 1.0
    return Y


def h_norm(labels, k):
    """h(Y) = (Y^T Y)^{-1/2} Y of Eq. (norm-y); empty cluster -> zero column (R12)."""
    c = np.bincount(labels, minlength=k).astype(F64)
    Y = bcm(labels, k)
    return Y * _inv_sqrt_or_zero(c)[None, :]


def _inv_sqrt_or_zero(c):
    out = np.zeros_like(c)
    nz = c > 0
    out[nz] = 1.0 / np.sqrt(c[nz])
    return out


def splitmix64(x):
    """One output of the splitmix64 generator for state x (uint64 array)."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, np.uint64) + np.uint64(0x9E3779B97F4A7C15))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def initial_block(labels, k):
    """Q^(0) = [n^{-1/2} 1 | h(Y^(0))] (Alg. 4 line 12) with reading R13."""
    n = labels.size
    Q = np.concatenate([np.full((n, 1), 1.0 / np.sqrt(n)), h_norm(labels, k)], axis=1)
    counts = np.bincount(labels, minlength=k)
    dependent = list(np.nonzero(counts == 0)[0]) + [int(np.nonzero(counts > 0)[0].max())]
    for c in dependent:
        bits = splitmix64(np.arange(n, dtype=np.uint64) * np.uint64(64) + np.uint64(c)) >> np.uint64(63)
        Q[:, 1 + c] = np.where(bits == 1, -1.0, 1.0) / np.sqrt(n)
    return Q


def argmax_rows(M):
    """Row argmax with ties to the lowest column (R6); np.argmax does that."""
    return np.argmax(M, axis=1).astype(np.int64)


# ----------------------------------------------------------------------------
# Algorithm 4, lines 3-11: InitBCM
# ----------------------------------------------------------------------------
def centre_nodes(degree, k):
    """V_c: the k largest-degree nodes (degree desc, id asc), sorted by id (R7)."""
    order = np.lexsort((np.arange(degree.size), -degree))
    return np.sort(order[:k])


def init_bcm(topo: Topology, k, alpha, T_i):
    """Pi^(t) = (1 - alpha) Pi^(t-1) P_N + alpha Z_0; g(v) = argmax_l Pi[l, v].

    Pi is k x n; it is carried transposed (n x k) so Pi P_N becomes P_N^T Pi^T.
    Returns (labels, V_c, Pi^T).
    """
    n = topo.n
    Vc = centre_nodes(topo.degree, k)
    Z0T = np.zeros((n, k))
    Z0T[Vc, np.arange(k)] = 1.0
    Pi0 = alpha * Z0T
    Pi = Pi0.copy()
    for _ in range(T_i):
        Pi = (1.0 - alpha) * topo.apply_T(Pi) + Pi0
    return argmax_rows(Pi), Vc, Pi


# ----------------------------------------------------------------------------
# Algorithm 1 / 4: QR step and Discretize
# ----------------------------------------------------------------------------
def qr_pos(Z):
    """Householder QR (LAPACK) with diag(R) > 0 (reading R10)."""
    Q, R = np.linalg.qr(Z)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s[None, :], R * s[:, None]


def discretize(Qk, max_iter=20, return_trace=False):
    """Discretize of Definition 2 / Algorithm 5 (readings R5, R6).

    Qk is n x k (the eigenvector block without the constant column).
    Returns the last labels Y (as an int vector) and, optionally, the trace of
    objective values and the final rotation.
    """
    Qk = np.asarray(Qk, F64)
    n, k = Qk.shape
    nrm = np.sqrt(np.einsum("ij,ij->i", Qk, Qk))
    Qt = Qk * _inv_or_zero(nrm)[:, None]             # row-normalised Q~
    R = np.eye(k)
    obj_prev = None
    objs = []
    labels = None
    for _ in range(max_iter):
        labels = argmax_rows(Qt @ R)                 # Eq. (updateY)
        c = np.bincount(labels, minlength=k).astype(F64)
        Yt = bcm(labels, k) * _inv_or_zero(c)[None, :]   # column-normalised Y~
        M = Yt.T @ Qt                                # Y~^T Q~  (k x k)
        U, Om, Vt = np.linalg.svd(M)                 # Eq. (svd-in-discr)
        R = Vt.T @ U.T                               # R = V U^T
        obj = n - 2.0 * Om.sum()
        objs.append(obj)
        if obj_prev is not None and abs(obj - obj_prev) <= 4 * EPS * max(1.0, abs(obj)):
            break
        obj_prev = obj
    if return_trace:
        return labels, objs, R
    return labels


# ----------------------------------------------------------------------------
# Algorithm 2 / Eq. (mhc-comp-ancka): multi-hop conductance
# ----------------------------------------------------------------------------
def cal_mhc(P: WalkOperator, labels, k, alpha, gamma):
    """phi = 1 - (1/k) tr(Yh^T F^(gamma)), F^(l) = (1-alpha) P F^(l-1) + F^(0)."""
    Yh = h_norm(labels, k)
    F0 = alpha * Yh
    F = F0
    for _ in range(gamma):
        F = (1.0 - alpha) * P.apply(F) + F0
    return 1.0 - np.einsum("ij,ij->", Yh, F) / k


def mhc_from_definition(S_dense, labels, k):
    """Phi of Eq. (mh-cond) evaluated from a dense S (small n only)."""
    total = 0.0
    for c in range(k):
        members = np.nonzero(labels == c)[0]
        if members.size == 0:
            continue
        outside = np.ones(labels.size, bool)
        outside[members] = False
        total += S_dense[np.ix_(members, outside)].sum() / members.size
    return total / k


def multi_hop_dense(P_dense, alpha, gamma):
    """S = alpha sum_{l=0..gamma} (1 - alpha)^l P^l of Eq. (approx-multi-hop)."""
    n = P_dense.shape[0]
    S = np.zeros((n, n))
    Pl = np.eye(n)
    for l in range(gamma + 1):
        S += alpha * (1.0 - alpha) ** l * Pl
        Pl = Pl @ P_dense
    return S


# ----------------------------------------------------------------------------
# Algorithm 4 end to end
# ----------------------------------------------------------------------------
def build_walk(topo_dict, X, K, beta, knn=None):
    """Alg. 4 lines 1-2: P_K from the KNN lists and P_N from the topology."""
    topo = Topology(topo_dict)
    if knn is None:
        idx, _ = knn_cosine(X, K)
    else:
        idx = np.asarray(knn, np.int64)
    A_K = knn_adjacency(X, idx)
    P_K, D_K = knn_transition(A_K)
    b = beta_vector(X, topo.degree, beta, D_K)
    return WalkOperator(topo, P_K, b), idx


def ancka(topo_dict, X, params=None, knn=None, init_labels=None, warm=None, warm_bf16=True, timings=None):
    """Algorithm 4 (ANCKA) in FP64 with the fixed schedule of reading R9.

    ``warm``: MLP weights (W1, b1, W2, b2) for the learned warm start of
    readings W1-W6.  ``timings``: an optional dict that receives the wall
    time (s) of each phase -- "build" (P_K, beta, P_N), "init" (InitBCM,
    Phi(Y0), Q0, the warm start), "iter" (the products and QR), "disc"
    (Discretize), "mhc" (CalMHC in the loop); it does not change the
    arithmetic.  Returns a dict with the labels, the final Q (n x (k+1)), the
    InitBCM labels, the phi trace and the Discretize inner-iteration counts.
    """
    from time import perf_counter
    tm = {} if timings is None else timings
    for key in ("build", "init", "iter", "disc", "mhc"):
        tm.setdefault(key, 0.0)
    p = dict(DEFAULTS)
    if params:
        p.update(params)
    k, alpha, T, tau, gamma = p["k"], p["alpha"], p["T"], p["tau"], p["gamma"]
    t0 = perf_counter()
    P, idx = build_walk(topo_dict, X, p["K"], p["beta"], knn)
    tm["build"] += perf_counter() - t0
    t0 = perf_counter()
    n = P.topo.n
    if init_labels is None:
        y0, Vc, _ = init_bcm(P.topo, k, alpha, p["T_i"])
    else:
        y0, Vc = np.asarray(init_labels, np.int64), None
    Y_best = y0.copy()
    phi_best = cal_mhc(P, y0, k, alpha, gamma)       # reading R8
    Q = initial_block(y0, k)
    warm_used = False
    if warm is not None:                              # reading W6
        Wm, _ = warm_forward(warm_features(P.topo, X), warm, warm_bf16)
        Q_w = warm_initial_block(Wm)
        y_w = discretize(Q_w[:, 1:], p["disc_max_iter"])
        phi_w = cal_mhc(P, y_w, k, alpha, gamma)
        if phi_w <= phi_best:
            Q, y0, Y_best, phi_best, warm_used = Q_w, y_w, y_w.copy(), phi_w, True
    tm["init"] += perf_counter() - t0
    phis = [phi_best]
    disc_iters = []
    taken = []
    t_run = 0
    for t in range(1, T + 1):
        Q_prev = Q
        t0 = perf_counter()
        Z = P.apply(Q)                                # Eq. (zt)
        Q, _ = qr_pos(Z)
        tm["iter"] += perf_counter() - t0
        t_run = t
        if t % tau == 0 or t == T:
            t0 = perf_counter()
            y_t, objs, _ = discretize(Q[:, 1:], p["disc_max_iter"], return_trace=True)
            tm["disc"] += perf_counter() - t0
            disc_iters.append(len(objs))
            t0 = perf_counter()
            phi_t = cal_mhc(P, y_t, k, alpha, gamma)
            tm["mhc"] += perf_counter() - t0
            phis.append(phi_t)
            take = phi_t < phi_best
            taken.append(bool(take))
            if take:
                Y_best, phi_best = y_t, phi_t
            if p["early_stop"]:
                conv = np.linalg.norm(Q - Q_prev) < p["eps_Q"]          # Eq. (tcond-1)
                rising = len(phis) >= 3 and phis[-3] < phis[-2] < phis[-1]  # Eq. (tcond-2)
                if conv or rising:
                    break
    return dict(labels=Y_best.astype(np.int64), Q=Q, init_labels=y0, centres=Vc,
                phi=np.array(phis), phi_best=phi_best, disc_iters=disc_iters,
                taken=taken, iters=t_run, knn_idx=idx, warm_used=warm_used)


# ----------------------------------------------------------------------------
# learned warm start (readings W1-W6)
# ----------------------------------------------------------------------------
def round_bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(a, np.float64).astype(np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(F64)


def warm_features(topo: Topology, X):
    """Reading W1: A = [U | P_N U]."""
    U = unit_rows(X)
    return np.hstack([U, topo.apply(U)])


def gelu(z):
    from scipy.special import erf
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def warm_forward(A, prm, bf16=False):
    """Reading W2: returns W and the cache (Z1, H) for the backward pass."""
    Ab = round_bf16(A) if bf16 else np.asarray(A, F64)
    W1 = round_bf16(prm["W1"]) if bf16 else prm["W1"]
    Z1 = Ab @ W1 + prm["b1"]
    H = gelu(Z1)
    W = H @ prm["W2"] + prm["b2"]
    return W, (Z1, H)


def warm_loss(W, Qt, lam):
    """Reading W3."""
    n, k = W.shape
    G = W.T @ W
    M = Qt.T @ W
    f = np.trace(np.linalg.solve(G, M.T @ M))
    return float(k - f + lam * np.sum((G / n - np.eye(k)) ** 2))


def warm_loss_grad(W, Qt, lam):
    """Reading W3: dL/dW in closed form."""
    n, k = W.shape
    G = W.T @ W
    M = Qt.T @ W
    Gi = np.linalg.inv(G)
    S = Gi @ M.T @ M @ Gi
    return -2.0 * (Qt @ M @ Gi - W @ S) + (4.0 * lam / n) * W @ (G / n - np.eye(k))


def warm_backward(A, prm, cache, dW, bf16=False):
    """Gradients of the loss w.r.t. W1, b1, W2, b2 given dL/dW."""
    Z1, H = cache
    g = {"W2": H.T @ dW, "b2": dW.sum(axis=0)}
    dH = dW @ prm["W2"].T
    dZ1 = dH * gelu_grad(Z1)
    g["b1"] = dZ1.sum(axis=0)
    if bf16:
        g["W1"] = round_bf16(A).T @ round_bf16(dZ1)
    else:
        g["W1"] = np.asarray(A, F64).T @ dZ1
    return g


def adam_step(prm, grads, state, lr, b1=0.9, b2=0.999, eps=1e-8):
    """Reading W4: one bias-corrected Adam update of every tensor in prm."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    out = {}
    for name, p in prm.items():
        m = state.setdefault("m_" + name, np.zeros_like(p))
        v = state.setdefault("v_" + name, np.zeros_like(p))
        m[...] = b1 * m + (1.0 - b1) * grads[name]
        v[...] = b2 * v + (1.0 - b2) * grads[name] ** 2
        mh = m / (1.0 - b1 ** t)
        vh = v / (1.0 - b2 ** t)
        out[name] = p - lr * mh / (np.sqrt(vh) + eps)
    return out


def warm_train(data, prm, epochs, lr=1e-3, lam=1e-3, bf16=False):
    """Reading W4: data = [(A_g, Qt_g)], one step per graph per epoch."""
    prm = {k_: np.array(v, F64) for k_, v in prm.items()}
    state, losses = {}, []
    for _ in range(epochs):
        for A, Qt in data:
            W, cache = warm_forward(A, prm, bf16)
            losses.append(warm_loss(W, Qt, lam))
            grads = warm_backward(A, prm, cache, warm_loss_grad(W, Qt, lam), bf16)
            prm = adam_step(prm, grads, state, lr)
    return prm, losses


def warm_initial_block(W):
    """Reading W6: Q^(0) = QR([n^-1/2 1 | W]) with diag(R) > 0."""
    n = W.shape[0]
    Q, _ = qr_pos(np.hstack([np.full((n, 1), 1.0 / np.sqrt(n)), W]))
    return Q


# ----------------------------------------------------------------------------
# evaluation helpers
# ----------------------------------------------------------------------------
def adjusted_rand_index(a, b):
    """Hubert-Arabie adjusted Rand index of two labelings."""
    a = np.asarray(a, np.int64)
    b = np.asarray(b, np.int64)
    _, ai = np.unique(a, return_inverse=True)
    _, bi = np.unique(b, return_inverse=True)
    C = sp.coo_matrix((np.ones(a.size), (ai, bi))).toarray()

    def comb2(x):
        return x * (x - 1) / 2.0

    s_ij = comb2(C).sum()
    s_a = comb2(C.sum(axis=1)).sum()
    s_b = comb2(C.sum(axis=0)).sum()
    total = comb2(float(a.size))
    expected = s_a * s_b / total if total > 0 else 0.0
    max_idx = 0.5 * (s_a + s_b)
    if max_idx == expected:
        return 1.0
    return (s_ij - expected) / (max_idx - expected)


def max_principal_angle(A, B):
    """Largest principal angle between span(A) and span(B) (arcsin form)."""
    Qa, _ = np.linalg.qr(np.asarray(A, F64))
    Qb, _ = np.linalg.qr(np.asarray(B, F64))
    resid = Qb - Qa @ (Qa.T @ Qb)
    s = np.linalg.norm(resid, 2)
    return float(np.arcsin(min(1.0, s)))
