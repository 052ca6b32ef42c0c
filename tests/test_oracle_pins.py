"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's own formula: each compares it with a
printed value (Figure 1 example), an exhaustive enumeration on a tiny input, a
closed form, an invariant, or an independent textbook / library routine.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import ancka_oracle as O
from paper_2408_05459_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# Section 3.1: KNN
# ----------------------------------------------------------------------------
def test_fig1_example_excludes_v7():
    g = json.load(open(os.path.join(GOLDEN, "fig1_knn_example.json")))
    X = np.array(g["X"])
    q = g["query_node"]
    for j, f in g["printed_similarities_to_query"].items():
        assert abs(O.cosine(X, q, int(j)) - f) < 1e-12
    idx, sim = O.knn_cosine(X, g["K"], rows=[q])
    assert sorted(idx[0].tolist()) == g["expected_knn_set"]
    assert g["excluded_node"] not in idx[0]
    # the next neighbour (K+1) is v7 with 0.41
    idx4, _ = O.knn_cosine(X, g["K"] + 1, rows=[q])
    assert idx4[0, -1] == g["excluded_node"]


def _fsum_cos(X, i, j):
    a, b = X[i].tolist(), X[j].tolist()
    na = math.sqrt(math.fsum(x * x for x in a))
    nb = math.sqrt(math.fsum(x * x for x in b))
    if na == 0 or nb == 0:
        return 0.0
    return math.fsum(x * y for x, y in zip(a, b)) / (na * nb)


def test_knn_exhaustive_property_small():
    rng = np.random.default_rng(3)
    n, d, K = 28, 5, 6
    X = rng.standard_normal((n, d))
    X[5] = 0.0                    # a zero row: all its similarities are 0
    X[9] = X[4] * 3.0             # a scaled duplicate: similarity 1 ties
    X[11] = X[4]
    idx, _ = O.knn_cosine(X, K)
    S = np.array([[_fsum_cos(X, i, j) for j in range(n)] for i in range(n)])
    for i in range(n):
        chosen = set(idx[i].tolist())
        assert i not in chosen and len(chosen) == K
        # exhaustive check of the (sim desc, index asc) definition
        for j in chosen:
            for jj in range(n):
                if jj == i or jj in chosen:
                    continue
                better = S[i, j] > S[i, jj] + 1e-12 or (abs(S[i, j] - S[i, jj]) <= 1e-12 and j < jj)
                assert better, (i, j, jj)
        # the list itself is ordered
        for a, b in zip(idx[i][:-1], idx[i][1:]):
            assert S[i, a] > S[i, b] + 1e-12 or (abs(S[i, a] - S[i, b]) <= 1e-12 and a < b)
    # zero row: neighbours are the K lowest other indices (all tie at 0)
    assert idx[5].tolist() == [j for j in range(n) if j != 5][:K]


def test_knn_invariant_to_positive_row_scaling():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((60, 7))
    scale = rng.uniform(0.1, 10.0, size=(60, 1))
    a, _ = O.knn_cosine(X, 5)
    b, _ = O.knn_cosine(X * scale, 5)
    assert np.array_equal(a, b)


def test_knn_permutation_equivariance():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((50, 6))
    perm = rng.permutation(50)
    a, _ = O.knn_cosine(X, 4)
    Xp = np.empty_like(X)
    Xp[perm] = X
    b, _ = O.knn_cosine(Xp, 4)
    assert np.array_equal(perm[a], b[perm])


def test_knn_adjacency_entries_enumerated():
    rng = np.random.default_rng(6)
    n, K = 25, 4
    X = rng.standard_normal((n, 3))
    idx, _ = O.knn_cosine(X, K)
    A = O.knn_adjacency(X, idx).toarray()
    lists = [set(r.tolist()) for r in idx]
    nnz = 0
    for i in range(n):
        for j in range(n):
            f = _fsum_cos(X, i, j)
            in_i, in_j = j in lists[i], i in lists[j]
            want = 2 * f if (in_i and in_j) else (f if (in_i or in_j) else 0.0)
            assert abs(A[i, j] - want) < 1e-12
            nnz += (in_i or in_j)
    assert np.allclose(A, A.T)
    assert n * K <= nnz <= 2 * n * K


# ----------------------------------------------------------------------------
# Section 6.1: walk matrices
# ----------------------------------------------------------------------------
def _tiny_hypergraph():
    # 7 nodes, hyperedges from the Figure 1 example (e1, e2) plus three more
    edges = [[0, 1, 3, 4], [0, 2, 3], [5, 6], [2, 5, 6], [1, 4]]
    he_ptr = np.concatenate([[0], np.cumsum([len(e) for e in edges])]).astype(np.int64)
    he_nodes = np.array(sum(edges, []), np.int32)
    return dict(kind="hypergraph", n=7, he_ptr=he_ptr, he_nodes=he_nodes), edges


def test_hypergraph_walk_matches_random_walk_definition():
    topo, edges = _tiny_hypergraph()
    P = O.Topology(topo).dense()
    n = 7
    want = np.zeros((n, n))
    for i in range(n):       # Definition 1: pick an incident hyperedge, then a member
        inc = [e for e in edges if i in e]
        for e in inc:
            for j in e:
                want[i, j] += (1.0 / len(inc)) * (1.0 / len(e))
    assert np.allclose(P, want, atol=1e-15)
    assert np.allclose(P.sum(axis=1), 1.0)


def test_multiplex_walk_matches_layer_choice_definition():
    rng = np.random.default_rng(7)
    n = 12
    layers, adj = [], []
    for _ in range(3):
        src = rng.integers(0, n, 30)
        dst = rng.integers(0, n, 30)
        rp, col = synth.csr_from_edges(n, src, dst, symmetric=True)
        layers.append((rp, col))
        nb = [set(col[rp[i]:rp[i + 1]].tolist()) for i in range(n)]
        adj.append(nb)
    P = O.Topology(dict(kind="multiplex", n=n, layers=layers)).dense()
    want = np.zeros((n, n))
    for i in range(n):        # choose a layer w.p. 1/L, then a neighbour uniformly
        for nb in adj:
            for j in nb[i]:
                want[i, j] += (1.0 / 3.0) / len(nb[i])
    assert np.allclose(P, want, atol=1e-15)


def test_directed_graph_is_symmetrised():
    n = 5
    row_ptr = np.array([0, 1, 2, 3, 3, 3], np.int64)   # 0->1, 1->2, 2->0
    col = np.array([1, 2, 0], np.int32)
    P = O.Topology(dict(kind="graph", n=n, layers=[(row_ptr, col)], directed=True)).dense()
    want = np.zeros((n, n))
    for a, b in [(0, 1), (1, 2), (2, 0)]:
        want[a, b] = want[b, a] = 0.5
    assert np.allclose(P, want)


def test_beta_rule_and_row_stochastic_P():
    topo, _ = _tiny_hypergraph()
    topo["n"] = 8                       # node 7 is in no hyperedge
    X = np.random.default_rng(8).standard_normal((8, 4))
    X[3] = 0.0                          # zero attributes
    P, _ = O.build_walk(topo, X, K=3, beta=0.4)
    assert P.b[3] == 0.0 and P.b[7] == 1.0
    assert np.allclose(np.delete(P.b, [3, 7]), 0.4)
    rows = P.dense().sum(axis=1)
    assert np.allclose(rows, 1.0)


def test_negative_knn_degree_reading_r3():
    """Reading R3 worked by hand on six nodes (Eq. AK with negative cosines):
    node 0 points away from everyone, so its K = 2 nearest are node 5
    (cos = -0.2/sqrt(1.04)) and node 3 (cos = -1/sqrt(1.09), tied with node 4,
    lowest index kept); no node lists node 0, so D_K[0] = -0.196 - 0.958 < 0
    and node 0 gets a zero P_K row and beta_0 = 0, while every other row of
    P_K still sums to 1 (its degree is positive)."""
    X = np.array([[1.0, 0.0], [-1.0, 0.1], [-1.0, -0.1], [-1.0, 0.3], [-1.0, -0.3], [-0.2, 1.0]])
    idx, _ = O.knn_cosine(X, 2)
    assert idx[0].tolist() == [5, 3]
    assert idx[5].tolist() == [3, 1] and 0 not in idx[1:].ravel()
    A = O.knn_adjacency(X, idx).toarray()
    f05, f03 = -0.2 / math.sqrt(1.04), -1.0 / math.sqrt(1.09)
    assert A[0, 5] == pytest.approx(f05, abs=1e-15) and A[5, 0] == pytest.approx(f05, abs=1e-15)
    assert A[0, 3] == pytest.approx(f03, abs=1e-15) and A[0, [1, 2, 4]].tolist() == [0.0, 0.0, 0.0]
    P_K, D = O.knn_transition(O.knn_adjacency(X, idx))
    assert D[0] == pytest.approx(f05 + f03, abs=1e-15) and D[0] < 0
    P_K = P_K.toarray()
    assert np.all(P_K[0] == 0.0)                      # not D_K^-1 A_K: that row would be positive
    assert np.all(D[1:] > 0) and np.allclose(P_K[1:].sum(axis=1), 1.0)
    b = O.beta_vector(X, np.ones(6), 0.5, D)
    assert b[0] == 0.0 and np.all(b[1:] == 0.5)
    # the walk of node 0 is then its topology walk alone
    row_ptr = np.array([0, 1, 2, 3, 4, 5, 6], np.int64)
    col = np.array([1, 0, 3, 2, 5, 4], np.int32)
    P, _ = O.build_walk(dict(kind="graph", n=6, layers=[(row_ptr, col)]), X, K=2, beta=0.5, knn=idx)
    Pd = P.dense()
    assert Pd[0].tolist() == [0.0, 1.0, 0.0, 0.0, 0.0, 0.0]
    assert np.allclose(Pd.sum(axis=1), 1.0)


def test_knn_transition_row_stochastic():
    X = np.abs(np.random.default_rng(9).standard_normal((40, 6)))  # positive cosines
    idx, _ = O.knn_cosine(X, 5)
    P_K, D = O.knn_transition(O.knn_adjacency(X, idx))
    assert np.all(D > 0)
    assert np.allclose(np.asarray(P_K.sum(axis=1)).ravel(), 1.0)


# ----------------------------------------------------------------------------
# Algorithm 2: MHC against Eq. (mh-cond) on a dense S
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("gamma", [1, 3, 5])
def test_calmhc_matches_conductance_definition(gamma):
    g = synth.sbm_graph(60, 3, 0.3, 0.05, 8, 1.0, seed=10)
    P, _ = O.build_walk(g, g["X"], K=4, beta=0.5)
    alpha = 0.2
    S = O.multi_hop_dense(P.dense(), alpha, gamma)
    labels = np.random.default_rng(11).integers(0, 3, 60)
    phi_alg2 = O.cal_mhc(P, labels, 3, alpha, gamma)
    phi_def = O.mhc_from_definition(S, labels, 3)
    # finite gamma: rows of S sum to 1 - (1-alpha)^(gamma+1), hence the offset
    assert abs((phi_alg2 - (1 - alpha) ** (gamma + 1)) - phi_def) < 1e-12


# ----------------------------------------------------------------------------
# Algorithm 4 lines 3-11: InitBCM
# ----------------------------------------------------------------------------
def test_initbcm_equals_truncated_rwr_series():
    g = synth.sbm_graph(80, 4, 0.25, 0.02, 4, 1.0, seed=12)
    topo = O.Topology(g)
    alpha, T_i, k = 0.2, 7, 4
    labels, Vc, PiT = O.init_bcm(topo, k, alpha, T_i)
    PN = topo.dense()
    Z0 = np.zeros((k, 80))
    Z0[np.arange(k), Vc] = 1
    series = sum(np.linalg.matrix_power((1 - alpha) * PN, t) for t in range(T_i + 1))
    Pi = alpha * Z0 @ series
    assert np.allclose(PiT.T, Pi, atol=1e-14)
    assert np.array_equal(labels, np.argmax(Pi, axis=0))


def test_initbcm_two_cliques_and_star():
    # cliques {0..4} and {5..10} joined by the edge 0-5: node 5 has degree 6,
    # node 0 ties with 6..10 at degree 5 and wins on the lower id
    src, dst = [], []
    for a, b in [(0, 5), (5, 11)]:
        for i in range(a, b):
            for j in range(i + 1, b):
                src.append(i)
                dst.append(j)
    src.append(0)
    dst.append(5)
    rp, col = synth.csr_from_edges(11, np.array(src), np.array(dst))
    topo = O.Topology(dict(kind="graph", n=11, layers=[(rp, col)]))
    labels, Vc, _ = O.init_bcm(topo, 2, 0.2, 25)
    assert Vc.tolist() == [0, 5]
    assert labels.tolist() == [0] * 5 + [1] * 6
    # star graph with one centre: every node goes to cluster 0
    rp, col = synth.csr_from_edges(9, np.zeros(8, np.int64), np.arange(1, 9))
    labels, Vc, _ = O.init_bcm(O.Topology(dict(kind="graph", n=9, layers=[(rp, col)])), 1, 0.2, 3)
    assert Vc.tolist() == [0] and np.all(labels == 0)


# ----------------------------------------------------------------------------
# QR, orthogonal iteration
# ----------------------------------------------------------------------------
def test_qr_pos_properties():
    Z = np.random.default_rng(13).standard_normal((200, 7))
    Q, R = O.qr_pos(Z)
    assert np.allclose(Q.T @ Q, np.eye(7), atol=1e-13)
    assert np.allclose(np.triu(R), R) and np.all(np.diag(R) > 0)
    assert np.allclose(Q @ R, Z, atol=1e-12)
    # unique thin QR with positive diagonal: Gram-Schmidt gives the same Q
    G = np.zeros_like(Z)
    for j in range(7):
        v = Z[:, j] - G[:, :j] @ (G[:, :j].T @ Z[:, j])
        v = v - G[:, :j] @ (G[:, :j].T @ v)
        G[:, j] = v / np.linalg.norm(v)
    assert np.allclose(G, Q, atol=1e-10)


def test_orthogonal_iteration_spans_power_subspace():
    g = synth.sbm_graph(90, 3, 0.3, 0.03, 6, 1.0, seed=14)
    P, _ = O.build_walk(g, g["X"], K=5, beta=0.5)
    Pd = P.dense()
    Q0 = np.random.default_rng(15).standard_normal((90, 4))
    Q = Q0
    for _ in range(6):
        Q, _ = O.qr_pos(P.apply(Q))
    W = np.linalg.matrix_power(Pd, 6) @ Q0
    assert O.max_principal_angle(Q, W) < 1e-9


# ----------------------------------------------------------------------------
# Discretize
# ----------------------------------------------------------------------------
def _rotation(k, angle, seed):
    A = np.random.default_rng(seed).standard_normal((k, k))
    Ks = (A - A.T) / 2
    Ks *= angle / np.linalg.norm(Ks, 2)
    return scipy.linalg.expm(Ks)


def test_discretize_rotation_is_polar_factor():
    rng = np.random.default_rng(16)
    n, k = 300, 5
    Qk = rng.standard_normal((n, k))
    labels, objs, R = O.discretize(Qk, max_iter=1, return_trace=True)
    Qt = Qk / np.linalg.norm(Qk, axis=1, keepdims=True)
    c = np.bincount(labels, minlength=k)
    M = (O.bcm(labels, k) / c).T @ Qt
    # orthogonal polar factor of M^T computed through an eigendecomposition
    w, V = np.linalg.eigh(M @ M.T)
    polar = M.T @ (V @ np.diag(w ** -0.5) @ V.T)
    assert np.allclose(R, polar, atol=1e-10)
    assert np.allclose(R.T @ R, np.eye(k), atol=1e-12)
    assert abs(objs[0] - (n - 2 * np.linalg.svd(M, compute_uv=False).sum())) < 1e-9


def test_discretize_recovers_rotated_indicators():
    rng = np.random.default_rng(17)
    n, k = 400, 6
    truth = rng.integers(0, k, n)
    Rot = _rotation(k, 0.5, 18)            # < pi/4: argmax with R = I is still right
    Qk = O.bcm(truth, k) @ Rot + 0.05 * rng.standard_normal((n, k))
    labels = O.discretize(Qk)
    assert O.adjusted_rand_index(labels, truth) == 1.0
    # a pure column permutation is also undone
    perm = rng.permutation(k)
    labels = O.discretize(O.bcm(truth, k)[:, perm])
    assert O.adjusted_rand_index(labels, truth) == 1.0


def test_h_norm_orthonormal_columns():
    labels = np.random.default_rng(19).integers(0, 7, 500)
    Yh = O.h_norm(labels, 7)
    assert np.allclose(Yh.T @ Yh, np.eye(7))


# ----------------------------------------------------------------------------
# evaluation helpers
# ----------------------------------------------------------------------------
def test_ari_hand_computed_and_library():
    # contingency [[2,1],[0,2]]: sum C(nij,2)=2, a: C(3,2)+C(2,2)=4, b: C(2,2)+C(3,2)=4
    # total C(5,2)=10, expected=1.6, max=4 -> (2-1.6)/(4-1.6) = 1/6
    a = [0, 0, 0, 1, 1]
    b = [0, 0, 1, 1, 1]
    assert abs(O.adjusted_rand_index(a, b) - 1.0 / 6.0) < 1e-15
    assert O.adjusted_rand_index([0, 0, 1, 1], [5, 5, 2, 2]) == 1.0
    sk = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(20)
    x, y = rng.integers(0, 4, 200), rng.integers(0, 5, 200)
    assert abs(O.adjusted_rand_index(x, y) - sk.adjusted_rand_score(x, y)) < 1e-12


def test_principal_angle_planted():
    th = 0.3
    A = np.array([[1.0], [0.0], [0.0]])
    B = np.array([[np.cos(th)], [np.sin(th)], [0.0]])
    assert abs(O.max_principal_angle(A, B) - th) < 1e-14
    rng = np.random.default_rng(21)
    U, V = rng.standard_normal((50, 4)), rng.standard_normal((50, 4))
    assert abs(O.max_principal_angle(U, V) - scipy.linalg.subspace_angles(U, V).max()) < 1e-10


# ----------------------------------------------------------------------------
# closed form: k disjoint cliques with per-clique identical attributes
# ----------------------------------------------------------------------------
def test_cliques_closed_form():
    k, c, K = 4, 16, 5
    g = synth.cliques_closed_form(k, c, seed=22)
    P, idx = O.build_walk(g, g["X"], K, 0.5)
    # KNN lists stay inside the clique (similarity 1 vs 0 outside)
    assert np.all(g["labels"][idx] == g["labels"][:, None])
    ev = np.sort(np.abs(np.linalg.eigvals(P.dense())))[::-1]
    assert np.allclose(ev[:k], 1.0) and ev[k] < 0.9
    init = np.random.default_rng(23).integers(0, k, k * c)
    T = 40
    res = O.ancka(g, g["X"], dict(k=k, K=K, T=T, tau=5), init_labels=init)
    ind = O.bcm(g["labels"], k)
    # the first k columns of Q span the cluster indicators
    assert O.max_principal_angle(res["Q"][:, :k], ind) <= max(1e-6, 10 * ev[k] ** T)
    assert O.adjusted_rand_index(res["labels"], g["labels"]) == 1.0


# ----------------------------------------------------------------------------
# reading R13: full-rank Q^(0) when InitBCM leaves a cluster empty
# ----------------------------------------------------------------------------
def test_splitmix64_reference_outputs():
    # first three outputs of splitmix64 seeded with 0 (state advances by the
    # golden-ratio increment; each output mixes the advanced state)
    g = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        states = np.array([0, g, g * np.uint64(2)], dtype=np.uint64)
    out = O.splitmix64(states)
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_initial_block_full_rank_with_empty_cluster():
    labels = np.array([0, 0, 2, 2, 2, 0, 2, 0, 0, 2] * 20)   # cluster 1 empty
    # the paper's block [1/sqrt(n) | h(Y)] is rank deficient twice over here
    raw = np.concatenate([np.full((200, 1), 1 / np.sqrt(200)), O.h_norm(labels, 3)], axis=1)
    assert np.linalg.matrix_rank(raw) == 2
    Q0 = O.initial_block(labels, 3)
    assert np.linalg.matrix_rank(Q0) == 4
    assert np.allclose(np.abs(Q0[:, [2, 3]]), 1 / np.sqrt(labels.size))
    # span(h(Y)) is kept: h(Y)'s columns lie in span(Q0)
    Yh = O.h_norm(labels, 3)
    coef, *_ = np.linalg.lstsq(Q0, Yh, rcond=None)
    assert np.allclose(Q0 @ coef, Yh)
    assert np.allclose(Q0[:, 1], Yh[:, 0])
    # a fully populated Y: only the last cluster's column is replaced
    full = np.arange(200) % 3
    Q1 = O.initial_block(full, 3)
    assert np.linalg.matrix_rank(Q1) == 4
    assert np.allclose(Q1[:, 1:3], O.h_norm(full, 3)[:, :2])


def test_paper_mode_stop_rules(monkeypatch):
    """Alg. 4 checks Eq. tcond-1 / tcond-2 after keep-best at each t with
    t mod tau = 0: a threshold every ||Q(t) - Q(t-1)|| meets stops at t = tau;
    with eps_Q = 0, three strictly rising phi values (phi(Y0) counted) stop
    the loop at their third check, and a flat phi never does (t runs to T)."""
    g = synth.cliques_closed_form(4, 30, 0)
    p = dict(k=4, K=10, T=40, tau=5, early_stop=True, eps_Q=10.0)
    assert O.ancka(g, g["X"], p)["iters"] == 5
    seq = iter([0.10, 0.20, 0.30, 0.40, 0.50, 0.60, 0.70, 0.80, 0.90])
    monkeypatch.setattr(O, "cal_mhc", lambda *a, **kw: next(seq))
    r = O.ancka(g, g["X"], dict(p, eps_Q=0.0))
    assert r["iters"] == 10 and list(r["phi"]) == [0.10, 0.20, 0.30]
    seq2 = iter([0.30, 0.20, 0.25, 0.10, 0.15, 0.40, 0.50, 0.60, 0.70])
    monkeypatch.setattr(O, "cal_mhc", lambda *a, **kw: next(seq2))
    # 0.30 0.20 0.25 0.10 0.15 0.40: the first strictly rising triple ends at t = 25
    assert O.ancka(g, g["X"], dict(p, eps_Q=0.0))["iters"] == 25
    monkeypatch.setattr(O, "cal_mhc", lambda *a, **kw: 0.5)
    r = O.ancka(g, g["X"], dict(p, eps_Q=0.0))
    assert r["iters"] == 40 and len(r["phi"]) == 9
