"""KNN parity of the CUDA path (ancka_knn through the C ABI) against the oracle."""
import numpy as np
import pytest

from oracle import ancka_oracle as O
from paper_2408_05459_gb300 import synth
from tests.parity_util import compare_knn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = ["fp32", "bf16", "fp8"]


@pytest.fixture(scope="module")
def ak():
    from paper_2408_05459_gb300 import ancka
    ancka.load()
    return ancka


def _run(ak, X, K, prec):
    Xd = torch.as_tensor(np.ascontiguousarray(X, np.float32), device="cuda")
    idx, sim, info = ak.knn(Xd, K, prec)
    torch.cuda.synchronize()
    return idx.cpu().numpy(), sim.cpu().numpy(), info


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,d,K", [(2000, 128, 10), (300, 5, 4), (129, 64, 16), (1000, 100, 10), (777, 130, 7)])
def test_knn_random_shapes(ak, prec, n, d, K):
    rng = np.random.default_rng(n + d + K)
    labels = rng.integers(0, 5, n)
    X = synth.gaussian_mixture(rng, labels, 5, d, 1.5)
    idx, sim, info = _run(ak, X, K, prec)
    c = compare_knn(X, K, np.arange(n), idx, sim)
    assert c["exact_rows"] + c["near_tie_rows"] == n
    # within the certified range (K <= 12 for BF16, 16 for FP32) few rows fall
    # back; FP8's wider margin leaves most rows to its BF16 second pass, whose
    # certificate then settles nearly all of them
    if prec != "fp8" and K <= (12 if prec == "bf16" else 16):
        assert info["knn_fallback_rows"] <= n // 20
    if prec == "fp8" and K <= 12:
        assert info["knn_exhaustive_rows"] <= n // 20


@pytest.mark.parametrize("prec", PRECS)
def test_knn_edge_cases(ak, prec):
    rng = np.random.default_rng(7)
    n, d, K = 260, 33, 6
    X = rng.standard_normal((n, d)).astype(np.float32)
    X[3] = 0.0                     # zero row: all similarities 0, lowest indices win
    X[10] = X[20] = X[30]          # exact duplicates: similarity-1 ties
    X[40] = 3.0 * X[41]            # scaled copy
    X[255:] = np.abs(X[255:])      # ragged tail rows
    idx, sim, _ = _run(ak, X, K, prec)
    compare_knn(X, K, np.arange(n), idx, sim)
    assert idx[3].tolist() == [j for j in range(n) if j != 3][:K]
    assert np.all(sim[3] == 0.0)
    assert set(idx[30][:2].tolist()) == {10, 20}


@pytest.mark.parametrize("prec", PRECS)
def test_knn_tiny_and_large_K(ak, prec):
    X = np.random.default_rng(1).standard_normal((3, 4)).astype(np.float32)
    idx, sim, _ = _run(ak, X, 2, prec)
    compare_knn(X, 2, np.arange(3), idx, sim)
    # K beyond the candidate list: the exhaustive exact path
    X = np.random.default_rng(2).standard_normal((400, 24)).astype(np.float32)
    idx, sim, info = _run(ak, X, 40, prec)
    compare_knn(X, 40, np.arange(400), idx, sim)
    assert info["knn_fallback_rows"] == 400


def test_knn_hypergraph_workload_sampled(ak):
    """Full-size sparse TF-IDF attributes (n = 1e5, d = 500) on sampled rows."""
    g = synth.config_hypergraph(0)
    X = g["X"]
    rows = np.random.default_rng(11).choice(X.shape[0], 192, replace=False)
    for prec in PRECS:
        idx, sim, info = _run(ak, X, 10, prec)
        c = compare_knn(X, 10, rows, idx, sim)
        assert c["exact_rows"] + c["near_tie_rows"] == rows.size
        if prec != "fp8":
            assert info["knn_fallback_rows"] < X.shape[0] // 100
        assert info["knn_exhaustive_rows"] < X.shape[0] // 100


@pytest.mark.parametrize("prec", PRECS)
def test_knn_sparse_rows_mixed(ak, prec):
    """Rows of every sparsity the re-rank meets: a few nonzeros spread over
    the lanes' strided shares (the sparse-row gather), nonzeros packed into
    one share (t = 5 mod 32: too many for one lane, the dense loop), dense
    rows, zero rows, duplicates and sign changes.  Every list must be exact."""
    rng = np.random.default_rng(31)
    n, d, K = 3000, 300, 8
    X = np.zeros((n, d), np.float32)
    topics = [rng.choice(d, 24, replace=False) for _ in range(6)]
    lab = rng.integers(0, 6, n)
    for i in range(n):
        nnz = int(rng.integers(1, 30))
        own = rng.random(nnz) < 0.7
        cols = np.where(own, rng.choice(topics[lab[i]], nnz), rng.integers(0, d, nnz))
        X[i, cols] = rng.exponential(1.0, nnz).astype(np.float32)
    packed = rng.choice(n, 200, replace=False)
    X[packed] = 0.0
    share = np.arange(5, d, 32)
    X[np.ix_(packed, share)] = rng.standard_normal((200, share.size)).astype(np.float32)
    dense = rng.choice(n, 150, replace=False)
    X[dense] = rng.standard_normal((150, d)).astype(np.float32)
    X[7] = 0.0
    X[100] = X[200] = X[300]
    X[400] = -X[401]
    X[500] = 2.5 * X[501]
    idx, sim, _ = _run(ak, X, K, prec)
    c = compare_knn(X, K, np.arange(n), idx, sim)
    assert c["exact_rows"] + c["near_tie_rows"] == n
    assert idx[7].tolist() == [j for j in range(n) if j != 7][:K]
    assert set(idx[300][:2].tolist()) == {100, 200}


def test_knn_invalid_arguments(ak):
    X = torch.zeros((5, 3), device="cuda")
    with pytest.raises(ak.AnckaError) as e:
        ak.knn(X, 5, "fp32")      # K >= n
    assert e.value.status == 1
    with pytest.raises(ak.AnckaError) as e:
        ak.knn(X, 0, "fp32")
    assert e.value.status == 1


def test_knn_deterministic(ak):
    X = np.random.default_rng(3).standard_normal((1500, 77)).astype(np.float32)
    for prec in PRECS:
        a = _run(ak, X, 9, prec)
        b = _run(ak, X, 9, prec)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_knn_collect_pass_dense_rows(ak):
    """Dense random rows: many rows cannot be certified from the two 16-entry
    lists and go through the collect pass; all lists must still be exact."""
    X = np.random.default_rng(12).standard_normal((12000, 256)).astype(np.float32)
    idx, sim, info = _run(ak, X, 10, "bf16")
    assert info["knn_fallback_rows"] > 0
    assert info["knn_exhaustive_rows"] <= max(1, info["knn_fallback_rows"] // 10)
    c = compare_knn(X, 10, np.arange(12000), idx, sim)
    assert c["exact_rows"] + c["near_tie_rows"] == 12000


@pytest.mark.parametrize("ordered", [False, True])
def test_knn_clustered_rows_parity(ak, ordered):
    """n = 20000 Gaussian mixture; ordered=True sorts the rows by cluster so
    that each row's neighbours sit in a narrow key range (one 128-key half
    of a tile holds most of them)."""
    rng = np.random.default_rng(21)
    n, d, K = 20000, 96, 10
    labels = rng.integers(0, 8, n)
    if ordered:
        labels = np.sort(labels)
    X = synth.gaussian_mixture(rng, labels, 8, d, 1.2)
    idx, sim, info = _run(ak, X, K, "bf16")
    rows = np.random.default_rng(22).choice(n, 1200, replace=False)
    c = compare_knn(X, K, rows, idx, sim)
    assert c["exact_rows"] + c["near_tie_rows"] == rows.size
    assert info["knn_fallback_rows"] <= n // 20


def test_knn_fp8_certified_groups(ak):
    """Groups of K + 1 near-duplicate rows (cosine ~0.99 inside a group,
    ~0.25 across): the FP8 margin is far below the gap after the K-th
    neighbour, so the FP8 lists certify nearly every row themselves."""
    rng = np.random.default_rng(31)
    g, K, d = 300, 10, 64
    centres = rng.standard_normal((g, d))
    X = (np.repeat(centres, K + 1, axis=0) + 0.05 * rng.standard_normal((g * (K + 1), d))).astype(np.float32)
    X = X[rng.permutation(X.shape[0])]
    idx, sim, info = _run(ak, X, K, "fp8")
    c = compare_knn(X, K, np.arange(X.shape[0]), idx, sim)
    assert c["exact_rows"] + c["near_tie_rows"] == X.shape[0]
    assert info["knn_fallback_rows"] <= X.shape[0] // 20


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("n,d", [(3000, 200), (2600, 130)])
def test_candidate_error_model(ak, prec, n, d):
    """The certificate's error model against exact arithmetic on the
    quantised rows: e_i >= ||q_i - u_i||, |score - q_i.q_j| <= acc |q_i||q_j|
    for every kept candidate, and every key a list left out scores at most the
    list's minimum (up to the same bound)."""
    rng = np.random.default_rng(n + d)
    labels = rng.integers(0, 6, n)
    X = synth.gaussian_mixture(rng, labels, 6, d, 1.0)
    cv, ci, q, err, acc = ak.knn_candidates(torch.as_tensor(X, device="cuda"), prec)
    torch.cuda.synchronize()
    cv, ci, q, err = [t.cpu().numpy() for t in (cv, ci, q, err)]
    q = q.astype(np.float64)
    U = O.unit_rows(X)
    assert np.all(np.linalg.norm(q - U, axis=1) <= err.astype(np.float64))
    G = q @ q.T
    nq = np.linalg.norm(q, axis=1)
    half_of = (np.arange(n) % 256) // 128
    worst = 0.0
    for i in range(n):
        for h in range(2):
            js = ci[i, 16 * h:16 * h + 16]
            vs = cv[i, 16 * h:16 * h + 16].astype(np.float64)
            assert np.all(js != i) and np.all(half_of[js[js >= 0]] == h)
            ok = js >= 0
            bound = acc * nq[i] * nq[js[ok]]
            worst = max(worst, float((np.abs(vs[ok] - G[i, js[ok]]) / bound).max()))
            others = half_of == h
            others[i] = False
            others[js[ok]] = False
            if ok.all() and others.any():
                assert np.all(G[i, others] <= vs.min() + acc * nq[i] * nq[others]), f"row {i} list {h}"
            else:
                assert not others.any(), f"row {i} list {h}: list not full but keys left out"
    print(f"{prec}: max |score - q.q| / (acc |q||q|) = {worst:.3g} (acc = {acc:.3g})")
    assert worst <= 1.0


class _SymmetricMinRows:
    """Sets the symmetric-contraction crossover for one block, then restores
    the default."""

    def __init__(self, ak, n_min):
        self.ak, self.n_min = ak, n_min

    def __enter__(self):
        self.ak.set_symmetric_knn_min_rows(self.n_min)

    def __exit__(self, *exc):
        self.ak.set_symmetric_knn_min_rows(2**63 - 1)


@pytest.mark.parametrize("n,d", [(70000, 64), (9000, 96)])
def test_symmetric_contraction_lists(ak, n, d):
    """The symmetric contraction (pairs j > i only, thresholds from every 8th
    key tile, scores pushed to both rows) leaves the same two 16-entry lists
    per row as the full sweep: s_ij and s_ji sum the same products in the same
    order, so the scores agree bit for bit; the keys agree except where equal
    scores sit at the 16th place."""
    rng = np.random.default_rng(n + d)
    labels = rng.integers(0, 8, n)
    X = torch.as_tensor(synth.gaussian_mixture(rng, labels, 8, d, 1.0), device="cuda")
    with _SymmetricMinRows(ak, 2**63 - 1):
        cv0, ci0, _, _, _ = ak.knn_candidates(X, "bf16")
    with _SymmetricMinRows(ak, 1):
        cv1, ci1, _, _, _ = ak.knn_candidates(X, "bf16")
    torch.cuda.synchronize()
    cv0, ci0, cv1, ci1 = [t.cpu().numpy() for t in (cv0, ci0, cv1, ci1)]
    same_keys = 0
    for h in range(2):
        a, b = cv0[:, 16 * h:16 * h + 16], cv1[:, 16 * h:16 * h + 16]
        assert np.array_equal(np.sort(a, axis=1), np.sort(b, axis=1)), f"half {h}: scores differ"
        ka, kb = np.sort(ci0[:, 16 * h:16 * h + 16], axis=1), np.sort(ci1[:, 16 * h:16 * h + 16], axis=1)
        same_keys += int(np.all(ka == kb, axis=1).sum())
        assert np.all((ci1[:, 16 * h:16 * h + 16] // 128) % 2 == h), "key in the wrong half"
    assert same_keys >= 2 * n - n // 1000, same_keys


@pytest.mark.parametrize("n,d,K", [(2000, 128, 10), (300, 5, 4), (777, 130, 7), (20000, 48, 10)])
def test_symmetric_contraction_knn_exact(ak, n, d, K):
    """Exact KNN through the symmetric contraction at small and ragged sizes
    (forced below its default crossover)."""
    rng = np.random.default_rng(n + 3 * d + K)
    labels = rng.integers(0, 5, n)
    X = synth.gaussian_mixture(rng, labels, 5, d, 1.5)
    with _SymmetricMinRows(ak, 1):
        idx, sim, info = _run(ak, X, K, "bf16")
    rows = np.arange(n) if n <= 4000 else np.random.default_rng(5).choice(n, 512, replace=False)
    c = compare_knn(X, K, rows, idx, sim)
    assert c["exact_rows"] + c["near_tie_rows"] == rows.size
