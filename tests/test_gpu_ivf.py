"""Approximate KNN by inverted lists (ancka_knn_ivf; the paper's large-n
KNN of Section 7 is Faiss IVFPQ) through the C ABI.  Its lists are not the
exact N_K, so this is a separate parity regime: every returned list is a
valid KNN list whose cosines are exact, recall@K against the oracle's exact
lists is measured on sampled rows, probing every cell gives the exact lists,
the result is deterministic, and Algorithm 4 run on these lists matches the
oracle's run on the same lists."""
import numpy as np
import pytest

from oracle import ancka_oracle as O
from paper_2408_05459_gb300 import synth
from tests.parity_util import ANGLE_MAX, ARI_MIN, compare_iteration

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ak():
    from paper_2408_05459_gb300 import ancka
    ancka.load()
    return ancka


def _x(n, seed=0):
    """Attributes of the large workload's generator (47 clusters, d = 100)."""
    rng = np.random.default_rng(seed)
    w = 1.0 / np.arange(1, 48)
    lab = rng.choice(47, n, p=w / w.sum())
    return synth.gaussian_mixture(rng, lab, 47, 100, 1.5)


def _check_lists(X, idx, sim, rows, K):
    """Valid lists (K distinct other rows, cosine desc then index asc) with
    exact cosines; returns recall@K against the oracle on `rows`."""
    o_idx, _ = O.knn_cosine(X, K, rows=rows)
    Xn = O.unit_rows(X)
    hits = 0
    for r, i in enumerate(rows):
        li = idx[i].astype(np.int64)
        assert np.all(li != i) and len(set(li.tolist())) == K
        true = Xn[li] @ Xn[i]
        assert np.all(np.abs(sim[i] - true) <= 1e-6)
        assert np.all(np.diff(true) <= 1e-6)              # cosine desc (within rounding)
        hits += len(set(li.tolist()) & set(o_idx[r].tolist()))
    return hits / (K * len(rows))


def test_ivf_lists_valid_and_recall(ak):
    n, K = 60000, 10
    X = _x(n)
    idx, sim, info = ak.knn_ivf(torch.as_tensor(X, device="cuda"), K, nlist=30, nprobe=4)
    torch.cuda.synchronize()
    rows = np.random.default_rng(1).choice(n, 256, replace=False)
    rec = _check_lists(X, idx.cpu().numpy(), sim.cpu().numpy(), rows, K)
    assert rec >= 0.97, rec
    # key tiles are skipped (a 128-row block sweeps the union of its rows'
    # probed cells, so at this small size most of the tiles remain)
    assert 0 < info["knn_tiles"] < info["knn_full_tiles"]


def test_ivf_probing_every_cell_gives_exact_lists(ak):
    """nprobe = nlist: every block sweeps every key tile, so the candidates
    are the exact path's and the re-ranked lists are the exact N_K (rows whose
    K-th and (K+1)-th cosines are within 1e-6 excepted)."""
    n, K = 12000, 10
    X = _x(n, seed=2)
    idx, sim, _ = ak.knn_ivf(torch.as_tensor(X, device="cuda"), K, nlist=8, nprobe=8)
    torch.cuda.synchronize()
    idx = idx.cpu().numpy()
    rows = np.random.default_rng(3).choice(n, 300, replace=False)
    o_idx, o_sim = O.knn_cosine(X, K, rows=rows, extra=1)
    tie = (o_sim[:, K - 1] - o_sim[:, K]) < 1e-6 * np.abs(o_sim[:, K - 1])
    same = np.array([set(idx[i].tolist()) == set(o_idx[r].tolist()) for r, i in enumerate(rows)])
    assert np.all(same | tie)


def test_ivf_deterministic(ak):
    X = torch.as_tensor(_x(40000, seed=4), device="cuda")
    a = ak.knn_ivf(X, 10, nlist=40, nprobe=3, with_info=False)
    b = ak.knn_ivf(X, 10, nlist=40, nprobe=3, with_info=False)
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_cluster_on_ivf_lists_matches_oracle(ak):
    """ancka_cluster with knn_nlist > 0 takes the approximate lists; the
    oracle's Algorithm 4 on the same lists gives the same labels and block."""
    g = synth.config_large_dcsbm(0, n=30000, m_edges=750000)
    p = ak.default_params(k=47, K=10, T=10, T_i=1, beta=0.4, knn_prec="bf16", knn_nlist=15, knn_nprobe=4)
    td = ak.topology_to_device(g)
    labels, ex, info = ak.cluster(td, torch.as_tensor(g["X"], device="cuda"), p, want_Q=True, want_knn=True,
                                  want_init=True)
    torch.cuda.synchronize()
    assert 0 < info["knn_tiles"] < info["knn_full_tiles"]
    knn = ex["knn_idx"].cpu().numpy()
    o = O.ancka(g, g["X"], dict(k=47, K=10, T=10, T_i=1, beta=0.4), knn=knn)
    assert np.array_equal(ex["init_labels"].cpu().numpy(), o["init_labels"])
    ari, ang = compare_iteration(o, labels.cpu().numpy(), ex["Q"].cpu().numpy())
    assert ari >= ARI_MIN and ang <= ANGLE_MAX, (ari, ang)


def test_ivf_invalid_arguments(ak):
    X = torch.as_tensor(_x(1000), device="cuda")
    for kw in (dict(nlist=0, nprobe=1), dict(nlist=10, nprobe=11), dict(nlist=10, nprobe=33),
               dict(nlist=2000, nprobe=1)):
        with pytest.raises(ak.AnckaError) as e:
            ak.knn_ivf(X, 10, **kw)
        assert e.value.status == 1
