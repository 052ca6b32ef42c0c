"""Learned warm start (features, MLP forward, gradients, training, the
warm-or-InitBCM start) and the paper's early-termination mode, through the C
ABI, against the FP64 oracle (readings W1-W6, Eq. tcond-1 / tcond-2)."""
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


def _dev(prm):
    return {k: torch.as_tensor(np.ascontiguousarray(v, np.float32), device="cuda") for k, v in prm.items()}


def _host(prm):
    return {k: v.detach().cpu().numpy().astype(np.float64) for k, v in prm.items()}


GRAPHS = {
    "sbm": lambda seed=5: synth.sbm_graph(1500, 4, 0.02, 0.002, 48, 1.5, seed),
    "hypergraph": lambda seed=6: synth.hypergraph_tfidf(1800, 4, 3000, 40, 6, seed=seed),
    "multiplex": lambda seed=7: synth.multiplex_sbm(1600, 4, 10.0, (6.0, 3.0), 32, 2.0, seed=seed),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_warm_forward_parity(ak, name):
    g = GRAPHS[name]()
    k, d = g["k"], g["X"].shape[1]
    prm = synth.warm_init(1, 2 * d, 256, k)
    W = ak.warm_predict(ak.topology_to_device(g), torch.as_tensor(g["X"], device="cuda"), _dev(prm))
    torch.cuda.synchronize()
    W = W.cpu().numpy().astype(np.float64)
    A = O.warm_features(O.Topology(g), g["X"])
    Wo, _ = O.warm_forward(A, {k_: v.astype(np.float64) for k_, v in prm.items()}, bf16=True)
    # BF16 operands on both sides; the unit rows and P_N U differ only in the
    # last FP32 bits before rounding
    assert np.max(np.abs(W - Wo)) <= 2e-3 * np.max(np.abs(Wo))


def test_warm_gradient_parity(ak):
    g = GRAPHS["sbm"]()
    k, d, lam = g["k"], g["X"].shape[1], 1e-2
    Qt = O.h_norm(g["labels"], k)
    prm = synth.warm_init(2, 2 * d, 256, k)
    grads, loss = ak.warm_gradients(ak.topology_to_device(g), torch.as_tensor(g["X"], device="cuda"),
                                    torch.as_tensor(Qt.astype(np.float32), device="cuda"), _dev(prm), lam)
    torch.cuda.synchronize()
    p64 = {k_: v.astype(np.float64) for k_, v in prm.items()}
    A = O.warm_features(O.Topology(g), g["X"])
    W, cache = O.warm_forward(A, p64, bf16=True)
    L = O.warm_loss(W, Qt, lam)
    go = O.warm_backward(A, p64, cache, O.warm_loss_grad(W, Qt, lam), bf16=True)
    assert abs(loss - L) <= 1e-4 * max(1.0, abs(L)), (loss, L)
    for name in ("W1", "b1", "W2", "b2"):
        gg = grads[name].cpu().numpy().astype(np.float64)
        rel = np.linalg.norm(gg - go[name]) / np.linalg.norm(go[name])
        assert rel <= 1e-2, (name, rel)


def test_warm_training_against_oracle(ak):
    gs = [GRAPHS["sbm"](10), GRAPHS["sbm"](11)]
    k, d, lam, lr, epochs = 4, 48, 1e-2, 3e-3, 25
    prm = synth.warm_init(3, 2 * d, 256, k)
    items, data = [], []
    for g in gs:
        Qt = O.h_norm(g["labels"], k)
        items.append((ak.topology_to_device(g), torch.as_tensor(g["X"], device="cuda"),
                      torch.as_tensor(Qt.astype(np.float32), device="cuda")))
        data.append((O.warm_features(O.Topology(g), g["X"]), Qt))
    w = _dev(prm)
    lg = ak.warm_train(items, w, epochs, lr, lam)
    torch.cuda.synchronize()
    _, lo = O.warm_train(data, {k_: v.astype(np.float64) for k_, v in prm.items()}, epochs, lr, lam, bf16=True)
    assert len(lg) == len(lo) == epochs * len(gs)
    assert np.allclose(lg[:6], lo[:6], rtol=2e-3, atol=1e-5), (lg[:6], lo[:6])
    assert lg[-1] < 0.5 * lg[0]
    assert abs(lg[-1] - lo[-1]) <= 0.1 * lo[-1] + 1e-3


def _oracle_params(p):
    return dict(k=p.k, K=p.K, alpha=p.alpha, beta=p.beta, T=p.T, gamma=p.gamma, T_i=p.T_i, tau=p.tau,
                disc_max_iter=p.disc_max_iter, early_stop=bool(p.early_stop), eps_Q=p.eps_Q)


@pytest.mark.parametrize("node_order", [1, 2])
def test_warm_start_cluster(ak, node_order):
    """Targets are ANCKA's own blocks on two training graphs; on a fresh graph
    the GPU and the oracle take the same start (warm or InitBCM) and agree,
    with the iteration on the caller's node order and on the degree order."""
    k = 4
    items = []
    for seed in (20, 21):
        g = GRAPHS["sbm"](seed)
        p = ak.default_params(k=k, knn_prec="fp32")
        _, ex, _ = ak.cluster(ak.topology_to_device(g), torch.as_tensor(g["X"], device="cuda"), p, want_Q=True)
        items.append((ak.topology_to_device(g), torch.as_tensor(g["X"], device="cuda"),
                      ex["Q"][:, 1:].contiguous()))
    w = _dev(synth.warm_init(4, 96, 256, k))
    ak.warm_train(items, w, 40, 3e-3, 1e-2)
    torch.cuda.synchronize()
    g = GRAPHS["sbm"](22)
    p = ak.default_params(k=k, knn_prec="fp32", node_order=node_order)
    td = ak.topology_to_device(g)
    labels, ex, info = ak.cluster(td, torch.as_tensor(g["X"], device="cuda"), p, want_Q=True, want_knn=True,
                                  warm=w)
    torch.cuda.synchronize()
    o = O.ancka(g, g["X"], _oracle_params(p), knn=ex["knn_idx"].cpu().numpy(), warm=_host(w))
    assert bool(info["warm_used"]) == bool(o["warm_used"])
    ari, ang = compare_iteration(o, labels.cpu().numpy(), ex["Q"].cpu().numpy())
    assert ari >= ARI_MIN and ang <= ANGLE_MAX, (ari, ang)
    assert O.adjusted_rand_index(labels.cpu().numpy(), g["labels"]) > 0.9


@pytest.mark.parametrize("eps_Q", [1.0, 0.95])
def test_paper_mode_parity(ak, eps_Q):
    """Eq. tcond-1 stops the loop at the first check point with ||Q(t) -
    Q(t-1)||_F < eps_Q.  On this graph the (k+1)-th column of Q is a bulk
    eigenvector that keeps rotating, so ||dQ||_F decreases slowly from ~1.3
    (t = 5) through 1.02 (t = 25), 0.977 (t = 30), 0.938 (t = 35): the
    thresholds stop the oracle at t = 30 and t = 35 with margins far above
    FP32 rounding."""
    g = synth.config_small_sbm(0)
    p = ak.default_params(k=g["k"], knn_prec="fp32", T=200, tau=5, early_stop=1, eps_Q=eps_Q)
    labels, ex, info = ak.cluster(ak.topology_to_device(g), torch.as_tensor(g["X"], device="cuda"), p,
                                  want_Q=True, want_knn=True)
    torch.cuda.synchronize()
    o = O.ancka(g, g["X"], _oracle_params(p), knn=ex["knn_idx"].cpu().numpy())
    assert info["iters_run"] == o["iters"] and info["iters_run"] < 200
    assert info["n_phi"] == min(len(o["phi"]), 64)
    ari, ang = compare_iteration(o, labels.cpu().numpy(), ex["Q"].cpu().numpy())
    assert ari >= ARI_MIN and ang <= ANGLE_MAX, (ari, ang)


def test_warm_invalid_arguments(ak):
    g = GRAPHS["sbm"]()
    X = torch.as_tensor(g["X"], device="cuda")
    bad = _dev(synth.warm_init(0, 50, 256, g["k"]))     # d_in != 2 d
    with pytest.raises(ak.AnckaError) as e:
        ak.warm_predict(ak.topology_to_device(g), X, bad)
    assert e.value.status == 1
    p = ak.default_params(k=g["k"] + 1, knn_prec="fp32")
    with pytest.raises(ak.AnckaError) as e:             # k of the model != clusters
        ak.cluster(ak.topology_to_device(g), X, p, warm=_dev(synth.warm_init(0, 96, 256, g["k"])))
    assert e.value.status == 1


def test_learned_start_gains_over_initbcm(ak):
    """What the trained network gains over the method without it.  The MLP
    is trained on ANCKA's own blocks of eight DC-SBM graphs (n = 2e4, k = 10,
    d = 64, T_i = 1 and beta = 0.4 as for the large graphs, where InitBCM's
    single hop from the k hubs leaves most nodes in one cluster), then four
    held-out graphs of the same generator are clustered from InitBCM's start
    and from the learned one:
      - the learned start is taken (its Phi is lower than InitBCM's) on every
        graph;
      - with a budget of five hops (one Discretize) the kept Phi is never
        higher and the labels agree better with the planted partition;
      - in the paper's early-termination mode (Eq. tcond-1/2) the learned
        start needs fewer hops in total, at a Phi no higher on any graph;
      - on the first graph the oracle, given the same weights, takes the same
        start and reaches the same labels and block."""
    k, d = 10, 64
    items = []
    for seed in range(100, 108):
        g = synth.dcsbm_graph(20000, k, 500000, d, 1.5, seed)
        td = ak.topology_to_device(g)
        X = torch.as_tensor(g["X"], device="cuda")
        p = ak.default_params(k=k, K=10, T=10, T_i=1, beta=0.4, knn_prec="bf16")
        _, ex, _ = ak.cluster(td, X, p, want_Q=True, with_info=False)
        items.append((td, X, ex["Q"][:, 1:].contiguous()))
    w = _dev(synth.warm_init(0, 2 * d, 256, k))
    losses = ak.warm_train(items, w, 60, 1e-3, 1e-2)
    torch.cuda.synchronize()
    assert losses[-1] < 0.5 * losses[0]
    hops = {"plain": 0, "learned": 0}
    ari5 = {"plain": [], "learned": []}
    for seed in (200, 201, 202, 203):
        g = synth.dcsbm_graph(20000, k, 500000, d, 1.5, seed)
        td = ak.topology_to_device(g)
        X = torch.as_tensor(g["X"], device="cuda")
        res = {}
        for mode in ("plain", "learned"):
            r = {}
            for tag, kw in (("paper", dict(T=100, early_stop=1, eps_Q=0.005)), ("T5", dict(T=5))):
                p = ak.default_params(k=k, K=10, T_i=1, beta=0.4, tau=5, knn_prec="bf16", **kw)
                lab, _, info = ak.cluster(td, X, p, warm=w if mode == "learned" else None)
                torch.cuda.synchronize()
                r[tag] = (info["iters_run"], info["phi"][0], info["phi_best"],
                          O.adjusted_rand_index(lab.cpu().numpy(), g["labels"]), info["warm_used"])
            res[mode] = r
            hops[mode] += r["paper"][0]
            ari5[mode].append(r["T5"][3])
        assert res["learned"]["T5"][4] == 1 and res["learned"]["T5"][1] < res["plain"]["T5"][1], res
        assert res["learned"]["T5"][2] <= res["plain"]["T5"][2] + 1e-5, res
        assert res["learned"]["paper"][2] <= res["plain"]["paper"][2] + 1e-4, res
        if seed == 200:
            p = ak.default_params(k=k, K=10, T=5, T_i=1, beta=0.4, tau=5, knn_prec="bf16")
            labels, ex, info = ak.cluster(td, X, p, want_Q=True, want_knn=True, warm=w)
            torch.cuda.synchronize()
            o = O.ancka(g, g["X"], _oracle_params(p), knn=ex["knn_idx"].cpu().numpy(), warm=_host(w))
            assert info["warm_used"] == 1 and bool(o["warm_used"])
            ari, ang = compare_iteration(o, labels.cpu().numpy(), ex["Q"].cpu().numpy())
            assert ari >= ARI_MIN and ang <= ANGLE_MAX, (ari, ang)
    assert hops["learned"] < hops["plain"], hops
    assert np.mean(ari5["learned"]) > np.mean(ari5["plain"]), ari5
