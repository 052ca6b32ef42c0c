"""Pins of the oracle's learned warm start (readings W1-W6) against
mathematics that does not come from the oracle itself: finite differences,
invariances, closed values of GELU and BF16 rounding, a hand-worked Adam step
and a hand-built walk."""
import numpy as np
import pytest

from oracle import ancka_oracle as O
from paper_2408_05459_gb300 import synth


def _orth(rng, n, k):
    q, _ = np.linalg.qr(rng.standard_normal((n, k)))
    return q


def test_gelu_values_and_derivative():
    # GELU(z) = z Phi(z): Phi(1) = 0.8413447460685429, Phi(-1) = 1 - Phi(1),
    # Phi(2) = 0.9772498680518208, Phi(-3) = 0.0013498980316300946
    z = np.array([0.0, 1.0, -1.0, 2.0, -3.0, 8.0])
    ref = np.array([0.0, 0.8413447460685429, -0.15865525393145707, 1.9544997361036416,
                    -3.0 * 0.0013498980316300946, 8.0])
    assert np.allclose(O.gelu(z), ref, rtol=1e-12, atol=1e-12)
    assert O.gelu_grad(np.array([0.0]))[0] == 0.5
    zs = np.linspace(-4, 4, 33)
    h = 1e-6
    fd = (O.gelu(zs + h) - O.gelu(zs - h)) / (2 * h)
    assert np.allclose(O.gelu_grad(zs), fd, rtol=1e-7, atol=1e-9)


def test_round_bf16_known_values():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -8 + 2 ** -20, -2.5, 3.14159265, 65504.0, 0.0])
    # spacing at 1 is 2^-7: 1 + 2^-8 is a tie -> even (1.0); 1 + 3*2^-8 is a tie -> even (1 + 2^-6)
    ref = np.array([1.0, 1.0, 1.0 + 2 ** -6, 1.0 + 2 ** -7, -2.5, 3.140625, 65536.0, 0.0])
    assert np.array_equal(O.round_bf16(x), ref)


def test_loss_gradient_against_finite_differences():
    rng = np.random.default_rng(0)
    n, k, lam = 14, 3, 0.05
    Qt = _orth(rng, n, k)
    W = rng.standard_normal((n, k))
    g = O.warm_loss_grad(W, Qt, lam)
    h = 1e-6
    fd = np.zeros_like(W)
    for i in range(n):
        for j in range(k):
            Wp, Wm = W.copy(), W.copy()
            Wp[i, j] += h
            Wm[i, j] -= h
            fd[i, j] = (O.warm_loss(Wp, Qt, lam) - O.warm_loss(Wm, Qt, lam)) / (2 * h)
    assert np.max(np.abs(g - fd)) < 1e-7 * max(1.0, np.max(np.abs(fd)))


def test_loss_invariances():
    rng = np.random.default_rng(1)
    n, k = 40, 4
    Qt = _orth(rng, n, k)
    W = rng.standard_normal((n, k))
    O_ = _orth(rng, k, k)
    base = O.warm_loss(W, Qt, 0.0)
    assert abs(O.warm_loss(W @ O_, Qt, 0.0) - base) < 1e-12       # rotation of W
    assert abs(O.warm_loss(7.5 * W, Qt, 0.0) - base) < 1e-12      # scale of W
    assert abs(O.warm_loss(Qt @ O_ * 3.0, Qt, 0.0)) < 1e-12       # span(W) = span(Q_t): zero
    assert base > 0.0 and base <= k                                # k - ||Q_t^T orth(W)||^2 in [0, k]
    # the first term equals k - ||Q_t^T orth(W)||_F^2 with orth from a QR of W
    Qw, _ = np.linalg.qr(W)
    assert abs(base - (k - np.sum((Qt.T @ Qw) ** 2))) < 1e-12
    # the penalty: lam ||G/n - I||^2 vanishes for W = sqrt(n) * orthonormal
    Wo = np.sqrt(n) * _orth(rng, n, k)
    assert abs(O.warm_loss(Wo, Qt, 3.0) - O.warm_loss(Wo, Qt, 0.0)) < 1e-10


def test_backward_against_finite_differences():
    rng = np.random.default_rng(2)
    n, din, hid, k, lam = 10, 4, 6, 2, 0.1
    A = rng.standard_normal((n, din))
    Qt = _orth(rng, n, k)
    prm = dict(W1=rng.standard_normal((din, hid)), b1=rng.standard_normal(hid) * 0.1,
               W2=rng.standard_normal((hid, k)), b2=rng.standard_normal(k) * 0.1)

    def loss(p):
        W, _ = O.warm_forward(A, p)
        return O.warm_loss(W, Qt, lam)

    W, cache = O.warm_forward(A, prm)
    grads = O.warm_backward(A, prm, cache, O.warm_loss_grad(W, Qt, lam))
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2"):
        fd = np.zeros_like(prm[name])
        for idx in np.ndindex(prm[name].shape):
            pp = {k_: v.copy() for k_, v in prm.items()}
            pm = {k_: v.copy() for k_, v in prm.items()}
            pp[name][idx] += h
            pm[name][idx] -= h
            fd[idx] = (loss(pp) - loss(pm)) / (2 * h)
        assert np.max(np.abs(grads[name] - fd)) < 1e-6 * max(1.0, np.max(np.abs(fd))), name


def test_adam_two_hand_worked_steps():
    prm = {"w": np.array([1.0, -2.0])}
    st = {}
    g1 = {"w": np.array([0.5, -4.0])}
    p1 = O.adam_step(prm, g1, st, lr=0.1)
    # step 1: m_hat = g, v_hat = g^2 -> update = lr * g / (|g| + eps)
    assert np.allclose(p1["w"], [1.0 - 0.1 * 0.5 / (0.5 + 1e-8), -2.0 + 0.1 * 4.0 / (4.0 + 1e-8)], rtol=0, atol=1e-15)
    g2 = {"w": np.array([1.0, 0.0])}
    p2 = O.adam_step(p1, g2, st, lr=0.1)
    m = 0.9 * 0.1 * np.array([0.5, -4.0]) + 0.1 * np.array([1.0, 0.0])
    v = 0.999 * 0.001 * np.array([0.25, 16.0]) + 0.001 * np.array([1.0, 0.0])
    mh, vh = m / (1 - 0.81), v / (1 - 0.999 ** 2)
    assert np.allclose(p2["w"], p1["w"] - 0.1 * mh / (np.sqrt(vh) + 1e-8), rtol=0, atol=1e-14)


def test_features_on_a_hand_built_graph():
    # path 0-1-2 plus isolated node 3: P_N = D^-1 A by hand
    row_ptr = np.array([0, 1, 3, 4, 4], np.int64)
    col = np.array([1, 0, 2, 1], np.int32)
    topo = O.Topology(dict(kind="graph", n=4, layers=[(row_ptr, col)]))
    X = np.array([[3.0, 4.0], [0.0, 2.0], [1.0, 0.0], [0.0, 0.0]])
    U = np.array([[0.6, 0.8], [0.0, 1.0], [1.0, 0.0], [0.0, 0.0]])
    PU = np.array([U[1], 0.5 * (U[0] + U[2]), U[1], [0.0, 0.0]])
    assert np.allclose(O.warm_features(topo, X), np.hstack([U, PU]), atol=1e-15)


def test_warm_initial_block_and_training_sanity():
    rng = np.random.default_rng(3)
    n, din, hid, k = 300, 8, 16, 3
    labels = rng.integers(0, k, n)
    A = np.eye(k)[labels] @ rng.standard_normal((k, din)) + 0.1 * rng.standard_normal((n, din))
    Qt = O.h_norm(labels, k)                      # target: the cluster indicator subspace
    prm0 = {k_: v.astype(np.float64) for k_, v in synth.warm_init(0, din, hid, k).items()}
    prm, losses = O.warm_train([(A, Qt)], prm0, epochs=300, lr=1e-2, lam=1e-3)
    assert losses[-1] < 0.1 * losses[0]
    W, _ = O.warm_forward(A, prm)
    Q0 = O.warm_initial_block(W)
    assert np.allclose(Q0.T @ Q0, np.eye(k + 1), atol=1e-12)
    assert np.allclose(np.abs(Q0[:, 0]), 1 / np.sqrt(n))
    assert O.max_principal_angle(np.hstack([np.ones((n, 1)), W]), Q0) < 1e-8
