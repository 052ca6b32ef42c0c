"""Discretize's k x k polar factor (Alg. 5, Eq. svd-in-discr) on the GPU
(FP32 Newton-Schulz, FP32 Jacobi SVD for a rank-deficient M) against the
oracle's FP64 SVD, through the C ABI (ancka_polar_factor)."""
import numpy as np
import pytest

from oracle import ancka_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# largest |R_gpu - R_fp64| entry accepted: the FP32 iteration stops once
# max |X^T X - I| < 1e-6 + 8 k 2^-24, and the rounding of M to FP32
# (2^-24 relative) moves the polar factor by at most ~2^-24 ||M|| / sigma_min
# per entry; at the planted blocks below sigma_min / ||M|| >= 1e-2
R_TOL = 2e-4


@pytest.fixture(scope="module")
def ak():
    from paper_2408_05459_gb300 import ancka
    ancka.load()
    return ancka


def _block(seed, n, k, noise=0.05, used=None, rotate=True):
    """Planted indicator rows of `used` clusters, rotated or not (with fewer
    clusters than columns and no rotation the last columns never win the
    argmax), plus noise."""
    rng = np.random.default_rng(seed)
    used = k if used is None else used
    truth = rng.integers(0, used, n)
    rot = np.linalg.qr(rng.standard_normal((k, k)))[0] if rotate else np.eye(k)
    return O.bcm(truth, k) @ rot * 0.3 + noise * rng.standard_normal((n, k))


def _first_step(Qk):
    """The oracle's first Discretize iteration (R = I): its labels, M and R."""
    labels, _, R = O.discretize(Qk, max_iter=1, return_trace=True)
    k = Qk.shape[1]
    nrm = np.sqrt(np.einsum("ij,ij->i", Qk, Qk))
    Qt = Qk / nrm[:, None]
    c = np.bincount(labels, minlength=k).astype(np.float64)
    Yt = O.bcm(labels, k) * np.where(c > 0, 1.0 / np.maximum(c, 1.0), 0.0)[None, :]
    return labels, Yt.T @ Qt, R


@pytest.mark.parametrize("k,rotate", [(5, True), (10, True), (20, True), (47, True), (64, False)])
def test_polar_factor_matches_fp64_svd(ak, k, rotate):
    Qk = _block(10 + k, 20000, k, rotate=rotate)
    _, M, R_o = _first_step(Qk)
    M32 = M.astype(np.float32)
    R_g, method = ak.polar_factor(torch.as_tensor(M32, device="cuda"))
    torch.cuda.synchronize()
    assert method == 0                               # Newton-Schulz settled
    R_g = R_g.cpu().numpy().astype(np.float64)
    err = np.max(np.abs(R_g - R_o))
    assert err <= R_TOL, err
    assert np.max(np.abs(R_g.T @ R_g - np.eye(k))) <= 1e-5


def test_polar_factor_of_the_bulk_column_block(ak):
    """M with one small singular value, as Discretize meets it on real blocks
    (one column of Q spans the bulk): still the FP64 polar factor."""
    k = 10
    rng = np.random.default_rng(3)
    U = np.linalg.qr(rng.standard_normal((k, k)))[0]
    V = np.linalg.qr(rng.standard_normal((k, k)))[0]
    sig = np.concatenate([np.linspace(1.0, 0.5, k - 1), [1e-2]])
    M = U @ np.diag(sig) @ V.T
    R_g, method = ak.polar_factor(torch.as_tensor(M.astype(np.float32), device="cuda"))
    R_g = R_g.cpu().numpy().astype(np.float64)
    assert method == 0
    assert np.max(np.abs(R_g - V @ U.T)) <= R_TOL


def test_polar_factor_with_an_empty_cluster(ak):
    """A zero row of M (an empty cluster, reading R12): the Jacobi path.  The
    factor is then unique only off the null direction, so the checks are the
    polar properties: R orthogonal and tr(M R) = the sum of the singular
    values (the Discretize objective)."""
    k = 12
    Qk = _block(5, 20000, k, noise=0.02, used=k - 1, rotate=False)
    labels, M, _ = _first_step(Qk)
    assert np.bincount(labels, minlength=k)[k - 1] == 0
    R_g, method = ak.polar_factor(torch.as_tensor(M.astype(np.float32), device="cuda"))
    R_g = R_g.cpu().numpy().astype(np.float64)
    assert method == 1
    assert np.max(np.abs(R_g.T @ R_g - np.eye(k))) <= 1e-5
    s = np.linalg.svd(M, compute_uv=False).sum()
    assert abs(np.trace(M @ R_g) - s) <= 1e-5 * s
