"""ancka_discretize_noalloc (the Discretize entry point for callers that must
not allocate device memory while they run) against ancka_discretize.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _block(seed, n, k):
    rng = np.random.default_rng(seed)
    truth = rng.integers(0, k, n)
    rot = np.linalg.qr(rng.standard_normal((k, k)))[0]
    Q = np.eye(k)[truth] @ rot * 0.3 + 0.05 * rng.standard_normal((n, k))
    return torch.as_tensor(Q.astype(np.float32), device="cuda")


def test_noalloc_matches_discretize_on_two_calls_in_a_row():
    from paper_2408_05459_gb300 import ancka
    ancka.load()
    labels = torch.empty(30000, dtype=torch.int32, device="cuda")
    for seed, (n, k) in [(1, (30000, 10)), (2, (20000, 7))]:
        Q = _block(seed, n, k)
        ref, ref_it = ancka.discretize(Q)
        out = labels[:n]
        it = ancka.discretize_noalloc(Q, out)
        torch.cuda.synchronize()
        # same kernels on the same input: identical labels and iteration count
        assert it == ref_it
        assert torch.equal(out, ref)


def test_noalloc_rejects_blocks_beyond_the_fixed_scratch():
    from paper_2408_05459_gb300 import ancka
    ancka.load()
    n, k = 300000, 64                        # ~77 MB of scratch > 32 MiB
    Q = torch.zeros((n, k), dtype=torch.float32, device="cuda")
    labels = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(ancka.AnckaError) as e:
        ancka.discretize_noalloc(Q, labels)
    assert e.value.status == 1 and "scratch" in str(e.value)
