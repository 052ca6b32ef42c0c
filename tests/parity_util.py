"""Comparison rules of the GPU path against the FP64 oracle.

KNN: index lists bit-exact with the (similarity desc, index asc) order, except
rows whose oracle K-th and (K+1)-th similarities differ by less than 1e-6
relative ("near-tie" rows, counted; their lists must still be valid within
that tolerance).  Similarities within 1e-6 absolute of the oracle's.
Iteration: largest principal angle <= 1e-3 rad, labels ARI >= 0.99.
"""
import numpy as np

from oracle import ancka_oracle as O

NEAR_TIE_REL = 1e-6
SIM_ABS = 1e-6
ANGLE_MAX = 1e-3
ARI_MIN = 0.99


def compare_knn(X, K, rows, gpu_idx, gpu_sim):
    """Returns a dict of counts; asserts the rule on every row."""
    rows = np.asarray(rows)
    o_idx, o_sim = O.knn_cosine(X, K, rows=rows, extra=1)
    g_idx = np.asarray(gpu_idx)[rows].astype(np.int64)
    g_sim = np.asarray(gpu_sim)[rows].astype(np.float64)
    Xn = O.unit_rows(X)
    kth, nxt = o_sim[:, K - 1], o_sim[:, K]
    tie = (kth - nxt) < NEAR_TIE_REL * np.maximum(np.abs(kth), 1e-300)
    exact_rows = ordered_rows = 0
    for r in range(rows.size):
        i = rows[r]
        true_sims = Xn[g_idx[r]] @ Xn[i]
        assert np.all(g_idx[r] != i), f"row {i}: self in list"
        assert len(set(g_idx[r].tolist())) == K, f"row {i}: repeated neighbour"
        assert np.all(np.abs(g_sim[r] - true_sims) <= SIM_ABS), f"row {i}: similarity off"
        if tie[r]:
            # valid list under the tolerance: nothing below the K-th value - tol
            assert np.all(true_sims >= kth[r] - NEAR_TIE_REL * max(abs(kth[r]), 1e-300) - 1e-12), f"row {i}"
            continue
        assert set(g_idx[r].tolist()) == set(o_idx[r].tolist()), f"row {i}: KNN set differs"
        exact_rows += 1
        gaps = -np.diff(o_sim[r, :K])
        if np.all(gaps >= NEAR_TIE_REL * np.maximum(np.abs(o_sim[r, :K - 1]), 1e-300)) or np.all(gaps == 0):
            assert np.array_equal(g_idx[r], o_idx[r]), f"row {i}: order differs"
            ordered_rows += 1
    return dict(rows=int(rows.size), near_tie_rows=int(tie.sum()), exact_rows=exact_rows,
                ordered_rows=ordered_rows)


def compare_iteration(o_res, labels, Q=None):
    ari = O.adjusted_rand_index(np.asarray(labels), o_res["labels"])
    ang = None
    if Q is not None:
        ang = O.max_principal_angle(np.asarray(Q, np.float64), o_res["Q"])
    return ari, ang
