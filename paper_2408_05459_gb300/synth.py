"""Seeded synthetic attributed networks shaped like the ANCKA workloads.

This module only draws inputs: it holds none of the clustering arithmetic, so
both the CUDA path and the FP64 oracle can be fed from it.  Every generator is
deterministic in its ``seed`` and returns a plain dict of numpy arrays:

``kind``      "graph" | "hypergraph" | "multiplex"
``n``, ``k``  number of nodes and of planted clusters
``X``         float32 n x d attribute matrix (row-major)
``labels``    int32 planted cluster of every node (context only)
graph / multiplex:  ``layers`` = list of (row_ptr int64[n+1], col int32[nnz]),
                    each layer a symmetric, duplicate-free, loop-free adjacency
hypergraph:         ``he_ptr`` int64[m+1], ``he_nodes`` int32[nnz]
                    (members of every hyperedge, no repeats)

Node ids are randomly permuted after generation so that no locality is handed
to the kernels.  The shapes follow the workloads the paper evaluates on
(Section 8: co-authorship / keyword hypergraphs, large co-purchase graphs,
multiplex academic graphs); the datasets themselves are not used.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "sbm_graph", "hypergraph_tfidf", "multiplex_sbm", "dcsbm_graph",
    "cliques_closed_form", "gaussian_mixture", "csr_from_edges",
    "config_small_sbm", "config_hypergraph", "config_multiplex", "config_large_dcsbm",
]


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------
def csr_from_edges(n: int, src: np.ndarray, dst: np.ndarray, symmetric: bool = True):
    """Binary CSR adjacency from an edge list: drops self loops and repeats.

    With ``symmetric`` every edge is stored in both directions.  Column indices
    are sorted inside each row.
    """
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    if symmetric:
        src, dst = np.concatenate([src, dst]), np.concatenate([dst, src])
    key = np.sort(src * n + dst)     # sorted unique keys (same result as np.unique, faster here)
    if key.size:
        first = np.empty(key.size, bool)
        first[0] = True
        np.not_equal(key[1:], key[:-1], out=first[1:])
        key = key[first]
    rows = key // n
    cols = (key % n).astype(np.int32)
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, cols


def _permute_graph(perm_new_of_old, row_ptr, col):
    """Relabel node ids of a CSR adjacency with the permutation old -> new."""
    n = row_ptr.shape[0] - 1
    rows_old = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    return csr_from_edges(n, perm_new_of_old[rows_old], perm_new_of_old[col.astype(np.int64)],
                          symmetric=False)


def gaussian_mixture(rng: np.random.Generator, labels: np.ndarray, k: int, d: int,
                     sigma: float) -> np.ndarray:
    """x_v = mu_{c(v)} + sigma * eps, mu_c ~ N(0, I_d), eps ~ N(0, I_d); float32."""
    mu = rng.standard_normal((k, d))
    X = mu[labels] + sigma * rng.standard_normal((labels.shape[0], d))
    return X.astype(np.float32)


def _block_pair_edges(rng, sizes, p_in, p_out):
    """Undirected SBM edges by sampling each block pair's edge count first.

    Endpoints are drawn uniformly inside the two blocks; repeated pairs are
    removed later by ``csr_from_edges`` (negligible at these densities).
    """
    k = len(sizes)
    starts = np.concatenate([[0], np.cumsum(sizes)])
    src, dst = [], []
    for a in range(k):
        for b in range(a, k):
            if a == b:
                pairs = sizes[a] * (sizes[a] - 1) // 2
                p = p_in
            else:
                pairs = sizes[a] * sizes[b]
                p = p_out
            cnt = rng.binomial(pairs, p) if pairs > 0 else 0
            if cnt == 0:
                continue
            src.append(starts[a] + rng.integers(0, sizes[a], cnt))
            dst.append(starts[b] + rng.integers(0, sizes[b], cnt))
    if not src:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(src), np.concatenate(dst)


# ----------------------------------------------------------------------------
# generators
# ----------------------------------------------------------------------------
def sbm_graph(n: int, k: int, p_in: float, p_out: float, d: int, sigma: float,
              seed: int) -> dict:
    """Undirected attributed SBM with k equal clusters and Gaussian-mixture X."""
    rng = np.random.default_rng(seed)
    sizes = np.full(k, n // k, np.int64)
    sizes[: n - sizes.sum()] += 1
    lab_sorted = np.repeat(np.arange(k), sizes)
    src, dst = _block_pair_edges(rng, sizes, p_in, p_out)
    perm = rng.permutation(n)  # old id -> new id
    row_ptr, col = csr_from_edges(n, perm[src], perm[dst], symmetric=True)
    labels = np.empty(n, np.int32)
    labels[perm] = lab_sorted
    X = gaussian_mixture(rng, labels, k, d, sigma)
    return dict(kind="graph", n=n, k=k, X=X, labels=labels, layers=[(row_ptr, col)])


def multiplex_sbm(n: int, k: int, mean_degree: float, ratios, d: int, sigma: float,
                  seed: int) -> dict:
    """L SBM layers over one node set; layer l has p_in/p_out = ratios[l].

    For block size c the per-layer probabilities give the requested mean degree:
    p_out = deg / (r (c - 1) + (n - c)), p_in = r p_out.
    """
    rng = np.random.default_rng(seed)
    sizes = np.full(k, n // k, np.int64)
    sizes[: n - sizes.sum()] += 1
    c = float(sizes[0])
    lab_sorted = np.repeat(np.arange(k), sizes)
    perm = rng.permutation(n)
    layers = []
    for r in ratios:
        p_out = mean_degree / (r * (c - 1.0) + (n - c))
        p_in = r * p_out
        src, dst = _block_pair_edges(rng, sizes, p_in, p_out)
        layers.append(csr_from_edges(n, perm[src], perm[dst], symmetric=True))
    labels = np.empty(n, np.int32)
    labels[perm] = lab_sorted
    X = gaussian_mixture(rng, labels, k, d, sigma)
    return dict(kind="multiplex", n=n, k=k, X=X, labels=labels, layers=layers)


def _zipf_probs(v: int, s: float) -> np.ndarray:
    p = 1.0 / np.arange(1, v + 1, dtype=np.float64) ** s
    return p / p.sum()


def hypergraph_tfidf(n: int, k: int, m: int, d: int, nnz_per_row: int, seed: int,
                     size_min: int = 2, size_max: int = 20, size_exp: float = 2.5,
                     p_home: float = 0.85, zipf_s: float = 1.1,
                     p_cluster_words: float = 0.7) -> dict:
    """Attributed hypergraph with planted clusters and TF-IDF-like attributes.

    Hyperedge sizes s in [size_min, size_max] with P(s) ~ s^-size_exp.  Each
    hyperedge picks a home cluster with probability proportional to its size
    and each member is in the home cluster w.p. ``p_home``, else uniform over
    the other clusters; members do not repeat.  Every node draws
    ``nnz_per_row`` distinct words from 0.7 * (cluster-specific Zipf over a
    per-cluster word permutation) + 0.3 * (background Zipf), term counts
    1 + Poisson(0.5), weighted by log(n / df).  Rows are never all-zero.
    """
    rng = np.random.default_rng(seed)
    sizes_c = np.full(k, n // k, np.int64)
    sizes_c[: n - sizes_c.sum()] += 1
    starts = np.concatenate([[0], np.cumsum(sizes_c)])
    lab_sorted = np.repeat(np.arange(k), sizes_c).astype(np.int32)

    # hyperedge sizes
    s_vals = np.arange(size_min, size_max + 1)
    ps = s_vals.astype(np.float64) ** (-size_exp)
    ps /= ps.sum()
    esz = rng.choice(s_vals, size=m, p=ps)
    home = rng.choice(k, size=m, p=sizes_c / sizes_c.sum())
    # draw members: oversample then dedupe per hyperedge
    total = int(esz.sum())
    eid = np.repeat(np.arange(m), esz)
    in_home = rng.random(total) < p_home
    other = rng.integers(0, k - 1, total) if k > 1 else np.zeros(total, np.int64)
    hc = home[eid]
    clus = np.where(in_home | (k == 1), hc, other + (other >= hc))
    node = starts[clus] + (rng.random(total) * sizes_c[clus]).astype(np.int64)
    # remove repeated members inside a hyperedge
    key = np.unique(eid.astype(np.int64) * n + node)
    eid_u = key // n
    node_u = key % n
    perm = rng.permutation(n)
    node_u = perm[node_u]
    cnt = np.bincount(eid_u, minlength=m)
    he_ptr = np.zeros(m + 1, np.int64)
    np.cumsum(cnt, out=he_ptr[1:])
    # sort members inside each hyperedge by their new id
    order = np.lexsort((node_u, eid_u))
    he_nodes = node_u[order].astype(np.int32)

    labels = np.empty(n, np.int32)
    labels[perm] = lab_sorted

    # attributes
    base = _zipf_probs(d, zipf_s)
    bg_perm = rng.permutation(d)
    bg = np.empty(d)
    bg[bg_perm] = base
    word_p = np.empty((k, d))
    for c in range(k):
        cp = np.empty(d)
        cp[rng.permutation(d)] = base
        word_p[c] = p_cluster_words * cp + (1.0 - p_cluster_words) * bg
    logp = np.log(word_p).astype(np.float32)
    X = np.zeros((n, d), np.float32)
    chunk = 20000
    cols_all = np.empty((n, nnz_per_row), np.int64)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        g = rng.gumbel(size=(e - s, d)).astype(np.float32)
        keys = logp[labels[s:e]] + g
        cols_all[s:e] = np.argpartition(-keys, nnz_per_row - 1, axis=1)[:, :nnz_per_row]
    tf = 1.0 + rng.poisson(0.5, size=(n, nnz_per_row))
    df = np.bincount(cols_all.ravel(), minlength=d).astype(np.float64)
    idf = np.log(n / np.maximum(df, 1.0))
    vals = (tf * idf[cols_all]).astype(np.float32)
    rows = np.repeat(np.arange(n), nnz_per_row)
    X[rows, cols_all.ravel()] = vals.ravel()
    zero = ~np.any(X != 0, axis=1)
    if zero.any():  # every row keeps at least one non-zero
        X[np.nonzero(zero)[0], cols_all[zero, 0]] = 1.0
    return dict(kind="hypergraph", n=n, k=k, X=X, labels=labels, he_ptr=he_ptr,
                he_nodes=he_nodes, m=m)


def dcsbm_graph(n: int, k: int, m_edges: int, d: int, sigma: float, seed: int,
                deg_exp: float = 2.5, in_frac: float = 0.8) -> dict:
    """Degree-corrected SBM: power-law propensities, Zipf(1) cluster sizes.

    Propensities theta_v ~ power law with exponent ``deg_exp`` (minimum 1,
    capped at sqrt(2 m)).  A fraction ``in_frac`` of edges is drawn inside a
    cluster (cluster chosen proportional to its squared theta mass, endpoints
    proportional to theta), the rest between any two nodes proportional to
    theta.  Self loops and repeats are dropped.
    """
    rng = np.random.default_rng(seed)
    w = 1.0 / np.arange(1, k + 1)
    sizes = np.maximum(1, np.floor(n * w / w.sum())).astype(np.int64)
    sizes[0] += n - sizes.sum()
    lab_sorted = np.repeat(np.arange(k), sizes).astype(np.int32)
    u = rng.random(n)
    theta = (1.0 - u) ** (-1.0 / (deg_exp - 1.0))
    theta = np.minimum(theta, np.sqrt(2.0 * m_edges))
    starts = np.concatenate([[0], np.cumsum(sizes)])
    mass = np.array([theta[starts[c]:starts[c + 1]].sum() for c in range(k)])
    m_in = int(round(in_frac * m_edges))
    m_out = m_edges - m_in
    pc = mass ** 2 / (mass ** 2).sum()
    ecl = rng.choice(k, size=m_in, p=pc)
    src = np.empty(m_in, np.int64)
    dst = np.empty(m_in, np.int64)
    for c in range(k):
        sel = np.nonzero(ecl == c)[0]
        if sel.size == 0:
            continue
        cdf = np.cumsum(theta[starts[c]:starts[c + 1]])
        cdf /= cdf[-1]
        src[sel] = starts[c] + np.searchsorted(cdf, rng.random(sel.size), side="right")
        dst[sel] = starts[c] + np.searchsorted(cdf, rng.random(sel.size), side="right")
    gcdf = np.cumsum(theta)
    gcdf /= gcdf[-1]
    src2 = np.searchsorted(gcdf, rng.random(m_out), side="right")
    dst2 = np.searchsorted(gcdf, rng.random(m_out), side="right")
    src = np.minimum(np.concatenate([src, src2]), n - 1)
    dst = np.minimum(np.concatenate([dst, dst2]), n - 1)
    perm = rng.permutation(n)
    row_ptr, col = csr_from_edges(n, perm[src], perm[dst], symmetric=True)
    labels = np.empty(n, np.int32)
    labels[perm] = lab_sorted
    X = gaussian_mixture(rng, labels, k, d, sigma)
    return dict(kind="graph", n=n, k=k, X=X, labels=labels, layers=[(row_ptr, col)])


def cliques_closed_form(k: int, c: int, seed: int, d: int | None = None) -> dict:
    """k disjoint cliques of c nodes; attributes identical inside a clique and
    orthogonal one-hot vectors across cliques (the closed-form test case)."""
    rng = np.random.default_rng(seed)
    n = k * c
    d = k if d is None else d
    lab_sorted = np.repeat(np.arange(k), c)
    src, dst = [], []
    for a in range(k):
        ii, jj = np.triu_indices(c, 1)
        src.append(a * c + ii)
        dst.append(a * c + jj)
    src = np.concatenate(src)
    dst = np.concatenate(dst)
    perm = rng.permutation(n)
    row_ptr, col = csr_from_edges(n, perm[src], perm[dst], symmetric=True)
    labels = np.empty(n, np.int32)
    labels[perm] = lab_sorted
    X = np.zeros((n, d), np.float32)
    X[np.arange(n), labels] = 1.0
    return dict(kind="graph", n=n, k=k, X=X, labels=labels, layers=[(row_ptr, col)])


# ----------------------------------------------------------------------------
# the workload configurations (sizes from the method's evaluation settings)
# ----------------------------------------------------------------------------
def config_small_sbm(seed: int = 0) -> dict:
    """Undirected attributed SBM: n=2000, k=5, p_in=0.01, p_out=0.001, d=128, sigma=1.5."""
    return sbm_graph(2000, 5, 0.01, 0.001, 128, 1.5, seed)


def config_hypergraph(seed: int = 0, n: int = 100_000, m: int = 200_000) -> dict:
    """Attributed hypergraph: n=1e5, k=10, m=2e5, sizes 2..20, d=500 at 2% density."""
    return hypergraph_tfidf(n, 10, m, 500, 10, seed)


def config_multiplex(seed: int = 0, n: int = 500_000) -> dict:
    """Multiplex: L=3 SBM layers, n=5e5, k=20, mean degree 20, ratios 8/4/2, d=256."""
    return multiplex_sbm(n, 20, 20.0, (8.0, 4.0, 2.0), 256, 2.0, seed)


def config_large_dcsbm(seed: int = 0, n: int = 2_400_000, m_edges: int = 60_000_000,
                       k: int = 47, d: int = 100) -> dict:
    """Large DC-SBM graph: n=2.4e6, 6e7 edges, k=47 Zipf-sized clusters, d=100."""
    return dcsbm_graph(n, k, m_edges, d, 1.5, seed)


def warm_init(seed: int, d_in: int, hidden: int, k: int) -> dict:
    """Seeded initial weights of the warm-start MLP (d_in -> hidden -> k):
    W1 ~ N(0, 2/d_in), W2 ~ N(0, 1/hidden), zero biases; float32."""
    rng = np.random.default_rng(seed)
    return dict(W1=(rng.standard_normal((d_in, hidden)) * np.sqrt(2.0 / d_in)).astype(np.float32),
                b1=np.zeros(hidden, np.float32),
                W2=(rng.standard_normal((hidden, k)) * np.sqrt(1.0 / hidden)).astype(np.float32),
                b2=np.zeros(k, np.float32))
