"""Python binding of ``libancka.so`` (the C ABI in ``include/ancka.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device buffers are torch tensors (PyTorch supplies device memory
and the current stream); host entry points take numpy arrays.  If the
library is missing the first call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libancka.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "ancka.h")

PREC = {"fp32": 0, "bf16": 1, "fp8": 2}
KIND = {"graph": 0, "hypergraph": 1, "multiplex": 2}
MAX_TRACE = 64


class Topology(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("L", ctypes.c_int32), ("n", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("nnz", ctypes.c_int64),
                ("directed", ctypes.c_int32), ("pad_", ctypes.c_int32), ("m", ctypes.c_int64),
                ("he_ptr", ctypes.c_void_p), ("he_nodes", ctypes.c_void_p)]


class WarmModel(ctypes.Structure):
    _fields_ = [("d_in", ctypes.c_int32), ("hidden", ctypes.c_int32), ("k", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("W1", ctypes.c_void_p), ("b1", ctypes.c_void_p),
                ("W2", ctypes.c_void_p), ("b2", ctypes.c_void_p)]


class WarmGraph(ctypes.Structure):
    _fields_ = [("topo", ctypes.POINTER(Topology)), ("X", ctypes.c_void_p), ("Qt", ctypes.c_void_p),
                ("d", ctypes.c_int32), ("pad_", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("K", ctypes.c_int32), ("alpha", ctypes.c_float),
                ("beta", ctypes.c_float), ("T", ctypes.c_int32), ("gamma", ctypes.c_int32),
                ("T_i", ctypes.c_int32), ("tau", ctypes.c_int32), ("disc_max_iter", ctypes.c_int32),
                ("knn_prec", ctypes.c_int32), ("init", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("init_labels", ctypes.c_void_p), ("early_stop", ctypes.c_int32), ("eps_Q", ctypes.c_float),
                ("warm", ctypes.POINTER(WarmModel)), ("knn_nlist", ctypes.c_int32), ("knn_nprobe", ctypes.c_int32),
                ("node_order", ctypes.c_int32)]


class Outputs(ctypes.Structure):
    _fields_ = [("Q", ctypes.c_void_p), ("init_labels", ctypes.c_void_p),
                ("knn_idx", ctypes.c_void_p), ("knn_sim", ctypes.c_void_p)]


class Info(ctypes.Structure):
    _fields_ = [("knn_candidates", ctypes.c_int64), ("knn_fallback_rows", ctypes.c_int64),
                ("knn_exhaustive_rows", ctypes.c_int64),
                ("iters_run", ctypes.c_int32), ("n_phi", ctypes.c_int32),
                ("phi", ctypes.c_double * MAX_TRACE), ("disc_iters", ctypes.c_int32 * MAX_TRACE),
                ("taken", ctypes.c_int32 * MAX_TRACE), ("phi_best", ctypes.c_double),
                ("numeric_flags", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("ms_knn", ctypes.c_float), ("ms_build", ctypes.c_float), ("ms_init", ctypes.c_float),
                ("ms_iter", ctypes.c_float), ("ms_disc", ctypes.c_float), ("ms_mhc", ctypes.c_float),
                ("ms_total", ctypes.c_float), ("ms_contract", ctypes.c_float),
                ("ms_rerank", ctypes.c_float), ("ms_spmm", ctypes.c_float),
                ("warm_used", ctypes.c_int32), ("pad2_", ctypes.c_int32),
                ("knn_tiles", ctypes.c_int64), ("knn_full_tiles", ctypes.c_int64)]

    def to_dict(self) -> dict:
        n = self.n_phi
        return dict(knn_candidates=self.knn_candidates, knn_fallback_rows=self.knn_fallback_rows,
                    knn_exhaustive_rows=self.knn_exhaustive_rows,
                    iters_run=self.iters_run, n_phi=n, phi=list(self.phi[:n]), disc_iters=list(self.disc_iters[:n]),
                    taken=list(self.taken[:n]), phi_best=self.phi_best, numeric_flags=self.numeric_flags,
                    ms_knn=self.ms_knn, ms_build=self.ms_build, ms_init=self.ms_init, ms_iter=self.ms_iter,
                    ms_disc=self.ms_disc, ms_mhc=self.ms_mhc, ms_total=self.ms_total,
                    ms_contract=self.ms_contract, ms_rerank=self.ms_rerank,
                    ms_spmm=self.ms_spmm, warm_used=self.warm_used, knn_tiles=self.knn_tiles,
                    knn_full_tiles=self.knn_full_tiles)


class AnckaError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__(f"{fn} -> status {status}: {msg}")
        self.status = status


_lib = None


def header_functions() -> list[str]:
    """Names of the functions declared in include/ancka.h."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ancka_[a-z0-9_]+)\s*\(", src)))


def load(path: str = LIB_PATH):
    """Load the library and declare the signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run paper_2408_05459_gb300.build.build() first "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    L.ancka_params_default.argtypes = [ctypes.POINTER(Params)]
    L.ancka_params_default.restype = None
    L.ancka_status_str.argtypes = [ctypes.c_int]
    L.ancka_status_str.restype = ctypes.c_char_p
    L.ancka_last_error.argtypes = []
    L.ancka_last_error.restype = ctypes.c_char_p
    L.ancka_device_check.argtypes = []
    L.ancka_device_check.restype = ctypes.c_int
    L.ancka_kernel_launches.argtypes = []
    L.ancka_kernel_launches.restype = ctypes.c_int64
    L.ancka_set_symmetric_knn_min_rows.argtypes = [ctypes.c_int64]
    L.ancka_set_symmetric_knn_min_rows.restype = None
    L.ancka_knn.argtypes = [vp, i64, i32, i32, i32, vp, vp, ctypes.POINTER(Info), vp]
    L.ancka_knn.restype = ctypes.c_int
    L.ancka_knn_candidates.argtypes = [vp, i64, i32, i32, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_float), vp]
    L.ancka_knn_candidates.restype = ctypes.c_int
    L.ancka_warm_predict.argtypes = [ctypes.POINTER(Topology), vp, i32, ctypes.POINTER(WarmModel), vp, vp]
    L.ancka_warm_predict.restype = ctypes.c_int
    L.ancka_warm_train.argtypes = [ctypes.POINTER(WarmGraph), i32, i32, ctypes.c_float, ctypes.c_float,
                                   ctypes.POINTER(WarmModel), ctypes.POINTER(ctypes.c_float), vp]
    L.ancka_warm_train.restype = ctypes.c_int
    L.ancka_warm_gradients.argtypes = [ctypes.POINTER(WarmGraph), ctypes.c_float, ctypes.POINTER(WarmModel),
                                       vp, vp, vp, vp, ctypes.POINTER(ctypes.c_double), vp]
    L.ancka_warm_gradients.restype = ctypes.c_int
    L.ancka_cluster.argtypes = [ctypes.POINTER(Topology), vp, i32, ctypes.POINTER(Params), vp,
                                ctypes.POINTER(Outputs), ctypes.POINTER(Info), vp]
    L.ancka_cluster.restype = ctypes.c_int
    L.ancka_cluster_with_knn.argtypes = [ctypes.POINTER(Topology), vp, i32, vp, vp, ctypes.POINTER(Params),
                                         vp, ctypes.POINTER(Outputs), ctypes.POINTER(Info), vp]
    L.ancka_cluster_with_knn.restype = ctypes.c_int
    L.ancka_cluster_host.argtypes = [ctypes.POINTER(Topology), vp, i32, ctypes.POINTER(Params), vp,
                                     ctypes.POINTER(Info), vp]
    L.ancka_cluster_host.restype = ctypes.c_int
    L.ancka_discretize.argtypes = [vp, i64, i32, i32, i32, vp, ctypes.POINTER(i32), vp]
    L.ancka_discretize.restype = ctypes.c_int
    L.ancka_discretize_noalloc.argtypes = [vp, i64, i32, i32, i32, vp, ctypes.POINTER(i32), vp]
    L.ancka_discretize_noalloc.restype = ctypes.c_int
    L.ancka_knn_ivf.argtypes = [vp, i64, i32, i32, i32, i32, vp, vp, ctypes.POINTER(Info), vp]
    L.ancka_knn_ivf.restype = ctypes.c_int
    L.ancka_polar_factor.argtypes = [vp, i32, vp, ctypes.POINTER(i32), vp]
    L.ancka_polar_factor.restype = ctypes.c_int
    _lib = L
    return L


def _check(fn: str, status: int):
    if status != 0:
        L = load()
        raise AnckaError(fn, status, f"{L.ancka_status_str(status).decode()}: {L.ancka_last_error().decode()}")


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def kernel_launches() -> int:
    """Kernels this library has launched in this process so far."""
    return int(load().ancka_kernel_launches())


def set_symmetric_knn_min_rows(n_min: int) -> None:
    """BF16 KNN lists of inputs with at least n_min rows come from the
    symmetric contraction (1 = always; the default, 2**63 - 1, never)."""
    load().ancka_set_symmetric_knn_min_rows(int(n_min))


def default_params(**kw) -> Params:
    p = Params()
    load().ancka_params_default(ctypes.byref(p))
    for key, v in kw.items():
        if key == "knn_prec" and isinstance(v, str):
            v = PREC[v]
        setattr(p, key, v)
    return p


# ----------------------------------------------------------------------------
# device entry points (torch tensors)
# ----------------------------------------------------------------------------
def knn(X, K: int, prec: str = "bf16", with_info: bool = True):
    """N_K lists (n x K int32) and cosines (n x K float32) of the rows of X."""
    import torch
    assert X.is_cuda and X.dtype == torch.float32 and X.is_contiguous()
    n, d = X.shape
    idx = torch.empty((n, K), dtype=torch.int32, device=X.device)
    sim = torch.empty((n, K), dtype=torch.float32, device=X.device)
    info = Info()
    st = load().ancka_knn(_ptr(X), n, d, K, PREC[prec], _ptr(idx), _ptr(sim),
                          ctypes.byref(info) if with_info else None, _stream())
    _check("ancka_knn", st)
    return idx, sim, (info.to_dict() if with_info else None)


def knn_ivf(X, K: int, nlist: int, nprobe: int, with_info: bool = True):
    """Approximate N_K lists by inverted lists (ancka_knn_ivf): (idx, sim, info)."""
    import torch
    assert X.is_cuda and X.dtype == torch.float32 and X.is_contiguous()
    n, d = X.shape
    idx = torch.empty((n, K), dtype=torch.int32, device=X.device)
    sim = torch.empty((n, K), dtype=torch.float32, device=X.device)
    info = Info()
    st = load().ancka_knn_ivf(_ptr(X), n, d, K, nlist, nprobe, _ptr(idx), _ptr(sim),
                              ctypes.byref(info) if with_info else None, _stream())
    _check("ancka_knn_ivf", st)
    return idx, sim, (info.to_dict() if with_info else None)


def knn_candidates(X, prec: str = "bf16"):
    """Diagnostic: the contraction's candidate lists before the exact re-rank
    (n x 32 scores and keys, two 16-entry lists per row), the quantised unit
    rows (n x d), the per-row error bounds (n) and the accumulation bound."""
    import torch
    assert X.is_cuda and X.dtype == torch.float32 and X.is_contiguous()
    n, d = X.shape
    cv = torch.empty((n, 32), dtype=torch.float32, device=X.device)
    ci = torch.empty((n, 32), dtype=torch.int32, device=X.device)
    q = torch.empty((n, d), dtype=torch.float32, device=X.device)
    err = torch.empty(n, dtype=torch.float32, device=X.device)
    acc = ctypes.c_float(0.0)
    st = load().ancka_knn_candidates(_ptr(X), n, d, PREC[prec], _ptr(cv), _ptr(ci), _ptr(q), _ptr(err),
                                     ctypes.byref(acc), _stream())
    _check("ancka_knn_candidates", st)
    return cv, ci, q, err, acc.value


def topology_to_device(g: dict, device="cuda"):
    """Copy a generator/numpy topology dict to device tensors (kept alive in the dict)."""
    import torch
    out = dict(kind=g["kind"], n=int(g["n"]), directed=int(g.get("directed", 0)))
    if g["kind"] == "hypergraph":
        out["he_ptr"] = torch.as_tensor(np.ascontiguousarray(g["he_ptr"], np.int64), device=device)
        out["he_nodes"] = torch.as_tensor(np.ascontiguousarray(g["he_nodes"], np.int32), device=device)
        out["m"] = int(len(g["he_ptr"]) - 1)
    else:
        n = int(g["n"])
        rps, cols, off = [], [], 0
        for rp, col in g["layers"]:
            rps.append(np.asarray(rp, np.int64) + off)
            cols.append(np.asarray(col, np.int32))
            off += len(col)
        out["row_ptr"] = torch.as_tensor(np.concatenate(rps), device=device)
        out["col_idx"] = torch.as_tensor(np.concatenate(cols) if cols else np.zeros(0, np.int32), device=device)
        out["L"] = len(g["layers"])
        out["nnz"] = int(off)
        assert out["row_ptr"].numel() == out["L"] * (n + 1)
    return out


def _topology_struct(t: dict) -> Topology:
    s = Topology()
    s.kind = KIND[t["kind"]]
    s.n = t["n"]
    s.directed = t.get("directed", 0)
    if t["kind"] == "hypergraph":
        s.L = 1
        s.m = t["m"]
        s.he_ptr = t["he_ptr"].data_ptr()
        s.he_nodes = t["he_nodes"].data_ptr()
    else:
        s.L = t["L"]
        s.row_ptr = t["row_ptr"].data_ptr()
        s.col_idx = t["col_idx"].data_ptr() if t["nnz"] > 0 else None
        s.nnz = t["nnz"]
    return s


def warm_model(weights: dict) -> tuple:
    """ctypes model over device tensors W1 (d_in x 256), b1, W2 (256 x k), b2
    (float32, contiguous; kept referenced by the caller)."""
    W1, b1, W2, b2 = (weights[k_] for k_ in ("W1", "b1", "W2", "b2"))
    for t in (W1, b1, W2, b2):
        assert t.is_cuda and t.is_contiguous() and t.dtype.is_floating_point and t.element_size() == 4
    m = WarmModel(d_in=W1.shape[0], hidden=W1.shape[1], k=W2.shape[1], W1=W1.data_ptr(), b1=b1.data_ptr(),
                  W2=W2.data_ptr(), b2=b2.data_ptr())
    return m


def warm_predict(topo_dev: dict, X, weights: dict):
    """W = MLP([U | P_N U]) (n x k) of the learned warm start."""
    import torch
    n, d = X.shape
    m = warm_model(weights)
    W = torch.empty((n, m.k), dtype=torch.float32, device=X.device)
    ts = _topology_struct(topo_dev)
    st = load().ancka_warm_predict(ctypes.byref(ts), _ptr(X), d, ctypes.byref(m), _ptr(W), _stream())
    _check("ancka_warm_predict", st)
    return W


def _warm_graphs(items):
    keep, arr = [], (WarmGraph * len(items))()
    for q, (topo_dev, X, Qt) in enumerate(items):
        assert Qt.is_cuda and Qt.is_contiguous() and Qt.dtype == X.dtype
        ts = _topology_struct(topo_dev)
        keep.append(ts)
        arr[q].topo = ctypes.pointer(ts)
        arr[q].X = X.data_ptr()
        arr[q].Qt = Qt.data_ptr()
        arr[q].d = X.shape[1]
    return arr, keep


def warm_train(items, weights: dict, epochs: int, lr: float = 1e-3, lam: float = 1e-3):
    """Trains the warm-start MLP in place on [(topo_dev, X, Qt)]; returns the
    loss before every step (epochs x graphs, graph order fixed)."""
    arr, keep = _warm_graphs(items)
    m = warm_model(weights)
    losses = (ctypes.c_float * (epochs * len(items)))()
    st = load().ancka_warm_train(arr, len(items), epochs, lr, lam, ctypes.byref(m), losses, _stream())
    _check("ancka_warm_train", st)
    return np.array(losses[:], np.float64)


def warm_gradients(topo_dev: dict, X, Qt, weights: dict, lam: float = 1e-3):
    """Gradients of the warm-start loss for one graph (no update) and the loss."""
    import torch
    arr, keep = _warm_graphs([(topo_dev, X, Qt)])
    m = warm_model(weights)
    dev = X.device
    g = dict(W1=torch.empty((m.d_in, 256), dtype=torch.float32, device=dev),
             b1=torch.empty(256, dtype=torch.float32, device=dev),
             W2=torch.empty((256, m.k), dtype=torch.float32, device=dev),
             b2=torch.empty(m.k, dtype=torch.float32, device=dev))
    loss = ctypes.c_double(0.0)
    st = load().ancka_warm_gradients(arr, lam, ctypes.byref(m), _ptr(g["W1"]), _ptr(g["b1"]), _ptr(g["W2"]),
                                     _ptr(g["b2"]), ctypes.byref(loss), _stream())
    _check("ancka_warm_gradients", st)
    return g, loss.value


def cluster(topo_dev: dict, X, params: Params | None = None, knn_lists=None, want_Q=False,
            want_init=False, want_knn=False, with_info=True, init_labels=None, warm=None):
    """Algorithm 4 on device buffers; returns (labels, extras dict, info dict).
    warm: device weights of the warm-start MLP (init = 2, InitBCM fallback)."""
    import torch
    n, d = X.shape
    p = params or default_params()
    if init_labels is not None:
        p.init = 1
        p.init_labels = init_labels.data_ptr()
    wm = None
    if warm is not None:
        wm = warm_model(warm)
        p.init = 2
        p.warm = ctypes.pointer(wm)
    labels = torch.empty(n, dtype=torch.int32, device=X.device)
    extras = {}
    o = Outputs()
    if want_Q:
        extras["Q"] = torch.empty((n, p.k + 1), dtype=torch.float32, device=X.device)
        o.Q = extras["Q"].data_ptr()
    if want_init:
        extras["init_labels"] = torch.empty(n, dtype=torch.int32, device=X.device)
        o.init_labels = extras["init_labels"].data_ptr()
    if want_knn and knn_lists is None:
        extras["knn_idx"] = torch.empty((n, p.K), dtype=torch.int32, device=X.device)
        extras["knn_sim"] = torch.empty((n, p.K), dtype=torch.float32, device=X.device)
        o.knn_idx = extras["knn_idx"].data_ptr()
        o.knn_sim = extras["knn_sim"].data_ptr()
    ts = _topology_struct(topo_dev)
    info = Info()
    ip = ctypes.byref(info) if with_info else None
    if knn_lists is None:
        st = load().ancka_cluster(ctypes.byref(ts), _ptr(X), d, ctypes.byref(p), _ptr(labels), ctypes.byref(o),
                                  ip, _stream())
        _check("ancka_cluster", st)
    else:
        ki, ks = knn_lists
        st = load().ancka_cluster_with_knn(ctypes.byref(ts), _ptr(X), d, _ptr(ki), _ptr(ks), ctypes.byref(p),
                                           _ptr(labels), ctypes.byref(o), ip, _stream())
        _check("ancka_cluster_with_knn", st)
    return labels, extras, (info.to_dict() if with_info else None)


def cluster_host(g: dict, X: np.ndarray, params: Params | None = None, with_info=True, stream=None):
    """Algorithm 4 on host numpy buffers (copies happen inside the library)."""
    X = np.ascontiguousarray(X, np.float32)
    n, d = X.shape
    p = params or default_params()
    keep = []
    s = Topology()
    s.kind = KIND[g["kind"]]
    s.n = n
    s.directed = int(g.get("directed", 0))
    if g["kind"] == "hypergraph":
        hp = np.ascontiguousarray(g["he_ptr"], np.int64)
        hn = np.ascontiguousarray(g["he_nodes"], np.int32)
        keep += [hp, hn]
        s.L = 1
        s.m = len(hp) - 1
        s.he_ptr = hp.ctypes.data
        s.he_nodes = hn.ctypes.data
    elif "row_ptr" in g:  # layers already in the ABI's layout (e.g. pinned host buffers)
        rp = g["row_ptr"]
        ci = g["col_idx"]
        assert rp.dtype == np.int64 and ci.dtype == np.int32 and rp.flags.c_contiguous and ci.flags.c_contiguous
        s.L = int(g["L"])
        assert rp.size == s.L * (n + 1)
        s.row_ptr = rp.ctypes.data
        s.col_idx = ci.ctypes.data if ci.size else None
        s.nnz = ci.size
    else:
        rps, cols, off = [], [], 0
        for rp, col in g["layers"]:
            rps.append(np.asarray(rp, np.int64) + off)
            cols.append(np.asarray(col, np.int32))
            off += len(col)
        rp = np.ascontiguousarray(np.concatenate(rps))
        ci = np.ascontiguousarray(np.concatenate(cols))
        keep += [rp, ci]
        s.L = len(g["layers"])
        s.row_ptr = rp.ctypes.data
        s.col_idx = ci.ctypes.data
        s.nnz = off
    labels = np.empty(n, np.int32)
    info = Info()
    st = load().ancka_cluster_host(ctypes.byref(s), X.ctypes.data, d, ctypes.byref(p), labels.ctypes.data,
                                   ctypes.byref(info) if with_info else None,
                                   stream if stream is not None else _stream())
    _check("ancka_cluster_host", st)
    del keep
    return labels, (info.to_dict() if with_info else None)


def discretize(Qk, max_iter: int = 20):
    """Discretize (Alg. 5) of an n x k device block; returns (labels, iterations)."""
    import torch
    assert Qk.is_cuda and Qk.dtype == torch.float32 and Qk.stride(1) == 1
    n, k = Qk.shape
    labels = torch.empty(n, dtype=torch.int32, device=Qk.device)
    it = ctypes.c_int32(0)
    st = load().ancka_discretize(_ptr(Qk), n, k, Qk.stride(0), max_iter, _ptr(labels), ctypes.byref(it), _stream())
    _check("ancka_discretize", st)
    return labels, it.value


def polar_factor(M):
    """ancka_polar_factor: R = V U^T of a k x k device matrix M = U Omega V^T
    by Discretize's own device routines; returns (R, method) with method 0 =
    Newton-Schulz, 1 = Jacobi."""
    import torch
    assert M.is_cuda and M.dtype == torch.float32 and M.dim() == 2 and M.shape[0] == M.shape[1]
    M = M.contiguous()
    k = M.shape[0]
    R = torch.empty_like(M)
    method = ctypes.c_int32(-1)
    st = load().ancka_polar_factor(_ptr(M), k, _ptr(R), ctypes.byref(method), _stream())
    _check("ancka_polar_factor", st)
    return R, method.value


def discretize_noalloc(Qk, labels, max_iter: int = 20):
    """ancka_discretize_noalloc: Discretize into a caller-owned ``labels``
    buffer using the library's fixed device scratch (no allocation inside the
    call).  Returns the number of inner iterations."""
    import torch
    assert Qk.is_cuda and Qk.dtype == torch.float32 and Qk.stride(1) == 1
    assert labels.is_cuda and labels.dtype == torch.int32 and labels.numel() == Qk.shape[0]
    n, k = Qk.shape
    it = ctypes.c_int32(0)
    st = load().ancka_discretize_noalloc(_ptr(Qk), n, k, Qk.stride(0), max_iter, _ptr(labels),
                                         ctypes.byref(it), _stream())
    _check("ancka_discretize_noalloc", st)
    return it.value
