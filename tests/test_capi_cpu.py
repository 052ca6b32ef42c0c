"""C ABI checks that need no GPU: the library builds, loads, exports every
function declared in include/ancka.h, and the ctypes mirrors of the structs
match the C layout (compiled with gcc from the header itself)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2408_05459_gb300 import ancka, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ancka.load()


def test_library_exports_every_declared_function(lib):
    names = ancka.header_functions()
    assert "ancka_knn" in names and "ancka_cluster" in names
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings_and_defaults(lib):
    assert lib.ancka_status_str(0) == b"ANCKA_OK"
    assert lib.ancka_status_str(1) == b"ANCKA_ERR_INVALID_ARG"
    p = ancka.default_params()
    assert (p.k, p.K, p.T, p.gamma, p.T_i, p.tau, p.disc_max_iter) == (5, 10, 10, 3, 25, 5, 20)
    assert abs(p.alpha - 0.2) < 1e-7 and abs(p.beta - 0.5) < 1e-7
    # exact KNN lists, the automatic node order, InitBCM, the fixed schedule
    assert (p.knn_nlist, p.knn_nprobe, p.node_order, p.init, p.early_stop) == (0, 0, 0, 0, 0)


def test_struct_layout_matches_header():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "ancka.h"
#define F(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
int main(void) {
  printf("ancka_topology %zu\nancka_params %zu\nancka_outputs %zu\nancka_info %zu\n",
         sizeof(ancka_topology), sizeof(ancka_params), sizeof(ancka_outputs), sizeof(ancka_info));
  F(ancka_topology, he_nodes); F(ancka_topology, m); F(ancka_params, init_labels);
  F(ancka_params, knn_prec); F(ancka_info, phi_best); F(ancka_info, ms_knn); F(ancka_info, ms_total);
  F(ancka_params, warm); F(ancka_params, knn_nlist); F(ancka_params, knn_nprobe); F(ancka_params, node_order);
  F(ancka_info, knn_tiles); F(ancka_info, knn_full_tiles);
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    vals = dict(line.split() for line in out if line.strip())
    assert int(vals["ancka_topology"]) == ctypes.sizeof(ancka.Topology)
    assert int(vals["ancka_params"]) == ctypes.sizeof(ancka.Params)
    assert int(vals["ancka_outputs"]) == ctypes.sizeof(ancka.Outputs)
    assert int(vals["ancka_info"]) == ctypes.sizeof(ancka.Info)
    assert int(vals["ancka_topology.he_nodes"]) == ancka.Topology.he_nodes.offset
    assert int(vals["ancka_topology.m"]) == ancka.Topology.m.offset
    assert int(vals["ancka_params.init_labels"]) == ancka.Params.init_labels.offset
    assert int(vals["ancka_params.knn_prec"]) == ancka.Params.knn_prec.offset
    assert int(vals["ancka_info.phi_best"]) == ancka.Info.phi_best.offset
    assert int(vals["ancka_info.ms_knn"]) == ancka.Info.ms_knn.offset
    assert int(vals["ancka_info.ms_total"]) == ancka.Info.ms_total.offset
    # the fields appended at the ends of the two structs
    for f in ("warm", "knn_nlist", "knn_nprobe", "node_order"):
        assert int(vals[f"ancka_params.{f}"]) == getattr(ancka.Params, f).offset, f
    for f in ("knn_tiles", "knn_full_tiles"):
        assert int(vals[f"ancka_info.{f}"]) == getattr(ancka.Info, f).offset, f


def test_oracle_and_cuda_path_are_independent():
    pkg = os.path.join(ROOT, "paper_2408_05459_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", text, re.M), f
    osrc = open(os.path.join(ROOT, "oracle", "ancka_oracle.py")).read()
    assert "paper_2408_05459_gb300" not in osrc


def test_no_gpu_means_an_error_not_a_host_fallback(lib):
    """Without a GPU the compute entry points return an error status (and the
    binding raises); nothing is computed on the host."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2408_05459_gb300 import synth
    assert lib.ancka_device_check() != 0
    assert lib.ancka_last_error()
    g = synth.config_small_sbm(0)
    with pytest.raises(ancka.AnckaError) as e:
        ancka.cluster_host(g, g["X"], ancka.default_params(k=5), stream=ctypes.c_void_p(0))
    assert e.value.status != 0
