"""The C-ABI library on the CPU: it builds, loads, exports every symbol that
include/dade.h declares, rejects invalid arguments before any GPU work, and
its host-side FP64 eigensolver (the PCA step of Section 3.2, Eq. 11) is
correct.  No GPU compute is called here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2411_17229_gb300 import build as libbuild
from paper_2411_17229_gb300 import dade

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    libbuild.build()
    return dade.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dade.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dade_[a-z_0-9]+)\s*\(", src)))


def test_header_and_binding_agree():
    names = declared_functions()
    assert len(names) >= 15
    assert set(names) == set(dade.SIGNATURES), set(names) ^ set(dade.SIGNATURES)


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L, name), name
    assert b"sm_103a" in L.dade_version()


def _c_layouts(tmp_path):
    """sizeof / offsetof of every field of the ABI structs, from a C program
    compiled against include/dade.h with the host C compiler."""
    structs = {"dade_build_opts": dade.BuildOpts, "dade_search_opts": dade.SearchOpts, "dade_info": dade.Info,
               "dade_server_opts": dade.ServerOpts, "dade_hnsw_build_opts": dade.HnswBuildOpts,
               "dade_hnsw_search_opts": dade.HnswSearchOpts, "dade_hnsw_info": dade.HnswInfo}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dade.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            cname, f, v = line.split()
            got[(cname, f)] = int(v)
    return structs, got


def test_struct_layouts_match_header(L, tmp_path):
    structs, got = _c_layouts(tmp_path)
    for cname, py in structs.items():
        assert C.sizeof(py) == got[(cname, "size")], cname
        for f, _ in py._fields_:
            assert getattr(py, f).offset == got[(cname, f)], (cname, f)


def test_invalid_arguments_rejected_without_gpu(L):
    o = dade.BuildOpts()
    L.dade_build_opts_default(C.byref(o))
    assert o.kmeans_iters == 10 and o.eps_pairs == 100000
    h = C.c_void_p()
    x = np.zeros((4, 8), np.float32)
    assert L.dade_build_index(x.ctypes.data, 1, 8, C.byref(o), C.byref(h), None) == dade.EINVAL
    assert b"n < 2" in L.dade_last_error()
    assert L.dade_build_index(x.ctypes.data, 4, 0, C.byref(o), C.byref(h), None) == dade.EINVAL
    assert L.dade_build_index(x.ctypes.data, 4, 2048, C.byref(o), C.byref(h), None) == dade.EINVAL
    o.n_clusters = 5
    assert L.dade_build_index(x.ctypes.data, 4, 8, C.byref(o), C.byref(h), None) == dade.EINVAL
    assert L.dade_build_index(None, 4, 8, C.byref(o), C.byref(h), None) == dade.EINVAL
    ids = np.zeros(10, np.int64)
    dists = np.zeros(10, np.float32)
    assert L.dade_search(None, x.ctypes.data, 1, 10, 1, 0.1, 32, None, ids.ctypes.data, dists.ctypes.data,
                         None) == dade.EINVAL
    assert L.dade_sync(None, None) == dade.EINVAL
    assert L.dade_free_index(None) is None


def test_hnsw_arguments_rejected_without_gpu(L):
    o = dade.HnswBuildOpts()
    L.dade_hnsw_build_opts_default(C.byref(o))
    assert (o.M, o.M0, o.kc, o.nprobe) == (16, 32, 64, 0)
    so = dade.HnswSearchOpts()
    L.dade_hnsw_search_opts_default(C.byref(so))
    assert so.mode == dade.MODE_DADE and so.max_visits == 0 and not so.entry and not so.coef
    h = C.c_void_p()
    x = np.zeros((4, 8), np.float32)
    nbr = np.zeros((4, 2), np.int32)
    assert L.dade_hnsw_build(None, x.ctypes.data, 4, C.byref(o), C.byref(h)) == dade.EINVAL
    for n, d, m0, entry, msg in ((0, 8, 2, 0, b"n outside"), (4, 0, 2, 0, b"d outside"),
                                 (4, 8, 33, 0, b"m0 outside"), (4, 8, 2, 4, b"entry outside")):
        assert L.dade_hnsw_create(None, x.ctypes.data, n, d, nbr.ctypes.data, m0, entry, C.byref(h)) == dade.EINVAL
        assert msg in L.dade_last_error()
    ids, dists = np.zeros(10, np.int64), np.zeros(10, np.float32)
    assert L.dade_hnsw_search(None, x.ctypes.data, 1, 10, 10, 0.1, 16, None, ids.ctypes.data, dists.ctypes.data,
                              None) == dade.EINVAL
    assert L.dade_hnsw_free(None) is None


def test_lead_options_rejected_without_gpu(L):
    h = C.c_void_p()
    x = np.zeros((64, 40), np.float32)
    for fmt, dims, msg in ((7, 16, b"lead_format"), (dade.LEAD_NONE, 16, b"lead_dims"),
                           (dade.LEAD_BF16, 0, b"lead_dims"), (dade.LEAD_BF16, 24, b"lead_dims"),
                           (dade.LEAD_FP8, 64, b"lead_dims")):   # D = 40 pads to 48
        o = dade.BuildOpts()
        L.dade_build_opts_default(C.byref(o))
        o.n_clusters, o.lead_format, o.lead_dims = 2, fmt, dims
        assert L.dade_build_index(x.ctypes.data, 64, 40, C.byref(o), C.byref(h), None) == dade.EINVAL
        assert msg in L.dade_last_error()


@pytest.mark.parametrize("n", [1, 2, 3, 7, 16, 64, 129])
def test_host_eigensolver_vs_lapack(L, n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    A = A + A.T
    w, v = dade.host_sym_eig(A)
    ref = np.sort(np.linalg.eigvalsh(A))[::-1]
    assert np.allclose(w, ref, atol=1e-12 * max(1.0, np.abs(ref).max()))
    assert np.all(np.diff(w) <= 0)
    assert np.allclose(v.T @ v, np.eye(n), atol=1e-12)
    assert np.allclose(A @ v, v * w[None, :], atol=1e-11 * max(1.0, np.abs(ref).max()))


def test_host_eigensolver_degenerate_and_diagonal(L):
    A = np.diag([3.0, 1.0, 3.0, 2.0, 0.0])
    w, v = dade.host_sym_eig(A)
    assert np.allclose(w, [3, 3, 2, 1, 0])
    assert np.allclose(A @ v, v * w[None, :], atol=1e-14)
    B = np.ones((6, 6))
    w, v = dade.host_sym_eig(B)
    assert np.allclose(w, [6, 0, 0, 0, 0, 0], atol=1e-12)
    assert np.allclose(B @ v, v * w[None, :], atol=1e-12)


def test_load_rejects_foreign_files_without_gpu(L, tmp_path):
    h = C.c_void_p()
    assert L.dade_load_index(str(tmp_path / "none.dade").encode(), C.byref(h)) == dade.EIO
    junk = tmp_path / "junk.dade"
    junk.write_bytes(bytes(range(256)) * 4)
    assert L.dade_load_index(str(junk).encode(), C.byref(h)) == dade.EINVAL
    assert b"not a libdade index file" in L.dade_last_error()
    hdr = tmp_path / "hdr.dade"    # right magic and version, impossible dimension
    hdr.write_bytes(b"DADEIX01" + (1).to_bytes(4, "little") + (0x01020304).to_bytes(4, "little") + bytes(72))
    assert L.dade_load_index(str(hdr).encode(), C.byref(h)) == dade.EINVAL
    assert b"header out of range" in L.dade_last_error()
    assert not h.value
