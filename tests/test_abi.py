"""The C-ABI library loads, exports every function that include/pdx.h
declares, agrees with the binding on struct layouts, and rejects bad
arguments before touching a GPU (none of these tests makes a compute call)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2503_04422_gb300 import build as pbuild
from paper_2503_04422_gb300 import pdx as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pdx.h")


@pytest.fixture(scope="module")
def L():
    pbuild.build()
    return P.lib()


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(pdx_[a-z_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_five_calls_and_helpers():
    names = _declared_functions()
    for n in ("pdx_build_layout", "pdx_ivf_build", "pdx_search_exact", "pdx_search_ivf", "pdx_free",
              "pdx_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(L):
    for n in _declared_functions():
        assert hasattr(L, n), n


def test_struct_layouts_match_c(tmp_path):
    prog = tmp_path / "sizes.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "pdx.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(pdx_build_opts), sizeof(pdx_ivf_opts),"
        " sizeof(pdx_search_opts), sizeof(pdx_search_stats), sizeof(pdx_index_info),"
        " offsetof(pdx_search_opts, mlp_ncentroids), offsetof(pdx_ivf_opts, init_centroids));"
        "printf(\"%zu %zu\\n\", sizeof(pdx_server_opts), sizeof(pdx_server_info_t));"
        "printf(\"%zu %zu %zu\\n\", offsetof(pdx_search_opts, engine), offsetof(pdx_build_opts, dense_rows),"
        " offsetof(pdx_search_stats, dense_fallbacks));"
        "printf(\"%zu %zu %zu %zu\\n\", offsetof(pdx_search_opts, tau_init), offsetof(pdx_search_opts, tau_fixed),"
        " offsetof(pdx_ivf_opts, rotation_seed), offsetof(pdx_search_stats, phase_ns));"
        "printf(\"%zu %zu %zu\\n\", offsetof(pdx_search_opts, layout), offsetof(pdx_build_opts, keep_dsm),"
        " offsetof(pdx_build_opts, start_clusters));"
        "printf(\"%zu %zu %zu\\n\", offsetof(pdx_build_opts, cs_first_step), offsetof(pdx_search_opts, finished_log),"
        " offsetof(pdx_search_opts, finished_cap));return 0;}\n")
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(P.pdx_build_opts), ctypes.sizeof(P.pdx_ivf_opts), ctypes.sizeof(P.pdx_search_opts),
            ctypes.sizeof(P.pdx_search_stats), ctypes.sizeof(P.pdx_index_info),
            P.pdx_search_opts.mlp_ncentroids.offset, P.pdx_ivf_opts.init_centroids.offset,
            ctypes.sizeof(P.pdx_server_opts), ctypes.sizeof(P.pdx_server_info_t),
            P.pdx_search_opts.engine.offset, P.pdx_build_opts.dense_rows.offset,
            P.pdx_search_stats.dense_fallbacks.offset, P.pdx_search_opts.tau_init.offset,
            P.pdx_search_opts.tau_fixed.offset, P.pdx_ivf_opts.rotation_seed.offset,
            P.pdx_search_stats.phase_ns.offset, P.pdx_search_opts.layout.offset, P.pdx_build_opts.keep_dsm.offset,
            P.pdx_build_opts.start_clusters.offset, P.pdx_build_opts.cs_first_step.offset,
            P.pdx_search_opts.finished_log.offset, P.pdx_search_opts.finished_cap.offset]
    assert got == want


def test_defaults(L):
    o = P.pdx_search_opts()
    L.pdx_default_search_opts(ctypes.byref(o))
    assert o.struct_size == ctypes.sizeof(P.pdx_search_opts)
    assert o.pruner == P.PRUNER["bond"] and o.first_step == 4 and o.means_scope == 2
    assert abs(o.selection_threshold - 0.20) < 1e-7 and abs(o.eps0 - 2.1) < 1e-6
    b = P.pdx_build_opts()
    L.pdx_default_build_opts(ctypes.byref(b))
    assert b.partition_size == 10000 and b.metric == 0 and b.dense_rows == 0
    assert o.engine == P.ENGINE["auto"]


def test_argument_errors_without_gpu(L):
    out = ctypes.c_void_p(123)
    # NULL vectors / output handle
    assert L.pdx_build_layout(None, 10, 4, None, None, ctypes.byref(out)) == P.PDX_ERR_ARG
    assert out.value is None
    assert "NULL" in P.pdx_last_error()
    x = (ctypes.c_float * 8)()
    assert L.pdx_build_layout(ctypes.addressof(x), 2, 0, None, None, ctypes.byref(out)) == P.PDX_ERR_ARG
    assert L.pdx_build_layout(ctypes.addressof(x), 2, 5000, None, None, ctypes.byref(out)) == P.PDX_ERR_ARG
    bad = P.pdx_build_opts()
    bad.struct_size = 4
    assert L.pdx_build_layout(ctypes.addressof(x), 2, 4, ctypes.byref(bad), None, ctypes.byref(out)) == P.PDX_ERR_ARG
    # searches on a NULL index
    d = (ctypes.c_float * 4)()
    i = (ctypes.c_int64 * 4)()
    assert L.pdx_search_exact(None, ctypes.addressof(x), 1, 4, None, ctypes.addressof(d), ctypes.addressof(i),
                              None) == P.PDX_ERR_ARG
    assert L.pdx_search_ivf(None, ctypes.addressof(x), 1, 4, 1, None, ctypes.addressof(d), ctypes.addressof(i),
                            None) in (P.PDX_ERR_ARG, P.PDX_ERR_UNSUPPORTED)
    L.pdx_free(None)  # NULL-safe
    assert L.pdx_index_info_get(None, None) == P.PDX_ERR_ARG
