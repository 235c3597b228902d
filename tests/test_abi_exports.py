"""The C-ABI library builds, loads without a GPU and exports every function
include/sgc.h declares (no compute calls: only the version and the default
options, which touch no device)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sgc.h")).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)          # drop comments
    text = re.sub(r"#[^\n]*", " ", text)                          # and preprocessor lines
    names = set()
    for decl in re.findall(r"[^;{}]+\([^;{}]*\)\s*;", text):     # prototypes end in ");"
        m = re.search(r"(\w+)\s*\([^()]*(?:\([^()]*\)[^()]*)*\)\s*;\s*$", decl.strip())
        if m and not decl.strip().startswith("typedef"):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2507_21253_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_path():
    names = declared_functions()
    for n in ("csr_cluster_build", "spgemm_symbolic", "spgemm_numeric", "spgemm_rowwise_symbolic",
              "spgemm_rowwise_numeric", "hcluster_reorder", "cluster_variable_length", "spgemm_learned_phase1",
              "spgemm_graph_create", "nnz_predictor_train", "nnz_predictor_save", "nnz_predictor_load",
              "sgc_fp64_rate", "csr_cluster_build_count_noalloc"):
        assert n in names
    assert len(names) >= 30


def test_every_declared_function_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared in include/sgc.h but not exported: {missing}"


def test_version_and_default_options(lib):
    lib.sgc_abi_version.restype = ctypes.c_int
    text = open(os.path.join(ROOT, "include", "sgc.h")).read()
    assert lib.sgc_abi_version() == int(re.search(r"#define SGC_ABI_VERSION (\d+)", text).group(1))
    opts = (ctypes.c_int32 * 16)()
    assert lib.sgc_default_options(ctypes.byref(opts)) == 0
