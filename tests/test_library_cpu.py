"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, and
exports every entry point include/tc.h declares.  No compute call is made
(there may be no GPU)."""
from __future__ import annotations

import ctypes
import os
import json
import re

import pytest

import paper_2105_00110_gb300 as tcg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "tc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tc_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def built():
    return tcg.build()


def test_library_builds_for_sm103a(built):
    # the build records the nvcc command lines it ran; every translation
    # unit and the link name exactly one target, sm_103a
    assert os.path.exists(built)
    from paper_2105_00110_gb300.build import BUILD_INFO
    with open(BUILD_INFO) as fh:
        info = json.load(fh)
    cmds = info["compile"] + [info["link"]]
    assert len(info["compile"]) >= 3
    for cmd in cmds:
        i = cmd.index("-gencode")
        assert cmd[i + 1] == "arch=compute_103a,code=sm_103a"
        assert cmd.count("-gencode") == 1


def test_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    names = declared_symbols()
    assert {"tc_build_csr", "tc_count", "tc_centrality"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) <= set(tcg.EXPORTED)


def test_status_strings(built):
    assert tcg.status_str(tcg.TC_OK) == "ok"
    assert "argument" in tcg.status_str(tcg.TC_ERR_INVALID_ARG)
    assert tcg.status_str(12345) == "unknown status"


def test_host_argument_checks_reject_without_device(built):
    # Invalid sizes are rejected before any device work.
    lib = tcg.lib()
    h = ctypes.c_void_p()
    assert lib.tc_build_csr(None, None, -1, 5, 0, None, ctypes.byref(h)) == tcg.TC_ERR_INVALID_ARG
    assert lib.tc_build_csr(None, None, 3, 5, 0, None, ctypes.byref(h)) == tcg.TC_ERR_INVALID_ARG
    assert lib.tc_build_csr(None, None, 0, 2**31, 0, None, ctypes.byref(h)) == tcg.TC_ERR_INVALID_ARG
    assert lib.tc_build_csr(None, None, 0, 5, 64, None, ctypes.byref(h)) == tcg.TC_ERR_INVALID_ARG
    assert lib.tc_count(None, None, None, None, None) == tcg.TC_ERR_INVALID_ARG
    assert lib.tc_centrality(None, None, None, None, None) == tcg.TC_ERR_INVALID_ARG
    assert lib.tc_set_strategy(None, 0) == tcg.TC_ERR_INVALID_ARG
    assert lib.tc_divide(None, -1, 3, None, None) == tcg.TC_ERR_INVALID_ARG
    # dense-core setting: host only; the build flag that keeps unions of
    # graphs without a core is not a public flag
    assert lib.tc_set_dense_core(-2) == tcg.TC_ERR_INVALID_ARG
    assert lib.tc_set_dense_core(32769) == tcg.TC_ERR_INVALID_ARG
    for c in (0, 4096, 32768, -1):
        assert lib.tc_set_dense_core(c) == tcg.TC_OK
    assert lib.tc_build_csr(None, None, 0, 5, 1 << 30, None, ctypes.byref(h)) == tcg.TC_ERR_INVALID_ARG


def test_no_cpu_fallback():
    # The binding has no host compute path: without CUDA the call raises.
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(Exception):
        tcg.triangle_centrality(torch.tensor([0, 1, 2], dtype=torch.int32),
                                torch.tensor([1, 2, 0], dtype=torch.int32), 3)


def test_package_does_not_import_oracle():
    src_dir = os.path.join(ROOT, "paper_2105_00110_gb300")
    for dirpath, _, files in os.walk(src_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "tc_oracle" not in text and "og_" not in text, f
