"""The C-ABI library loads and exports every symbol include/colden.h declares
(no GPU needed: nothing here launches work)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1410_0624_gb300 import _build, colden

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(cd_[a-z_0-9]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return colden.load()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert "cd_column_density" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (cd_[a-z_0-9]+)", out))
    assert declared <= exported, declared - exported
    assert declared == set(colden.EXPORTS)
    for name in declared:
        assert getattr(lib, name) is not None


def test_opts_default_and_errors_without_gpu(lib):
    o = colden.opts_default()
    assert o.precision == colden.FP32
    assert abs(o.av_per_nh * 1.87e21 - 1.0) < 1e-15 and o.shield_k == 2.5
    h = ctypes.c_void_p()
    # argument checks run before any device work
    assert lib.cd_build_tree_uniform(0, 1.0, None, 1, None, ctypes.byref(h)) == colden.CD_EINVAL
    assert b"leaf_level" in lib.cd_last_error()
    assert lib.cd_build_tree_uniform(3, -1.0, None, 1, None, ctypes.byref(h)) == colden.CD_EINVAL
    assert lib.cd_precompute_geometry(0, 1, 0, None, 0, 7, None, ctypes.byref(h)) == colden.CD_EINVAL
    assert b"mode" in lib.cd_last_error()
    assert lib.cd_precompute_geometry(99, 1, 0, None, 0, 0, None, ctypes.byref(h)) == colden.CD_EINVAL
    assert lib.cd_column_density(None, None, None, None, None, None, None) == colden.CD_EINVAL
    assert lib.cd_stats_get(len(colden.KERNEL_KINDS), None, None) == colden.CD_EINVAL


def test_no_oracle_in_product_path():
    pkg = os.path.join(ROOT, "paper_1410_0624_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "liboracle" not in src, f


def test_checked_entry_points_refuse_in_the_normal_build(lib):
    site, index = ctypes.c_int(), ctypes.c_int64()
    assert lib.cd_checked_status(ctypes.byref(site), ctypes.byref(index)) == colden.CD_EUNSUPPORTED
    assert lib.cd_debug_check_probe(ctypes.c_int64(9), None) == colden.CD_EUNSUPPORTED
