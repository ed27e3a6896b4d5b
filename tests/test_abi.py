"""The C-ABI library builds for sm_103a and exports every symbol hss.h declares.

No CUDA call is made (this runs without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hss.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hss_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__ as g
    g.build()
    from paper_1503_05464_gb300 import build
    return build.LIB


def test_header_declares_the_entry_points():
    names = _declared()
    for want in ("hss_compress", "hss_matvec", "hss_factor", "hss_solve", "hss_info",
                 "hss_destroy", "hss_last_error", "hss_sample", "hss_random_gaussian",
                 "hss_id_batched", "hss_node_ranks", "hss_default_opts"):
        assert want in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\b[TW] (hss_[a-z_0-9]+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_ctypes_binding_loads_without_gpu(lib_path):
    from paper_1503_05464_gb300 import hss
    L = hss.load(lib_path)
    for name in hss.EXPORTS:
        assert hasattr(L, name)
    o = hss.hss_default_opts(rtol=1e-4, sample_mode="tf32")
    assert o.leaf_size == 128 and o.rtol == 1e-4 and o.sample_mode == 1
