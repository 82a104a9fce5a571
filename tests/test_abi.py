"""The C-ABI library builds, loads and exports every entry point of
include/acr.h; its host-side block structure equals the oracle's (integer
index work: compared exactly).  No CUDA compute call is made here."""
import os
import re

import numpy as np
import pytest

from oracle.hstructure import Structure

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1712_08872_gb300 import _build, acr
    _build.build()
    return acr.load_library()


def header_functions():
    txt = open(os.path.join(ROOT, "include", "acr.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(acr_\w+)\s*\(", txt, flags=re.M)))


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert "acr_setup" in names and "acr_apply_transpose" in names and len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name


def test_missing_library_fails_loudly(tmp_path):
    from paper_1712_08872_gb300 import acr
    saved = acr._lib
    acr._lib = None
    try:
        with pytest.raises(ImportError):
            acr.load_library(str(tmp_path / "nope.so"))
    finally:
        acr._lib = saved


@pytest.mark.parametrize("n,eta,leaf", [(16, 1.0, 32), (16, 2.0, 16), (32, 2.0, 64),
                                        (64, 2.0, 64), (32, 16.0, 64), (12, 2.0, 20)])
def test_structure_equals_oracle(lib, n, eta, leaf):
    from paper_1712_08872_gb300 import acr_structure_query
    counts, leaves, perm = acr_structure_query(n, eta, leaf, with_leaves=True)
    st = Structure(n, eta, leaf)
    assert list(perm) == st.perm
    mine = sorted(map(tuple, leaves.tolist()))
    ref = sorted((st.clusters[a].begin, st.clusters[a].size, st.clusters[b].begin,
                  st.clusters[b].size, 1 if k == "L" else 0) for a, b, k in st.leaves())
    assert mine == ref
    assert counts[0] == len(st.clusters)
    assert counts[1] == sum(1 for *_, k in st.leaves() if k == "D")
    assert counts[2] == sum(1 for *_, k in st.leaves() if k == "L")


def test_structure_query_rejects_bad_arguments(lib):
    import ctypes
    counts = (ctypes.c_int64 * 6)()
    assert lib.acr_structure_query(0, 2.0, 32, counts, None, None) == 1
    assert lib.acr_structure_query(16, -1.0, 32, counts, None, None) == 1
    assert lib.acr_structure_query(16, 2.0, 0, counts, None, None) == 1
