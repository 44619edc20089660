"""The C ABI: the library builds for sm_103a, loads, exports every symbol the
header declares, and rejects bad arguments on the host (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_2507_17094_gb300 as A
from paper_2507_17094_gb300.build import INCLUDE


def header_functions():
    text = open(os.path.join(INCLUDE, "ann.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ann_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def L():
    A.build()
    return A.lib()


def test_exports_every_declared_symbol(L):
    declared = header_functions()
    assert set(declared) == set(A.EXPORTS), declared
    for name in declared:
        assert hasattr(L, name), name


def test_params_struct_matches_defaults(L):
    assert C.sizeof(A.SearchParams) == 72
    p = A.make_params()
    assert (p.k, p.itopk, p.search_width, p.max_iters) == (10, 64, 1, 64)
    assert abs(p.dgs_cooldown - 0.3) < 1e-7 and p.ghost_max_iters == 16 and p.ghost_max_iters_given == 4


def test_host_side_validation(L):
    X = np.zeros((4, 8), np.float32)
    with pytest.raises(A.AnnError) as e:
        A.Index(X, np.full((4, 2), 9, np.uint32))            # neighbour id out of range
    assert e.value.status == 1
    with pytest.raises(A.AnnError) as e:
        A.Index(X, np.zeros((4, 2), np.uint32), ghost_ids=np.array([2, 1], np.uint32),
                ghost_graph=np.zeros((2, 1), np.uint32))      # ghost ids not ascending
    assert e.value.status == 1
    assert L.ann_search(None, None, 0, None, None, 0, None, None, None, None) == 1
    assert L.ann_index_load(b"/nonexistent/file", 0, 0, 1, 1, C.byref(C.c_void_p())) == 4
