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
    assert C.sizeof(A.SearchParams) == 88
    p = A.make_params()
    assert (p.k, p.itopk, p.search_width, p.max_iters) == (10, 64, 1, 64)
    assert abs(p.dgs_cooldown - 0.3) < 1e-7 and p.ghost_max_iters == 16 and p.ghost_max_iters_given == 4
    assert p.ghost_search_width == 1 and p.dgs_min_match == 0.0 and p.ghost_judge == 0.0


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


def test_mlp_file_errors_on_host(L, tmp_path):
    """ann_mlp_load checks the file before it touches a device."""
    h = C.c_void_p()
    assert L.ann_mlp_load(b"/nonexistent/mlp.bin", 0, 8, C.byref(h)) == 4
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"NOTANMLP" + np.array([8, 8, 8, 8], np.uint32).tobytes())
    assert L.ann_mlp_load(str(bad).encode(), 0, 8, C.byref(h)) == 1
    short = tmp_path / "short.bin"
    short.write_bytes(b"ANNMLP01" + np.array([8, 8, 8, 8], np.uint32).tobytes() + b"\0" * 40)
    assert L.ann_mlp_load(str(short).encode(), 0, 8, C.byref(h)) == 4
    odd = tmp_path / "odd.bin"
    odd.write_bytes(b"ANNMLP01" + np.array([8, 12, 8, 8], np.uint32).tobytes())
    assert L.ann_mlp_load(str(odd).encode(), 0, 8, C.byref(h)) == 1
    assert not h.value
    assert L.ann_mlp_save(None, b"x") == 1
