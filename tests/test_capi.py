"""The C ABI library: builds for sm_103a, loads, and exports every function that
include/sced.h declares (no compute call; runs without a GPU)."""
import os
import re

import paper_1804_05028_gb300 as ed

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "sced.h")


def declared_functions():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ed_\w+)\s*\(", src, flags=re.M)))


def test_library_builds_and_exports_every_declared_symbol():
    ed.build()
    L = ed.lib()
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n
    assert sorted(ed.SYMBOLS) == names
    assert L.ed_version().decode().startswith("sced")


def test_error_path_without_device():
    # validation runs on the host before any CUDA call: a bad descriptor is refused
    import ctypes
    import numpy as np
    with_err = None
    try:
        ed.build_basis(n_sites=65, n_sublat=1, bonds=np.array([[0, 1]]), bond_class=[0],
                       n_classes=1, perm=np.zeros((1, 65), np.int32), phase_num=[0],
                       phase_denom=1, n_up=1, stream=0)
    except ed.EdError as e:
        with_err = e
    assert with_err is not None and with_err.code == 1 and "n_sites" in str(with_err)
