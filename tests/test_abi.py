"""The C ABI without a GPU: the library loads, exports every entry point include/hom.h
declares, and rejects invalid arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import microstructure as ms

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hom.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hom_[a-z_]+)\s*\(", src)))


def test_header_symbols_exported():
    H = pytest.importorskip("paper_1508_02045_gb300")
    lib = ctypes.CDLL(H.LIB_PATH)
    names = declared_functions()
    assert "hom_create" in names and "hom_solve" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) <= set(H.EXPORTED)


def test_invalid_arguments_rejected_on_host():
    H = pytest.importorskip("paper_1508_02045_gb300")
    ph = ms.box_phase((9, 9), 0.6)
    mat = H.phase_material(ph, ms.isotropic_table([1.0, 10.0], 2))
    for d, N in [(2, (8, 9)), (4, (9, 9, 9, 9)), (2, (1, 9)), (2, (9, 9001))]:
        with pytest.raises(H.HomError) as ei:
            H.hom_create(d, N, mat, stream=0)
        assert ei.value.status == H.HOM_ERR_INVALID
    fm = H.fourier_material(np.zeros((17, 17), complex), 1.0, 10.0)
    with pytest.raises(H.HomError) as ei:
        H.hom_create(2, (9, 9), fm, H.HOM_APPROX, stream=0)
    assert ei.value.status == H.HOM_ERR_INVALID
    # exact integration of an image takes scalar coefficients only: a tensor table is refused
    # before the device is touched
    tmat = H.phase_material(ph, ms.random_spd_table(2, 2, seed=1, scales=[1.0, 10.0]))
    with pytest.raises(H.HomError) as ei:
        H.hom_create(2, (9, 9), tmat, H.HOM_EXACT, stream=0)
    assert ei.value.status == H.HOM_ERR_UNSUPPORTED


def test_strerror():
    H = pytest.importorskip("paper_1508_02045_gb300")
    assert H.hom_strerror(0) == "ok"
    assert "unsupported" in H.hom_strerror(H.HOM_ERR_UNSUPPORTED)
