"""CPU checks of the C-ABI library: it loads without a GPU, exports every symbol the
header declares, and its own quadrature agrees with the oracle's."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char)\s*\*?\s*(lbm_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1405_1253_b300 import build
    build.build()
    from paper_1405_1253_b300 import lbm
    return lbm


def test_library_exports_every_declared_symbol(lib):
    names = header_symbols()
    assert len(names) >= 17
    cdll = ctypes.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(cdll, n), n
    assert set(names) == set(lib.exported_symbols())


def test_library_quadrature_matches_oracle(lib):
    c, w, r = lib.lattice()
    oc, _ = oracle.velocities()
    ow, orr = oracle.weights()
    np.testing.assert_array_equal(c, oc)
    assert abs(r - orr) < 1e-15
    np.testing.assert_allclose(w, ow, rtol=1e-14)


def test_create_rejects_bad_arguments_without_a_gpu(lib):
    ctx = ctypes.c_void_p()
    rc = lib._lib.lbm_create(ctypes.byref(ctx), 0, 128, 0, 0.8, 1e-4, None, None, 0, None)
    assert rc == lib.LBM_EINVAL and not ctx.value
    assert b"Lx" in lib._lib.lbm_last_error()
    rc = lib._lib.lbm_create(ctypes.byref(ctx), 8, 16, 0, 0.4, 1e-4, None, None, 0, None)
    assert rc == lib.LBM_EINVAL and b"tau" in lib._lib.lbm_last_error()
    rc = lib._lib.lbm_create(ctypes.byref(ctx), 8, 16, 9, 0.8, 1e-4, None, None, 0, None)
    assert rc == lib.LBM_EINVAL
    assert lib._lib.lbm_destroy(None) == lib.LBM_OK


def test_precision_numbering_matches_header(lib):
    """The storage precisions keep the numbering the boundary fixes: LBM_F64 = 0,
    LBM_F32 = 1 and LBM_F32_DEV = 2 (FP32 deviation storage); the float-float FP64 form
    sits after them.  The binding's table must say the same, and other values are refused."""
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    m = re.search(r"typedef enum \{([^}]*)\} lbm_prec;", src)
    assert m, "lbm_prec enum not found"
    vals = {k: int(v) for k, v in re.findall(r"(LBM_\w+)\s*=\s*(\d+)", m.group(1))}
    assert vals == {"LBM_F64": 0, "LBM_F32": 1, "LBM_F32_DEV": 2, "LBM_F64_FF": 3}
    assert lib.PREC == {"f64": vals["LBM_F64"], "f32": vals["LBM_F32"], "f32_dev": vals["LBM_F32_DEV"],
                        "f64_ff": vals["LBM_F64_FF"]}
    ctx = ctypes.c_void_p()
    for bad in (4, 5, -1):
        rc = lib._lib.lbm_create(ctypes.byref(ctx), 8, 16, bad, 0.8, 1e-4, None, None, 0, None)
        assert rc == lib.LBM_EINVAL and b"precision" in lib._lib.lbm_last_error()
        assert not ctx.value
