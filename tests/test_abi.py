"""CPU checks of the C ABI: the library loads, exports every function that
include/sps.h declares, and its host-side spherical-harmonic tables (grid,
analysis and synthesis matrices) agree with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1909_06623_gb300 import _lib, build, unit_tables

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sps.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sps_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, n


def test_default_params(lib):
    prm = _lib.sps_params()
    assert lib.sps_default_params(ctypes.byref(prm)) == 0
    assert prm.p == 6 and prm.beta == 1.75 and prm.bb_variant == 1
    # the fields appended last: the Python mirror of the struct ends where the C one does
    assert prm.delta_rel == 0.0 and prm.bb_warm == 0 and prm.contact_search == 0
    assert prm.ir_dw == 1 and prm.lcp_solver == 0


def test_create_rejects_bad_params(lib):
    prm = _lib.sps_params()
    lib.sps_default_params(ctypes.byref(prm))
    prm.p = 0
    h = ctypes.c_void_p()
    assert lib.sps_create(ctypes.byref(prm), None, ctypes.byref(h)) == 1
    assert lib.sps_unit_tables(0, None, None, None, None) == 1
    for field, bad in (("delta_rel", -0.1), ("delta_rel", float("inf")), ("bb_warm", 3),
                       ("delta", -1.0), ("mobility", 5), ("ir_dw", 2), ("precision", 3),
                       ("lcp_solver", 3), ("lcp_solver", -1), ("bb_variant", 4)):
        lib.sps_default_params(ctypes.byref(prm))
        setattr(prm, field, bad)
        assert lib.sps_create(ctypes.byref(prm), None, ctypes.byref(h)) == 1, field


@pytest.mark.parametrize("p", [2, 4, 6, 8])
def test_unit_tables_match_oracle(lib, p):
    from oracle import sph
    nodes, w, A, S = unit_tables(p)
    th, ph, nrm, wo = sph.unit_grid(p)
    assert np.abs(nodes.T - nrm).max() < 1e-14
    assert np.abs(w - wo).max() < 1e-14
    rng = np.random.default_rng(p)
    sig = rng.standard_normal((len(wo), 3))
    coef = A @ sig.T.ravel()                 # columns c*P + k
    ref = sph.analysis(sig, p)
    NC = (p + 1) * (p + 2) // 2
    for (n, m), (sv, sw, sx) in ref.items():
        if m < 0:
            continue
        ci = n * (n + 1) // 2 + m
        for ty, val in enumerate((sv, sw, sx)):
            r = (ty * NC + ci) * 2
            assert abs(coef[r] + 1j * coef[r + 1] - val) < 1e-13, (n, m, ty)
    back = (S @ coef).reshape(3, -1).T
    assert np.abs(back - sph.grid_synthesis(ref, p)).max() < 1e-13
