"""Host-side validation of lelbm_create (include/lelbm.h): every invalid parameter set is
rejected with LELBM_E_INVAL and its reason before any CUDA call, so this runs without a GPU.

The cases follow the documented contract of lelbm_params: dimensions 1-3, boundary kinds and
their pairing per axis (Sec. VI.B: periodic, inflow, outflow), the stencil constants of
Sec. II.C, the Newton limits of Sec. II.D, and the restrictions of the paths that are built
(no-slip walls and deterministic streaming on the 2D FP64 path, 3D on the FP64 path only).
"""
import ctypes
import math

import numpy as np
import pytest

from paper_2508_06911_gb300 import build, lelbm as L


@pytest.fixture(scope="module")
def lib():
    build.build()
    return L.load()


def _p(**kw):
    p = L.lelbm_default_params()
    for k, v in kw.items():
        if k in ("bc", "bc_z", "inlet", "wall_u"):
            for i, x in enumerate(v):
                getattr(p, k)[i] = x
        else:
            setattr(p, k, v)
    return p


OUT, IN, PER = L.LELBM_BC_OUTFLOW, L.LELBM_BC_INFLOW, L.LELBM_BC_PERIODIC
G2 = dict(dims=2, nx=8, ny=6)  # a fully periodic 2D grid
G3 = dict(dims=3, nx=4, ny=4, nz=4)  # a fully periodic 3D grid

# parameter sets are made when a test runs, after the library fixture has built and loaded
# the current library
INVALID = {
    "dims 0": (lambda: _p(dims=0), "dims"),
    "dims 4": (lambda: _p(dims=4), "dims"),
    "nx 0": (lambda: _p(nx=0), "nx"),
    "1D with ny 2": (lambda: _p(ny=2), "ny must be 1"),
    "2D batch": (lambda: _p(n_batch=2, **G2), "1D only"),
    "bc kind 3": (lambda: _p(bc=(3, 3, PER, PER)), "bc kind"),
    "periodic on one side": (lambda: _p(bc=(PER, OUT, PER, PER)), "both sides"),
    "outflow without pads": (lambda: _p(bc=(OUT, OUT, PER, PER), pad=0), "pad >= 1"),
    "3D z outflow without pads": (lambda: _p(bc_z=(OUT, OUT), **G3), "axis 2"),
    "K < 0": (lambda: _p(K=-1.0), "K must"),
    "K NaN": (lambda: _p(K=math.nan), "K must"),
    "nu < 0": (lambda: _p(nu_shear=-1e-3), "nu_shear"),
    "Pr 0": (lambda: _p(prandtl=0.0), "prandtl"),
    "n 0": (lambda: _p(n_conform=0.0), "stencil radius"),
    "R_min 0.5": (lambda: _p(r_min=0.5), "stencil radius"),
    "refinement divisor 0": (lambda: _p(refine_div=0.0), "refinement"),
    "refinement radius NaN": (lambda: _p(refine_rad=math.nan), "refinement"),
    "max_refine 5": (lambda: _p(max_refine=5), "max_refine"),
    "tol 0": (lambda: _p(tol=0.0), "tol"),
    "max_newton 0": (lambda: _p(max_newton=0), "max_newton"),
    "max_newton 61": (lambda: _p(max_newton=61), "max_newton"),
    "precision 7": (lambda: _p(precision=7), "precision"),
    "pad on a fully periodic 2D grid": (lambda: _p(pad=1, **G2), "fully periodic"),
    "pad on a fully periodic 3D grid": (lambda: _p(pad=1, **G3), "fully periodic"),
    "inflow with rho 0": (lambda: _p(bc=(IN, OUT, PER, PER), pad=2, inlet=(0.0, 0.0, 0.0, 1.0)), "inflow"),
    "inflow with RT 0": (lambda: _p(bc=(IN, OUT, PER, PER), pad=2, inlet=(1.0, 0.0, 0.0, 0.0)), "inflow"),
    "wall_u infinite": (lambda: _p(wall_u=(math.inf, 0.0), **G2), "wall_u"),
    "deterministic 1D": (lambda: _p(deterministic=1), "deterministic"),
    "deterministic mixed": (lambda: _p(deterministic=1, precision=L.LELBM_MIXED, **G2), "deterministic"),
    "3D nz 0": (lambda: _p(dims=3, nx=4, ny=4, nz=0), "nz"),
    "3D mixed": (lambda: _p(precision=L.LELBM_MIXED, **G3), "FP64 path only"),
    "3D inlet_uz NaN": (lambda: _p(inlet_uz=math.nan, **G3), "inlet_uz"),
}


def _create_rc(p, lengths=None, pads=None, solid=None):
    try:
        h = L.lelbm_create(p, lengths=lengths, pads=pads, solid=solid)
    except L.LelbmError as e:
        return e.code, str(e)
    L.lelbm_destroy(h)
    return L.LELBM_OK, ""


@pytest.mark.parametrize("case", sorted(INVALID))
def test_invalid_parameters_are_rejected_before_any_cuda_call(lib, case):
    make, reason = INVALID[case]
    code, msg = _create_rc(make())
    assert code == L.LELBM_E_INVAL, (case, code, msg)
    assert reason in msg, (case, msg)


def test_invalid_host_arrays_are_rejected(lib):
    # a 1D batch with an empty instance, and one with an outflow instance without pads
    p = _p(bc=(OUT, OUT, PER, PER), pad=2)
    code, msg = _create_rc(p, lengths=[8, 0, 5], pads=[2, 2, 2])
    assert code == L.LELBM_E_INVAL and "lengths[1]" in msg
    code, msg = _create_rc(_p(bc=(OUT, OUT, PER, PER), pad=2), lengths=[8, 4, 5], pads=[2, 2, 0])
    assert code == L.LELBM_E_INVAL and "pads[2]" in msg
    # no-slip (2) and moving no-slip (3) walls need the FP64 path; slip walls (1) do not
    solid = np.zeros((6, 8), np.uint8)
    for kind in (2, 3):
        solid[2, 3] = kind
        for prec in (L.LELBM_MIXED, L.LELBM_FP32):
            code, msg = _create_rc(_p(precision=prec, **G2), solid=solid)
            assert code == L.LELBM_E_INVAL and "FP64" in msg, (kind, prec, msg)
    # a solid mask excludes deterministic streaming and 3D
    code, msg = _create_rc(_p(deterministic=1, **G2), solid=solid)
    assert code == L.LELBM_E_INVAL and "deterministic" in msg
    code, msg = _create_rc(_p(**G3), solid=np.zeros((4, 4, 4), np.uint8))
    assert code == L.LELBM_E_INVAL and "solid" in msg


def test_null_arguments(lib):
    h = L._H()
    assert lib.lelbm_create(None, ctypes.byref(L.lelbm_default_params())) == L.LELBM_E_INVAL
    assert b"out" in lib.lelbm_last_error(None)
    assert lib.lelbm_create(ctypes.byref(h), None) == L.LELBM_E_INVAL
    assert b"params" in lib.lelbm_last_error(None)


def test_valid_parameters_pass_validation(lib):
    """Sets the contract allows get past validation: without a GPU they stop at the first
    CUDA call (E_CUDA), with one they create a handle."""
    import torch

    valid = [
        _p(),
        _p(**G2),
        _p(**G3),  # the default z boundaries are periodic
        _p(bc=(IN, OUT, OUT, OUT), pad=2, **G2),
        _p(bc=(IN, OUT, OUT, OUT), bc_z=(OUT, IN), pad=1, inlet_uz=0.5, **G3),
        _p(deterministic=1, **G2),
        _p(precision=L.LELBM_MIXED, **G2),
        _p(precision=L.LELBM_FP32, wall_u=(0.3, -0.1), **G2),
    ]
    for p in valid:
        code, msg = _create_rc(p)
        if torch.cuda.is_available():
            assert code == L.LELBM_OK, msg
        else:
            assert code == L.LELBM_E_CUDA, msg


def test_create_leaves_the_callers_parameters_unchanged(lib):
    p = _p(bc=(OUT, OUT, PER, PER), pad=2)
    before = bytes(p)
    _create_rc(p, lengths=[8, 4, 5], pads=[2, 2, 2], solid=None)
    assert bytes(p) == before
