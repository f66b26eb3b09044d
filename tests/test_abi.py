"""The C-ABI library builds, loads and exports every function include/lelbm.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2508_06911_gb300 import build, lelbm as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(lelbm_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return L.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(L.EXPORTS) == names


def test_struct_layouts_match(lib):
    ps, ss = L.lelbm_abi_sizes()
    assert ps == ctypes.sizeof(L.lelbm_params)
    assert ss == ctypes.sizeof(L.lelbm_stats)


def test_defaults_are_the_papers_constants(lib):
    p = L.lelbm_default_params()
    assert (p.n_conform, p.r_min, p.refine_div, p.refine_rad, p.tol) == (4.0, 2.0, 3.0, 3.0, 1e-12)
    assert p.limiter == 1 and p.nu_bulk < 0


def test_no_cpu_fallback_without_device(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(L.LelbmError) as e:
        L.lelbm_create(L.lelbm_default_params())
    assert e.value.code == L.LELBM_E_CUDA
