"""The C ABI library builds for sm_103a, loads, exports every symbol include/iga.h
declares, and rejects bad arguments on the host before touching a GPU (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_1904_06971_gb300 as iga

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "iga.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(iga_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = iga.load()
    syms = declared_symbols()
    assert len(syms) >= 14
    for s in syms:
        assert hasattr(L, s), s


def test_version_and_kernel_names():
    L = iga.load()
    assert L.iga_version() >= 10000
    names = iga.kernel_names()
    assert "spmv" in names and "stage_x" in names and "fill" in names
    assert len(set(names)) == len(names)


class P:
    def __init__(self, **kw):
        base = dict(dim=2, p=2, n_el=(8, 8), map_kind="identity", map_amp=0.0, affine=None,
                    kappa_kind="const", kappa_a=1.0, kappa_b=0.0, kappa_deg=0, kappa_poly=None)
        base.update(kw)
        self.__dict__.update(base)


@pytest.mark.parametrize("kw,code", [
    (dict(p=0), -4), (dict(p=6), -4), (dict(dim=4, n_el=(8, 8, 8)), -4),
    (dict(n_el=(2, 8)), -1), (dict(kappa_kind="expsin3d"), -1),
    (dict(kappa_kind="poly", kappa_deg=4), -1),
])
def test_host_validation_rejects_bad_problems(kw, code):
    with pytest.raises(iga.IgaError) as ei:
        iga.assemble_exact(P(**kw), stream=0)
    assert ei.value.code == code
    assert iga.load().iga_last_error().decode() != ""


@pytest.mark.parametrize("M,q,code", [(0, 3, -1), (4, -1, -4), (4, 8, -4)])
def test_host_validation_rejects_bad_sampling(M, q, code):
    with pytest.raises(iga.IgaError) as ei:
        iga.assemble_surrogate(P(), M, q, stream=0)
    assert ei.value.code == code


def test_bad_dtype_and_null_pointers():
    L = iga.load()
    with pytest.raises(ValueError):
        iga.assemble_exact(P(), dtype="f16", stream=0)
    pt, mp, kp = iga._structs(P())
    h = ctypes.c_void_p()
    assert L.iga_assemble_exact(None, 2, ctypes.byref(mp), ctypes.byref(kp), 0, None, ctypes.byref(h)) == -1
    assert L.iga_assemble_exact(ctypes.byref(pt), 2, ctypes.byref(mp), ctypes.byref(kp), 7, None, ctypes.byref(h)) == -1
    assert L.iga_assemble_exact(ctypes.byref(pt), 2, ctypes.byref(mp), ctypes.byref(kp), 0, None, None) == -1
    assert L.iga_apply(None, None, None, None) == -1
    assert L.iga_matrix_info(None, None, None, None, None) == -1
    assert L.iga_matrix_destroy(None) == 0
    assert L.iga_profile_read(-1, None, None) == -1
