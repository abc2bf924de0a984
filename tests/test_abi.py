"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every
symbol include/scw.h declares, and rejects bad descriptors before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2404_07293_gb300 as scw
from paper_2404_07293_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(scw_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2404_07293_gb300 import build
        build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, f"binding lacks {n}"


def test_status_strings_and_version(lib):
    assert lib.scw_version() >= 1
    for s in range(9):
        assert lib.scw_status_string(s)
    assert lib.scw_status_string(99) == b"unknown status"


def _desc(**kw):
    zb = np.array([0.0, 0.25, 0.5])
    zp = np.array([0.1, 0.3])
    base = dict(U=3, V=3, L=2, lam=1.0, X=2.0, Y=2.0, Fx=16, Fy=16, Fz=2, x0=0.0, y0=0.0, n_top=1.0,
                n_bot_re=1.0, n_bot_im=0.0, z_inc=0.0, precision=0, flags=0, k_split=0)
    base.update(kw)
    zb = base.pop("zb", zb)
    zp = base.pop("zp", zp)
    d = _lib.ScwDesc(**base)
    d.z_bounds = zb.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.z_planes = zp.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return d, (zb, zp)


@pytest.mark.parametrize("bad", [
    dict(U=0), dict(L=0), dict(lam=0.0), dict(X=-1.0), dict(Fx=12), dict(Fy=4), dict(Fx=8192), dict(Fz=0),
    dict(precision=7), dict(k_split=-1), dict(n_top=0.0), dict(illuminations=-1), dict(illuminations=257),
    dict(illuminations=200, Fz=400, zp=np.linspace(0.0, 0.5, 400)), dict(pupil_na=-0.1),
    dict(pupil_na=float("inf")), dict(tiles_x=65), dict(tiles_y=-1), dict(out_ld=17), dict(out_ld=14),
    dict(out_ld=32, out_plane_stride=32 * 15), dict(out_plane_stride=257),
    dict(zb=np.array([0.0, 0.5, 0.5])), dict(zp=np.array([0.3, 0.1])), dict(zp=np.array([0.1, np.nan])),
])
def test_bad_descriptors_are_rejected(lib, bad):
    d, keep = _desc(**bad)
    h = ctypes.c_void_p()
    st = lib.scw_plan_create(ctypes.byref(d), ctypes.byref(h))
    assert st == 1, (st, lib.scw_last_error())
    assert not h.value
    assert lib.scw_last_error()


@pytest.mark.parametrize("entry", ["scw_plan", "scw_plan_batched"])
def test_stream_forms_reject_bad_descriptors(lib, entry):
    """The stream-taking plan constructors validate before they touch a device."""
    for bad in (dict(U=0), dict(Fx=12), dict(zp=np.array([0.3, 0.1]))):
        d, keep = _desc(**bad)
        h = ctypes.c_void_p()
        if entry == "scw_plan":
            st = lib.scw_plan(ctypes.byref(d), None, ctypes.byref(h))
        else:
            st = lib.scw_plan_batched(ctypes.byref(d), 1, None, ctypes.byref(h))
        assert st == 1, (entry, bad, st)
        assert not h.value


def test_boundary_names_of_the_scope_table(lib):
    """Every entry point the hot path's boundary names is exported and callable through
    ctypes; with NULL handles each returns INVALID_ARGUMENT (host checks, no device)."""
    h = ctypes.c_void_p()
    assert lib.scw_plan(None, None, ctypes.byref(h)) == 1
    assert lib.scw_plan_batched(None, 1, None, ctypes.byref(h)) == 1
    assert lib.scw_plan_set_layers(None, None, None, None, None, None, None, None) == 1
    assert lib.scw_synthesize(None, None, None) == 1
    table = ctypes.c_void_p(256)
    outs = (ctypes.c_void_p * 1)(256)
    assert lib.scw_synthesize_batched(None, table, None, None) == 1
    assert lib.scw_synthesize_batched(None, None, outs, None) == 1
    assert lib.scw_surrogate_create(None, ctypes.byref(h)) == 1
    assert lib.scw_surrogate_train_step(None, None, None, 1, ctypes.c_float(1e-3), None, None) == 1
    assert lib.scw_surrogate_infer(None, None, 1, None, None, None, ctypes.c_float(5e-2), None) == 1
    assert lib.scw_surrogate_destroy(None) == 0
    assert lib.scw_plan_destroy(None) == 0
    assert lib.scw_status_string(0) == b"ok"
    assert lib.scw_last_error() is not None


def test_host_io_with_custom_pitch_is_unsupported(lib):
    d, keep = _desc(out_ld=32, flags=2)
    h = ctypes.c_void_p()
    assert lib.scw_plan_create(ctypes.byref(d), ctypes.byref(h)) == 2
    assert not h.value


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.scw_plan_create(None, ctypes.byref(h)) == 1
    assert lib.scw_synthesize(None, None, None) == 1
    assert lib.scw_plan_set_layers(None, None, None, None, None, None, None, None) == 1
    assert lib.scw_plan_destroy(None) == 0


def test_no_cpu_fallback_without_gpu(lib):
    """On a machine without a usable sm_103a device plan creation fails loudly."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    d, keep = _desc()
    h = ctypes.c_void_p()
    st = lib.scw_plan_create(ctypes.byref(d), ctypes.byref(h))
    assert st == 4
    with pytest.raises(scw.ScwError):
        scw.Plan(3, 3, 2, 1.0, 2.0, 2.0, [0, 0.25, 0.5], 16, 16, [0.1, 0.3])


def test_noalloc_rejects_sizes_above_its_scratch(lib):
    """The allocation-free recompose checks its fixed scratch size on the host,
    before looking at the device or launching anything."""
    dummy = ctypes.c_void_p(256)  # never dereferenced: the size check comes first
    st = lib.scw_recompose_noalloc(4096, 1, 16.0, 16.0, 4096, 4096, 100, 0.0, 0.0, dummy, dummy, None)
    assert st == 2
    assert b"scratch" in lib.scw_last_error()
    assert lib.scw_recompose_noalloc(21, 21, 16.0, 16.0, 256, 256, 8, 0.0, 0.0, None, dummy, None) == 1
    assert lib.scw_recompose_noalloc(21, 97, 16.0, 16.0, 256, 256, 8, 0.0, 0.0, dummy, dummy, None) == 1


def _solve_desc(**kw):
    zb = np.array([0.0, 0.25, 0.5])
    base = dict(U=3, V=3, L=2, lam=1.0, X=2.0, Y=2.0, Nx=8, Ny=8, n_top=1.0, n_bot_re=1.0, n_bot_im=0.0, z_inc=0.0)
    base.update(kw)
    zb = base.pop("zb", zb)
    d = _lib.ScwSolveDesc(**base)
    d.z_bounds = zb.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return d, zb


@pytest.mark.parametrize("bad", [dict(U=0), dict(L=0), dict(lam=-1.0), dict(Nx=4), dict(Ny=4), dict(n_top=0.0),
                                 dict(U=64, V=64, Nx=128, Ny=128), dict(zb=np.array([0.0, 0.5, 0.4]))])
def test_bad_solver_descriptors_are_rejected(lib, bad):
    d, keep = _solve_desc(**bad)
    h = ctypes.c_void_p()
    st = lib.scw_solver_create(ctypes.byref(d), ctypes.byref(h))
    assert st in (1, 2), (st, lib.scw_last_error())
    assert not h.value
