"""CPU-side checks of the C ABI: the library builds, loads, exports every symbol
declared in include/nb.h, and rejects bad arguments before touching a GPU."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2006_09167_gb300 import build, _abi
    build.build()
    return _abi.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "nb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nb_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("nb_grid_sort", "nb_pairlist_build", "nb_prune_rolling", "nb_forces", "nb_forces_batched",
              "nb_forces_vjp"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2006_09167_gb300 import _abi
    names = declared_symbols()
    assert set(names) == set(_abi.EXPORTED)
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    for s in range(8):
        assert lib.nb_status_str(s)


def _params(**over):
    from paper_2006_09167_gb300 import _abi
    c6 = np.array([0.0026], dtype=np.float32)
    c12 = np.array([2.6e-6], dtype=np.float32)
    p = _abi.NbParams()
    p.n_atoms = 4
    p.n_types = 1
    p.coulomb = 0
    p.reserved = 0
    p.eps_r = 1.0
    p.eps_rf = math.inf
    p.beta = 0.0
    p.rc = 0.9
    p.rlist = 1.0
    p.r_in = 0.9
    for k, v in over.items():
        setattr(p, k, v)
    f32p = ctypes.POINTER(ctypes.c_float)
    p.c6_host = c6.ctypes.data_as(f32p)
    p.c12_host = c12.ctypes.data_as(f32p)
    return p, (c6, c12)


@pytest.mark.parametrize("over", [
    dict(n_atoms=0), dict(n_types=0), dict(n_types=65), dict(coulomb=3), dict(reserved=1),
    dict(eps_r=0.0), dict(rc=-1.0), dict(rc=9.0, rlist=9.5, r_in=9.0), dict(r_in=0.8),
    dict(rlist=0.85), dict(coulomb=1, beta=0.0), dict(coulomb=1, beta=5.0), dict(rc=float("nan")),
])
def test_create_rejects_bad_parameters_without_gpu(lib, over):
    p, keep = _params(**over)
    n = max(int(p.n_atoms), 1)
    q = np.zeros(n, np.float32)
    t = np.zeros(n, np.int32)
    off = np.zeros(n + 1, np.int32)
    idx = np.zeros(1, np.int32)
    h = ctypes.c_void_p()
    i32p = ctypes.POINTER(ctypes.c_int32)
    f32p = ctypes.POINTER(ctypes.c_float)
    st = lib.nb_create(ctypes.byref(p), q.ctypes.data_as(f32p), t.ctypes.data_as(i32p),
                       off.ctypes.data_as(i32p), idx.ctypes.data_as(i32p), ctypes.byref(h))
    assert st == 1 and not h.value


@pytest.mark.parametrize("case", ["type_range", "self_excl", "asym_excl", "too_many_excl", "nan_q"])
def test_create_rejects_bad_topology_without_gpu(lib, case):
    p, keep = _params()
    n = 4
    q = np.zeros(n, np.float32)
    t = np.zeros(n, np.int32)
    off = np.zeros(n + 1, np.int32)
    idx = np.zeros(1, np.int32)
    if case == "type_range":
        t[2] = 3
    elif case == "self_excl":
        off = np.array([0, 1, 1, 1, 1], np.int32)
        idx = np.array([0], np.int32)
    elif case == "asym_excl":
        off = np.array([0, 1, 1, 1, 1], np.int32)
        idx = np.array([2], np.int32)
    elif case == "too_many_excl":
        p, keep = _params(n_atoms=20)
        n = 20
        q = np.zeros(n, np.float32)
        t = np.zeros(n, np.int32)
        off = np.concatenate([[0], np.full(n, 17)]).astype(np.int32)
        idx = np.arange(1, 18, dtype=np.int32)
    elif case == "nan_q":
        q[1] = np.nan
    h = ctypes.c_void_p()
    i32p = ctypes.POINTER(ctypes.c_int32)
    f32p = ctypes.POINTER(ctypes.c_float)
    st = lib.nb_create(ctypes.byref(p), q.ctypes.data_as(f32p), t.ctypes.data_as(i32p),
                       off.ctypes.data_as(i32p), idx.ctypes.data_as(i32p), ctypes.byref(h))
    assert st == 1 and not h.value


def test_null_handles_are_rejected(lib):
    assert lib.nb_grid_sort(None, None, None, None) == 1
    assert lib.nb_pairlist_build(None, ctypes.c_float(1.0), None) == 1
    assert lib.nb_prune_rolling(None, ctypes.c_float(1.0), 0, 1, None) == 1
    assert lib.nb_forces(None, 0, None, None, None, None, None) == 1
    assert lib.nb_forces_vjp(None, None, None, ctypes.c_double(0.0), None, None, None, None, None) == 1
    assert lib.nb_forces_batched(None, 0, None, None, None, None, None) == 1
    lib.nb_destroy(None)
    lib.nb_batch_destroy(None)


@pytest.mark.parametrize("over", [dict(n_atoms=0), dict(order=2), dict(order=9), dict(grid=(6, 16, 16)),
                                  dict(grid=(16, 16, 5000)), dict(beta=0.0), dict(beta=float("nan")),
                                  dict(eps_r=0.0), dict(reserved=1)])
def test_pme_create_rejects_bad_parameters_without_gpu(lib, over):
    from paper_2006_09167_gb300 import _abi
    p = _abi.NbPmeParams()
    p.n_atoms, p.order, p.reserved, p.beta, p.eps_r = 10, 4, 0, 3.0, 1.0
    for a in range(3):
        p.grid[a] = 16
    for k, v in over.items():
        if k == "grid":
            for a in range(3):
                p.grid[a] = v[a]
        else:
            setattr(p, k, v)
    h = ctypes.c_void_p()
    assert lib.nb_pme_create(ctypes.byref(p), ctypes.byref(h)) == 1 and not h.value


def test_pme_and_corrections_reject_null_handles(lib):
    box = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    assert lib.nb_pme_forces(None, 0, None, None, box, None, None, None, None) == 1
    assert lib.nb_ewald_corrections(None, 0, None, None, None, None, None) == 1
    lib.nb_pme_destroy(None)
