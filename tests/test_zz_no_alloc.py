"""The allocation-free entry point (nb_forces_small_noalloc) against nb_forces.

nb_forces_small_noalloc is for callers that cannot allocate device memory (for
example while a stream is being captured into a CUDA graph, or when another
allocator owns the device memory): it takes only inputs and outputs and keeps
its scratch in a static device array.  This test calls it through the C ABI
twice in a row -- the second call reuses the scratch the first one left
behind -- and checks both results against the context-based nb_forces within
the bars the other parity tests use.  It lives in its own file so that pytest
collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2006_09167_gb300 import synth
from helpers import TOL_F, TOL_W, energy_tolerances, rel, rms_rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_09167_gb300 import api as a
    return a


def _params(api, s):
    from paper_2006_09167_gb300 import _abi
    p = _abi.NbParams()
    p.n_atoms = s.n
    p.n_types = s.n_types
    p.coulomb = s.coulomb
    p.reserved = 0
    p.eps_r = s.eps_r
    p.eps_rf = s.eps_rf
    p.beta = s.beta
    p.rc = s.rc
    p.rlist = s.rlist
    p.r_in = s.r_in
    c6 = np.ascontiguousarray(s.c6, np.float32)
    c12 = np.ascontiguousarray(s.c12, np.float32)
    f32p = ctypes.POINTER(ctypes.c_float)
    p.c6_host = c6.ctypes.data_as(f32p)
    p.c12_host = c12.ctypes.data_as(f32p)
    return p, (c6, c12)


def _noalloc_call(lib, p, s, x, q, t, eo, ei, f, e, w):
    box = (ctypes.c_double * 3)(*[float(v) for v in s.box])
    vp = ctypes.c_void_p
    st = lib.nb_forces_small_noalloc(ctypes.byref(p), vp(x.data_ptr()), vp(q.data_ptr()), vp(t.data_ptr()),
                                     vp(eo.data_ptr()), vp(ei.data_ptr()), box, 3, vp(f.data_ptr()),
                                     vp(e.data_ptr()), vp(w.data_ptr()),
                                     vp(torch.cuda.current_stream().cuda_stream))
    return st


@pytest.mark.parametrize("which", ["rf648", "ewald3000"])
def test_noalloc_matches_nb_forces_twice(api, which):
    from paper_2006_09167_gb300 import _abi
    lib = _abi.load()
    s = synth.water_648() if which == "rf648" else synth.water_box(1000, 3.1, seed=61, rc=1.0, rlist=1.1)
    # the existing entry point
    ctx = api.NbContext.from_system(s)
    x = torch.tensor(s.x, device="cuda")
    ctx.build(x, s.box)
    f_ref, e_ref, w_ref = ctx.forces(x, energy=True, virial=True)
    torch.cuda.synchronize()
    f_ref = f_ref.cpu().numpy()
    e_ref = e_ref.cpu().numpy()
    w_ref = w_ref.cpu().numpy()
    tol_lj, tol_c = energy_tolerances(s, oracle.celllist(s))
    # the allocation-free entry point, twice in a row on the same stream
    p, keep = _params(api, s)
    q = torch.tensor(s.q, device="cuda")
    t = torch.tensor(s.types, dtype=torch.int32, device="cuda")
    eo = torch.tensor(s.excl_off, dtype=torch.int32, device="cuda")
    ei = torch.tensor(s.excl_idx, dtype=torch.int32, device="cuda")
    for call in range(2):
        f = torch.full((s.n, 3), float("nan"), device="cuda")
        e = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        w = torch.full((9,), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc_call(lib, p, s, x, q, t, eo, ei, f, e, w) == 0
        torch.cuda.synchronize()
        fn, en, wn = f.cpu().numpy(), e.cpu().numpy(), w.cpu().numpy().reshape(3, 3)
        assert rms_rel(fn, f_ref) < TOL_F, f"call {call}"
        assert rel(en[0], e_ref[0]) < 2 * tol_lj, f"call {call}"
        assert rel(en[1], e_ref[1]) < 2 * tol_c, f"call {call}"
        assert np.sqrt(((wn - w_ref) ** 2).sum() / (w_ref ** 2).sum()) < TOL_W, f"call {call}"
    del keep


def test_noalloc_rejects_sizes_beyond_its_maximum(api):
    from paper_2006_09167_gb300 import _abi
    lib = _abi.load()
    s = synth.water_648()
    p, keep = _params(api, s)
    p.n_atoms = _abi.NB_NOALLOC_MAX_ATOMS + 1
    dummy = torch.zeros(8, device="cuda")
    box = (ctypes.c_double * 3)(*[float(v) for v in s.box])
    vp = ctypes.c_void_p(dummy.data_ptr())
    st = lib.nb_forces_small_noalloc(ctypes.byref(p), vp, vp, vp, None, None, box, 0, vp, None, None, None)
    assert st == _abi.NB_ERR_CAPACITY
    del keep
