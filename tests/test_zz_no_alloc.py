"""The allocation-free entry point (nb_forces_small_noalloc) against nb_forces.

nb_forces_small_noalloc is for callers that cannot allocate device memory (for
example when another allocator owns the device memory, or when the caller may
not allocate once it is running): it takes only inputs and outputs and keeps
its scratch in a static device array.  This test calls it through the C ABI
twice in a row -- the second call reuses the scratch the first one left
behind -- and checks both results against the context-based nb_forces within
the bars the other parity tests use.  It also checks the sizes it must refuse
on the host and the inputs it must refuse on the device (an atom type out of
range, an exclusion row longer than the kernel can hold), after which every
output is NaN.  It lives in its own file so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2006_09167_gb300 import synth
from helpers import TOL_W, assert_forces, energy_tolerances, rel

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
        assert_forces(fn, f_ref)
        assert rel(en[0], e_ref[0]) < 2 * tol_lj, f"call {call}"
        assert rel(en[1], e_ref[1]) < 2 * tol_c, f"call {call}"
        assert np.sqrt(((wn - w_ref) ** 2).sum() / (w_ref ** 2).sum()) < TOL_W, f"call {call}"
    del keep


@pytest.mark.parametrize("case", ["atoms", "types", "exclusion_pointers", "box"])
def test_noalloc_rejects_on_the_host(api, case):
    """Sizes beyond the maximum and bad arguments return an error before any launch."""
    from paper_2006_09167_gb300 import _abi
    lib = _abi.load()
    s = synth.water_648()
    p, keep = _params(api, s)
    dummy = torch.zeros(8, device="cuda")
    vp = ctypes.c_void_p(dummy.data_ptr())
    box = [float(v) for v in s.box]
    excl = (None, None)
    want = _abi.NB_ERR_CAPACITY
    if case == "atoms":
        p.n_atoms = _abi.NB_NOALLOC_MAX_ATOMS + 1
    elif case == "types":
        big = np.zeros((_abi.NB_NOALLOC_MAX_TYPES + 1,) * 2, np.float32)
        f32p = ctypes.POINTER(ctypes.c_float)
        p.n_types = big.shape[0]
        p.c6_host = big.ctypes.data_as(f32p)
        p.c12_host = big.ctypes.data_as(f32p)
        keep = (keep, big)
    elif case == "exclusion_pointers":
        excl = (vp, None)  # one of the two CSR arrays without the other
        want = _abi.NB_ERR_INVALID_ARG
    else:
        box[0] = 1.9 * s.rc  # rc >= L/2 on one axis
        want = _abi.NB_ERR_BOX_TOO_SMALL
    hbox = (ctypes.c_double * 3)(*box)
    st = lib.nb_forces_small_noalloc(ctypes.byref(p), vp, vp, vp, excl[0], excl[1], hbox, 0, vp, None, None, None)
    assert st == want
    del keep


@pytest.mark.parametrize("case", ["17_exclusion_partners", "type_out_of_range", "negative_type"])
def test_noalloc_refuses_invalid_device_inputs(api, case):
    """Inputs only the device can check give NaN outputs (not a silently wrong result),
    and the next valid call is correct again (the status word is cleared per call)."""
    from paper_2006_09167_gb300 import _abi
    lib = _abi.load()
    s = synth.water_648()
    p, keep = _params(api, s)
    x = torch.tensor(s.x, device="cuda")
    q = torch.tensor(s.q, device="cuda")
    types = s.types.astype(np.int32).copy()
    off, idx = s.excl_off.astype(np.int32), s.excl_idx.astype(np.int32)
    if case == "17_exclusion_partners":
        # atom 0 lists 17 partners: its own two hydrogens and 15 atoms of other molecules
        rows = [list(idx[off[i]:off[i + 1]]) for i in range(s.n)]
        extra = [j for j in range(3, s.n) if j not in rows[0]][:15]
        rows[0] = rows[0] + extra
        for j in extra:
            rows[j] = rows[j] + [0]
        off = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
        idx = np.concatenate([np.asarray(r, np.int32) for r in rows])
        assert off[1] - off[0] == 17
    elif case == "type_out_of_range":
        types[5] = s.n_types
    else:
        types[5] = -1
    t = torch.tensor(types, device="cuda")
    eo = torch.tensor(off, device="cuda")
    ei = torch.tensor(idx, device="cuda")
    f = torch.zeros((s.n, 3), device="cuda")
    e = torch.zeros(2, dtype=torch.float64, device="cuda")
    w = torch.zeros(9, dtype=torch.float64, device="cuda")
    assert _noalloc_call(lib, p, s, x, q, t, eo, ei, f, e, w) == 0
    torch.cuda.synchronize()
    assert torch.isnan(f).all() and torch.isnan(e).all() and torch.isnan(w).all()
    # the next call with valid inputs is unaffected by the failed one
    t = torch.tensor(s.types, dtype=torch.int32, device="cuda")
    eo = torch.tensor(s.excl_off, dtype=torch.int32, device="cuda")
    ei = torch.tensor(s.excl_idx, dtype=torch.int32, device="cuda")
    assert _noalloc_call(lib, p, s, x, q, t, eo, ei, f, e, w) == 0
    torch.cuda.synchronize()
    ref = oracle.brute(s)
    assert_forces(f.cpu().numpy(), ref)
    tol_lj, tol_c = energy_tolerances(s, ref)
    assert rel(e[0].item(), ref["E_lj"]) < tol_lj and rel(e[1].item(), ref["E_c"]) < tol_c
    del keep
