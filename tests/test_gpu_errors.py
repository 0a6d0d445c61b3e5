"""Error handling on the GPU: calls out of order, bad arguments and device-detected
errors come back as status codes (no trap, fault or hang)."""
import numpy as np
import pytest

from paper_2006_09167_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_09167_gb300 import api as a
    return a


def status_of(api, fn):
    with pytest.raises(api.NbError) as ei:
        fn()
    return ei.value.status


def test_calls_out_of_order(api):
    s = synth.water_648()
    ctx = api.NbContext.from_system(s)
    x = torch.tensor(s.x, device="cuda")
    f = torch.empty((s.n, 3), device="cuda")
    assert status_of(api, lambda: ctx.nb_forces(0, x, f)) == 3
    assert status_of(api, lambda: ctx.nb_prune_rolling(0, 2)) == 3
    assert status_of(api, lambda: ctx.nb_pairlist_build()) == 3
    ctx.nb_grid_sort(x, s.box)
    assert status_of(api, lambda: ctx.nb_forces(0, x, f)) == 3  # sorted, no list yet
    ctx.nb_pairlist_build()
    ctx.nb_forces(0, x, f)
    # a new grid sort invalidates the list
    ctx.nb_grid_sort(x, s.box)
    assert status_of(api, lambda: ctx.nb_forces(0, x, f)) == 3


def test_bad_arguments(api):
    s = synth.water_box(1000, 3.1, seed=71, rc=1.0, rlist=1.1)
    ctx = api.NbContext.from_system(s)
    x = torch.tensor(s.x, device="cuda")
    f = torch.empty((s.n, 3), device="cuda")
    # box too small for rc (rc >= L/2) or rlist (>= L)
    assert status_of(api, lambda: ctx.nb_grid_sort(x, [1.9, 3.1, 3.1])) == 2
    ctx.build(x, s.box)
    # rlist below r_in
    assert status_of(api, lambda: ctx.nb_pairlist_build(rlist=0.95)) == 1
    ctx.build(x, s.box)
    # prune radius outside [rc, rlist]
    assert status_of(api, lambda: ctx.nb_prune_rolling(0, 2, r_in=0.9)) == 1
    assert status_of(api, lambda: ctx.nb_prune_rolling(0, 2, r_in=1.2)) == 1
    assert status_of(api, lambda: ctx.nb_prune_rolling(2, 2)) == 1
    # unknown flag bits, missing energy buffer
    assert status_of(api, lambda: ctx.nb_forces(4, x, f)) == 1
    from paper_2006_09167_gb300 import _abi
    import ctypes
    st = _abi.load().nb_forces(ctx.handle, 1, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                               None, None, None)
    assert st == 1
    torch.cuda.synchronize()
    assert ctx.nb_get_error() == 0


def test_nonfinite_coordinates_are_reported(api):
    s = synth.water_box(1000, 3.1, seed=72, rc=1.0, rlist=1.1)
    ctx = api.NbContext.from_system(s)
    x = torch.tensor(s.x, device="cuda")
    ctx.build(x, s.box)
    x2 = x.clone()
    x2[17, 1] = float("nan")
    f, e, _ = ctx.forces(x2, energy=True)
    torch.cuda.synchronize()
    assert ctx.nb_get_error() == 7
    assert ctx.nb_get_error() == 0  # reading clears the flag
    # the same coordinates given to the grid sort
    ctx.nb_grid_sort(x2, s.box)
    torch.cuda.synchronize()
    assert ctx.nb_get_error() == 7


def test_column_capacity_overflow(api):
    # 10,000 atoms in a thin pillar of a sparse box: one grid column holds them all
    rng = np.random.default_rng(3)
    n = 10000
    L = 20.0
    x = np.empty((n, 3), np.float32)
    x[:, 0] = 10.0 + rng.uniform(-0.2, 0.2, n)
    x[:, 1] = 10.0 + rng.uniform(-0.2, 0.2, n)
    x[:, 2] = np.sort(rng.uniform(0, L, n))
    c6, c12 = synth.geometric_tables([0.0026], [2.6e-6])
    off, idx = synth.csr_from_pairs(n, np.zeros((0, 2)))
    ctx = api.NbContext(n, np.zeros(n, np.float32), np.zeros(n, np.int32), c6, c12, off, idx,
                        coulomb=api.NB_COULOMB_RF, rc=0.9, rlist=1.0)
    xt = torch.tensor(x, device="cuda")
    assert status_of(api, lambda: ctx.nb_grid_sort(xt, [L, L, L])) == 4


def test_forces_are_reproducible(api):
    s = synth.water_box(3375, 4.66, seed=73, rc=1.0, rlist=1.1)
    ctx = api.NbContext.from_system(s)
    x = torch.tensor(s.x, device="cuda")
    ctx.build(x, s.box)
    outs = [ctx.forces(x, energy=True, virial=True) for _ in range(3)]
    torch.cuda.synchronize()
    f0 = outs[0][0].cpu().numpy().astype(np.float64)
    for f, e, w in outs[1:]:
        fd = f.cpu().numpy().astype(np.float64)
        # atomics change only the FP32 summation order
        assert np.sqrt(((fd - f0) ** 2).sum() / (f0 ** 2).sum()) < 1e-6
        assert abs(e[0].item() - outs[0][1][0].item()) <= 1e-9 * abs(outs[0][1][0].item())
    # the list itself is deterministic: a rebuild exports the same pair set
    p1 = ctx.nb_debug_export_pairs(api.NB_LIST_OUTER)
    ctx.build(x, s.box)
    p2 = ctx.nb_debug_export_pairs(api.NB_LIST_OUTER)
    assert np.array_equal(np.sort(p1.view([("", p1.dtype)] * 5), axis=0), np.sort(p2.view([("", p2.dtype)] * 5), axis=0))


def test_trace_selected_kinds(api):
    """nb_trace_enable times only the kinds it is given; unknown kinds are rejected."""
    s = synth.water_648()
    ctx = api.NbContext.from_system(s)
    x = torch.tensor(s.x, device="cuda")
    f = torch.empty((s.n, 3), device="cuda")
    ctx.build(x, s.box)
    ctx.nb_trace_enable(True, kinds=[api.NB_TRACE_FORCES])
    for k in range(3):
        ctx.nb_forces(0, x, f)
        ctx.nb_prune_rolling(k % 2, 2)
    ms, n = ctx.nb_trace_read(api.NB_TRACE_FORCES)
    assert n == 3 and ms > 0.0
    assert ctx.nb_trace_read(api.NB_TRACE_PRUNE) == (0.0, 0)
    assert ctx.nb_trace_read(api.NB_TRACE_GATHER) == (0.0, 0)
    ctx.nb_trace_enable(True)  # every kind
    ctx.nb_forces(0, x, f)
    ctx.nb_prune_rolling(0, 2)
    assert ctx.nb_trace_read(api.NB_TRACE_GATHER)[1] == 1
    assert ctx.nb_trace_read(api.NB_TRACE_PRUNE)[1] == 1
    # switching the selection keeps traced launches pending until they are read
    ctx.nb_trace_enable(False)
    ctx.nb_forces(0, x, f)
    ctx.nb_trace_enable(True, kinds=[api.NB_TRACE_FORCES])
    ctx.nb_forces(0, x, f)
    assert ctx.nb_trace_read(api.NB_TRACE_FORCES)[1] == 2
    assert ctx.nb_trace_read(api.NB_TRACE_FORCES) == (0.0, 0)
    assert status_of(api, lambda: ctx.nb_trace_enable(True, kinds=[api.NB_TRACE_KINDS])) == 1
