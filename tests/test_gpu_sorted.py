"""Sorted-layout mode: positions and forces in the context's cluster order between list builds.

nb_sorted_export hands out the sorted positions (the periodic images the grid
sort chose) and the slot -> atom permutation; nb_forces_sorted evaluates at
positions the caller keeps in that order and writes forces in that order, so an
MD step needs no gather into and no scatter out of the cluster layout.  Checked:
the same forces, energies and virial as the caller-order path at the same
positions, padding slots untouched, and an MD-like loop run entirely in the
sorted layout (forces, rolling prune, position update, a rebuild through caller
order) against the oracle's evaluation of the exported pair set.
"""
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


def _to_caller(xq, perm, n):
    """Caller-order positions [n, 3] from the sorted ones."""
    valid = perm >= 0
    x = torch.empty((n, 3), dtype=torch.float32, device=xq.device)
    x[perm[valid].long()] = xq[valid, :3]
    return x


@pytest.mark.parametrize("which", ["ewald3000", "rf648"])
def test_sorted_matches_caller_order(api, which):
    s = synth.water_648() if which == "rf648" else synth.water_box(1000, 3.1, seed=71, rc=1.0, rlist=1.1)
    flags = api.NB_ENERGY | api.NB_VIRIAL
    ctx = api.NbContext.from_system(s)
    x = torch.tensor(s.x, device="cuda")
    ctx.build(x, s.box)
    f_ref, e_ref, w_ref = ctx.forces(x, energy=True, virial=True)
    xq, perm = ctx.nb_sorted_export()
    xq0 = xq.clone()
    f = torch.full_like(xq, float("nan"))
    e = torch.empty(2, dtype=torch.float64, device="cuda")
    w = torch.empty(9, dtype=torch.float64, device="cuda")
    ctx.nb_forces_sorted(flags, xq, f, e, w)
    torch.cuda.synchronize()
    assert ctx.nb_get_error() == 0
    valid = perm >= 0
    assert int(valid.sum()) == s.n and torch.equal(xq, xq0)
    assert torch.all(f[~valid] == 0) and torch.all(f[:, 3] == 0)
    fb = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
    fb[perm[valid].long()] = f[valid, :3]
    assert_forces(fb.cpu().numpy(), f_ref.cpu().numpy(), tol_rms=1e-6, tol_atom=1e-5)
    assert rel(e[0].item(), e_ref[0].item()) < 1e-9 and rel(e[1].item(), e_ref[1].item()) < 1e-9
    assert np.abs(w.cpu().numpy() - w_ref.cpu().numpy().ravel()).max() <= 1e-6 * np.abs(w_ref.cpu().numpy()).max()
    # and against the oracle
    ref = oracle.brute(s) if which == "rf648" else oracle.celllist(s)
    assert_forces(fb.cpu().numpy(), ref)
    tol_lj, tol_c = energy_tolerances(s, ref)
    assert rel(e[0].item(), ref["E_lj"]) < tol_lj and rel(e[1].item(), ref["E_c"]) < tol_c
    W = w.cpu().numpy().reshape(3, 3)
    assert np.sqrt(((W - ref["W"]) ** 2).sum() / (ref["W"] ** 2).sum()) < TOL_W


def test_sorted_md_loop(api):
    """Forces, rolling prune over 2 parts and the position update in the sorted layout, a
    rebuild every 20 steps through caller order; forces and energies against the oracle's
    evaluation of exactly the exported inner pair set."""
    s = synth.water_box(1000, 3.1, seed=72, rc=1.0, rlist=1.1, r_in=1.03)
    vel = torch.tensor(synth.maxwell_boltzmann(s, 300.0, seed=5), dtype=torch.float32, device="cuda")
    flags = api.NB_ENERGY | api.NB_VIRIAL
    ctx = api.NbContext.from_system(s)
    xc0 = torch.tensor(s.x, device="cuda")  # caller coordinates of the last build
    ctx.build(xc0, s.box)
    xq, perm = ctx.nb_sorted_export()
    xq0 = xq.clone()  # the sorted positions as exported (the images the sort chose)
    f = torch.empty_like(xq)
    e = torch.empty(2, dtype=torch.float64, device="cuda")
    w = torch.empty(9, dtype=torch.float64, device="cuda")

    def sorted_velocities():
        v = torch.zeros((xq.shape[0], 3), dtype=torch.float32, device="cuda")
        valid = perm >= 0
        v[valid] = vel[perm[valid].long()]
        return v
    vs = sorted_velocities()
    for t in range(45):
        if t and t % 20 == 0:
            xc0 = _to_caller(xq, perm, s.n)
            ctx.build(xc0, s.box)
            xq, perm = ctx.nb_sorted_export()  # the slot count may change with the new sort
            xq0 = xq.clone()
            f = torch.empty_like(xq)
            vs = sorted_velocities()
        ctx.nb_forces_sorted(flags, xq, f, e, w)
        if t in (3, 21, 44):
            torch.cuda.synchronize()
            # the exported pair shifts refer to the caller coordinates the sort was given: move
            # those by the displacement since the export (the sorted images may differ by box vectors)
            xh = (xc0 + _to_caller(xq - xq0, perm, s.n)).cpu().numpy()
            ref = oracle.listset(s, ctx.nb_debug_export_pairs(api.NB_LIST_INNER), x=xh)
            valid = perm >= 0
            fb = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
            fb[perm[valid].long()] = f[valid, :3]
            assert_forces(fb.cpu().numpy(), ref)
            tol_lj, tol_c = energy_tolerances(s, ref, x=xh)
            assert rel(e[0].item(), ref["E_lj"]) < tol_lj and rel(e[1].item(), ref["E_c"]) < tol_c
        ctx.nb_prune_rolling(t % 2, 2)
        xq[:, :3].add_(vs, alpha=0.002)
    torch.cuda.synchronize()
    assert ctx.nb_get_error() == 0


def test_sorted_argument_errors(api):
    import ctypes
    vp = ctypes.c_void_p
    s = synth.water_648()
    ctx = api.NbContext.from_system(s)
    lib = ctx._lib
    buf = torch.zeros((64, 4), device="cuda")
    # before a grid sort there is no layout to export (NB_ERR_NOT_READY)
    assert lib.nb_sorted_export(ctx.handle, vp(buf.data_ptr()), None, None) == 3
    ctx.build(torch.tensor(s.x, device="cuda"), s.box)
    xq, perm = ctx.nb_sorted_export()
    f = torch.empty_like(xq)
    # misaligned arrays and missing outputs are rejected before any launch
    assert lib.nb_forces_sorted(ctx.handle, 0, vp(xq.data_ptr() + 4), vp(f.data_ptr()), None, None, None) == 1
    assert lib.nb_forces_sorted(ctx.handle, api.NB_ENERGY, vp(xq.data_ptr()), vp(f.data_ptr()), None, None,
                                None) == 1
