"""First-use prune fused into the force kernel (nb_set_fused_prune, Sec. V.D):
the inner list it compacts equals the separate prune's at the same positions
(as integer pair sets), forces and energies match the oracle and the separate
path, and calls that need the inner list before the first force call prune it
first."""
import numpy as np
import pytest

import oracle
from helpers import assert_forces, canonical_pairs, energy_tolerances, rel
from paper_2006_09167_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_09167_gb300 import api as a
    return a


def inner_pairs(api, ctx):
    """The inner list as a sorted list of canonical image pairs (export order depends on scheduling)."""
    return sorted(canonical_pairs(ctx.nb_debug_export_pairs(api.NB_LIST_INNER)))


def contexts(api, s, x):
    sep = api.NbContext.from_system(s)
    fus = api.NbContext.from_system(s)
    fus.nb_set_fused_prune(True)
    sep.build(x, s.box)
    fus.build(x, s.box)
    return sep, fus


@pytest.mark.parametrize("coulomb", [synth.COULOMB_RF, synth.COULOMB_EWALD])
def test_fused_prune_equals_separate_prune(api, coulomb):
    import torch
    s = synth.water_box(1000, 3.1, seed=61, coulomb=coulomb, rc=1.0, rlist=1.1)
    x = torch.tensor(s.x, device="cuda")
    sep, fus = contexts(api, s, x)
    f1, e1, w1 = sep.forces(x, energy=True, virial=True)
    f2, e2, w2 = fus.forces(x, energy=True, virial=True)  # evaluates the outer list, prunes on the way
    torch.cuda.synchronize()
    assert sep.nb_get_error() == 0 and fus.nb_get_error() == 0
    assert inner_pairs(api, sep) == inner_pairs(api, fus)
    ref = oracle.brute(s)
    tol_lj, tol_c = energy_tolerances(s, ref)
    for f, e in ((f1, e1), (f2, e2)):
        assert_forces(f.cpu().numpy(), ref)
        assert rel(e[0].item(), ref["E_lj"]) < tol_lj and rel(e[1].item(), ref["E_c"]) < tol_c
    assert_forces(f2.cpu().numpy(), f1.cpu().numpy(), tol_rms=1e-6, tol_atom=1e-5)
    assert np.abs(w2.cpu().numpy() - w1.cpu().numpy()).max() < 1e-5 * np.abs(w1.cpu().numpy()).max()


def test_fused_prune_then_rolling_steps(api):
    import torch
    s = synth.water_box(1000, 3.1, seed=62, rc=1.0, rlist=1.1, coulomb=synth.COULOMB_EWALD)
    x = torch.tensor(s.x, device="cuda")
    v = torch.tensor(synth.maxwell_boltzmann(s, 300.0, seed=3), dtype=torch.float32, device="cuda")
    sep, fus = contexts(api, s, x)
    for t in range(12):
        f1, e1, _ = sep.forces(x, energy=True)
        f2, e2, _ = fus.forces(x, energy=True)
        assert_forces(f2.cpu().numpy(), f1.cpu().numpy(), tol_rms=1e-6, tol_atom=1e-5)
        assert rel(e2.sum().item(), e1.sum().item()) < 1e-6
        sep.nb_prune_rolling(t % 2, 2)
        fus.nb_prune_rolling(t % 2, 2)
        x.add_(v, alpha=0.002)
    torch.cuda.synchronize()
    assert inner_pairs(api, sep) == inner_pairs(api, fus)


def test_pending_inner_list_is_pruned_on_demand(api):
    import torch
    s = synth.water_box(1000, 3.1, seed=63, rc=1.0, rlist=1.1)
    x = torch.tensor(s.x, device="cuda")
    sep, fus = contexts(api, s, x)
    # before any force call the fused context still answers inner-list queries correctly
    assert fus.nb_count_pairs(api.NB_LIST_INNER) == sep.nb_count_pairs(api.NB_LIST_INNER)
    assert inner_pairs(api, fus) == inner_pairs(api, sep)
    f1, _, _ = sep.forces(x, energy=False)
    f2, _, _ = fus.forces(x, energy=False)
    assert_forces(f2.cpu().numpy(), f1.cpu().numpy(), tol_rms=1e-6, tol_atom=1e-5)
