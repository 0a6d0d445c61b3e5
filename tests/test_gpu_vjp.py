"""GPU adjoint (nb_forces_vjp) against the oracle's analytic adjoint, and the
torch.autograd wrapper on a force-matching loss."""
import numpy as np
import pytest

import oracle
from paper_2006_09167_gb300 import synth
from helpers import TOL_F_ATOM, energy_tolerances, max_atom_err, rms_rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_G = 1e-5


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_09167_gb300 import api as a
    return a


def gpu_vjp(api, s, gF, gE):
    ctx = api.NbContext.from_system(s)
    x = torch.tensor(s.x, device="cuda")
    ctx.build(x, s.box)
    T = s.n_types
    gx = torch.empty((s.n, 3), device="cuda")
    gq = torch.empty(s.n, device="cuda")
    gc6 = torch.empty((T, T), dtype=torch.float64, device="cuda")
    gc12 = torch.empty((T, T), dtype=torch.float64, device="cuda")
    ctx.nb_forces_vjp(x, torch.tensor(gF, dtype=torch.float32, device="cuda"), gE, gx, gq, gc6, gc12)
    torch.cuda.synchronize()
    assert ctx.nb_get_error() == 0
    return dict(gx=gx.cpu().numpy(), gq=gq.cpu().numpy(), gc6=gc6.cpu().numpy(), gc12=gc12.cpu().numpy())


def check(g, r):
    assert rms_rel(g["gx"], r["gx"]) < TOL_G
    assert max_atom_err(g["gx"], r["gx"]) < TOL_F_ATOM
    assert rms_rel(g["gq"], r["gq"]) < TOL_G
    assert rms_rel(g["gc6"], r["gc6"]) < TOL_G
    assert rms_rel(g["gc12"], r["gc12"]) < TOL_G


@pytest.mark.parametrize("coulomb", [synth.COULOMB_RF, synth.COULOMB_EWALD])
def test_vjp_small_box(api, coulomb):
    rng = np.random.default_rng(1)
    extra = [(0.3166 * rng.uniform(0.95, 1.05), 0.65 * rng.uniform(0.8, 1.2)) for _ in range(4)]
    s = synth.water_box(1000, 3.1, seed=51, coulomb=coulomb, rc=1.0, rlist=1.1, extra_o_types=extra)
    gF = rng.normal(size=(s.n, 3))
    g = gpu_vjp(api, s, gF, 0.7)
    r = oracle.vjp(s, gF, 0.7)
    check(g, r)


@pytest.mark.parametrize("n_extra", [6, 10])
def test_vjp_many_types(api, n_extra):
    """8 types (per-lane parameter accumulators, the largest such case) and 12 types
    (shared-memory atomics)."""
    rng = np.random.default_rng(3 + n_extra)
    extra = [(0.3166 * rng.uniform(0.9, 1.1), 0.65 * rng.uniform(0.7, 1.3)) for _ in range(n_extra)]
    s = synth.water_box(1000, 3.1, seed=53, coulomb=synth.COULOMB_EWALD, rc=1.0, rlist=1.1, extra_o_types=extra)
    assert s.n_types == 2 + n_extra
    gF = rng.normal(size=(s.n, 3))
    check(gpu_vjp(api, s, gF, 0.4), oracle.vjp(s, gF, 0.4))


def test_vjp_24k_six_types(api):
    s = synth.water_24k_types()
    rng = np.random.default_rng(2)
    gF = rng.normal(size=(s.n, 3))
    g = gpu_vjp(api, s, gF, -0.3)
    r = oracle.vjp(s, gF, -0.3)
    check(g, r)


def test_autograd_force_matching_loss(api):
    s = synth.water_24k_types()
    ctx = api.NbContext.from_system(s)
    x = torch.tensor(s.x, device="cuda")
    ctx.build(x, s.box)
    # reference forces: the same box with C6/C12 scaled by 1.05 (oracle)
    s_ref = synth.System(**{**s.__dict__, "c6": s.c6 * np.float32(1.05), "c12": s.c12 * np.float32(1.05)})
    f_ref = torch.tensor(oracle.celllist(s_ref)["F"], dtype=torch.float32, device="cuda")
    xq = x.clone().requires_grad_(True)
    q = torch.tensor(s.q, device="cuda", requires_grad=True)
    c6 = torch.tensor(s.c6, device="cuda", requires_grad=True)
    c12 = torch.tensor(s.c12, device="cuda", requires_grad=True)
    F, E = api.forces(ctx, xq, q, c6, c12)
    loss = ((F - f_ref) ** 2).sum() / (3 * s.n) + 1e-4 * E
    loss.backward()
    torch.cuda.synchronize()
    # the same gradients from the oracle: gF = 2 (F - F_ref) / (3N) at the GPU forces, gE = 1e-4
    gF = (2.0 / (3 * s.n)) * (F.detach().cpu().numpy().astype(np.float64) - f_ref.cpu().numpy())
    r = oracle.vjp(s, gF, 1e-4)
    assert rms_rel(xq.grad.cpu().numpy(), r["gx"]) < TOL_G
    assert max_atom_err(xq.grad.cpu().numpy(), r["gx"]) < TOL_F_ATOM
    assert rms_rel(q.grad.cpu().numpy(), r["gq"]) < TOL_G
    assert rms_rel(c6.grad.cpu().numpy(), r["gc6"]) < TOL_G
    assert rms_rel(c12.grad.cpu().numpy(), r["gc12"]) < TOL_G
    # forward values
    o = oracle.celllist(s)
    assert rms_rel(F.detach().cpu().numpy(), o["F"]) < 1e-5
    assert max_atom_err(F.detach().cpu().numpy(), o["F"]) < TOL_F_ATOM
    tol_lj, tol_c = energy_tolerances(s, o)
    etot = o["E_lj"] + o["E_c"]
    bound = (tol_lj * abs(o["E_lj"]) + tol_c * abs(o["E_c"])) / abs(etot)
    assert abs(E.item() - etot) / abs(etot) < bound


def test_vjp_energy_weight_from_device_memory(api):
    """nb_forces_vjp_dev reads gE on the device (no host synchronisation): the same gradients
    as nb_forces_vjp given the same weight on the host."""
    s = synth.water_box(1000, 3.1, seed=93, rc=1.0, rlist=1.1)
    rng = np.random.default_rng(9)
    gF = torch.tensor(rng.normal(size=(s.n, 3)), dtype=torch.float32, device="cuda")
    ctx = api.NbContext.from_system(s)
    x = torch.tensor(s.x, device="cuda")
    ctx.build(x, s.box)
    T = s.n_types
    outs = []
    for dev in (False, True):
        gx = torch.empty((s.n, 3), device="cuda")
        gq = torch.empty(s.n, device="cuda")
        gc6 = torch.empty((T, T), dtype=torch.float64, device="cuda")
        gc12 = torch.empty((T, T), dtype=torch.float64, device="cuda")
        if dev:
            ctx.nb_forces_vjp_dev(x, gF, torch.tensor([0.37], dtype=torch.float64, device="cuda"), gx, gq, gc6, gc12)
        else:
            ctx.nb_forces_vjp(x, gF, 0.37, gx, gq, gc6, gc12)
        torch.cuda.synchronize()
        outs.append([t.cpu().numpy() for t in (gx, gq, gc6, gc12)])
    for a, b in zip(*outs):
        assert rms_rel(b, a) < 1e-6
    r = oracle.vjp(s, gF.cpu().numpy().astype(np.float64), 0.37)
    check(dict(zip(("gx", "gq", "gc6", "gc12"), outs[1])), r)
