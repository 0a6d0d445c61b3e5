"""GPU parity of the Ewald completion: smooth PME against the FP64 PME oracle
(same grid and order), the exclusion and self terms against the oracle, and the
whole Ewald sum (short-range kernel + PME + corrections) against the exact
direct sum, including a Madelung constant."""
import math

import numpy as np
import pytest

import oracle
from helpers import assert_forces, rel, rms_rel
from paper_2006_09167_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_09167_gb300 import api as a
    return a


def water_ewald(n_mol=216, box_len=1.862, seed=1, rc=0.9):
    return synth.water_box(n_mol, box_len, seed=seed, rc=rc, rlist=rc + 0.1)


def run_pme(api, s, grid, order, x=None, flags=3):
    import torch
    xx = torch.tensor(s.x if x is None else x, device="cuda")
    q = torch.tensor(s.q, device="cuda")
    pme = api.NbPme(s.n, s.beta, grid=grid, order=order, eps_r=s.eps_r)
    f = torch.zeros((s.n, 3), dtype=torch.float32, device="cuda")
    e = torch.empty(1, dtype=torch.float64, device="cuda")
    w = torch.empty(9, dtype=torch.float64, device="cuda")
    pme.nb_pme_forces(flags, xx, q, s.box, f, e, w)
    torch.cuda.synchronize()
    return f.cpu().numpy().astype(np.float64), float(e.item()), w.cpu().numpy().reshape(3, 3)


@pytest.mark.parametrize("order,spacing", [(4, 0.12), (5, 0.1), (6, 0.08), (8, 0.06)])
def test_pme_matches_pme_oracle(api, order, spacing):
    s = water_ewald()
    grid = api.pme_grid(s.box, spacing)
    f, e, w = run_pme(api, s, grid, order)
    ref = oracle.pme(s, grid=grid, order=order)
    assert_forces(f, ref)
    assert rel(e, ref["E"]) < 2e-6
    assert np.abs(w - ref["W"]).max() < 1e-5 * np.abs(ref["W"]).max()


def test_pme_96k_full_size(api):
    s = synth.water_96k()
    grid = api.pme_grid(s.box, 0.12)
    assert grid == (84, 84, 84)
    f, e, w = run_pme(api, s, grid, 4)
    ref = oracle.pme(s, grid=grid, order=4)
    assert_forces(f, ref)
    assert rel(e, ref["E"]) < 2e-6
    assert np.abs(w - ref["W"]).max() < 1e-5 * np.abs(ref["W"]).max()


def test_pme_positions_outside_the_box(api):
    s = water_ewald()
    grid = api.pme_grid(s.box, 0.12)
    shift = np.array([-1, 2, 3], np.float64) * s.box
    x2 = (s.x.astype(np.float64) + shift).astype(np.float32)
    f1, e1, _ = run_pme(api, s, grid, 4)
    f2, e2, _ = run_pme(api, s, grid, 4, x=x2)
    ref = oracle.pme(s, x=x2.astype(np.float64), grid=grid, order=4)
    assert_forces(f2, ref)
    assert_forces(f1, f2)
    assert rel(e1, e2) < 1e-5


@pytest.mark.parametrize("box", ["648", "24k"])
def test_corrections_match_oracle(api, box):
    import torch
    s = water_ewald() if box == "648" else synth.water_24k_types()
    ctx = api.NbContext.from_system(s)
    x = torch.tensor(s.x, device="cuda")
    ctx.build(x, s.box)
    f = torch.zeros((s.n, 3), dtype=torch.float32, device="cuda")
    e = torch.empty(2, dtype=torch.float64, device="cuda")
    w = torch.empty(9, dtype=torch.float64, device="cuda")
    ctx.nb_ewald_corrections(3, x, f, e, w)
    torch.cuda.synchronize()
    ref = oracle.ewald_excl(s)
    assert_forces(f.cpu().numpy(), ref, tol_rms=2e-6)
    assert rel(e[0].item(), ref["E"]) < 1e-6
    assert rel(e[1].item(), oracle.ewald_self(s)) < 1e-12
    assert np.abs(w.cpu().numpy().reshape(3, 3) - ref["W"]).max() < 1e-5 * np.abs(ref["W"]).max()


def full_ewald(api, s, grid, order):
    import torch
    ctx = api.NbContext.from_system(s)
    x = torch.tensor(s.x, device="cuda")
    q = torch.tensor(s.q, device="cuda")
    ctx.build(x, s.box)
    pme = api.NbPme(s.n, s.beta, grid=grid, order=order, eps_r=s.eps_r)
    f = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
    e_sr = torch.empty(2, dtype=torch.float64, device="cuda")
    e_rec = torch.empty(1, dtype=torch.float64, device="cuda")
    e_cor = torch.empty(2, dtype=torch.float64, device="cuda")
    ctx.nb_forces(api.NB_ENERGY, x, f, e_sr)
    pme.nb_pme_forces(api.NB_ENERGY, x, q, s.box, f, e_rec)
    ctx.nb_ewald_corrections(api.NB_ENERGY, x, f, e_cor)
    torch.cuda.synchronize()
    E = float(e_sr.sum().item() + e_rec.item() + e_cor.sum().item())
    return f.cpu().numpy().astype(np.float64), E


def exact_ewald(s):
    real = oracle.brute(s) if s.n <= 30000 else oracle.celllist(s)
    rec = oracle.ewald_recip(s)
    exc = oracle.ewald_excl(s)
    E = real["E_lj"] + real["E_c"] + rec["E"] + exc["E"] + oracle.ewald_self(s)
    return real["F"] + rec["F"] + exc["F"], E


def test_full_ewald_sum_matches_exact_direct_sum(api):
    s = water_ewald()
    Fx, Ex = exact_ewald(s)
    # fine PME: the interpolation error is below the FP32 level
    f, E = full_ewald(api, s, api.pme_grid(s.box, 0.06), 8)
    assert rms_rel(f, Fx) < 1e-5
    assert rel(E, Ex) < 1e-5
    # the usual settings (order 4, 0.12 nm): equal to the FP64 sum with the same PME,
    # which differs from the exact sum by the interpolation error (~2e-3 of the total force)
    grid4 = api.pme_grid(s.box, 0.12)
    f4, E4 = full_ewald(api, s, grid4, 4)
    real, exc = oracle.brute(s), oracle.ewald_excl(s)
    p4 = oracle.pme(s, grid=grid4, order=4)
    F4 = real["F"] + p4["F"] + exc["F"]
    E4x = real["E_lj"] + real["E_c"] + p4["E"] + exc["E"] + oracle.ewald_self(s)
    assert_forces(f4, F4)
    assert rel(E4, E4x) < 1e-5
    assert 1e-4 < rms_rel(f4, Fx) < 5e-3


def test_madelung_constant_through_the_gpu_path(api):
    a, cells = 0.5640, 3
    L = a * cells
    rc = 0.499 * L
    s = synth.ionic_crystal("NaCl", a=a, cells=cells, beta=3.95 / rc, rc=rc)
    f, E = full_ewald(api, s, api.pme_grid(s.box, 0.04), 8)
    M = -E / (s.n / 2 * 138.935458 / (0.5 * a))
    assert M == pytest.approx(1.747564594633, rel=2e-6)
    assert np.abs(f).max() < 1e-3 * 138.935458 / (0.5 * a) ** 2


def test_pme_in_a_cuda_graph(api):
    import torch
    s = water_ewald()
    grid = api.pme_grid(s.box, 0.12)
    x = torch.tensor(s.x, device="cuda")
    q = torch.tensor(s.q, device="cuda")
    pme = api.NbPme(s.n, s.beta, grid=grid, order=4, eps_r=s.eps_r)
    f = torch.zeros((s.n, 3), dtype=torch.float32, device="cuda")
    e = torch.empty(1, dtype=torch.float64, device="cuda")
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        pme.nb_pme_forces(1, x, q, s.box, f, e)  # warm-up outside capture
    torch.cuda.synchronize()
    e0 = e.item()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        f.zero_()
        pme.nb_pme_forces(1, x, q, s.box, f, e)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    ref = oracle.pme(s, grid=grid, order=4)
    assert rel(e.item(), e0) < 1e-6 and rms_rel(f.cpu().numpy(), ref["F"]) < 1e-5
