"""Degenerate inputs of the cluster pair path against the FP64 oracle: a single
atom, two atoms inside and outside the cut-off, one full plus one partial
cluster, all atoms in one plane, the maximum number of atom types, a fully
excluded molecule, an empty pair list and a cut-off just below half the box."""
import math

import numpy as np
import pytest

import oracle
from helpers import EPS32, TOL_F, assert_forces, energy_tolerances, rel
from paper_2006_09167_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_09167_gb300 import api as a
    return a


def make_system(x, box, *, q=None, types=None, c6=None, c12=None, pairs=None, coulomb=synth.COULOMB_RF, rc=0.9,
                rlist=1.0):
    x = np.asarray(x, np.float32).reshape(-1, 3)
    n = x.shape[0]
    q = np.asarray(q if q is not None else np.zeros(n), np.float32)
    types = np.asarray(types if types is not None else np.zeros(n), np.int32)
    T = int(types.max()) + 1 if c6 is None else np.asarray(c6).shape[0]
    c6 = np.asarray(c6 if c6 is not None else np.full((T, T), 0.0026), np.float32)
    c12 = np.asarray(c12 if c12 is not None else np.full((T, T), 2.6e-6), np.float32)
    off, idx = synth.csr_from_pairs(n, np.zeros((0, 2)) if pairs is None else pairs)
    beta = synth.ewald_beta(rc) if coulomb == synth.COULOMB_EWALD else 0.0
    return synth.System(name="edge", x=x, q=q, types=types, c6=c6, c12=c12, excl_off=off, excl_idx=idx,
                        box=np.asarray(box, np.float64), coulomb=coulomb, rc=rc, rlist=rlist, r_in=rc, beta=beta)


def run(api, s):
    import torch
    ctx = api.NbContext.from_system(s)
    x = torch.tensor(s.x, device="cuda")
    ctx.build(x, s.box)
    f, e, w = ctx.forces(x, energy=True, virial=True)
    torch.cuda.synchronize()
    assert ctx.nb_get_error() == 0
    return f.cpu().numpy().astype(np.float64), e.cpu().numpy(), w.cpu().numpy()


def check(api, s, force_scale=None, energy_scale=None):
    """Forces within TOL_F (relative RMS; or TOL_F times force_scale, the size of the
    terms a force is the difference of, where it nearly cancels); energies within the
    suite's bars (1e-6, or the FP32 rounding floor of the sum where it is higher: near
    the cut-off a shifted potential is a tiny difference of large terms)."""
    f, e, w = run(api, s)
    ref = oracle.brute(s)
    if force_scale is not None:
        assert np.abs(f - ref["F"]).max() < TOL_F * force_scale, (f, ref["F"])
    elif np.abs(ref["F"]).max() > 0:
        assert_forces(f, ref)
    else:
        assert np.all(f == 0)
    if energy_scale is not None:
        # absolute: a few FP32 roundings of the terms each energy is the difference of
        for got, exp, sc in zip(e, (ref["E_lj"], ref["E_c"]), energy_scale):
            assert abs(got - exp) <= 8 * EPS32 * sc, (got, exp, sc)
        return f, e, w, ref
    tol_lj, tol_c = energy_tolerances(s, ref)
    for got, exp, tol in ((e[0], ref["E_lj"], tol_lj), (e[1], ref["E_c"], tol_c)):
        if exp == 0.0:
            assert got == 0.0
        else:
            assert rel(got, exp) < tol, (got, exp, tol)
    return f, e, w, ref


def test_single_atom(api):
    s = make_system([[1.0, 1.0, 1.0]], [3.0, 3.0, 3.0], q=[0.5])
    f, e, w = run(api, s)
    assert np.all(f == 0) and np.all(e == 0) and np.all(w == 0)


@pytest.mark.parametrize("coulomb", [synth.COULOMB_RF, synth.COULOMB_EWALD, synth.COULOMB_NONE])
@pytest.mark.parametrize("r", [0.31, 0.8999, 0.95])
def test_two_atoms(api, coulomb, r):
    s = make_system([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]], [3.0, 3.0, 3.0], q=[0.4, -0.4], coulomb=coulomb)
    # with eps_rf = inf the reaction-field force vanishes at rc: near rc it is the
    # difference of terms of size f q q / r^2 (and the LJ terms 12 C12/r^13, 6 C6/r^7)
    scale = 138.935458 * 0.16 / r ** 2 + 12 * 2.6e-6 / r ** 13 + 6 * 0.0026 / r ** 7
    # energies: V_LJ = C12/r^12 - C6/r^6 - shift, V_C = f qq (1/r + k_rf r^2 - c_rf) (or erfc(beta r)/r - shift)
    e_scale = (2.6e-6 / r ** 12 + 0.0026 / r ** 6 + 2.6e-6 / 0.9 ** 12 + 0.0026 / 0.9 ** 6,
               138.935458 * 0.16 * (1 / r + 0.5 * r ** 2 / 0.9 ** 3 + 1.5 / 0.9))
    f, e, w, ref = check(api, s, force_scale=scale, energy_scale=e_scale)
    if r >= s.rc:
        assert np.all(f == 0) and np.all(e == 0)
    else:
        assert np.abs(f.sum(0)).max() <= 1e-6 * np.abs(f).max()


def test_two_atoms_across_the_boundary(api):
    # the pair vector crosses the periodic boundary on all three axes
    s = make_system([[0.05, 0.05, 0.05], [2.85, 2.9, 2.95]], [3.0, 3.0, 3.0], q=[0.3, 0.3])
    check(api, s)


def test_full_plus_partial_cluster(api):
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 2.5, (9, 3))
    s = make_system(x, [2.5, 2.5, 2.5], q=rng.normal(0, 0.3, 9), rc=1.0, rlist=1.1)
    check(api, s)


def test_all_atoms_in_one_plane(api):
    rng = np.random.default_rng(6)
    n = 400
    x = np.column_stack([rng.uniform(0, 4, n), rng.uniform(0, 4, n), np.full(n, 1.3)])
    # keep atoms at least 0.15 nm apart so the LJ terms stay moderate
    keep = [0]
    for i in range(1, n):
        if np.min(np.linalg.norm(x[keep] - x[i], axis=1)) > 0.15:
            keep.append(i)
    x = x[keep]
    s = make_system(x, [4.0, 4.0, 4.0], q=rng.normal(0, 0.3, len(x)), rc=1.0, rlist=1.1)
    check(api, s)


def test_maximum_number_of_types(api):
    rng = np.random.default_rng(7)
    w = synth.water_648()
    T = 64
    types = rng.integers(0, T, w.n)
    sig = rng.uniform(0.25, 0.35, T)
    eps = rng.uniform(0.2, 1.0, T)
    c6t, c12t = synth.lj_c6_c12(sig, eps)
    c6, c12 = synth.geometric_tables(c6t, c12t)
    s = synth.System(**{**w.__dict__, "types": types.astype(np.int32), "c6": c6, "c12": c12})
    check(api, s)


def test_fully_excluded_molecule(api):
    w = synth.water_648()
    x = w.x[:3]
    s = make_system(x, [3.0, 3.0, 3.0], q=w.q[:3], pairs=[[0, 1], [0, 2], [1, 2]])
    f, e, wv = run(api, s)
    assert np.all(f == 0) and np.all(e == 0) and np.all(wv == 0)


def test_no_pair_within_rlist(api):
    # 8 atoms on a 2 nm lattice in a 4 nm box: every distance exceeds rlist
    g = np.array([[i, j, k] for i in range(2) for j in range(2) for k in range(2)], np.float64) * 2.0 + 0.5
    s = make_system(g, [4.0, 4.0, 4.0], q=np.linspace(-0.5, 0.5, 8))
    f, e, w = run(api, s)
    assert np.all(f == 0) and np.all(e == 0) and np.all(w == 0)


def test_cutoff_just_below_half_the_box(api):
    w = synth.water_648()
    s = synth.System(**{**w.__dict__, "rc": 0.9305, "rlist": 1.0, "r_in": 0.9305})
    assert s.rc < s.box[0] / 2
    check(api, s)
