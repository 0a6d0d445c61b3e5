"""Pins of the Ewald long-range oracle (ewald.c, pme.py) against facts it does not
compute itself: Madelung constants of ionic crystals, the independence of the
total Ewald sum from the splitting parameter, finite differences, box-scaling
virials, the image-dipole energy of one molecule in a large box, and the
convergence of smooth PME to the exact reciprocal sum."""
import math

import numpy as np
import pytest

import oracle
from paper_2006_09167_gb300 import synth

F = 138.935458


def water_ewald():
    """The 648-atom water box with Ewald electrostatics (beta from erfc(beta rc) = 1e-5 at rc 0.9)."""
    w = synth.water_648()
    return synth.System(**{**w.__dict__, "coulomb": synth.COULOMB_EWALD, "beta": synth.ewald_beta(w.rc)})


def total_ewald(s, beta=None, x=None):
    """Real-space pairs inside rc (oracle brute force, Ewald flavour) + reciprocal + self + exclusion."""
    b = s.beta if beta is None else beta
    t = synth.System(**{**s.__dict__, "beta": b, "coulomb": synth.COULOMB_EWALD})
    real = oracle.brute(t, x)
    rec = oracle.ewald_recip(t, x)
    exc = oracle.ewald_excl(t, x)
    E = real["E_c"] + real["E_lj"] + rec["E"] + exc["E"] + oracle.ewald_self(t)
    return E, real["F"] + rec["F"] + exc["F"]


@pytest.mark.parametrize("kind,a,cells,madelung,r0_over_a", [
    ("NaCl", 0.5640, 2, 1.747564594633, 0.5),
    ("CsCl", 0.4123, 3, 1.762674773070, math.sqrt(3) / 2),
])
def test_madelung_constants(kind, a, cells, madelung, r0_over_a):
    # beta * rc >= 4.5 makes the real-space truncation (and the potential shift) < 1e-9 relative
    L = cells * a
    s = synth.ionic_crystal(kind, a=a, cells=cells, beta=9.5 / L)
    E, Fo = total_ewald(s)
    n_pairs = s.n / 2
    M = -E / (n_pairs * F / (r0_over_a * a))
    assert M == pytest.approx(madelung, rel=2e-7)
    # every ion sits at a centre of symmetry: no force
    assert np.abs(Fo).max() < 1e-6 * F / (r0_over_a * a) ** 2


def test_total_independent_of_beta():
    s = synth.System(**{**water_ewald().__dict__, "rc": 0.92})
    E1, F1 = total_ewald(s, beta=4.9)
    E2, F2 = total_ewald(s, beta=5.6)
    assert E1 == pytest.approx(E2, rel=2e-8, abs=1e-5)
    assert np.sqrt(((F1 - F2) ** 2).sum() / (F1 ** 2).sum()) < 1e-7
    # and a beta change moves each part by much more than that
    r1 = oracle.ewald_recip(synth.System(**{**s.__dict__, "beta": 4.9}))["E"]
    r2 = oracle.ewald_recip(synth.System(**{**s.__dict__, "beta": 5.6}))["E"]
    assert abs(r1 - r2) > 1e3 * abs(E1 - E2)


def test_reciprocal_forces_are_minus_gradient():
    s = water_ewald()
    base = oracle.ewald_recip(s)
    x0 = s.x.astype(np.float64)
    rng = np.random.default_rng(3)
    h = 1e-5
    for i in rng.choice(s.n, 6, replace=False):
        for a in range(3):
            xp = x0.copy()
            xm = x0.copy()
            xp[i, a] += h
            xm[i, a] -= h
            fd = -(oracle.ewald_recip(s, xp)["E"] - oracle.ewald_recip(s, xm)["E"]) / (2 * h)
            assert base["F"][i, a] == pytest.approx(fd, rel=1e-6, abs=1e-6)


def test_exclusion_forces_are_minus_gradient():
    s = water_ewald()
    base = oracle.ewald_excl(s)
    x0 = s.x.astype(np.float64)
    h = 1e-6
    for i in (0, 1, 2, 300):
        for a in range(3):
            xp = x0.copy()
            xm = x0.copy()
            xp[i, a] += h
            xm[i, a] -= h
            fd = -(oracle.ewald_excl(s, xp)["E"] - oracle.ewald_excl(s, xm)["E"]) / (2 * h)
            assert base["F"][i, a] == pytest.approx(fd, rel=1e-6, abs=1e-6)


@pytest.mark.parametrize("part", ["recip", "excl"])
def test_virial_from_box_scaling(part):
    """W_aa = 1/2 dE/d(eps_aa) for scaling axis a of the box and of all coordinates."""
    s = water_ewald()
    fn = oracle.ewald_recip if part == "recip" else oracle.ewald_excl
    W = fn(s)["W"]
    h = 1e-6
    for a in range(3):
        def energy(eps):
            sc = np.ones(3)
            sc[a] += eps
            t = synth.System(**{**s.__dict__, "box": s.box * sc})
            return fn(t, s.x.astype(np.float64) * sc)["E"]
        dE = (energy(h) - energy(-h)) / (2 * h)
        assert W[a, a] == pytest.approx(0.5 * dE, rel=1e-6, abs=1e-4)


def test_single_molecule_image_dipole_energy():
    """One neutral water in a cubic box with tin-foil boundaries: reciprocal + self +
    exclusion terms leave only the image-dipole energy -2 pi f mu^2 / (3 L^3)."""
    w = synth.water_648()
    x = w.x[:3].astype(np.float64)
    q = w.q[:3].astype(np.float64)
    mu = (q[:, None] * x).sum(0)
    mu2 = float(mu @ mu)
    devs = []
    for L in (4.0, 6.0, 8.0):
        xx = x - x.mean(0) + L / 2
        off = np.array([0, 2, 4, 6], np.int32)
        idx = np.array([1, 2, 0, 2, 0, 1], np.int32)
        s = synth.System(name="one", x=xx.astype(np.float32), q=w.q[:3], types=w.types[:3], c6=w.c6, c12=w.c12,
                         excl_off=off, excl_idx=idx, box=np.full(3, L), coulomb=1, rc=1.0, rlist=1.0, r_in=1.0,
                         beta=3.0)
        xs = s.x.astype(np.float64)
        E = oracle.ewald_recip(s, xs)["E"] + oracle.ewald_excl(s, xs)["E"] + oracle.ewald_self(s)
        expect = -2 * math.pi * F * mu2 / (3 * L ** 3)
        devs.append(abs(E / expect - 1))
    # higher multipoles fall off faster than the dipole term
    assert devs[-1] < 0.02 and devs[0] > devs[1] > devs[2]


def test_bspline_partition_of_unity_and_derivative():
    from oracle.pme import bspline
    w = np.linspace(0, 1, 101, endpoint=False)
    for n in (3, 4, 5, 6, 8):
        m, dm = bspline(w, n)
        assert np.allclose(m.sum(1), 1.0, atol=1e-14)
        assert np.allclose(dm.sum(1), 0.0, atol=1e-13)
        # M_n(u) matches the closed form for n = 4 (cubic B-spline)
        if n == 4:
            def m4(u):
                return np.where(u < 1, u ** 3 / 6, np.where(u < 2, (-3 * u ** 3 + 12 * u ** 2 - 12 * u + 4) / 6,
                                np.where(u < 3, (3 * u ** 3 - 24 * u ** 2 + 60 * u - 44) / 6, (4 - u) ** 3 / 6)))
            for j in range(4):
                assert np.allclose(m[:, j], m4(w + j), atol=1e-14)
        # derivative by central differences
        eps = 1e-6
        mp, _ = bspline(np.clip(w + eps, 0, 1 - 1e-12), n)
        mm, _ = bspline(np.clip(w - eps, 0, 1), n)
        inner = (w > 2 * eps) & (w < 1 - 2 * eps)
        assert np.allclose(((mp - mm) / (2 * eps))[inner], dm[inner], atol=1e-6)


def test_pme_converges_to_the_exact_reciprocal_sum():
    s = water_ewald()
    ref = oracle.ewald_recip(s)
    errs = []
    for order, spacing in ((4, 0.12), (6, 0.08), (8, 0.04)):
        grid = oracle.pme_grid(s.box, spacing)
        p = oracle.pme(s, grid=grid, order=order)
        ef = np.sqrt(((p["F"] - ref["F"]) ** 2).sum() / (ref["F"] ** 2).sum())
        ee = abs(p["E"] - ref["E"]) / abs(ref["E"])
        ew = np.abs(p["W"] - ref["W"]).max() / np.abs(ref["W"]).max()
        errs.append((ef, ee, ew, np.abs(p["F"].sum(0)).max()))
    # the usual settings (order 4, 0.12 nm) carry a ~1e-2 interpolation error; it falls
    # by orders of magnitude with the order and the grid
    assert errs[0][0] < 1e-2 and errs[1][0] < 5e-5 and errs[2][0] < 1e-8
    assert errs[2][1] < 1e-8 and errs[2][2] < 5e-8
    assert errs[0][0] > errs[1][0] > errs[2][0]
    # the net PME force vanishes with the interpolation error
    assert errs[0][3] > errs[1][3] > errs[2][3] and errs[2][3] < 1e-4


def test_pme_grid_sizes():
    assert oracle.pme_grid(np.array([9.86, 9.86, 9.86])) == (84, 84, 84)
    for K in oracle.pme_grid(np.array([1.862, 3.1, 24.63]), 0.12):
        m = K
        for p in (2, 3, 5, 7):
            while m % p == 0:
                m //= p
        assert m == 1 and K % 2 == 0
