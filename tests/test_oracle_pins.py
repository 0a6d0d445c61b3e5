"""Pins for the FP64 oracle, against facts other than the oracle itself.

Each check is chosen so that a plausible slip in oracle.c (a dropped term, a
wrong sign or exponent, a transposed table index, a mishandled exclusion or
periodic image) fails at least one of them:
  - closed-form properties of the pair potentials (LJ minimum at 2^(1/6) sigma
    with depth eps, zero crossing at sigma; reaction-field force and energy
    vanishing at rc for eps_rf = inf; the eps_rf = eps_r and beta -> 0 special
    cases reducing to plain cut-off Coulomb; the Coulomb constant from CODATA;
    erfc from an independent multiprecision routine),
  - F = -dE/dx by central differences, Newton's third law, translation and
    permutation invariance, pairwise additivity with exclusions,
  - the virial from box-scaling and shear derivatives of the energy,
  - the cell list against brute force, the image-pair evaluator against brute
    force, the pair set against a numpy distance matrix (brute force on tiny inputs),
  - the analytic adjoint against central differences.
"""
import dataclasses
import math

import mpmath
import numpy as np
import pytest

import oracle
from paper_2006_09167_gb300 import synth


def make_sys(x, q, types, c6, c12, box, coulomb=synth.COULOMB_RF, rc=0.9, eps_rf=math.inf,
             beta=0.0, excl_pairs=()):
    n = len(x)
    off, idx = synth.csr_from_pairs(n, np.array(excl_pairs, dtype=np.int64).reshape(-1, 2))
    return synth.System(name="t", x=np.asarray(x, np.float64), q=np.asarray(q, np.float64),
                        types=np.asarray(types, np.int32), c6=np.asarray(c6, np.float64),
                        c12=np.asarray(c12, np.float64), excl_off=off, excl_idx=idx,
                        box=np.asarray(box, np.float64), coulomb=coulomb, rc=rc, rlist=rc,
                        r_in=rc, eps_rf=eps_rf, beta=beta)


def two_atoms(r, q=(0.0, 0.0), sigma=0.34, eps=0.8, **kw):
    c6, c12 = synth.lj_c6_c12(sigma, eps)
    box = kw.pop("box", [5.0, 5.0, 5.0])
    return make_sys([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]], q, [0, 0], [[c6]], [[c12]], box, **kw)


def energy(s, x=None):
    o = oracle.brute(s, x)
    return o["E_lj"] + o["E_c"]


# --------------------------------------------------------------- closed forms
def test_coulomb_constant_from_codata():
    e = 1.602176634e-19
    na = 6.02214076e23
    eps0 = 8.8541878128e-12
    f_codata = e * e * na / (4 * math.pi * eps0) / 1e-9 / 1e3  # kJ mol^-1 nm e^-2
    # two unit charges at 0.5 nm, eps_rf = eps_r: V = f (1/r - 1/rc)
    s = two_atoms(0.5, q=(1.0, 1.0), eps=0.0, rc=1.2, eps_rf=1.0)
    v = oracle.brute(s)["E_c"]
    assert v == pytest.approx(f_codata * (1 / 0.5 - 1 / 1.2), rel=2e-8)


def test_lj_minimum_depth_and_zero_crossing():
    sigma, eps = 0.34, 0.8
    rmin = 2 ** (1 / 6) * sigma
    s = two_atoms(rmin, sigma=sigma, eps=eps)
    o = oracle.brute(s)
    scale = 12 * eps / sigma  # magnitude of LJ forces near sigma
    assert abs(o["F"][0, 0]) < 1e-10 * scale
    v_min = o["E_lj"]
    v_sig = oracle.brute(two_atoms(sigma, sigma=sigma, eps=eps))["E_lj"]
    # the shift cancels in the difference: V(rmin) - V(sigma) = -eps
    assert v_min - v_sig == pytest.approx(-eps, rel=1e-12)
    # the shift makes the energy vanish at the cut-off
    v_rc = oracle.brute(two_atoms(0.9 * (1 - 1e-12), sigma=sigma, eps=eps))["E_lj"]
    assert abs(v_rc) < 1e-9
    # repulsive inside rmin: force on atom 0 points away from atom 1 (-x)
    assert oracle.brute(two_atoms(0.95 * rmin, sigma=sigma, eps=eps))["F"][0, 0] < 0
    # outside the cut-off nothing
    o_out = oracle.brute(two_atoms(0.9 * (1 + 1e-9), sigma=sigma, eps=eps))
    assert o_out["npairs"] == 0 and o_out["E_lj"] == 0.0


def test_reaction_field_vanishes_at_cutoff():
    for rc in (0.9, 1.1):
        s = two_atoms(rc * (1 - 1e-10), q=(0.7, -0.4), eps=0.0, rc=rc)
        o = oracle.brute(s)
        assert abs(o["E_c"]) < 1e-7
        assert np.abs(o["F"]).max() < 1e-6
        # like charges repel at short range
        s2 = two_atoms(0.3, q=(0.5, 0.5), eps=0.0, rc=rc)
        assert oracle.brute(s2)["F"][0, 0] < 0


def test_reaction_field_finite_eps_rf_limits():
    # eps_rf = eps_r gives k_rf = 0: plain shifted Coulomb, V = f qq (1/r - 1/rc)
    s = two_atoms(0.4, q=(0.5, -0.3), eps=0.0, rc=1.0, eps_rf=1.0)
    o = oracle.brute(s)
    f = 138.935458
    assert o["E_c"] == pytest.approx(f * 0.5 * -0.3 * (1 / 0.4 - 1.0), rel=1e-12)
    # a large finite eps_rf approaches the conducting limit
    e_inf = oracle.brute(two_atoms(0.4, q=(0.5, -0.3), eps=0.0, rc=1.0))["E_c"]
    e_big = oracle.brute(two_atoms(0.4, q=(0.5, -0.3), eps=0.0, rc=1.0, eps_rf=1e9))["E_c"]
    assert e_big == pytest.approx(e_inf, rel=1e-8)


def test_ewald_small_beta_is_plain_cutoff_coulomb():
    s_ew = two_atoms(0.37, q=(0.8, -0.6), eps=0.0, rc=1.0, coulomb=synth.COULOMB_EWALD, beta=1e-7)
    s_pl = two_atoms(0.37, q=(0.8, -0.6), eps=0.0, rc=1.0, eps_rf=1.0)
    a, b = oracle.brute(s_ew), oracle.brute(s_pl)
    assert a["E_c"] == pytest.approx(b["E_c"], rel=1e-9)
    assert a["F"][0, 0] == pytest.approx(b["F"][0, 0], rel=1e-9)


@pytest.mark.parametrize("r", [0.12, 0.3, 0.55, 0.8, 0.99])
def test_ewald_energy_against_multiprecision_erfc(r):
    beta, rc = 3.123413274340875, 1.0
    qq = 0.8 * -0.6
    s = two_atoms(r, q=(0.8, -0.6), eps=0.0, rc=rc, coulomb=synth.COULOMB_EWALD, beta=beta)
    mpmath.mp.dps = 40
    ref = 138.935458 * qq * (float(mpmath.erfc(beta * r)) / r - float(mpmath.erfc(beta * rc)) / rc)
    assert oracle.brute(s)["E_c"] == pytest.approx(ref, rel=1e-12, abs=1e-14)


def test_generator_beta_solves_rtol():
    mpmath.mp.dps = 30
    for rc, beta in ((1.0, synth.ewald_beta(1.0)), (1.2, synth.ewald_beta(1.2))):
        assert float(mpmath.erfc(beta * rc)) == pytest.approx(1e-5, rel=1e-9)
    assert synth.ewald_beta(1.0) == pytest.approx(3.123413, abs=1e-6)
    assert synth.ewald_beta(1.2) == pytest.approx(2.602844, abs=1e-6)


# ------------------------------------------------------- small random systems
def random_system(n=60, L=2.3, seed=0, coulomb=synth.COULOMB_EWALD, rc=1.0, n_types=3,
                  excl_frac=0.05, min_dist=0.18):
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < n:
        p = rng.uniform(0, L, 3)
        ok = True
        for o in pts:
            d = p - o
            d -= L * np.rint(d / L)
            if np.dot(d, d) < min_dist ** 2:
                ok = False
                break
        if ok:
            pts.append(p)
    x = np.array(pts)
    sig = rng.uniform(0.25, 0.35, n_types)
    eps = rng.uniform(0.3, 1.0, n_types)
    c6t, c12t = synth.lj_c6_c12(sig, eps)
    c6 = np.sqrt(np.outer(c6t, c6t))
    c12 = np.sqrt(np.outer(c12t, c12t))
    types = rng.integers(0, n_types, n)
    q = rng.normal(0, 0.5, n)
    allp = [(i, j) for i in range(n) for j in range(i + 1, n)]
    sel = rng.choice(len(allp), size=int(excl_frac * n), replace=False)
    ex = [allp[k] for k in sel]
    beta = synth.ewald_beta(rc) if coulomb == synth.COULOMB_EWALD else 0.0
    return make_sys(x, q, types, c6, c12, [L, L, L], coulomb=coulomb, rc=rc, beta=beta,
                    excl_pairs=ex)


@pytest.mark.parametrize("coulomb", [synth.COULOMB_RF, synth.COULOMB_EWALD])
def test_forces_are_minus_energy_gradient(coulomb):
    s = random_system(n=40, seed=1, coulomb=coulomb)
    o = oracle.brute(s)
    rng = np.random.default_rng(5)
    h = 1e-6
    for i in rng.choice(s.n, 8, replace=False):
        for k in range(3):
            xp = s.x.copy()
            xm = s.x.copy()
            xp[i, k] += h
            xm[i, k] -= h
            fd = -(energy(s, xp) - energy(s, xm)) / (2 * h)
            assert fd == pytest.approx(o["F"][i, k], rel=2e-6, abs=2e-4)


def test_newton_third_law_and_invariances():
    s = random_system(n=70, seed=2)
    o = oracle.brute(s)
    fnorm = np.abs(o["F"]).sum()
    assert np.abs(o["F"].sum(0)).max() < 1e-12 * fnorm
    # translation (with re-wrapping) leaves everything unchanged
    t = np.array([0.71, -1.3, 2.9])
    x2 = np.mod(s.x + t, s.box)
    o2 = oracle.brute(s, x2)
    assert np.allclose(o2["F"], o["F"], rtol=1e-10, atol=1e-9 * np.abs(o["F"]).max())
    assert o2["E_lj"] == pytest.approx(o["E_lj"], rel=1e-11)
    assert o2["E_c"] == pytest.approx(o["E_c"], rel=1e-11)
    # permutation of the atom order permutes the forces
    perm = np.random.default_rng(3).permutation(s.n)
    inv = np.argsort(perm)
    ex = [(inv[i], inv[j]) for i in range(s.n)
          for j in s.excl_idx[s.excl_off[i]:s.excl_off[i + 1]] if i < j]
    sp = make_sys(s.x[perm], s.q[perm], s.types[perm], s.c6, s.c12, s.box, coulomb=s.coulomb,
                  rc=s.rc, beta=s.beta, excl_pairs=ex)
    op = oracle.brute(sp)
    assert np.allclose(op["F"], o["F"][perm], rtol=1e-10, atol=1e-9 * np.abs(o["F"]).max())
    assert op["E_c"] == pytest.approx(o["E_c"], rel=1e-11)


def test_pairwise_additivity_and_exclusions():
    s = random_system(n=30, seed=4, excl_frac=0.3)
    total = energy(s)
    no_ex = dataclasses.replace(s, excl_off=np.zeros(s.n + 1, np.int32), excl_idx=np.zeros(0, np.int32))
    total_noex = energy(no_ex)
    # sum of two-atom energies over the excluded pairs, each evaluated alone in the same box
    ex_sum = 0.0
    for i in range(s.n):
        for j in s.excl_idx[s.excl_off[i]:s.excl_off[i + 1]]:
            if i < j:
                sub = synth.subsystem(no_ex, np.array([i, j]))
                ex_sum += energy(sub)
    assert total_noex - total == pytest.approx(ex_sum, rel=1e-10, abs=1e-10)
    # and the total is the sum over all non-excluded two-atom energies
    pair_sum = 0.0
    exset = {(i, j) for i in range(s.n) for j in s.excl_idx[s.excl_off[i]:s.excl_off[i + 1]]}
    for i in range(s.n):
        for j in range(i + 1, s.n):
            if (i, j) not in exset:
                pair_sum += energy(synth.subsystem(no_ex, np.array([i, j])))
    assert total == pytest.approx(pair_sum, rel=1e-10)


def test_virial_from_box_scaling():
    s = random_system(n=50, seed=6, coulomb=synth.COULOMB_RF)
    W = oracle.brute(s)["W"]
    h = 1e-6
    for a in range(3):
        sc = np.ones(3)
        sc[a] = 1 + h
        sp = dataclasses.replace(s, box=s.box * sc)
        sc[a] = 1 - h
        sm = dataclasses.replace(s, box=s.box * sc)
        sc[a] = 1 + h
        ep = energy(sp, s.x * np.where(np.arange(3) == a, 1 + h, 1.0))
        em = energy(sm, s.x * np.where(np.arange(3) == a, 1 - h, 1.0))
        # x_a -> (1+e) x_a:  dE/de = -sum phi r_a^2 = 2 W_aa
        assert (ep - em) / (2 * h) == pytest.approx(2 * W[a, a], rel=1e-5, abs=1e-5)
    assert np.allclose(W, W.T, atol=1e-10 * np.abs(W).max())


def test_virial_offdiagonal_from_shear_of_isolated_cluster():
    # atoms confined to a small region of a large box: no periodic image is within rc,
    # so an affine shear x_a -> x_a + e x_b is a valid deformation; dE/de = 2 W_ab
    rng = np.random.default_rng(8)
    core = random_system(n=25, L=1.6, seed=8, coulomb=synth.COULOMB_RF, rc=0.7)
    s = dataclasses.replace(core, box=np.array([9.0, 9.0, 9.0]), x=core.x + 3.0)
    W = oracle.brute(s)["W"]
    h = 1e-6
    for a, b in ((0, 1), (0, 2), (1, 2), (2, 0)):
        xp = s.x.copy()
        xm = s.x.copy()
        xp[:, a] += h * (s.x[:, b] - 4.0)
        xm[:, a] -= h * (s.x[:, b] - 4.0)
        d = (energy(s, xp) - energy(s, xm)) / (2 * h)
        assert d == pytest.approx(2 * W[a, b], rel=1e-5, abs=1e-5)
    del rng


def test_celllist_equals_brute():
    s = synth.water_box(300, 2.1 * 1.0 * 3.0 ** 0 * 1.5, seed=11, rc=0.9, rlist=1.0)
    a, b = oracle.brute(s), oracle.celllist(s)
    assert a["npairs"] == b["npairs"]
    assert np.allclose(a["F"], b["F"], rtol=1e-12, atol=1e-12 * np.abs(a["F"]).max())
    assert b["E_c"] == pytest.approx(a["E_c"], rel=1e-12)
    assert b["E_lj"] == pytest.approx(a["E_lj"], rel=1e-12)
    assert np.allclose(a["W"], b["W"], rtol=1e-11, atol=1e-11 * np.abs(a["W"]).max())
    sub = np.array([0, 5, 17, 299, 400, 899])
    fs = oracle.celllist(s, subset=sub)["F"]
    assert np.allclose(fs, a["F"][sub], rtol=1e-12, atol=1e-12 * np.abs(a["F"]).max())


def test_listset_equals_brute_and_ignores_far_pairs():
    s = random_system(n=60, seed=9)
    a = oracle.brute(s)
    p_rc = oracle.pairs_within(s, s.rc)
    b = oracle.listset(s, p_rc)
    assert b["npairs"] == a["npairs"]
    assert np.allclose(a["F"], b["F"], rtol=1e-12, atol=1e-12 * np.abs(a["F"]).max())
    assert b["E_c"] == pytest.approx(a["E_c"], rel=1e-12)
    # adding every pair out to 1.15 nm (and far images) changes nothing
    p_far = oracle.pairs_within(s, 1.15)
    extra = p_far.copy()
    extra[:, 2] += 1  # a far image of each pair
    c = oracle.listset(s, np.concatenate([p_far, extra]))
    assert c["npairs"] == a["npairs"]
    assert c["E_lj"] == pytest.approx(a["E_lj"], rel=1e-12)


def test_pairs_within_against_distance_matrix():
    s = random_system(n=45, seed=12, excl_frac=0.1)
    d = s.x[:, None, :] - s.x[None, :, :]
    d -= s.box * np.rint(d / s.box)
    r = np.sqrt((d * d).sum(-1))
    exset = {(i, j) for i in range(s.n) for j in s.excl_idx[s.excl_off[i]:s.excl_off[i + 1]]}
    want = {(i, j) for i in range(s.n) for j in range(i + 1, s.n)
            if r[i, j] < 0.8 and (i, j) not in exset}
    got = oracle.pairs_within(s, 0.8)
    assert {(int(a), int(b)) for a, b in got[:, :2]} == want
    # recorded shifts reproduce the minimum-image vector
    for i, j, sx, sy, sz in got:
        v = s.x[i] - s.x[j] + np.array([sx, sy, sz]) * s.box
        assert np.linalg.norm(v) < 0.8


def _loss(s, gF, gE, x=None, q=None, c6=None, c12=None):
    s2 = dataclasses.replace(s, q=s.q if q is None else q, c6=s.c6 if c6 is None else c6,
                             c12=s.c12 if c12 is None else c12)
    o = oracle.brute(s2, x)
    return float((gF * o["F"]).sum() + gE * (o["E_lj"] + o["E_c"]))


@pytest.mark.parametrize("coulomb", [synth.COULOMB_RF, synth.COULOMB_EWALD])
def test_vjp_against_central_differences(coulomb):
    s = random_system(n=36, seed=13, coulomb=coulomb, n_types=3)
    rng = np.random.default_rng(14)
    gF = rng.normal(size=(s.n, 3))
    gE = 0.37
    g = oracle.vjp(s, gF, gE)
    h = 1e-6
    for i in rng.choice(s.n, 6, replace=False):
        for k in range(3):
            xp = s.x.copy()
            xm = s.x.copy()
            xp[i, k] += h
            xm[i, k] -= h
            fd = (_loss(s, gF, gE, x=xp) - _loss(s, gF, gE, x=xm)) / (2 * h)
            assert fd == pytest.approx(g["gx"][i, k], rel=1e-5, abs=1e-3)
    for i in rng.choice(s.n, 6, replace=False):
        hq = 1e-6
        qp = s.q.copy()
        qm = s.q.copy()
        qp[i] += hq
        qm[i] -= hq
        fd = (_loss(s, gF, gE, q=qp) - _loss(s, gF, gE, q=qm)) / (2 * hq)
        assert fd == pytest.approx(g["gq"][i], rel=1e-6, abs=1e-4)
    # parameter tables: perturb (a,b) and (b,a) together (a symmetric direction)
    T = s.c6.shape[0]
    for a in range(T):
        for b in range(a, T):
            for name in ("c6", "c12"):
                tab = getattr(s, name)
                hp = 1e-4 * abs(tab[a, b])
                tp = tab.copy()
                tm = tab.copy()
                tp[a, b] += hp
                tm[a, b] -= hp
                if a != b:
                    tp[b, a] += hp
                    tm[b, a] -= hp
                fd = (_loss(s, gF, gE, **{name: tp}) - _loss(s, gF, gE, **{name: tm})) / (2 * hp)
                ga = g["g" + name]
                an = ga[a, b] + (ga[b, a] if a != b else 0.0)
                assert fd == pytest.approx(an, rel=1e-5, abs=1e-6 * max(1.0, abs(an)))
    # a single off-diagonal slot carries half of the symmetric derivative
    assert np.allclose(g["gc6"], g["gc6"].T)


def test_energy_moments_are_squared_radial_derivatives():
    # two atoms: m = (r dV/dr)^2 for each term, with dV/dr from central differences of the energy
    for coulomb, beta, eps_rf in ((synth.COULOMB_RF, 0.0, math.inf), (synth.COULOMB_EWALD, 3.123413274340875, 1.0)):
        r, h = 0.37, 1e-6
        kw = dict(q=(0.7, -0.4), rc=1.0, coulomb=coulomb, beta=beta, eps_rf=eps_rf)
        s = two_atoms(r, **kw)
        m_lj, m_c = oracle.energy_moments(s)
        op, om = oracle.brute(two_atoms(r + h, **kw)), oracle.brute(two_atoms(r - h, **kw))
        d_lj = r * (op["E_lj"] - om["E_lj"]) / (2 * h)
        d_c = r * (op["E_c"] - om["E_c"]) / (2 * h)
        assert m_lj == pytest.approx(d_lj ** 2, rel=1e-6)
        assert m_c == pytest.approx(d_c ** 2, rel=1e-6)


def _three_atoms(coulomb, beta):
    # three atoms on a line: pair energies of both signs (LJ attractive and repulsive
    # pairs, Coulomb like and unlike charges)
    c6, c12 = synth.lj_c6_c12(0.34, 0.8)
    return make_sys([[1.0, 1.0, 1.0], [1.33, 1.0, 1.0], [1.88, 1.0, 1.0]], (0.7, 0.4, -0.5), [0, 0, 0],
                    [[c6]], [[c12]], [5.0, 5.0, 5.0], coulomb=coulomb, rc=1.0, beta=beta, eps_rf=1.0)


def _pair_energies(s):
    """Energies of each pair alone (two-atom sub-systems evaluated by brute force)."""
    out = []
    for i, j in ((0, 1), (0, 2), (1, 2)):
        sub = dataclasses.replace(s, x=s.x[[i, j]], q=s.q[[i, j]], types=s.types[[i, j]],
                                  excl_off=np.zeros(3, np.int32), excl_idx=np.zeros(0, np.int32))
        o = oracle.brute(sub)
        out.append((float(np.linalg.norm(s.x[i] - s.x[j])), o["E_lj"], o["E_c"]))
    return out


@pytest.mark.parametrize("coulomb,beta", [(synth.COULOMB_RF, 0.0), (synth.COULOMB_EWALD, 3.123413274340875)])
def test_energy_moments_absolute_sums(coulomb, beta):
    # sum |V| over pairs = sum of the absolute two-atom energies (the pair terms differ in sign,
    # so this is not |E|)
    s = _three_atoms(coulomb, beta)
    pe = _pair_energies(s)
    _, _, a_lj, a_c = oracle.energy_moments(s, with_abs=True)
    assert a_lj == pytest.approx(sum(abs(v) for _, v, _ in pe), rel=1e-12)
    assert a_c == pytest.approx(sum(abs(v) for _, _, v in pe), rel=1e-12)
    assert a_lj > abs(sum(v for _, v, _ in pe)) * 1.01
    assert a_c > abs(sum(v for _, _, v in pe)) * 1.01


@pytest.mark.parametrize("coulomb,beta", [(synth.COULOMB_RF, 0.0), (synth.COULOMB_EWALD, 3.123413274340875)])
def test_energy_hist_bins_the_pair_terms(coulomb, beta):
    # each pair lands in bin floor(r / rc * nbins) with its own energy, square and charge product
    s = _three_atoms(coulomb, beta)
    nb = 40
    h = oracle.energy_hist(s, nb)
    want = np.zeros((nb, 6))
    for (r, vlj, vc), (i, j) in zip(_pair_energies(s), ((0, 1), (0, 2), (1, 2))):
        k = int(r / s.rc * nb)
        want[k] += [1.0, s.q[i] * s.q[j], vlj, vlj * vlj, vc, vc * vc]
    assert np.allclose(h, want, rtol=1e-12, atol=0.0)


def test_energy_hist_adds_up_to_the_cell_list():
    s = random_system(n=300, L=3.2, seed=17, n_types=3)
    h = oracle.energy_hist(s, 64)
    c = oracle.celllist(s)
    assert int(h[:, 0].sum()) == c["npairs"]
    assert h[:, 2].sum() == pytest.approx(c["E_lj"], rel=1e-12)
    assert h[:, 4].sum() == pytest.approx(c["E_c"], rel=1e-12)
    qq = sum(s.q[i] * s.q[j] for i, j, *_ in oracle.pairs_within(s, s.rc))
    assert h[:, 1].sum() == pytest.approx(qq, rel=1e-12)


def test_force_magnitude_sums():
    # two atoms: each atom's sum of pair-force magnitudes is its force's magnitude; three
    # atoms on a line: the sum of the two-atom force magnitudes, which exceeds the net force
    s2 = two_atoms(0.37, q=(0.7, -0.4), rc=1.0)
    o = oracle.brute(s2)
    assert np.allclose(o["Fabs"], np.linalg.norm(o["F"], axis=1), rtol=1e-12)
    s = _three_atoms(synth.COULOMB_EWALD, 3.123413274340875)
    o = oracle.brute(s)
    want = np.zeros(3)
    for i, j in ((0, 1), (0, 2), (1, 2)):
        sub = dataclasses.replace(s, x=s.x[[i, j]], q=s.q[[i, j]], types=s.types[[i, j]],
                                  excl_off=np.zeros(3, np.int32), excl_idx=np.zeros(0, np.int32))
        fij = np.linalg.norm(oracle.brute(sub)["F"][0])
        want[i] += fij
        want[j] += fij
    assert np.allclose(o["Fabs"], want, rtol=1e-12)
    assert np.all(o["Fabs"] >= np.linalg.norm(o["F"], axis=1))
    # the cell list, its subset path and the image-pair evaluator agree with brute force
    r = random_system(n=300, L=3.2, seed=19, n_types=3)
    b = oracle.brute(r)
    assert np.allclose(oracle.celllist(r)["Fabs"], b["Fabs"], rtol=1e-12)
    sub = np.array([3, 50, 299])
    assert np.allclose(oracle.celllist(r, subset=sub)["Fabs"], b["Fabs"][sub], rtol=1e-12)
    assert np.allclose(oracle.listset(r, oracle.pairs_within(r, r.rc))["Fabs"], b["Fabs"], rtol=1e-12)
