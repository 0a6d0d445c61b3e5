"""Central finite differences of the FP64 oracle's adjoint on the differentiation box.

The adjoint (not in the paper) returns the gradients of
    L = <gF, F> + gE * (E_LJ + E_C)
with respect to positions, charges and the C6 / C12 type-pair tables.  Here it
is checked on the 24,000-atom SPC/E box with six Lennard-Jones types (the
differentiation workload) with the force-matching residual as gF:
gF = 2 (F - F_ref) / (3N), F_ref the forces of the same box with C6 and C12
scaled by 1.05, and gE = 0.5.

The pair set is frozen (every pair inside rc at the unperturbed positions is
summed at the perturbed ones, and no other pair), so no step moves a pair
across the cut-off and no coordinate has to be skipped.  A step changes only
the pairs that contain the perturbed atom (or type pair), so each difference is
evaluated over those pairs alone; for <gF, F> this is exact because the forces
of the other pairs cancel in the difference.

Steps: h = 1e-4 nm for coordinates, 1e-4 relative for charges and table
entries.  Checked: 256 seeded coordinates, 256 seeded charges, every entry of
both T x T tables, and one random direction in all parameters at once.  Bar:
relative RMS error 1e-5.  The loss is linear in each charge and table entry, so
those differences are exact up to rounding; for the coordinates the h^2 term of
the central difference is about 1e-6 of the gradient at h = 1e-4 nm (the
random-direction derivative, which cancels strongly, also uses h/2 to remove it)."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2006_09167_gb300 import synth

H_X = 1e-4   # nm
H_REL = 1e-4  # relative step for q, C6, C12
TOL = 1e-5   # relative RMS


@pytest.fixture(scope="module")
def diff_box():
    s = synth.water_24k_types()
    pairs = oracle.pairs_within(s, s.rc)
    s_ref = dataclasses.replace(s, c6=(s.c6 * np.float32(1.05)).astype(np.float32),
                                c12=(s.c12 * np.float32(1.05)).astype(np.float32))
    F_ref = oracle.celllist(s_ref)["F"]
    F = oracle.celllist(s)["F"]
    gF = 2.0 * (F - F_ref) / (3 * s.n)
    gE = 0.5
    g = oracle.vjp(s, gF, gE)
    # pairs of each atom (CSR over both ends)
    ends = np.concatenate([pairs[:, 0], pairs[:, 1]])
    rows = np.concatenate([np.arange(len(pairs)), np.arange(len(pairs))])
    order = np.argsort(ends, kind="stable")
    off = np.searchsorted(ends[order], np.arange(s.n + 1))
    by_atom = (rows[order], off)
    return dict(s=s, pairs=pairs, gF=gF, gE=gE, g=g, by_atom=by_atom, x=s.x.astype(np.float64))


def _loss(d, sel, x=None, q=None, c6=None, c12=None):
    """L over the frozen pairs `sel` (rows of the pair set), with optional replacements."""
    s = d["s"]
    s2 = dataclasses.replace(s, q=s.q if q is None else q, c6=s.c6 if c6 is None else c6,
                             c12=s.c12 if c12 is None else c12)
    o = oracle.listset(s2, d["pairs"][sel], x=d["x"] if x is None else x, frozen=True)
    return float((d["gF"] * o["F"]).sum() + d["gE"] * (o["E_lj"] + o["E_c"]))


def _atom_pairs(d, i):
    rows, off = d["by_atom"]
    return rows[off[i]:off[i + 1]]


def _rms_rel(fd, an):
    fd, an = np.asarray(fd), np.asarray(an)
    return float(np.sqrt(((fd - an) ** 2).sum() / (an ** 2).sum()))


def test_fd_positions_24k(diff_box):
    d = diff_box
    rng = np.random.default_rng(401)
    atoms = rng.choice(d["s"].n, 256, replace=False)
    axes = rng.integers(0, 3, 256)
    fd, an = [], []
    for i, k in zip(atoms, axes):
        sel = _atom_pairs(d, i)
        xp, xm = d["x"].copy(), d["x"].copy()
        xp[i, k] += H_X
        xm[i, k] -= H_X
        fd.append((_loss(d, sel, x=xp) - _loss(d, sel, x=xm)) / (2 * H_X))
        an.append(d["g"]["gx"][i, k])
    assert _rms_rel(fd, an) < TOL


def test_fd_charges_24k(diff_box):
    d = diff_box
    s = d["s"]
    rng = np.random.default_rng(402)
    fd, an = [], []
    for i in rng.choice(s.n, 256, replace=False):
        h = H_REL * abs(float(s.q[i]))
        qp, qm = s.q.astype(np.float64), s.q.astype(np.float64)
        qp[i] += h
        qm[i] -= h
        sel = _atom_pairs(d, i)
        fd.append((_loss(d, sel, q=qp) - _loss(d, sel, q=qm)) / (2 * h))
        an.append(d["g"]["gq"][i])
    assert _rms_rel(fd, an) < TOL


def test_fd_type_pair_tables_24k(diff_box):
    """Every entry of both tables; a single off-diagonal slot carries half of its type
    pair's derivative (the pair parameter is (C[a][b] + C[b][a]) / 2)."""
    d = diff_box
    s = d["s"]
    T = s.n_types
    ti, tj = s.types[d["pairs"][:, 0]], s.types[d["pairs"][:, 1]]
    for name in ("c6", "c12"):
        tab = getattr(s, name).astype(np.float64)
        scale = np.abs(tab).max()
        fd, an = [], []
        for a in range(T):
            for b in range(T):
                sel = np.nonzero(((ti == a) & (tj == b)) | ((ti == b) & (tj == a)))[0]
                h = H_REL * (abs(tab[a, b]) if tab[a, b] != 0 else scale)
                tp, tm = tab.copy(), tab.copy()
                tp[a, b] += h
                tm[a, b] -= h
                fd.append((_loss(d, sel, **{name: tp}) - _loss(d, sel, **{name: tm})) / (2 * h))
                an.append(d["g"]["g" + name][a, b])
        assert _rms_rel(fd, an) < TOL, name


def test_fd_random_direction_24k(diff_box):
    """One random direction in positions, charges and both tables at once, over all pairs."""
    d = diff_box
    s = d["s"]
    rng = np.random.default_rng(403)
    ux = rng.normal(size=d["x"].shape)
    uq = rng.normal(size=s.n) * np.abs(s.q.astype(np.float64))
    u6 = rng.normal(size=s.c6.shape) * np.abs(s.c6.astype(np.float64))
    u12 = rng.normal(size=s.c12.shape) * np.abs(s.c12.astype(np.float64))
    g = d["g"]
    every = np.arange(len(d["pairs"]))

    def at(t):
        return _loss(d, every, x=d["x"] + t * H_X * ux, q=s.q + t * H_REL * uq, c6=s.c6 + t * H_REL * u6,
                     c12=s.c12 + t * H_REL * u12)

    # derivative per unit step along (H_X ux, H_REL uq, H_REL u6, H_REL u12).  The directional
    # derivative sums 72,000 position terms of either sign, which cancel far more than the
    # h^2 terms of the central difference do (measured 7e-5 relative at h alone), so the h^2
    # term is removed by Richardson extrapolation from the steps h and h/2
    def cd(t):
        return (at(t) - at(-t)) / (2 * t)
    fd = (4.0 * cd(0.5) - cd(1.0)) / 3.0
    an_scaled = (g["gx"] * H_X * ux).sum() + (g["gq"] * H_REL * uq).sum() + \
        (g["gc6"] * H_REL * u6).sum() + (g["gc12"] * H_REL * u12).sum()
    assert fd == pytest.approx(an_scaled, rel=TOL)
