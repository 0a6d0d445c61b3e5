"""Shared helpers for the test suite (error norms, pair-set canonicalisation)."""
import itertools

import numpy as np

# parity bars (FP32 pair arithmetic against the FP64 oracle)
TOL_F = 1e-5      # RMS relative force error
TOL_F_ATOM = 1e-4  # largest per-atom force error, relative to the atom's scale (max_atom_err)
TOL_E = 1e-6      # relative energy error (each of E_LJ, E_C)
TOL_W = 1e-5      # relative Frobenius virial error
TOL_NET = 1e-6    # |sum F| / sum |F_i|
EPS32 = 2.0 ** -24  # FP32 unit roundoff


def energy_budget(s, ref, x=None, nbins=100):
    """Relative energy bars (E_LJ, E_C) with the parts they are made of.

    The bar is 1e-6 or, where the system's energy cancels so strongly that FP32 pair
    terms cannot resolve 1e-6 of it, the FP32 floor of the sum:
      - E_LJ (and E_C for reaction field): a relative error of order EPS32 in each FP32
        pair distance moves a term by EPS32 |r dV/dr| with random sign; 4x the root sum
        of squares, EPS32 sqrt(sum (r dV/dr)^2), from the oracle's energy moments.
      - E_C for Ewald: the FP32 rounding model of the kernels' erfc sequence
        (fp32_ewald_model) on the oracle's radial histogram of the exact terms: the
        deterministic error of the fits |sys| plus 5 standard deviations of the
        roundings (5, not 4: the suite checks hundreds of such sums, e.g. 256 replicas,
        and a 4-sigma excursion among them is expected now and then).  floor_c_ideal
        is 4 standard deviations of the same sequence with a correctly rounded FP32
        erfc, the best FP32 pair terms can do.
    Returns dict(tol_lj, tol_c, floor_lj, floor_c, sys_c, sigma_c, floor_c_ideal)."""
    import oracle
    m_lj, m_c = oracle.energy_moments(s, x)
    floor_lj = 4 * EPS32 * np.sqrt(m_lj) / max(abs(ref["E_lj"]), 1e-300)
    out = dict(floor_lj=floor_lj, tol_lj=max(TOL_E, floor_lj))
    if s.coulomb == 1:  # Ewald
        import fp32_ewald_model
        h = oracle.energy_hist(s, nbins, x)
        fl = fp32_ewald_model.coulomb_floor(h, s.beta, s.rc, 138.935458 / s.eps_r, ref["E_c"], float(np.max(s.box)))
        floor_c = abs(fl["sys"]) + 5 * fl["sigma"]
        out.update(floor_c=floor_c, sys_c=fl["sys"], sigma_c=fl["sigma"], floor_c_ideal=4 * fl["sigma_ideal"])
    else:
        floor_c = 4 * EPS32 * np.sqrt(m_c) / max(abs(ref["E_c"]), 1e-300)
        out.update(floor_c=floor_c, sys_c=0.0, sigma_c=floor_c / 4, floor_c_ideal=floor_c)
    out["tol_c"] = max(TOL_E, floor_c)
    return out


def energy_tolerances(s, ref, x=None):
    """Relative energy bars (E_LJ, E_C); see energy_budget."""
    b = energy_budget(s, ref, x)
    return b["tol_lj"], b["tol_c"]


# rows of the per-configuration energy table printed at the end of a test run (conftest)
ENERGY_ROWS = []


def check_energies(name, s, ref, e, x=None):
    """Assert E_LJ and E_C within their bars and record a row of the energy table."""
    b = energy_budget(s, ref, x)
    el, ec = rel(e[0], ref["E_lj"]), rel(e[1], ref["E_c"]) if ref["E_c"] != 0 else 0.0
    ENERGY_ROWS.append(dict(name=name, n=int(s.n), err_lj=el, err_c=ec, **b))
    assert el < b["tol_lj"], f"{name}: E_LJ relative error {el:.3g} (bar {b['tol_lj']:.3g})"
    assert ec < b["tol_c"], f"{name}: E_C relative error {ec:.3g} (bar {b['tol_c']:.3g})"
    return b


def rms_rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def max_atom_err(a, b, fabs=None):
    """Largest per-atom force error |F_i - F_i^ref| relative to the atom's own scale
    max(|F_i^ref|, RMS force) + 0.1 Fabs_i, Fabs_i = sum_j |F_ij| (oracle): one
    mis-handled cluster, face or image shows here even when the RMS norm over many
    atoms hides it.  Relative to the atom's own force because FP32 rounding scales
    with it (an argon atom in a close contact carries a force 50x the RMS and an error
    to match); the Fabs term, at the bar of 1e-4, allows 1e-5 of the summed pair-force
    magnitudes (about 170 FP32 roundings of the terms) for atoms whose pair forces
    cancel to a small net force; the RMS floor covers atoms without that sum."""
    a = np.asarray(a, np.float64).reshape(-1, 3)
    b = np.asarray(b, np.float64).reshape(-1, 3)
    rms = np.sqrt((b * b).sum(1).mean())
    scale = np.maximum(np.sqrt((b * b).sum(1)), max(rms, 1e-300))
    if fabs is not None:
        scale = scale + 0.1 * np.asarray(fabs, np.float64)
    return float((np.sqrt(((a - b) ** 2).sum(1)) / scale).max())


def assert_forces(f, ref, tol_rms=None, tol_atom=None):
    """Force parity: RMS relative error and the largest per-atom error.  ref: the
    reference forces, or an oracle result (its F, and its Fabs for the per-atom scale)."""
    tol_rms = TOL_F if tol_rms is None else tol_rms
    tol_atom = TOL_F_ATOM if tol_atom is None else tol_atom
    fabs = None
    if isinstance(ref, dict):
        ref, fabs = ref["F"], ref.get("Fabs")
    e_rms, e_max = rms_rel(f, ref), max_atom_err(f, ref, fabs)
    assert e_rms < tol_rms, f"force RMS relative error {e_rms:.3g} (bar {tol_rms:g})"
    assert e_max < tol_atom, f"largest per-atom force error {e_max:.3g} relative (bar {tol_atom:g})"
    return e_rms, e_max


def rel(a, b):
    return abs(float(a) - float(b)) / max(abs(float(b)), 1e-300)


def canonical_pairs(p):
    """Rows (i, j, sx, sy, sz) -> set of canonical tuples (i <= j; for i == j, shift > 0)."""
    out = []
    for i, j, sx, sy, sz in np.asarray(p, dtype=np.int64):
        s = (int(sx), int(sy), int(sz))
        if i > j or (i == j and s < (0, 0, 0)):
            i, j, s = j, i, (-s[0], -s[1], -s[2])
        out.append((int(i), int(j)) + s)
    return out


def all_images_within(x, box, rcut, excl_off, excl_idx):
    """Every image pair (i, j, s) with |x_i - x_j + s L| < rcut, s in {-1,0,1}^3 (brute force)."""
    x = np.asarray(x, np.float64)
    box = np.asarray(box, np.float64)
    n = x.shape[0]
    ex = set()
    for i in range(n):
        for j in excl_idx[excl_off[i]:excl_off[i + 1]]:
            ex.add((i, int(j)))
    res = set()
    d0 = x[:, None, :] - x[None, :, :]
    for s in itertools.product((-1, 0, 1), repeat=3):
        d = d0 + np.array(s) * box
        r2 = (d * d).sum(-1)
        ii, jj = np.nonzero(r2 < rcut * rcut)
        for i, j in zip(ii, jj):
            if (i, j) in ex:
                continue
            if i < j or (i == j and s > (0, 0, 0)):
                res.add((int(i), int(j)) + s)
    return res
