"""Shared helpers for the test suite (error norms, pair-set canonicalisation)."""
import itertools

import numpy as np

# parity bars (FP32 pair arithmetic against the FP64 oracle)
TOL_F = 1e-5      # RMS relative force error
TOL_E = 1e-6      # relative energy error (each of E_LJ, E_C)
TOL_W = 1e-5      # relative Frobenius virial error
TOL_NET = 1e-6    # |sum F| / sum |F_i|
EPS32 = 2.0 ** -24  # FP32 unit roundoff


# relative bias bound of the FP32 complementary error function on the GPU (CUDA erfcf,
# measured against FP64 erfc over 0.05 <= z <= 3.2, weighted by the pair distribution: 4e-9)
ERFC_BIAS = 1e-8


def energy_tolerances(s, ref, x=None):
    """Relative energy bars (E_LJ, E_C): 1e-6, or the FP32 rounding floor of the sum
    where the system's energy cancels so strongly that 1e-6 is below it.

    A pair term computed in FP32 carries a relative error of order EPS32 in r, which
    moves it by EPS32 |r dV/dr| with random sign; summed over all pairs that is
    EPS32 sqrt(sum (r dV/dr)^2).  The Ewald energy also inherits the FP32 erfc's
    pointwise error, which does not average out: it adds up to ERFC_BIAS sum |V_C|.
    The floor is 4x the random part plus the systematic part, relative to |E|."""
    import oracle
    m_lj, m_c, a_lj, a_c = oracle.energy_moments(s, x, with_abs=True)
    f_lj = 4 * EPS32 * np.sqrt(m_lj) / max(abs(ref["E_lj"]), 1e-300)
    sys_c = ERFC_BIAS * a_c if s.coulomb == 1 else 0.0
    f_c = (4 * EPS32 * np.sqrt(m_c) + sys_c) / max(abs(ref["E_c"]), 1e-300)
    return max(TOL_E, f_lj), max(TOL_E, f_c)


def rms_rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


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
