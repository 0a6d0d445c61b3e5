"""Pair-list buffer from an energy-drift tolerance (paper Sec. V.B).

The paper sets the Verlet buffer from a user tolerance on the energy drift
(default 0.005 kJ/mol/ps per atom), using the particle masses, the temperature
and the pair potentials; it gives the idea but not the formula.  This module
derives an estimate from first principles:

- Over the list lifetime t (the time from the search to the last step that uses
  the list), atoms move ballistically with Maxwell-Boltzmann velocities, so the
  change of a pair's separation along the pair axis is Gaussian with variance
  sigma^2 = k T t^2 (1/m_i + 1/m_j).
- A pair that starts at r0 = rc + u outside the list radius (u >= b = rlist - rc)
  and ends at rc - w inside the cut-off is missed; with the potential shifted to
  zero at rc its missing energy is, to second order, |V'(rc)| w + |V''(rc)| w^2 / 2.
- Summing over partner atoms of each type (number density rho_j, shell 4 pi r0^2)
  and over the atom types gives the expected energy error per atom that a list
  rebuild adds after one lifetime; divided by the lifetime it is the drift.

Swapping the order of integration reduces the double integral to one:
    int_b^inf du int_0^inf dw G(u + w) f(w) = int_b^inf G(s) F(s - b) ds,
with G the Gaussian density and F(x) = a x^2 / 2 + c x^3 / 3 for f(w) = a w + c w^2.
The estimate ignores the extra (implicit) buffer of the cluster setup -- pairs
of listed cluster pairs beyond rlist are computed too (Sec. V.B) -- so it errs on
the safe side.
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np

KB = 0.0083144626  # kJ/mol/K
F_COUL = 138.935458


def _pair_derivatives(system, a: int, b: int, qa: float, qb: float):
    """|V'(rc)| and |V''(rc)| of the shifted pair potential for types a, b and charges qa, qb."""
    rc = system.rc
    c6 = 0.5 * (float(system.c6[a, b]) + float(system.c6[b, a]))
    c12 = 0.5 * (float(system.c12[a, b]) + float(system.c12[b, a]))
    d1 = -12.0 * c12 / rc ** 13 + 6.0 * c6 / rc ** 7
    d2 = 156.0 * c12 / rc ** 14 - 42.0 * c6 / rc ** 8
    qq = F_COUL / system.eps_r * qa * qb
    if system.coulomb == 0:  # reaction field
        eps_rf, eps_r = system.eps_rf, system.eps_r
        krf = 1.0 / (2 * rc ** 3) if (not math.isfinite(eps_rf) or eps_rf <= 0) else \
            (eps_rf - eps_r) / ((2 * eps_rf + eps_r) * rc ** 3)
        d1 += qq * (-1.0 / rc ** 2 + 2 * krf * rc)
        d2 += qq * (2.0 / rc ** 3 + 2 * krf)
    elif system.coulomb == 1:  # Ewald real space
        beta = system.beta
        g = 2 * beta / math.sqrt(math.pi) * math.exp(-(beta * rc) ** 2)
        ec = math.erfc(beta * rc)
        d1 += qq * (-ec / rc ** 2 - g / rc)
        d2 += qq * (2 * ec / rc ** 3 + 2 * g / rc ** 2 + 2 * beta ** 2 * g)
    return abs(d1), abs(d2)


def missed_energy_per_pair_density(sigma: float, buffer: float, rc: float, d1: float, d2: float,
                                   n_grid: int = 4000) -> float:
    """Expected missed energy summed over partners at unit number density:
    int_b^inf 4 pi (rc + u)^2 du int_0^inf dw G(u + w) (d1 w + d2 w^2 / 2), with G the
    N(0, sigma^2) density.  Evaluated as int_b^inf G(s) H(s) ds on a grid, where
    H(s) = int_0^{s-b} 4 pi (rc + s - w)^2 (d1 w + d2 w^2/2) dw (exact polynomial)."""
    if sigma <= 0:
        return 0.0
    smax = buffer + 10.0 * sigma
    s = np.linspace(buffer, smax, n_grid)
    x = s - buffer  # penetration range
    # H(s) with R = rc + s: int_0^x (R - w)^2 (d1 w + c w^2) dw, c = d2/2
    R = rc + s
    c = 0.5 * d2
    # expand (R - w)^2 = R^2 - 2 R w + w^2
    h = (R ** 2 * (d1 * x ** 2 / 2 + c * x ** 3 / 3)
         - 2 * R * (d1 * x ** 3 / 3 + c * x ** 4 / 4)
         + (d1 * x ** 4 / 4 + c * x ** 5 / 5))
    gauss = np.exp(-0.5 * (s / sigma) ** 2) / (math.sqrt(2 * math.pi) * sigma)
    trap = getattr(np, "trapezoid", None) or np.trapz
    return float(4 * math.pi * trap(gauss * h, s))


def drift_estimate(system, temperature: float, nstlist: int, dt: float, rlist: Optional[float] = None) -> float:
    """Estimated energy drift (kJ/mol/ps per atom) for a list rebuilt every nstlist steps."""
    rl = system.rlist if rlist is None else rlist
    buffer = rl - system.rc
    t = max(nstlist - 1, 1) * dt
    n = system.n
    vol = float(np.prod(system.box))
    masses = system.mass if system.mass is not None else np.ones(n)
    # atom classes: (type, charge, mass) with their counts
    keys = np.stack([system.types.astype(np.float64), np.asarray(system.q, np.float64),
                     np.asarray(masses, np.float64)], 1)
    uniq, counts = np.unique(keys, axis=0, return_counts=True)
    total = 0.0
    for (ta, qa, ma), na in zip(uniq, counts):
        for (tb, qb, mb), nb in zip(uniq, counts):
            d1, d2 = _pair_derivatives(system, int(ta), int(tb), float(qa), float(qb))
            if d1 == 0.0 and d2 == 0.0:
                continue
            sigma = math.sqrt(KB * temperature * t * t * (1.0 / ma + 1.0 / mb))
            rho_b = nb / vol
            # per atom of class a, half of each pair's energy is its own
            total += 0.5 * na * rho_b * missed_energy_per_pair_density(sigma, buffer, system.rc, d1, d2)
    return total / n / t


def estimate_rlist(system, temperature: float, nstlist: int, dt: float, tolerance: float = 0.005,
                   max_buffer: float = 0.6) -> float:
    """Smallest rlist >= rc whose estimated drift is at most `tolerance` (kJ/mol/ps/atom)."""
    lo, hi = 0.0, max_buffer
    if drift_estimate(system, temperature, nstlist, dt, rlist=system.rc) <= tolerance:
        return system.rc
    if drift_estimate(system, temperature, nstlist, dt, rlist=system.rc + hi) > tolerance:
        raise ValueError("no buffer up to max_buffer meets the tolerance")
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        if drift_estimate(system, temperature, nstlist, dt, rlist=system.rc + mid) <= tolerance:
            hi = mid
        else:
            lo = mid
    return system.rc + hi
