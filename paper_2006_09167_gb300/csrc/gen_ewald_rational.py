"""Generate ewald_rational.h: rational approximations used by the Ewald pair kernels.

The paper evaluates the real-space Ewald correction in the pair kernel with an
analytical, FMA-based approximation instead of a table (Sec. V.A) but does not
print it.  This script derives our own from the mathematics.  With z = beta*r
and s = z^2 / ZMAX^2 (ZMAX = 4, i.e. beta*rc <= 4):

  H(z) = (erf(z)/z - (2/sqrt(pi)) exp(-z^2)) / z^2       (force correction)
  E(z) = erf(z) / z                                    (energy correction)
  X(z) = exp(z^2) erfc(z)                              (scaled complementary error function)

so that the Ewald pair terms become
  phi_C = f qi qj (1/r^3 - beta^3 H(z)),   V_C = f qi qj (erfc(z)/r - erfc(beta rc)/rc)
with erfc(z) = exp(-z^2) X(z).  The energy uses X rather than 1/r - beta E(z):
far from the origin erfc(z)/r is a small difference of two O(1/r) numbers, and
forming it by subtraction in FP32 would cost most of its digits.

H and E are even, smooth and positive on [0, ZMAX] and are fitted as P(s)/Q(s)
in s = z^2 / ZMAX^2; X is fitted as P(t)/Q(t) in t = z / ZMAX.  Each fit
(Q(0) = 1) minimising the maximum relative error against 40-digit mpmath
values, by iteratively re-weighted linear least squares (Sanathanan-Koerner
linearisation with Lawson-style weight updates) on Chebyshev nodes.

Run:  python gen_ewald_rational.py   (writes ewald_rational.h next to this file)
"""
import os

import mpmath
import numpy as np

ZMAX = 4.0
DEG_H = (6, 5)
DEG_E = (5, 5)
DEG_X = (4, 4)
mpmath.mp.dps = 40


def h_ref(z):
    z = mpmath.mpf(z)
    if z == 0:
        return 4 / (3 * mpmath.sqrt(mpmath.pi))
    return (mpmath.erf(z) / z - 2 / mpmath.sqrt(mpmath.pi) * mpmath.exp(-z * z)) / (z * z)


def e_ref(z):
    z = mpmath.mpf(z)
    if z == 0:
        return 2 / mpmath.sqrt(mpmath.pi)
    return mpmath.erf(z) / z


def x_ref(z):
    z = mpmath.mpf(z)
    return mpmath.erfc(z) * mpmath.exp(z * z)


def fit(fun, m, n, iters=40, npts=3000, squared=True):
    k = np.arange(npts)
    s = 0.5 * (1 - np.cos(np.pi * (k + 0.5) / npts))
    f = np.array([float(fun(ZMAX * (np.sqrt(v) if squared else v))) for v in s])
    w = np.ones_like(s)
    q = np.ones_like(s)
    best = None
    for _ in range(iters):
        A = np.concatenate([np.vander(s, m + 1, increasing=True),
                            -f[:, None] * np.vander(s, n + 1, increasing=True)[:, 1:]], 1)
        wt = w / (np.abs(q) * np.abs(f))
        sol, *_ = np.linalg.lstsq(A * wt[:, None], f * wt, rcond=None)
        p = sol[:m + 1]
        qc = np.concatenate([[1.0], sol[m + 1:]])
        q = np.polyval(qc[::-1], s)
        r = (np.polyval(p[::-1], s) / q - f) / f
        e = np.abs(r).max()
        if best is None or e < best[0]:
            best = (e, p.copy(), qc.copy())
        w = w * np.abs(r) ** 0.5 + 1e-30
        w /= w.max()
    return best


def f32_horner_error(fun, p, qc, squared=True):
    z = np.linspace(0.0, ZMAX, 8001)
    s = ((z * z / ZMAX ** 2) if squared else (z / ZMAX)).astype(np.float32)
    P = np.float32(p[-1])
    for c in p[-2::-1]:
        P = (P * s + np.float32(c)).astype(np.float32)
    Q = np.float32(qc[-1])
    for c in qc[-2::-1]:
        Q = (Q * s + np.float32(c)).astype(np.float32)
    v = (P / Q).astype(np.float64)
    ref = np.array([float(fun(t)) for t in z])
    r = (v - ref) / ref
    return float(np.abs(r).max()), float(r.mean())


def main():
    out = []
    out.append("/* Generated by gen_ewald_rational.py -- do not edit.\n"
               " * Rational approximations, z = beta r, of\n"
               " *   H(z) = (erf(z)/z - 2/sqrt(pi) exp(-z^2)) / z^2 and E(z) = erf(z)/z  (in s = z^2/ZMAX^2)\n"
               " *   X(z) = exp(z^2) erfc(z)                                              (in t = z/ZMAX)\n"
               " * on 0 <= z <= ZMAX (relative errors below are measured against mpmath).\n */")
    out.append("#pragma once")
    out.append(f"#define NB_EW_ZMAX {ZMAX:.1f}f")
    for name, fun, (m, n), sq in (("H", h_ref, DEG_H, True), ("E", e_ref, DEG_E, True),
                                  ("X", x_ref, DEG_X, False)):
        e, p, qc = fit(fun, m, n, squared=sq)
        e32, b32 = f32_horner_error(fun, p, qc, squared=sq)
        out.append(f"/* {name}: degrees ({m},{n}); fp64 max rel err {e:.3g}; "
                   f"fp32 Horner max rel err {e32:.3g}, mean {b32:.3g} */")
        for i, c in enumerate(p):
            out.append(f"#define NB_EW_{name}P{i} {float(np.float32(c))!r}f")
        for i, c in enumerate(qc[1:], start=1):
            out.append(f"#define NB_EW_{name}Q{i} {float(np.float32(c))!r}f")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ewald_rational.h")
    with open(path, "w") as fh:
        fh.write("\n".join(out) + "\n")
    print("\n".join(out))


if __name__ == "__main__":
    main()
