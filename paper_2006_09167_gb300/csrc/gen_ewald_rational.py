"""Generate ewald_rational.h: the approximations used by the Ewald pair kernels.

The paper evaluates the real-space Ewald correction in the pair kernel with an
analytical, FMA-based approximation instead of a table (Sec. V.A) but does not
print it.  This script derives our own from the mathematics.  With z = beta*r:

  H(z) = (erf(z)/z - (2/sqrt(pi)) exp(-z^2)) / z^2     (force correction, force-only kernels)
  X(z) = exp(z^2) erfc(z)                              (scaled complementary error function)
  exp(w), |w| <= ln2/2                                 (core of exp(-x) after range reduction)

Force-only kernels use phi_C = f qi qj (1/r^3 - beta^3 H(z)), exp-free.  Energy
kernels form e = exp(-z^2) once (Cody-Waite reduction x = n ln2 + u, the
product n * LN2_HI exact, then the polynomial for exp(-u), times 2^-n) and take
both terms from it:
  erfc(z) = e X(z),   phi_C = f qi qj (erfc(z)/r + (2 beta/sqrt(pi)) e) / r^2.
Forming erfc(z)/r as 1/r - beta erf(z)/z instead would subtract two O(1/r)
numbers and lose most FP32 digits near the cut-off.

Accuracy requirement.  The Coulomb energy of water is a sum of terms that cancel
by a factor of about 3000 (sum |V| / |sum V|; 44,000 for the 1.5M-atom polymer
box), so a pointwise relative error that varies smoothly with r -- such as the
equioscillating error of a fit -- is amplified by that factor instead of
averaging out.  The fits are therefore taken to a fit error well below the FP32
rounding level (exp: ~5e-11, degree 7; a degree-6 polynomial with 2e-9 moved
the energy of a 96,000-atom water box by 4e-6 relative, the degree-7 one leaves
it at the FP32 floor).  For X the limit is not the fit but the FP32 rounding
of its coefficients: rounding the coefficients of a minimax (4,4) rational
(fit error 1.1e-8) to FP32 leaves a smooth error of 3.5e-8, which the
polymer box's energy amplified to 1.4e-5.  X is therefore a (6,6) rational
whose coefficients are chosen among FP32 values: starting from the FP64 fit,
the coefficient whose rounding moves the function most is rounded and fixed,
the remaining ones are fitted again, and so on (largest smooth error 2.9e-9;
the polymer box's energy error predicted from it 2e-7).

H is fitted as P(s)/Q(s) in s = z^2/ZMAX^2 and X as P(t)/Q(t) in t = z/ZMAX
(ZMAX = 4, i.e. beta*rc <= 4), each with Q(0) = 1, and exp(w) as
1 + w q(w); all minimise the maximum relative error against 40-digit mpmath
values by iteratively re-weighted linear least squares (Sanathanan-Koerner
linearisation with Lawson-style weight updates) on Chebyshev nodes.

Run:  python gen_ewald_rational.py   (writes ewald_rational.h next to this file)
"""
import os

import mpmath
import numpy as np

ZMAX = 4.0
DEG_H = (6, 5)
DEG_X = (6, 6)
DEG_EXP = 7
mpmath.mp.dps = 40


def h_ref(z):
    z = mpmath.mpf(z)
    if z == 0:
        return 4 / (3 * mpmath.sqrt(mpmath.pi))
    return (mpmath.erf(z) / z - 2 / mpmath.sqrt(mpmath.pi) * mpmath.exp(-z * z)) / (z * z)


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


def fit_fp32_coefficients(fun, m, n, squared=False, iters=60, npts=3000):
    """Minimax relative fit P/Q (Q(0) = 1, P(0) = fun(0) = 1) with FP32 coefficients.

    Rounding all FP64 coefficients to FP32 at once leaves an error far above the
    fit's (each coefficient of a rational moves the function by up to ~1e-8).
    Instead, one coefficient at a time -- the one whose rounding moves the
    function most, at the current fit -- is rounded to FP32 and fixed, and the
    free ones are fitted again (the same re-weighted least squares as fit()),
    so the later coefficients absorb the rounding of the earlier ones."""
    k = np.arange(npts)
    s = 0.5 * (1 - np.cos(np.pi * (k + 0.5) / npts))
    f = np.array([float(fun(ZMAX * (np.sqrt(v) if squared else v))) for v in s])
    ncoef = m + 1 + n
    A = np.concatenate([np.vander(s, m + 1, increasing=True),
                        -f[:, None] * np.vander(s, n + 1, increasing=True)[:, 1:]], 1)

    def solve(frozen):
        free = [c for c in range(ncoef) if c not in frozen]
        rhs0 = f - sum(A[:, c] * v for c, v in frozen.items())
        w = np.ones_like(s)
        q = np.ones_like(s)
        best = None
        for _ in range(iters if free else 1):
            coef = np.zeros(ncoef)
            if free:
                wt = w / (np.abs(q) * np.abs(f))
                sol, *_ = np.linalg.lstsq(A[:, free] * wt[:, None], rhs0 * wt, rcond=None)
                coef[free] = sol
            for c, v in frozen.items():
                coef[c] = v
            q = np.polyval(np.concatenate([[1.0], coef[m + 1:]])[::-1], s)
            r = (np.polyval(coef[:m + 1][::-1], s) / q - f) / f
            e = np.abs(r).max()
            if best is None or e < best[0]:
                best = (e, coef.copy())
            w = w * np.abs(r) ** 0.5 + 1e-30
            w /= w.max()
        return best

    frozen = {0: 1.0}
    e, coef = solve(frozen)
    while len(frozen) < ncoef:
        P = np.polyval(coef[:m + 1][::-1], s)
        Q = np.polyval(np.concatenate([[1.0], coef[m + 1:]])[::-1], s)
        moved = {}
        for c in range(ncoef):
            if c not in frozen:
                basis = s ** c / P if c <= m else s ** (c - m) / Q
                moved[c] = np.abs((float(np.float32(coef[c])) - coef[c]) * basis).max()
        c = max(moved, key=moved.get)
        frozen[c] = float(np.float32(coef[c]))
        e, coef = solve(frozen)
    return e, coef[:m + 1], np.concatenate([[1.0], coef[m + 1:]])


def fit_exp(deg, iters=60, npts=4000):
    """exp(w) = 1 + w q(w) on |w| <= ln2/2, q of degree deg - 1 (minimax relative error)."""
    h = float(mpmath.log(2)) / 2
    k = np.arange(npts)
    w = -h + 2 * h * 0.5 * (1 - np.cos(np.pi * (k + 0.5) / npts))
    f = np.array([float(mpmath.exp(v)) for v in w])
    g = (f - 1) / w
    wt = np.ones_like(w)
    best = None
    for _ in range(iters):
        A = np.vander(w, deg, increasing=True)
        scale = wt * np.abs(w) / f
        sol, *_ = np.linalg.lstsq(A * scale[:, None], g * scale, rcond=None)
        r = (1 + w * np.polyval(sol[::-1], w) - f) / f
        e = np.abs(r).max()
        if best is None or e < best[0]:
            best = (e, sol.copy())
        wt = wt * np.abs(r) ** 0.5 + 1e-30
        wt /= wt.max()
    return best


def cody_waite_constants():
    """LN2_HI: ln2 truncated to 16 significant bits (n * LN2_HI is exact for |n| < 2^8);
    LN2_LO: the FP32 rounding of the remainder; LOG2E: FP32 rounding of 1/ln2."""
    ln2 = mpmath.log(2)
    hi = mpmath.mpf(int(ln2 * 2 ** 16)) / 2 ** 16
    return float(hi), float(np.float32(float(ln2 - hi))), float(np.float32(float(1 / ln2)))


def f32_expm_error(c, hi, lo, l2e):
    """Max and mean relative error of the FP32 exp(-x) sequence on 0 <= x <= 16."""
    f32 = np.float32
    x = np.linspace(0.0, 16.0, 400001).astype(f32)

    def fma(a, b, d):
        return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(d, np.float64)).astype(f32)
    n = np.rint((x * f32(l2e)).astype(f32)).astype(f32)
    u = fma(-n, f32(hi), x)
    u = fma(-n, f32(lo), u)
    w = (-u).astype(f32)
    q = np.full_like(w, f32(c[-1]))
    for cc in c[-2::-1]:
        q = fma(q, w, f32(cc))
    p = fma(q, w, f32(1.0))
    v = p.astype(np.float64) * np.exp2(-n.astype(np.float64))
    ref = np.exp(-x.astype(np.float64))
    r = (v - ref) / ref
    return float(np.abs(r).max()), float(r.mean())


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
               " * Rational approximations, z = beta r, on 0 <= z <= ZMAX of\n"
               " *   H(z) = (erf(z)/z - 2/sqrt(pi) exp(-z^2)) / z^2   (in s = z^2/ZMAX^2)\n"
               " *   X(z) = exp(z^2) erfc(z)                          (in t = z/ZMAX)\n"
               " * and exp(w) = 1 + w (C1 + C2 w + ...) on |w| <= ln2/2 with the Cody-Waite\n"
               " * constants of exp(-x) = 2^-n exp(-(x - n ln2)).\n"
               " * Relative errors below are measured against mpmath / FP64.\n */")
    out.append("#pragma once")
    out.append(f"#define NB_EW_ZMAX {ZMAX:.1f}f")
    for name, fun, (m, n), sq in (("H", h_ref, DEG_H, True), ("X", x_ref, DEG_X, False)):
        if name == "X":
            e, p, qc = fit_fp32_coefficients(fun, m, n, squared=sq)
            kind = "FP32 coefficients, exact evaluation"
        else:
            e, p, qc = fit(fun, m, n, squared=sq)
            kind = "fp64"
        e32, b32 = f32_horner_error(fun, p, qc, squared=sq)
        out.append(f"/* {name}: degrees ({m},{n}); {kind}: max rel err {e:.3g}; "
                   f"fp32 Horner max rel err {e32:.3g}, mean {b32:.3g} */")
        for i, c in enumerate(p):
            out.append(f"#define NB_EW_{name}P{i} {float(np.float32(c))!r}f")
        for i, c in enumerate(qc[1:], start=1):
            out.append(f"#define NB_EW_{name}Q{i} {float(np.float32(c))!r}f")
    e, c = fit_exp(DEG_EXP)
    hi, lo, l2e = cody_waite_constants()
    c32 = [float(np.float32(v)) for v in c]
    e32, b32 = f32_expm_error(c32, hi, lo, l2e)
    out.append(f"/* exp: degree {DEG_EXP}; fp64 max rel err {e:.3g}; "
               f"fp32 exp(-x) on [0,16] max rel err {e32:.3g}, mean {b32:.3g} */")
    out.append(f"#define NB_EXP_LOG2E {l2e!r}f")
    out.append(f"#define NB_EXP_LN2_HI {hi!r}f")
    out.append(f"#define NB_EXP_LN2_LO {lo!r}f")
    for i, v in enumerate(c32, start=1):
        out.append(f"#define NB_EXP_C{i} {v!r}f")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ewald_rational.h")
    with open(path, "w") as fh:
        fh.write("\n".join(out) + "\n")
    print("\n".join(out))


if __name__ == "__main__":
    main()
