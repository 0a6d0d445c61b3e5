"""FP32 rounding model of the Ewald energy term of the pair kernels (test infrastructure).

The energy kernels form, per pair and in FP32 (every FMA rounded once):
    d = x_i - x_j,  r2 = d.d,  1/r (hardware estimate refined by one Newton step),
    r = r2 / r,  z = beta r  and  x = beta^2 r2  (beta, beta^2 as float pairs; the
    kernels form t = z / ZMAX directly from beta / ZMAX, the same value because ZMAX
    is a power of two),
    exp(-x) by Cody-Waite reduction and a degree-7 polynomial,
    X(z) = exp(z^2) erfc(z) as a (6,6) rational with a refined reciprocal,
    erfc(z) = exp(-x) X(z),  v = erfc(z) / r - erfc(beta rc) / rc,  term = qi qj v.
The Coulomb energy of a water box is a sum of millions of such terms that cancel
several thousand-fold, so its error is not bounded by a relative error per term.
It is the sum of two parts:
  - a deterministic part, the smooth error of the approximations (the fits with
    their FP32 coefficients, evaluated without rounding): relative error b(r);
  - a random part, the roundings of every step, zero-mean and independent from
    pair to pair: relative standard deviation s(r).
With the oracle's radial histogram of the exact terms (oracle.energy_hist), an
energy sum over bins k then has error
    sum_k U_k b_k  +-  sqrt(sum_k V2_k s_k^2),
U_k the sum of the unshifted terms qi qj erfc(beta r)/r and V2_k the sum of the
squared terms in bin k.  This module re-states the kernel sequence in numpy to
measure b_k and s_k; it shares no code with the CUDA library (its constants are
read from the generated header as text, like tests/test_ewald_rational.py does).
The same sequence with erfc(z) correctly rounded to FP32 instead of exp(-x) X(z)
gives the floor an ideal FP32 erfc would have (s_ideal)."""
import functools
import os
import re

import numpy as np
from scipy.special import erfc

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2006_09167_gb300", "csrc",
                   "ewald_rational.h")
f32 = np.float32
EPS32 = 2.0 ** -24


@functools.lru_cache(maxsize=1)
def constants():
    return {n: f32(float(v)) for n, v in re.findall(r"#define\s+(NB_\w+)\s+([-+0-9.eE]+)f", open(HDR).read())}


def _fma(a, b, c):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(f32)


def _horner(coefs, t):
    acc = np.full(t.shape, coefs[-1], f32)
    for c in coefs[-2::-1]:
        acc = _fma(acc, t, c)
    return acc


def _split(v):
    hi = f32(v)
    return hi, f32(v - float(hi))


def expm32(x):
    """exp(-x) as the kernels evaluate it, in FP32."""
    c = constants()
    # n = rint of the exact product x log2e (the kernels round x log2e + 1.5 * 2^23 once, in an FMA)
    n = np.rint(np.asarray(x, np.float64) * np.float64(c["NB_EXP_LOG2E"])).astype(f32)
    u = _fma(-n, c["NB_EXP_LN2_HI"], x)
    u = _fma(-n, c["NB_EXP_LN2_LO"], u)
    w = (-u).astype(f32)
    q = _horner([c[f"NB_EXP_C{k}"] for k in range(1, 8)], w)
    p = _fma(q, w, f32(1.0))
    return (p.astype(np.float64) * np.exp2(-n.astype(np.float64))).astype(f32)


def _xcoefs():
    """Numerator and denominator coefficients of X, lowest power first (degrees as in the header)."""
    c = constants()
    m = max(int(k[8:]) for k in c if k.startswith("NB_EW_XP"))
    n = max(int(k[8:]) for k in c if k.startswith("NB_EW_XQ"))
    return [c[f"NB_EW_XP{k}"] for k in range(m + 1)], [f32(1.0)] + [c[f"NB_EW_XQ{k}"] for k in range(1, n + 1)]


def x32(z):
    """X(z) = exp(z^2) erfc(z) as the kernels evaluate it: the reciprocal of the
    denominator is refined to about half an ulp, so it is modelled as rounded."""
    p, q = _xcoefs()
    t = (z * f32(1.0 / constants()["NB_EW_ZMAX"])).astype(f32)
    P = _horner(p, t)
    Q = _horner(q, t)
    return (P * (1.0 / Q.astype(np.float64)).astype(f32)).astype(f32)


def kernel_terms(d32, qq, beta, rc, ideal=False):
    """Per-pair energy terms qi qj v(r) (without the Coulomb constant) in FP32 from FP32
    pair vectors d32 [n,3] and FP32 charge products qq [n]; ideal=True replaces
    exp(-x) X(z) by the correctly rounded FP32 erfc."""
    r2 = _fma(d32[:, 2], d32[:, 2], _fma(d32[:, 1], d32[:, 1], (d32[:, 0] * d32[:, 0]).astype(f32)))
    y = (1.0 / np.sqrt(r2.astype(np.float64))).astype(f32)
    e = _fma(-(r2 * y).astype(f32), y, f32(1.0))
    rinv = _fma((f32(0.5) * y).astype(f32), e, y)
    r = (r2 * rinv).astype(f32)
    bh, bl = _split(beta)
    b2h, b2l = _split(beta * beta)
    z = _fma(bh, r, (bl * r).astype(f32))
    x = _fma(r2, b2h, (r2 * b2l).astype(f32))
    if ideal:
        erfcz = erfc(beta * np.sqrt(r2.astype(np.float64))).astype(f32)
    else:
        erfcz = (expm32(x) * x32(z)).astype(f32)
    v = _fma(erfcz, rinv, -f32(erfc(beta * rc) / rc))
    return (qq * v).astype(f32)


def smooth_error(z):
    """Relative error of exp(-z^2) X(z) from the fits alone (FP32 coefficients, exact
    arithmetic): the deterministic part of the kernels' erfc."""
    c = constants()
    z = np.asarray(z, np.float64)
    xx = z * z
    n = np.rint(xx / np.log(2.0))
    w = -(xx - n * np.log(2.0))
    q = np.full_like(w, float(c["NB_EXP_C7"]))
    for k in range(6, 0, -1):
        q = q * w + float(c[f"NB_EXP_C{k}"])
    ex = (1.0 + q * w) * np.exp2(-n)
    p, qc = _xcoefs()
    t = z / float(c["NB_EW_ZMAX"])
    P = np.polyval([float(v) for v in p[::-1]], t)
    Q = np.polyval([float(v) for v in qc[::-1]], t)
    return ex * (P / Q) / erfc(z) - 1.0


@functools.lru_cache(maxsize=16)
def bin_model(beta, rc, box_len, nbins=100, samples=4000, seed=1):
    """(b, s, s_ideal) per radial bin of [0, rc): smooth relative error of the unshifted
    term, and the standard deviation of the relative error of the whole FP32 sequence
    for the kernels' erfc and for a correctly rounded one.  The roundings of the pair
    vector are included: both atoms are random FP32 positions in a box of edge
    box_len (larger coordinates have larger ulps).  The summation of the terms in FP32
    (short per-lane sums of a few terms per list entry, then compensated) adds about
    one rounding at the scale of a few terms per term: modelled as 2 EPS32 standard
    deviation per term."""
    rng = np.random.default_rng(seed)
    edges = np.linspace(0.0, rc, nbins + 1)
    b = np.zeros(nbins)
    s = np.zeros(nbins)
    s_ideal = np.zeros(nbins)
    acc = 2.0 * EPS32
    for k in range(nbins):
        lo, hi = max(edges[k], 0.05), max(edges[k + 1], 0.06)
        # pair distribution within the bin ~ r^2
        r = np.cbrt(rng.uniform(lo ** 3, hi ** 3, samples))
        zg = beta * np.linspace(lo, hi, 257)
        wg = np.linspace(lo, hi, 257) ** 2
        b[k] = float((smooth_error(zg) * wg).sum() / wg.sum())
        u = rng.normal(size=(samples, 3))
        u /= np.linalg.norm(u, axis=1)[:, None]
        xi = rng.uniform(0.0, box_len, (samples, 3)).astype(f32)
        xj = (xi.astype(np.float64) - u * r[:, None]).astype(f32)
        d32 = (xi - xj).astype(f32)
        rex = np.linalg.norm(xi.astype(np.float64) - xj.astype(np.float64), axis=1)
        qq = rng.uniform(0.1, 1.0, samples).astype(f32)
        exact_unshifted = qq.astype(np.float64) * erfc(beta * rex) / rex
        exact = exact_unshifted - qq.astype(np.float64) * erfc(beta * rc) / rc
        for ideal, out in ((False, s), (True, s_ideal)):
            rel = (kernel_terms(d32, qq, beta, rc, ideal=ideal).astype(np.float64) - exact) / exact_unshifted
            rel -= rel.mean()
            out[k] = float(np.sqrt(rel.var() + acc ** 2))
    return b, s, s_ideal


def coulomb_floor(hist, beta, rc, coul_f, E_c, box_len):
    """Error terms of an FP32 Ewald energy sum relative to |E_C|, from the oracle's radial
    histogram (columns: pairs, sum qq, sum V_LJ, sum V_LJ^2, sum V_C, sum V_C^2; V_C with
    the Coulomb constant) of a box with largest edge box_len: dict(sys, sigma, sigma_ideal)."""
    nb = hist.shape[0]
    b, s, s_ideal = bin_model(float(beta), float(rc), float(box_len), nb)
    unshifted = hist[:, 4] + coul_f * (erfc(beta * rc) / rc) * hist[:, 1]
    sys = float((unshifted * b).sum())
    sig = float(np.sqrt((hist[:, 5] * s ** 2).sum()))
    sig_i = float(np.sqrt((hist[:, 5] * s_ideal ** 2).sum()))
    a = max(abs(E_c), 1e-300)
    return dict(sys=sys / a, sigma=sig / a, sigma_ideal=sig_i / a)
