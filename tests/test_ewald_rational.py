"""CPU checks of the Ewald approximation constants in csrc/ewald_rational.h.

The force and energy kernels evaluate exp(-z^2), X(z) = exp(z^2) erfc(z) and the
force correction H(z) from these constants in FP32.  Here the same operation
sequences are emulated in FP32 (each FMA rounded once) and compared with the
library functions exp and erfc: pointwise accuracy near the FP32 rounding level,
and a mean error far below it, since the Coulomb energy of water cancels by a
factor of ~3000 and a smooth pointwise bias would not average out."""
import os
import re

import numpy as np
import pytest
from scipy.special import erf, erfc

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2006_09167_gb300", "csrc",
                   "ewald_rational.h")
f32 = np.float32


@pytest.fixture(scope="module")
def consts():
    out = {}
    for name, val in re.findall(r"#define\s+(NB_\w+)\s+([-+0-9.eE]+)f", open(HDR).read()):
        out[name] = f32(float(val))
    return out


def fma(a, b, c):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(f32)


def horner(coefs, t):
    acc = np.full(t.shape, coefs[-1], f32)
    for c in coefs[-2::-1]:
        acc = fma(acc, t, c)
    return acc


def expm(c, x):
    # n = rint of the exact product x log2e (the kernels round x log2e + 1.5 * 2^23 once, in an FMA)
    n = np.rint(np.asarray(x, np.float64) * np.float64(c["NB_EXP_LOG2E"])).astype(f32)
    u = fma(-n, c["NB_EXP_LN2_HI"], x)
    u = fma(-n, c["NB_EXP_LN2_LO"], u)
    w = (-u).astype(f32)
    q = horner([c[f"NB_EXP_C{k}"] for k in range(1, 8)], w)
    p = fma(q, w, f32(1.0))
    return (p.astype(np.float64) * np.exp2(-n.astype(np.float64))).astype(f32)


def xfun(c, z):
    # the kernels refine the reciprocal of the denominator to about half an ulp: modelled
    # here as the rounded quotient
    t = (z * f32(1.0 / c["NB_EW_ZMAX"])).astype(f32)
    m = max(int(k[8:]) for k in c if k.startswith("NB_EW_XP"))
    n = max(int(k[8:]) for k in c if k.startswith("NB_EW_XQ"))
    p = horner([c[f"NB_EW_XP{k}"] for k in range(m + 1)], t)
    q = horner([f32(1.0)] + [c[f"NB_EW_XQ{k}"] for k in range(1, n + 1)], t)
    return (p.astype(np.float64) / q).astype(f32)


def test_cody_waite_split_is_exact_for_the_range(consts):
    hi = float(consts["NB_EXP_LN2_HI"])
    # 16 significant bits: n * LN2_HI is exact in FP32 for every n the kernels reach (z^2 < 80)
    assert hi * 2 ** 16 == int(hi * 2 ** 16)
    for n in range(0, 120):
        assert float(f32(n) * f32(hi)) == n * hi
    assert abs(hi + float(consts["NB_EXP_LN2_LO"]) - np.log(2.0)) < 1e-12


def test_exp_minus_x_accuracy_and_bias(consts):
    x = np.linspace(0.0, 20.0, 400001).astype(f32)
    ref = np.exp(-x.astype(np.float64))
    r = expm(consts, x).astype(np.float64) / ref - 1.0
    assert np.abs(r).max() < 1.5e-7          # ~1.2 ulp
    assert abs(r.mean()) < 2e-9              # no smooth bias at the fit level
    # the bias per interval between powers of two stays small too (the fit error is periodic)
    for a in range(0, 20, 2):
        sel = (x >= a) & (x < a + 2)
        assert abs(r[sel].mean()) < 5e-9
    assert expm(consts, np.zeros(1, f32))[0] == f32(1.0)


def test_erfc_from_exp_and_x(consts):
    z = np.linspace(0.05, 4.0, 200001).astype(f32)
    zd = z.astype(np.float64)
    z2 = (z * z).astype(f32)   # rounded like the kernel's z^2 argument; compare with the same input
    ref = np.exp(-z2.astype(np.float64)) * erfc(zd) * np.exp(zd * zd)
    got = (expm(consts, z2).astype(np.float64) * xfun(consts, z)).astype(f32).astype(np.float64)
    r = got / ref - 1.0
    assert np.abs(r).max() < 5e-7
    assert abs(r.mean()) < 2e-8


def test_force_rational_h(consts):
    zmax = float(consts["NB_EW_ZMAX"])
    z = np.linspace(0.05, 4.0, 20001)
    ref = (erf(z) / z - 2 / np.sqrt(np.pi) * np.exp(-z * z)) / (z * z)
    s = (z * z / zmax ** 2).astype(f32)
    p = horner([consts[f"NB_EW_HP{k}"] for k in range(7)], s)
    q = horner([f32(1.0)] + [consts[f"NB_EW_HQ{k}"] for k in range(1, 6)], s)
    r = (p.astype(np.float64) / q) / ref - 1.0
    assert np.abs(r).max() < 5e-7


def test_ewald_force_forms_agree(consts):
    """The energy kernels' force (erfc/r + 2 beta/sqrt(pi) e^{-z^2}) / r^2 and the
    force-only kernels' 1/r^3 - beta^3 H(z) are the same function."""
    beta, r = 3.123413, np.linspace(0.08, 1.0, 5001)
    z = beta * r
    a = (erfc(z) / r + 2 * beta / np.sqrt(np.pi) * np.exp(-z * z)) / r ** 2
    h = (erf(z) / z - 2 / np.sqrt(np.pi) * np.exp(-z * z)) / (z * z)
    b = 1 / r ** 3 - beta ** 3 * h
    assert np.allclose(a, b, rtol=1e-10, atol=0)
