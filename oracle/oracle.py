"""ctypes binding of the FP64 oracle in oracle.c and ewald.c (test infrastructure only).

Inputs are the caller's arrays promoted exactly to float64 (float32 values are
exactly representable), so the oracle evaluates the same system the CUDA
library is given.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "ewald.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_i = ctypes.POINTER(ctypes.c_int)
_l = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile oracle.c and ewald.c with gcc (-O2, OpenMP, no fast-math) into liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(p) for p in _SRCS):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               "-D_GNU_SOURCE"] + _SRCS + ["-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        common = [ctypes.c_int, _d, _d, _i, ctypes.c_int, _d, _d]
        _lib.or_brute.argtypes = common + [_i, _i, _d, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, _d, _d, _d, _l, _d]
        _lib.or_celllist.argtypes = common + [_i, _i, _d, ctypes.c_int, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_int, _i, _d, _d, _d, _l, _d]
        _lib.or_listset.argtypes = common + [_d, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_int64, _l,
                                             ctypes.c_int, _d, _d, _d, _l, _d]
        _lib.or_pairs_within.argtypes = [ctypes.c_int, _d, _d, _i, _i, ctypes.c_double,
                                         ctypes.c_int64, _l]
        _lib.or_pairs_within.restype = ctypes.c_int64
        _lib.or_vjp.argtypes = common + [_i, _i, _d, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, _d, ctypes.c_double, _d,
                                         _d, _d, _d]
        _lib.or_energy_moments.argtypes = common + [_i, _i, _d, ctypes.c_int, ctypes.c_double,
                                                    ctypes.c_double, ctypes.c_double, ctypes.c_double, _d]
        _lib.or_energy_hist.argtypes = common + [_i, _i, _d, ctypes.c_int, ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                 _d]
        _lib.or_ewald_recip.argtypes = [ctypes.c_int, _d, _d, _d, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, _d, _d, _d]
        _lib.or_ewald_excl.argtypes = [ctypes.c_int, _d, _d, _d, _i, _i, ctypes.c_double, ctypes.c_double,
                                       _d, _d, _d]
        _lib.or_ewald_self.argtypes = [ctypes.c_int, _d, ctypes.c_double, ctypes.c_double]
        _lib.or_ewald_self.restype = ctypes.c_double
        _lib.or_num_threads.restype = ctypes.c_int
        _lib.or_set_num_threads.argtypes = [ctypes.c_int]
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _arrays(sys_or_kw):
    s = sys_or_kw
    x = np.ascontiguousarray(s.x, dtype=np.float64)
    q = np.ascontiguousarray(s.q, dtype=np.float64)
    ty = np.ascontiguousarray(s.types, dtype=np.int32)
    c6 = np.ascontiguousarray(s.c6, dtype=np.float64)
    c12 = np.ascontiguousarray(s.c12, dtype=np.float64)
    off = np.ascontiguousarray(s.excl_off, dtype=np.int32)
    idx = np.ascontiguousarray(s.excl_idx, dtype=np.int32)
    if idx.size == 0:
        idx = np.zeros(1, dtype=np.int32)
    box = np.ascontiguousarray(s.box, dtype=np.float64)
    return x, q, ty, c6, c12, off, idx, box


def _coul(s):
    eps_rf = s.eps_rf if math.isfinite(s.eps_rf) else math.inf
    return int(s.coulomb), float(s.eps_r), float(eps_rf), float(s.beta)


def brute(s, x=None):
    """O(N^2) evaluation. Returns dict(F [N,3], E_lj, E_c, W [3,3], npairs, Fabs [N]);
    Fabs[i] is the sum over atom i's pairs of the magnitude of the pair force."""
    lib = _load()
    xx, q, ty, c6, c12, off, idx, box = _arrays(s)
    if x is not None:
        xx = np.ascontiguousarray(x, dtype=np.float64)
    n = xx.shape[0]
    F = np.zeros((n, 3))
    E = np.zeros(2)
    W = np.zeros(9)
    npairs = ctypes.c_int64(0)
    Fabs = np.zeros(n)
    co, er, erf_, be = _coul(s)
    rc = lib.or_brute(n, _p(xx, _d), _p(q, _d), _p(ty, _i), c6.shape[0], _p(c6, _d), _p(c12, _d),
                      _p(off, _i), _p(idx, _i), _p(box, _d), co, er, erf_, be, float(s.rc),
                      _p(F, _d), _p(E, _d), _p(W, _d), ctypes.byref(npairs), _p(Fabs, _d))
    if rc != 0:
        raise ValueError("oracle: rc must be < L/2")
    return dict(F=F, E_lj=E[0], E_c=E[1], W=W.reshape(3, 3), npairs=npairs.value, Fabs=Fabs)


def celllist(s, x=None, subset=None):
    """Cell-list evaluation (all cores), the keys of brute().  With subset: forces (F, Fabs)
    on those atoms only."""
    lib = _load()
    xx, q, ty, c6, c12, off, idx, box = _arrays(s)
    if x is not None:
        xx = np.ascontiguousarray(x, dtype=np.float64)
    n = xx.shape[0]
    co, er, erf_, be = _coul(s)
    if subset is not None:
        sub = np.ascontiguousarray(subset, dtype=np.int32)
        F = np.zeros((sub.size, 3))
        Fabs = np.zeros(sub.size)
        E = np.zeros(2)
        W = np.zeros(9)
        rc = lib.or_celllist(n, _p(xx, _d), _p(q, _d), _p(ty, _i), c6.shape[0], _p(c6, _d),
                             _p(c12, _d), _p(off, _i), _p(idx, _i), _p(box, _d), co, er, erf_, be,
                             float(s.rc), sub.size, _p(sub, _i), _p(F, _d), _p(E, _d), _p(W, _d),
                             None, _p(Fabs, _d))
        if rc != 0:
            raise ValueError("oracle: subset evaluation needs >= 3 cells per axis and rc < L/2")
        return dict(F=F, Fabs=Fabs)
    F = np.zeros((n, 3))
    Fabs = np.zeros(n)
    E = np.zeros(2)
    W = np.zeros(9)
    npairs = ctypes.c_int64(0)
    rc = lib.or_celllist(n, _p(xx, _d), _p(q, _d), _p(ty, _i), c6.shape[0], _p(c6, _d), _p(c12, _d),
                         _p(off, _i), _p(idx, _i), _p(box, _d), co, er, erf_, be, float(s.rc), 0,
                         None, _p(F, _d), _p(E, _d), _p(W, _d), ctypes.byref(npairs), _p(Fabs, _d))
    if rc != 0:
        raise ValueError("oracle: rc must be < L/2")
    return dict(F=F, E_lj=E[0], E_c=E[1], W=W.reshape(3, 3), npairs=npairs.value, Fabs=Fabs)


def listset(s, pairs, x=None, frozen=False):
    """Sum exactly the given image pairs [(i, j, sx, sy, sz)] that lie inside rc.

    frozen=True sums every given pair whatever its distance (a frozen pair set: the
    shifted potentials continue smoothly beyond rc), so that finite differences of
    the result are those of a fixed list even where a step moves a pair across rc."""
    lib = _load()
    xx, q, ty, c6, c12, off, idx, box = _arrays(s)
    if x is not None:
        xx = np.ascontiguousarray(x, dtype=np.float64)
    pr = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 5)
    if pr.shape[0] == 0:
        pr = np.zeros((1, 5), dtype=np.int64)
        npair = 0
    else:
        npair = pr.shape[0]
    n = xx.shape[0]
    F = np.zeros((n, 3))
    Fabs = np.zeros(n)
    E = np.zeros(2)
    W = np.zeros(9)
    n_in = ctypes.c_int64(0)
    co, er, erf_, be = _coul(s)
    rc = lib.or_listset(n, _p(xx, _d), _p(q, _d), _p(ty, _i), c6.shape[0], _p(c6, _d), _p(c12, _d),
                        _p(box, _d), co, er, erf_, be, float(s.rc), npair, _p(pr, _l), int(bool(frozen)), _p(F, _d),
                        _p(E, _d), _p(W, _d), ctypes.byref(n_in), _p(Fabs, _d))
    if rc != 0:
        raise ValueError("oracle: pair index out of range")
    return dict(F=F, E_lj=E[0], E_c=E[1], W=W.reshape(3, 3), npairs=n_in.value, Fabs=Fabs)


def pairs_within(s, rcut, x=None):
    """Brute-force set of unordered non-excluded pairs within rcut: int64 [P,5]."""
    lib = _load()
    xx, q, ty, c6, c12, off, idx, box = _arrays(s)
    if x is not None:
        xx = np.ascontiguousarray(x, dtype=np.float64)
    n = xx.shape[0]
    cap = 1 << 16
    while True:
        out = np.zeros((cap, 5), dtype=np.int64)
        cnt = lib.or_pairs_within(n, _p(xx, _d), _p(box, _d), _p(off, _i), _p(idx, _i),
                                  float(rcut), cap, _p(out, _l))
        if cnt <= cap:
            return out[:cnt]
        cap = int(cnt)


def vjp(s, gF, gE, x=None):
    """Analytic gradients of <gF, F> + gE*E: dict(gx [N,3], gq [N], gc6 [T,T], gc12 [T,T])."""
    lib = _load()
    xx, q, ty, c6, c12, off, idx, box = _arrays(s)
    if x is not None:
        xx = np.ascontiguousarray(x, dtype=np.float64)
    n = xx.shape[0]
    T = c6.shape[0]
    g = np.ascontiguousarray(gF, dtype=np.float64)
    gx = np.zeros((n, 3))
    gq = np.zeros(n)
    gc6 = np.zeros((T, T))
    gc12 = np.zeros((T, T))
    co, er, erf_, be = _coul(s)
    rc = lib.or_vjp(n, _p(xx, _d), _p(q, _d), _p(ty, _i), T, _p(c6, _d), _p(c12, _d), _p(off, _i),
                    _p(idx, _i), _p(box, _d), co, er, erf_, be, float(s.rc), _p(g, _d), float(gE),
                    _p(gx, _d), _p(gq, _d), _p(gc6, _d), _p(gc12, _d))
    if rc != 0:
        raise ValueError("oracle: rc must be < L/2")
    return dict(gx=gx, gq=gq, gc6=gc6, gc12=gc12)


def energy_moments(s, x=None, with_abs=False):
    """(m_lj, m_c): sums over pairs inside rc of (r dV/dr)^2 for the LJ and Coulomb terms;
    with_abs also returns (sum |V_LJ|, sum |V_C|)."""
    lib = _load()
    xx, q, ty, c6, c12, off, idx, box = _arrays(s)
    if x is not None:
        xx = np.ascontiguousarray(x, dtype=np.float64)
    m = np.zeros(4)
    co, er, erf_, be = _coul(s)
    rc = lib.or_energy_moments(xx.shape[0], _p(xx, _d), _p(q, _d), _p(ty, _i), c6.shape[0], _p(c6, _d),
                               _p(c12, _d), _p(off, _i), _p(idx, _i), _p(box, _d), co, er, erf_, be,
                               float(s.rc), _p(m, _d))
    if rc != 0:
        raise ValueError("oracle: rc must be < L/2")
    if with_abs:
        return float(m[0]), float(m[1]), float(m[2]), float(m[3])
    return float(m[0]), float(m[1])


def energy_hist(s, nbins, x=None):
    """Radial histogram of the pair terms inside rc (nbins equal bins of r on [0, rc)):
    float64 [nbins, 6] with columns (pairs, sum qi qj, sum V_LJ, sum V_LJ^2, sum V_C, sum V_C^2)."""
    lib = _load()
    xx, q, ty, c6, c12, off, idx, box = _arrays(s)
    if x is not None:
        xx = np.ascontiguousarray(x, dtype=np.float64)
    h = np.zeros((int(nbins), 6))
    co, er, erf_, be = _coul(s)
    rc = lib.or_energy_hist(xx.shape[0], _p(xx, _d), _p(q, _d), _p(ty, _i), c6.shape[0], _p(c6, _d), _p(c12, _d),
                            _p(off, _i), _p(idx, _i), _p(box, _d), co, er, erf_, be, float(s.rc), int(nbins),
                            _p(h, _d))
    if rc != 0:
        raise ValueError("oracle: rc must be < L/2 and nbins >= 1")
    return h


def num_threads() -> int:
    return int(_load().or_num_threads())


def set_num_threads(t: int) -> None:
    _load().or_set_num_threads(int(t))


def ewald_kmax(box, beta: float, tol: float = 1e-12):
    """Per-axis k-vector range beyond which the terms exp(-k^2/(4 beta^2)) are below tol."""
    kcut = 2.0 * beta * math.sqrt(-math.log(tol))
    return tuple(int(math.ceil(kcut * L / (2.0 * math.pi))) for L in np.asarray(box, np.float64))


def ewald_recip(s, x=None, kmax=None, beta=None):
    """Direct reciprocal-space Ewald sum (the plain definition PME approximates):
    dict(F, E, W).  kmax per axis defaults to ewald_kmax(box, beta)."""
    lib = _load()
    xx = np.ascontiguousarray(s.x if x is None else x, dtype=np.float64)
    q = np.ascontiguousarray(s.q, dtype=np.float64)
    box = np.ascontiguousarray(s.box, dtype=np.float64)
    b = float(s.beta if beta is None else beta)
    if kmax is None:
        kmax = ewald_kmax(s.box, b)
    F = np.zeros((s.n, 3))
    E = np.zeros(1)
    W = np.zeros(9)
    rc = lib.or_ewald_recip(s.n, _p(xx, _d), _p(q, _d), _p(box, _d), b, float(s.eps_r),
                            int(kmax[0]), int(kmax[1]), int(kmax[2]), _p(F, _d), _p(E, _d), _p(W, _d))
    if rc != 0:
        raise RuntimeError(f"or_ewald_recip failed ({rc})")
    return dict(F=F, E=float(E[0]), W=W.reshape(3, 3))


def ewald_excl(s, x=None, beta=None):
    """Exclusion correction -f qi qj erf(beta r)/r over the excluded pairs: dict(F, E, W)."""
    lib = _load()
    xx, q, _, _, _, off, idx, box = _arrays(s)
    if x is not None:
        xx = np.ascontiguousarray(x, dtype=np.float64)
    F = np.zeros((s.n, 3))
    E = np.zeros(1)
    W = np.zeros(9)
    rc = lib.or_ewald_excl(s.n, _p(xx, _d), _p(q, _d), _p(box, _d), _p(off, _i), _p(idx, _i),
                           float(s.beta if beta is None else beta), float(s.eps_r), _p(F, _d), _p(E, _d), _p(W, _d))
    if rc != 0:
        raise RuntimeError(f"or_ewald_excl failed ({rc})")
    return dict(F=F, E=float(E[0]), W=W.reshape(3, 3))


def ewald_self(s, beta=None):
    """Self energy -f beta/sqrt(pi) sum q^2."""
    q = np.ascontiguousarray(s.q, dtype=np.float64)
    return float(_load().or_ewald_self(s.n, _p(q, _d), float(s.beta if beta is None else beta), float(s.eps_r)))
