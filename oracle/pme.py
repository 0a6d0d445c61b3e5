"""Smooth particle-mesh Ewald in FP64 (test infrastructure only).

The paper runs the reciprocal part of the Ewald sum as a separate PME task on
its own stream, dominated by two 3-D FFTs (Sec. IV), and cites smooth PME
(Essmann et al., J. Chem. Phys. 103, 8577, 1995) for the method.  This module
takes that method's steps in its order and notation, in plain numpy, so the
CUDA PME can be compared with it step for step; the exact reciprocal sum it
approximates is oracle.ewald_recip (ewald.c), which pins it.

  u_a     = K_a x_a / L_a                         scaled fractional coordinates (wrapped into [0, K_a))
  M_n     cardinal B-spline of order n: M_2(u) = 1 - |u - 1| on [0, 2],
          M_n(u) = u/(n-1) M_{n-1}(u) + (n-u)/(n-1) M_{n-1}(u-1),  M_n' (u) = M_{n-1}(u) - M_{n-1}(u-1)
  Q(k)    = sum_i q_i prod_a M_n(u_ai - k_a)      charge grid (periodic in k)
  B(m)    = prod_a |b_a(m_a)|^2,  b_a(m) = exp(2 pi i (n-1) m/K_a) / sum_{k=0}^{n-2} M_n(k+1) exp(2 pi i m k/K_a)
  C(m)    = exp(-pi^2 |m|^2 / beta^2) / (pi V |m|^2),  m = (m'_1/L_1, m'_2/L_2, m'_3/L_3),  C(0) = 0
  E       = f/2 sum_m B(m) C(m) |F(Q)(m)|^2       F the discrete Fourier transform
  theta*Q = inverse DFT of B C F(Q), scaled by K_1 K_2 K_3 (the convolution of Q with the
            pair kernel on the grid), and F_i = -f q_i sum_k grad_i[prod_a M_n(u_ai - k_a)] (theta*Q)(k)
  W_ab    = -1/2 sum_m e_m (delta_ab - 2 (1 + pi^2 |m|^2/beta^2) m_a m_b / |m|^2),  e_m = f/2 B C |F(Q)|^2

with f = 138.935458/eps_r (W in the convention -1/2 sum r (x) F of the short-range part).
"""
from __future__ import annotations

import math

import numpy as np

F_COUL = 138.935458


def pme_grid(box, spacing: float = 0.12):
    """Smallest even grid sizes >= L/spacing whose only prime factors are 2, 3, 5, 7."""
    def nice(n):
        while True:
            if n % 2 == 0:
                m = n
                for p in (2, 3, 5, 7):
                    while m % p == 0:
                        m //= p
                if m == 1:
                    return n
            n += 1
    return tuple(nice(max(int(math.ceil(float(L) / spacing)), 4)) for L in np.asarray(box, np.float64))


def bspline(w: np.ndarray, order: int):
    """M_n(w + j) and M_n'(w + j) for j = 0..n-1 and fractional parts w in [0, 1): arrays (len(w), n)."""
    w = np.asarray(w, np.float64)
    # order 2: M_2(w) = w, M_2(w + 1) = 1 - w, zero elsewhere
    m = np.zeros((w.size, order))
    m[:, 0] = w
    m[:, 1] = 1.0 - w
    dm = None
    for n in range(3, order + 1):
        if n == order:
            # derivative of M_n at w + j is M_{n-1}(w + j) - M_{n-1}(w + j - 1)
            dm = np.zeros_like(m)
            dm[:, 0] = m[:, 0]
            dm[:, 1:n] = m[:, 1:n] - m[:, 0:n - 1]
        new = np.zeros_like(m)
        for j in range(n):
            u = w + j
            a = m[:, j] if j < n - 1 else 0.0          # M_{n-1}(u)
            b = m[:, j - 1] if j >= 1 else 0.0         # M_{n-1}(u - 1)
            new[:, j] = (u * a + (n - u) * b) / (n - 1)
        m = new
    if dm is None:  # order 2
        dm = np.zeros_like(m)
        dm[:, 0] = 1.0
        dm[:, 1] = -1.0
    return m, dm


def bspline_moduli(K: int, order: int) -> np.ndarray:
    """|b(m)|^2 for m = 0..K-1."""
    vals, _ = bspline(np.zeros(1), order)          # M_n(j), j = 0..n-1
    mk = vals[0, 1:order]                          # M_n(k + 1), k = 0..n-2
    m = np.arange(K)[:, None]
    k = np.arange(order - 1)[None, :]
    den = np.abs((mk[None, :] * np.exp(2j * np.pi * m * k / K)).sum(1)) ** 2
    out = np.empty(K)
    ok = den > 1e-7
    out[ok] = 1.0 / den[ok]
    # odd orders vanish at m = K/2: use the mean of the neighbours there
    for i in np.nonzero(~ok)[0]:
        out[i] = 0.5 * (out[(i - 1) % K] + out[(i + 1) % K])
    return out


def pme(s, x=None, grid=None, order: int = 4, beta=None):
    """Reciprocal-space energy, forces and virial by smooth PME: dict(F, E, W, Q).

    grid: (K1, K2, K3), default pme_grid(box, 0.12); order: B-spline order n."""
    xx = np.asarray(s.x if x is None else x, np.float64)
    q = np.asarray(s.q, np.float64)
    L = np.asarray(s.box, np.float64)
    b = float(s.beta if beta is None else beta)
    K = np.asarray(grid if grid is not None else pme_grid(L), np.int64)
    f = F_COUL / float(s.eps_r)
    n = int(order)
    N = xx.shape[0]
    # scaled fractional coordinates, wrapped into [0, K)
    u = np.mod(xx / L * K, K)
    fl = np.floor(u).astype(np.int64)
    w = u - fl
    theta, dtheta, idx = [], [], []
    for a in range(3):
        t, dt = bspline(w[:, a], n)
        theta.append(t)
        dtheta.append(dt * (K[a] / L[a]))          # d/dx_a of M_n(u_a - k)
        idx.append(np.mod(fl[:, a][:, None] - np.arange(n)[None, :], K[a]))
    # charge grid
    Q = np.zeros(tuple(K))
    wgt = q[:, None, None, None] * theta[0][:, :, None, None] * theta[1][:, None, :, None] * theta[2][:, None, None, :]
    ix = np.broadcast_to(idx[0][:, :, None, None], wgt.shape)
    iy = np.broadcast_to(idx[1][:, None, :, None], wgt.shape)
    iz = np.broadcast_to(idx[2][:, None, None, :], wgt.shape)
    np.add.at(Q, (ix.ravel(), iy.ravel(), iz.ravel()), wgt.ravel())
    # influence function B C on the full grid
    ms = [np.fft.fftfreq(int(K[a]), d=1.0 / int(K[a])) / L[a] for a in range(3)]   # m'_a / L_a
    mx, my, mz = np.meshgrid(ms[0], ms[1], ms[2], indexing="ij")
    m2 = mx * mx + my * my + mz * mz
    V = float(np.prod(L))
    with np.errstate(divide="ignore", invalid="ignore"):
        C = np.exp(-np.pi ** 2 * m2 / b ** 2) / (np.pi * V * m2)
    C[0, 0, 0] = 0.0
    B = bspline_moduli(int(K[0]), n)[:, None, None] * bspline_moduli(int(K[1]), n)[None, :, None] * \
        bspline_moduli(int(K[2]), n)[None, None, :]
    FQ = np.fft.fftn(Q)
    e_m = 0.5 * f * B * C * np.abs(FQ) ** 2
    E = float(e_m.sum())
    W = np.zeros((3, 3))
    with np.errstate(divide="ignore", invalid="ignore"):
        g = 2.0 * (1.0 + np.pi ** 2 * m2 / b ** 2) / m2
    g[0, 0, 0] = 0.0
    mv = (mx, my, mz)
    for a in range(3):
        for c in range(3):
            W[a, c] = -0.5 * float((e_m * ((1.0 if a == c else 0.0) - g * mv[a] * mv[c])).sum())
    conv = np.real(np.fft.ifftn(B * C * FQ)) * float(np.prod(K))
    # forces: gather the convolved grid with the B-spline gradients
    cv = conv[ix, iy, iz]                               # (N, n, n, n)
    t0, t1, t2 = theta
    d0, d1, d2 = dtheta
    Fx = (d0[:, :, None, None] * t1[:, None, :, None] * t2[:, None, None, :] * cv).sum((1, 2, 3))
    Fy = (t0[:, :, None, None] * d1[:, None, :, None] * t2[:, None, None, :] * cv).sum((1, 2, 3))
    Fz = (t0[:, :, None, None] * t1[:, None, :, None] * d2[:, None, None, :] * cv).sum((1, 2, 3))
    # d/dx of M_n(u - k) where u - k = w + j: the derivative arrays are indexed like theta
    F = -f * q[:, None] * np.stack([Fx, Fy, Fz], 1)
    return dict(F=F, E=E, W=W, Q=Q)
