"""Verlet buffer from a drift tolerance (Sec. V.B): the estimate's integral against
a Monte-Carlo simulation of the same model, its limits and monotonicity; on the GPU,
an NVE run with the estimated buffer stays within the tolerance."""
import math

import numpy as np
import pytest

from paper_2006_09167_gb300 import synth, verlet_buffer as vb


def test_missed_energy_integral_against_monte_carlo():
    rng = np.random.default_rng(0)
    rc, b, sigma, d1, d2 = 0.9, 0.03, 0.025, 1.7, 30.0
    # partners at unit density in the shell [rc + b, rc + b + 8 sigma]; radial Gaussian moves
    r_lo, r_hi = rc + b, rc + b + 8 * sigma
    n = 4_000_000
    r0 = np.cbrt(rng.uniform(r_lo ** 3, r_hi ** 3, n))
    r1 = r0 + rng.normal(0.0, sigma, n)
    w = np.clip(rc - r1, 0.0, None)
    shell = 4.0 / 3.0 * math.pi * (r_hi ** 3 - r_lo ** 3)
    mc = shell * np.mean(d1 * w + 0.5 * d2 * w * w)
    est = vb.missed_energy_per_pair_density(sigma, b, rc, d1, d2)
    assert est == pytest.approx(mc, rel=0.03)


def test_drift_estimate_limits_and_monotonicity():
    s = synth.argon_box(1000, rc=0.9, rlist=1.0)
    d = [vb.drift_estimate(s, 120.0, 40, 0.002, rlist=0.9 + bb) for bb in (0.0, 0.01, 0.02, 0.05)]
    assert all(a > b for a, b in zip(d, d[1:]))
    assert vb.drift_estimate(s, 1e-9, 40, 0.002, rlist=0.9) < 1e-12
    # longer list lifetimes need larger buffers
    r10 = vb.estimate_rlist(s, 120.0, 10, 0.002, tolerance=1e-4)
    r80 = vb.estimate_rlist(s, 120.0, 80, 0.002, tolerance=1e-4)
    assert 0.9 <= r10 < r80
    # a loose tolerance needs no buffer
    assert vb.estimate_rlist(s, 120.0, 10, 0.002, tolerance=1.0) == 0.9


@pytest.mark.gpu
def test_nve_drift_within_tolerance_with_estimated_buffer():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_09167_gb300 import api
    tol, T, nst, dt = 0.005, 120.0, 50, 0.002
    s0 = synth.argon_box(1000, seed=7, rc=0.9, rlist=1.0)
    rl = vb.estimate_rlist(s0, T, nst, dt, tolerance=tol)
    s = synth.argon_box(1000, seed=7, rc=0.9, rlist=rl, r_in=rl)  # single list: no rolling prune
    ctx = api.NbContext.from_system(s)
    x = torch.tensor(s.x, device="cuda")
    m = torch.tensor(s.mass, dtype=torch.float32, device="cuda")[:, None]
    v = torch.tensor(synth.maxwell_boltzmann(s, T, seed=5), dtype=torch.float32, device="cuda")
    ctx.build(x, s.box)
    f, e, _ = ctx.forces(x, energy=True)
    etot = []
    for t in range(1000):
        v += 0.5 * dt * f / m
        x += dt * v
        if (t + 1) % nst == 0:
            ctx.build(x, s.box)
        f, e, _ = ctx.forces(x, energy=True)
        v += 0.5 * dt * f / m
        etot.append((0.5 * (m * v * v).sum(dtype=torch.float64) + e.sum()).item())
    drift = np.polyfit(dt * np.arange(1, 1001), np.array(etot), 1)[0] / s.n
    est = vb.drift_estimate(s, T, nst, dt)
    print(f"rlist {rl:.4f}: measured drift {drift:.3e}, estimate {est:.3e} kJ/mol/ps/atom")
    assert abs(drift) <= tol
