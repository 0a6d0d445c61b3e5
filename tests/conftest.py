"""Shared pytest configuration: the `gpu` marker and import paths."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


def pytest_terminal_summary(terminalreporter):
    """Per-configuration table of the energy errors against the FP64 oracle, with the bar
    each was held to: 1e-6, or the FP32 floor of the sum (helpers.energy_budget)."""
    try:
        from helpers import ENERGY_ROWS
    except ImportError:
        return
    if not ENERGY_ROWS:
        return
    tr = terminalreporter
    tr.section("energy relative errors against the FP64 oracle (stated bar 1e-6)")
    tr.write_line(f"{'configuration':34s} {'atoms':>9s} {'E_LJ err':>9s} {'bar':>8s} {'E_C err':>9s} {'bar':>8s} "
                  f"{'C sys':>9s} {'C 4 sigma':>9s} {'ideal erfc':>10s}")
    for r in ENERGY_ROWS:
        tr.write_line(f"{r['name'][:34]:34s} {r['n']:9d} {r['err_lj']:9.2e} {r['tol_lj']:8.1e} {r['err_c']:9.2e} "
                      f"{r['tol_c']:8.1e} {r['sys_c']:+9.1e} {4 * r['sigma_c']:9.1e} {r['floor_c_ideal']:10.1e}")
