"""Pins of the scalar solver on the step-profile advection test (Table 3):
the inlet-driven front against the closed-form solution of the 1D
advection-diffusion equation with a held inlet concentration (Ogata & Banks),
and the paper's finding on the four cases of Table 3 (section "Results",
Figure 3): at Pe ~ 4100 the front carries large spurious oscillations that a
tenfold smaller time step does not remove; at Pe ~ 800 they are gone."""
import numpy as np
import pytest
from scipy.special import erfc

import oracle
from paper_1307_4703_gb300 import workloads as W


def _front(u0, D, T, nx=300, ny=3):
    ports = [dict(channel=0, side=0, x=0, y0=0, y1=ny, kind=0),
             dict(channel=0, side=1, x=nx - 1, y0=0, y1=ny, kind=1, rho=1.0)]
    eu, ec = np.zeros((2, ny)), np.zeros((2, ny))
    ec[0] = 1.0
    L = oracle.OracleLattice(np.zeros((ny, nx)), 0.8, 2 * D + 0.5, w0=0.0, ports=ports, edge_u=eu, edge_C=ec)
    L.scalar_step(1, np.full((ny, nx), u0), np.zeros((ny, nx)), T)
    C = L.fields()[3]
    assert np.abs(C - C[1]).max() < 1e-12  # one-dimensional
    x = np.arange(nx)
    s = 2 * np.sqrt(D * T)
    exact = 0.5 * (erfc((x - u0 * T) / s) + np.exp(u0 * x / D) * erfc((x + u0 * T) / s))
    reach = int(2 * u0 * T)
    return np.abs(C[1] - exact)[:reach].max()


def test_inlet_front_matches_the_closed_form():
    """Uniform flow u0 = 0.05, D = 0.05 (paper's D2Q4 lattice, tau_g = 2D +
    1/2), C = 1 held at x = 0: within 2.5e-3 of the closed form after 1000
    steps, and closer after 2000 (the start-up error decays)."""
    e1, e2 = _front(0.05, 0.05, 1000), _front(0.05, 0.05, 2000)
    assert e1 < 2.5e-3 and e2 < e1


@pytest.mark.parametrize("case", ["a", "b", "c", "d"])
def test_table3_cases(case):
    p = W.step_advection(case)
    L = oracle.from_problem(p)
    ux, uy = p["velocity"]
    L.scalar_step(1, ux, uy, p["steps"])
    mid = L.fields()[3][p["ny"] // 2]
    front = int(np.argmin(np.abs(mid - 0.5)))
    assert 180 <= front <= 210  # the front travels U * T = 200 nodes
    overshoot = mid.max() - 1.0
    if case in ("a", "b"):   # Pe ~ 4100: strong oscillations, not cured by the smaller time step
        assert overshoot > 0.1
    else:                    # Pe ~ 800: smooth
        assert overshoot < 0.01
