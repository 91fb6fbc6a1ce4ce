"""Pins of the oracle's scalar-only step with a stored velocity field (the
paper's workflow in section "Results": stationary velocity fields computed
once, read by the advection-diffusion solver)."""
import numpy as np

import oracle
from paper_1307_4703_gb300 import workloads as W


def test_scalar_step_with_the_fluid_velocity_equals_the_coupled_step():
    """Driven by the velocity the fluid has at the start of each step, the
    scalar-only step reproduces the coupled step's scalar populations exactly,
    over several steps with every port kind open and closed."""
    prob, init = W.random_case(17, 24, 16)
    a = oracle.from_problem(prob)
    b = oracle.from_problem(prob)
    a.init_equilibrium(**init)
    b.init_equilibrium(**init)
    for t, mask in enumerate([7, 7, 5, 0, 3, 7]):
        _, ux, uy, _ = a.fields()
        b.scalar_step(mask, ux, uy)
        a.step(mask)
        f_a, g_a = a.populations()
        f_b, g_b = b.populations()
        assert np.array_equal(g_a, g_b), t
        b.set_populations(f_a, g_b)  # the fluid of b follows a


def test_scalar_step_diffusion_coefficient():
    """At rest, variance growth 2 D per step with D = c_s^2 (tau_g - 1/2)."""
    n, tau_g = 80, 0.7
    L = oracle.OracleLattice(np.zeros((n, n), np.uint8), 0.8, tau_g)
    y, x = np.mgrid[0:n, 0:n]
    c0 = (n - 1) / 2
    L.init_equilibrium(1.0, 0.0, 0.0, np.exp(-((x - c0) ** 2 + (y - c0) ** 2) / 32.0))

    def var(C):
        m = C.sum()
        return (C * (x - (C * x).sum() / m) ** 2).sum() / m

    zero = np.zeros((n, n))
    L.scalar_step(0, zero, zero, 40)
    v1 = var(L.fields()[3])
    L.scalar_step(0, zero, zero, 40)
    v2 = var(L.fields()[3])
    D = (tau_g - 0.5) / 3
    assert abs((v2 - v1) / 40 - 2 * D) < 1e-9 * D


def test_scalar_step_advects_with_the_given_field():
    """A uniform stored field u0 moves the centroid by u0 per step exactly
    (from the equilibrium of that field), and the fluid populations stay
    as they are."""
    n, m = 128, 96
    L = oracle.OracleLattice(np.zeros((m, n), np.uint8), 0.8, 0.7, periodic=True)
    y, x = np.mgrid[0:m, 0:n]
    u0 = (0.3, -0.2)  # a field rescaled to a larger scalar time step
    # scalar at the equilibrium of the field that will drive it
    L.init_equilibrium(1.0, u0[0], u0[1], np.exp(-((x - 40.0) ** 2 + (y - 50.0) ** 2) / 18.0))
    f0, _ = L.populations()

    def cen(C):
        return (C * x).sum() / C.sum(), (C * y).sum() / C.sum()

    a = cen(L.fields()[3])
    L.scalar_step(0, np.full((m, n), u0[0]), np.full((m, n), u0[1]), 50)
    b = cen(L.fields()[3])
    assert abs(b[0] - a[0] - 50 * u0[0]) < 1e-9 and abs(b[1] - a[1] - 50 * u0[1]) < 1e-9
    assert np.array_equal(L.populations()[0], f0)  # the fluid populations are not touched
