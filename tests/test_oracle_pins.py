"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the
lattice of Eq. lattice written in its cos/sin form, moment identities of the
equilibria, conservation laws, and closed-form solutions (Poiseuille flow and
its pressure drop, diffusive spreading, exact advection of a centroid, the
linear steady gradient between two held concentrations).  Every one of them
fails for a plausible slip in the oracle (a dropped term, a wrong sign or
direction index, a swapped relaxation time).
"""
import numpy as np
import pytest

import oracle
from oracle import EAST, PRESSURE, VELOCITY, WEST
from paper_1307_4703_gb300 import workloads as W


def _single_node_populations(rho, ux, uy, C, w0=1.0 / 3.0):
    L = oracle.OracleLattice(np.zeros((1, 1), np.uint8), 0.8, 0.8, w0=w0)
    L.init_equilibrium(rho, ux, uy, C)
    f, g = L.populations()
    return f[0, 0], g[0, 0]


def test_lattice_vectors_follow_eq_lattice():
    """Eq. lattice gives e_i by angle; the oracle's integer table must match,
    and the weights must satisfy the isotropy conditions that define D2Q9
    (sum 1, second moment c_s^2 = 1/3, fourth moments 1/3 and 1/9)."""
    ex, ey, w = oracle.lattice_vectors()
    for i in range(9):
        if i == 0:
            ref = (0.0, 0.0)
        elif i <= 4:
            a = np.pi * (i - 1) / 2
            ref = (np.cos(a), np.sin(a))
        else:
            a = np.pi * (i - 4.5) / 2
            ref = (np.sqrt(2) * np.cos(a), np.sqrt(2) * np.sin(a))
        assert abs(ex[i] - ref[0]) < 1e-12 and abs(ey[i] - ref[1]) < 1e-12, i
    assert abs(w.sum() - 1) < 1e-15
    assert abs((w * ex * ex).sum() - 1 / 3) < 1e-15
    assert abs((w * ey * ey).sum() - 1 / 3) < 1e-15
    assert abs((w * ex * ey).sum()) < 1e-15
    assert abs((w * ex ** 4).sum() - 1 / 3) < 1e-15
    assert abs((w * ex ** 2 * ey ** 2).sum() - 1 / 9) < 1e-15
    # opposite pairs are what bounce-back needs: e_i and -e_i both present
    pairs = {(int(a), int(b)) for a, b in zip(ex, ey)}
    assert all((-a, -b) in pairs for a, b in pairs)


@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (1.07, 0.05, -0.02), (0.93, -0.08, 0.11)])
def test_fluid_equilibrium_moments(rho, ux, uy):
    """f_eq reproduces rho, rho u and the Euler stress rho c_s^2 I + rho u u
    (the moments behind Eq. moments and the viscosity relation)."""
    f, _ = _single_node_populations(rho, ux, uy, 0.0)
    ex, ey, _ = oracle.lattice_vectors()
    assert abs(f.sum() - rho) < 1e-14
    assert abs((f * ex).sum() - rho * ux) < 1e-14
    assert abs((f * ey).sum() - rho * uy) < 1e-14
    assert abs((f * ex * ex).sum() - (rho / 3 + rho * ux * ux)) < 1e-14
    assert abs((f * ey * ey).sum() - (rho / 3 + rho * uy * uy)) < 1e-14
    assert abs((f * ex * ey).sum() - rho * ux * uy) < 1e-14


@pytest.mark.parametrize("w0", [1.0 / 3.0, 0.0])
def test_scalar_equilibrium_moments(w0):
    """g_eq carries C, the advective flux C u and an isotropic second moment
    c_s^2 C I with c_s^2 = (1 - w0)/2; w0 = 0 is the paper's D2Q4 lattice
    (Eq. cdeequilibrium), whose rest population is empty."""
    C, ux, uy = 0.7, 0.04, -0.03
    _, g = _single_node_populations(1.0, ux, uy, C, w0=w0)
    ex, ey, _ = oracle.lattice_vectors()
    ex, ey = ex[:5], ey[:5]
    cs2 = (1 - w0) / 2
    assert abs(g.sum() - C) < 1e-15
    assert abs((g * ex).sum() - C * ux) < 1e-15
    assert abs((g * ey).sum() - C * uy) < 1e-15
    assert abs((g * ex * ex).sum() - cs2 * C) < 1e-15
    assert abs((g * ey * ey).sum() - cs2 * C) < 1e-15
    if w0 == 0.0:
        assert g[0] == 0.0


def test_collision_conserves_mass_momentum_and_scalar():
    """BGK relaxation (Eq. lbequation, right-hand side) leaves rho, rho u and
    C unchanged at every node."""
    prob, init = W.random_case(11, 12, 10)
    L = oracle.from_problem(prob)
    L.init_equilibrium(**init)
    r = W.rng(5)
    f, g = L.populations()
    f = f * (1 + 0.05 * (r.random(f.shape) - 0.5))
    g = g * (1 + 0.05 * (r.random(g.shape) - 0.5))
    L.set_populations(f, g)
    fp, gp = L.post_collision()
    ex, ey, _ = oracle.lattice_vectors()
    fl = ~L.solid
    for a, b in ((f, fp),):
        assert np.abs(a.sum(-1) - b.sum(-1))[fl].max() < 1e-14
        assert np.abs((a * ex).sum(-1) - (b * ex).sum(-1))[fl].max() < 1e-14
        assert np.abs((a * ey).sum(-1) - (b * ey).sum(-1))[fl].max() < 1e-14
    assert np.abs(g.sum(-1) - gp.sum(-1))[fl].max() < 1e-14


def test_closed_box_conserves_mass_and_scalar_exactly():
    """With every wall and valve closed, halfway bounce-back and BGK conserve
    total mass and total scalar exactly (to round-off) for 10^4 steps, also
    across a closed valve's port nodes."""
    prob, init = W.random_case(3, 24, 16)
    L = oracle.from_problem(prob)
    L.init_equilibrium(**init)
    rho, _, _, C = L.fields()
    m0, c0 = rho.sum(), C.sum()
    L.step(0, 10000)
    rho, ux, _, C = L.fields()
    assert abs(rho.sum() - m0) / m0 < 1e-12
    assert abs(C.sum() - c0) / c0 < 1e-12
    assert np.isfinite(ux).all()


def _channel(nx, width, tau, tau_c, u_prof, C_in=0.0, east_kind=PRESSURE):
    solid = np.zeros((width, nx), np.uint8)
    ports = [dict(channel=0, side=WEST, x=0, y0=0, y1=width, kind=VELOCITY),
             dict(channel=0, side=EAST, x=nx - 1, y0=0, y1=width, kind=east_kind, rho=1.0)]
    eu = np.zeros((2, width))
    eu[WEST] = u_prof
    ec = np.zeros((2, width))
    ec[WEST] = C_in
    return oracle.OracleLattice(solid, tau, tau_c, ports=ports, edge_u=eu, edge_C=ec)


def test_poiseuille_profile_and_pressure_drop():
    """Plane Poiseuille flow between halfway bounce-back walls: the developed
    profile is the parabola 4 U s (W - s)/W^2 and the pressure gradient is
    -dp/dx = 8 rho nu U / W^2 with p = rho c_s^2 and nu = c_s^2 (tau - 1/2)
    (the paper's Poiseuille channels and linear pressure drop, section
    "Results"; its check that the imposed pressure difference gives U within
    1%, section "Choice of Parameter Values").  Both to within 1%."""
    width, nx, tau, umax = 16, 64, 0.8, 0.01
    nu = (tau - 0.5) / 3
    L = _channel(nx, width, tau, 0.6, W.parabolic_profile(width, umax))
    L.step(1, 8000)
    rho, ux, uy, _ = L.fields()
    s = np.arange(width) + 0.5
    p = 4 * s * (width - s) / width ** 2
    xm = nx // 2
    A = (ux[:, xm] * p).sum() / (p * p).sum()
    assert np.abs(ux[:, xm] - A * p).max() / A < 0.01
    assert abs(A / umax - 1) < 0.01
    xs = np.arange(8, nx - 8)
    G = -np.polyfit(xs, rho[width // 2, xs], 1)[0] / 3.0
    pred = 8 * rho[:, xm].mean() * nu * A / width ** 2
    assert abs(G / pred - 1) < 0.01
    assert np.abs(uy[:, 8:-8]).max() < 1e-3 * umax


def test_plug_inflow_develops_into_poiseuille():
    """A uniform inflow develops into the parabolic profile whose peak is
    1.5 times the mean velocity, within 1%, downstream of the entrance."""
    width, nx = 16, 128
    L = _channel(nx, width, 0.8, 0.6, np.full(width, 0.01))
    L.step(1, 12000)
    rho, ux, _, _ = L.fields()
    s = np.arange(width) + 0.5
    p = 4 * s * (width - s) / width ** 2
    for xm in (64, 96):
        A = (ux[:, xm] * p).sum() / (p * p).sum()
        assert np.abs(ux[:, xm] - A * p).max() / A < 0.01
        assert abs(A / ux[:, xm].mean() - 1.5) < 0.015


def test_zou_he_port_nodes_hold_prescribed_values():
    """Every open velocity node carries exactly the prescribed u_x, zero u_y
    and C_in; every open pressure node exactly the prescribed rho and zero
    u_y; on all four (side, kind) combinations."""
    prob, init = W.random_case(7, 16, 16)
    L = oracle.from_problem(prob)
    L.init_equilibrium(**init)
    L.step(7, 3)  # channels 0, 1, 2 open
    rho, ux, uy, C = L.fields()
    kinds = set()
    for p in prob["ports"]:
        ys = slice(p["y0"], p["y1"])
        kinds.add((p["side"], p["kind"]))
        assert np.abs(uy[ys, p["x"]]).max() < 1e-15
        if p["kind"] == VELOCITY:
            assert np.abs(ux[ys, p["x"]] - prob["edge_u"][p["side"], ys]).max() < 1e-15
            assert np.abs(C[ys, p["x"]] - prob["edge_C"][p["side"], ys]).max() < 1e-14
        else:
            assert np.abs(rho[ys, p["x"]] - p["rho"]).max() < 1e-14
    assert kinds == {(WEST, VELOCITY), (WEST, PRESSURE), (EAST, VELOCITY), (EAST, PRESSURE)}


@pytest.mark.parametrize("w0", [1.0 / 3.0, 0.0])
def test_diffusion_coefficient(w0):
    """A Gaussian in fluid at rest spreads with variance growing by 2 D per
    step and axis, D = c_s^2 (tau_g - 1/2); for w0 = 0 this is the paper's
    D = (2 tau_g - 1)/4 (Eq. cdeequilibrium).  The growth rate is exact
    once the start-up transient, which decays as (1 - 1/tau_g)^t, is gone."""
    n, tau_g = 96, 0.8
    L = oracle.OracleLattice(np.zeros((n, n), np.uint8), 0.8, tau_g, w0=w0)
    y, x = np.mgrid[0:n, 0:n]
    c0 = (n - 1) / 2
    L.init_equilibrium(1.0, 0.0, 0.0, np.exp(-((x - c0) ** 2 + (y - c0) ** 2) / 32.0))

    def var(C):
        m = C.sum()
        return (C * (x - (C * x).sum() / m) ** 2).sum() / m, (C * (y - (C * y).sum() / m) ** 2).sum() / m

    L.step(0, 60)
    v1 = var(L.fields()[3])
    L.step(0, 40)
    v2 = var(L.fields()[3])
    D = (1 - w0) / 2 * (tau_g - 0.5)
    for a, b in zip(v1, v2):
        assert abs((b - a) / 40 - 2 * D) < 1e-9 * D
    if w0 == 0.0:
        assert abs(D - (2 * tau_g - 1) / 4) < 1e-15


def test_uniform_flow_advects_centroid_exactly():
    """Passive advection by the fluid's own velocity: in a uniform periodic
    flow the centroid of C moves by u per step (the sum of C e_i over the
    lattice is conserved as C u under BGK), and the flow stays uniform."""
    n, m = 128, 96
    L = oracle.OracleLattice(np.zeros((m, n), np.uint8), 0.8, 0.7, periodic=True)
    y, x = np.mgrid[0:m, 0:n]
    u0 = (0.05, -0.03)
    L.init_equilibrium(1.0, u0[0], u0[1], np.exp(-((x - 40.0) ** 2 + (y - 50.0) ** 2) / 18.0))

    def cen(C):
        return (C * x).sum() / C.sum(), (C * y).sum() / C.sum()

    a = cen(L.fields()[3])
    L.step(0, 100)
    rho, ux, uy, C = L.fields()
    b = cen(C)
    assert abs(b[0] - a[0] - 100 * u0[0]) < 1e-10
    assert abs(b[1] - a[1] - 100 * u0[1]) < 1e-10
    assert np.abs(ux - u0[0]).max() < 1e-14 and np.abs(uy - u0[1]).max() < 1e-14


def test_linear_steady_gradient_between_held_concentrations():
    """A flow-free chamber held at C = 1 on one side and C = 0 on the other,
    no-flux walls elsewhere: the steady profile is linear between the two
    held node columns (the linear steady gradient without decay, section
    "Results"), uniform across, and the fluid stays at rest."""
    nx, ny = 32, 6
    solid = np.zeros((ny, nx), np.uint8)
    ports = [dict(channel=0, side=WEST, x=0, y0=0, y1=ny, kind=VELOCITY),
             dict(channel=1, side=EAST, x=nx - 1, y0=0, y1=ny, kind=VELOCITY)]
    ec = np.zeros((2, ny))
    ec[WEST] = 1.0
    L = oracle.OracleLattice(solid, 0.8, 1.0, ports=ports, edge_u=np.zeros((2, ny)), edge_C=ec)
    L.step(3, 20000)
    rho, ux, uy, C = L.fields()
    lin = 1.0 - np.arange(nx) / (nx - 1)
    assert np.abs(C - lin[None, :]).max() < 1e-10
    assert np.abs(ux).max() < 1e-14 and np.abs(rho - 1).max() < 1e-14


def test_do_nothing_outlet_fills_to_inlet_concentration_at_rest():
    """With the fluid at rest, a held inlet concentration and a do-nothing
    outlet (zeroth-order extrapolation in time, section "Boundary
    Conditions"), nothing leaves at steady state: the channel fills to the
    inlet value everywhere."""
    L = _channel(16, 2, 0.8, 0.9, np.zeros(2), C_in=1.0)
    L.step(1, 25000)
    C = L.fields()[3]
    assert np.abs(C - 1.0).max() < 1e-9


def test_do_nothing_outlet_lets_scalar_leave_with_the_flow():
    """With through-flow, the do-nothing outlet lets the advected scalar out:
    the total scalar settles to a steady value and C never exceeds the inlet
    value (a wall in its place would let the scalar pile up without
    bound)."""
    L = _channel(32, 8, 0.8, 0.8, W.parabolic_profile(8, 0.02), C_in=1.0)
    L.step(1, 16000)
    c1 = L.fields()[3].sum()
    L.step(1, 1000)
    C = L.fields()[3]
    assert abs(C.sum() - c1) / c1 < 1e-5
    assert C.max() < 1.0 + 1e-9


def test_outlet_fluxes_balance_inlet_in_steady_flow():
    """Mass and scalar conservation: in a steady channel the outlet
    diagnostics (sum of rho u_x and of C u_x over the open pressure-port
    nodes) carry what the inlet nodes inject, within 0.1% (mass) and 1%
    (scalar, whose inlet also has a small diffusive part); the totals are
    the plain sums of the fields."""
    L = _channel(48, 8, 0.8, 0.8, W.parabolic_profile(8, 0.01), C_in=1.0)
    L.step(1, 20000)
    d = L.diagnostics(1)
    rho, ux, _, C = L.fields()
    assert abs(d[2] / (rho[:, 0] * ux[:, 0]).sum() - 1) < 1e-3
    assert abs(d[3] / (C[:, 0] * ux[:, 0]).sum() - 1) < 1e-2
    assert abs(d[0] - rho.sum()) < 1e-9 and abs(d[1] - C.sum()) < 1e-9
    assert L.diagnostics(0)[2] == 0.0


def test_closed_valve_is_a_wall():
    """Closing both valves of a channel stops the through-flow: the velocity
    decays by more than a thousandfold (what is left is a slowly damped
    acoustic mode of the closed box) and mass is conserved from then on
    (section "Results": closed valves are ordinary walls)."""
    width, nx = 8, 32
    L = _channel(nx, width, 0.8, 0.7, W.parabolic_profile(width, 0.02), C_in=1.0)
    L.step(1, 3000)
    d_open = L.diagnostics(1)
    assert d_open[2] > 0.01 and d_open[3] > 0
    rho, _, _, C = L.fields()
    L.step(0, 1)
    m0 = L.fields()[0].sum()
    c0 = L.fields()[3].sum()
    L.step(0, 4000)
    rho, ux, _, C = L.fields()
    assert abs(rho.sum() - m0) / m0 < 1e-12
    assert abs(C.sum() - c0) / c0 < 1e-12
    assert np.abs(ux).max() < 1e-3 * 0.02
    assert L.diagnostics(0)[2] == 0.0


def test_valve_schedule_reading():
    """The chip of the small workload: top channel open first for one
    period, then the bottom one; the source concentration reaches the
    chamber from the top channel only while the top valves are open."""
    prob = W.config_small()
    assert W.valve_word(prob, 0) == 1 and W.valve_word(prob, 499) == 1
    assert W.valve_word(prob, 500) == 2 and W.valve_word(prob, 1000) == 1
    top = [p for p in prob["ports"] if p["channel"] == 0]
    assert all(p["y0"] == 112 and p["y1"] == 128 for p in top)
    assert np.all(prob["edge_C"][WEST, 112:128] == 1.0)
    assert W.fluid_count(prob) == 14336
