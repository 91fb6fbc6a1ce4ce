"""Pins of the oracle's paper-specific terms: the decay term -kC of Eq. cde
and the paper's own port boundary of section "Boundary Conditions"
(do-nothing for the unknown populations, then a rescaling of all of them to
the prescribed density or concentration)."""
import numpy as np

import oracle

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def test_decay_in_a_uniform_closed_box_is_geometric():
    """No gradients, no flow: each step removes k C, so C(t) = C0 (1 - k)^t
    exactly, for the coupled step and the scalar-only step alike."""
    k, C0, n = 3e-3, 0.7, 50
    for scalar_only in (False, True):
        L = oracle.OracleLattice(np.zeros((6, 9)), 0.8, 0.65, decay=k)
        L.init_equilibrium(1.0, 0.0, 0.0, C0)
        if scalar_only:
            z = np.zeros((6, 9))
            L.scalar_step(0, z, z, n)
        else:
            L.step(0, n)
        C = L.fields()[3]
        assert np.abs(C / (C0 * (1 - k) ** n) - 1).max() < 1e-13, scalar_only


def _decay_profile_error(length):
    """Steady state between C = 1 (x = 0) and C = 0 (x = length) with decay:
    the closed form C = sinh(lambda (L - x)) / sinh(lambda L), lambda =
    sqrt(k / D), lambda L = 2, D = c_s^2 (tau_g - 1/2) = 1/6."""
    nx, ny, tau_g = length + 1, 3, 1.0
    D = (tau_g - 0.5) / 3
    k = D * (2.0 / length) ** 2
    ports = [dict(channel=0, side=0, x=0, y0=0, y1=ny, kind=0),
             dict(channel=0, side=1, x=nx - 1, y0=0, y1=ny, kind=0)]
    eu, ec = np.zeros((2, ny)), np.zeros((2, ny))
    ec[0] = 1.0
    L = oracle.OracleLattice(np.zeros((ny, nx)), 0.8, tau_g, ports=ports, edge_u=eu, edge_C=ec, decay=k)
    z = np.zeros((ny, nx))
    L.scalar_step(1, z, z, 20 * length * length)
    C = L.fields()[3]
    x = np.arange(nx)
    lam = np.sqrt(k / D)
    exact = np.sinh(lam * (length - x)) / np.sinh(lam * length)
    assert np.abs(C - C[1]).max() < 1e-12  # uniform across the channel
    return np.abs(C[1] - exact).max()


def test_decay_steady_profile_converges_to_the_sinh_closed_form():
    e32, e64 = _decay_profile_error(32), _decay_profile_error(64)
    assert e32 < 1e-4
    assert 3.6 < e32 / e64 < 4.4  # second order in the lattice spacing


def _pressure_channel(tau, n_steps):
    """Straight channel W = 20 rows between halfway walls, the paper's
    rescaling ports at x = 0 (inlet, C_in = 1) and x = 200 (outlet), density
    difference 3 dp with dp = 8 rho nu U L / W^2 for U = 0.00125 (section
    "Choice of Parameter Values")."""
    W_, Lc, U = 20, 200, 0.00125
    nx, ny = Lc + 1, W_
    nu = (tau - 0.5) / 3
    dp = 8 * nu * U * Lc / W_ ** 2
    rho_in, rho_out = 1 + 1.5 * dp, 1 - 1.5 * dp
    ports = [dict(channel=0, side=0, x=0, y0=0, y1=ny, kind=oracle.INLET_RESCALE, rho=rho_in),
             dict(channel=0, side=1, x=nx - 1, y0=0, y1=ny, kind=oracle.PRESSURE_RESCALE, rho=rho_out)]
    eu, ec = np.zeros((2, ny)), np.zeros((2, ny))
    ec[0] = 1.0
    L = oracle.OracleLattice(np.zeros((ny, nx)), tau, 0.6, ports=ports, edge_u=eu, edge_C=ec)
    for _ in range(n_steps // 1000):
        L.step(1, 1000)
        rho, ux, uy, C = L.fields()
        # the ports hold their density and the inlet its concentration exactly
        assert np.abs(rho[:, 0] - rho_in).max() < 1e-14 and np.abs(rho[:, -1] - rho_out).max() < 1e-14
        assert np.abs(C[:, 0] - 1.0).max() < 1e-14
    return L, U, nu, W_


def test_pressure_driven_channel_is_poiseuille():
    """At tau = 1/2 + sqrt(3/16), where halfway bounce-back places the wall
    exactly, the mid-channel profile is the parabola of the local pressure
    gradient to 1e-4, and its maximum is within 1% of the U the end-to-end
    pressure difference was chosen for (the paper's own accuracy)."""
    tau = 0.5 + np.sqrt(3 / 16)
    L, U, nu, W_ = _pressure_channel(tau, 12000)
    rho, ux, uy, C = L.fields()
    grad = (rho[:, 50].mean() - rho[:, 150].mean()) / 100 / 3
    U_local = grad * W_ ** 2 / (8 * rho[:, 100].mean() * nu)
    s = np.arange(W_) + 0.5
    prof = 4 * U_local * s * (W_ - s) / W_ ** 2
    assert np.abs(ux[:, 100] - prof).max() < 1e-4 * U_local
    assert abs(ux[:, 100].max() / U - 1) < 0.01
    assert np.abs(uy[:, 20:180]).max() < 1e-3 * U


def _post_stream_node(f_post, solid, x, y):
    """Populations arriving at (x, y) by free flight, None where the link
    starts outside the fluid (numpy restatement for one node)."""
    ny, nx = solid.shape
    out = []
    for i in range(9):
        xs, ys = x - EX[i], y - EY[i]
        if 0 <= xs < nx and 0 <= ys < ny and not solid[ys, xs]:
            out.append(f_post[ys, xs, i])
        else:
            out.append(None)
    return out


def test_rescaling_port_node_from_first_principles():
    """One step from a flowing state: at an outlet node the unknown
    populations (e_x = -1) are the node's own post-collision values, known
    ones arrive by free flight (walls bounce back), and the nine are scaled to
    the port density, so u is that of the do-nothing populations.  At an
    inlet node that starts without compound, the five scalar populations
    are the equilibrium of C_in at the node's velocity."""
    ny, nx = 6, 12
    ports = [dict(channel=0, side=0, x=0, y0=1, y1=5, kind=oracle.INLET_RESCALE, rho=1.002),
             dict(channel=0, side=1, x=nx - 1, y0=1, y1=5, kind=oracle.PRESSURE_RESCALE, rho=0.999)]
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = solid[-1, :] = 1
    eu, ec = np.zeros((2, ny)), np.zeros((2, ny))
    ec[0, 1:5] = 0.8
    L = oracle.OracleLattice(solid, 0.7, 0.6, ports=ports, edge_u=eu, edge_C=ec)
    yy, xx = np.mgrid[0:ny, 0:nx]
    L.init_equilibrium(1.0 + 0.001 * np.sin(xx), 0.04 + 0.01 * np.cos(yy), 0.005 * np.sin(xx + yy), 0.0)
    fp, gp = L.post_collision()
    L.step(1)
    f, g = L.populations()
    rho, ux, uy, C = L.fields()
    x, y = nx - 1, 3
    arrived = _post_stream_node(fp, solid.astype(bool), x, y)
    col = []
    for i in range(9):
        if EX[i] == -1:                      # unknown at an east port: do-nothing
            col.append(fp[y, x, i])
        elif arrived[i] is None:             # wall link: bounce-back
            col.append(fp[y, x, [0, 3, 4, 1, 2, 7, 8, 5, 6][i]])
        else:
            col.append(arrived[i])
    col = np.array(col)
    expect = col * 0.999 / col.sum()
    assert np.abs(f[y, x] - expect).max() < 1e-15
    assert abs(ux[y, x] - (col * EX).sum() / col.sum()) < 1e-15
    # inlet scalar: equilibrium of C_in = 0.8 at the node's velocity (w0 = 1/3)
    w = np.array([1 / 3] + [1 / 6] * 4)
    ge = 0.8 * w * (1 + 3 * (EX[:5] * ux[2, 0] + EY[:5] * uy[2, 0]))
    assert np.abs(g[2, 0] - ge).max() < 1e-15
    assert abs(C[2, 0] - 0.8) < 1e-15
    # the next step finds compound there: do-nothing for g_1, free flight for
    # the others, then the five scaled to C_in
    fp, gp = L.post_collision()
    L.step(1)
    g2 = L.populations()[1]
    x, y = 0, 2
    col = np.array([gp[y, x, 0], gp[y, x, 1], gp[y - 1, x, 2], gp[y, x + 1, 3], gp[y + 1, x, 4]])
    assert np.abs(g2[y, x] - col * 0.8 / col.sum()).max() < 1e-15
    assert np.abs(L.fields()[3][1:5, 0] - 0.8).max() < 1e-15


def test_equilibrium_wall_keeps_a_fluid_at_rest_exactly():
    solid = np.zeros((20, 30), np.uint8)
    solid[8:12, 10:14] = 1
    L = oracle.OracleLattice(solid, 0.8, 0.7, wall_scheme=1)
    L.step(0, 50)
    f = L.populations()[0]
    assert np.abs(f[solid == 0] - W9).max() < 1e-15


def test_equilibrium_wall_node_from_first_principles():
    """One step from known fields: at a fluid node next to an obstacle, every
    population whose source is solid equals f_eq of rho = 2 rho(x + e_m) -
    rho(x + 2 e_m) and j = j(x + e_m) / 3 (the paper's first-order
    extrapolation and interpolation), the other populations arrive by free
    flight."""
    ny, nx = 12, 16
    solid = np.zeros((ny, nx), np.uint8)
    solid[5:7, 6:9] = 1
    yy, xx = np.mgrid[0:ny, 0:nx]
    rho = 1.0 + 0.01 * np.sin(0.7 * xx + 0.3 * yy)
    ux = 0.03 * np.cos(0.5 * yy)
    uy = 0.02 * np.sin(0.4 * xx)
    L = oracle.OracleLattice(solid, 0.75, 0.6, wall_scheme=1)
    L.init_equilibrium(rho, ux, uy, 0.0)
    fp, _ = L.post_collision()
    L.step(0)
    f = L.populations()[0]

    def feq(i, r, vx, vy):
        eu = EX[i] * vx + EY[i] * vy
        return W9[i] * r * (1 + 3 * eu + 4.5 * eu * eu - 1.5 * (vx * vx + vy * vy))

    checked = 0
    for (x, y) in ((5, 5), (9, 6), (7, 4), (7, 7), (5, 7)):
        assert not solid[y, x]
        for m in range(9):
            xs, ys = x - EX[m], y - EY[m]
            if solid[ys, xs]:
                x1, y1, x2, y2 = x + EX[m], y + EY[m], x + 2 * EX[m], y + 2 * EY[m]
                r = 2 * rho[y1, x1] - rho[y2, x2]
                jx, jy = rho[y1, x1] * ux[y1, x1] / 3, rho[y1, x1] * uy[y1, x1] / 3
                assert abs(f[y, x, m] - feq(m, r, jx / r, jy / r)) < 1e-15, (x, y, m)
                checked += 1
            else:
                assert abs(f[y, x, m] - fp[ys, xs, m]) < 1e-15
    assert checked >= 8


def test_equilibrium_wall_channel_profile():
    """Pressure-driven channel with the paper's walls and ports: the steady
    profile is a symmetric parabola (residual < 1e-3 of its maximum) whose
    zeros lie 0.5 to 1.2 nodes beyond the halfway positions at tau = 0.65
    (the equilibrium wall's slip; the paper tuned its pressure difference to
    reach U within 1%)."""
    tau, W_, Lc, U = 0.65, 20, 200, 0.00125
    nx, ny = Lc + 1, W_
    nu = (tau - 0.5) / 3
    dp = 8 * nu * U * Lc / W_ ** 2
    ports = [dict(channel=0, side=0, x=0, y0=0, y1=ny, kind=oracle.INLET_RESCALE, rho=1 + 1.5 * dp),
             dict(channel=0, side=1, x=nx - 1, y0=0, y1=ny, kind=oracle.PRESSURE_RESCALE, rho=1 - 1.5 * dp)]
    eu, ec = np.zeros((2, ny)), np.zeros((2, ny))
    ec[0] = 1.0
    L = oracle.OracleLattice(np.zeros((ny, nx)), tau, 0.6, ports=ports, edge_u=eu, edge_C=ec, wall_scheme=1)
    L.step(1, 12000)
    u = L.fields()[1][:, 100]
    y = np.arange(ny) + 0.5
    c = np.polyfit(y, u, 2)
    assert np.abs(np.polyval(c, y) - u).max() < 1e-3 * u.max()
    lo, hi = np.sort(np.roots(c).real)
    assert abs((lo + hi) / 2 - W_ / 2) < 1e-6
    assert -1.2 < lo < -0.5 and W_ + 0.5 < hi < W_ + 1.2
