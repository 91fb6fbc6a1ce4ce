"""Pins of the oracle's adjoint (reverse-mode derivative of the time step).

The adjoint is checked against what differentiation fixes, not against
itself: central finite differences of the oracle's own forward runs
(Richardson-extrapolated, so that the check is accurate to ~1e-8 even close
to tau_g = 1/2 where plain differences with a large step are off by a few
per cent), and the dot-product identity <a, J v> = <J^T a, v> for single
steps on random lattices with every port kind, which checks the transposed
collision, free flight, bounce-back and port completions at every node.
"""
import numpy as np
import pytest

import oracle
from paper_1307_4703_gb300 import workloads as W


def _objective(prob):
    cx0, cx1, cy0, cy1 = prob["chamber"]
    oy = np.arange(cy0, cy1)
    ox = np.full_like(oy, (cx0 + cx1) // 2)
    target = (oy - cy0) / max(1, cy1 - 1 - cy0)
    return ox, oy, target.astype(float), np.ones(len(oy))


def _J(prob, n, masks, obj, **over):
    p = dict(prob)
    p.update(over)
    L = oracle.from_problem(p)
    for t in range(n):
        L.step(masks[t])
    C = L.fields()[3]
    ox, oy, target, weight = obj
    return float((weight * (C[oy, ox] - target) ** 2).sum())


def _fd(fun, h):
    """Richardson-extrapolated central difference (error O(h^4))."""
    d1 = (fun(h) - fun(-h)) / (2 * h)
    d2 = (fun(h / 2) - fun(-h / 2)) / h
    return (4 * d2 - d1) / 3


@pytest.fixture(scope="module")
def chip_case():
    prob = W.config_large_chip(96, 48)
    prob["period"] = 40
    n = 120
    masks = [W.valve_word(prob, t) for t in range(n)]
    obj = _objective(prob)
    L = oracle.from_problem(prob)
    J, dtau, du, dc = L.adjoint(n, masks, *obj)
    return prob, n, masks, obj, (J, dtau, du, dc)


def test_adjoint_objective_matches_forward(chip_case):
    prob, n, masks, obj, (J, _, _, _) = chip_case
    assert abs(J - _J(prob, n, masks, obj)) < 1e-12 * max(1.0, J)


def test_gradient_wrt_tau_g(chip_case):
    prob, n, masks, obj, (_, dtau, _, _) = chip_case
    fd = _fd(lambda h: _J(prob, n, masks, obj, tau_c=prob["tau_c"] + h), 2e-5)
    assert abs(dtau / fd - 1) < 1e-6


def test_gradient_wrt_inlet_velocity_scale(chip_case):
    prob, n, masks, obj, (_, _, du, _) = chip_case
    fd = _fd(lambda h: _J(prob, n, masks, obj, edge_u=prob["edge_u"] * (1 + h)), 1e-4)
    adj = float((du * prob["edge_u"]).sum())
    assert abs(adj / fd - 1) < 1e-6


@pytest.mark.parametrize("row_from_top", [0, 3, 7])
def test_gradient_wrt_inlet_concentration_per_row(chip_case, row_from_top):
    prob, n, masks, obj, (_, _, _, dc) = chip_case
    y = prob["ny"] - 1 - row_from_top

    def J_at(h):
        ec = prob["edge_C"].copy()
        ec[W.WEST, y] += h
        return _J(prob, n, masks, obj, edge_C=ec)

    fd = _fd(J_at, 1e-4)
    assert abs(dc[W.WEST, y] - fd) < 1e-7 * max(1e-3, abs(fd))
    # rows that are not velocity-port rows carry no derivative
    assert dc[W.WEST, prob["ny"] // 2] == 0.0


@pytest.mark.parametrize("seed", [3, 8])
def test_dot_product_identity_single_step(seed):
    """<a, (F(S + e v) - F(S - e v)) / 2e> = <F'(S)^T a, v> for random a, v."""
    prob, init = W.random_case(seed, 18, 16)
    L = oracle.from_problem(prob)
    L.init_equilibrium(**init)
    r = W.rng(seed + 100)
    f0, g0 = L.populations()
    fl = ~L.solid
    vf = r.standard_normal(f0.shape) * fl[..., None]
    vg = r.standard_normal(g0.shape) * fl[..., None]
    af = r.standard_normal(f0.shape) * fl[..., None]
    ag = r.standard_normal(g0.shape) * fl[..., None]
    mask = 7  # every port open: all completions take part
    L.step(mask)
    f1, g1 = L.populations()

    def F(eps):
        M = oracle.from_problem(prob)
        M.set_populations(f0 + eps * vf, g0 + eps * vg)
        M.step(mask)
        return M.populations()

    eps = 1e-5
    fp, gp = F(eps)
    fm, gm = F(-eps)
    lhs = ((af * (fp - fm)).sum() + (ag * (gp - gm)).sum()) / (2 * eps)
    bf, bg, _ = L.adjoint_step(mask, (f0, g0), (f1, g1), af, ag)
    rhs = (bf * vf).sum() + (bg * vg).sum()
    assert abs(lhs - rhs) < 1e-7 * max(1.0, abs(lhs))


def test_parameter_gradients_on_every_port_kind():
    """Derivatives with respect to u_in and C_in of west and east velocity
    ports, checked against differences on a random lattice."""
    prob, init = W.random_case(5, 20, 16)
    n = 12
    masks = [7] * n
    ox = np.array([10, 11, 12])
    oy = np.array([7, 8, 9])
    obj = (ox, oy, np.array([0.3, 0.5, 0.7]), np.ones(3))

    def J_of(**over):
        p = dict(prob)
        p.update(over)
        L = oracle.from_problem(p)
        L.init_equilibrium(**init)
        for t in range(n):
            L.step(masks[t])
        C = L.fields()[3]
        return float(((C[oy, ox] - obj[2]) ** 2).sum())

    L = oracle.from_problem(prob)
    L.init_equilibrium(**init)
    _, _, du, dc = L.adjoint(n, masks, *obj)
    for p in prob["ports"]:
        if p["kind"] != W.VELOCITY:
            continue
        side, y = p["side"], p["y0"]

        def Ju(h):
            eu = prob["edge_u"].copy()
            eu[side, y] += h
            return J_of(edge_u=eu)

        def Jc(h):
            ec = prob["edge_C"].copy()
            ec[side, y] += h
            return J_of(edge_C=ec)

        fu, fc = _fd(Ju, 1e-4), _fd(Jc, 1e-4)
        assert abs(du[side, y] - fu) < 1e-7 * max(1e-4, abs(fu)), (side, y)
        assert abs(dc[side, y] - fc) < 1e-7 * max(1e-4, abs(fc)), (side, y)
