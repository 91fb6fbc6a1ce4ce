"""GPU adjoint (lbm_adjoint) against the FP64 oracle adjoint.

The oracle adjoint is itself pinned by finite differences and dot-product
identities (tests/test_oracle_adjoint.py).  Target: gradients within 1e-3
relative of the FP64 reference (FP32 forward and adjoint populations, FP64
gradient accumulation; observed agreement is ~1e-6).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1307_4703_gb300 import lbm, workloads as W  # noqa: E402

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

GRAD_TOL = 1e-3


def _objective(prob):
    """Chamber concentration profile along y at the chamber's centre column
    against a linear target from 0 (bottom) to 1 (top)."""
    cx0, cx1, cy0, cy1 = prob["chamber"]
    oy = np.arange(cy0, cy1)
    ox = np.full_like(oy, (cx0 + cx1) // 2)
    return ox, oy, ((oy - cy0) / max(1, cy1 - 1 - cy0)).astype(float), np.ones(len(oy))


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(1e-300, np.linalg.norm(np.ravel(b))))


def _check(gpu, ref):
    J, dt, du, dc = gpu
    rJ, rt, ru, rc = ref
    assert abs(J / rJ - 1) < 1e-5
    assert abs(dt - rt) <= GRAD_TOL * max(abs(rt), 1e-12)
    assert _rel(du, ru) < GRAD_TOL
    assert _rel(dc, rc) < GRAD_TOL


@pytest.mark.parametrize("ckpt", [50, 7, 1])
def test_adjoint_matches_oracle_on_small_chip(ckpt):
    prob = W.config_large_chip(96, 48)
    prob["period"] = 40
    n = 120
    masks = [W.valve_word(prob, t) for t in range(n)]
    obj = _objective(prob)
    ref = oracle.from_problem(prob).adjoint(n, masks, *obj)
    chip = lbm.Chip.from_problem(prob)
    chip.set_valve_schedule(prob["period"], prob["states"])
    got = chip.adjoint(n, obj[0], obj[1], obj[2], obj[3], ckpt_every=ckpt)
    _check(got, ref)
    assert chip.step_count() == n
    chip.close()


def test_adjoint_every_port_kind():
    """West and east velocity ports (u_in and C_in derivatives on both sides),
    west and east pressure ports (do-nothing transpose), random obstacles; the
    lattice is small enough that every port reaches the objective in n steps."""
    prob, init = W.random_case(5, 16, 16)
    n = 12
    fy, fx = np.nonzero(prob["solid"] == 0)
    sel = np.arange(0, len(fx), max(1, len(fx) // 5))[:5]
    ox, oy = fx[sel], fy[sel]
    tg = np.linspace(0.2, 0.8, len(sel))
    L = oracle.from_problem(prob)
    L.init_equilibrium(**init)
    ref = L.adjoint(n, [7] * n, ox, oy, tg, np.ones(len(sel)))
    chip = lbm.Chip.from_problem(prob)
    chip.init_equilibrium(**init)
    chip.set_valves(7)
    got = chip.adjoint(n, ox, oy, tg, ckpt_every=5)
    _check(got, ref)
    ru = ref[2]
    assert np.count_nonzero(ru[W.WEST]) > 0 and np.count_nonzero(ru[W.EAST]) > 0
    chip.close()


def test_adjoint_on_the_128x64_copy_of_the_gradient_chip():
    """The gradient workload scaled to 128 x 64 (the size the FP64 reference
    adjoint runs at), with the seeded per-row inlet concentrations: 4000
    steps, valves toggling every 1500 steps, checkpoints every 250 steps."""
    prob = W.config_adjoint_chip(128, 64)
    n = 4000
    masks = [W.valve_word(prob, t) for t in range(n)]
    obj = _objective(prob)
    ref = oracle.from_problem(prob).adjoint(n, masks, *obj)
    chip = lbm.Chip.from_problem(prob)
    chip.set_valve_schedule(prob["period"], prob["states"])
    got = chip.adjoint(n, obj[0], obj[1], obj[2], obj[3], ckpt_every=250)
    _check(got, ref)
    # the derivatives are not degenerate on this workload
    assert abs(ref[1]) > 1e-3 and np.abs(ref[3]).max() > 1e-4
    chip.close()


def test_adjoint_leaves_the_forward_state_and_diagnostics():
    prob = W.config_large_chip(96, 48)
    prob["period"] = 30
    obj = _objective(prob)
    a = lbm.Chip.from_problem(prob)
    b = lbm.Chip.from_problem(prob)
    for c in (a, b):
        c.set_valve_schedule(prob["period"], prob["states"])
    a.adjoint(90, obj[0], obj[1], obj[2], obj[3], ckpt_every=20)
    b.step(90)
    fa, ga = a.populations()
    fb, gb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    assert np.array_equal(a.diagnostics(), b.diagnostics())
    assert a.step_count() == b.step_count() == 90
    # every state kept: the same final state, step count and gradients
    a.adjoint(31, obj[0], obj[1], obj[2], obj[3], ckpt_every=1)
    b.step(31)
    fa, ga = a.populations()
    fb, gb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    assert a.step_count() == b.step_count() == 121
    a.close()
    b.close()


@pytest.mark.parametrize("K", [13, 7, 69, 70, 100])
def test_adjoint_keeping_every_state_equals_checkpointed(K):
    """Checkpoints every K of 70 steps (last segment 5, 7 = K, 1, 70 = the
    whole run, and K > n): the forward sweep keeps the last segment's states
    and the others are recomputed, so every reverse step reads the same
    states as with every state kept: the same J, the gradients up to the
    order of the FP64 gradient atomics, and the same final populations."""
    prob = W.config_large_chip(96, 48)
    prob["period"] = 30
    obj = _objective(prob)
    res = []
    for k in (1, K):
        c = lbm.Chip.from_problem(prob)
        c.set_valve_schedule(prob["period"], prob["states"])
        res.append(c.adjoint(70, obj[0], obj[1], obj[2], obj[3], ckpt_every=k))
        res.append(c.populations())
        assert c.step_count() == 70
        c.close()
    (J1, t1, u1, c1), (f1, g1), (J2, t2, u2, c2), (f2, g2) = res
    assert np.array_equal(f1, f2) and np.array_equal(g1, g2)
    assert J1 == J2
    assert abs(t1 - t2) <= 1e-9 * abs(t2)
    assert np.allclose(u1, u2, rtol=1e-9, atol=0) and np.allclose(c1, c2, rtol=1e-9, atol=0)


@pytest.mark.parametrize("K,multi_step", [(1, 16), (1, 1000), (13, 5), (250, 64)])
def test_adjoint_with_multi_step_launches_equals_single_launches(K, multi_step):
    """Forward sweep, recomputation and reverse sweep in cooperative
    multi-step launches (runs split by valve switches every 30 steps and by
    the run cap) against one launch per step: the same populations, J
    identical and the gradients equal up to the order of their FP64 sums;
    both against the FP64 oracle adjoint."""
    prob = W.config_large_chip(256, 128)
    prob["period"] = 30
    obj = _objective(prob)
    res = []
    for ms in (0, multi_step):
        c = lbm.Chip.from_problem(prob, multi_step=ms)
        c.set_valve_schedule(prob["period"], prob["states"])
        res.append(c.adjoint(97, obj[0], obj[1], obj[2], obj[3], ckpt_every=K))
        res.append(c.populations())
        c.close()
    (J1, t1, u1, c1), (f1, g1), (J2, t2, u2, c2), (f2, g2) = res
    assert np.array_equal(f1, f2) and np.array_equal(g1, g2)
    assert J1 == J2
    assert abs(t1 - t2) <= 1e-6 * abs(t1)
    assert _rel(u2, u1) < 1e-6 and _rel(c2, c1) < 1e-6
    masks = [W.valve_word(prob, t) for t in range(97)]
    _check((J2, t2, u2, c2), oracle.from_problem(prob).adjoint(97, masks, *obj))


def test_adjoint_rejects_bad_objectives():
    prob = W.config_large_chip(96, 48)
    chip = lbm.Chip.from_problem(prob)
    with pytest.raises(lbm.LbmError) as e:
        chip.adjoint(10, [0], [prob["ny"] // 2], [0.0])  # a solid node
    assert e.value.status == lbm.LBM_ERR_ARG
    with pytest.raises(lbm.LbmError):
        chip.adjoint(0, [5], [1], [0.0])
    chip.close()


def test_autograd_function_returns_the_adjoint_gradients():
    """The torch.autograd.Function's backward gives the adjoint's
    derivatives: dJ/dtau_c, dJ/du_scale = sum u_in dJ/du_in, and dJ/dC_in of
    the listed inlet rows; a finite difference in u_scale agrees."""
    from paper_1307_4703_gb300.autograd import chamber_objective

    prob = W.config_large_chip(96, 48)
    prob["period"] = 40
    n = 120
    obj = _objective(prob)
    top = [p for p in prob["ports"] if p["channel"] == 0 and p["side"] == W.WEST][0]
    rows = np.arange(top["y0"], top["y1"])
    tau = torch.tensor(prob["tau_c"], dtype=torch.float64, requires_grad=True)
    us = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    cin = torch.tensor(prob["edge_C"][W.WEST, rows], dtype=torch.float64, requires_grad=True)
    J = chamber_objective(tau, us, cin, prob, rows, obj, n, ckpt_every=40)
    J.backward()
    masks = [W.valve_word(prob, t) for t in range(n)]
    rJ, rt, ru, rc = oracle.from_problem(prob).adjoint(n, masks, *obj)
    assert abs(float(J.detach()) / rJ - 1) < 1e-5
    assert abs(float(tau.grad) / rt - 1) < GRAD_TOL
    assert abs(float(us.grad) / float((ru * prob["edge_u"]).sum()) - 1) < GRAD_TOL
    assert _rel(cin.grad.numpy(), rc[W.WEST, rows]) < GRAD_TOL
    # the scalar's sensitivity to the inlet velocity scale, by differences
    h = 1e-2
    Jp = float(chamber_objective(torch.tensor(prob["tau_c"]), torch.tensor(1 + h), cin.detach(), prob, rows, obj, n))
    Jm = float(chamber_objective(torch.tensor(prob["tau_c"]), torch.tensor(1 - h), cin.detach(), prob, rows, obj, n))
    fd = (Jp - Jm) / (2 * h)
    assert abs(float(us.grad) / fd - 1) < 1e-2
