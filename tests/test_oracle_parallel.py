"""The all-cores build of the oracle (OpenMP over rows) gives the same bits
as the serial build.

Both libraries compile the same source; the OpenMP build spreads only row
loops whose every destination value has one writer (collision, free flight,
moments, fields, equilibrium set-up, scalar-only step), so each value is the
same expression evaluated once either way.  Checked population by
population, bit for bit, on lattices with every port kind, both wall
schemes, decay, and the scalar-only step.
"""
import numpy as np
import pytest

import oracle
from paper_1307_4703_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def _team():
    oracle.set_num_threads(4)  # several threads even on a one-core host
    yield


def _pair(prob, **kw):
    return oracle.from_problem(prob, **kw), oracle.from_problem(prob, parallel=True, **kw)


def _same(a, b):
    fa, ga = a.populations()
    fb, gb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    for x, y in zip(a.fields(), b.fields()):
        assert np.array_equal(x, y)


def test_thread_counts():
    assert oracle.num_threads(False) == 1
    assert oracle.num_threads(True) == 4


@pytest.mark.parametrize("paper_ports,decay,wall", [(False, 0.0, 0), (True, 0.01, 0), (False, 0.0, 1),
                                                    (True, 0.0, 1)])
def test_coupled_steps_bit_identical(paper_ports, decay, wall):
    prob, init = W.random_case(11, 53, 37, paper_ports=paper_ports, decay=decay)
    prob["wall_scheme"] = wall
    a, b = _pair(prob)
    for L in (a, b):
        L.init_equilibrium(**init)
    _same(a, b)
    for t in range(25):
        a.step(prob["states"][t])
        b.step(prob["states"][t])
    _same(a, b)
    pa, pb = a.post_collision(), b.post_collision()
    assert np.array_equal(pa[0], pb[0]) and np.array_equal(pa[1], pb[1])
    assert np.array_equal(a.diagnostics(7), b.diagnostics(7))


def test_chip_run_bit_identical():
    prob = W.config_small()
    a, b = _pair(prob)
    sched = lambda t: W.valve_word(prob, t)  # noqa: E731
    a.run(600, sched)
    b.run(600, sched)
    _same(a, b)


def test_scalar_step_bit_identical():
    prob, init = W.random_case(12, 40, 24, decay=0.02)
    a, b = _pair(prob)
    r = W.rng(5)
    ux = 0.05 * (r.random((prob["ny"], prob["nx"])) - 0.5)
    uy = 0.05 * (r.random((prob["ny"], prob["nx"])) - 0.5)
    for L in (a, b):
        L.init_equilibrium(**init)
        L.scalar_step(7, ux, uy, n=15)
    _same(a, b)


def test_adjoint_bit_identical():
    prob = W.config_large_chip(96, 48)
    prob["period"] = 20
    n = 45
    masks = [W.valve_word(prob, t) for t in range(n)]
    cx0, cx1, cy0, cy1 = prob["chamber"]
    oy = np.arange(cy0, cy1)
    ox = np.full_like(oy, (cx0 + cx1) // 2)
    obj = (ox, oy, (oy - cy0) / (cy1 - 1 - cy0), np.ones(len(oy)))
    a, b = _pair(prob)
    ra = a.adjoint(n, masks, *obj)
    rb = b.adjoint(n, masks, *obj)
    assert ra[0] == rb[0] and ra[1] == rb[1]
    assert np.array_equal(ra[2], rb[2]) and np.array_equal(ra[3], rb[3])
