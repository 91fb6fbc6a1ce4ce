"""CUDA-graph replay of step runs (graph_steps) and the launch-shape
autotuner (lbm_autotune): both change how steps are launched, never what
they compute, so the populations must stay bit-identical."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1307_4703_gb300 import lbm, workloads as W  # noqa: E402

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1307_4703_gb300 import build
    build.build()
    lbm.load()


def _same(a, b):
    fa, ga = a.populations()
    fb, gb = b.populations()
    return np.array_equal(fa, fb) and np.array_equal(ga, gb)


@pytest.mark.parametrize("graph_steps,variant", [(2, 0), (10, 0), (64, 0), (10, 5)])
def test_graph_replay_is_bit_identical(graph_steps, variant):
    """Valve switches every 25 steps split the runs: graphs where the valve
    word holds for graph_steps steps, single launches elsewhere (with the
    default kernel and with variant 5).  The reference chip runs the same
    kernel without graphs: the diagnostics' summation order follows the
    kernel's tiles, so they are compared bit for bit within one variant."""
    prob, init = W.random_case(12, 300, 20)
    a = lbm.Chip.from_problem(prob, variant=variant)
    b = lbm.Chip.from_problem(prob, graph_steps=graph_steps, variant=variant)
    for c in (a, b):
        c.init_equilibrium(**init)
        c.set_valve_schedule(25, prob["states"])
    for n in (137, 1, 64, 3):
        a.step(n)
        b.step(n)
    assert a.step_count() == b.step_count() == 205
    assert _same(a, b)
    assert np.array_equal(a.diagnostics(), b.diagnostics())
    a.close()
    b.close()


def test_graph_replay_on_a_batch_with_own_valve_programs():
    chips = W.config_batch(3, seed=6)
    a = lbm.Chip.batch(chips)
    b = lbm.Chip.batch(chips, graph_steps=20)
    for c in (a, b):
        for k, p in enumerate(chips):
            c.set_instance_schedule(k, 30 + 17 * k, p["states"])
        c.step(250)
    assert _same(a, b)
    a.close()
    b.close()


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_autotune_keeps_the_state_and_the_results(prec):
    prob = W.config_small()
    a = lbm.Chip.from_problem(prob, precision=prec)
    b = lbm.Chip.from_problem(prob, precision=prec, graph_steps=8)
    for c in (a, b):
        c.set_valve_schedule(prob["period"], prob["states"])
        c.step(100)
    d0 = b.diagnostics()
    f0, g0 = b.populations()
    info = b.autotune(trial_steps=5)
    assert info["variant"] in (1, 2, 3, 4, 5) and info["grid"] >= 1
    assert b.step_count() == 100
    f1, g1 = b.populations()
    assert np.array_equal(f0, f1) and np.array_equal(g0, g1)
    assert np.array_equal(b.diagnostics(), d0)
    for c in (a, b):
        c.step(300)
    assert _same(a, b)
    a.close()
    b.close()


def test_graph_steps_must_be_even():
    prob = W.config_small()
    with pytest.raises(lbm.LbmError) as e:
        lbm.Chip.from_problem(prob, graph_steps=3)
    assert e.value.status == lbm.LBM_ERR_ARG


@pytest.mark.parametrize("multi_step", [16, 7, 1000])
def test_multi_step_launch_is_bit_identical(multi_step):
    """Runs of steps in one cooperative launch (a grid-wide barrier between
    steps): valve switches every 25 steps split the runs, odd run lengths
    leave the state in the other buffer.  Populations are bit-identical; the
    diagnostics are sums over another grouping of blocks, equal to round-off."""
    prob, init = W.random_case(12, 300, 20)
    a = lbm.Chip.from_problem(prob)
    b = lbm.Chip.from_problem(prob, multi_step=multi_step)
    for c in (a, b):
        c.init_equilibrium(**init)
        c.set_valve_schedule(25, prob["states"])
    for n in (137, 1, 64, 3):
        a.step(n)
        b.step(n)
    assert a.step_count() == b.step_count() == 205
    assert _same(a, b)
    assert np.allclose(a.diagnostics(), b.diagnostics(), rtol=1e-6, atol=1e-9)
    a.close()
    b.close()


def test_multi_step_launch_on_larger_chips_and_batches():
    """A chip of several tiles per row with a ragged last segment, and a
    batch of chips with their own valve programs."""
    prob = W.two_channel_chip(600, 300, 40, 580, 120, 0.6, 0.52, 0.04, 30, 200)
    a = lbm.Chip.from_problem(prob)
    b = lbm.Chip.from_problem(prob, multi_step=64)
    for c in (a, b):
        c.set_valve_schedule(prob["period"], prob["states"])
        c.step(173)
    assert _same(a, b)
    assert np.allclose(a.diagnostics(), b.diagnostics(), rtol=1e-6, atol=1e-9)
    a.close()
    b.close()
    chips = W.config_batch(3, seed=6)
    a = lbm.Chip.batch(chips)
    b = lbm.Chip.batch(chips, multi_step=50)
    for c in (a, b):
        for k, p in enumerate(chips):
            c.set_instance_schedule(k, 30 + 17 * k, p["states"])
        c.step(250)
    assert _same(a, b)
    a.close()
    b.close()


def test_multi_step_barrier_timeout_is_reported_and_recoverable():
    """The grid barrier's bounded wait runs out (the test hook makes it wait
    for an arrival that never comes): the kernel stops with the timeout bit,
    the host reports LBM_ERR_TIMEOUT, and after clearing it the context and
    the handle work again.  No fault, trap or endless wait."""
    prob, init = W.random_case(12, 300, 20)
    chip = lbm.Chip.from_problem(prob, multi_step=8)
    chip.init_equilibrium(**init)
    chip.debug_barrier_extra(1)
    chip.step(4)
    with pytest.raises(lbm.LbmError) as e:
        chip.synchronize()
    assert e.value.status == lbm.LBM_ERR_TIMEOUT
    chip.clear_error()
    chip.debug_barrier_extra(0)
    chip.init_equilibrium(**init)
    ref = lbm.Chip.from_problem(prob)
    ref.init_equilibrium(**init)
    for c in (chip, ref):
        c.step(10)
    chip.synchronize()
    assert _same(chip, ref)
    chip.close()
    ref.close()
