"""Scalar-only steps on stored velocity fields (lbm_store_velocity,
lbm_set_velocity_field, lbm_scalar_step) against the FP64 oracle.

Convention: GPU step t completes the open ports of valve word w(t) and then
relaxes the scalar with the field of w(t).  In the oracle's collide-then-
stream order that relaxation is the collision at the start of oracle step
t + 1, so the oracle is driven with the field of w(t - 1) and the ports of
w(t); both start from a scalar at the equilibrium of the first field.
Concentrations are compared (they are the moments of both the pre- and the
post-collision populations).  Tolerances: see each test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1307_4703_gb300 import lbm, workloads as W  # noqa: E402

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _run_oracle(prob, init, fields, words, u_scale):
    L = oracle.from_problem(prob)
    first = fields[words[0]]
    L.init_equilibrium(init["rho"], u_scale * first[0], u_scale * first[1], init["C"])
    for t, w in enumerate(words):
        fx, fy = fields[words[max(t - 1, 0)]]
        L.scalar_step(w, u_scale * fx, u_scale * fy)
    return L


@pytest.mark.parametrize("scalar_variant", [1, 2])
@pytest.mark.parametrize("seed,nx,ny", [(2, 40, 24), (9, 150, 20)])
def test_scalar_steps_match_oracle_random_fields(seed, nx, ny, scalar_variant):
    prob, init = W.random_case(seed, nx, ny)
    r = W.rng(seed + 50)
    fields = {w: (0.05 * (r.random((ny, nx)) - 0.5), 0.05 * (r.random((ny, nx)) - 0.5)) for w in (7, 3, 0)}
    words = [7] * 4 + [3] * 5 + [0] * 3 + [7] * 4
    u_scale = 1.5
    chip = lbm.Chip.from_problem(prob, scalar_variant=scalar_variant)
    first = fields[words[0]]
    chip.init_equilibrium(init["rho"], u_scale * first[0], u_scale * first[1], init["C"])
    for w, (fx, fy) in fields.items():
        chip.set_velocity_field(w, fx, fy)
    f0, _ = chip.populations()
    for w in words:
        chip.set_valves(w)
        chip.scalar_step(1, u_scale)
    L = _run_oracle(prob, init, fields, words, u_scale)
    fl = ~L.solid
    C = chip.fields()[3]
    assert np.abs(C - L.fields()[3])[fl].max() < 1e-5
    f1, _ = chip.populations()
    assert np.array_equal(f0, f1)  # the fluid populations are not touched
    chip.close()


@pytest.mark.parametrize("own_fields", [True, False])
def test_stored_fields_workflow_on_the_small_chip(own_fields):
    """The paper's workflow: run the fluid to its flow field for each valve
    state, store the three fields, then advance the scalar alone with a
    larger time step (u_scale = 2) under the toggling valves, 600 steps.

    own_fields=False gives the GPU the oracle's fields and scalar state: only
    the scalar steps differ (FP32 against FP64), tolerance 1e-5.
    own_fields=True stores the GPU's own FP32 flow fields, which differ from
    the FP64 ones by du ~ 1e-7: tolerance 1e-4, the coupled-run bound."""
    prob = W.config_small()
    chip = lbm.Chip.from_problem(prob)
    ref = oracle.from_problem(prob)
    fields = {}
    for w, n in ((1, 400), (2, 400), (0, 200)):
        chip.set_valves(w)
        chip.step(n)
        ref.step(w, n)
        _, ux, uy, _ = ref.fields()
        fields[w] = (ux, uy)
        if own_fields:
            chip.store_velocity(w)
        else:
            chip.set_velocity_field(w, ux, uy)
    if not own_fields:  # the same scalar start on both sides (the GPU stores post-collision values)
        _, g = ref.post_collision()
        chip_f, _ = chip.populations()
        chip.set_populations(chip_f, np.moveaxis(g, -1, 0))
    u_scale = 2.0
    chip.set_valve_schedule(50, [1, 0, 2, 0])
    t0 = chip.step_count()
    words = [[1, 0, 2, 0][((t0 + t) // 50) % 4] for t in range(600)]
    chip.scalar_step(600, u_scale)
    # the oracle continues from its own state, with its own fields; its first
    # collision is the one that produced the GPU's starting state: the
    # coupled step's, with the fluid's own (unscaled) velocity
    for t, w in enumerate(words):
        if t == 0:
            fx, fy = fields[0]
            ref.scalar_step(w, fx, fy)
        else:
            fx, fy = fields[words[t - 1]]
            ref.scalar_step(w, u_scale * fx, u_scale * fy)
    fl = ~ref.solid
    C = chip.fields()[3]
    err = np.abs(C - ref.fields()[3])[fl].max()
    assert err < (1e-4 if own_fields else 1e-5), err
    d = chip.diagnostics()
    assert abs(d[1] - ref.fields()[3][fl].sum()) < 1e-3 * max(1.0, d[1])
    chip.close()


def test_scalar_steps_split_into_calls_and_need_fields():
    prob = W.config_small()
    a = lbm.Chip.from_problem(prob)
    with pytest.raises(lbm.LbmError) as e:
        a.scalar_step(1)
    assert e.value.status == lbm.LBM_ERR_STATE
    b = lbm.Chip.from_problem(prob)
    for c in (a, b):
        c.set_valves(1)
        c.step(100)
        c.store_velocity(1)
    a.scalar_step(7, 3.0)          # odd count: the scalar planes are copied back
    b.scalar_step(3, 3.0)
    b.scalar_step(4, 3.0)
    fa, ga = a.populations()
    fb, gb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    a.step(5)                      # coupled steps continue from the combined state
    b.step(5)
    assert np.array_equal(a.populations()[1], b.populations()[1])
    a.close()
    b.close()


@pytest.mark.parametrize("paper_ports,decay", [(False, 0.0), (True, 0.002)])
def test_scalar_kernel_variants_are_bit_identical(paper_ports, decay):
    """The register and bulk-copy kernels of lbm_scalar_step do the same
    arithmetic per node: identical populations and diagnostics after
    scalar steps across valve switches (a 600 x 300 chip, several tiles per
    row and a ragged last segment)."""
    prob = W.two_channel_chip(600, 300, 40, 580, 120, 0.6, 0.52, 0.04, 30, 200, paper_ports=paper_ports,
                              decay=decay)
    out = []
    for sv in (1, 2):
        chip = lbm.Chip.from_problem(prob, scalar_variant=sv)
        chip.set_valve_schedule(prob["period"], prob["states"])
        chip.step(40)
        for w in sorted(set(prob["states"])):
            chip.store_velocity(w)
        chip.scalar_step(100, 2.0)
        d = chip.diagnostics()
        f, g = chip.populations()
        out.append((f, g, d))
        chip.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert np.allclose(out[0][2], out[1][2], rtol=1e-12, atol=1e-9)


def test_full_chip_chamber_profile_in_the_papers_workflow():
    """The 1024 x 768 chip (tau_c = 0.52, the largest diffusivity of its
    range) in the paper's workflow: a stationary velocity field per valve
    state (the channel-flow stand-ins of workloads.channel_flow_fields) and
    40000 scalar-only steps with the valves switching every 2000 steps, so
    that compound has reached the chamber (the top channel's front passes
    the chamber's centre column near step 22000) and the gradient along y at
    its centre column has started to form.  Every concentration against the
    FP64 oracle (its all-cores build) within the whole-run bound 1e-4.
    (The steady chamber gradient itself needs about (568 rows)^2 / D = 5e7
    steps at this size, out of the oracle's reach.)"""
    prob = W.config_full_chip(tau_c=0.52)
    fields = W.channel_flow_fields(prob)
    n, period = 40000, prob["period"]
    chip = lbm.Chip.from_problem(prob)
    for w, (fx, fy) in fields.items():
        chip.set_velocity_field(w, fx, fy)
    chip.set_valve_schedule(period, prob["states"])
    chip.scalar_step(n, 1.0)
    C = chip.fields()[3]
    chip.close()
    # the oracle: step t completes the ports of w(t) and collides with the
    # field of w(t - 1) (see the module docstring); both start at C = 0
    L = oracle.from_problem(prob, parallel=True)
    t = 0
    while t < n:
        w = W.valve_word(prob, t)
        L.scalar_step(w, *fields[W.valve_word(prob, max(t - 1, 0))], n=1)
        t += 1
        m = min(period - t % period, n - t) if t % period else 0
        if m:
            L.scalar_step(w, *fields[w], n=m)
            t += m
    rC = L.fields()[3]
    fl = ~L.solid
    dC = np.abs(C - rC)[fl].max()
    cx0, cx1, cy0, cy1 = prob["chamber"]
    col = rC[cy0:cy1, (cx0 + cx1) // 2]
    print("chip-1024x768 frozen-velocity run, %d steps: max|dC| %.3e; chamber centre column C top %.4f, "
          "rows above 1e-3: %d" % (n, dC, col[-1], int((col > 1e-3).sum())))
    assert dC <= 1e-4, dC
    # compound has entered the chamber from the top channel, and none from the bottom one
    assert col[-1] > 1e-3 and abs(col[0]) < 1e-6
    L.close()
