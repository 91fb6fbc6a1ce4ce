"""16-bit storage of the populations (LBM_FP16, LBM_BF16) against the FP64
oracle.

The step's arithmetic is FP32; only the stored populations are rounded, to
16-bit deviations f_i - w_i and g_i - w_i C_ref (C_ref = 1/2).  Tolerances
follow from the unit roundoff u of the format (FP16 2^-11, BF16 2^-8):

  * codec: storing and reading back a population gives exactly the
    round-to-nearest-even 16-bit value of its deviation (checked bit for bit
    against numpy's rounding).
  * populations after n steps from a random state: every step rounds every
    stored deviation (|deviation| <= 1/2 for these states) once, with an
    error <= u/2 x 1/2, and the step itself does not amplify errors, so
    |f - f_oracle| <= n u / 4 plus the FP32 bound.
  * whole runs of the chip workloads: the conserved moments are not damped
    by the collision, so their rounding errors add up over the time the flow
    needs to relax (~10^3 steps on these chips) like a random walk,
    sqrt(10^3) x (u/2) x (a few planes) ~ 20 u.  Bound: max |du| / u_max and
    max |dC| <= 20 u, relative total mass <= u.  (Observed on the 256 x 128
    chip after 2000 steps: FP16 du/u_max 2.1e-3 = 4.3 u, dC 3.4e-3 = 7 u;
    BF16 du/u_max 4.1e-2 = 10 u, dC 1.3e-2 = 3.4 u.)
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1307_4703_gb300 import lbm, workloads as W  # noqa: E402

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

UNIT_ROUNDOFF = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, np.float32)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1307_4703_gb300 import build
    build.build()
    lbm.load()


def _round16(x, prec):
    """Round-to-nearest-even of float32 values to the 16-bit format, back as
    float32 (numpy's float16 cast for FP16; the upper half of the float32
    bits, rounded, for BF16)."""
    x = np.asarray(x, np.float32)
    if prec == "fp16":
        return x.astype(np.float16).astype(np.float32)
    b = x.view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32)


def _field_errors(prob, chip, ref):
    rho, ux, uy, C = chip.fields()
    r_rho, r_ux, r_uy, r_C = ref.fields()
    fl = ~ref.solid
    du = max(np.abs(ux - r_ux)[fl].max(), np.abs(uy - r_uy)[fl].max()) / prob["u_max"]
    dC = np.abs(C - r_C)[fl].max()
    dm = abs(rho[fl].astype(np.float64).sum() - r_rho[fl].sum()) / r_rho[fl].sum()
    return du, dC, dm


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_codec_rounds_to_nearest_even(prec):
    """set_populations then populations: every value comes back as the
    16-bit rounding of its deviation plus the offset, bit for bit."""
    prob, _ = W.random_case(3, 40, 24)
    chip = lbm.Chip.from_problem(prob, precision=prec)
    r = W.rng(77)
    ny, nx = prob["ny"], prob["nx"]
    f = (W9[:, None, None] * (1 + 0.3 * (r.random((9, ny, nx)) - 0.5))).astype(np.float32)
    g = (r.random((5, ny, nx)) * 0.3).astype(np.float32)
    chip.set_populations(f, g)
    f1, g1 = chip.populations()
    w0 = 1.0 / 3.0
    off = np.array([np.float32(w0) * np.float32(0.5)] + [np.float32(0.25 * (1 - w0)) * np.float32(0.5)] * 4,
                   np.float32)
    fd = (f - W9[:, None, None]).astype(np.float32)
    ef = (_round16(fd, prec) + W9[:, None, None]).astype(np.float32)
    eg = (_round16((g - off[:, None, None]).astype(np.float32), prec) + off[:, None, None]).astype(np.float32)
    assert np.array_equal(f1, ef)
    assert np.array_equal(g1, eg)
    # the scalar planes alone leave the fluid planes as they are
    chip.set_populations(None, g * 0.5)
    f2, _ = chip.populations()
    assert np.array_equal(f2, f1)
    chip.close()


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("nx,ny,seed", [(17, 9, 2), (130, 12, 4), (300, 20, 7)])
def test_population_parity_random_lattices(nx, ny, seed, prec, variant):
    """Random obstacles, every port kind, random fields and valve words:
    every post-collision population within n u / 4 (+ the FP32 bound) of the
    oracle after n = 10 steps; diagnostics to the same accuracy."""
    prob, init = W.random_case(seed, nx, ny)
    chip = lbm.Chip.from_problem(prob, precision=prec, variant=variant)
    ref = oracle.from_problem(prob)
    chip.init_equilibrium(**init)
    ref.init_equilibrium(**init)
    states = prob["states"]
    chip.set_valve_schedule(1, states)
    n = 10
    for t in range(n):
        chip.step(1)
        ref.step(states[t])
    f, g = chip.populations()
    fp, gp = ref.post_collision()
    rf, rg = np.moveaxis(fp, -1, 0), np.moveaxis(gp, -1, 0)
    fl = ~ref.solid
    tol = n * UNIT_ROUNDOFF[prec] / 4 + 2e-5
    ef = np.abs(f - rf)[:, fl].max()
    eg = np.abs(g - rg)[:, fl].max()
    assert ef <= tol and eg <= tol, (ef, eg, tol)
    d = chip.diagnostics()
    rd = ref.diagnostics(states[n - 1])
    nf = fl.sum()
    assert abs(d[0] - rd[0]) <= 9 * nf * tol
    assert abs(d[1] - rd[1]) <= 5 * nf * tol
    chip.close()


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_small_chip_full_run(prec):
    """The 256 x 128 chip from rest, 2000 steps, valves toggling every 500
    steps: velocity, concentration and mass within the 20 u bounds."""
    u = UNIT_ROUNDOFF[prec]
    prob = W.config_small()
    ref = oracle.from_problem(prob)
    ref.run(prob["steps"], lambda t: W.valve_word(prob, t))
    for variant in (1, 2):
        chip = lbm.Chip.from_problem(prob, precision=prec, variant=variant)
        chip.set_valve_schedule(prob["period"], prob["states"])
        chip.step(prob["steps"])
        du, dC, dm = _field_errors(prob, chip, ref)
        assert du <= 20 * u and dC <= 20 * u and dm <= u, (variant, du, dC, dm)
        chip.close()


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_full_chip_parity(prec):
    """The 1024 x 768 chip, tau_c = 0.505, 400 steps."""
    u = UNIT_ROUNDOFF[prec]
    prob = W.config_full_chip(tau_c=0.505)
    chip = lbm.Chip.from_problem(prob, precision=prec)
    chip.set_valve_schedule(200, prob["states"])
    ref = oracle.from_problem(prob)
    chip.step(400)
    ref.run(400, lambda t: prob["states"][(t // 200) % 2])
    du, dC, dm = _field_errors(prob, chip, ref)
    assert du <= 20 * u and dC <= 20 * u and dm <= u, (du, dC, dm)
    chip.close()


@pytest.fixture(scope="module")
def _oracle_runs():
    """The FP64 oracle (its all-cores build) on the 4096 x 2048 chip and its
    512 x 256 downscaled copy, 1000 steps from rest, computed once."""
    cache = {}

    def get(nx, ny):
        if (nx, ny) not in cache:
            prob = W.config_large_chip(nx, ny)
            ref = oracle.from_problem(prob, parallel=True)
            ref.run(1000, lambda t: W.valve_word(prob, t))
            cache[(nx, ny)] = (prob, ref, ref.fields())
        return cache[(nx, ny)]

    yield get
    for _, ref, _ in cache.values():
        ref.close()


@pytest.mark.parametrize("nx,ny", [(512, 256), (4096, 2048)])
def test_large_chip_1000_steps_against_oracle(nx, ny, _oracle_runs):
    """The precision workload (the 4096 x 2048 chip, tau = 0.6, tau_c =
    0.51) and its 512 x 256 copy, 1000 steps from rest with the valve
    schedule, stored as FP32, FP16 and BF16: every field against the FP64
    oracle.  Bounds: FP32 max |du| / u_max and max |dC| <= 1e-4 and the
    relative mass <= 1e-6; 16-bit storage the 20 u bounds above.  The
    errors are printed (pytest -s)."""
    prob, ref, (r_rho, r_ux, r_uy, r_C) = _oracle_runs(nx, ny)
    fl = ~ref.solid
    for prec in ("fp32", "fp16", "bf16"):
        with lbm.Chip.from_problem(prob, precision=prec) as chip:
            chip.set_valve_schedule(prob["period"], prob["states"])
            chip.step(1000)
            rho, ux, uy, C = chip.fields()
        drho = np.abs(rho - r_rho)[fl].max()
        du = max(np.abs(ux - r_ux)[fl].max(), np.abs(uy - r_uy)[fl].max()) / prob["u_max"]
        dC = np.abs(C - r_C)[fl].max()
        dm = abs(rho[fl].astype(np.float64).sum() - r_rho[fl].sum()) / r_rho[fl].sum()
        print("chip-%dx%d 1000 steps %s vs FP64 oracle: max|drho| %.3e max|du|/u_max %.3e max|dC| %.3e "
              "mass %.3e" % (nx, ny, prec, drho, du, dC, dm))
        if prec == "fp32":
            assert du <= 1e-4 and dC <= 1e-4 and dm <= 1e-6, (prec, du, dC, dm)
        else:
            u = UNIT_ROUNDOFF[prec]
            assert du <= 20 * u and dC <= 20 * u and dm <= u, (prec, du, dC, dm)


def test_large_chip_at_benchmark_launch_shape():
    """The 4096 x 2048 chip in FP16 from a perturbed state: three steps,
    every node against the oracle, and the 16-bit handle's bytes and
    footprint are half the FP32 handle's."""
    prob = W.config_large_chip()
    ny, nx = prob["ny"], prob["nx"]
    yy, xx = np.mgrid[0:ny, 0:nx]
    init = dict(rho=1.0 + 0.01 * np.sin(xx / 37.0) * np.cos(yy / 23.0),
                ux=0.02 * np.cos(yy / 41.0), uy=0.01 * np.sin(xx / 29.0),
                C=0.5 + 0.5 * np.sin(xx / 17.0 + yy / 13.0))
    chip = lbm.Chip.from_problem(prob, precision="fp16")
    ref = oracle.from_problem(prob)
    chip.init_equilibrium(**init)
    ref.init_equilibrium(**init)
    chip.set_valve_schedule(prob["period"], prob["states"])
    chip.step(3)
    ref.run(3, lambda t: W.valve_word(prob, t))
    du, dC, dm = _field_errors(prob, chip, ref)
    u = UNIT_ROUNDOFF["fp16"]
    assert du <= 20 * u and dC <= 20 * u and dm <= u, (du, dC, dm)
    info = chip.info()
    assert info["precision"] == lbm.LBM_FP16
    assert info["algorithmic_bytes_per_step"] == 56 * W.fluid_count(prob)
    with lbm.Chip.from_problem(prob) as c32:
        assert c32.info()["algorithmic_bytes_per_step"] == 2 * info["algorithmic_bytes_per_step"]
    chip.close()


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("opts", [dict(variant=1, block_threads=128),
                                  dict(variant=2, consumer_warps=1, pipeline_stages=1),
                                  dict(variant=2, consumer_warps=7, pipeline_stages=3),
                                  dict(variant=2, consumer_warps=3, pipeline_stages=2, max_blocks=5),
                                  dict(variant=4), dict(variant=4, block_threads=64, max_blocks=5),
                                  dict(variant=4, max_blocks=1), dict(variant=4, max_blocks=2),
                                  dict(variant=1, max_blocks=1)])
def test_16bit_variants_are_bit_identical(prec, opts):
    """Every 16-bit kernel variant and launch shape rounds the same FP32
    values: identical stored bits after 300 steps (a 700-wide lattice whose
    fluid spans are not multiples of the 8-element copy unit)."""
    prob, init = W.random_case(31, 700, 64, solid_frac=0.1)
    prob["states"] = [1, 2, 4, 3, 7, 0]
    a = lbm.Chip.from_problem(prob, precision=prec, variant=1)
    b = lbm.Chip.from_problem(prob, precision=prec, **opts)
    for c in (a, b):
        c.init_equilibrium(**init)
        c.set_valve_schedule(37, prob["states"])
        c.step(300)
    assert a.save_state() == b.save_state()
    a.close()
    b.close()


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_16bit_save_load_and_fp32_only_calls(prec):
    prob = W.config_small()
    a = lbm.Chip.from_problem(prob, precision=prec)
    assert a.info()["variant"] == 4  # the 16-bit default: registers + asynchronous prefetch
    a.set_valve_schedule(prob["period"], prob["states"])
    a.step(120)
    blob = a.save_state()
    assert len(blob) < 0.6 * len(lbm.Chip.from_problem(prob).save_state())
    a.step(80)
    b = lbm.Chip.from_problem(prob, precision=prec)
    b.load_state(blob)
    b.step(80)
    assert a.save_state() == b.save_state()
    with pytest.raises(lbm.LbmError) as e:  # a state of another precision does not load
        lbm.Chip.from_problem(prob).load_state(blob)
    assert e.value.status == lbm.LBM_ERR_ARG
    for call in (lambda: a.store_velocity(1), lambda: a.scalar_step(1),
                 lambda: a.set_velocity_field(1, np.zeros((128, 256)), np.zeros((128, 256))),
                 lambda: a.adjoint(10, [100], [64], [0.5])):
        with pytest.raises(lbm.LbmError) as e:
            call()
        assert e.value.status == lbm.LBM_ERR_STATE
    a.close()
    b.close()
