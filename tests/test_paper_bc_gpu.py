"""The paper's own port boundary (do-nothing + rescaling to the prescribed
density or concentration) and the decay term -kC on the GPU, against the FP64
oracle (whose pins are in tests/test_oracle_paper_bc.py).  Tolerances as for
the Zou-He lattices (tests/test_parity_gpu.py): FP32 populations drift by
at most n * 30 * 2^-24 over n steps; whole runs within 1e-4 of u_max and
in C."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1307_4703_gb300 import lbm, workloads as W  # noqa: E402

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

POP_ATOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1307_4703_gb300 import build
    build.build()
    lbm.load()


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("nx,ny,seed", [(17, 9, 2), (130, 12, 4), (300, 20, 7)])
def test_population_parity_with_paper_ports_and_decay(nx, ny, seed, variant):
    prob, init = W.random_case(seed, nx, ny, paper_ports=True, decay=2e-3)
    chip = lbm.Chip.from_problem(prob, variant=variant)
    ref = oracle.from_problem(prob)
    chip.init_equilibrium(**init)
    ref.init_equilibrium(**init)
    chip.set_valve_schedule(1, prob["states"])
    for t in range(10):
        chip.step(1)
        ref.step(prob["states"][t])
    f, g = chip.populations()
    fp, gp = ref.post_collision()
    fl = ~ref.solid
    ef = np.abs(f - np.moveaxis(fp, -1, 0))[:, fl].max()
    eg = np.abs(g - np.moveaxis(gp, -1, 0))[:, fl].max()
    assert ef <= POP_ATOL and eg <= POP_ATOL, (ef, eg)
    d = chip.diagnostics()
    rd = ref.diagnostics(prob["states"][9])
    assert abs(d[0] - rd[0]) / rd[0] < 1e-6
    assert abs(d[1] - rd[1]) <= 1e-5 * max(1.0, abs(rd[1]))
    assert abs(d[2] - rd[2]) <= 1e-5 and abs(d[3] - rd[3]) <= 1e-5
    chip.close()


def test_fp16_storage_with_paper_ports():
    prob, init = W.random_case(4, 130, 12, paper_ports=True, decay=2e-3)
    chip = lbm.Chip.from_problem(prob, precision="fp16")
    ref = oracle.from_problem(prob)
    chip.init_equilibrium(**init)
    ref.init_equilibrium(**init)
    chip.set_valve_schedule(1, prob["states"])
    for t in range(10):
        chip.step(1)
        ref.step(prob["states"][t])
    f, g = chip.populations()
    fp, gp = ref.post_collision()
    fl = ~ref.solid
    tol = 10 * 2.0 ** -11 / 4 + POP_ATOL
    assert np.abs(f - np.moveaxis(fp, -1, 0))[:, fl].max() <= tol
    assert np.abs(g - np.moveaxis(gp, -1, 0))[:, fl].max() <= tol
    chip.close()


def test_pressure_driven_chip_with_decay_matches_oracle():
    """The two-channel chip driven the paper's way (rescaling inlet and
    outlet, u_max = 0.01 by the Poiseuille pressure drop) with a decaying
    compound, 2000 steps with the valves toggling every 500."""
    prob = W.two_channel_chip(256, 128, 16, 256, 64, 0.8, 0.55, 0.01, 500, 2000, paper_ports=True,
                              decay=1e-4, name="paper-chip-256x128")
    chip = lbm.Chip.from_problem(prob)
    chip.set_valve_schedule(prob["period"], prob["states"])
    ref = oracle.from_problem(prob)
    chip.step(2000)
    ref.run(2000, lambda t: W.valve_word(prob, t))
    rho, ux, uy, C = chip.fields()
    r_rho, r_ux, r_uy, r_C = ref.fields()
    fl = ~ref.solid
    du = max(np.abs(ux - r_ux)[fl].max(), np.abs(uy - r_uy)[fl].max()) / prob["u_max"]
    dC = np.abs(C - r_C)[fl].max()
    dm = abs(rho[fl].astype(np.float64).sum() - r_rho[fl].sum()) / r_rho[fl].sum()
    assert du <= 1e-4 and dC <= 1e-4 and dm <= 1e-6, (du, dC, dm)
    # the open channel (bottom, channel 1, in the last 500 steps) holds its port densities
    bottom = [p for p in prob["ports"] if p["channel"] == 1]
    for p in bottom:
        assert np.abs(rho[p["y0"]:p["y1"], p["x"]] - p["rho"]).max() < 1e-5
    # the pressure drop drives the open channel's flow towards +x
    assert ux[0:16, 40].min() > 0
    with pytest.raises(lbm.LbmError) as e:
        chip.adjoint(10, [128], [64], [0.0])
    assert e.value.status == lbm.LBM_ERR_STATE
    chip.close()


def test_decay_on_the_gpu():
    """Uniform closed box: C(t) = C0 (1 - k)^t (FP32); the sinh steady
    profile by scalar-only steps against the oracle."""
    k, C0, n = 3e-3, 0.7, 50
    solid = np.zeros((8, 40), np.uint8)
    chip = lbm.Chip(solid, 0.8, 0.65, decay=k)
    chip.init_equilibrium(np.ones((8, 40)), np.zeros((8, 40)), np.zeros((8, 40)), np.full((8, 40), C0))
    chip.step(n)
    C = chip.fields()[3]
    assert np.abs(C / (C0 * (1 - k) ** n) - 1).max() < 1e-5
    chip.close()
    length, ny, tau_g = 64, 4, 1.0
    nx = length + 1
    D = (tau_g - 0.5) / 3
    kk = D * (2.0 / length) ** 2
    ports = [dict(channel=0, side=0, x=0, y0=0, y1=ny, kind=0, rho=1.0),
             dict(channel=0, side=1, x=nx - 1, y0=0, y1=ny, kind=0, rho=1.0)]
    eu, ec = np.zeros((2, ny)), np.zeros((2, ny))
    ec[0] = 1.0
    prob = dict(solid=np.zeros((ny, nx), np.uint8), tau=0.8, tau_c=tau_g, ports=ports, edge_u=eu, edge_C=ec,
                decay=kk)
    chip = lbm.Chip.from_problem(prob)
    ref = oracle.from_problem(prob)
    z = np.zeros((ny, nx))
    chip.set_velocity_field(1, z, z)
    chip.set_valves(1)
    chip.scalar_step(20000)
    ref.scalar_step(1, z, z, 20000)
    # a whole run (20000 steps): the 1e-4 bound of the chip runs
    assert np.abs(chip.fields()[3] - ref.fields()[3]).max() < 1e-4
    x = np.arange(nx)
    lam = np.sqrt(kk / D)
    exact = np.sinh(lam * (length - x)) / np.sinh(lam * length)
    assert np.abs(chip.fields()[3][1] - exact).max() < 1e-4
    chip.close()


def test_scalar_only_step_with_the_paper_inlet():
    """Stored velocity field, rescaling inlet starting without compound (the
    equilibrium fallback) and then with it (the rescaling), do-nothing
    outlet: against the oracle's scalar-only step."""
    prob, init = W.random_case(9, 150, 20, paper_ports=True, decay=1e-3)
    chip = lbm.Chip.from_problem(prob)
    ref = oracle.from_problem(prob)
    r = W.rng(71)
    ux = 0.05 * (r.random((20, 150)) - 0.5)
    uy = 0.05 * (r.random((20, 150)) - 0.5)
    init["C"] = np.zeros((20, 150))
    chip.init_equilibrium(init["rho"], ux, uy, init["C"])
    ref.init_equilibrium(init["rho"], ux, uy, init["C"])
    chip.set_velocity_field(7, ux, uy)
    chip.set_valves(7)
    chip.scalar_step(30)
    ref.scalar_step(7, ux, uy, 30)
    fl = ~ref.solid
    assert np.abs(chip.fields()[3] - ref.fields()[3])[fl].max() < 1e-5
    chip.close()


@pytest.mark.parametrize("variant,precision", [(1, "fp32"), (2, "fp32"), (1, "bf16"), (2, "fp16")])
@pytest.mark.parametrize("paper_ports", [False, True])
def test_equilibrium_walls_match_oracle(variant, precision, paper_ports):
    """The paper's equilibrium-interpolation walls (random obstacles, every
    port kind), 10 steps from random fields: populations against the oracle
    (FP32 bound, or the 16-bit bound n u / 4)."""
    prob, init = W.random_case(7, 300, 20, paper_ports=paper_ports)
    prob["wall_scheme"] = 1
    chip = lbm.Chip.from_problem(prob, variant=variant, precision=precision)
    ref = oracle.from_problem(prob)
    chip.init_equilibrium(**init)
    ref.init_equilibrium(**init)
    chip.set_valve_schedule(1, prob["states"])
    for t in range(10):
        chip.step(1)
        ref.step(prob["states"][t])
    f, g = chip.populations()
    fp, gp = ref.post_collision()
    fl = ~ref.solid
    u = {"fp32": 0.0, "fp16": 2.0 ** -11, "bf16": 2.0 ** -8}[precision]
    tol = 10 * u / 4 + POP_ATOL
    assert np.abs(f - np.moveaxis(fp, -1, 0))[:, fl].max() <= tol
    assert np.abs(g - np.moveaxis(gp, -1, 0))[:, fl].max() <= tol
    chip.close()


def test_equilibrium_wall_chip_run_matches_oracle():
    prob = W.two_channel_chip(256, 128, 16, 256, 64, 0.8, 0.55, 0.01, 500, 1000, paper_ports=True,
                              name="paper-walls-256x128")
    prob["wall_scheme"] = 1
    chip = lbm.Chip.from_problem(prob)
    chip.set_valve_schedule(prob["period"], prob["states"])
    ref = oracle.from_problem(prob)
    chip.step(1000)
    ref.run(1000, lambda t: W.valve_word(prob, t))
    rho, ux, uy, C = chip.fields()
    r_rho, r_ux, r_uy, r_C = ref.fields()
    fl = ~ref.solid
    du = max(np.abs(ux - r_ux)[fl].max(), np.abs(uy - r_uy)[fl].max()) / prob["u_max"]
    dC = np.abs(C - r_C)[fl].max()
    dm = abs(rho[fl].astype(np.float64).sum() - r_rho[fl].sum()) / r_rho[fl].sum()
    assert du <= 1e-4 and dC <= 1e-4 and dm <= 1e-6, (du, dC, dm)
    with pytest.raises(lbm.LbmError) as e:
        chip.adjoint(10, [128], [64], [0.0])
    assert e.value.status == lbm.LBM_ERR_STATE
    chip.close()


def test_equilibrium_walls_with_graphs_and_batches():
    """The wall values are written by two extra kernels per step: CUDA-graph
    replay and a batch of two chips give the same bits as direct steps of
    single chips."""
    prob, init = W.random_case(3, 130, 16)
    prob["wall_scheme"] = 1
    prob["states"] = [7, 7, 3, 1]
    a = lbm.Chip.from_problem(prob)
    b = lbm.Chip.from_problem(prob, graph_steps=6)
    for c in (a, b):
        c.init_equilibrium(**init)
        c.set_valve_schedule(20, prob["states"])
        c.step(90)
    fa, ga = a.populations()
    fb, gb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    chips = W.config_batch(2, seed=3)
    for p in chips:
        p["wall_scheme"] = 1
    batch = lbm.Chip.batch(chips, wall_scheme=1)
    alone = [lbm.Chip.from_problem(p) for p in chips]
    for c in alone:
        c.set_valves(1)
        c.step(60)
    batch.set_valves(1)
    batch.step(60)
    f, g = batch.populations()
    for k, c in enumerate(alone):
        i = batch.instance(k)
        fk = f[:, i["row0"]:i["row0"] + i["ny"], :i["nx"]]
        fa = c.populations()[0]
        fl = ~c.solid
        assert np.array_equal(fa[:, fl], fk[:, fl])
        c.close()
    a.close()
    b.close()
    batch.close()
