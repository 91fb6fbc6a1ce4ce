"""CUDA path against the FP64 oracle, through the C ABI, on the same seeded
inputs.

Tolerances (FP32 path against FP64 arithmetic):
  * populations after n steps from a random state: every stored value is
    the result of about 30 FP32 roundings per step of quantities of size
    <= 1, so |f_gpu - f_oracle| <= n * 30 * 2^-24 bounds the drift;
    POP_ATOL uses that bound for n = 10 (1.8e-5, rounded up to 2e-5).
  * whole runs of the chip workloads (the figures the method's users need):
    max |u_gpu - u_oracle| / u_max <= 1e-4, max |C_gpu - C_oracle| <= 1e-4,
    total mass |M_gpu - M_oracle| / M_oracle <= 1e-6.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1307_4703_gb300 import lbm, workloads as W  # noqa: E402

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

POP_ATOL = 2e-5
U_TOL = 1e-4
C_TOL = 1e-4
MASS_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1307_4703_gb300 import build
    build.build()
    lbm.load()


def _oracle_pops(ref):
    """Oracle post-collision populations in the library's [i][y][x] layout."""
    fp, gp = ref.post_collision()
    return np.moveaxis(fp, -1, 0), np.moveaxis(gp, -1, 0)


def _field_errors(prob, chip, ref):
    rho, ux, uy, C = chip.fields()
    r_rho, r_ux, r_uy, r_C = ref.fields()
    fl = ~ref.solid
    du = max(np.abs(ux - r_ux)[fl].max(), np.abs(uy - r_uy)[fl].max()) / prob["u_max"]
    dC = np.abs(C - r_C)[fl].max()
    dm = abs(rho[fl].astype(np.float64).sum() - r_rho[fl].sum()) / r_rho[fl].sum()
    assert np.all(rho[~fl] == 0) and np.all(C[~fl] == 0)
    return du, dC, dm


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("nx,ny,seed", [(8, 8, 1), (17, 9, 2), (64, 32, 3), (130, 12, 4),
                                        (300, 20, 5), (129, 16, 6), (300, 20, 7), (260, 8, 5)])
def test_population_parity_random_lattices(nx, ny, seed, variant):
    """Random obstacles, every port kind on both sides, random initial
    fields and a random valve word per step: every post-collision
    population of every fluid node agrees with the oracle, for both kernel
    variants.  The sizes span one to three 128-node tiles with ragged
    tails."""
    prob, init = W.random_case(seed, nx, ny)
    chip = lbm.Chip.from_problem(prob, variant=variant)
    ref = oracle.from_problem(prob)
    chip.init_equilibrium(**init)
    ref.init_equilibrium(**init)
    states = prob["states"]
    chip.set_valve_schedule(1, states)
    for t in range(10):
        chip.step(1)
        ref.step(states[t])
    f, g = chip.populations()
    rf, rg = _oracle_pops(ref)
    fl = ~ref.solid
    ef = np.abs(f - rf)[:, fl].max()
    eg = np.abs(g - rg)[:, fl].max()
    assert ef <= POP_ATOL and eg <= POP_ATOL, (ef, eg)
    d = chip.diagnostics()
    rd = ref.diagnostics(states[9])
    assert abs(d[0] - rd[0]) / rd[0] < 1e-6
    assert abs(d[1] - rd[1]) <= 1e-5 * max(1.0, abs(rd[1]))
    assert abs(d[2] - rd[2]) <= 1e-5 and abs(d[3] - rd[3]) <= 1e-5
    chip.close()


@pytest.mark.parametrize("opts", [dict(variant=1), dict(variant=2, pipeline_stages=1, consumer_warps=1),
                                  dict(variant=2, pipeline_stages=3, consumer_warps=7),
                                  dict(variant=2, pipeline_stages=1, consumer_warps=7, max_blocks=3),
                                  dict(variant=2, pipeline_stages=5, consumer_warps=3, max_blocks=7),
                                  dict(variant=3), dict(variant=3, pipeline_stages=3, consumer_warps=8),
                                  dict(variant=3, pipeline_stages=1, consumer_warps=1, max_blocks=5),
                                  dict(variant=4), dict(variant=4, block_threads=256),
                                  dict(variant=4, block_threads=64, max_blocks=3),
                                  dict(variant=5), dict(variant=5, block_threads=64, max_blocks=3),
                                  dict(variant=1, max_blocks=1), dict(variant=1, max_blocks=2),
                                  dict(variant=1, block_threads=64, max_blocks=9),
                                  dict(variant=4, max_blocks=1), dict(variant=4, block_threads=64, max_blocks=2)])
def test_kernel_variants_are_bit_identical(opts):
    """Both step kernels and any pipeline shape run the same arithmetic on
    the same values: identical bits after 300 steps with valve toggles and
    a random obstacle field.  The register variants run tiles that hold a
    port node in their own blocks: one block (every tile through the port
    loop), two (one block each) and small grids check that split."""
    prob, init = W.random_case(31, 700, 64, solid_frac=0.1)
    prob["states"] = [1, 2, 4, 3, 7, 0]
    ref = lbm.Chip.from_problem(prob)
    other = lbm.Chip.from_problem(prob, **opts)
    for c in (ref, other):
        c.init_equilibrium(**init)
        c.set_valve_schedule(37, prob["states"])
        c.step(300)
    fa, ga = ref.populations()
    fb, gb = other.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    da, db = ref.diagnostics(), other.diagnostics()
    # lanes sum in compensated FP32, so launch shapes agree to FP32 rounding
    assert np.allclose(da, db, rtol=1e-6, atol=1e-6)
    assert ref.info()["variant"] == 1 and other.info()["variant"] == opts["variant"]
    ref.close()
    other.close()


def test_small_chip_full_run():
    """The 256 x 128 chip from rest: 2000 steps with the valves toggling
    every 500 steps."""
    prob = W.config_small()
    chip = lbm.Chip.from_problem(prob)
    chip.set_valve_schedule(prob["period"], prob["states"])
    ref = oracle.from_problem(prob)
    chip.step(prob["steps"])
    ref.run(prob["steps"], lambda t: W.valve_word(prob, t))
    du, dC, dm = _field_errors(prob, chip, ref)
    assert du <= U_TOL and dC <= C_TOL and dm <= MASS_TOL, (du, dC, dm)
    d = chip.diagnostics()
    rd = ref.diagnostics(W.valve_word(prob, prob["steps"] - 1))
    assert abs(d[0] - rd[0]) / rd[0] <= MASS_TOL
    assert abs(d[2] - rd[2]) <= 1e-4 * abs(rd[2])
    assert chip.step_count() == prob["steps"]
    chip.close()


@pytest.mark.parametrize("tau_c", [0.505, 0.52])
def test_full_chip_parity(tau_c):
    """The 1024 x 768 chip at both ends of its tau_c range, 400 steps
    (the channels' flow has reached the chamber by then)."""
    prob = W.config_full_chip(tau_c=tau_c)
    chip = lbm.Chip.from_problem(prob)
    chip.set_valve_schedule(200, prob["states"])
    ref = oracle.from_problem(prob)
    chip.step(400)
    ref.run(400, lambda t: prob["states"][(t // 200) % 2])
    du, dC, dm = _field_errors(prob, chip, ref)
    assert du <= U_TOL and dC <= C_TOL and dm <= MASS_TOL, (du, dC, dm)
    chip.close()


def test_large_chip_parity_at_benchmark_launch_shape():
    """The 4096 x 2048 chip in the launch shape the benchmark times, from a
    perturbed state (so every node moves), three steps, every node compared."""
    prob = W.config_large_chip()
    r = W.rng(99)
    ny, nx = prob["ny"], prob["nx"]
    yy, xx = np.mgrid[0:ny, 0:nx]
    init = dict(rho=1.0 + 0.01 * np.sin(xx / 37.0) * np.cos(yy / 23.0),
                ux=0.02 * np.cos(yy / 41.0), uy=0.01 * np.sin(xx / 29.0),
                C=0.5 + 0.5 * np.sin(xx / 17.0 + yy / 13.0))
    chip = lbm.Chip.from_problem(prob)
    ref = oracle.from_problem(prob)
    chip.init_equilibrium(**init)
    ref.init_equilibrium(**init)
    chip.set_valve_schedule(prob["period"], prob["states"])
    chip.step(3)
    ref.run(3, lambda t: W.valve_word(prob, t))
    du, dC, dm = _field_errors(prob, chip, ref)
    assert du <= U_TOL and dC <= C_TOL and dm <= MASS_TOL, (du, dC, dm)
    info = chip.info()
    assert info["fluid_nodes"] == W.fluid_count(prob)
    chip.close()
    del r


def test_paper_d2q4_scalar_lattice():
    """w0 = 0: the paper's D2Q4 scalar lattice (Eq. cdeequilibrium)."""
    prob = W.config_small()
    prob["w0"] = 0.0
    chip = lbm.Chip.from_problem(prob)
    chip.set_valve_schedule(prob["period"], prob["states"])
    ref = oracle.from_problem(prob)
    chip.step(600)
    ref.run(600, lambda t: W.valve_word(prob, t))
    du, dC, dm = _field_errors(prob, chip, ref)
    assert du <= U_TOL and dC <= C_TOL and dm <= MASS_TOL, (du, dC, dm)
    chip.close()


def test_closed_chip_conserves_mass():
    """All valves closed: total mass and scalar are constant (FP32 storage,
    FP64 sums)."""
    prob, init = W.random_case(21, 200, 40)
    chip = lbm.Chip.from_problem(prob)
    chip.init_equilibrium(**init)
    chip.set_valves(0)
    chip.step(1)
    d0 = chip.diagnostics()
    chip.step(2000)
    d1 = chip.diagnostics()
    assert abs(d1[0] - d0[0]) / d0[0] < 1e-6
    assert abs(d1[1] - d0[1]) / d0[1] < 1e-5
    chip.close()


def test_schedule_equals_manual_valves_and_is_deterministic():
    prob = W.config_small()
    a = lbm.Chip.from_problem(prob)
    a.set_valve_schedule(7, [1, 2, 3, 0])
    a.step(50)
    b = lbm.Chip.from_problem(prob)
    for t in range(50):
        b.set_valves([1, 2, 3, 0][(t // 7) % 4])
        b.step(1)
    fa, ga = a.populations()
    fb, gb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    assert np.array_equal(a.diagnostics(), b.diagnostics())
    a.close()
    b.close()


def test_save_load_resumes_bit_exactly():
    prob = W.config_small()
    a = lbm.Chip.from_problem(prob)
    a.set_valve_schedule(prob["period"], prob["states"])
    a.step(480)
    blob = a.save_state()
    a.step(40)
    b = lbm.Chip.from_problem(prob)
    b.load_state(blob)
    assert b.step_count() == 480
    b.step(40)
    fa, ga = a.populations()
    fb, gb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    a.close()
    b.close()


def test_numeric_error_is_flagged_and_cleared():
    prob = W.config_small()
    chip = lbm.Chip.from_problem(prob)
    f, g = chip.populations()
    f[0, 5, 40] = np.nan
    chip.set_populations(f, g)
    chip.step(1)
    with pytest.raises(lbm.LbmError) as ei:
        chip.diagnostics()
    assert ei.value.status == lbm.LBM_ERR_NUMERIC
    chip.init_equilibrium(1.0, 0.0, 0.0, 0.0)
    chip.clear_error()
    chip.step(1)
    chip.diagnostics()
    chip.close()


def test_torch_stream_and_allocator():
    """PyTorch supplies the stream and the device memory; results are the
    same bits as with the library's own allocator on the default stream."""
    prob = W.config_small()
    s = torch.cuda.Stream()
    a = lbm.Chip.from_problem(prob, stream=s, torch_alloc=True)
    a.set_valve_schedule(prob["period"], prob["states"])
    a.step(300)
    rho_t = torch.empty((prob["ny"], prob["nx"]), device="cuda", dtype=torch.float32)
    C_t = torch.empty_like(rho_t)
    a.fields_device(rho=rho_t, C=C_t)
    s.synchronize()
    b = lbm.Chip.from_problem(prob)
    b.set_valve_schedule(prob["period"], prob["states"])
    b.step(300)
    rho, _, _, C = b.fields()
    assert np.array_equal(rho_t.cpu().numpy(), rho) and np.array_equal(C_t.cpu().numpy(), C)
    a.close()
    b.close()


def test_degenerate_single_row_channel_and_odd_widths():
    """A one-row channel (every node has walls north and south) and a
    channel that ends one node into a second tile."""
    for nx, ny in ((5, 1), (129, 3)):
        solid = np.zeros((ny, nx), np.uint8)
        ports = [dict(channel=0, side=W.WEST, x=0, y0=0, y1=ny, kind=W.VELOCITY, rho=1.0),
                 dict(channel=0, side=W.EAST, x=nx - 1, y0=0, y1=ny, kind=W.PRESSURE, rho=1.0)]
        eu = np.zeros((2, ny))
        eu[0] = 0.02
        ec = np.zeros((2, ny))
        ec[0] = 1.0
        prob = dict(solid=solid, tau=0.7, tau_c=0.6, ports=ports, edge_u=eu, edge_C=ec, u_max=0.02)
        chip = lbm.Chip.from_problem(prob)
        chip.set_valves(1)
        ref = oracle.from_problem(prob)
        chip.step(200)
        ref.step(1, 200)
        du, dC, dm = _field_errors(prob, chip, ref)
        assert du <= U_TOL and dC <= C_TOL and dm <= MASS_TOL, (nx, ny, du, dC, dm)
        chip.close()


def test_async_diagnostics_match_the_synchronous_read():
    """lbm_get_diagnostics_async queues each step's diagnostics into pinned
    host memory without waiting; after one synchronisation every row equals
    what the synchronous read gives step by step; a set error word is
    reported by lbm_synchronize."""
    prob = W.config_small()
    a = lbm.Chip.from_problem(prob)
    b = lbm.Chip.from_problem(prob)
    for c in (a, b):
        c.set_valve_schedule(3, prob["states"])
    ring = torch.zeros((6, 4), dtype=torch.float64, pin_memory=True)
    want = []
    for k in range(6):
        a.step(1)
        a.diagnostics_async(ring[k].data_ptr())
        b.step(1)
        want.append(b.diagnostics())
    a.synchronize()
    assert np.array_equal(ring.numpy(), np.array(want))
    f, g = a.populations()
    f[0, 5, 40] = np.nan
    a.set_populations(f, g)
    a.step(1)
    a.diagnostics_async(ring[0].data_ptr())
    with pytest.raises(lbm.LbmError) as ei:
        a.synchronize()
    assert ei.value.status == lbm.LBM_ERR_NUMERIC
    a.close()
    b.close()


@pytest.mark.parametrize("opts", [dict(), dict(variant=2, pipeline_stages=2, consumer_warps=3),
                                  dict(variant=4, block_threads=64), dict(variant=5), dict(precision="fp16"),
                                  dict(precision="bf16", variant=1), dict(wall_scheme=1),
                                  dict(max_blocks=5), dict(max_blocks=17), dict(variant=3, consumer_warps=1)])
def test_in_kernel_diagnostics_equal_the_reduction_launch(opts):
    """lbm_step_diagnostics: the step kernel's last block writes the totals
    of every step (into pinned host memory and into device memory); each row
    has the same bits as lbm_get_diagnostics after that step (same order of
    additions), the populations match lbm_step's, and the ticket counter is
    back at zero after every step (a second run gives the same rows).  The
    register and asynchronous-copy variants fold in the kernel (grids of 5
    and 17 blocks included); the bulk-copy, pipeline and pair variants, the
    paper's walls and blocks of fewer than 128 threads take the totals from
    the reduction kernel launched after each step instead."""
    prob, init = W.random_case(41, 300, 48, solid_frac=0.1)
    prob["states"] = [1, 2, 3, 0]
    a = lbm.Chip.from_problem(prob, **opts)
    b = lbm.Chip.from_problem(prob, **opts)
    for c in (a, b):
        c.init_equilibrium(**init)
        c.set_valve_schedule(4, prob["states"])
    n = 12
    host = torch.zeros((n, 4), dtype=torch.float64, pin_memory=True)
    dev = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
    a.step_diagnostics(n // 2, host.data_ptr())
    a.step_diagnostics(n - n // 2, host[n // 2].data_ptr())
    want = []
    for k in range(n):
        b.step(1)
        want.append(b.diagnostics())
    a.synchronize()
    assert np.array_equal(host.numpy(), np.array(want))
    fa, ga = a.populations()
    fb, gb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    a.step_diagnostics(n, dev.data_ptr())
    for k in range(n):
        b.step(1)
        want[k] = b.diagnostics()
    a.synchronize()
    assert np.array_equal(dev.cpu().numpy(), np.array(want))
    a.step_diagnostics(0, 0)  # no steps: out is not touched
    pageable = np.zeros(8)
    with pytest.raises(lbm.LbmError) as ei:
        a.step_diagnostics(2, pageable.ctypes.data)
    assert ei.value.status == lbm.LBM_ERR_ARG
    with pytest.raises(lbm.LbmError):
        a.step_diagnostics(1, 0)
    assert a.step_count() == 2 * n
    a.close()
    b.close()


def test_diagnostics_over_more_than_1024_block_partials():
    """Blocks of two warps on a 512 x 600 lattice of about 2400 tiles: a grid
    of more than 1024 blocks, whose partials the reduction adds in two rounds
    per thread.  The totals after three steps agree with the oracle's
    diagnostics, and the rows of lbm_step_diagnostics (the reduction kernel
    after each step, for blocks of fewer than 128 threads) have the bits of
    lbm_get_diagnostics."""
    prob, init = W.random_case(43, 512, 600, solid_frac=0.05)
    a = lbm.Chip.from_problem(prob, variant=1, block_threads=64)
    assert a.info()["grid"] > 1024
    b = lbm.Chip.from_problem(prob, variant=1, block_threads=64)
    ref = oracle.from_problem(prob)
    states = prob["states"]
    for c in (a, b, ref):
        c.init_equilibrium(**init)
    for c in (a, b):
        c.set_valve_schedule(1, states)
    rows = torch.zeros((3, 4), dtype=torch.float64, device="cuda")
    a.step_diagnostics(3, rows.data_ptr())
    want = []
    for t in range(3):
        b.step(1)
        want.append(b.diagnostics())
        ref.step(states[t])
    a.synchronize()
    assert np.array_equal(rows.cpu().numpy(), np.array(want))
    d, rd = want[-1], ref.diagnostics(states[2])
    assert abs(d[0] - rd[0]) / rd[0] < 1e-6
    assert abs(d[1] - rd[1]) <= 1e-5 * max(1.0, abs(rd[1]))
    assert abs(d[2] - rd[2]) <= 1e-5 and abs(d[3] - rd[3]) <= 1e-5
    a.close()
    b.close()


def test_misaligned_allocator_memory_is_refused(monkeypatch):
    """A caller's allocator that returns memory off the 256-byte boundary:
    lbm_create hands every such pointer straight back and fails with
    LBM_ERR_OOM before any kernel runs on it."""
    held = {}

    def _alloc(nbytes, user):
        base = torch.cuda.caching_allocator_alloc(int(nbytes) + 256)
        held[base + 16] = base
        return base + 16

    def _free(ptr, nbytes, user):
        torch.cuda.caching_allocator_delete(held.pop(int(ptr)))

    hooks = (lbm.ALLOC_FN(_alloc), lbm.FREE_FN(_free))
    monkeypatch.setattr(lbm, "_torch_hooks", lambda device: hooks)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Chip.from_problem(W.config_small(), torch_alloc=True)
    assert ei.value.status == lbm.LBM_ERR_OOM
    assert not held  # every pointer went back to the caller's free


@pytest.mark.parametrize("opts", [dict(), dict(multi_step=8), dict(precision="fp16")])
def test_zero_steps_change_nothing(opts):
    """lbm_step(0) and lbm_scalar_step(0) are no-ops: same stored bytes,
    same step count, same diagnostics."""
    prob = W.config_small()
    chip = lbm.Chip.from_problem(prob, **opts)
    chip.set_valve_schedule(prob["period"], prob["states"])
    chip.step(3)
    before, d0 = chip.save_state(), chip.diagnostics()
    chip.step(0)
    if opts.get("precision", "fp32") == "fp32":
        chip.scalar_step(0, 1.0)
    assert chip.save_state() == before and chip.step_count() == 3
    assert np.array_equal(chip.diagnostics(), d0)
    chip.close()


@pytest.mark.parametrize("nx,ny", [(524160, 3), (4, 131071)])
def test_largest_width_and_height(nx, ny):
    """The largest lattices the tile encoding admits (524160 columns, the
    last tile starting at column 524032; 2^17 - 1 rows): a closed box (every edge a wall) from
    random fields near rest, two steps, every population against the
    oracle.  Exercises the last segment index and the last row in the tile
    table, the row clamping at both edges and the halos at the last
    segment."""
    r = W.rng(77)
    prob = {"solid": np.zeros((ny, nx), np.uint8), "tau": 0.7, "tau_c": 0.6, "ports": [],
            "edge_u": np.zeros((2, ny)), "edge_C": np.zeros((2, ny)), "w0": 1.0 / 3.0, "u_max": 0.05}
    init = {"rho": 1.0 + 0.01 * (r.random((ny, nx)) - 0.5), "ux": 0.04 * (r.random((ny, nx)) - 0.5),
            "uy": 0.04 * (r.random((ny, nx)) - 0.5), "C": r.random((ny, nx))}
    chip = lbm.Chip.from_problem(prob)
    ref = oracle.from_problem(prob)
    chip.init_equilibrium(**init)
    ref.init_equilibrium(**init)
    for _ in range(2):
        chip.step(1)
        ref.step(0)
    f, g = chip.populations()
    rf, rg = _oracle_pops(ref)
    assert np.abs(f - rf).max() <= POP_ATOL and np.abs(g - rg).max() <= POP_ATOL
    chip.close()
