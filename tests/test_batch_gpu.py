"""Batches of independent chips in one launch (lbm_create_batch).

Stacked with a solid row between neighbours, each chip sees exactly the
links, ports and relaxation rates it has alone, and every node's update uses
the same FP32 operations on the same operands, so a chip in a batch must
match the same chip run alone bit for bit (and therefore the oracle as
closely as a single chip does)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1307_4703_gb300 import lbm, workloads as W  # noqa: E402

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1307_4703_gb300 import build
    build.build()
    lbm.load()


def _instance_pops(chip, k, f, g):
    i = chip.instance(k)
    sl = (slice(None), slice(i["row0"], i["row0"] + i["ny"]), slice(0, i["nx"]))
    return f[sl], g[sl]


def _mixed_chips():
    """Random obstacle lattices of different sizes and relaxation times
    (every port kind), plus two chip workloads of different shapes."""
    chips, inits = [], []
    for seed, nx, ny in ((3, 40, 24), (8, 150, 20), (11, 300, 12)):
        prob, init = W.random_case(seed, nx, ny)
        prob["tau"] = 0.6 + 0.05 * seed
        prob["tau_c"] = 0.52 + 0.01 * seed
        chips.append(prob)
        inits.append(init)
    for prob in W.config_batch(2, seed=5):
        chips.append(prob)
        inits.append(None)
    return chips, inits


@pytest.mark.parametrize("opts", [dict(), dict(variant=1), dict(variant=3), dict(variant=5), dict(precision="fp16"),
                                  dict(precision="bf16", variant=1)])
def test_batch_equals_chips_run_alone(opts):
    chips, inits = _mixed_chips()
    batch = lbm.Chip.batch(chips, **opts)
    alone = [lbm.Chip.from_problem(p, **opts) for p in chips]
    assert batch.info()["instances"] == len(chips)
    # initial states: random fields where the case has them
    rho, ux, uy, C = (np.ones((batch.ny, batch.nx)), np.zeros((batch.ny, batch.nx)),
                      np.zeros((batch.ny, batch.nx)), np.zeros((batch.ny, batch.nx)))
    for k, (c, init) in enumerate(zip(alone, inits)):
        if init is None:
            continue
        c.init_equilibrium(**init)
        i = batch.instance(k)
        sl = (slice(i["row0"], i["row0"] + i["ny"]), slice(0, i["nx"]))
        rho[sl], ux[sl], uy[sl], C[sl] = init["rho"], init["ux"], init["uy"], init["C"]
    batch.init_equilibrium(rho, ux, uy, C)
    # every chip its own valve program
    for k, (c, p) in enumerate(zip(alone, chips)):
        period = 7 + 5 * k
        c.set_valve_schedule(period, p["states"])
        batch.set_instance_schedule(k, period, p["states"])
    for c in alone:
        c.step(150)
    batch.step(150)
    f, g = batch.populations()
    for k, c in enumerate(alone):
        fa, ga = c.populations()
        fb, gb = _instance_pops(batch, k, f, g)
        fl = ~c.solid
        assert np.array_equal(fa[:, fl], fb[:, fl]), k
        assert np.array_equal(ga[:, fl], gb[:, fl]), k
    # diagnostics are totals over the chips
    d = batch.diagnostics()
    da = np.sum([c.diagnostics() for c in alone], axis=0)
    assert abs(d[0] - da[0]) <= 1e-6 * abs(da[0]) and abs(d[1] - da[1]) <= 1e-5 * max(1.0, abs(da[1]))
    batch.close()
    for c in alone:
        c.close()


def test_batch_matches_oracle_per_chip():
    """Two chip workloads in one batch, each against its own FP64 oracle run
    with its own valve period: the single-chip tolerances hold."""
    chips = W.config_batch(2, steps=600, seed=9)
    batch = lbm.Chip.batch(chips)
    for k, p in enumerate(chips):
        batch.set_instance_schedule(k, 150 + 100 * k, p["states"])
    batch.step(600)
    fields = batch.fields()
    for k, p in enumerate(chips):
        ref = oracle.from_problem(p)
        ref.run(600, lambda t, k=k, p=p: p["states"][(t // (150 + 100 * k)) % 2])
        rho, ux, uy, C = batch.instance_fields(k, fields)
        r_rho, r_ux, r_uy, r_C = ref.fields()
        fl = ~ref.solid
        du = max(np.abs(ux - r_ux)[fl].max(), np.abs(uy - r_uy)[fl].max()) / p["u_max"]
        dC = np.abs(C - r_C)[fl].max()
        dm = abs(rho[fl].astype(np.float64).sum() - r_rho[fl].sum()) / r_rho[fl].sum()
        assert du <= 1e-4 and dC <= 1e-4 and dm <= 1e-6, (k, du, dC, dm)
        assert np.all(rho[~fl] == 0)
    batch.close()


def test_batch_valve_calls():
    chips = W.config_batch(3, seed=4)
    batch = lbm.Chip.batch(chips)
    bases = [batch.instance(k)["channel_base"] for k in range(3)]
    assert bases == [0, 2, 4]
    # one valve word for every chip equals the same word set chip by chip
    other = lbm.Chip.batch(chips)
    batch.set_valves(1)
    for k in range(3):
        other.set_instance_valves(k, 1)
    batch.step(40)
    other.step(40)
    fa, ga = batch.populations()
    fb, gb = other.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    # chip 1 alone closed from the start: it stays exactly at rest while the
    # others flow
    third = lbm.Chip.batch(chips)
    third.set_valves(1)
    third.set_instance_valves(1, 0)
    third.step(200)
    fields = third.fields()
    assert np.abs(third.instance_fields(1, fields)[1]).max() == 0.0
    assert np.abs(third.instance_fields(0, fields)[1]).max() > 0.02
    assert np.abs(third.instance_fields(2, fields)[1]).max() > 0.02
    third.close()
    with pytest.raises(lbm.LbmError) as e:
        batch.adjoint(10, [5], [5], [0.0])
    assert e.value.status == lbm.LBM_ERR_STATE
    with pytest.raises(lbm.LbmError) as e:
        batch.set_instance_valves(3, 1)
    assert e.value.status == lbm.LBM_ERR_ARG
    batch.close()
    other.close()
