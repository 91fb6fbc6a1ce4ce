"""Unit conversion against the values the paper prints (Tables 1-3 and the
conversion section), stored in tests/golden/paper_tables.json."""
import json
import os

import pytest

from paper_1307_4703_gb300 import units

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def _close(a, b, rel=1e-9):
    return abs(a - b) <= rel * max(abs(a), abs(b))


def test_table1_fluid_parameters():
    t = GOLDEN["table1_fluid"]
    s = GOLDEN["section_choice_of_parameters"]
    c = units.Conversion.from_resolution(t["L_phys_um"], t["L_lb"], t["U_phys_um_s"], t["U_lb"])
    assert _close(c.dx, s["dx_um"]) and _close(c.dt, s["dt_fluid_s"])
    assert _close(c.viscosity(t["nu_phys_um2_s"]), t["nu_lb"])
    assert _close(c.steps(t["T_phys_s"]), t["T_lb"])
    assert _close(c.velocity(t["U_phys_um_s"]), t["U_lb"])
    assert _close(units.reynolds(t["L_lb"], t["U_lb"], t["nu_lb"]), s["Re"])
    assert _close(units.reynolds(t["L_phys_um"], t["U_phys_um_s"], t["nu_phys_um2_s"]), s["Re"])
    assert _close(units.tau_fluid(t["nu_lb"]), 0.65)


def test_table2_cde_parameters():
    t = GOLDEN["table2_cde"]
    s = GOLDEN["section_choice_of_parameters"]
    c = units.Conversion.from_resolution(t["L_phys_um"], t["L_lb"], t["U_phys_um_s"], t["U_lb"])
    assert _close(c.dt, s["dt_cde_s"])
    assert _close(c.diffusivity(t["D_phys_um2_s"]), t["D_lb"])
    assert _close(c.rate(t["k_phys_per_s"]), t["k_lb"])
    assert _close(c.steps(t["T_phys_s"]), t["T_lb"])
    pe = units.peclet(t["L_lb"], t["U_lb"], t["D_lb"])
    assert _close(pe, units.peclet(t["L_phys_um"], t["U_phys_um_s"], t["D_phys_um2_s"]))
    assert abs(pe - s["Pe_approx"]) / s["Pe_approx"] < 0.01
    # the paper's D2Q4 lattice: D = (2 tau - 1) / 4
    tau = units.tau_scalar(t["D_lb"], w0=0.0)
    assert _close((2 * tau - 1) / 4, t["D_lb"])
    # the fluid field of Table 1 read with the CDE time step
    f = GOLDEN["table1_fluid"]
    assert _close(units.rescale_velocity(f["U_lb"], s["dt_fluid_s"], s["dt_cde_s"]), t["U_lb"])


@pytest.mark.parametrize("case", ["a", "b", "c", "d"])
def test_table3_step_advection_parameters(case):
    t = GOLDEN["table3_step_advection"][case]
    c = units.Conversion(t["dx_um"], t["dt_s"])
    assert _close(c.velocity(t["U_phys_um_s"]), t["U_lb"])
    assert _close(c.diffusivity(t["D_phys_um2_s"]), t["D_lb"])
    assert _close(c.velocity_phys(t["U_lb"]), t["U_phys_um_s"])
    pe = units.peclet(20, t["U_lb"], t["D_lb"])
    s = GOLDEN["section_choice_of_parameters"]
    ref = s["Pe_approx"] if t["U_phys_um_s"] == 5000.0 else s["Pe_low_approx"]
    assert abs(pe - ref) / ref < 0.03
