"""The gradient workload (a 1024 x 512 chip, 4000 coupled FP32 steps with two
valve toggles, checkpoints every 250 steps) and its 128 x 64 copy: the GPU
adjoint (lbm_adjoint) against central finite differences of the GPU's own
forward runs.

Parameters: tau_c, the inlet amplitude u_max (the parabolic inlet profile is
linear in it) and the top inlet's per-row held concentrations C_in, a vector
drawn uniformly from [0.8, 1.0) with a fixed seed.  The objective is the
squared mismatch between the final concentration profile along y at the
chamber's centre column and a linear target from 0 (bottom) to 1 (top).

Finite differences.  A central difference D(h) = (J(p + h) - J(p - h)) / 2h
carries a truncation error of about h^2 J''' / 6.  J depends on tau_c through
the diffusivity (tau_c - 1/2) / 3, which changes on the scale
tau_c - 1/2 = 0.01, so at h = 1e-3 that error is about 3% for dJ/dtau_c (the
FP64 oracle on the 128 x 64 copy: D(1e-3) = -10.830 against the exact
-10.528).  Every derivative is therefore compared with the Richardson
extrapolation (4 D(h/2) - D(h)) / 3 of the central differences at h = 1e-3
and h/2, which removes the h^2 term, within 1e-3 relative; the plain
D(1e-3) must agree within 1e-3 plus its own truncation error, estimated as
(4/3) |D(h) - D(h/2)|.

The forward runs are FP32, so J itself carries rounding noise; between two
runs whose inputs differ slightly it is about 2e-6 on these workloads
(measured: the C_in differences below at h = 1e-3 and h/2 scatter by 1e-3
around the exact value), i.e. about 1e-3 in D(1e-3).  That is small next to
dJ/dtau_c and dJ/du_max (10 to 180 here) but not next to a C_in derivative
(0.017 to 0.4 on the copy).  J is exactly quadratic in C_in, though: for a
given flow the scalar lattice is linear in its populations and affine in the
held concentrations, so C at the objective is affine in C_in and a central
difference is exact at any step.  The C_in rows therefore take the step
H_CIN = 0.5, where the noise is 2e-6 relative to the differences in J; the
differences at h = 1e-3 are printed beside them.

The full-size chip starts the 4000-step window from the state a spin-up of
SPINUP steps from rest leaves: from rest, the scalar front advances about
100 nodes in 4000 steps and stays 300 nodes short of the chamber, so every
derivative of the chamber objective would be zero to working precision.
The window ends (step 30000) before the compound reaches the outlets: at
tau_c = 0.51 the scalar's do-nothing outlet does not stay bounded once it
carries compound (the FP64 oracle on this chip: max C 1.09 at step 30000,
1e15 at 35000, growing from the outlet column next to the channel walls).
Within any 4000-step window a change at the inlet travels at most about 160
nodes (u_max = 0.04), so dJ/dC_in is zero on this chip: the adjoint gives
zero and the differences give zero, which the test checks as such; the
128 x 64 copy, whose chamber is 51 nodes from the inlet, checks the C_in
derivatives with non-zero values.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1307_4703_gb300 import lbm, workloads as W  # noqa: E402

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

H = 1e-3        # finite-difference step (tau_c, u_max)
H_CIN = 0.5     # step of the C_in rows, on which J depends quadratically
GRAD_TOL = 1e-3  # relative
SPINUP = 26000   # steps from rest before the window of the full-size chip


def _objective(prob):
    cx0, cx1, cy0, cy1 = prob["chamber"]
    oy = np.arange(cy0, cy1)
    ox = np.full_like(oy, (cx0 + cx1) // 2)
    return ox, oy, ((oy - cy0) / max(1, cy1 - 1 - cy0)).astype(float), np.ones(len(oy))


def _J(prob, blob, n, obj):
    """J after n steps of the chip of `prob` from the saved state `blob`
    (None: from rest with the problem's valve schedule)."""
    ox, oy, tg, wt = obj
    with lbm.Chip.from_problem(prob) as c:
        if blob is None:
            c.set_valve_schedule(prob["period"], prob["states"])
        else:
            c.load_state(blob)
        c.step(n)
        C = c.fields()[3].astype(np.float64)
    assert np.abs(C).max() < 2.0  # the run stayed in the stable regime (see SPINUP)
    return float((wt * (C[oy, ox] - tg) ** 2).sum())


def _perturbations(prob, rows):
    def tau(p, d):
        q = dict(p)
        q["tau_c"] = p["tau_c"] + d
        return q

    def umax(p, d):
        q = dict(p)
        q["edge_u"] = p["edge_u"] * ((p["u_max"] + d) / p["u_max"])
        return q

    def cin(r):
        def f(p, d):
            q = dict(p)
            q["edge_C"] = p["edge_C"].copy()
            q["edge_C"][W.WEST, r] += d
            return q
        return f

    return [("tau_c", tau), ("u_max", umax)] + [("C_in[%d]" % r, cin(r)) for r in rows]


def _D(prob, blob, n, obj, perturb, h):
    """Central difference at step h."""
    return (_J(perturb(prob, h), blob, n, obj) - _J(perturb(prob, -h), blob, n, obj)) / (2 * h)


def _differences(prob, blob, n, obj, perturb):
    """Central differences at h and h/2."""
    return _D(prob, blob, n, obj, perturb, H), _D(prob, blob, n, obj, perturb, H / 2)


def _check_cin(name, adj, prob, blob, n, obj, perturb, zero_scale=None):
    """A C_in row: the adjoint against the (exact) central difference at
    H_CIN; zero_scale set: the derivative is zero, within the FP32 noise."""
    d = _D(prob, blob, n, obj, perturb, H_CIN)
    d3 = _D(prob, blob, n, obj, perturb, H)
    print("%-10s adjoint %.8g  D(%.1f) %.8g  rel %.2e  (D(1e-3) %.8g)"
          % (name, adj, H_CIN, d, abs(adj - d) / max(abs(adj), 1e-300), d3))
    if zero_scale is None:
        assert abs(adj - d) <= GRAD_TOL * abs(adj), (name, adj, d)
    else:
        assert abs(adj) <= 1e-9 * zero_scale and abs(d) <= 1e-6 * zero_scale, (name, adj, d)


def _adjoint_values(prob, got, rows):
    J, dt, du, dc = got
    return [dt, float((du * prob["edge_u"]).sum() / prob["u_max"])] + [float(dc[W.WEST, r]) for r in rows]


def _check_against_differences(name, adj, dh, dh2):
    rich = (4 * dh2 - dh) / 3
    trunc = 4.0 / 3.0 * abs(dh - dh2)
    print("%-10s adjoint %.8g  D(h) %.8g  D(h/2) %.8g  Richardson %.8g  rel %.2e (D(h): %.2e)"
          % (name, adj, dh, dh2, rich, abs(adj - rich) / max(abs(adj), 1e-300), abs(adj - dh) / max(abs(adj), 1e-300)))
    assert abs(adj - rich) <= GRAD_TOL * abs(adj), (name, adj, rich, dh, dh2)
    assert abs(adj - dh) <= GRAD_TOL * abs(adj) + trunc, (name, adj, dh, trunc)
    return rich


def test_gradient_chip_against_central_differences():
    """1024 x 512, 4000 steps from the spun-up state, checkpoints every 250
    steps: dJ/dtau_c and dJ/du_max against central differences (h = 1e-3,
    with Richardson extrapolation against h/2); five C_in rows, whose
    derivatives are zero on this chip, both ways."""
    prob = W.config_adjoint_chip()
    n = prob["steps"]
    obj = _objective(prob)
    rows = prob["c_in_rows"][[0, 25, 50, 75, 99]]
    with lbm.Chip.from_problem(prob) as c:
        c.set_valve_schedule(prob["period"], prob["states"])
        c.step(SPINUP)
        blob = c.save_state()
        # the window holds two valve toggles
        words = [W.valve_word(prob, SPINUP + t) for t in range(n)]
        assert sum(words[t] != words[t - 1] for t in range(1, n)) == 2
        got = c.adjoint(n, *obj, ckpt_every=250)
    adj = _adjoint_values(prob, got, rows)
    J0 = _J(prob, blob, n, obj)
    print("chip-1024x512 window %d..%d: J %.9g, adjoint dJ/dtau_c %.6g dJ/du_max %.6g dJ/dC_in %s"
          % (SPINUP, SPINUP + n, got[0], adj[0], adj[1], adj[2:]))
    assert abs(got[0] / J0 - 1) < 1e-6
    # the spun-up state puts compound at the chamber's centre column
    assert abs(adj[0]) > 1e-4 and abs(adj[1]) > 1e-4, adj
    scale = max(abs(adj[0]), abs(adj[1]))
    for (name, perturb), a in zip(_perturbations(prob, rows), adj):
        if name.startswith("C_in"):
            # no inlet change reaches the chamber within the window
            _check_cin(name, a, prob, blob, n, obj, perturb, zero_scale=scale)
        else:
            dh, dh2 = _differences(prob, blob, n, obj, perturb)
            _check_against_differences(name, a, dh, dh2)


def test_gradient_copy_128x64_against_central_differences():
    """The 128 x 64 copy from rest, 4000 steps, checkpoints every 250 steps:
    every derivative is non-zero here, the C_in rows included."""
    prob = W.config_adjoint_chip(128, 64)
    n = prob["steps"]
    obj = _objective(prob)
    rows = prob["c_in_rows"][[0, 3, 6, 9, 11]]
    with lbm.Chip.from_problem(prob) as c:
        c.set_valve_schedule(prob["period"], prob["states"])
        got = c.adjoint(n, *obj, ckpt_every=250)
    adj = _adjoint_values(prob, got, rows)
    assert abs(got[0] / _J(prob, None, n, obj) - 1) < 1e-6
    assert min(abs(a) for a in adj) > 1e-3, adj
    for (name, perturb), a in zip(_perturbations(prob, rows), adj):
        if name.startswith("C_in"):
            _check_cin(name, a, prob, None, n, obj, perturb)
        else:
            dh, dh2 = _differences(prob, None, n, obj, perturb)
            _check_against_differences(name, a, dh, dh2)
