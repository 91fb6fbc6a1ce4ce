"""Seeded synthetic inputs for the coupled lattice Boltzmann step.

This module builds problem descriptions only: solid masks, port tables,
inlet velocity profiles, source/sink concentrations and valve schedules.  It
holds none of the method's arithmetic, so both the CUDA path and the FP64
oracle take their inputs from here.

The chip topology follows the gradient generator of Tanaka & Iber (arXiv
1307.4703, "Experimental Layout and Conditions"): two parallel channels whose
inlet and outlet valves open alternately, joined by a chamber in which the
gradient forms.  The exact drawing of the paper's Figure 1a is not part of
the paper's text, so rectangular chips of the stated proportions stand in for
it.  Every random draw uses numpy's PCG64 generator with an explicit seed.

Problem dict keys: name, nx, ny, solid (ny, nx) uint8 (1 = solid), tau,
tau_c, w0, ports (list of dicts: channel, side, x, y0, y1, kind, rho),
edge_u / edge_C ((2, ny) float64: u_x and C_in of velocity-port nodes per
side and row), period, states (valve words cycled every ``period`` steps),
steps, u_max.
"""
import numpy as np

WEST, EAST = 0, 1
VELOCITY, PRESSURE, PRESSURE_RESCALE, INLET_RESCALE = 0, 1, 2, 3
SEED = 0x1307


def rng(seed=SEED):
    return np.random.Generator(np.random.PCG64(seed))


def parabolic_profile(width, u_max):
    """Inlet u_x across a channel of ``width`` rows whose walls lie half a
    cell outside its first and last row: u = 4 u_max s (W - s) / W^2 with
    s = row + 1/2 (the developed Poiseuille profile the paper's channels
    approach, section "Results")."""
    s = np.arange(width, dtype=np.float64) + 0.5
    return 4.0 * u_max * s * (width - s) / float(width) ** 2


def valve_word(problem, t):
    """Valve word of time step t under the problem's schedule."""
    st = problem["states"]
    return int(st[(t // int(problem["period"])) % len(st)])


def two_channel_chip(nx, ny, ch_w, ch_len, chamber_w, tau, tau_c, u_max, period, steps,
                     x0=0, C_top=1.0, C_bottom=0.0, w0=1.0 / 3.0, name="chip", paper_ports=False, decay=0.0):
    """Two channels of ``ch_w`` rows along x (rows [0, ch_w) and
    [ny - ch_w, ny), columns [x0, x0 + ch_len)) joined by a chamber of
    ``chamber_w`` columns centred in the grid.  Channel 0 is the top channel
    (largest y, fed with C_top) and opens first; channel 1 is the bottom
    channel (C_bottom).  Each channel has a velocity inlet on its west end
    and a pressure outlet (rho = 1) on its east end.

    paper_ports: the paper's pressure-driven channels instead (section
    "Boundary Conditions"): a rescaling inlet at density 1 + drho / 2 holding
    C_in and a rescaling outlet at 1 - drho / 2, with drho = 3 dp and dp the
    Poiseuille pressure drop 8 nu u_max L / W^2 of a channel of length L and
    width W (section "Choice of Parameter Values").  decay: rate k of the
    compound."""
    assert 0 < ch_w and 2 * ch_w < ny and 0 <= x0 and x0 + ch_len <= nx
    solid = np.ones((ny, nx), dtype=np.uint8)
    solid[0:ch_w, x0:x0 + ch_len] = 0
    solid[ny - ch_w:ny, x0:x0 + ch_len] = 0
    cx0 = (nx - chamber_w) // 2
    solid[ch_w:ny - ch_w, cx0:cx0 + chamber_w] = 0
    edge_u = np.zeros((2, ny))
    edge_C = np.zeros((2, ny))
    prof = parabolic_profile(ch_w, u_max)
    ports = []
    drho = 3 * 8 * (tau - 0.5) / 3 * u_max * (ch_len - 1) / ch_w ** 2
    for chan, (y0, c_in) in enumerate(((ny - ch_w, C_top), (0, C_bottom))):
        if paper_ports:
            ports.append(dict(channel=chan, side=WEST, x=x0, y0=y0, y1=y0 + ch_w, kind=INLET_RESCALE,
                              rho=1.0 + drho / 2))
            ports.append(dict(channel=chan, side=EAST, x=x0 + ch_len - 1, y0=y0, y1=y0 + ch_w,
                              kind=PRESSURE_RESCALE, rho=1.0 - drho / 2))
        else:
            ports.append(dict(channel=chan, side=WEST, x=x0, y0=y0, y1=y0 + ch_w, kind=VELOCITY, rho=1.0))
            ports.append(dict(channel=chan, side=EAST, x=x0 + ch_len - 1, y0=y0, y1=y0 + ch_w,
                              kind=PRESSURE, rho=1.0))
            edge_u[WEST, y0:y0 + ch_w] = prof
        edge_C[WEST, y0:y0 + ch_w] = c_in
    return dict(name=name, nx=nx, ny=ny, solid=solid, tau=float(tau), tau_c=float(tau_c),
                w0=float(w0), ports=ports, edge_u=edge_u, edge_C=edge_C, period=int(period),
                states=[1, 2], steps=int(steps), u_max=float(u_max),
                chamber=(cx0, cx0 + chamber_w, ch_w, ny - ch_w), decay=float(decay))


def config_small():
    """256 x 128 chip: channels rows 0-15 and 112-127 over x = 0..255, chamber
    x = 96..159; tau = 0.8, tau_c = 0.55, u_max = 0.05, valves toggle every
    500 steps, 2000 steps."""
    return two_channel_chip(256, 128, 16, 256, 64, 0.8, 0.55, 0.05, 500, 2000, name="chip-256x128")


def config_full_chip(tau_c=0.51):
    """1024 x 768 chip at 1 um per cell: channels 100 rows wide over
    x = 0..999 (columns 1000-1023 solid), chamber 200 columns wide spanning
    rows 100..667; tau = 0.6, u_max = 0.04, valve period 2000 steps."""
    return two_channel_chip(1024, 768, 100, 1000, 200, 0.6, tau_c, 0.04, 2000, 200000,
                            name="chip-1024x768")


def config_large_chip(nx=4096, ny=2048, tau_c=0.51, steps=50000):
    """The 1024 x 768 chip scaled to 4096 x 2048 (x by 4, y by 8/3): channels
    267 rows wide over x = 0..3999, chamber 800 columns wide.  Other sizes
    keep the same proportions (used for downscaled copies)."""
    ch_w = int(round(ny * 267 / 2048))
    ch_len = int(round(nx * 4000 / 4096))
    cw = int(round(nx * 800 / 4096))
    return two_channel_chip(nx, ny, ch_w, ch_len, cw, 0.6, tau_c, 0.04, 2000, steps,
                            name="chip-%dx%d" % (nx, ny))


def config_adjoint_chip(nx=1024, ny=512, seed=SEED):
    """1024 x 512 chip for the gradient workload: channels rows 0..99 and
    412..511 over x = 0..999, chamber 200 wide; tau = 0.6, tau_c = 0.51,
    u_max = 0.04, valve period 1500 (two toggles in 4000 steps), 4000
    steps.  The top inlet holds a per-row concentration vector drawn
    uniformly from [0.8, 1.0) with PCG64 (``seed``), one entry per inlet row
    (100 on this chip); its rows are ``c_in_rows``.  Other sizes keep the
    proportions (the 128 x 64 copy: channels 12 rows wide and 125 long,
    chamber 25 wide, the first 12 draws of the same vector)."""
    ch_w = int(round(ny * 100 / 512))
    ch_len = int(round(nx * 1000 / 1024))
    cw = int(round(nx * 200 / 1024))
    prob = two_channel_chip(nx, ny, ch_w, ch_len, cw, 0.6, 0.51, 0.04, 1500, 4000,
                            name="chip-%dx%d" % (nx, ny))
    top = [p for p in prob["ports"] if p["channel"] == 0 and p["side"] == WEST][0]
    rows = np.arange(top["y0"], top["y1"])
    prob["edge_C"][WEST, rows] = rng(seed).uniform(0.8, 1.0, size=len(rows))
    prob["c_in_rows"] = rows
    return prob


def channel_flow_fields(problem):
    """Stand-in stationary velocity fields of a two-channel chip, one per
    valve word of its schedule, for the scalar-only workflow of the paper
    (section "Results": the flow of each valve state is computed once and
    stored, and the compound is advanced on it): every open channel carries
    its inlet's parabolic profile u_x(y) unchanged from its inlet column to
    its outlet column; the closed channel and the chamber are at rest.
    Returns {valve word: (ux, uy)} of (ny, nx) arrays."""
    ny, nx = problem["ny"], problem["nx"]
    eu = np.asarray(problem["edge_u"], np.float64)
    out = {}
    for word in sorted(set(int(w) for w in problem["states"])):
        ux = np.zeros((ny, nx))
        for p in problem["ports"]:
            if p["side"] != WEST or p["kind"] != VELOCITY or not (word >> p["channel"]) & 1:
                continue
            east = [q for q in problem["ports"] if q["channel"] == p["channel"] and q["side"] == EAST]
            x1 = east[0]["x"] if east else nx - 1
            ux[p["y0"]:p["y1"], p["x"]:x1 + 1] = eu[WEST, p["y0"]:p["y1"], None]
        ux[np.asarray(problem["solid"]) != 0] = 0.0
        out[word] = (ux, np.zeros((ny, nx)))
    return out


def config_batch(n=64, steps=10000, seed=SEED):
    """``n`` independent two-channel chips for the batched step, drawn with
    PCG64: nx uniform over the multiples of 64 in [256, 1024], ny = nx / 2,
    channels ny / 8 rows wide over the full length, chamber centred with a
    width uniform in [40, 200] (at most nx / 2), tau = 0.8, u_max = 0.05,
    tau_c uniform in [0.505, 0.6), valve period uniform in [250, 4000]."""
    r = rng(seed)
    chips = []
    for k in range(n):
        nx = 64 * int(r.integers(4, 17))
        ny = nx // 2
        cw = min(int(r.integers(40, 201)), nx // 2)
        tau_c = float(r.uniform(0.505, 0.6))
        period = int(r.integers(250, 4001))
        chips.append(two_channel_chip(nx, ny, ny // 8, nx, cw, 0.8, tau_c, 0.05, period, steps,
                                      name="batch-%d-%dx%d" % (k, nx, ny)))
    return chips


STEP_ADVECTION_CASES = {  # Table 3: (U_lb, D_lb, T_phys / dt)
    "a": (0.5, 0.00244, 400),
    "b": (0.05, 0.000244, 4000),
    "c": (0.1, 0.00244, 2000),
    "d": (0.01, 0.000244, 20000),
}


def step_advection(case, length=400, width=20):
    """The step-profile advection test of Table 3 (cases a-d): a straight
    channel `width` nodes wide (the paper resolves the 100 um channel by 20
    nodes) between halfway walls, at rest with C = 0, opened at t = 0 with a
    prescribed-density inlet holding C = 1 (the paper's rescaling inlet) and
    a do-nothing outlet.  The stored velocity field is the Poiseuille
    profile u(s) = 4 U s (W - s) / W^2 (s = y + 1/2) with the case's maximal
    speed U, standing in for the pre-computed channel flow; the scalar runs
    on the paper's D2Q4 lattice (w0 = 0) with tau_g = 2 D + 1/2.  Every case
    advects the front 200 nodes."""
    U, D, steps = STEP_ADVECTION_CASES[case]
    ny, nx = width, length
    solid = np.zeros((ny, nx), dtype=np.uint8)
    edge_u = np.zeros((2, ny))
    edge_C = np.zeros((2, ny))
    edge_C[WEST, :] = 1.0
    ports = [dict(channel=0, side=WEST, x=0, y0=0, y1=ny, kind=INLET_RESCALE, rho=1.0),
             dict(channel=0, side=EAST, x=nx - 1, y0=0, y1=ny, kind=PRESSURE_RESCALE, rho=1.0)]
    s = np.arange(ny) + 0.5
    ux = np.repeat((4 * U * s * (ny - s) / ny ** 2)[:, None], nx, axis=1)
    return dict(name="step-advection-%s" % case, nx=nx, ny=ny, solid=solid, tau=0.8,
                tau_c=float(2 * D + 0.5), w0=0.0, ports=ports, edge_u=edge_u, edge_C=edge_C,
                period=int(steps), states=[1], steps=int(steps), u_max=float(U), D=float(D),
                velocity=(ux, np.zeros((ny, nx))))


def has_isolated_fluid(solid):
    """True when some fluid cell has no fluid cell among its 8 neighbours
    inside the grid (such masks are rejected by the library)."""
    fl = np.asarray(solid) == 0
    ny, nx = fl.shape
    pad = np.zeros((ny + 2, nx + 2), dtype=bool)
    pad[1:-1, 1:-1] = fl
    nb = np.zeros_like(fl)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dx or dy:
                nb |= pad[1 + dy:ny + 1 + dy, 1 + dx:nx + 1 + dx]
    return bool(np.any(fl & ~nb))


def random_case(seed, nx, ny, solid_frac=0.2, paper_ports=False, decay=0.0):
    """A small lattice with every kind of node: random solid obstacles, one
    port of each (side, kind) pair on three valve channels, random inlet
    profiles and concentrations, and random initial fields near rest.

    Returns (problem, init) where init = dict(rho, ux, uy, C) of (ny, nx)
    arrays, and problem["states"] holds a random valve word per step
    (period 1).  paper_ports: the velocity ports become the paper's
    rescaling inlets and the pressure ports its rescaling outlets (the same
    random draws otherwise).  decay: rate k of the compound."""
    r = rng(seed)
    assert nx >= 4 and ny >= 8
    solid = (r.random((ny, nx)) < solid_frac).astype(np.uint8)
    # ports: rows split into bands; each band is a port on the west or east edge
    h = ny // 4
    bands = [(0, h), (h, 2 * h), (2 * h, 3 * h), (3 * h, ny)]
    ports = []
    edge_u = np.zeros((2, ny))
    edge_C = np.zeros((2, ny))
    specs = [(0, WEST, VELOCITY, bands[0]), (0, EAST, PRESSURE, bands[1]),
             (1, EAST, VELOCITY, bands[2]), (1, WEST, PRESSURE, bands[3]),
             (2, WEST, VELOCITY, bands[2]), (2, EAST, PRESSURE, bands[0])]
    for chan, side, kind, (y0, y1) in specs:
        y0 = y0 + (1 if y1 - y0 > 2 else 0)
        x = 0 if side == WEST else nx - 1
        solid[y0:y1, x] = 0
        solid[y0:y1, x + (1 if side == WEST else -1)] = 0
        ports.append(dict(channel=chan, side=side, kind=kind if not paper_ports else
                          (INLET_RESCALE if kind == VELOCITY else PRESSURE_RESCALE), x=x, y0=y0, y1=y1,
                          rho=float(1.0 + 0.01 * (r.random() - 0.5))))
        if kind == VELOCITY:
            sgn = 1.0 if side == WEST else -1.0
            edge_u[side, y0:y1] = sgn * 0.04 * r.random(y1 - y0)
            edge_C[side, y0:y1] = r.random(y1 - y0)
    # drop isolated fluid cells (never port nodes, which have a fluid neighbour)
    while has_isolated_fluid(solid):
        fl = solid == 0
        pad = np.zeros((ny + 2, nx + 2), dtype=bool)
        pad[1:-1, 1:-1] = fl
        nb = np.zeros_like(fl)
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dx or dy:
                    nb |= pad[1 + dy:ny + 1 + dy, 1 + dx:nx + 1 + dx]
        solid[fl & ~nb] = 1
    init = dict(rho=1.0 + 0.01 * (r.random((ny, nx)) - 0.5),
                ux=0.03 * (r.random((ny, nx)) - 0.5),
                uy=0.03 * (r.random((ny, nx)) - 0.5),
                C=r.random((ny, nx)))
    states = [int(s) for s in r.integers(0, 8, size=64)]
    prob = dict(name="random-%dx%d-s%d" % (nx, ny, seed), nx=nx, ny=ny, solid=solid,
                tau=float(0.55 + 0.5 * r.random()), tau_c=float(0.52 + 0.5 * r.random()),
                w0=1.0 / 3.0, ports=ports, edge_u=edge_u, edge_C=edge_C, period=1,
                states=states, steps=len(states), u_max=0.04, decay=float(decay))
    return prob, init


def fluid_count(problem):
    return int(np.count_nonzero(np.asarray(problem["solid"]) == 0))
