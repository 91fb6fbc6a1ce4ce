"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
function ``include/lbm.h`` declares, and rejects invalid arguments before it
touches the device (so these checks run on a CPU-only machine)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1307_4703_gb300 import build, lbm, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return lbm.load()


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(lbm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("lbm_create", "lbm_set_valves", "lbm_step", "lbm_get_fields", "lbm_destroy"):
        assert required in names
    assert names == set(lbm.SIGNATURES), names ^ set(lbm.SIGNATURES)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_library_is_built_for_sm_103a_only():
    src = open(os.path.join(ROOT, "paper_1307_4703_gb300", "build.py")).read()
    assert "arch=compute_103a,code=sm_103a" in src


def _create(lib, nx, ny, mask, tau=0.8, tau_c=0.6, ports=(), edge_u=None, edge_C=None, opt=None):
    parr = (lbm.lbm_port * max(1, len(ports)))()
    for k, p in enumerate(ports):
        parr[k] = lbm.lbm_port(*p)
    h = ctypes.c_void_p()
    eu = None if edge_u is None else np.ascontiguousarray(edge_u, np.float32)
    ec = None if edge_C is None else np.ascontiguousarray(edge_C, np.float32)
    st = lib.lbm_create(ctypes.byref(h), nx, ny,
                        None if mask is None else np.ascontiguousarray(mask, np.uint8).ctypes.data_as(lbm._u8p),
                        tau, tau_c, len(ports), parr,
                        None if eu is None else eu.ctypes.data_as(lbm._f32p),
                        None if ec is None else ec.ctypes.data_as(lbm._f32p),
                        None if opt is None else ctypes.byref(opt))
    return st, lib.lbm_last_error(None).decode()


@pytest.mark.parametrize("case,needle", [
    (dict(tau=0.5), "relaxation time"),
    (dict(tau_c=0.4), "scalar relaxation"),
    (dict(tau=float("nan")), "relaxation time"),
    (dict(mask="none"), "mask is NULL"),
    (dict(mask="allsolid"), "no fluid"),
    (dict(mask="isolated"), "no fluid neighbour"),
    (dict(nx=0), "empty"),
    (dict(ports=[(0, 0, 0, 0, 4, 0, 1.0)]), "need edge_u"),
    (dict(ports=[(0, 0, 3, 0, 4, 1, 1.0)]), "outside the port is fluid"),
    (dict(ports=[(40, 0, 0, 0, 4, 1, 1.0)]), "channel"),
    (dict(ports=[(0, 0, 0, 0, 4, 1, -1.0)]), "pressure density"),
    (dict(ports=[(0, 0, 0, 0, 4, 1, 1.0), (1, 0, 0, 2, 6, 1, 1.0)]), "already has a port"),
    (dict(ports=[(0, 2, 0, 0, 4, 1, 1.0)]), "side"),
    (dict(ports=[(0, 0, 0, 0, 99, 1, 1.0)]), "outside the grid"),
    (dict(opt="badsize"), "struct_size"),
    (dict(opt="badblock"), "block_threads"),
    (dict(opt="badprecision"), "precision = 3"),
    (dict(opt="fp16pipe"), "variants 1, 2 and 4"),
    (dict(opt="wallpipe"), "runs variants 1 and 2"),
    (dict(opt="badwall"), "wall_scheme = 2"),
    (dict(opt="badscalar"), "scalar_variant = 3"),
    (dict(nx=524161, mask="wide"), "too large"),
    (dict(opt="multifp16"), "multi_step needs FP32"),
    (dict(opt="badmulti"), "multi_step = 70000"),
    (dict(opt="badvariant"), "variant = 6"),
    (dict(opt="pairs16"), "variant 5 needs FP32"),
    (dict(opt="pairswall"), "variant 5 needs FP32"),
    (dict(opt="pairsblock"), "variant 5 runs blocks"),
])
def test_create_rejects_invalid_arguments(lib, case, needle):
    nx, ny = case.get("nx", 8), 6
    mask = np.zeros((ny, max(nx, 1)), np.uint8)
    m = case.get("mask")
    if m == "none":
        mask = None
    elif m == "allsolid":
        mask[:] = 1
    elif m == "isolated":
        mask[:] = 1
        mask[2, 2] = 0
    elif m == "wide":
        pass  # all fluid, one node wider than the tile encoding admits
    opt = None
    if case.get("opt"):
        opt = lbm.lbm_options()
        lib.lbm_default_options(ctypes.byref(opt))
        if case["opt"] == "badsize":
            opt.struct_size = 3
        elif case["opt"] == "badprecision":
            opt.precision = 3
        elif case["opt"] == "fp16pipe":
            opt.precision, opt.variant = lbm.LBM_FP16, 3
        elif case["opt"] == "wallpipe":
            opt.wall_scheme, opt.variant = lbm.LBM_WALL_EQUILIBRIUM, 3
        elif case["opt"] == "badwall":
            opt.wall_scheme = 2
        elif case["opt"] == "badscalar":
            opt.scalar_variant = 3
        elif case["opt"] == "multifp16":
            opt.precision, opt.multi_step = lbm.LBM_FP16, 8
        elif case["opt"] == "badmulti":
            opt.multi_step = 70000
        elif case["opt"] == "badvariant":
            opt.variant = 6
        elif case["opt"] == "pairs16":
            opt.precision, opt.variant = lbm.LBM_BF16, 5
        elif case["opt"] == "pairswall":
            opt.wall_scheme, opt.variant = lbm.LBM_WALL_EQUILIBRIUM, 5
        elif case["opt"] == "pairsblock":
            opt.variant, opt.block_threads = 5, 256
        else:
            opt.block_threads = 100
    st, msg = _create(lib, nx, ny, mask, tau=case.get("tau", 0.8), tau_c=case.get("tau_c", 0.6),
                      ports=case.get("ports", ()), opt=opt)
    assert st == lbm.LBM_ERR_ARG, (st, msg)
    assert needle in msg, msg


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.lbm_step(None, 1) == lbm.LBM_ERR_ARG
    assert lib.lbm_step_diagnostics(None, 1, None) == lbm.LBM_ERR_ARG
    assert lib.lbm_get_diagnostics_async(None, None) == lbm.LBM_ERR_ARG
    assert lib.lbm_set_valves(None, 1) == lbm.LBM_ERR_ARG
    lib.lbm_destroy(None)
    assert lib.lbm_status_string(4) == b"LBM_ERR_NUMERIC"


def test_valid_arguments_reach_the_device_step(lib):
    """Valid input passes every host check; without a GPU the first device
    call then reports a CUDA error instead of crashing."""
    import torch

    prob = workloads.config_small()
    ports = [(p["channel"], p["side"], p["x"], p["y0"], p["y1"], p["kind"], p["rho"]) for p in prob["ports"]]
    st, msg = _create(lib, prob["nx"], prob["ny"], prob["solid"], ports=ports,
                      edge_u=prob["edge_u"], edge_C=prob["edge_C"])
    if torch.cuda.is_available():
        assert st == lbm.LBM_OK, msg
    else:
        assert st == lbm.LBM_ERR_CUDA, msg


def test_batch_creation_checks_run_on_the_host(lib):
    """lbm_create_batch rejects an empty batch and more than 256 valve
    channels before any device call."""
    h = ctypes.c_void_p()
    assert lib.lbm_create_batch(ctypes.byref(h), 0, None, None) == lbm.LBM_ERR_ARG
    mask = np.zeros((8, 8), np.uint8)
    eu = np.zeros((2, 8), np.float32)
    port = (lbm.lbm_port * 1)(lbm.lbm_port(1, 0, 0, 0, 4, 1, 1.0))  # channel 1: two channels per chip
    descs = (lbm.lbm_chip_desc * 129)()
    for k in range(129):
        descs[k] = lbm.lbm_chip_desc(8, 8, mask.ctypes.data, 0.8, 0.6, 1, ctypes.cast(port, ctypes.c_void_p),
                                     eu.ctypes.data, eu.ctypes.data)
    assert lib.lbm_create_batch(ctypes.byref(h), 129, descs, None) == lbm.LBM_ERR_ARG
    assert b"valve channels" in lib.lbm_last_error(None)
    descs[0].tau_c = 0.5
    assert lib.lbm_create_batch(ctypes.byref(h), 1, descs, None) == lbm.LBM_ERR_ARG
    assert b"chip 0" in lib.lbm_last_error(None)


def test_create_reports_the_first_isolated_node_of_a_large_mask(lib):
    """Masks of a million nodes or more are scanned by several host threads,
    each over its own rows; the error still names the first bad node in row
    order."""
    nx, ny = 1024, 1024
    mask = np.zeros((ny, nx), np.uint8)
    for x, y in ((300, 1000), (500, 900), (700, 900)):  # three isolated fluid nodes
        mask[y - 1:y + 2, x - 1:x + 2] = 1
        mask[y, x] = 0
    st, msg = _create(lib, nx, ny, mask)
    assert st == lbm.LBM_ERR_ARG
    assert "(500, 900)" in msg and "no fluid neighbour" in msg


def test_create_rejects_grids_beyond_the_tile_encoding(lib):
    """Tile entries hold the row in 17 bits and the first column / 16 in 15
    (a tile ends at most at column 2^19 - 1: 524160 columns); one more row or
    column than that is rejected before any device call."""
    for nx, ny in ((4, 1 << 17), (524161, 2)):
        st, msg = _create(lib, nx, ny, np.zeros((ny, nx), np.uint8))
        assert st == lbm.LBM_ERR_ARG and "too large" in msg, (nx, ny, msg)
