"""lbm_step_noalloc against the ordinary handle path.

lbm_step_noalloc exists for callers that cannot allocate device memory
through the library (code inside another framework's memory pool, or under
a rule against cudaMalloc after start-up).  They own every buffer; the call
runs the same step kernel with its scratch in a fixed array of the library.

This test prepares the caller-owned buffers (the allocation is the caller's
job, so the test makes it with PyTorch), fills them with the same state and
tables a handle uses, then runs two no-alloc calls in a row and compares
populations and diagnostics with two steps of lbm_step, and the populations
with the FP64 oracle.  It lives in a file
of its own, collected last, and passes alone or after the other tests.
"""
import ctypes
import struct

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1307_4703_gb300 import lbm, workloads as W  # noqa: E402

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

TILE = 128
# directions 1..8 of the D2Q9 lattice (e_x, e_y)
EX = [1, 0, -1, 0, 1, -1, -1, 1]
EY = [0, 1, 0, -1, 1, 1, -1, -1]


def _tables(prob, pitch):
    """Wall-link bytes, per-row port entries and tile list in the formats the
    header documents for lbm_step_noalloc."""
    solid = np.asarray(prob["solid"]) != 0
    ny, nx = solid.shape
    fl = ~solid
    pad = np.zeros((ny + 2, nx + 2), bool)
    pad[1:-1, 1:-1] = fl
    lb = np.zeros((ny, nx), np.uint8)
    for i in range(8):  # bit i: the pull source x - e_(i+1) is not fluid
        src = pad[1 - EY[i]:1 - EY[i] + ny, 1 - EX[i]:1 - EX[i] + nx]
        lb |= ((~src).astype(np.uint8) << i)
    links = np.full((ny, pitch), 0xFF, np.uint8)
    links[:, :nx] = np.where(fl, lb, 0xFF)

    ports = np.zeros(2 * ny, dtype=[("x", "<i4"), ("ck", "<i4"), ("a", "<f4"), ("c", "<f4")])
    ports["x"] = -1
    eu = np.asarray(prob["edge_u"], np.float32)
    ec = np.asarray(prob["edge_C"], np.float32)
    for p in prob["ports"]:
        for y in range(p["y0"], p["y1"]):
            e = ports[p["side"] * ny + y]
            e["x"] = p["x"]
            e["ck"] = p["channel"] | (p["kind"] << 8)
            if p["kind"] == W.VELOCITY:
                e["a"] = eu[p["side"], y]
                e["c"] = ec[p["side"], y]
            else:
                e["a"] = np.float32(p.get("rho", 1.0) - 1.0)
            ports[p["side"] * ny + y] = e

    tiles = []
    for y in range(ny):
        for seg in range(pitch // TILE):
            q = np.nonzero(fl[y, seg * TILE:min(nx, (seg + 1) * TILE)])[0] // 4  # fluid quads
            if len(q):
                tiles.append(((y << 15) | (seg * TILE // 16), int(q[0]) | (int(q[-1]) << 8)))
    return links, ports, np.array(tiles, dtype=np.uint32).reshape(-1, 2)


def _raw_state(chip):
    """The handle's stored populations, bit for bit, as [14][ny][nx]."""
    blob = chip.save_state()
    n_sched = struct.unpack_from("<i", blob, 12)[0]
    off = 40 + 4 * n_sched
    return np.frombuffer(blob, dtype=np.float32, offset=off).reshape(14, chip.ny, chip.nx).copy()


def _pitched(arr, pitch):
    planes, ny, nx = arr.shape
    out = np.zeros((planes, ny, pitch), np.float32)
    out[:, :, :nx] = arr
    return out


def _case(name):
    if name == "random-300x40":  # about 120 tiles: at most one per block
        return W.random_case(41, 300, 40, solid_frac=0.15)
    # 1100 x 280: 9 segments x 280 rows = 2520 tiles, more than the 2048-block cap;
    # the grid is one wave of resident blocks (several hundred partials to add)
    return W.random_case(43, 1100, 280, solid_frac=0.1)


@pytest.mark.parametrize("name,max_blocks", [("random-300x40", 0), ("random-300x40", 5),
                                             ("random-1100x280", 0), ("random-1100x280", 7)])
def test_noalloc_step_matches_handle_step_twice(name, max_blocks):
    """Two no-alloc calls in a row: the stored populations equal the handle
    path's bit for bit and the FP64 oracle's post-collision populations
    within the FP32 parity bound (n x 30 x 2^-24 for n steps), and the
    diagnostics equal the handle's.  max_blocks = 5 or 7 makes every block
    take many tiles; the 1100 x 280 lattice has more tiles than the fixed
    scratch has block slots."""
    import oracle

    lib = lbm.load()
    prob, init = _case(name)
    ny, nx = prob["ny"], prob["nx"]
    pitch = (nx + TILE - 1) // TILE * TILE
    words = [5, 3]  # valve words of the two steps

    chip = lbm.Chip.from_problem(prob)
    chip.init_equilibrium(**init)
    start = _raw_state(chip)
    ref = oracle.from_problem(prob)
    ref.init_equilibrium(**init)

    links, ports, tiles = _tables(prob, pitch)
    if name == "random-1100x280":
        assert len(tiles) > 2048
    dev = torch.device("cuda")
    bufs = [torch.from_numpy(_pitched(start, pitch)).to(dev), torch.zeros((14, ny, pitch), device=dev)]
    links_d = torch.from_numpy(links).to(dev)
    ports_d = torch.from_numpy(ports.view(np.uint8)).to(dev)
    tiles_d = torch.from_numpy(tiles.view(np.uint8).reshape(-1)).to(dev)
    diag_d = torch.zeros(4, dtype=torch.float64, device=dev)
    err_d = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    msg = ctypes.create_string_buffer(256)
    fl = ~np.asarray(prob["solid"], bool)

    for call, word in enumerate(words):
        # ordinary path: one step with this valve word
        chip.set_valves(word)
        chip.step(1)
        ref_diag = chip.diagnostics()
        ref_state = _raw_state(chip)
        ref.step(word)
        # allocation-free path: one call, src -> dst
        src, dst = bufs[call % 2], bufs[(call + 1) % 2]
        d = lbm.lbm_noalloc_step()
        d.struct_size = ctypes.sizeof(lbm.lbm_noalloc_step)
        d.nx, d.ny, d.pitch = nx, ny, pitch
        d.src, d.dst = src.data_ptr(), dst.data_ptr()
        d.links, d.ports, d.tiles = links_d.data_ptr(), ports_d.data_ptr(), tiles_d.data_ptr()
        d.n_tiles = len(tiles)
        d.max_blocks = max_blocks
        d.tau, d.tau_c, d.w0 = prob["tau"], prob["tau_c"], prob["w0"]
        d.open_mask = word
        d.diag, d.err = diag_d.data_ptr(), err_d.data_ptr()
        d.stream = stream.cuda_stream
        d.message = ctypes.cast(msg, ctypes.c_char_p)
        d.message_len = len(msg)
        st = lib.lbm_step_noalloc(ctypes.byref(d))
        assert st == lbm.LBM_OK, msg.value.decode()
        torch.cuda.synchronize()
        assert int(err_d.item()) == 0
        got = dst.cpu().numpy()[:, :, :nx]
        # same kernel, same inputs: identical bits on every fluid node
        assert np.array_equal(got[:, fl], ref_state[:, fl]), "populations differ after call %d" % (call + 1)
        got_diag = diag_d.cpu().numpy()
        assert np.allclose(got_diag, ref_diag, rtol=1e-6, atol=1e-6), (got_diag, ref_diag)
        # and against the FP64 oracle directly: stored f_i - w_i and g_i
        fp, gp = ref.post_collision()
        w9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
        rf = np.moveaxis(fp, -1, 0) - w9[:, None, None]
        rg = np.moveaxis(gp, -1, 0)
        tol = (call + 1) * 30 * 2.0 ** -24
        ef = np.abs(got[:9].astype(np.float64) - rf)[:, fl].max()
        eg = np.abs(got[9:].astype(np.float64) - rg)[:, fl].max()
        assert ef <= tol and eg <= tol, (ef, eg, tol)
    chip.close()


def test_noalloc_rejects_oversized_launch_and_bad_descriptor():
    lib = lbm.load()
    msg = ctypes.create_string_buffer(256)
    d = lbm.lbm_noalloc_step()
    d.struct_size = ctypes.sizeof(lbm.lbm_noalloc_step)
    d.nx, d.ny, d.pitch = 64, 8, 128
    d.max_blocks = 2049
    d.message = ctypes.cast(msg, ctypes.c_char_p)
    d.message_len = len(msg)
    assert lib.lbm_step_noalloc(ctypes.byref(d)) == lbm.LBM_ERR_ARG
    assert b"2048" in msg.value
    d.max_blocks = 0
    d.pitch = 100
    assert lib.lbm_step_noalloc(ctypes.byref(d)) == lbm.LBM_ERR_ARG
    assert b"pitch" in msg.value
