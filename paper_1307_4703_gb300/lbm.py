"""Thin ctypes binding of the C ABI in ``include/lbm.h``.

Argument marshalling only: every step of the time step runs in the CUDA
library ``_lib/liblbm_gb300.so``.  PyTorch, when given, supplies the CUDA
stream and the device memory (through its caching allocator); it computes
nothing.  If the library is missing, ``load()`` raises: there is no CPU
fallback.
"""
import ctypes
import os

import numpy as np

WEST, EAST = 0, 1
VELOCITY, PRESSURE = 0, 1

LBM_OK, LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_OOM, LBM_ERR_NUMERIC, LBM_ERR_TIMEOUT, LBM_ERR_STATE = range(7)
LBM_FP32, LBM_FP16, LBM_BF16 = range(3)
LBM_PORT_VELOCITY, LBM_PORT_PRESSURE, LBM_PORT_PRESSURE_RESCALE, LBM_PORT_INLET_RESCALE = range(4)
LBM_WALL_BOUNCE_BACK, LBM_WALL_EQUILIBRIUM = range(2)
PRECISIONS = {"fp32": LBM_FP32, "fp16": LBM_FP16, "bf16": LBM_BF16}

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "liblbm_gb300.so")


class LbmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (_STATUS_NAMES.get(status, status), message))
        self.status = status


_STATUS_NAMES = {0: "LBM_OK", 1: "LBM_ERR_ARG", 2: "LBM_ERR_CUDA", 3: "LBM_ERR_OOM",
                 4: "LBM_ERR_NUMERIC", 5: "LBM_ERR_TIMEOUT", 6: "LBM_ERR_STATE"}


class lbm_port(ctypes.Structure):
    _fields_ = [("channel", ctypes.c_int32), ("side", ctypes.c_int32), ("x", ctypes.c_int32),
                ("y0", ctypes.c_int32), ("y1", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("rho", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class lbm_options(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("device", ctypes.c_int32),
                ("w0", ctypes.c_double), ("rho0", ctypes.c_double), ("C0", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_user", ctypes.c_void_p), ("block_threads", ctypes.c_int32),
                ("max_blocks", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("pipeline_stages", ctypes.c_int32), ("consumer_warps", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("decay", ctypes.c_double), ("wall_scheme", ctypes.c_int32),
                ("graph_steps", ctypes.c_int32), ("scalar_variant", ctypes.c_int32),
                ("multi_step", ctypes.c_int32)]


class lbm_info(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("pitch", ctypes.c_int32),
                ("n_tiles", ctypes.c_int32), ("grid", ctypes.c_int32), ("block", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("stages", ctypes.c_int32), ("fluid_nodes", ctypes.c_int64),
                ("algorithmic_bytes_per_step", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("precision", ctypes.c_int32), ("instances", ctypes.c_int32)]


class lbm_chip_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("mask", ctypes.c_void_p),
                ("tau", ctypes.c_double), ("tau_c", ctypes.c_double), ("n_ports", ctypes.c_int32),
                ("ports", ctypes.c_void_p), ("edge_u", ctypes.c_void_p), ("edge_C", ctypes.c_void_p)]


class lbm_instance(ctypes.Structure):
    _fields_ = [("row0", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("channel_base", ctypes.c_int32)]


class lbm_objective(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("target", ctypes.c_void_p), ("weight", ctypes.c_void_p)]


class lbm_row_port(ctypes.Structure):
    _fields_ = [("x", ctypes.c_int32), ("channel_kind", ctypes.c_int32), ("a", ctypes.c_float),
                ("c", ctypes.c_float)]


class lbm_tile(ctypes.Structure):
    _fields_ = [("row_segment", ctypes.c_uint32), ("quads", ctypes.c_uint32)]


class lbm_noalloc_step(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("pitch", ctypes.c_int32), ("src", ctypes.c_void_p), ("dst", ctypes.c_void_p),
                ("links", ctypes.c_void_p), ("ports", ctypes.c_void_p), ("tiles", ctypes.c_void_p),
                ("n_tiles", ctypes.c_int32), ("max_blocks", ctypes.c_int32), ("tau", ctypes.c_double),
                ("tau_c", ctypes.c_double), ("w0", ctypes.c_double), ("open_mask", ctypes.c_uint32),
                ("diag", ctypes.c_void_p), ("err", ctypes.c_void_p), ("stream", ctypes.c_void_p),
                ("message", ctypes.c_char_p), ("message_len", ctypes.c_int32)]


_lib = None
_P = ctypes.POINTER
_f32p = _P(ctypes.c_float)
_f64p = _P(ctypes.c_double)
_u8p = _P(ctypes.c_uint8)
_u32p = _P(ctypes.c_uint32)

# name -> (restype, argtypes); the same names and order as include/lbm.h
SIGNATURES = {
    "lbm_default_options": (None, [_P(lbm_options)]),
    "lbm_create": (ctypes.c_int, [_P(ctypes.c_void_p), ctypes.c_int32, ctypes.c_int32, _u8p,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_int32, _P(lbm_port),
                                  _f32p, _f32p, _P(lbm_options)]),
    "lbm_destroy": (None, [ctypes.c_void_p]),
    "lbm_set_valves": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32]),
    "lbm_set_valve_schedule": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, _u32p]),
    "lbm_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "lbm_get_fields": (ctypes.c_int, [ctypes.c_void_p, _f32p, _f32p, _f32p, _f32p]),
    "lbm_get_fields_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p]),
    "lbm_get_diagnostics": (ctypes.c_int, [ctypes.c_void_p, _f64p]),
    "lbm_get_diagnostics_async": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "lbm_step_diagnostics": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "lbm_get_populations": (ctypes.c_int, [ctypes.c_void_p, _f32p, _f32p]),
    "lbm_set_populations": (ctypes.c_int, [ctypes.c_void_p, _f32p, _f32p]),
    "lbm_init_equilibrium": (ctypes.c_int, [ctypes.c_void_p, _f32p, _f32p, _f32p, _f32p]),
    "lbm_save_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, _P(ctypes.c_size_t)]),
    "lbm_load_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "lbm_get_step": (ctypes.c_int, [ctypes.c_void_p, _P(ctypes.c_int64)]),
    "lbm_synchronize": (ctypes.c_int, [ctypes.c_void_p]),
    "lbm_clear_error": (ctypes.c_int, [ctypes.c_void_p]),
    "lbm_debug_barrier_extra": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "lbm_get_info": (ctypes.c_int, [ctypes.c_void_p, _P(lbm_info)]),
    "lbm_step_noalloc": (ctypes.c_int, [_P(lbm_noalloc_step)]),
    "lbm_adjoint": (ctypes.c_int, [ctypes.c_void_p, _P(lbm_objective), ctypes.c_int64, ctypes.c_int32,
                                   _f64p, _f64p, _f64p, _f64p]),
    "lbm_store_velocity": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32]),
    "lbm_set_velocity_field": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, _f32p, _f32p]),
    "lbm_scalar_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double]),
    "lbm_create_batch": (ctypes.c_int, [_P(ctypes.c_void_p), ctypes.c_int32, _P(lbm_chip_desc),
                                        _P(lbm_options)]),
    "lbm_get_instance": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _P(lbm_instance)]),
    "lbm_set_instance_valves": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32]),
    "lbm_set_instance_schedule": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                                 _u32p]),
    "lbm_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "lbm_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "lbm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
}


def load(path=None):
    """Load the CUDA library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("the CUDA library %s is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ports(ports):
    ports = list(ports)
    parr = (lbm_port * max(1, len(ports)))()
    for k, p in enumerate(ports):
        parr[k] = lbm_port(int(p["channel"]), int(p["side"]), int(p["x"]), int(p["y0"]),
                           int(p["y1"]), int(p["kind"]), float(p.get("rho", 1.0)))
    parr._keep = ports
    return parr


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _fp(a):
    return a.ctypes.data_as(_f32p)


def _torch_hooks(device_index):
    """Allocator hooks that hand out memory from PyTorch's caching allocator."""
    import torch

    def _alloc(nbytes, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device=device_index)
        except Exception:
            return None

    def _free(ptr, nbytes, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    return ALLOC_FN(_alloc), FREE_FN(_free)


class Chip:
    """One chip on one GPU: the handle of ``lbm_create`` and its calls.

    ``solid`` (ny, nx): non-zero = solid.  ``ports``: dicts with channel,
    side, x, y0, y1, kind, rho.  ``edge_u`` / ``edge_C``: (2, ny) per side
    and row.  ``stream``: a ``torch.cuda.Stream`` (or raw cudaStream_t int);
    ``torch_alloc``: take device memory from PyTorch's caching allocator.
    ``precision``: storage of the populations, "fp32" (default), "fp16" or
    "bf16" (16-bit deviations, FP32 arithmetic).
    """

    def __init__(self, solid, tau, tau_c, ports=(), edge_u=None, edge_C=None, w0=1.0 / 3.0,
                 rho0=1.0, C0=0.0, stream=None, torch_alloc=False, device=-1, block_threads=0,
                 max_blocks=0, variant=0, pipeline_stages=0, consumer_warps=0, precision="fp32",
                 graph_steps=0, decay=0.0, wall_scheme=0, scalar_variant=0, multi_step=0, _batch=None):
        self._lib = load()
        if _batch is None:
            solid = np.asarray(solid)
            if solid.dtype != np.uint8 or not solid.flags.c_contiguous:
                solid = np.ascontiguousarray(solid != 0, dtype=np.uint8)  # the library reads non-zero as solid
            self.ny, self.nx = solid.shape
            parr = _ports(ports)
            eu = _f32(np.zeros((2, self.ny)) if edge_u is None else edge_u, (2, self.ny))
            ec = _f32(np.zeros((2, self.ny)) if edge_C is None else edge_C, (2, self.ny))
        opt = lbm_options()
        self._lib.lbm_default_options(ctypes.byref(opt))
        opt.device = int(device)
        opt.w0, opt.rho0, opt.C0 = float(w0), float(rho0), float(C0)
        opt.block_threads = int(block_threads)
        opt.max_blocks = int(max_blocks)
        opt.variant = int(variant)
        opt.pipeline_stages = int(pipeline_stages)
        opt.consumer_warps = int(consumer_warps)
        opt.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        opt.graph_steps = int(graph_steps)
        opt.decay = float(decay)
        opt.wall_scheme = int(wall_scheme)
        opt.scalar_variant = int(scalar_variant)
        opt.multi_step = int(multi_step)
        self.stream = stream
        if stream is not None:
            opt.stream = ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        self._hooks = None
        if torch_alloc:
            import torch
            dev = torch.cuda.current_device() if device < 0 else int(device)
            self._hooks = _torch_hooks(dev)
            opt.alloc, opt.free = self._hooks
        h = ctypes.c_void_p()
        if _batch is None:
            st = self._lib.lbm_create(ctypes.byref(h), self.nx, self.ny, solid.ctypes.data_as(_u8p),
                                      float(tau), float(tau_c), len(parr._keep), parr, _fp(eu), _fp(ec),
                                      ctypes.byref(opt))
        else:
            descs, keep = _batch
            st = self._lib.lbm_create_batch(ctypes.byref(h), len(descs), descs, ctypes.byref(opt))
        if st != LBM_OK:
            raise LbmError(st, self._lib.lbm_last_error(None).decode())
        self._h = h
        if _batch is None:
            self._mask = solid
            self._solid = None
        else:
            inf = self.info()
            self.nx, self.ny = inf["nx"], inf["ny"]
            self._solid = np.ones((self.ny, self.nx), bool)
            for k in range(inf["instances"]):
                i = self.instance(k)
                self._solid[i["row0"]:i["row0"] + i["ny"], :i["nx"]] = keep[4 * k] != 0

    @property
    def solid(self):
        """(ny, nx) bool, True = solid (formed on first use)."""
        if self._solid is None:
            self._solid = self._mask != 0
        return self._solid

    @classmethod
    def from_problem(cls, prob, **kw):
        kw.setdefault("decay", prob.get("decay", 0.0))
        kw.setdefault("wall_scheme", prob.get("wall_scheme", 0))
        return cls(prob["solid"], prob["tau"], prob["tau_c"], ports=prob["ports"],
                   edge_u=prob["edge_u"], edge_C=prob["edge_C"], w0=prob.get("w0", 1.0 / 3.0), **kw)

    @classmethod
    def batch(cls, problems, **kw):
        """One handle over many independent chips (lbm_create_batch), each a
        problem dict as ``from_problem`` takes; chip k is ``instance(k)``."""
        problems = list(problems)
        descs = (lbm_chip_desc * len(problems))()
        keep = []
        for k, prob in enumerate(problems):
            solid = np.ascontiguousarray(np.asarray(prob["solid"]) != 0, dtype=np.uint8)
            ny, nx = solid.shape
            parr = _ports(prob["ports"])
            eu = _f32(prob["edge_u"], (2, ny))
            ec = _f32(prob["edge_C"], (2, ny))
            keep += [solid, eu, ec, parr]
            descs[k] = lbm_chip_desc(nx, ny, solid.ctypes.data, float(prob["tau"]), float(prob["tau_c"]),
                                     len(parr._keep), ctypes.cast(parr, ctypes.c_void_p), eu.ctypes.data,
                                     ec.ctypes.data)
        kw.setdefault("w0", problems[0].get("w0", 1.0 / 3.0))
        chip = cls(None, None, None, _batch=(descs, keep), **kw)
        chip.problems = problems
        return chip

    def instance(self, k):
        i = lbm_instance()
        self._check(self._lib.lbm_get_instance(self._h, int(k), ctypes.byref(i)))
        return {n: getattr(i, n) for n, _ in lbm_instance._fields_}

    def instance_fields(self, k, fields=None):
        """rho, ux, uy, C of chip k of a batch (slices of ``fields()``)."""
        i = self.instance(k)
        fields = self.fields() if fields is None else fields
        return tuple(a[i["row0"]:i["row0"] + i["ny"], :i["nx"]] for a in fields)

    def set_instance_valves(self, k, open_mask):
        self._check(self._lib.lbm_set_instance_valves(self._h, int(k), int(open_mask) & 0xFFFFFFFF))

    def set_instance_schedule(self, k, period, states):
        arr = np.ascontiguousarray(states, dtype=np.uint32)
        self._check(self._lib.lbm_set_instance_schedule(self._h, int(k), int(period), len(arr),
                                                        arr.ctypes.data_as(_u32p)))

    # -- plumbing ------------------------------------------------------------
    def _check(self, st):
        if st != LBM_OK:
            raise LbmError(st, self._lib.lbm_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- the ABI calls -------------------------------------------------------
    def set_valves(self, open_mask):
        self._check(self._lib.lbm_set_valves(self._h, int(open_mask) & 0xFFFFFFFF))

    def set_valve_schedule(self, period, states):
        arr = np.ascontiguousarray(states, dtype=np.uint32)
        self._check(self._lib.lbm_set_valve_schedule(self._h, int(period), len(arr),
                                                     arr.ctypes.data_as(_u32p)))

    def step(self, n=1):
        self._check(self._lib.lbm_step(self._h, int(n)))

    def fields(self, out=None):
        """rho, ux, uy, C as (ny, nx) float32 arrays; ``out``: four
        C-contiguous float32 arrays of that shape to fill instead (e.g.
        page-locked ones, which the device copies into faster)."""
        if out is None:
            out = [np.empty((self.ny, self.nx), np.float32) for _ in range(4)]
        else:
            out = list(out)
            for a in out:
                if a.dtype != np.float32 or a.shape != (self.ny, self.nx) or not a.flags.c_contiguous:
                    raise ValueError("fields(out=...): four C-contiguous float32 (ny, nx) arrays")
        self._check(self._lib.lbm_get_fields(self._h, *[_fp(a) for a in out]))
        return tuple(out)  # rho, ux, uy, C

    def fields_device(self, rho=None, ux=None, uy=None, C=None):
        """Moments into device buffers (torch tensors or raw pointers)."""
        ptrs = [ctypes.c_void_p(0 if a is None else int(getattr(a, "data_ptr", lambda: a)()))
                for a in (rho, ux, uy, C)]
        self._check(self._lib.lbm_get_fields_device(self._h, *ptrs))

    def diagnostics(self):
        out = np.zeros(4)
        self._check(self._lib.lbm_get_diagnostics(self._h, out.ctypes.data_as(_f64p)))
        return out

    def populations(self):
        f = np.empty((9, self.ny, self.nx), np.float32)
        g = np.empty((5, self.ny, self.nx), np.float32)
        self._check(self._lib.lbm_get_populations(self._h, _fp(f), _fp(g)))
        return f, g

    def set_populations(self, f=None, g=None):
        fa = None if f is None else _f32(f, (9, self.ny, self.nx))
        ga = None if g is None else _f32(g, (5, self.ny, self.nx))
        self._check(self._lib.lbm_set_populations(self._h, None if fa is None else _fp(fa),
                                                  None if ga is None else _fp(ga)))

    def init_equilibrium(self, rho, ux, uy, C):
        a = [_f32(np.broadcast_to(v, (self.ny, self.nx))) for v in (rho, ux, uy, C)]
        self._check(self._lib.lbm_init_equilibrium(self._h, *[_fp(v) for v in a]))

    def save_state(self):
        n = ctypes.c_size_t(0)
        self._check(self._lib.lbm_save_state(self._h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._check(self._lib.lbm_save_state(self._h, buf, ctypes.byref(n)))
        return buf.raw[:n.value]

    def load_state(self, data):
        buf = ctypes.create_string_buffer(bytes(data), len(data))
        self._check(self._lib.lbm_load_state(self._h, buf, len(data)))

    def step_count(self):
        t = ctypes.c_int64()
        self._check(self._lib.lbm_get_step(self._h, ctypes.byref(t)))
        return t.value

    def synchronize(self):
        self._check(self._lib.lbm_synchronize(self._h))

    def clear_error(self):
        self._check(self._lib.lbm_clear_error(self._h))

    def debug_barrier_extra(self, extra):
        """Test hook: make the multi-step kernel's barriers wait for arrivals
        that never come (extra > 0), so that their bounded wait runs out."""
        self._check(self._lib.lbm_debug_barrier_extra(self._h, int(extra)))

    def adjoint(self, n_steps, obj_x, obj_y, target, weight=None, ckpt_every=250):
        """Gradient of J = sum weight (C(x, y) - target)^2 after n_steps
        (the chip advances by n_steps).  Returns (J, dJ/dtau_c,
        dJ/du_in (2, ny), dJ/dC_in (2, ny))."""
        ox = np.ascontiguousarray(obj_x, np.int32)
        oy = np.ascontiguousarray(obj_y, np.int32)
        tg = np.ascontiguousarray(target, np.float32)
        wt = np.ascontiguousarray(np.ones(len(ox)) if weight is None else weight, np.float32)
        o = lbm_objective(len(ox), ox.ctypes.data, oy.ctypes.data, tg.ctypes.data, wt.ctypes.data)
        J = ctypes.c_double()
        dtau = ctypes.c_double()
        du = np.zeros((2, self.ny))
        dc = np.zeros((2, self.ny))
        self._check(self._lib.lbm_adjoint(self._h, ctypes.byref(o), int(n_steps), int(ckpt_every),
                                          ctypes.byref(J), ctypes.byref(dtau), du.ctypes.data_as(_f64p),
                                          dc.ctypes.data_as(_f64p)))
        return J.value, dtau.value, du, dc

    def store_velocity(self, open_mask):
        self._check(self._lib.lbm_store_velocity(self._h, int(open_mask) & 0xFFFFFFFF))

    def set_velocity_field(self, open_mask, ux, uy):
        a = _f32(np.broadcast_to(ux, (self.ny, self.nx)))
        b = _f32(np.broadcast_to(uy, (self.ny, self.nx)))
        self._check(self._lib.lbm_set_velocity_field(self._h, int(open_mask) & 0xFFFFFFFF, _fp(a), _fp(b)))

    def scalar_step(self, n=1, u_scale=1.0):
        self._check(self._lib.lbm_scalar_step(self._h, int(n), float(u_scale)))

    def autotune(self, trial_steps=0):
        """Keep the fastest launch shape of the step kernel (lbm_autotune)."""
        self._check(self._lib.lbm_autotune(self._h, int(trial_steps)))
        return self.info()

    def diagnostics_async(self, out_ptr):
        """Enqueue the diagnostics read into host memory at out_ptr (4
        doubles, page-locked, e.g. a pinned torch tensor's data_ptr());
        valid after synchronize()."""
        self._check(self._lib.lbm_get_diagnostics_async(self._h, ctypes.c_void_p(int(out_ptr))))

    def step_diagnostics(self, n, out_ptr):
        """Advance n steps, one launch each, the k-th step's four diagnostics
        written by the step kernel to out_ptr + 32 k (4 n doubles of device
        memory or page-locked host memory, e.g. a CUDA or pinned torch
        tensor's data_ptr()); valid after synchronize()."""
        self._check(self._lib.lbm_step_diagnostics(self._h, int(n), ctypes.c_void_p(int(out_ptr))))

    def info(self):
        i = lbm_info()
        self._check(self._lib.lbm_get_info(self._h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in lbm_info._fields_}
