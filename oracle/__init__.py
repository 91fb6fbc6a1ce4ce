"""FP64 CPU oracle of the coupled D2Q9 + scalar lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference leg of ``bench.py`` import this package.  The
CUDA library and its Python binding never do, and share no code with it.

The arithmetic lives in ``lbm_oracle.c`` (Tanaka & Iber, arXiv 1307.4703,
"Numerical Methods" and "Boundary Conditions"); this module only marshals
numpy arrays through ctypes.
"""
import ctypes
import os

import numpy as np

from .build import build_oracle

WEST, EAST = 0, 1
VELOCITY, PRESSURE, PRESSURE_RESCALE, INLET_RESCALE = 0, 1, 2, 3


class _Port(ctypes.Structure):
    _fields_ = [("channel", ctypes.c_int), ("side", ctypes.c_int), ("x", ctypes.c_int),
                ("y0", ctypes.c_int), ("y1", ctypes.c_int), ("kind", ctypes.c_int),
                ("rho", ctypes.c_double)]


_libs = {}


def _load(parallel=False):
    """The serial library, or (``parallel``) the OpenMP build of the same
    source, whose row loops run on all host cores with the same bits."""
    lib = _libs.get(bool(parallel))
    if lib is None:
        lib = ctypes.CDLL(build_oracle(parallel=bool(parallel)))
        P = ctypes.POINTER
        d = P(ctypes.c_double)
        lib.orc_new.restype = ctypes.c_void_p
        lib.orc_new.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_ubyte), ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                P(_Port), d, d]
        lib.orc_free.argtypes = [ctypes.c_void_p]
        lib.orc_init_equilibrium.argtypes = [ctypes.c_void_p, d, d, d, d]
        lib.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_uint]
        lib.orc_fields.argtypes = [ctypes.c_void_p, d, d, d, d]
        lib.orc_get_populations.argtypes = [ctypes.c_void_p, d, d]
        lib.orc_set_populations.argtypes = [ctypes.c_void_p, d, d]
        lib.orc_post_collision.argtypes = [ctypes.c_void_p, d, d]
        lib.orc_diagnostics.argtypes = [ctypes.c_void_p, ctypes.c_uint, d]
        lib.orc_lattice_vectors.argtypes = [P(ctypes.c_int), P(ctypes.c_int), d]
        lib.orc_adjoint_step.argtypes = [ctypes.c_void_p, ctypes.c_uint, d, d, d, d, d, d, d]
        lib.orc_scalar_step.argtypes = [ctypes.c_void_p, ctypes.c_uint, d, d]
        lib.orc_set_decay.argtypes = [ctypes.c_void_p, ctypes.c_double]
        lib.orc_set_wall_scheme.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.orc_set_wall_scheme.restype = ctypes.c_int
        lib.orc_adjoint.restype = ctypes.c_double
        lib.orc_adjoint.argtypes = [ctypes.c_void_p, ctypes.c_int, P(ctypes.c_uint), ctypes.c_int,
                                    P(ctypes.c_int), P(ctypes.c_int), d, d, d, d, d]
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_num_threads.argtypes = []
        lib.orc_set_num_threads.argtypes = [ctypes.c_int]
        _libs[bool(parallel)] = lib
    return lib


def num_threads(parallel=False):
    """Host threads the oracle's row loops use (1 for the serial build)."""
    return int(_load(parallel).orc_num_threads())


def set_num_threads(n):
    """Team size of the OpenMP build (the serial build ignores it)."""
    _load(True).orc_set_num_threads(int(n))


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def lattice_vectors():
    """(ex, ey, w) exactly as the oracle uses them."""
    lib = _load()
    ex = (ctypes.c_int * 9)()
    ey = (ctypes.c_int * 9)()
    w = np.zeros(9)
    lib.orc_lattice_vectors(ex, ey, _dptr(w))
    return np.array(ex[:]), np.array(ey[:]), w


class OracleLattice:
    """One lattice held by the oracle.

    ``parallel``: run on the OpenMP build (all host cores, same bits).
    ``solid``: (ny, nx) array, non-zero = solid.  ``ports``: iterable of
    dicts with keys channel, side, x, y0, y1, kind and (pressure ports) rho.
    ``edge_u`` / ``edge_C``: (2, ny) arrays of u_x and C_in per side and row
    at velocity-port nodes.  ``w0``: rest weight of the scalar lattice
    (1/3: D2Q5; 0: the paper's D2Q4).
    """

    def __init__(self, solid, tau_f, tau_g, w0=1.0 / 3.0, periodic=False, ports=(),
                 edge_u=None, edge_C=None, decay=0.0, wall_scheme=0, parallel=False):
        lib = _load(parallel)
        solid = np.ascontiguousarray(np.asarray(solid) != 0, dtype=np.uint8)
        self.ny, self.nx = solid.shape
        self.solid = solid.astype(bool)
        ports = list(ports)
        arr = (_Port * max(1, len(ports)))()
        for k, p in enumerate(ports):
            arr[k] = _Port(int(p["channel"]), int(p["side"]), int(p["x"]), int(p["y0"]),
                           int(p["y1"]), int(p["kind"]), float(p.get("rho", 1.0)))
        self.ports = ports
        eu = np.zeros((2, self.ny)) if edge_u is None else np.ascontiguousarray(edge_u, np.float64)
        ec = np.zeros((2, self.ny)) if edge_C is None else np.ascontiguousarray(edge_C, np.float64)
        assert eu.shape == (2, self.ny) and ec.shape == (2, self.ny)
        self._keep = (solid, arr, eu, ec)
        h = lib.orc_new(self.nx, self.ny, solid.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)),
                        float(tau_f), float(tau_g), float(w0), 1 if periodic else 0,
                        len(ports), arr, _dptr(eu), _dptr(ec))
        if not h:
            raise ValueError("oracle rejected the lattice arguments")
        self._h = ctypes.c_void_p(h)
        self._lib = lib
        self.t = 0
        if decay:
            lib.orc_set_decay(self._h, float(decay))
        if wall_scheme and lib.orc_set_wall_scheme(self._h, int(wall_scheme)) != 0:
            raise ValueError("oracle: wall scheme %r" % wall_scheme)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_free(self._h)
            self._h = None

    def __del__(self):
        self.close()

    # -- state ---------------------------------------------------------------
    def init_equilibrium(self, rho, ux, uy, C):
        a = [np.ascontiguousarray(np.broadcast_to(v, (self.ny, self.nx)), np.float64)
             for v in (rho, ux, uy, C)]
        self._lib.orc_init_equilibrium(self._h, *[_dptr(v) for v in a])

    def step(self, open_mask, n=1):
        for _ in range(int(n)):
            self._lib.orc_step(self._h, ctypes.c_uint(int(open_mask) & 0xFFFFFFFF))
            self.t += 1

    def run(self, n, schedule):
        """Advance n steps; ``schedule(t)`` gives the valve word of step t."""
        for _ in range(int(n)):
            self.step(schedule(self.t))

    def fields(self):
        out = [np.zeros((self.ny, self.nx)) for _ in range(4)]
        self._lib.orc_fields(self._h, *[_dptr(v) for v in out])
        return tuple(out)  # rho, ux, uy, C

    def populations(self):
        f = np.zeros((self.ny, self.nx, 9))
        g = np.zeros((self.ny, self.nx, 5))
        self._lib.orc_get_populations(self._h, _dptr(f), _dptr(g))
        return f, g

    def set_populations(self, f, g):
        f = np.ascontiguousarray(f, np.float64).reshape(self.ny, self.nx, 9)
        g = np.ascontiguousarray(g, np.float64).reshape(self.ny, self.nx, 5)
        self._lib.orc_set_populations(self._h, _dptr(f), _dptr(g))

    def post_collision(self):
        f = np.zeros((self.ny, self.nx, 9))
        g = np.zeros((self.ny, self.nx, 5))
        self._lib.orc_post_collision(self._h, _dptr(f), _dptr(g))
        return f, g

    def scalar_step(self, open_mask, ux, uy, n=1):
        """Scalar-only steps with a given (already scaled) velocity field."""
        ux = np.ascontiguousarray(np.broadcast_to(ux, (self.ny, self.nx)), np.float64)
        uy = np.ascontiguousarray(np.broadcast_to(uy, (self.ny, self.nx)), np.float64)
        for _ in range(int(n)):
            self._lib.orc_scalar_step(self._h, ctypes.c_uint(int(open_mask) & 0xFFFFFFFF), _dptr(ux), _dptr(uy))
            self.t += 1

    def adjoint_step(self, open_mask, S_t, S_t1, af, ag):
        """One reverse step: (af, ag) = dJ/dS_{t+1} -> dJ/dS_t, given the
        pre-collision states S_t = (f, g) and S_{t+1}.  Returns (af, ag, grad)
        with grad = [dJ/d(1/tau_g), dJ/du_in (2*ny), dJ/dC_in (2*ny)]."""
        c = lambda a, k: np.ascontiguousarray(a, np.float64).reshape(self.ny, self.nx, k)
        ft, gt, ft1, gt1 = c(S_t[0], 9), c(S_t[1], 5), c(S_t1[0], 9), c(S_t1[1], 5)
        af = c(af, 9).copy()
        ag = c(ag, 5).copy()
        grad = np.zeros(1 + 4 * self.ny)
        self._lib.orc_adjoint_step(self._h, ctypes.c_uint(int(open_mask) & 0xFFFFFFFF), _dptr(ft), _dptr(gt),
                                   _dptr(ft1), _dptr(gt1), _dptr(af), _dptr(ag), _dptr(grad))
        return af, ag, grad

    def adjoint(self, n, masks, obj_x, obj_y, target, weight):
        """n forward steps (the lattice advances) and the reverse pass of
        J = sum weight (C(x, y) - target)^2 at the final step.  Returns
        (J, dJ/dtau_g, dJ/du_in (2, ny), dJ/dC_in (2, ny))."""
        masks = np.ascontiguousarray(masks, np.uint32)
        assert len(masks) >= n
        ox = np.ascontiguousarray(obj_x, np.int32)
        oy = np.ascontiguousarray(obj_y, np.int32)
        tg = np.ascontiguousarray(target, np.float64)
        wt = np.ascontiguousarray(weight, np.float64)
        dtau = np.zeros(1)
        du = np.zeros((2, self.ny))
        dc = np.zeros((2, self.ny))
        ip = ctypes.POINTER(ctypes.c_int)
        J = self._lib.orc_adjoint(self._h, int(n), masks.ctypes.data_as(ctypes.POINTER(ctypes.c_uint)), len(ox),
                                  ox.ctypes.data_as(ip), oy.ctypes.data_as(ip), _dptr(tg), _dptr(wt),
                                  _dptr(dtau), _dptr(du), _dptr(dc))
        if J < 0:
            raise ValueError("oracle adjoint: needs Zou-He ports and no decay, and the trajectory in host memory")
        self.t += int(n)
        return J, float(dtau[0]), du, dc

    def diagnostics(self, open_mask):
        out = np.zeros(4)
        self._lib.orc_diagnostics(self._h, ctypes.c_uint(int(open_mask) & 0xFFFFFFFF), _dptr(out))
        return out


def schedule_fn(period=None, states=None, fixed=None):
    """Valve word of step t: fixed, or states[(t // period) % len(states)]."""
    if fixed is not None:
        return lambda t: int(fixed)
    states = [int(s) for s in states]
    return lambda t: states[(t // int(period)) % len(states)]


def from_problem(prob, **over):
    """Build an OracleLattice from a problem dict of the seeded generators."""
    kw = dict(tau_f=prob["tau"], tau_g=prob["tau_c"], w0=prob.get("w0", 1.0 / 3.0),
              ports=prob["ports"], edge_u=prob["edge_u"], edge_C=prob["edge_C"],
              decay=prob.get("decay", 0.0), wall_scheme=prob.get("wall_scheme", 0))
    kw.update(over)
    return OracleLattice(prob["solid"], **kw)
