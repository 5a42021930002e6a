"""FP64 CPU oracle for the regularized Particles-on-Demand finite-volume step.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline leg of
the benchmark are the only callers.  The product library never imports this package
and shares no code with it (see ``pond_oracle.c`` for the paper passages each
function follows).  ``riemann.py`` holds the exact Riemann solution used to pin the
oracle on shock tubes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pond_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

BC_TRANSMISSIVE, BC_PERIODIC, BC_INFLOW, BC_REFLECTIVE = 0, 1, 2, 3
VANLEER, MINMOD = 0, 1


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (IEEE round-to-nearest, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC",
           "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_create.restype = ctypes.c_void_p
        lib.oracle_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ip, dp, ip, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_int]
        lib.oracle_create3.restype = ctypes.c_void_p
        lib.oracle_create3.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ip, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int]
        lib.oracle_set_primitive3.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, dp]
        lib.oracle_conserved3.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, dp]
        lib.oracle_face_gauges3.argtypes = [ctypes.c_void_p, dp, dp, dp]
        lib.oracle_set_face_gauges3.argtypes = [ctypes.c_void_p, dp, dp, dp]
        lib.oracle_free.argtypes = [ctypes.c_void_p]
        lib.oracle_set_primitive.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
        lib.oracle_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.oracle_step.restype = ctypes.c_int
        lib.oracle_sl_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.oracle_sl_step.restype = ctypes.c_int
        lib.oracle_conserved.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
        lib.oracle_regauged_state.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
        lib.oracle_raw_state.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
        lib.oracle_set_state.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
        lib.oracle_face_gauges.argtypes = [ctypes.c_void_p, dp, dp]
        lib.oracle_set_face_gauges.argtypes = [ctypes.c_void_p, dp, dp]
        lib.oracle_stats.argtypes = [ctypes.c_void_p, dp, dp, ctypes.POINTER(ctypes.c_longlong)]
        lib.oracle_lattice.argtypes = [ctypes.c_int, dp, dp, dp]
        lib.oracle_lattice.restype = ctypes.c_int
        lib.oracle_grad_transform.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_double,
                                              dp, ctypes.c_double, dp]
        lib.oracle_limiter.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
        lib.oracle_limiter.restype = ctypes.c_double
        lib.oracle_force_dt.argtypes = [ctypes.c_void_p, ctypes.c_double]
        lib.oracle_set_equilibration.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.oracle_grad_transform_eq.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_double,
                                                 dp, ctypes.c_double, dp]
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def lattice(D: int):
    """Lattice speeds c [Q, D], weights W [Q] and T_L (Table I, Eq. wi; D3Q64 as the
    three-dimensional tensor product)."""
    lib = _load()
    c = np.zeros((64, D))
    w = np.zeros(64)
    tl = np.zeros(1)
    q = lib.oracle_lattice(D, _dp(c), _dp(w), _dp(tl))
    return c[:q].copy(), w[:q].copy(), float(tl[0])


def grad_transform(D: int, order: int, f_in, u_in, T_in: float, u_out, T_out: float) -> np.ndarray:
    """Eq. (f_transformed) with Eqs. (a0)-(a3): populations f_in in frame (u_in, T_in)
    re-expressed in frame (u_out, T_out); order 3 (f) or 2 (g)."""
    lib = _load()
    f_in = _f64(f_in)
    out = np.zeros_like(f_in)
    ui = _f64(np.atleast_1d(u_in))
    uo = _f64(np.atleast_1d(u_out))
    lib.oracle_grad_transform(D, order, _dp(f_in), _dp(ui), float(T_in), _dp(uo), float(T_out), _dp(out))
    return out


def regularized_transform(D: int, order: int, f_in, u_in, T_in: float, u_out, T_out: float,
                          equilibrate: bool) -> np.ndarray:
    """The regularized transformation with Grad's projection (equilibrate False, as
    grad_transform) or with the fast moments set to the equilibrium's (Sec. II.C)."""
    lib = _load()
    f_in = _f64(f_in)
    out = np.zeros_like(f_in)
    ui = _f64(np.atleast_1d(u_in))
    uo = _f64(np.atleast_1d(u_out))
    lib.oracle_grad_transform_eq(D, order, int(bool(equilibrate)), _dp(f_in), _dp(ui), float(T_in), _dp(uo),
                                 float(T_out), _dp(out))
    return out


def limiter(kind: int, a: float, b: float) -> float:
    return float(_load().oracle_limiter(kind, float(a), float(b)))


class Solver:
    """The FP64 oracle solver: one instance per problem.

    Grid of nx (x ny (x nz)) cells, D = 1 (D1Q4), 2 (D2Q16) or 3 (D3Q64).  ``bc`` lists
    x-lo, x-hi, y-lo, y-hi (and z-lo, z-hi in 3D); ``inflow`` is a 4x4 array of
    (rho, ux, uy, p) per side and ``inflow_range`` a 4x2 array of [lo, hi) cell ranges
    along that side (1D and 2D only).
    """

    def __init__(self, D, nx, ny=1, nz=1, *, dx, dy=None, dz=None, gamma, tau, cfl, t_end=0.0,
                 bc=(0, 0, 0, 0), inflow=None, inflow_range=None, limiter=VANLEER,
                 tol=1e-12, max_iter=50, fixed_iters=0):
        self.lib = _load()
        self.D, self.nx, self.ny, self.nz = D, nx, (ny if D >= 2 else 1), (nz if D == 3 else 1)
        _, w, _ = lattice(D)
        self.Q = len(w)
        if D == 3:
            bc6 = tuple(bc) + (0,) * (6 - len(bc))
            self.h = self.lib.oracle_create3(nx, self.ny, self.nz, float(dx), float(dy if dy is not None else dx),
                                             float(dz if dz is not None else dx), float(gamma), float(tau),
                                             float(cfl), float(t_end), (ctypes.c_int * 6)(*[int(b) for b in bc6]),
                                             int(limiter), float(tol), int(max_iter), int(fixed_iters))
            if not self.h:
                raise ValueError("oracle_create3 failed")
            return
        bc_arr = (ctypes.c_int * 4)(*[int(b) for b in bc])
        infl = _f64(np.zeros((4, 4)) if inflow is None else inflow).reshape(16)
        rng = np.zeros((4, 2), dtype=np.int32) if inflow_range is None else np.asarray(inflow_range, dtype=np.int32)
        rng_arr = (ctypes.c_int * 8)(*[int(v) for v in rng.reshape(8)])
        self._infl = infl
        self.h = self.lib.oracle_create(D, nx, self.ny, float(dx), float(dy if dy is not None else dx),
                                        float(gamma), float(tau), float(cfl), float(t_end), bc_arr,
                                        _dp(infl), rng_arr, int(limiter), float(tol), int(max_iter),
                                        int(fixed_iters))
        if not self.h:
            raise ValueError("oracle_create failed")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.oracle_free(h)
            self.h = None

    @property
    def ncell(self):
        return self.nx * self.ny * self.nz

    def set_primitive3(self, rho, ux, uy, uz, p):
        n = self.ncell
        rho, ux, uy, uz, p = (_f64(np.ravel(a)) for a in (rho, ux, uy, uz, p))
        assert all(a.size == n for a in (rho, ux, uy, uz, p))
        self.lib.oracle_set_primitive3(self.h, _dp(rho), _dp(ux), _dp(uy), _dp(uz), _dp(p))

    def set_primitive(self, rho, ux, uy, p):
        n = self.ncell
        rho, ux, p = (_f64(np.ravel(a)) for a in (rho, ux, p))
        uy = _f64(np.zeros(n) if uy is None else np.ravel(uy))
        assert rho.size == n and ux.size == n and p.size == n and uy.size == n
        self.lib.oracle_set_primitive(self.h, _dp(rho), _dp(ux), _dp(uy), _dp(p))

    def step(self, n: int) -> int:
        return int(self.lib.oracle_step(self.h, int(n)))

    def sl_step(self, n: int) -> int:
        """n steps of the semi-Lagrangian realization (Sec. III.A) instead of the FV step."""
        return int(self.lib.oracle_sl_step(self.h, int(n)))

    def conserved(self):
        """rho, mx, my, E per cell (1D, 2D); rho, mx, my, mz, E in 3D."""
        n = self.ncell
        if self.D == 3:
            out = [np.zeros(n) for _ in range(5)]
            self.lib.oracle_conserved3(self.h, *(_dp(a) for a in out))
            return out
        out = [np.zeros(n) for _ in range(4)]
        self.lib.oracle_conserved(self.h, *(_dp(a) for a in out))
        return out  # rho, mx, my, E

    def primitive(self):
        """rho, ux, uy, p (1D, 2D); rho, ux, uy, uz, p in 3D."""
        cv = 1.0 / (self.gamma - 1.0)
        if self.D == 3:
            rho, mx, my, mz, E = self.conserved()
            T = (E - 0.5 * (mx * mx + my * my + mz * mz) / rho) / (cv * rho)
            return rho, mx / rho, my / rho, mz / rho, rho * T
        rho, mx, my, E = self.conserved()
        ux, uy = mx / rho, my / rho
        T = (E - 0.5 * (mx * mx + my * my) / rho) / (cv * rho)
        return rho, ux, uy, rho * T

    gamma = None

    def regauged_state(self):
        n = self.ncell
        f = np.zeros((n, self.Q)); g = np.zeros((n, self.Q))
        u = np.zeros((n, self.D)); T = np.zeros(n)
        self.lib.oracle_regauged_state(self.h, _dp(f), _dp(g), _dp(u), _dp(T))
        return f, g, u, T

    def raw_state(self):
        n = self.ncell
        f = np.zeros((n, self.Q)); g = np.zeros((n, self.Q))
        u = np.zeros((n, self.D)); T = np.zeros(n)
        self.lib.oracle_raw_state(self.h, _dp(f), _dp(g), _dp(u), _dp(T))
        return f, g, u, T

    def set_state(self, f, g, u, T):
        f, g, u, T = (_f64(a) for a in (f, g, u, T))
        self.lib.oracle_set_state(self.h, _dp(f), _dp(g), _dp(u), _dp(T))

    def face_gauges(self):
        D = self.D
        if D == 3:
            nx, ny, nz = self.nx, self.ny, self.nz
            out = [np.zeros(((nx + 1) * ny * nz, 4)), np.zeros((nx * (ny + 1) * nz, 4)),
                   np.zeros((nx * ny * (nz + 1), 4))]
            self.lib.oracle_face_gauges3(self.h, *(_dp(a) for a in out))
            return tuple(out)
        xg = np.zeros(((self.nx + 1) * self.ny, D + 1))
        yg = np.zeros((self.nx * (self.ny + 1), D + 1)) if D == 2 else np.zeros((1, D + 1))
        self.lib.oracle_face_gauges(self.h, _dp(xg), _dp(yg))
        return xg, (yg if D == 2 else None)

    def set_face_gauges(self, xg, yg=None, zg=None):
        if self.D == 3:
            xg, yg, zg = (_f64(a) for a in (xg, yg, zg))
            self.lib.oracle_set_face_gauges3(self.h, _dp(xg), _dp(yg), _dp(zg))
            return
        xg = _f64(xg)
        yg = _f64(yg) if yg is not None else np.zeros(1)
        self.lib.oracle_set_face_gauges(self.h, _dp(xg), _dp(yg))

    def force_dt(self, dt: float):
        """Test hook: fixed time step instead of the CFL rule (dt <= 0 restores it)."""
        self.lib.oracle_force_dt(self.h, float(dt))

    def set_equilibration(self, on: bool):
        """Ablation: the equilibration alternative of Sec. II.C in every transformation."""
        self.lib.oracle_set_equilibration(self.h, int(bool(on)))

    def stats(self):
        t = np.zeros(1); dt = np.zeros(1)
        counts = (ctypes.c_longlong * 6)()
        self.lib.oracle_stats(self.h, _dp(t), _dp(dt), counts)
        keys = ("steps", "face_iters", "faces", "nonconverged", "nonphysical", "fallbacks")
        d = {k: int(v) for k, v in zip(keys, counts)}
        d["t"] = float(t[0]); d["dt"] = float(dt[0])
        return d


def make_solver(D, nx, ny=1, nz=1, *, gamma, **kw) -> Solver:
    s = Solver(D, nx, ny, nz, gamma=gamma, **kw)
    s.gamma = gamma
    return s
