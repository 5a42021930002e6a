"""Python binding of the GB300 regularized Particles-on-Demand library (libpond.so).

The binding only marshals arguments: every step of the method runs in the library's
CUDA kernels.  PyTorch provides device memory (the caching allocator is handed to the
library through the allocator hook of ``pond_options``) and the CUDA stream.  The
functions ``pond_*`` are the C entry points of ``include/pond.h`` with the same names;
``Solver`` wraps them for numpy/torch callers.  There is no CPU fallback: without the
compiled library every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import inputs  # noqa: F401  (problem generators, no method arithmetic)

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libpond.so")
_lock = threading.Lock()
_lib = None

POND_OK, POND_ERR_INVALID_ARG, POND_ERR_UNSUPPORTED, POND_ERR_OOM, POND_ERR_CUDA = 0, 1, 2, 3, 4
POND_ERR_NONPHYSICAL, POND_ERR_NOT_CONVERGED, POND_ERR_TIMEOUT = 5, 6, 7
POND_D1Q3, POND_D1Q4, POND_D2Q16, POND_D2Q9, POND_D3Q64 = 0, 1, 2, 3, 4
POND_FP64, POND_FP32 = 0, 1
POND_VANLEER, POND_MINMOD = 0, 1
POND_FV, POND_SL = 0, 1
MLP_PARAMS, MLP_FEATURES, MLP_PAIR_STRIDE = 8336, 48, 52

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class pond_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double), ("y0", ctypes.c_double),
                ("y1", ctypes.c_double), ("bc", ctypes.c_int * 4),
                ("inflow", (ctypes.c_double * 4) * 4), ("inflow_lo", ctypes.c_int64 * 4),
                ("inflow_hi", ctypes.c_int64 * 4)]


class pond_grid3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double), ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("z0", ctypes.c_double), ("z1", ctypes.c_double), ("bc", ctypes.c_int * 6)]


class pond_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("limiter", ctypes.c_int), ("cfl", ctypes.c_double),
                ("t_end", ctypes.c_double), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("fixed_iters", ctypes.c_int), ("strict_convergence", ctypes.c_int),
                ("learned", ctypes.c_int), ("stream", ctypes.c_void_p), ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p), ("scheme", ctypes.c_int)]


class pond_diag(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("dt", ctypes.c_double), ("steps", ctypes.c_int64),
                ("face_solves", ctypes.c_int64), ("face_iters", ctypes.c_int64),
                ("nonconverged", ctypes.c_int64), ("fallbacks", ctypes.c_int64),
                ("nonphysical", ctypes.c_int64), ("first_bad_cell", ctypes.c_int64),
                ("flags", ctypes.c_uint32), ("staged_tma", ctypes.c_int64)]


POND_TUNE_MAX = 32


class pond_tune_result(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("face", ctypes.c_int), ("cell", ctypes.c_int), ("tube", ctypes.c_int),
                ("from_cache", ctypes.c_int), ("ms", ctypes.c_double * POND_TUNE_MAX)]


class PondError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("pond status %d: %s" % (status, msg))
        self.status = status


def library_path() -> str:
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise ImportError("libpond.so is not built (run __graft_entry__.build() or "
                              "paper_2203_05477_gb300._build.build()); there is no CPU fallback")
        lib = ctypes.CDLL(_LIB_PATH)
        vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
        sigs = {
            "pond_init": (ctypes.c_int, [ctypes.POINTER(pond_grid), ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, ctypes.POINTER(pond_options), ctypes.POINTER(vp)]),
            "pond_set_primitive": (ctypes.c_int, [vp, vp, vp, vp, vp, ctypes.c_int]),
            "pond_init3": (ctypes.c_int, [ctypes.POINTER(pond_grid3), ctypes.c_double, ctypes.c_double,
                                          ctypes.POINTER(pond_options), ctypes.POINTER(vp)]),
            "pond_set_primitive3": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, ctypes.c_int]),
            "pond_moments3": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, vp, ctypes.c_int]),
            "pond_get_face_gauges3": (ctypes.c_int, [vp, vp, vp, vp]),
            "pond_set_face_gauges3": (ctypes.c_int, [vp, vp, vp, vp]),
            "pond_step": (ctypes.c_int, [vp, ctypes.c_int64]),
            "pond_step_timed": (ctypes.c_int, [vp, ctypes.c_int64, vp]),
            "pond_moments": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, ctypes.c_int]),
            "pond_get_state": (ctypes.c_int, [vp, vp, vp, vp]),
            "pond_get_face_gauges": (ctypes.c_int, [vp, vp, vp]),
            "pond_set_face_gauges": (ctypes.c_int, [vp, vp, vp]),
            "pond_sync": (ctypes.c_int, [vp, ctypes.POINTER(pond_diag)]),
            "pond_launch_count": (ctypes.c_int64, [vp]),
            "pond_init_batch": (ctypes.c_int, [ctypes.c_int64, vp, vp, vp, ctypes.c_double,
                                               ctypes.POINTER(pond_options), ctypes.POINTER(vp)]),
            "pond_batch_times": (ctypes.c_int, [vp, vp, vp]),
            "pond_batch_status": (ctypes.c_int, [vp, vp, vp]),
            "pond_gauge_collect": (ctypes.c_int, [vp, ctypes.c_int64, vp, ctypes.c_int64, ctypes.c_int, vp]),
            "pond_gauge_train": (ctypes.c_int, [vp, vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_float, vp]),
            "pond_gauge_enable": (ctypes.c_int, [vp, ctypes.c_int]),
            "pond_set_equilibration": (ctypes.c_int, [vp, ctypes.c_int]),
            "pond_wait_timeout_check": (ctypes.c_int, [ctypes.c_int64, vp]),
            "pond_gauge_set_gate": (ctypes.c_int, [vp, ctypes.c_float]),
            "pond_gauge_set_trust": (ctypes.c_int, [vp, ctypes.c_float]),
            "pond_gauge_set_params": (ctypes.c_int, [vp, vp]),
            "pond_gauge_get_params": (ctypes.c_int, [vp, vp]),
            "pond_gauge_save": (ctypes.c_int, [vp, vp, ctypes.POINTER(ctypes.c_size_t)]),
            "pond_gauge_load": (ctypes.c_int, [vp, vp, ctypes.c_size_t]),
            "pond_mlp_forward": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int64, vp, vp]),
            "pond_mlp_gradient": (ctypes.c_int, [vp, vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int64, vp, vp, vp]),
            "pond_autotune": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_char_p, ctypes.POINTER(pond_tune_result)]),
            "pond_variant_count": (ctypes.c_int, [vp]),
            "pond_variant_name": (ctypes.c_char_p, [vp, ctypes.c_int]),
            "pond_set_variants": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
            "pond_destroy": (None, [vp]),
            "pond_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def __getattr__(name):
    # pond_* entry points of the C ABI under their own names
    if name.startswith("pond_"):
        return getattr(_load(), name)
    raise AttributeError(name)


def _check(st):
    if st != POND_OK:
        raise PondError(st, _load().pond_last_error().decode())


def _ptr(a):
    """Device or host pointer of a torch tensor / numpy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


class _TorchAllocator:
    """Hands torch's CUDA caching allocator to the library (device memory only)."""

    def __init__(self, device, stream):
        import torch
        self.torch = torch
        self.device = device
        self.stream = stream
        self.live = {}

        def alloc(nbytes, ctx):
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), device=self.device, stream=self.stream)
            except Exception:
                return None
            self.live[p] = nbytes
            return p

        def free(ptr, ctx):
            if ptr and ptr in self.live:
                del self.live[ptr]
                torch.cuda.caching_allocator_delete(ptr)

        self.alloc_fn = ALLOC_FN(alloc)
        self.free_fn = FREE_FN(free)


class Solver:
    """One PonD problem on the current CUDA device (see ``inputs.Problem``)."""

    def __init__(self, problem, *, tau, cfl, precision="fp64", limiter=POND_VANLEER, t_end=0.0,
                 tol=None, max_iter=16, fixed_iters=0, strict=False, stream=None, torch_alloc=True,
                 scheme="fv"):
        import torch
        lib = _load()
        self.problem = problem
        self.D = problem.dim
        self.nx, self.ny = problem.nx, (problem.ny if problem.dim == 2 else 1)
        self.prec = POND_FP32 if precision in ("fp32", POND_FP32) else POND_FP64
        g = pond_grid()
        g.dim = problem.dim
        g.nx, g.ny = problem.nx, self.ny
        g.x0, g.x1, g.y0, g.y1 = problem.x0, problem.x1, problem.y0, problem.y1
        for k in range(4):
            g.bc[k] = int(problem.bc[k])
            g.inflow_lo[k] = int(problem.inflow_range[k][0])
            g.inflow_hi[k] = int(problem.inflow_range[k][1])
            for q in range(4):
                g.inflow[k][q] = float(problem.inflow[k][q])
        self.device = torch.cuda.current_device()
        # a stream of our own: torch's default stream is the legacy one, which cannot be
        # captured into a CUDA graph
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        o = pond_options()
        o.precision = self.prec
        o.limiter = int(limiter)
        o.cfl = float(cfl)
        o.t_end = float(t_end)
        o.tol = float(tol if tol is not None else (1e-10 if self.prec == POND_FP64 else 1e-6))
        o.max_iter = int(max_iter)
        o.fixed_iters = int(fixed_iters)
        o.strict_convergence = int(bool(strict))
        o.scheme = POND_SL if scheme in ("sl", POND_SL) else POND_FV
        o.stream = self.stream.cuda_stream
        self._alloc = _TorchAllocator(self.device, self.stream) if torch_alloc else None
        if self._alloc:
            o.alloc = self._alloc.alloc_fn
            o.free = self._alloc.free_fn
        self._grid, self._opts = g, o
        self.h = ctypes.c_void_p()
        velset = POND_D1Q4 if problem.dim == 1 else POND_D2Q16
        _check(lib.pond_init(ctypes.byref(g), velset, float(problem.gamma), float(tau), ctypes.byref(o),
                             ctypes.byref(self.h)))
        self.lib = lib
        self.ncell = self.nx * self.ny
        self.nfc = 4 if self.D == 1 else 10
        self.ngc = 3 if self.D == 1 else 6

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.lib.pond_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_primitive(self, rho=None, ux=None, uy=None, p=None):
        pb = self.problem
        vals = [pb.rho if rho is None else rho, pb.ux if ux is None else ux,
                (pb.uy if uy is None else uy) if self.D == 2 else None, pb.p if p is None else p]
        on_dev = not isinstance(vals[0], np.ndarray)
        if not on_dev:
            vals = [None if v is None else np.ascontiguousarray(v, dtype=np.float64) for v in vals]
        self._keep = vals
        _check(self.lib.pond_set_primitive(self.h, *[_ptr(v) for v in vals], int(on_dev)))

    def step(self, n=1):
        _check(self.lib.pond_step(self.h, int(n)))

    def step_timed(self, n):
        """n steps with every kernel timed by CUDA events on the stream: (face ms, cell ms)."""
        ms = np.zeros(2)
        _check(self.lib.pond_step_timed(self.h, int(n), _ptr(ms)))
        return float(ms[0]), float(ms[1])

    def moments(self, totals=True):
        out = [np.zeros(self.ncell) for _ in range(4)]
        tot = np.zeros(4)
        _check(self.lib.pond_moments(self.h, *[_ptr(a) for a in out], _ptr(tot) if totals else None, 0))
        return out, tot

    def moments_device(self, outs, totals=None):
        """Conserved fields into device tensors (each may be None); totals into a host array."""
        _check(self.lib.pond_moments(self.h, *[_ptr(a) for a in outs], _ptr(totals), 1))

    def state(self):
        cf = np.zeros((self.ncell, self.nfc))
        cg = np.zeros((self.ncell, self.ngc))
        fr = np.zeros((self.ncell, self.D + 1))
        _check(self.lib.pond_get_state(self.h, _ptr(cf), _ptr(cg), _ptr(fr)))
        return cf, cg, fr

    def face_gauges(self):
        D = self.D
        xg = np.zeros(((self.nx + 1) * self.ny, D + 1))
        yg = np.zeros((self.nx * (self.ny + 1), D + 1)) if D == 2 else None
        _check(self.lib.pond_get_face_gauges(self.h, _ptr(xg), _ptr(yg)))
        return xg, yg

    def set_face_gauges(self, xg, yg=None):
        xg = np.ascontiguousarray(xg, dtype=np.float64)
        yg = None if yg is None else np.ascontiguousarray(yg, dtype=np.float64)
        _check(self.lib.pond_set_face_gauges(self.h, _ptr(xg), _ptr(yg)))

    def sync(self, raise_on_error=False):
        d = pond_diag()
        st = self.lib.pond_sync(self.h, ctypes.byref(d))
        out = {f: getattr(d, f) for f, _ in pond_diag._fields_}
        out["status"] = st
        if raise_on_error:
            _check(st)
        elif st not in (POND_OK, POND_ERR_NONPHYSICAL, POND_ERR_NOT_CONVERGED):
            _check(st)
        return out

    def launch_count(self):
        return int(self.lib.pond_launch_count(self.h))

    # ---- kernel-variant autotuning
    def variants(self):
        """Names of the compiled kernel variants (face then cell variants; tube variants for a batch)."""
        return [self.lib.pond_variant_name(self.h, i).decode() for i in range(self.lib.pond_variant_count(self.h))]

    def autotune(self, steps=3, cache=None):
        """Times every variant on the current state (restored afterwards) and keeps the fastest;
        returns the choice and the per-variant mean ms per launch."""
        r = pond_tune_result()
        path = None if cache is None else os.fsencode(cache)
        _check(self.lib.pond_autotune(self.h, int(steps), path, ctypes.byref(r)))
        names = self.variants()
        return {"face": r.face, "cell": r.cell, "tube": r.tube, "from_cache": bool(r.from_cache),
                "ms": {names[i]: r.ms[i] for i in range(r.n)}}

    def set_variants(self, face=0, cell=0, tube=0):
        _check(self.lib.pond_set_variants(self.h, int(face), int(cell), int(tube)))

    def set_equilibration(self, on=True):
        """The equilibration alternative of Sec. II.C instead of Grad's projection (ablation)."""
        _check(self.lib.pond_set_equilibration(self.h, int(bool(on))))

    # ---- learned face-gauge predictor (D2Q16)
    def gauge_collect(self, n_steps, cap, every=4):
        """Runs n_steps plain steps and returns the sampled training pairs (device tensor)."""
        import torch
        pairs = torch.empty((int(cap), MLP_PAIR_STRIDE), dtype=torch.float32, device="cuda")
        n = ctypes.c_int64()
        _check(self.lib.pond_gauge_collect(self.h, int(n_steps), pairs.data_ptr(), int(cap), int(every), ctypes.byref(n)))
        return pairs[: n.value]

    def gauge_train(self, pairs, epochs=10, batch=4096, lr=1e-3):
        pairs = pairs.contiguous()
        losses = np.zeros(int(epochs), dtype=np.float32)
        _check(self.lib.pond_gauge_train(self.h, pairs.data_ptr(), int(pairs.shape[0]), int(epochs), int(batch),
                                         float(lr), _ptr(losses)))
        return losses

    def gauge_enable(self, on=True, gate=None, trust=None):
        if gate is not None:
            _check(self.lib.pond_gauge_set_gate(self.h, float(gate)))
        if trust is not None:
            _check(self.lib.pond_gauge_set_trust(self.h, float(trust)))
        _check(self.lib.pond_gauge_enable(self.h, int(bool(on))))

    def gauge_params(self):
        p = np.zeros(MLP_PARAMS, dtype=np.float32)
        _check(self.lib.pond_gauge_get_params(self.h, _ptr(p)))
        return p

    def gauge_save(self) -> bytes:
        n = ctypes.c_size_t(0)
        _check(self.lib.pond_gauge_save(self.h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(self.lib.pond_gauge_save(self.h, buf, ctypes.byref(n)))
        return buf.raw

    def gauge_load(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(self.lib.pond_gauge_load(self.h, buf, len(blob)))

    def set_gauge_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == MLP_PARAMS
        _check(self.lib.pond_gauge_set_params(self.h, _ptr(p)))


class Solver3(Solver):
    """One PonD problem on a D3Q64 grid (see ``inputs.Problem3``): the finite-volume scheme."""

    def __init__(self, problem, *, tau, cfl, precision="fp64", limiter=POND_VANLEER, t_end=0.0,
                 tol=None, max_iter=16, fixed_iters=0, strict=False, stream=None, torch_alloc=True):
        import torch
        lib = _load()
        self.problem = problem
        self.D = 3
        self.nx, self.ny, self.nz = problem.nx, problem.ny, problem.nz
        self.prec = POND_FP32 if precision in ("fp32", POND_FP32) else POND_FP64
        g = pond_grid3()
        g.nx, g.ny, g.nz = problem.nx, problem.ny, problem.nz
        g.x0, g.x1, g.y0, g.y1, g.z0, g.z1 = problem.x0, problem.x1, problem.y0, problem.y1, problem.z0, problem.z1
        for k in range(6):
            g.bc[k] = int(problem.bc[k])
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        o = pond_options()
        o.precision = self.prec
        o.limiter = int(limiter)
        o.cfl = float(cfl)
        o.t_end = float(t_end)
        o.tol = float(tol if tol is not None else (1e-10 if self.prec == POND_FP64 else 1e-6))
        o.max_iter = int(max_iter)
        o.fixed_iters = int(fixed_iters)
        o.strict_convergence = int(bool(strict))
        o.scheme = POND_FV
        o.stream = self.stream.cuda_stream
        self._alloc = _TorchAllocator(self.device, self.stream) if torch_alloc else None
        if self._alloc:
            o.alloc = self._alloc.alloc_fn
            o.free = self._alloc.free_fn
        self._grid, self._opts = g, o
        self.h = ctypes.c_void_p()
        _check(lib.pond_init3(ctypes.byref(g), float(problem.gamma), float(tau), ctypes.byref(o), ctypes.byref(self.h)))
        self.lib = lib
        self.ncell = self.nx * self.ny * self.nz
        self.nfc, self.ngc = 20, 10

    def set_primitive(self, rho=None, ux=None, uy=None, uz=None, p=None):
        pb = self.problem
        vals = [pb.rho if rho is None else rho, pb.ux if ux is None else ux, pb.uy if uy is None else uy,
                pb.uz if uz is None else uz, pb.p if p is None else p]
        on_dev = not isinstance(vals[0], np.ndarray)
        if not on_dev:
            vals = [np.ascontiguousarray(v, dtype=np.float64) for v in vals]
        self._keep = vals
        _check(self.lib.pond_set_primitive3(self.h, *[_ptr(v) for v in vals], int(on_dev)))

    def moments(self, totals=True):
        """(rho, mx, my, mz, E) per cell and their compensated totals over the box."""
        out = [np.zeros(self.ncell) for _ in range(5)]
        tot = np.zeros(5)
        _check(self.lib.pond_moments3(self.h, *[_ptr(a) for a in out], _ptr(tot) if totals else None, 0))
        return out, tot

    def moments_device(self, outs, totals=None):
        _check(self.lib.pond_moments3(self.h, *[_ptr(a) for a in outs], _ptr(totals), 1))

    def face_gauges(self):
        nx, ny, nz = self.nx, self.ny, self.nz
        out = (np.zeros(((nx + 1) * ny * nz, 4)), np.zeros((nx * (ny + 1) * nz, 4)), np.zeros((nx * ny * (nz + 1), 4)))
        _check(self.lib.pond_get_face_gauges3(self.h, *[_ptr(a) for a in out]))
        return out

    def set_face_gauges(self, xg, yg=None, zg=None):
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in (xg, yg, zg)]
        _check(self.lib.pond_set_face_gauges3(self.h, *[_ptr(a) for a in arrs]))


class BatchSolver(Solver):
    """Many independent 1D shock tubes (D1Q4) advanced by one persistent launch per call."""

    def __init__(self, lengths, gammas, *, tau, cfl, dx=None, precision="fp32", limiter=POND_VANLEER,
                 tol=None, max_iter=16, fixed_iters=0, stream=None, torch_alloc=True):
        import torch
        lib = _load()
        self.lengths = np.ascontiguousarray(lengths, dtype=np.int64)
        self.gammas = np.ascontiguousarray(gammas, dtype=np.float64)
        self.dxs = None if dx is None else np.ascontiguousarray(dx, dtype=np.float64)
        self.n_tubes = len(self.lengths)
        self.D = 1
        self.prec = POND_FP32 if precision in ("fp32", POND_FP32) else POND_FP64
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        o = pond_options()
        o.precision = self.prec
        o.limiter = int(limiter)
        o.cfl = float(cfl)
        o.tol = float(tol if tol is not None else (1e-10 if self.prec == POND_FP64 else 1e-6))
        o.max_iter = int(max_iter)
        o.fixed_iters = int(fixed_iters)
        o.stream = self.stream.cuda_stream
        self._alloc = _TorchAllocator(self.device, self.stream) if torch_alloc else None
        if self._alloc:
            o.alloc = self._alloc.alloc_fn
            o.free = self._alloc.free_fn
        self._opts = o
        self.h = ctypes.c_void_p()
        _check(lib.pond_init_batch(self.n_tubes, _ptr(self.lengths), _ptr(self.gammas), _ptr(self.dxs), float(tau),
                                   ctypes.byref(o), ctypes.byref(self.h)))
        self.lib = lib
        self.ncell = int(self.lengths.sum())
        self.nx, self.ny = self.ncell, 1
        self.nfc, self.ngc = 4, 3
        self.offsets = np.concatenate([[0], np.cumsum(self.lengths)])

    def set_primitive(self, rho, ux, uy=None, p=None):
        vals = [rho, ux, None, p]
        on_dev = not isinstance(rho, np.ndarray)
        if not on_dev:
            vals = [None if v is None else np.ascontiguousarray(v, dtype=np.float64) for v in vals]
        self._keep = vals
        _check(self.lib.pond_set_primitive(self.h, *[_ptr(v) for v in vals], int(on_dev)))

    def times(self):
        t = np.zeros(self.n_tubes)
        dt = np.zeros(self.n_tubes)
        _check(self.lib.pond_batch_times(self.h, _ptr(t), _ptr(dt)))
        return t, dt

    def status(self):
        st = np.zeros(self.n_tubes, dtype=np.int32)
        done = np.zeros(self.n_tubes, dtype=np.int64)
        _check(self.lib.pond_batch_status(self.h, _ptr(st), _ptr(done)))
        return st, done

    def face_gauges(self):
        g = np.zeros((int((self.lengths + 1).sum()), 2))
        _check(self.lib.pond_get_face_gauges(self.h, _ptr(g), None))
        return g, None


def mlp_forward(params, x):
    """Forward pass of the predictor network on device tensors: params [8336], x [n][>=48]."""
    import torch
    n, ld = x.shape
    out = torch.empty((n, 16), dtype=torch.float32, device=x.device)
    st = torch.cuda.current_stream().cuda_stream
    _check(_load().pond_mlp_forward(params.data_ptr(), x.data_ptr(), int(ld), int(n), out.data_ptr(), st))
    return out


def mlp_gradient(params, x, y):
    """Mean squared error and its gradient; targets in columns 48..50 of y."""
    import torch
    n, ldx = x.shape
    grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device=x.device)
    loss = torch.zeros(1, dtype=torch.float32, device=x.device)
    st = torch.cuda.current_stream().cuda_stream
    _check(_load().pond_mlp_gradient(params.data_ptr(), x.data_ptr(), int(ldx), y.data_ptr(), int(y.shape[1]), int(n),
                                     grad.data_ptr(), loss.data_ptr(), st))
    return float(loss.item()), grad
