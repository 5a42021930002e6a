"""The C-ABI library builds for sm_103a, loads without a GPU, exports every entry point
that include/pond.h declares, and validates its arguments before touching the device."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2203_05477_gb300 as pond
from paper_2203_05477_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return ctypes.CDLL(pond.library_path())


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(pond_\w+)\s*\(", text))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert "pond_init" in names and "pond_step" in names and "pond_moments" in names
    for n in names:
        assert hasattr(lib, n), n


def _grid(dim=1, nx=8):
    g = pond.pond_grid()
    g.dim, g.nx, g.ny, g.x0, g.x1, g.y0, g.y1 = dim, nx, 1 if dim == 1 else nx, 0.0, 1.0, 0.0, 1.0
    return g


def _opts():
    o = pond.pond_options()
    o.precision, o.limiter, o.cfl, o.tol, o.max_iter = pond.POND_FP64, 0, 0.2, 1e-10, 16
    return o


@pytest.mark.parametrize("velset,dim,gamma,want", [
    (pond.POND_D1Q3, 1, 1.4, pond.POND_ERR_UNSUPPORTED),
    (pond.POND_D2Q9, 2, 1.4, pond.POND_ERR_UNSUPPORTED),
    (pond.POND_D1Q4, 2, 1.4, pond.POND_ERR_INVALID_ARG),     # dim mismatch
    (pond.POND_D2Q16, 2, 2.5, pond.POND_ERR_UNSUPPORTED),    # gamma > 1 + 2/D
    (pond.POND_D1Q4, 1, 1.0, pond.POND_ERR_INVALID_ARG),
])
def test_init_rejects_bad_arguments(lib, velset, dim, gamma, want):
    L = pond._load()
    g, o = _grid(dim), _opts()
    h = ctypes.c_void_p()
    st = L.pond_init(ctypes.byref(g), velset, gamma, 1e-5, ctypes.byref(o), ctypes.byref(h))
    assert st == want
    assert not h.value
    assert L.pond_last_error()


def test_null_arguments(lib):
    L = pond._load()
    h = ctypes.c_void_p()
    assert L.pond_init(None, pond.POND_D1Q4, 1.4, 1e-5, None, ctypes.byref(h)) == pond.POND_ERR_INVALID_ARG
    assert L.pond_step(None, 1) == pond.POND_ERR_INVALID_ARG
    assert L.pond_sync(None, None) == pond.POND_ERR_INVALID_ARG


def _grid3(n=4, bc=(0,) * 6):
    g = pond.pond_grid3()
    g.nx, g.ny, g.nz = n, n, n
    g.x0, g.x1, g.y0, g.y1, g.z0, g.z1 = 0.0, 1.0, 0.0, 1.0, 0.0, 1.0
    for k in range(6):
        g.bc[k] = bc[k]
    return g


@pytest.mark.parametrize("change,want", [
    (lambda g, o: None, "gamma"),                                               # gamma 1.7 > 5/3
    (lambda g, o: setattr(g, "nz", 0), pond.POND_ERR_INVALID_ARG),
    (lambda g, o: g.bc.__setitem__(4, 2), pond.POND_ERR_INVALID_ARG),          # no inflow sides in 3D
    (lambda g, o: g.bc.__setitem__(0, 1), pond.POND_ERR_INVALID_ARG),          # unpaired periodic side
    (lambda g, o: setattr(o, "scheme", pond.POND_SL), pond.POND_ERR_UNSUPPORTED),
    (lambda g, o: setattr(o, "learned", 1), pond.POND_ERR_UNSUPPORTED),
], ids=["gamma", "empty", "inflow", "periodic_pair", "sl", "learned"])
def test_init3_rejects_bad_arguments(lib, change, want):
    L = pond._load()
    g, o = _grid3(), _opts()
    change(g, o)
    gamma = 1.7 if want == "gamma" else 1.4
    h = ctypes.c_void_p()
    st = L.pond_init3(ctypes.byref(g), gamma, 1e-5, ctypes.byref(o), ctypes.byref(h))
    assert st == (pond.POND_ERR_UNSUPPORTED if want == "gamma" else want)
    assert not h.value and L.pond_last_error()


def test_d3q64_goes_through_init3(lib):
    L = pond._load()
    g, o = _grid(2), _opts()
    h = ctypes.c_void_p()
    assert L.pond_init(ctypes.byref(g), pond.POND_D3Q64, 1.4, 1e-5, ctypes.byref(o), ctypes.byref(h)) == pond.POND_ERR_UNSUPPORTED
    assert L.pond_init3(None, 1.4, 1e-5, None, ctypes.byref(h)) == pond.POND_ERR_INVALID_ARG
    assert L.pond_set_primitive3(None, None, None, None, None, None, 0) == pond.POND_ERR_INVALID_ARG
    assert L.pond_moments3(None, None, None, None, None, None, None, 0) == pond.POND_ERR_INVALID_ARG


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes structures and constants of the binding have the sizes, field offsets and
    values that a C compiler gives the declarations of include/pond.h."""
    structs = {"pond_grid": pond.pond_grid, "pond_grid3": pond.pond_grid3, "pond_options": pond.pond_options,
               "pond_diag": pond.pond_diag, "pond_tune_result": pond.pond_tune_result}
    consts = ["POND_OK", "POND_ERR_INVALID_ARG", "POND_ERR_UNSUPPORTED", "POND_ERR_OOM", "POND_ERR_CUDA",
              "POND_ERR_NONPHYSICAL", "POND_ERR_NOT_CONVERGED", "POND_ERR_TIMEOUT", "POND_D1Q3", "POND_D1Q4",
              "POND_D2Q16", "POND_D2Q9", "POND_D3Q64", "POND_FP64", "POND_FP32", "POND_VANLEER", "POND_MINMOD",
              "POND_FV", "POND_SL", "POND_TUNE_MAX"]
    lines = ['#include <stdio.h>', '#include "pond.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, field, name, field))
    for c in consts:
        lines.append('printf("%s %%ld\\n", (long)%s);' % (c, c))
    for c in ("POND_MLP_PARAMS", "POND_MLP_FEATURES", "POND_MLP_PAIR_STRIDE"):
        lines.append('printf("%s %%ld\\n", (long)%s);' % (c, c))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                              text=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got["%s size" % name]) == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(got["%s.%s" % (name, field)]) == getattr(cls, field).offset, (name, field)
    for c in consts:
        assert int(got[c]) == getattr(pond, c), c
    assert int(got["POND_MLP_PARAMS"]) == pond.MLP_PARAMS
    assert int(got["POND_MLP_FEATURES"]) == pond.MLP_FEATURES
    assert int(got["POND_MLP_PAIR_STRIDE"]) == pond.MLP_PAIR_STRIDE


def test_wait_timeout_check_validates_before_touching_the_device(lib):
    assert pond.pond_wait_timeout_check(0, None) == pond.POND_ERR_INVALID_ARG
    assert pond.pond_wait_timeout_check(1 << 25, None) == pond.POND_ERR_INVALID_ARG
