"""The equilibration alternative of Sec. II.C (an ablation of Grad's projection) on the GPU
against the oracle with the same option (oracle_set_equilibration): FP64 in corrector
parity mode at 1e-12 with the same corrector pass and fallback counts, FP32 at 1e-4
relative L1, on D1Q4 and D2Q16 grids; and the runs differ from the Grad ones, so the
option reaches the kernels."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2203_05477_gb300 as pond  # noqa: E402
from paper_2203_05477_gb300 import inputs as I  # noqa: E402
from tests.common import gpu_primitive, max_rel, oracle_for, rel_l1  # noqa: E402
from tests.test_gpu_parity import compare_fp64  # noqa: E402

pytestmark = pytest.mark.gpu


def cases():
    return [
        ("sod_400", I.sod_400(), 0.5),
        ("periodic_1d_97", I.smooth_periodic(1, 97, 1, seed=5, amp=0.15), 0.3),
        ("strong_shock_120", I.paper_tube("strong_shock", 120)[0], 0.2),
        ("quadrants_29", I.quadrants_2d(29, seed=0), 0.2),
        ("lax_liu_24", I.lax_liu_2d(24), 0.2),
        ("periodic_19x13", I.smooth_periodic(2, 19, 13, seed=2, amp=0.15), 0.2),
    ]


@pytest.mark.parametrize("name,pb,cfl", cases(), ids=[c[0] for c in cases()])
def test_equilibration_fp64_parity(name, pb, cfl):
    kw = dict(tau=1e-5, cfl=cfl, fixed_iters=3, max_iter=8)
    gs = pond.Solver(pb, precision="fp64", **kw)
    gs.set_primitive()
    gs.set_equilibration(True)
    os_ = oracle_for(pb, **kw)
    os_.set_equilibration(True)
    for chunk in (1, 4):
        gs.step(chunk)
        os_.step(chunk)
        d, st = gs.sync(), os_.stats()
        assert d["steps"] == st["steps"] and d["face_iters"] == st["face_iters"] and d["fallbacks"] == st["fallbacks"]
        assert d["nonphysical"] == st["nonphysical"] == 0
        compare_fp64(gs, os_)
    # the same steps with Grad's projection end elsewhere
    gg = pond.Solver(pb, precision="fp64", **kw)
    gg.set_primitive()
    gg.step(5)
    (r_eq, _, _, E_eq), _ = gs.moments(totals=False)
    (r_gr, _, _, E_gr), _ = gg.moments(totals=False)
    assert max(max_rel(r_eq, r_gr), max_rel(E_eq, E_gr)) > 1e-9


@pytest.mark.parametrize("dim", [1, 2])
def test_equilibration_fp32_against_fp64_oracle(dim):
    pb = I.sod_400() if dim == 1 else I.quadrants_2d(32, seed=6, mach_max=1.0)
    cfl, steps = (0.5, 200) if dim == 1 else (0.2, 30)
    gs = pond.Solver(pb, precision="fp32", tau=1e-5, cfl=cfl, max_iter=16)
    gs.set_primitive()
    gs.set_equilibration(True)
    os_ = oracle_for(pb, tau=1e-5, cfl=cfl, tol=1e-6, max_iter=16)
    os_.set_equilibration(True)
    gs.step(steps)
    os_.step(steps)
    assert gs.sync()["nonphysical"] == 0
    r, ux, uy, p = gpu_primitive(gs)
    ro, uxo, uyo, po = os_.primitive()
    so = np.hypot(uxo, uyo)
    assert rel_l1(r, ro) < 1e-4 and rel_l1(p, po) < 1e-4
    assert np.abs(np.hypot(ux, uy) - so).sum() / so.sum() < 1e-4


def test_equilibration_option_is_refused_where_it_does_not_apply():
    pb = I.quadrants_2d(16, seed=0)
    s = pond.Solver(pb, precision="fp32", tau=1e-5, cfl=0.2, scheme="sl")
    with pytest.raises(pond.PondError):
        s.set_equilibration(True)
    b = pond.BatchSolver([50], [1.4], precision="fp32", tau=1e-5, cfl=0.2)
    with pytest.raises(pond.PondError):
        b.set_equilibration(True)
    g = pond.Solver(pb, precision="fp32", tau=1e-5, cfl=0.2)
    g.set_equilibration(True)
    with pytest.raises(pond.PondError):
        g.gauge_enable(True)
