"""The D3Q64 finite-volume step on the GPU against the oracle's: FP64 at 1e-12 in corrector
parity mode (a fixed number of passes) on periodic, transmissive and walled boxes, through
single launches and captured graphs, the stored state compared coefficient by coefficient
with the oracle's populations; FP32 against the FP64 oracle; conservation on a periodic box;
the bench workload checked on sampled cells after its first step."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import paper_2203_05477_gb300 as pond  # noqa: E402
from paper_2203_05477_gb300 import inputs as I  # noqa: E402
from tests.common import gpu_primitive, max_rel, oracle_for, rel_l1  # noqa: E402

KW64 = dict(tau=1e-5, fixed_iters=3, max_iter=8)


def he(k, x):
    return [np.ones_like(x), x, x * x - 1.0, x ** 3 - 3.0 * x][k]


def hermite3(f, order):
    """Hermite moments of D3Q64 populations in the library's packed order."""
    c, _, _ = O.lattice(3)
    cols = []
    for n in range(order + 1):
        for j in range(n + 1):
            for t in range(j + 1):
                s, r = j - t, n - j
                cols.append(f @ (he(r, c[:, 0]) * he(s, c[:, 1]) * he(t, c[:, 2])))
    return np.stack(cols, 1)


def pair(pb, cfl=0.3, precision="fp64", **kw):
    gs = pond.Solver3(pb, precision=precision, cfl=cfl, **kw)
    gs.set_primitive()
    os_ = oracle_for(pb, cfl=cfl, **kw)
    return gs, os_


def compare(gs, os_, tol=1e-12):
    (r, mx, my, mz, E), _ = gs.moments(totals=False)
    ro, mxo, myo, mzo, Eo = os_.conserved()
    assert max_rel(r, ro) <= tol and max_rel(E, Eo) <= tol
    scale = max(np.abs(mxo).max(), np.abs(myo).max(), np.abs(mzo).max(), np.sqrt(np.abs(Eo * ro).max()))
    for a, b in ((mx, mxo), (my, myo), (mz, mzo)):
        assert np.abs(a - b).max() <= tol * scale
    cf, cg, fr = gs.state()
    fo, go, uo, To = os_.regauged_state()
    Af, Ag = hermite3(fo, 3), hermite3(go, 2)
    mach = np.sqrt((uo ** 2).sum(1) / To)
    order_f = np.array([0] + [1] * 3 + [2] * 6 + [3] * 10)
    cond = (1.0 + mach)[:, None] ** order_f[None, :]
    allow_f = 10 * tol * np.abs(ro)[:, None] * np.maximum(1.0, np.abs(Af) / np.abs(ro)[:, None]) + 1e-14 * np.abs(ro)[:, None] * cond
    assert (np.abs(cf - Af) <= allow_f).all(), np.abs(cf - Af).max()
    e_scale = (np.abs(ro) * np.abs(To))[:, None]
    allow_g = 10 * tol * e_scale * np.maximum(1.0, np.abs(Ag) / e_scale) + 1e-14 * e_scale * cond[:, :10]
    assert (np.abs(cg - Ag) <= allow_g).all(), np.abs(cg - Ag).max()
    assert max_rel(fr[:, 3], To) <= tol
    for a in range(3):
        assert np.abs(fr[:, a] - uo[:, a]).max() <= tol * max(1.0, np.abs(uo).max(), np.sqrt(To.max()))
    for g_, o_ in zip(gs.face_gauges(), os_.face_gauges()):
        assert max_rel(g_[:, 3], o_[:, 3]) <= 10 * tol
        assert np.abs(g_[:, :3] - o_[:, :3]).max() <= 10 * tol * max(1.0, np.abs(o_[:, :3]).max())


def walled_box(n, seed):
    rng = np.random.default_rng(seed)
    pb = I.smooth_periodic_3d(n, n, n, seed=seed, amp=0.2)
    pb.rho = pb.rho * np.exp(0.2 * rng.uniform(-1, 1, pb.ncell))
    pb.bc = (I.REFLECTIVE,) * 6
    return pb


CASES = [
    ("periodic_5x4x3", lambda: I.smooth_periodic_3d(5, 4, 3, seed=8, amp=0.2)),
    ("octants_4", lambda: I.octants_3d(4, seed=2)),
    ("walled_3", lambda: walled_box(3, 6)),
    ("tube_z_12", lambda: I.shock_tube_3d((1.0, 0.3, 1.0), (0.4, -0.5, 0.3), 1.4, 12, axis=2, nt=2)),
    ("mixed_bc_6x5x4", lambda: _mixed()),
    ("anisotropic_5x4x3", lambda: _anisotropic()),
]


def _anisotropic():
    """Cells of three different sizes (dx = 0.2, dy = 0.125, dz = 0.4)."""
    pb = I.smooth_periodic_3d(5, 4, 3, seed=9, amp=0.2)
    pb.y1, pb.z1 = 0.5, 1.2
    return pb


def _mixed():
    pb = I.smooth_periodic_3d(6, 5, 4, seed=3, amp=0.2)
    pb.bc = (I.TRANSMISSIVE, I.TRANSMISSIVE, I.REFLECTIVE, I.REFLECTIVE, I.PERIODIC, I.PERIODIC)
    return pb


@pytest.mark.parametrize("limiter", [0, 1], ids=["vanleer", "minmod"])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_fp64_parity(name, make, limiter):
    gs, os_ = pair(make(), limiter=limiter, **KW64)
    for chunk in (1, 3):
        gs.step(chunk)
        os_.step(chunk)
        d, st = gs.sync(), os_.stats()
        assert d["steps"] == st["steps"] and d["face_iters"] == st["face_iters"]
        assert d["fallbacks"] == st["fallbacks"] and d["nonphysical"] == st["nonphysical"] == 0
        assert d["t"] == pytest.approx(st["t"], rel=1e-13)
        compare(gs, os_)


def test_graph_replays():
    gs, os_ = pair(I.smooth_periodic_3d(4, 3, 3, seed=1, amp=0.15), **KW64)
    for chunk in (32, 2):
        gs.step(chunk)
        os_.step(chunk)
        assert gs.sync()["steps"] == os_.stats()["steps"]
        compare(gs, os_)


def test_fp32_against_fp64_oracle():
    # the spherical explosion on 8^3 cells (the random octant problems at 6^3 cells fail in
    # the oracle itself for most draws: under-resolved jumps of up to 100 in density)
    pb = I.spherical_blast_3d(8)
    kw = dict(tau=1e-5, max_iter=16)
    gs = pond.Solver3(pb, precision="fp32", cfl=0.3, tol=1e-6, **kw)
    gs.set_primitive()
    os_ = oracle_for(pb, cfl=0.3, tol=1e-6, **kw)
    gs.step(6)
    os_.step(6)
    assert gs.sync()["nonphysical"] == 0
    r, ux, uy, uz, p = gpu_primitive(gs)
    ro, uxo, uyo, uzo, po = os_.primitive()
    assert rel_l1(r, ro) <= 1e-4 and rel_l1(p, po) <= 1e-4
    sp, spo = np.sqrt(ux ** 2 + uy ** 2 + uz ** 2), np.sqrt(uxo ** 2 + uyo ** 2 + uzo ** 2)
    assert np.abs(sp - spo).sum() / spo.sum() <= 2e-4


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_periodic_box_conserves(precision, tol):
    pb = I.smooth_periodic_3d(16, 12, 10, seed=4, amp=0.2)
    gs = pond.Solver3(pb, precision=precision, tau=1e-5, cfl=0.3, max_iter=16)
    gs.set_primitive()
    _, t0 = gs.moments()
    gs.step(40)
    _, t1 = gs.moments()
    assert gs.sync()["status"] == pond.POND_OK
    assert abs(t1[0] - t0[0]) <= tol * t0[0] and abs(t1[4] - t0[4]) <= tol * t0[4]
    for k in (1, 2, 3):
        assert abs(t1[k] - t0[k]) <= tol * t0[0]


def test_full_size_sampled_first_step():
    """The bench workload (the spherical explosion on 128^3 cells, FP32 and FP64) on sampled
    cells: one step depends only on a radius-2 neighbourhood, so the oracle runs it on
    patches cut from the same initial condition with the full grid's first time step."""
    n, cfl = 128, 0.3
    pb = I.spherical_blast_3d(n)
    T = pb.p / pb.rho
    dt = cfl / ((np.sqrt(T) * 2.3344142183389773) / pb.dx).max()
    rng = np.random.default_rng(1)
    X = I.cell_centres(n, -1, 1)
    # cells on the sphere's surface (where the step is non-trivial), and random ones
    surf = [(int(i), int(j), int(k)) for i, j, k in rng.integers(0, n, (400, 3))
            if abs(np.sqrt(X[i] ** 2 + X[j] ** 2 + X[k] ** 2) - 0.4) < 2.0 / n][:5]
    samples = surf + [(int(i), int(j), int(k)) for i, j, k in rng.integers(0, n, (2, 3))] + [(0, 0, 0), (n - 1, 64, 3)]
    results = {}
    for prec in ("fp64", "fp32"):
        gs = pond.Solver3(pb, precision=prec, tau=1e-5, cfl=cfl, fixed_iters=3, max_iter=8)
        gs.set_primitive()
        gs.step(1)
        d = gs.sync()
        assert d["status"] == pond.POND_OK and d["t"] == pytest.approx(dt, rel=1e-6)
        results[prec] = gs.moments(totals=False)[0]
        gs.close()
    m = 3
    for (i, j, k) in samples:
        lo = [max(0, v - m) for v in (i, j, k)]
        hi = [min(n, v + m + 1) for v in (i, j, k)]
        sub = lambda a: np.asarray(a).reshape(n, n, n)[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]].ravel()
        ext = [h - l for l, h in zip(lo, hi)]
        patch = I.Problem3(ext[0], ext[1], ext[2], 0, ext[0] * pb.dx, 0, ext[1] * pb.dy, 0, ext[2] * pb.dz, pb.gamma,
                           sub(pb.rho), sub(pb.ux), sub(pb.uy), sub(pb.uz), sub(pb.p))
        os_ = oracle_for(patch, tau=1e-5, cfl=cfl, fixed_iters=3, max_iter=8)
        os_.force_dt(dt)
        os_.step(1)
        ro = os_.conserved()
        kp = ((k - lo[2]) * ext[1] + (j - lo[1])) * ext[0] + (i - lo[0])
        kg = (k * n + j) * n + i
        for fld in range(5):
            ref = ro[fld][kp]
            scale = max(abs(ref), abs(ro[0][kp]), abs(ro[4][kp]))
            assert abs(results["fp64"][fld][kg] - ref) <= 1e-12 * scale, ("fp64", i, j, k, fld)
            assert abs(results["fp32"][fld][kg] - ref) <= 1e-5 * scale, ("fp32", i, j, k, fld)


def test_abi_round_trips():
    """Face frames written and read back, device-side moments equal to host-side ones, and
    the compensated totals equal to the volume-weighted sums of the fields."""
    pb = I.octants_3d(5, seed=2)
    gs = pond.Solver3(pb, precision="fp64", tau=1e-5, cfl=0.3, max_iter=16)
    gs.set_primitive()
    gs.step(2)
    xg, yg, zg = gs.face_gauges()
    rng = np.random.default_rng(0)
    new = [g * (1.0 + 0.01 * rng.uniform(-1, 1, g.shape)) for g in (xg, yg, zg)]
    gs.set_face_gauges(*new)
    for a, b in zip(gs.face_gauges(), new):
        np.testing.assert_array_equal(a, b)
    gs.set_face_gauges(None, None, zg)       # NULL arrays are skipped
    got = gs.face_gauges()
    np.testing.assert_array_equal(got[0], new[0])
    np.testing.assert_array_equal(got[2], zg)
    fields, tot = gs.moments()
    dev = [torch.empty(gs.ncell, dtype=torch.float64, device="cuda") for _ in range(5)]
    tot_d = np.zeros(5)
    gs.moments_device(dev, tot_d)
    torch.cuda.synchronize()
    for f, d in zip(fields, dev):
        np.testing.assert_array_equal(f, d.cpu().numpy())
    vol = pb.dx * pb.dy * pb.dz
    for t_, f in zip(tot, fields):
        assert abs(t_ - f.sum() * vol) <= 1e-13 * np.abs(f).sum() * vol
    np.testing.assert_array_equal(tot, tot_d)
    # the calls of the other grids refuse a 3D state
    assert gs.lib.pond_moments(gs.h, None, None, None, None, None, 0) == pond.POND_ERR_INVALID_ARG
    assert gs.lib.pond_set_primitive(gs.h, None, None, None, None, 0) == pond.POND_ERR_INVALID_ARG
    buf = np.zeros(4 * xg.shape[0])
    assert gs.lib.pond_get_face_gauges(gs.h, buf.ctypes.data, None) == pond.POND_ERR_INVALID_ARG


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_every_3d_variant(precision):
    """The D3Q64 face kernel's tile variants and the cell kernel's block variants (the
    autotuner's search space): in FP64 parity mode every one matches the oracle at 1e-12 on a
    box that leaves ragged tiles for every shape; in FP32 they agree with each other to FP32
    rounding.  Tuning restores the state it times on and keeps a valid choice."""
    pb = I.smooth_periodic_3d(9, 6, 5, seed=8, amp=0.2) if precision == "fp64" else I.spherical_blast_3d(12)
    kw = KW64 if precision == "fp64" else dict(tau=1e-5, max_iter=16, tol=1e-6)
    gs = pond.Solver3(pb, precision=precision, cfl=0.3, **kw)
    names = gs.variants()
    nf = sum(1 for n in names if n.startswith("face3"))
    nc = sum(1 for n in names if n.startswith("cell3"))
    assert nf >= 3 and nc >= 3 and nf + nc == len(names), names
    ref = None
    if precision == "fp64":
        os_ = oracle_for(pb, cfl=0.3, **kw)
        os_.step(3)
    for f, c in [(f, 0) for f in range(nf)] + [(0, c) for c in range(1, nc)]:
        gs.set_variants(face=f, cell=c)
        gs.set_primitive()
        gs.step(3)
        d = gs.sync()
        assert d["steps"] == 3 and d["nonphysical"] == 0, (names[f], names[nf + c], d)
        if precision == "fp64":
            compare(gs, os_)
        else:
            prims = [np.asarray(a) for a in gpu_primitive(gs)]
            if ref is None:
                ref = prims
            for a, b in zip(prims, ref):
                assert rel_l1(a, b) <= 1e-5, (names[f], names[nf + c], rel_l1(a, b))
    # the tuner restores the state it times on and keeps a valid choice
    gs.set_variants(0, 0)
    gs.set_primitive()
    gs.step(2)
    before = [np.asarray(a).copy() for a in gs.state()]
    r = gs.autotune(steps=2)
    assert 0 <= r["face"] < nf and 0 <= r["cell"] < nc and len(r["ms"]) == nf + nc
    for a, b in zip(gs.state(), before):
        assert np.array_equal(np.asarray(a), b)
    gs.close()
