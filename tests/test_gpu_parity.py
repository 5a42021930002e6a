"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element,
on the same seeded inputs.  FP64 mode: 1e-12 relative in corrector parity mode (a fixed
number of corrector passes, so rounding cannot change iteration counts).  FP32 mode:
1e-4 relative L1 on density, pressure and velocity with shocks within one cell."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2203_05477_gb300 as pond  # noqa: E402
from paper_2203_05477_gb300 import inputs as I  # noqa: E402
from tests.common import gpu_primitive, hermite_of_pops, max_rel, oracle_for, rel_l1  # noqa: E402

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def gpu_for(pb, **kw):
    s = pond.Solver(pb, **kw)
    s.set_primitive()
    return s


def compare_fp64(gs, os_, tol=FP64_TOL, what="conserved", faces=True):
    (r, mx, my, E), _ = gs.moments(totals=False)
    ro, mxo, myo, Eo = os_.conserved()
    scale_m = max(np.abs(mxo).max(), np.abs(myo).max(), np.sqrt(np.abs(Eo * ro).max()))
    assert max_rel(r, ro) <= tol, ("rho", max_rel(r, ro))
    assert np.abs(mx - mxo).max() <= tol * scale_m, ("mx", np.abs(mx - mxo).max() / scale_m)
    assert np.abs(my - myo).max() <= tol * scale_m, ("my", np.abs(my - myo).max() / scale_m)
    assert max_rel(E, Eo) <= tol, ("E", max_rel(E, Eo))
    # the stored state: Hermite coefficients of each cell in its own frame, and the frame.
    # The oracle evaluates Eqs. (a0)-(a3) with lab-frame moments M_k, whose terms grow like
    # rho |u|^k: its coefficient of order k carries a rounding error ~ eps rho (1 + M)^k
    # (M = |u| / sqrt(T)), which bounds what can be compared at high Mach.
    cf, cg, fr = gs.state()
    fo, go, uo, To = os_.regauged_state()
    D = gs.D
    Af = hermite_of_pops(fo, D)
    Ag = hermite_of_pops(go, D)[:, : cg.shape[1]]
    mach = np.sqrt((uo ** 2).sum(1) / To)
    order = np.array([0, 1, 2, 3] if D == 1 else [0, 1, 1, 2, 2, 2, 3, 3, 3, 3])
    cond = (1.0 + mach)[:, None] ** order[None, :]
    allow_f = 10 * tol * np.abs(ro)[:, None] * np.maximum(1.0, np.abs(Af) / np.abs(ro)[:, None]) + 1e-14 * np.abs(ro)[:, None] * cond
    assert (np.abs(cf - Af) <= allow_f).all(), np.abs(cf - Af).max()
    e_scale = (np.abs(ro) * np.abs(To))[:, None]
    ng = cg.shape[1]
    allow_g = 10 * tol * e_scale * np.maximum(1.0, np.abs(Ag) / e_scale) + 1e-14 * e_scale * cond[:, :ng]
    assert (np.abs(cg - Ag) <= allow_g).all(), np.abs(cg - Ag).max()
    assert max_rel(fr[:, D], To) <= tol
    for a in range(D):
        assert np.abs(fr[:, a] - uo[:, a]).max() <= tol * max(1.0, np.abs(uo).max(), np.sqrt(To.max()))
    if not faces:
        return
    # face predictors for the next step
    xg, yg = gs.face_gauges()
    xo, yo = os_.face_gauges()
    assert max_rel(xg[:, -1], xo[:, -1]) <= 10 * tol
    if D == 2:
        assert max_rel(yg[:, -1], yo[:, -1]) <= 10 * tol


def parity_cases_1d():
    sod = I.sod_400()
    lax, _ = I.paper_tube("lax", 150)
    strong, _ = I.paper_tube("strong_shock", 120)
    jet, _ = I.paper_tube("jet_1d", 160)
    periodic = I.smooth_periodic(1, 97, 1, seed=5, amp=0.15)
    tiny = I.shock_tube((1.0, 0.3, 1.0), (0.5, -0.2, 0.4), 1.4, 3)
    return [("sod_400", sod, 0.5), ("lax", lax, 0.2), ("strong", strong, 0.2), ("jet", jet, 0.2),
            ("periodic_97", periodic, 0.3), ("tiny_3", tiny, 0.3)]


@pytest.mark.parametrize("name,pb,cfl", parity_cases_1d(), ids=[c[0] for c in parity_cases_1d()])
@pytest.mark.parametrize("steps", [1, 12])
def test_fp64_parity_1d(name, pb, cfl, steps):
    kw = dict(tau=1e-5, cfl=cfl, fixed_iters=3, max_iter=8)
    gs = gpu_for(pb, precision="fp64", **kw)
    os_ = oracle_for(pb, **kw)
    gs.step(steps)
    os_.step(steps)
    d = gs.sync()
    st = os_.stats()
    assert d["steps"] == st["steps"]
    assert d["t"] == pytest.approx(st["t"], rel=1e-13)
    assert d["face_iters"] == st["face_iters"] and d["fallbacks"] == st["fallbacks"]
    assert d["nonphysical"] == st["nonphysical"] == 0
    compare_fp64(gs, os_)


def parity_cases_2d():
    return [
        ("quadrants_29x29", I.quadrants_2d(29, seed=0)),
        ("lax_liu_24", I.lax_liu_2d(24)),
        ("periodic_19x13", I.smooth_periodic(2, 19, 13, seed=2, amp=0.15)),
        ("shocked_interface_37x13", I.shocked_interface_2d(37, 13, seed=1)),
        ("jet_24", I.jet_2d(24, seed=3)),
        ("strip_1x6", I.Problem(2, 1, 6, 0, 1, 0, 6, 1.4, np.linspace(1, 2, 6), np.zeros(6), np.linspace(-0.2, 0.2, 6),
                                np.ones(6), bc=(I.PERIODIC, I.PERIODIC, I.TRANSMISSIVE, I.TRANSMISSIVE))),
    ]


@pytest.mark.parametrize("name,pb", parity_cases_2d(), ids=[c[0] for c in parity_cases_2d()])
def test_fp64_parity_2d(name, pb):
    kw = dict(tau=1e-5, cfl=0.2, fixed_iters=3, max_iter=8)
    gs = gpu_for(pb, precision="fp64", **kw)
    os_ = oracle_for(pb, **kw)
    for chunk in (1, 3):
        gs.step(chunk)
        os_.step(chunk)
        d = gs.sync()
        st = os_.stats()
        assert d["steps"] == st["steps"] and d["face_iters"] == st["face_iters"]
        assert d["fallbacks"] == st["fallbacks"]
        compare_fp64(gs, os_)


def test_fp64_parity_converged_corrector():
    """Convergence mode (tol 1e-10): iteration counts may differ by rounding, so the
    bound is the corrector tolerance, not round-off."""
    pb = I.sod_400()
    kw = dict(tau=1e-5, cfl=0.5, t_end=0.2, tol=1e-10, max_iter=16)
    gs = gpu_for(pb, precision="fp64", **kw)
    os_ = oracle_for(pb, **kw)
    gs.step(700)
    os_.step(700)
    d = gs.sync()
    assert d["t"] == pytest.approx(0.2, abs=1e-14) and d["steps"] == os_.stats()["steps"]
    compare_fp64(gs, os_, tol=1e-8)


def shock_cell(r, start):
    return start + int(np.argmax(np.abs(np.diff(r[start:]))))


def test_fp32_against_fp64_oracle_sod():
    pb = I.sod_400()
    gs = gpu_for(pb, precision="fp32", tau=1e-5, cfl=0.5, t_end=0.2)
    os_ = oracle_for(pb, tau=1e-5, cfl=0.5, t_end=0.2, tol=1e-10)
    gs.step(700)
    os_.step(700)
    d = gs.sync()
    assert d["status"] == pond.POND_OK, d
    r, u, _, p = gpu_primitive(gs)
    ro, uo, _, po = os_.primitive()
    assert rel_l1(r, ro) < 1e-4 and rel_l1(p, po) < 1e-4
    assert np.abs(u - uo).sum() / np.abs(uo).sum() < 1e-4
    assert abs(shock_cell(r, 300) - shock_cell(ro, 300)) <= 1


@pytest.mark.parametrize("seed", [0, 3])
def test_fp32_against_fp64_oracle_quadrants(seed):
    pb = I.quadrants_2d(32, seed=seed)
    gs = gpu_for(pb, precision="fp32", tau=1e-5, cfl=0.2)
    os_ = oracle_for(pb, tau=1e-5, cfl=0.2, tol=1e-10)
    gs.step(40)
    os_.step(40)
    d = gs.sync()
    assert d["status"] == pond.POND_OK, d
    r, ux, uy, p = gpu_primitive(gs)
    ro, uxo, uyo, po = os_.primitive()
    assert rel_l1(r, ro) < 1e-4 and rel_l1(p, po) < 1e-4
    sp, spo = np.hypot(ux, uy), np.hypot(uxo, uyo)
    assert np.abs(sp - spo).sum() / np.abs(spo).sum() < 1e-4


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
@pytest.mark.parametrize("dim", [1, 2])
def test_conservation_periodic(precision, tol, dim):
    pb = I.smooth_periodic(dim, 64 if dim == 1 else 24, 20, seed=7, amp=0.15)
    gs = gpu_for(pb, precision=precision, tau=1e-4, cfl=0.3)
    _, t0 = gs.moments()
    gs.step(200 if dim == 1 else 40)
    _, t1 = gs.moments()
    assert gs.sync()["status"] == pond.POND_OK
    for k in range(4):
        if dim == 1 and k == 2:
            continue
        assert abs(t1[k] - t0[k]) <= tol * max(abs(t0[k]), t0[0]), (k, t0[k], t1[k])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_uniform_mach80_any_gauge(precision):
    n, g, T = 16, 5.0 / 3.0, 0.02
    u = 80 * np.sqrt(g * T)
    N = n * n
    pb = I.Problem(2, n, n, 0, 1, 0, 1, g, np.full(N, 2.0), np.full(N, u), np.full(N, -0.4 * u), np.full(N, 2.0 * T),
                   bc=(I.PERIODIC,) * 4)
    gs = gpu_for(pb, precision=precision, tau=1e-5, cfl=0.2, max_iter=40,
                 tol=1e-9 if precision == "fp64" else 1e-6)
    xg, yg = gs.face_gauges()
    xg[:, 0] += 0.5 * np.sqrt(T)
    yg[:, -1] *= 1.7
    gs.set_face_gauges(xg, yg)
    gs.step(20)
    d = gs.sync()
    assert d["status"] == pond.POND_OK, d
    r, ux, uy, p = gpu_primitive(gs)
    tol = 1e-9 if precision == "fp64" else 2e-5
    assert max_rel(r, np.full(N, 2.0)) < tol and max_rel(p, np.full(N, 2.0 * T)) < 10 * tol
    assert np.abs(ux - u).max() < tol * u and np.abs(uy + 0.4 * u).max() < tol * u


def test_graph_replay_matches_single_launches():
    pb = I.quadrants_2d(40, seed=3)
    a = gpu_for(pb, precision="fp32", tau=1e-5, cfl=0.2)
    b = gpu_for(pb, precision="fp32", tau=1e-5, cfl=0.2)
    a.step(70)            # two captured 32-step graphs + 6 launches
    for _ in range(70):
        b.step(1)
    ca, ga, fa = a.state()
    cb, gb, fb = b.state()
    assert np.array_equal(ca, cb) and np.array_equal(ga, gb) and np.array_equal(fa, fb)
    assert a.launch_count() == b.launch_count()


def test_nonphysical_input_is_reported():
    pb = I.sod_400()
    gs = pond.Solver(pb, precision="fp64", tau=1e-5, cfl=0.5)
    rho = pb.rho.copy()
    rho[17] = -1.0
    gs.set_primitive(rho=rho)
    d = gs.sync()
    assert d["status"] == pond.POND_ERR_NONPHYSICAL and d["first_bad_cell"] == 17
    # the device and the context stay usable
    ok = gpu_for(pb, precision="fp64", tau=1e-5, cfl=0.5)
    ok.step(3)
    assert ok.sync()["status"] == pond.POND_OK


C_MAX = 2.3344142183389773  # the largest D1Q4 node, sqrt(3 + sqrt(6))


def sampled_first_step(pb, samples, cfl, m=4):
    """A bench-size workload (FP32 and FP64, in the autotuned launch configuration the bench
    uses) checked on sampled cells: one step depends only on a radius-3 neighbourhood, so
    the oracle runs that step on (2m+1)^2 patches cut from the same initial condition, with
    the full grid's first time step and the grid's own sides where a patch touches them
    (periodic axes are cut with wrap-around)."""
    nx, ny = pb.nx, pb.ny
    T = pb.p / pb.rho
    rate = max(((np.abs(pb.ux) + np.sqrt(T) * C_MAX) / pb.dx).max(), ((np.abs(pb.uy) + np.sqrt(T) * C_MAX) / pb.dy).max())
    dt = cfl / rate
    results = {}
    for prec in ("fp64", "fp32"):
        gs = gpu_for(pb, precision=prec, tau=1e-5, cfl=cfl, fixed_iters=3, max_iter=8)
        tuned = gs.autotune(steps=1)
        assert not tuned["from_cache"]
        gs.step(1)
        d = gs.sync()
        assert d["dt"] > 0 and d["nonphysical"] == 0, d
        results[prec] = gs.moments(totals=False)[0]
        gs.close()
    per_y = pb.bc[2] == I.PERIODIC
    for (i, j) in samples:
        i0, i1 = max(0, i - m), min(nx, i + m + 1)
        js = np.arange(j - m, j + m + 1) % ny if per_y else np.arange(max(0, j - m), min(ny, j + m + 1))
        grid = lambda a: a.reshape(ny, nx)[js][:, i0:i1].ravel()
        bc = [pb.bc[0] if i0 == 0 else I.TRANSMISSIVE, pb.bc[1] if i1 == nx else I.TRANSMISSIVE,
              I.TRANSMISSIVE if per_y or js[0] != 0 else pb.bc[2], I.TRANSMISSIVE if per_y or js[-1] != ny - 1 else pb.bc[3]]
        inflow = np.zeros((4, 4))
        rng = np.zeros((4, 2), dtype=np.int64)
        if bc[0] == I.INFLOW:
            inflow[0] = pb.inflow[0]
            rows = np.nonzero((js >= pb.inflow_range[0][0]) & (js < pb.inflow_range[0][1]))[0]
            if rows.size:
                assert rows.size == rows[-1] - rows[0] + 1
                rng[0] = (rows[0], rows[-1] + 1)
        assert bc[1] != I.INFLOW and bc[2] != I.INFLOW and bc[3] != I.INFLOW
        pw, ph = i1 - i0, len(js)
        patch = I.Problem(2, pw, ph, 0, pw * pb.dx, 0, ph * pb.dy, pb.gamma, grid(pb.rho), grid(pb.ux), grid(pb.uy),
                          grid(pb.p), bc=tuple(bc), inflow=inflow, inflow_range=rng)
        os_ = oracle_for(patch, tau=1e-5, cfl=cfl, fixed_iters=3, max_iter=8)
        os_.force_dt(dt)
        os_.step(1)
        assert os_.stats()["nonphysical"] == 0
        ro = os_.conserved()
        k_patch = int(np.nonzero(js == j)[0][0]) * pw + (i - i0)
        k = j * nx + i
        for fld in range(4):
            ref = ro[fld][k_patch]
            scale = max(abs(ref), abs(ro[0][k_patch]), abs(ro[3][k_patch]))
            assert abs(results["fp64"][fld][k] - ref) <= FP64_TOL * scale, ("fp64", i, j, fld)
            assert abs(results["fp32"][fld][k] - ref) <= 1e-5 * scale, ("fp32", i, j, fld)


def test_full_size_sampled_first_step():
    """Configuration 2 at the bench's size: 1024^2 quadrants, seed 0."""
    n = 1024
    pb = I.quadrants_2d(n, seed=0)
    rng = np.random.default_rng(0)
    samples = [(int(i), int(j)) for i, j in rng.integers(0, n, (6, 2))] + [(511, 511), (512, 512), (0, 0), (n - 1, 700)]
    sampled_first_step(pb, samples, 0.2)


def test_full_size_sampled_first_step_shocked_interface():
    """Configuration 4 at its stated size: the shocked perturbed interface on 4096 x 1024
    cells (left inflow at the post-shock state, periodic in y), sampled at the inflow side,
    across the shock (x = 0.5) and the interface (x ~ 1), at the periodic seam and at
    random cells."""
    pb = I.shocked_interface_2d(4096, 1024, seed=0)
    rng = np.random.default_rng(1)
    samples = [(int(i), int(j)) for i, j in zip(rng.integers(0, 4096, 6), rng.integers(0, 1024, 6))]
    samples += [(0, 0), (0, 1023), (1, 500), (511, 3), (512, 1020), (4095, 0), (4095, 777)]
    r = pb.rho.reshape(1024, 4096)
    for j in (0, 100, 255, 600):
        i_if = int(np.argmax(r[j, 600:] > 1.5)) + 600   # first heavy-gas cell of row j
        samples += [(i_if - 1, j), (i_if, j)]
    sampled_first_step(pb, samples, 0.2)


def test_full_size_sampled_first_step_jet():
    """Configuration 5 at its stated size: the Mach-80 jet on 4096^2 cells, sampled at the
    edges of the inflow band, next to it on the inflow side, in the corners and at random
    cells."""
    n = 4096
    pb = I.jet_2d(n, seed=0)
    lo, hi = int(pb.inflow_range[0][0]), int(pb.inflow_range[0][1])
    rng = np.random.default_rng(2)
    samples = [(int(i), int(j)) for i, j in rng.integers(0, n, (4, 2))]
    samples += [(0, lo - 1), (0, lo), (0, (lo + hi) // 2), (0, hi - 1), (0, hi), (1, lo), (2, hi - 1), (0, 0),
                (n - 1, n - 1), (0, n - 1)]
    sampled_first_step(pb, samples, 0.2)


@pytest.mark.parametrize("name,pb,cfl", [
    ("sod_400", I.sod_400(), 0.5),
    ("quadrants_29x29", I.quadrants_2d(29, seed=0), 0.2),
    ("lax_liu_24", I.lax_liu_2d(24), 0.2),
], ids=["sod_400", "quadrants_29x29", "lax_liu_24"])
def test_fp64_parity_minmod(name, pb, cfl):
    """The second limiter the paper names (Sec. III.B.3), minmod, in every slope."""
    kw = dict(tau=1e-5, cfl=cfl, fixed_iters=3, max_iter=8, limiter=1)
    gs = gpu_for(pb, precision="fp64", **kw)
    os_ = oracle_for(pb, **kw)
    for chunk in (1, 5):
        gs.step(chunk)
        os_.step(chunk)
        d, st = gs.sync(), os_.stats()
        assert d["steps"] == st["steps"] and d["face_iters"] == st["face_iters"]
        assert d["nonphysical"] == st["nonphysical"] == 0
        compare_fp64(gs, os_)


def test_fp32_minmod_against_fp64_oracle():
    pb = I.quadrants_2d(48, seed=0)
    kw = dict(tau=1e-5, cfl=0.2, max_iter=16, limiter=1)
    gs = gpu_for(pb, precision="fp32", tol=1e-6, **kw)
    os_ = oracle_for(pb, tol=1e-6, **kw)
    gs.step(10)
    os_.step(10)
    assert gs.sync()["nonphysical"] == 0
    r, _, _, p = gpu_primitive(gs)
    ro, _, _, po = os_.primitive()
    assert rel_l1(r, ro) <= 1e-4 and rel_l1(p, po) <= 1e-4


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_compensated_totals_against_exact_sum(precision):
    """The double-double totals of pond_moments (the conserved moments of Sec. II.B summed
    over the grid, times the cell area) against the exactly rounded sum (math.fsum) of the
    per-cell fields the same call returns, on ill-conditioned fields: densities alternating
    1e16 and O(1), with momenta of the heavy cells cancelling in pairs, so that a plain
    double sum loses every light cell's contribution.  Bound: one rounding of the result."""
    import math
    nx, ny = 129, 67
    N = nx * ny
    k = np.arange(N)
    heavy = k % 2 == 0
    sign = np.where((k // 2) % 2 == 0, 1.0, -1.0)
    rho = np.where(heavy, 1e16, 1.0 + 0.37 * (k % 7))
    ux = np.where(heavy, sign, 0.3 + 0.011 * (k % 5))
    uy = np.where(heavy, -sign * 0.5, -0.2 + 0.013 * (k % 3))
    p = 0.5 * rho
    pb = I.Problem(2, nx, ny, 0, 1.0, 0, 0.75, 1.4, rho, ux, uy, p, bc=(I.PERIODIC,) * 4)
    gs = gpu_for(pb, precision=precision, tau=1e-5, cfl=0.2)
    fields, tot = gs.moments(totals=True)
    vol = pb.dx * pb.dy
    naive_lost = 0
    for q in range(4):
        exact = math.fsum(fields[q].tolist()) * vol
        assert abs(tot[q] - exact) <= np.spacing(abs(exact)), (q, tot[q], exact)
        naive_lost += int(float(np.cumsum(fields[q])[-1]) * vol != exact)
    assert naive_lost >= 2   # the fields defeat a plain left-to-right double sum


@pytest.mark.parametrize("name,pb,steps", [
    ("shocked_interface_64x16", I.shocked_interface_2d(64, 16, seed=0), 120),
    ("jet_32", I.jet_2d(32, seed=0), 20),
], ids=["shocked_interface_64x16", "jet_32"])
def test_fp32_configurations_4_and_5_against_fp64_oracle(name, pb, steps):
    """Configurations 4 and 5 downscaled (the shocked interface at 64 x 16 over 120 steps;
    the Mach-80 jet at 32^2 over 20 of the ~22 steps the method survives there), FP32 with
    the bench's stopping rule against the FP64 oracle with the same rule: relative L1 of rho,
    p and speed within 1e-4, or within twice the oracle's own change when the pass limit
    moves by one where that is larger (faces that reach the limit without converging end on
    an iterate that depends on where the iteration stops); where a row or column has one
    clearly steepest density jump, the FP32 run's lies within one cell of the oracle's."""
    kw = dict(tau=1e-5, cfl=0.2, tol=1e-6, max_iter=16)
    gs = gpu_for(pb, precision="fp32", **kw)
    gs.step(steps)
    d = gs.sync()
    assert d["nonphysical"] == 0, d
    os_ = oracle_for(pb, **kw)
    os_.step(steps)
    ro, uxo, uyo, po = os_.primitive()
    so = np.hypot(uxo, uyo)

    def err(r, ux, uy, p):
        return max(rel_l1(r, ro), rel_l1(p, po), np.abs(np.hypot(ux, uy) - so).sum() / max(so.sum(), 1e-300))

    prim = gpu_primitive(gs)
    e = err(*prim)
    # shock positions: in every row and column where the oracle's steepest density jump
    # stands out (every jump more than 3 cells away from it is below 80% of it), the FP32
    # run's steepest jump lies within one cell of it
    r2, ro2 = prim[0].reshape(pb.ny, pb.nx), ro.reshape(pb.ny, pb.nx)
    off, used = 0, 0
    for a, b in ((r2, ro2), (r2.T, ro2.T)):
        g, go = np.abs(np.diff(a, axis=1)), np.abs(np.diff(b, axis=1))
        for k in range(go.shape[0]):
            i = int(np.argmax(go[k]))
            rest = np.concatenate([go[k, :max(0, i - 3)], go[k, i + 4:]])
            if rest.size and rest.max() >= 0.8 * go[k, i]:
                continue
            used += 1
            off = max(off, abs(int(np.argmax(g[k])) - i))
    print("%s: shock positions checked in %d rows and columns, largest offset %d" % (name, used, off))
    assert used >= 10 and off <= 1, (used, off)
    bound = 1e-4
    if os_.stats()["nonconverged"]:
        for mi in (15, 17):
            o2 = oracle_for(pb, **dict(kw, max_iter=mi))
            o2.step(steps)
            bound = max(bound, 2.0 * err(*o2.primitive()))
    print("%s: FP32 vs oracle %.2e, bound %.2e, oracle non-converged faces %d" % (name, e, bound, os_.stats()["nonconverged"]))
    assert e <= bound, (e, bound, os_.stats()["nonconverged"])
