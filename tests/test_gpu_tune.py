"""Kernel variants and the autotuner.  Every compiled variant of the face, cell and tube
kernels reproduces the FP64 oracle at 1e-12 in corrector parity mode, on sizes that leave
ragged tiles for every tile shape; FP32 variants agree with each other to FP32 rounding;
tuning restores the state it times on; a cache file short-cuts a second tuning."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2203_05477_gb300 as pond  # noqa: E402
from paper_2203_05477_gb300 import inputs as I  # noqa: E402
from tests.common import gpu_primitive, max_rel, oracle_for, rel_l1  # noqa: E402
from tests.test_gpu_batch import run_pair, small_batch  # noqa: E402
from tests.test_gpu_parity import compare_fp64, gpu_for  # noqa: E402

pytestmark = pytest.mark.gpu

KW64 = dict(tau=1e-5, cfl=0.2, fixed_iters=3, max_iter=8)


def split(names):
    """(face variants, cell variants, whole-step choices) of a grid state's variant names."""
    nf = sum(1 for n in names if n.startswith("face"))
    nc = sum(1 for n in names if n.startswith("cell"))
    return nf, nc, len(names) - nf - nc


@pytest.mark.parametrize("name,pb", [
    ("shocked_interface_37x13", I.shocked_interface_2d(37, 13, seed=1)),
    ("quadrants_29x29", I.quadrants_2d(29, seed=0)),
    ("lax_150", I.paper_tube("lax", 150)[0]),
], ids=lambda x: x if isinstance(x, str) else "")
def test_every_grid_variant_matches_oracle_fp64(name, pb):
    os_ = oracle_for(pb, **KW64)
    os_.step(4)
    gs = gpu_for(pb, precision="fp64", **KW64)
    nf, nc, ns = split(gs.variants())
    assert nf >= 3 and nc == 9 and ns >= 2
    for f in range(nf):
        for c in range(nc):
            if f and c != f % nc:
                continue  # every face variant once, every cell variant with face variant 0
            gs.set_variants(face=f, cell=c)
            gs.set_primitive()
            gs.step(4)
            d = gs.sync()
            assert d["steps"] == 4 and d["nonphysical"] == 0, (f, c, d)
            compare_fp64(gs, os_)
    # every fused step variant (faces and cell update of a tile in one kernel)
    for k in range(1, ns):
        gs.set_variants(face=0, cell=0, tube=k)
        gs.set_primitive()
        gs.step(4)
        d = gs.sync()
        st = os_.stats()
        assert d["steps"] == 4 and d["nonphysical"] == 0, (k, d)
        assert d["face_iters"] == st["face_iters"] and d["fallbacks"] == st["fallbacks"], (k, d, st)
        compare_fp64(gs, os_)


def _prims(s):
    return [np.asarray(a) for a in gpu_primitive(s)]  # rho, ux, uy, p


def test_fp32_grid_variants_agree():
    pb = I.quadrants_2d(61, seed=0)
    kw = dict(tau=1e-5, cfl=0.2, max_iter=16, tol=1e-6)
    gs = gpu_for(pb, precision="fp32", **kw)
    nf, nc, ns = split(gs.variants())
    gs.step(10)
    ref = _prims(gs)
    for f in list(range(nf)) + [(0, k) for k in range(1, ns)]:
        if isinstance(f, tuple):
            gs.set_variants(face=0, cell=0, tube=f[1])
            f = 0
        else:
            gs.set_variants(face=f, cell=f % nc)
        gs.set_primitive()
        gs.step(10)
        assert gs.sync()["nonphysical"] == 0
        got = _prims(gs)
        for a, b in zip(got, ref):
            assert rel_l1(a, b) <= 1e-5, (gs.variants()[f], rel_l1(a, b))


def test_autotune_restores_state_and_uses_cache(tmp_path):
    pb = I.quadrants_2d(64, seed=0)
    kw = dict(tau=1e-5, cfl=0.2, max_iter=16, tol=1e-6)
    gs = gpu_for(pb, precision="fp32", **kw)
    gs.step(3)
    assert gs.sync()["nonphysical"] == 0
    before = gs.state()
    gb = gs.face_gauges()
    t0 = gs.sync()["t"]
    cache = tmp_path / "tune.txt"
    r = gs.autotune(steps=2, cache=str(cache))
    assert not r["from_cache"] and len(r["ms"]) == len(gs.variants())
    assert all(v > 0 for v in r["ms"].values())
    after = gs.state()
    for a, b in zip(after, before):
        assert np.array_equal(a, b)
    for a, b in zip(gs.face_gauges(), gb):
        assert np.array_equal(a, b)
    assert gs.sync()["t"] == t0
    # the tuned solver continues like an untuned one
    ref = gpu_for(pb, precision="fp32", **kw)
    ref.step(3 + 40)
    gs.step(40)
    for a, b in zip(_prims(gs), _prims(ref)):
        assert rel_l1(a, b) <= 1e-5
    # a second solver of the same problem takes the choice from the cache without timing
    other = gpu_for(pb, precision="fp32", **kw)
    r2 = other.autotune(steps=2, cache=str(cache))
    assert r2["from_cache"] and (r2["face"], r2["cell"]) == (r["face"], r["cell"])
    assert len(cache.read_text().splitlines()) == 1


@pytest.mark.parametrize("dim", [1, 2])
def test_fused_step_graphs_and_parity(dim):
    """The fused step alternates between two sets of state planes: runs of captured 32-step
    graphs entered at either parity, and single launches, give the same state bit for bit;
    an odd number of fused steps, then the face and cell kernels, continue the same run."""
    pb = I.quadrants_2d(40, seed=3) if dim == 2 else I.paper_tube("lax", 300)[0]
    kw = dict(tau=1e-5, cfl=0.2, max_iter=16, tol=1e-6)
    a = gpu_for(pb, precision="fp32", **kw)
    b = gpu_for(pb, precision="fp32", **kw)
    ns = split(a.variants())[2]
    a.set_variants(0, 0, ns - 1)
    b.set_variants(0, 0, ns - 1)
    a.step(1)              # odd parity, then two graphs entered there, then single launches
    a.step(69)
    for _ in range(70):
        b.step(1)
    for x, y in zip(a.state(), b.state()):
        assert np.array_equal(x, y)
    for x, y in zip(a.face_gauges(), b.face_gauges()):
        assert x is None or np.array_equal(x, y)
    # switching to the separate kernels after an odd number of fused steps
    c = gpu_for(pb, precision="fp64", **KW64)
    o = oracle_for(pb, **KW64)
    c.set_variants(0, 0, 1)
    c.step(3)
    c.set_variants(0, 0, 0)
    c.step(2)
    o.step(5)
    compare_fp64(c, o)


def test_every_tube_variant_matches_oracle_fp64():
    bt = small_batch()
    gs, oracles = run_pair(bt, "fp64", 5, **KW64)
    rho0, ux0, p0 = I.tube_batch_fields(bt)
    names = gs.variants()
    assert len(names) >= 2 and all(n.startswith("tube") for n in names)
    for v in range(len(names)):
        gs.set_variants(tube=v)
        gs.set_primitive(rho0, ux0, None, p0)
        gs.step(5)
        assert gs.sync()["status"] == pond.POND_OK
        (rho, mx, _, E), _ = gs.moments()
        for k, os_ in enumerate(oracles):
            a, b = gs.offsets[k], gs.offsets[k + 1]
            ro, mo, _, Eo = os_.conserved()
            assert max_rel(rho[a:b], ro) <= 1e-12 and max_rel(E[a:b], Eo) <= 1e-12, (names[v], k)


def test_tube_autotune_restores_state():
    bt = small_batch()
    gs = pond.BatchSolver(bt.lengths, bt.gammas, precision="fp32", tau=1e-5, cfl=0.2, max_iter=16, tol=1e-6)
    rho0, ux0, p0 = I.tube_batch_fields(bt)
    gs.set_primitive(rho0, ux0, None, p0)
    gs.step(4)
    before = gs.state()
    t_before = gs.times()
    r = gs.autotune(steps=3)
    assert 0 <= r["tube"] < len(gs.variants()) and len(r["ms"]) == len(gs.variants())
    for a, b in zip(gs.state(), before):
        assert np.array_equal(a, b)
    for a, b in zip(gs.times(), t_before):
        assert np.array_equal(a, b)


def test_scratch_variants_are_the_same_arithmetic():
    """The face variants that keep the corrector's centre cells (level 1) or also its moment
    sums (level 2) in shared scratch do the same arithmetic in the same order: their states
    agree bit for bit after ten steps of a Mach-3 draw, and with the register-only variant of
    the same tile to FP32 rounding."""
    pb = I.quadrants_2d(61, seed=0)
    kw = dict(tau=1e-5, cfl=0.2, max_iter=16, tol=1e-6)
    gs = gpu_for(pb, precision="fp32", **kw)
    names = gs.variants()
    tile = "face 8x8 cells, 128 threads, 4 CTA/SM"
    picks = [i for i, n in enumerate(names) if n.startswith(tile) and "TMA" not in n]
    assert len(picks) == 3, names
    out = {}
    for f in picks:
        gs.set_variants(face=f, cell=0)
        gs.set_primitive()
        gs.step(10)
        assert gs.sync()["nonphysical"] == 0
        out[names[f]] = ([np.asarray(a) for a in gs.state()], _prims(gs))
    plain, l1, l2 = (out[names[f]] for f in picks)
    for a, b in zip(l1[0], l2[0]):
        assert np.array_equal(a, b)
    for a, b in zip(l1[1], plain[1]):
        assert rel_l1(a, b) <= 1e-5


def _quadrants_64x48():
    q = I.quadrants_2d(64, seed=0)
    keep = np.arange(64 * 48)   # rows 0..47 of the 64 x 64 draw (x fastest)
    return I.Problem(2, 64, 48, 0.0, 1.0, 0.0, 0.75, q.gamma, q.rho[keep], q.ux[keep], q.uy[keep], q.p[keep],
                     bc=q.bc, name="quadrants_64x48")


@pytest.mark.parametrize("name,make", [
    ("quadrants_64x48", _quadrants_64x48),
    ("shocked_interface_96x40", lambda: I.shocked_interface_2d(96, 40, seed=2)),
    ("jet_64", lambda: I.jet_2d(64, seed=0)),
    ("explosion_box_48", lambda: I.explosion_box_2d(48)),
    ("smooth_periodic_64x40", lambda: I.smooth_periodic(2, 64, 40, seed=1)),
], ids=lambda x: x if isinstance(x, str) else "")
def test_tma_staging_is_the_same_arithmetic(name, make):
    """The TMA variants of the 8 x 8 face tile (both scratch levels) copy the state planes of
    an interior tile's box into shared memory with tensor-map loads and form phi-bar-plus
    there, with the arithmetic of the per-thread staging; tiles that touch a side (ghost
    rules) stage per thread.  Over twelve steps of transmissive, inflow, reflective and
    periodic problems their states and face frames equal those of the per-thread variants of
    the same tile bit for bit, and the diagnostics count the tiles staged by TMA (every
    interior tile of every step)."""
    pb = make()
    kw = dict(tau=1e-5, cfl=0.2, max_iter=16, tol=1e-6)
    steps = 12
    # interior tiles: x origin i0 = 8 bx with 2 <= i0 and i0 + 8 <= nx - 1, likewise in y
    nxt = sum(1 for i0 in range(0, pb.nx + 1, 8) if i0 >= 2 and i0 + 8 <= pb.nx - 1)
    nyt = sum(1 for j0 in range(0, pb.ny + 1, 8) if j0 >= 2 and j0 + 8 <= pb.ny - 1)
    for level in ("centre cells in shared scratch", "centre cells and moment sums in shared scratch"):
        out = {}
        for which in ("per-thread", "TMA"):
            gs = gpu_for(pb, precision="fp32", **kw)
            names = gs.variants()
            base = "face 8x8 cells, 128 threads, 4 CTA/SM, " + level
            f = names.index(base + (", TMA staging" if which == "TMA" else ""))
            gs.set_variants(face=f, cell=0)
            gs.set_primitive()
            gs.step(steps)
            d = gs.sync()
            assert d["nonphysical"] == 0 and d["steps"] == steps, (level, which, d)
            out[which] = ([np.asarray(a) for a in gs.state()], [a for a in gs.face_gauges()], d)
            gs.close()
        (sa, fa, da), (sb, fb, db) = out["per-thread"], out["TMA"]
        for a, b in zip(sa, sb):
            assert np.array_equal(a, b), level
        for a, b in zip(fa, fb):
            assert a is None or np.array_equal(a, b), level
        assert da["face_iters"] == db["face_iters"] and da["fallbacks"] == db["fallbacks"]
        assert da["staged_tma"] == 0
        assert db["staged_tma"] == steps * nxt * nyt > 0, (level, db["staged_tma"], nxt, nyt)


def test_tma_variant_stages_per_thread_without_maps():
    """A grid whose rows are not a multiple of 16 bytes (nx = 61) gets no tensor maps: the TMA
    variant then stages every tile per thread and gives the per-thread variant's state."""
    pb = I.quadrants_2d(61, seed=0)
    kw = dict(tau=1e-5, cfl=0.2, max_iter=16, tol=1e-6)
    res = []
    for tma in (False, True):
        gs = gpu_for(pb, precision="fp32", **kw)
        names = gs.variants()
        base = "face 8x8 cells, 128 threads, 4 CTA/SM, centre cells in shared scratch"
        gs.set_variants(face=names.index(base + (", TMA staging" if tma else "")), cell=0)
        gs.set_primitive()
        gs.step(5)
        d = gs.sync()
        assert d["staged_tma"] == 0
        res.append([np.asarray(a) for a in gs.state()])
        gs.close()
    for a, b in zip(*res):
        assert np.array_equal(a, b)
