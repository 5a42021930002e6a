"""Reflective walls on the GPU (two-blast-wave and explosion-in-a-box cases of Sec. IV):
FP64 parity with the oracle at 1e-12 in corrector parity mode, on walls alone, walls in
corners, walls beside transmissive and inflow sides, and with nonzero wall-normal
velocities; mass and energy conservation in a closed box; FP32 against the FP64 oracle."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2203_05477_gb300 as pond  # noqa: E402
from paper_2203_05477_gb300 import inputs as I  # noqa: E402
from tests.common import oracle_for, rel_l1  # noqa: E402
from tests.test_gpu_parity import compare_fp64, gpu_for  # noqa: E402
from tests.test_oracle_reflective import perturbed  # noqa: E402

pytestmark = pytest.mark.gpu

KW64 = dict(tau=1e-5, cfl=0.2, fixed_iters=3, max_iter=8)
R, T, P, F = I.REFLECTIVE, I.TRANSMISSIVE, I.PERIODIC, I.INFLOW


def _inflow_left(pb):
    inflow = np.zeros((4, 4))
    inflow[0] = (2.0, 0.6, 0.1, 2.5)
    rng = np.zeros((4, 2), dtype=np.int64)
    rng[0] = (pb.ny // 3, 2 * pb.ny // 3)
    return dataclasses.replace(pb, bc=(F, T, R, R), inflow=inflow, inflow_range=rng)


CASES = [
    ("two_blast_120", lambda: I.two_blast_1d(120)),
    ("wall_reflection_90", lambda: I.wall_reflection_1d(90)),
    ("random_tube_walls_37", lambda: dataclasses.replace(
        perturbed(I.shock_tube((1.0, 0.4, 1.0), (0.3, -0.6, 0.4), 1.4, 37), 4), bc=(R, R, T, T))),
    ("explosion_box_27", lambda: I.explosion_box_2d(27)),
    ("explosion_box_moving_21", lambda: perturbed(I.explosion_box_2d(21), 6)),
    ("walls_x_periodic_y_23x17", lambda: dataclasses.replace(
        perturbed(I.smooth_periodic(2, 23, 17, seed=3, amp=0.15), 7), bc=(R, R, P, P))),
    ("wall_transmissive_mix_19x26", lambda: dataclasses.replace(
        perturbed(I.smooth_periodic(2, 19, 26, seed=4, amp=0.15), 8), bc=(R, T, T, R))),
    ("inflow_window_and_walls_18", lambda: _inflow_left(perturbed(I.explosion_box_2d(18), 9))),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_fp64_parity_reflective(name, make):
    pb = make()
    gs = gpu_for(pb, precision="fp64", **KW64)
    os_ = oracle_for(pb, **KW64)
    for chunk in (1, 5):
        gs.step(chunk)
        os_.step(chunk)
        d = gs.sync()
        st = os_.stats()
        assert d["steps"] == st["steps"] and d["face_iters"] == st["face_iters"]
        assert d["nonphysical"] == st["nonphysical"] == 0
        compare_fp64(gs, os_)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_closed_box_conserves_mass_and_energy(precision, tol):
    pb = perturbed(I.explosion_box_2d(32), 5)
    gs = gpu_for(pb, precision=precision, tau=1e-4, cfl=0.3)
    _, t0 = gs.moments()
    gs.step(60)
    _, t1 = gs.moments()
    assert gs.sync()["status"] == pond.POND_OK
    for k in (0, 3):
        assert abs(t1[k] - t0[k]) <= tol * t0[k], (k, t0[k], t1[k])


def test_fp32_explosion_box_against_fp64_oracle():
    pb = I.explosion_box_2d(48)
    kw = dict(tau=1e-5, cfl=0.2, max_iter=16, tol=1e-6)
    gs = gpu_for(pb, precision="fp32", **kw)
    os_ = oracle_for(pb, **kw)
    gs.step(40)
    os_.step(40)
    assert gs.sync()["nonphysical"] == 0 and os_.stats()["nonphysical"] == 0
    r, ux, uy, p = gs.primitive()
    ro, uxo, uyo, po = os_.primitive()
    assert rel_l1(r, ro) <= 1e-4 and rel_l1(p, po) <= 1e-4
    speed = np.sqrt(uxo ** 2 + uyo ** 2)
    assert np.abs(ux - uxo).sum() / speed.sum() <= 1e-4 and np.abs(uy - uyo).sum() / speed.sum() <= 1e-4
