"""Pins for the oracle's semi-Lagrangian realization (Sec. III.A): the exact Riemann
solution of Sod's tube with first-order-like convergence under refinement; uniform flow at
any Mach number stays uniform; a small acoustic wave travels at the sound speed sqrt(gamma T)
(closed form of linear acoustics), in both the semi-Lagrangian and the finite-volume
realizations; the x<->y symmetry of a symmetric 2D state; reflective walls unfold into a
periodic problem.  The scheme is not conservative (Sec. IV, comparison of the schemes):
the mass drift is reported, small but not zero."""
import numpy as np
import pytest

from oracle.riemann import cell_averaged_profile
from paper_2203_05477_gb300 import inputs as I
from tests.common import max_rel, oracle_for, rel_l1
from tests.test_oracle_reflective import perturbed, unfolded_view, walled

SOD = ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4)


def sod_sl(n):
    pb = I.shock_tube(*SOD, n)
    s = oracle_for(pb, tau=1e-5, cfl=0.5, t_end=0.2, tol=1e-10, max_iter=16)
    s.sl_step(100000)
    return pb, s


def test_sl_sod_converges_to_exact_solution():
    errs = []
    for n in (100, 200, 400):
        pb, s = sod_sl(n)
        st = s.stats()
        assert st["t"] == pytest.approx(0.2, rel=1e-12) and st["nonphysical"] == 0
        r, u, _, p = s.primitive()
        re, ue, pe = cell_averaged_profile(SOD[0], SOD[1], SOD[2], np.linspace(0, 1, n + 1), 0.5, 0.2)
        errs.append((rel_l1(r, re), rel_l1(p, pe)))
    assert errs[-1][0] < 6e-3 and errs[-1][1] < 6e-3
    for k in range(2):
        assert errs[0][k] > errs[1][k] > errs[2][k]


def test_sl_is_not_conservative_but_close():
    pb, s = sod_sl(200)
    m0 = pb.rho.sum()
    m1 = s.primitive()[0].sum()
    drift = abs(m1 - m0) / m0
    assert 1e-6 < drift < 1e-2


@pytest.mark.parametrize("mach", [0.0, 3.0, 80.0])
@pytest.mark.parametrize("dim", [1, 2])
def test_sl_uniform_flow_stays_uniform(mach, dim):
    g, T, rho = 5.0 / 3.0, 0.02, 1.3
    u = mach * np.sqrt(g * T)
    n = 12
    if dim == 1:
        pb = I.Problem(1, n, 1, 0.0, 1.0, 0.0, 1.0, g, np.full(n, rho), np.full(n, u), np.zeros(n),
                       np.full(n, rho * T), bc=(I.PERIODIC,) * 4)
    else:
        pb = I.Problem(2, n, n, 0.0, 1.0, 0.0, 1.0, g, np.full(n * n, rho), np.full(n * n, u * 0.8),
                       np.full(n * n, -u * 0.6), np.full(n * n, rho * T), bc=(I.PERIODIC,) * 4)
    s = oracle_for(pb, tau=1e-5, cfl=0.4, tol=1e-12, max_iter=16)
    s.sl_step(30)
    r, ux, uy, p = s.primitive()
    tol = 1e-12 * (1.0 + mach) ** 2
    assert max_rel(r, pb.rho) <= tol and max_rel(p, pb.p) <= tol
    assert np.abs(ux - pb.ux).max() <= tol * max(1.0, abs(u))


def _wave_phase(rho, n):
    return np.angle(np.fft.rfft(rho - rho.mean())[1])


@pytest.mark.parametrize("scheme", ["sl", "fv"])
def test_acoustic_wave_travels_at_sound_speed(scheme):
    """Linear acoustics: rho = rho0 (1 + eps sin kx), u = c eps sin kx, p = p0 (1 + gamma eps
    sin kx) is a right-running wave of speed c = sqrt(gamma p0 / rho0)."""
    n, g, rho0, p0, eps = 64, 1.4, 1.0, 1.0, 1e-4
    c = np.sqrt(g * p0 / rho0)
    x = I.cell_centres(n, 0.0, 1.0)
    w = np.sin(2 * np.pi * x)
    pb = I.Problem(1, n, 1, 0.0, 1.0, 0.0, 1.0, g, rho0 * (1 + eps * w), c * eps * w, np.zeros(n),
                   p0 * (1 + g * eps * w), bc=(I.PERIODIC,) * 4)
    t_end = 0.3 / c
    s = oracle_for(pb, tau=1e-5, cfl=0.4, t_end=t_end, tol=1e-12, max_iter=16)
    (s.sl_step if scheme == "sl" else s.step)(100000)
    assert s.stats()["t"] == pytest.approx(t_end, rel=1e-12)
    r = s.primitive()[0]
    shift = ((_wave_phase(pb.rho, n) - _wave_phase(r, n)) / (2 * np.pi)) % 1.0
    assert shift == pytest.approx(c * t_end, rel=1e-2)
    # amplitude: little dissipation over 0.3 periods at 64 cells per wavelength
    amp = np.abs(np.fft.rfft(r - r.mean())[1]) / (n / 2) / rho0
    assert 0.9 * eps < amp <= 1.0001 * eps


def test_sl_2d_keeps_xy_symmetry():
    pb = I.lax_liu_2d(16)
    s = oracle_for(pb, tau=1e-5, cfl=0.3, fixed_iters=3, max_iter=8)
    s.sl_step(6)
    r, ux, uy, p = s.primitive()
    n = pb.nx
    R, U, V, P = (a.reshape(n, n) for a in (r, ux, uy, p))
    assert max_rel(R, R.T) <= 1e-13 and max_rel(P, P.T) <= 1e-13
    assert np.abs(U - V.T).max() <= 1e-13 * max(1.0, np.abs(U).max())


@pytest.mark.parametrize("make", [
    lambda: walled(perturbed(I.shock_tube((1.0, 0.3, 1.0), (0.4, -0.5, 0.3), 1.4, 23), 2)),
    lambda: perturbed(I.explosion_box_2d(10), 3),
], ids=["random_tube_23", "explosion_box_10"])
def test_sl_reflective_equals_unfolded_periodic(make):
    pb = make()
    big = I.mirror_extend(pb)
    kw = dict(tau=1e-5, cfl=0.3, fixed_iters=3, max_iter=8)
    a, b = oracle_for(pb, **kw), oracle_for(big, **kw)
    a.sl_step(5)
    b.sl_step(5)
    assert a.stats()["nonphysical"] == 0
    ra, _, _, Ea = a.conserved()
    rb, _, _, Eb = b.conserved()
    assert max_rel(ra, unfolded_view(pb, rb)) <= 1e-13 and max_rel(Ea, unfolded_view(pb, Eb)) <= 1e-13
