"""Pins for the exact Riemann solver used as the shock-tube yardstick (Sec. IV.A-C):
the sampled solution must satisfy the Rankine-Hugoniot conditions across shocks, the
isentropic Riemann invariants across rarefactions and pressure/velocity continuity
across the contact."""
import numpy as np
import pytest

from oracle.riemann import RiemannSolution

CASES = {
    "sod": ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4),
    "lax": ((0.445, 0.698, 3.528), (0.5, 0.0, 0.571), 1.4),
    "strong": ((1.0, 0.0, 1000.0), (1.0, 0.0, 0.01), 1.4),
    "jet": ((5.0, 30.0, 0.4127), (0.5, 0.0, 0.4127), 5.0 / 3.0),
    "leblanc": ((1.0, 0.0, 2.0 / 3.0 * 1e-1), (1e-3, 0.0, 2.0 / 3.0 * 1e-10), 5.0 / 3.0),
}


def rh_residual(s, a, b, g):
    """Mass, momentum and energy flux jumps in the frame of a discontinuity moving at s."""
    (r1, u1, p1), (r2, u2, p2) = a, b
    w1, w2 = u1 - s, u2 - s
    e1 = p1 / ((g - 1) * r1) + 0.5 * w1 * w1 + p1 / r1
    e2 = p2 / ((g - 1) * r2) + 0.5 * w2 * w2 + p2 / r2
    return (r1 * w1 - r2 * w2, r1 * w1 * w1 + p1 - r2 * w2 * w2 - p2, r1 * w1 * e1 - r2 * w2 * e2)


@pytest.mark.parametrize("name", list(CASES))
def test_wave_relations(name):
    L, R, g = CASES[name]
    sol = RiemannSolution(L, R, g)
    assert not sol.vacuum
    scale = max(L[2], R[2], sol.pstar)
    for side, K, rs in (("L", L, sol.rstar_l), ("R", R, sol.rstar_r)):
        S = sol.shock_speed(side)
        star = (rs, sol.ustar, sol.pstar)
        if S is not None:
            res = rh_residual(S, K, star, g)
            mscale = max(K[0], rs) * (abs(S) + abs(K[1]) + np.sqrt(g * scale / K[0]))
            assert abs(res[0]) < 1e-10 * mscale
            assert abs(res[1]) < 1e-10 * mscale * (abs(S) + 1e-300 + np.sqrt(scale))
        else:
            # isentropic fan: p rho^-g and u +- 2a/(g-1) preserved
            assert sol.pstar / rs ** g == pytest.approx(K[2] / K[0] ** g, rel=1e-10)
            a_k, a_s = np.sqrt(g * K[2] / K[0]), np.sqrt(g * sol.pstar / rs)
            sign = 1.0 if side == "L" else -1.0
            assert K[1] + sign * 2 * a_k / (g - 1) == pytest.approx(sol.ustar + sign * 2 * a_s / (g - 1), rel=1e-10, abs=1e-10)


def test_sod_star_state_and_profile_continuity():
    sol = RiemannSolution(*CASES["sod"])
    # star values implied by the RH + isentrope relations above, to 6 digits
    assert sol.pstar == pytest.approx(0.303130, rel=1e-5)
    assert sol.ustar == pytest.approx(0.927453, rel=1e-5)
    s = np.linspace(-2, 2, 4001)
    r, u, p = sol.sample(s)
    # across the contact (s = u*) pressure and velocity are continuous
    k = np.searchsorted(s, sol.ustar)
    assert abs(p[k + 1] - p[k - 1]) < 1e-12 and abs(u[k + 1] - u[k - 1]) < 1e-12
    assert r[k - 1] == pytest.approx(sol.rstar_l) and r[k + 1] == pytest.approx(sol.rstar_r)


def test_vacuum_generation():
    sol = RiemannSolution((1.0, -2.0, 0.1), (1.0, 2.0, 0.1), 1.4)
    assert sol.vacuum
    r, u, p = sol.sample(np.array([-3.0, 0.0, 3.0]))
    assert r[0] == 1.0 and r[2] == 1.0 and r[1] == 0.0 and p[1] == 0.0
