"""Pin for the oracle's inflow side (the RMI and jet set-ups of Sec. IV, equilibrium ghost
cells at a prescribed state): a supersonic stream entering a gas at rest.  When both waves
of the Riemann problem between the inflow state (left) and the gas (right) move into the
domain, the solution inside is that Riemann problem's exact solution centred on the side,
which the exact solver (written from the gas dynamics) gives independently."""
import numpy as np
import pytest

from oracle.riemann import RiemannSolution, cell_averaged_profile
from paper_2203_05477_gb300 import inputs as I
from tests.common import oracle_for, rel_l1

GAMMA = 1.4
STREAM = (1.5, 2.5, 1.2)   # rho, u, p entering at x = 0 (Mach 2.4)
GAS = (0.5, 0.0, 0.4)


def inflow_tube(n):
    inflow = np.zeros((4, 4))
    inflow[0] = (STREAM[0], STREAM[1], 0.0, STREAM[2])
    rng = np.zeros((4, 2), dtype=np.int64)
    rng[0] = (0, 1)
    return I.Problem(1, n, 1, 0.0, 1.0, 0.0, 1.0, GAMMA, np.full(n, GAS[0]), np.full(n, GAS[1]), np.zeros(n),
                     np.full(n, GAS[2]), bc=(I.INFLOW, I.TRANSMISSIVE, I.TRANSMISSIVE, I.TRANSMISSIVE),
                     inflow=inflow, inflow_range=rng)


def test_both_waves_enter_the_domain():
    sol = RiemannSolution(STREAM, GAS, GAMMA)
    assert sol.pstar > STREAM[2] and sol.pstar > GAS[2]          # two shocks
    assert sol.shock_speed("L") > 0.5 and sol.shock_speed("R") > sol.shock_speed("L")


@pytest.mark.parametrize("n,tol", [(200, 1.2e-2), (400, 7e-3)])
def test_supersonic_inflow_matches_exact_solution(n, tol):
    t_end = 0.2
    s = oracle_for(inflow_tube(n), tau=1e-5, cfl=0.3, t_end=t_end, tol=1e-10, max_iter=16)
    s.step(100000)
    st = s.stats()
    assert st["t"] == pytest.approx(t_end, rel=1e-12) and st["nonphysical"] == 0
    r, u, _, p = s.primitive()
    edges = np.linspace(0.0, 1.0, n + 1)
    re, ue, pe = cell_averaged_profile(STREAM, GAS, GAMMA, edges, 0.0, t_end)
    # measured (rho / p / u) 8.7e-3 / 2.9e-3 / 4.3e-3 at 200 cells, 5.5e-3 / 2.7e-3 / 2.7e-3 at 400
    assert rel_l1(r, re) < tol and rel_l1(p, pe) < tol and rel_l1(u, ue) < tol
    # the cells next to the side hold the stream's state
    assert abs(r[:5] - STREAM[0]).max() < 1e-3 and abs(u[:5] - STREAM[1]).max() < 1e-3
