"""The Richtmyer-Meshkov set-ups of Sec. IV.  The printed post-shock states are the
Rankine-Hugoniot states of the named shocks (density and velocity of both types, pressure
of type 2 to the printed digits); type 1's printed pressure 0.151332 is one tenth of the
Rankine-Hugoniot value 1.51332, and the generator takes the latter (a reading).  The oracle
keeps the set-ups' mirror symmetry about mid-height."""
import os

import numpy as np
import pytest

from paper_2203_05477_gb300 import inputs as I
from tests.common import oracle_for


def printed_states():
    rows = []
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "rmi_post_shock_states.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append([float(v) for v in line.split()])
    return rows


@pytest.mark.parametrize("row", printed_states(), ids=["type1", "type2"])
def test_printed_post_shock_states_are_rankine_hugoniot(row):
    kind, mach, rho, ux, uy, p = row
    r2, u2, p2 = I.rankine_hugoniot(mach, 1.0, 1.0, 1.4)
    assert r2 == pytest.approx(rho, rel=5e-3) and u2 == pytest.approx(ux, rel=5e-3)
    if kind == 1:
        assert p2 == pytest.approx(10.0 * p, rel=1e-5)   # printed one tenth of the shock state
    else:
        assert p2 == pytest.approx(p, rel=1e-5)
    pb = I.rmi_2d(int(kind), 60, 10)
    assert pb.rho[0] == r2 and pb.p[0] == p2 and pb.inflow[0][3] == p2


@pytest.mark.parametrize("kind", [1, 2])
def test_rmi_keeps_mirror_symmetry(kind):
    pb = I.rmi_2d(kind, 60, 10)
    s = oracle_for(pb, tau=1e-5, cfl=0.2, fixed_iters=3, max_iter=8)
    s.step(6)
    assert s.stats()["nonphysical"] == 0
    r, ux, uy, p = (a.reshape(10, 60) for a in s.primitive())
    assert np.abs(r - r[::-1]).max() <= 1e-13 * r.max()
    assert np.abs(p - p[::-1]).max() <= 1e-13 * p.max()
    assert np.abs(uy + uy[::-1]).max() <= 1e-13 * np.abs(ux).max()
