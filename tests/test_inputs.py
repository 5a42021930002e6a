"""The seeded synthetic inputs hold the stated recipes: value ranges, structure and the
shock relations of the set-ups that carry a shock (host logic, no method arithmetic)."""
import numpy as np
import pytest

from paper_2203_05477_gb300 import inputs as I


@pytest.mark.parametrize("seed", range(8))
def test_quadrants_recipe(seed):
    pb = I.quadrants_2d(32, seed=seed)
    assert pb.rho.size == 32 * 32 and len(np.unique(pb.rho)) <= 4
    assert pb.rho.min() >= 0.1 and pb.rho.max() <= 10 and pb.p.min() >= 0.1 and pb.p.max() <= 10
    c = np.sqrt(pb.gamma * pb.p / pb.rho)
    mach = np.hypot(pb.ux, pb.uy) / c
    assert mach.max() <= 3.0 + 1e-12
    # each quadrant moves towards the domain centre within 45 degrees (measured from the
    # quadrant's own centre)
    U, V = pb.ux.reshape(32, 32), pb.uy.reshape(32, 32)
    for (jy, ix), (cx, cy) in zip([(0, 0), (0, 31), (31, 0), (31, 31)], [(0.25, 0.25), (0.75, 0.25), (0.25, 0.75), (0.75, 0.75)]):
        u = np.array([U[jy, ix], V[jy, ix]])
        d = np.array([0.5 - cx, 0.5 - cy])
        if np.linalg.norm(u) > 0:
            assert u @ d / (np.linalg.norm(u) * np.linalg.norm(d)) >= np.cos(np.pi / 4) - 1e-12
    # same seed, same draw
    assert np.array_equal(I.quadrants_2d(32, seed=seed).p, pb.p)


def test_tube_batch_recipe():
    b = I.tube_batch(4096, seed=0)
    assert b.lengths.min() >= 200 and b.lengths.max() <= 8000
    assert 1800 < b.lengths.mean() < 2400           # log-uniform on [200, 8000]: mean 2114
    assert set(np.unique(b.gammas)) == {1.4, 5.0 / 3.0}
    hi = np.maximum(b.left[:, 0], b.right[:, 0])
    lo = np.minimum(b.left[:, 0], b.right[:, 0])
    assert (hi / lo <= 1e5 * (1 + 1e-12)).all() and (hi >= 0.1 - 1e-12).all() and (hi <= 10 + 1e-12).all()
    phi = np.maximum(b.left[:, 2], b.right[:, 2])
    plo = np.minimum(b.left[:, 2], b.right[:, 2])
    assert (phi / plo <= 1e5 * (1 + 1e-12)).all()
    # the velocity jump is at most Mach 20 of the denser side's sound speed
    dense = np.where(b.left[:, 0] >= b.right[:, 0], 0, 1)
    side = np.where(dense[:, None] == 0, b.left, b.right)
    cs = np.sqrt(b.gammas * side[:, 2] / side[:, 0])
    assert (np.abs(b.left[:, 1] - b.right[:, 1]) <= 20 * cs * (1 + 1e-12)).all()
    rho, ux, p = I.tube_batch_fields(b)
    assert rho.size == b.total_cells and ux.size == p.size == rho.size


@pytest.mark.parametrize("seed", range(5))
def test_shocked_interface_is_a_rankine_hugoniot_shock(seed):
    pb = I.shocked_interface_2d(64, 16, seed=seed)
    rho2, u2, _, p2 = pb.inflow[0]
    g = pb.gamma
    # shock speed from mass conservation across a shock into gas at rest (rho 1, p 1)
    S = rho2 * u2 / (rho2 - 1.0)
    assert rho2 * (S - u2) ** 2 + p2 == pytest.approx(S * S + 1.0, rel=1e-12)               # momentum
    e1, e2 = 1.0 / (g - 1.0), p2 / ((g - 1.0) * rho2)
    assert (S - u2) * rho2 * (e2 + p2 / rho2 + 0.5 * (S - u2) ** 2) == pytest.approx(
        S * (e1 + 1.0 + 0.5 * S * S), rel=1e-12)                                                # energy
    M = S / np.sqrt(g)
    assert 1.5 <= M <= 3.0
    heavy = pb.rho.max()
    A = (heavy - 1.0) / (heavy + 1.0)
    assert 0.5 <= A <= 0.9
    assert pb.bc == (I.INFLOW, I.TRANSMISSIVE, I.PERIODIC, I.PERIODIC)


@pytest.mark.parametrize("seed", range(5))
def test_jet_recipe(seed):
    pb = I.jet_2d(48, seed=seed)
    rho_j, u_j, _, p_j = pb.inflow[0]
    p_amb = pb.p[0]
    assert 0.1 <= p_amb <= 1.0 and np.all(pb.rho == 1.0)
    T_ratio = (p_j / rho_j) / p_amb
    assert 0.01 <= T_ratio <= 1.0 and rho_j == pytest.approx(10.0)
    assert u_j / np.sqrt(pb.gamma * p_j / rho_j) == pytest.approx(80.0, rel=1e-12)
    lo, hi = pb.inflow_range[0]
    y = I.cell_centres(48, -0.5, 0.5)
    assert np.all(np.abs(y[lo:hi]) <= 0.05) and abs(y[lo - 1]) > 0.05 and abs(y[hi]) > 0.05
