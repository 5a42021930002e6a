"""The equilibration alternative to Grad's projection (Sec. II.C), an ablation of the
regularized transformation.  Pinned by what the construction fixes: the slow moments (orders
up to 3 for f, 2 for g) are those of the input, as with Grad's projection; the fast
tensor-Hermite components equal the equilibrium's, M0 d_x^r d_y^s with d = (M1/M0 - u') /
sqrt(T'); a discrete equilibrium moved to a frame of the same temperature becomes the
product of two 1D shifted equilibria (the closed form of a shifted Maxwellian on a
tensor-product lattice); a solver step with it still conserves mass, momentum and energy."""
import numpy as np
import pytest

import oracle as O
from paper_2203_05477_gb300 import inputs as I
from tests.common import oracle_for
from tests.test_oracle_transform import lab_moments, random_case


def he(k, x):
    return [np.ones_like(x), x, x * x - 1.0, x ** 3 - 3.0 * x][k]


@pytest.mark.parametrize("D", [1, 2, 3])
@pytest.mark.parametrize("order", [2, 3])
def test_slow_moments_are_kept(D, order):
    rng = np.random.default_rng(7 * D + order)
    for _ in range(20):
        c, W, f, u, T, up, Tp = random_case(rng, D)
        fo = O.regularized_transform(D, order, f, u, T, up, Tp, equilibrate=True)
        for a, b in zip(lab_moments(f, c, u, T, order), lab_moments(fo, c, up, Tp, order)):
            np.testing.assert_allclose(b, a, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("order", [2, 3])
def test_fast_components_are_the_equilibrium(order):
    rng = np.random.default_rng(30 + order)
    for _ in range(20):
        c, W, f, u, T, up, Tp = random_case(rng, 2)
        fo = O.regularized_transform(2, order, f, u, T, up, Tp, equilibrate=True)
        M = lab_moments(f, c, u, T, 1)
        d = (M[1] / M[0] - up) / np.sqrt(Tp)
        for r in range(4):
            for s in range(4):
                a_rs = np.sum(fo * he(r, c[:, 0]) * he(s, c[:, 1]))
                if r + s > order:
                    assert a_rs == pytest.approx(M[0] * d[0] ** r * d[1] ** s, rel=1e-10, abs=1e-12)
        # Grad's projection leaves those components at zero
        fg = O.grad_transform(2, order, f, u, T, up, Tp)
        assert abs(np.sum(fg * he(3, c[:, 0]) * he(3, c[:, 1]))) < 1e-12


def test_shifted_equilibrium_is_a_product_of_1d_ones():
    c, W, _ = O.lattice(2)
    rho, T = 1.7, 0.6
    u, up = np.array([0.3, -0.2]), np.array([-0.1, 0.25])
    fo = O.regularized_transform(2, 3, rho * W, u, T, up, T, equilibrate=True)
    d = (u - up) / np.sqrt(T)
    e = lambda x, dd: sum(dd ** k * he(k, x) / [1, 1, 2, 6][k] for k in range(4))
    np.testing.assert_allclose(fo, rho * W * e(c[:, 0], d[0]) * e(c[:, 1], d[1]), rtol=1e-12, atol=1e-14)


def test_solver_with_equilibration_conserves():
    pb = I.smooth_periodic(2, 12, 10, seed=4, amp=0.2)
    s = oracle_for(pb, tau=1e-4, cfl=0.3, tol=1e-12, max_iter=16)
    s.set_equilibration(True)
    r0, mx0, my0, E0 = (a.sum() for a in s.conserved())
    s.step(20)
    assert s.stats()["nonphysical"] == 0
    r1, mx1, my1, E1 = (a.sum() for a in s.conserved())
    assert abs(r1 - r0) <= 1e-13 * r0 and abs(E1 - E0) <= 1e-13 * E0
    assert abs(mx1 - mx0) <= 1e-13 * r0 and abs(my1 - my0) <= 1e-13 * r0


@pytest.mark.parametrize("order", [2, 3])
def test_fast_components_are_the_equilibrium_3d(order):
    """D3Q64: every tensor component He_r He_s He_t with r, s, t <= 3 and r + s + t > order is
    the equilibrium's M0 d_x^r d_y^s d_z^t."""
    from tests.test_oracle_3d import random_case_3d
    rng = np.random.default_rng(40 + order)
    for _ in range(6):
        c, W, f, u, T, up, Tp = random_case_3d(rng)
        fo = O.regularized_transform(3, order, f, u, T, up, Tp, equilibrate=True)
        M = lab_moments(f, c, u, T, 1)
        d = (M[1] / M[0] - up) / np.sqrt(Tp)
        for r in range(4):
            for s_ in range(4):
                for t in range(4):
                    if r + s_ + t > order:
                        a = np.sum(fo * he(r, c[:, 0]) * he(s_, c[:, 1]) * he(t, c[:, 2]))
                        assert a == pytest.approx(M[0] * d[0] ** r * d[1] ** s_ * d[2] ** t, rel=1e-9, abs=1e-11)
