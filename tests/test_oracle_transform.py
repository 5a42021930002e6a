"""Pins for the oracle's regularized frame transformation (Sec. II.C).

The transformation is defined by two things: the Grad form Eq. (f_transformed) of the
output and the invariance of the moments of order <= 3 (f) or <= 2 (g), Eq. (Mcondition).
These tests check the oracle's implementation of Eqs. (a0)-(a3) against that definition,
against an independent route (central moments expanded directly), against a brute-force
least-squares solve of the moment conditions, and against the algebraic consequences
(identity, round trip, idempotence)."""
import itertools

import numpy as np
import pytest

import oracle as O


def lab_moments(f, c, u, T, kmax):
    v = np.sqrt(T) * c + np.asarray(u)[None, :]
    out = []
    for k in range(kmax + 1):
        if k == 0:
            out.append(f.sum())
        else:
            ops = ",".join(["i"] + ["i" + "abc"[j] for j in range(k)])
            out.append(np.einsum(ops + "->" + "abc"[:k], f, *([v] * k)))
    return out


def grad_basis(c, order):
    """Columns: W_i * Hermite tensor components He_{r,s}(c_i) for r + s <= order (D2) or r <= order (D1)."""
    D = c.shape[1]
    def he(k, x):
        return [np.ones_like(x), x, x * x - 1, x ** 3 - 3 * x][k]
    cols = []
    if D == 1:
        for r in range(order + 1):
            cols.append(he(r, c[:, 0]))
    else:
        for r in range(order + 1):
            for s in range(order + 1 - r):
                cols.append(he(r, c[:, 0]) * he(s, c[:, 1]))
    return np.stack(cols, 1)


def random_case(rng, D, spread=1.0):
    c, W, _ = O.lattice(D)
    Q = len(W)
    f = W * (1.0 + 0.3 * rng.standard_normal(Q))
    u = rng.uniform(-spread, spread, D)
    T = np.exp(rng.uniform(-1, 1))
    up = rng.uniform(-spread, spread, D)
    Tp = np.exp(rng.uniform(-1, 1))
    return c, W, f, u, T, up, Tp


@pytest.mark.parametrize("D", [1, 2])
@pytest.mark.parametrize("order", [2, 3])
def test_moments_invariant(D, order):
    rng = np.random.default_rng(10 * D + order)
    for _ in range(20):
        c, W, f, u, T, up, Tp = random_case(rng, D)
        fo = O.grad_transform(D, order, f, u, T, up, Tp)
        Min = lab_moments(f, c, u, T, order)
        Mout = lab_moments(fo, c, up, Tp, order)
        for a, b in zip(Min, Mout):
            np.testing.assert_allclose(b, a, rtol=1e-12, atol=1e-12)


def central_route(f, c, W, u, T, up, Tp, order):
    """Independent route: central moments P_k of xi = (v - u')/sqrt(T') expanded directly,
    Hermite coefficients a0 = P0, a1 = P1, a2 = P2 - P0 I, a3 = P3 - sym(P1 x I)."""
    D = c.shape[1]
    xi = (np.sqrt(T) * c + u[None, :] - up[None, :]) / np.sqrt(Tp)
    P0 = f.sum()
    P1 = np.einsum("i,ia->a", f, xi)
    P2 = np.einsum("i,ia,ib->ab", f, xi, xi)
    P3 = np.einsum("i,ia,ib,ic->abc", f, xi, xi, xi)
    I = np.eye(D)
    a2 = P2 - P0 * I
    a3 = P3 - (np.einsum("a,bc->abc", P1, I) + np.einsum("b,ac->abc", P1, I) + np.einsum("c,ab->abc", P1, I))
    H2 = np.einsum("ia,ib->iab", c, c) - I[None]
    H3 = (np.einsum("ia,ib,ic->iabc", c, c, c)
          - np.einsum("ia,bc->iabc", c, I) - np.einsum("ib,ac->iabc", c, I) - np.einsum("ic,ab->iabc", c, I))
    out = P0 + c @ P1 + 0.5 * np.einsum("iab,ab->i", H2, a2)
    if order >= 3:
        out = out + np.einsum("iabc,abc->i", H3, a3) / 6.0
    return W * out


@pytest.mark.parametrize("D", [1, 2])
@pytest.mark.parametrize("order", [2, 3])
def test_matches_central_moment_route(D, order):
    rng = np.random.default_rng(7 + D + order)
    for _ in range(20):
        c, W, f, u, T, up, Tp = random_case(rng, D, spread=2.0)
        fo = O.grad_transform(D, order, f, u, T, up, Tp)
        ref = central_route(f, c, W, u, T, up, Tp, order)
        np.testing.assert_allclose(fo, ref, rtol=1e-11, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("D,order,nparam", [(1, 3, 4), (1, 2, 3), (2, 3, 10), (2, 2, 6)])
def test_brute_force_moment_conditions(D, order, nparam):
    """Solve Eq. (Mcondition) directly: unknown Grad coefficients, one equation per moment
    component of order <= `order`, least squares over the (consistent) overdetermined set."""
    rng = np.random.default_rng(100 + D + order)
    for _ in range(5):
        c, W, f, u, T, up, Tp = random_case(rng, D)
        B = W[:, None] * grad_basis(c, order)
        assert B.shape[1] == nparam
        vp = np.sqrt(Tp) * c + up[None, :]
        rows, rhs = [], []
        Min = lab_moments(f, c, u, T, order)
        for k in range(order + 1):
            for idx in itertools.product(range(D), repeat=k):
                w = np.ones(len(W))
                for a in idx:
                    w = w * vp[:, a]
                rows.append(w @ B)
                rhs.append(Min[k][idx] if k else Min[0])
        coef, *_ = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)
        np.testing.assert_allclose(O.grad_transform(D, order, f, u, T, up, Tp), B @ coef,
                                   rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("D", [1, 2])
def test_identity_round_trip_and_idempotence(D):
    rng = np.random.default_rng(42 + D)
    for _ in range(10):
        c, W, f, u, T, up, Tp = random_case(rng, D)
        g3 = O.grad_transform(D, 3, f, u, T, u, T)           # Grad form in lambda
        np.testing.assert_allclose(O.grad_transform(D, 3, g3, u, T, u, T), g3, atol=1e-13)  # idempotent
        there = O.grad_transform(D, 3, g3, u, T, up, Tp)
        back = O.grad_transform(D, 3, there, up, Tp, u, T)
        np.testing.assert_allclose(back, g3, atol=1e-12)     # round trip on Grad-form populations
        if D == 1:  # four populations, four moments: the f-transform is a change of basis
            np.testing.assert_allclose(g3, f, atol=1e-13)


def test_equilibrium_maps_to_equilibrium():
    """f^eq = rho W_i in frame (u, T) is the Maxwellian; in its own frame it stays rho W_i,
    and its conserved moments are rho, rho u, rho u^2/2 + D rho T/2 (Eqs. feqPond, E)."""
    for D in (1, 2):
        c, W, _ = O.lattice(D)
        rho, u, T = 1.7, np.array([0.4, -0.3])[:D], 0.8
        feq = rho * W
        M = lab_moments(feq, c, u, T, 2)
        assert M[0] == pytest.approx(rho)
        np.testing.assert_allclose(M[1], rho * u, atol=1e-14)
        np.testing.assert_allclose(M[2], rho * np.outer(u, u) + rho * T * np.eye(D), atol=1e-14)
