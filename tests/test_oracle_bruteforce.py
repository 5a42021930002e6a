"""Brute force on tiny periodic grids: a second, independent implementation of the
finite-volume step (Secs. II.C, III.B) in extended precision (numpy long double), written
population by population, against the oracle.

The brute force takes the regularized transformation through central Hermite moments (the
Grad form written as a Hermite expansion in the new frame, not the oracle's Eqs. a0-a3 in
lab moments), iterates every face corrector to its fixed point (up to 300 passes, until the
frame stops moving in extended precision), and assembles fluxes and updates cell by cell.
It follows the same readings as the oracle (initial face predictor, van Leer slopes over
one-sided differences, upwind tie-break, face populations at the frame of the last pass's
moments).  It pins the oracle's step after a few steps to 1e-12 and checks that every face
frame it converged to is a fixed point of the corrector map to 1e-14.

The semi-Lagrangian step (Sec. III.A) has its own brute force on the same footing: each
node's frame iterated to its fixed point, the cubic interpolant through the four nearest
nodes evaluated by Neville's recursion (the oracle uses Lagrange weights), the limiter's
linear fallback, and the BGK collision of the transformed populations."""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from tests.common import max_rel

LD = np.longdouble


def d1q4():
    s6 = np.sqrt(LD(6))
    c = np.array([-np.sqrt(LD(3) + s6), -np.sqrt(LD(3) - s6), np.sqrt(LD(3) - s6), np.sqrt(LD(3) + s6)])
    w = np.array([(LD(3) - s6) / 12, (LD(3) + s6) / 12, (LD(3) + s6) / 12, (LD(3) - s6) / 12])
    return c, w


def lattice(D):
    c1, w1 = d1q4()
    if D == 1:
        return c1[:, None], w1
    idx = list(itertools.product(range(4), repeat=D))
    return (np.array([[c1[k] for k in i] for i in idx], dtype=LD),
            np.array([np.prod([w1[k] for k in i]) for i in idx], dtype=LD))


def he(n, x):
    return [np.ones_like(x), x, x * x - 1, x ** 3 - 3 * x][n]


class Brute:
    """One periodic grid (nx; nx x ny; nx x ny x nz cells), state as populations per cell."""

    def __init__(self, D, shape, dx, gamma, tau, cfl):
        self.D, self.shape = D, shape
        # cell size along each axis (a scalar: the same along all of them)
        self.sp = np.array(list(dx) if np.ndim(dx) else [dx] * D, dtype=LD)
        self.c, self.W = lattice(D)
        self.Q = len(self.W)
        self.Cv = LD(1) / (LD(gamma) - 1)
        self.tau, self.cfl = LD(tau), LD(cfl)
        self.orders = [o for o in itertools.product(range(4), repeat=D)]
        self.cmax = max(abs(self.c.astype(float)).ravel())

    # ---- regularized transformation through central Hermite moments
    def transform(self, f, u, T, u2, T2, order):
        v = np.sqrt(T) * self.c + u[None, :]
        xi = (v - u2[None, :]) / np.sqrt(T2)
        out = np.zeros(self.Q, dtype=LD)
        for o in self.orders:
            if sum(o) > order:
                continue
            a = np.sum(f * np.prod([he(o[k], xi[:, k]) for k in range(self.D)], axis=0))
            basis = np.prod([he(o[k], self.c[:, k]) for k in range(self.D)], axis=0)
            out += a * basis / np.prod([math.factorial(k) for k in o])
        return self.W * out

    def moments(self, f, g, u, T):
        v = np.sqrt(T) * self.c + u[None, :]
        rho = f.sum()
        m = (f[:, None] * v).sum(0)
        E = (0.5 * (v * v).sum(1) * f).sum() + g.sum()
        uu = m / rho
        Tn = (E - 0.5 * (m * m).sum() / rho) / (self.Cv * rho)
        return rho, uu, Tn

    def equilibria(self, rho, T):
        return rho * self.W, (self.Cv - LD(self.D) / 2) * T * rho * self.W

    # ---- grid helpers (periodic)
    def cells(self):
        return list(itertools.product(*[range(n) for n in self.shape]))

    def at(self, cell, axis, off):
        c = list(cell)
        c[axis] = (c[axis] + off) % self.shape[axis]
        return tuple(c)

    def set_state(self, f, g, u, T):
        self.f, self.g, self.u, self.T = f, g, u, T

    def init_faces(self):
        self.face = {}
        for cell in self.cells():
            for a in range(self.D):
                L = self.at(cell, a, -1)
                rA, uA, TA = self.moments(self.f[L], self.g[L], self.u[L], self.T[L])
                rB, uB, TB = self.moments(self.f[cell], self.g[cell], self.u[cell], self.T[cell])
                EA = rA * (self.Cv * TA + 0.5 * (uA * uA).sum())
                EB = rB * (self.Cv * TB + 0.5 * (uB * uB).sum())
                r, m, E = (rA + rB) / 2, (rA * uA + rB * uB) / 2, (EA + EB) / 2
                self.face[(cell, a)] = (m / r, (E - 0.5 * (m * m).sum() / r) / (self.Cv * r))

    minmod = False   # the other limiter the paper names (Sec. III.B.3)

    def vanleer(self, a, b):
        """The slope from the two one-sided differences: van Leer's harmonic form, or minmod."""
        if self.minmod:
            return LD(0) if a * b <= 0 else (a if abs(a) < abs(b) else b)
        den = abs(a) + abs(b)
        return np.where(den == 0, LD(0), (np.sign(a) + np.sign(b)) * abs(a) * abs(b) / np.where(den == 0, 1, den))

    def face_pass(self, cell, a, fp, gp, lam_u, lam_T, h):
        """One corrector pass at the face of axis a below `cell`: reconstructed populations."""
        L, R = self.at(cell, a, -1), cell
        LL, RR = self.at(cell, a, -2), self.at(cell, a, 1)
        tang = [t for t in range(self.D) if t != a]
        need = {L, R, LL, RR}
        for t in tang:
            for base in (L, R):
                need |= {self.at(base, t, -1), self.at(base, t, 1)}
        P = {k: (self.transform(fp[k], self.u[k], self.T[k], lam_u, lam_T, 3),
                 self.transform(gp[k], self.u[k], self.T[k], lam_u, lam_T, 2)) for k in need}
        v = np.sqrt(lam_T) * self.c + lam_u[None, :]
        out = []
        for pop in range(2):
            val = np.zeros(self.Q, dtype=LD)
            for i in range(self.Q):
                up, lo, hi = (L, LL, R) if v[i, a] > 0 else (R, L, RR)
                off = (self.sp[a] / 2 if v[i, a] > 0 else -self.sp[a] / 2) - v[i, a] * h
                s = self.vanleer((P[up][pop][i] - P[lo][pop][i]) / self.sp[a], (P[hi][pop][i] - P[up][pop][i]) / self.sp[a])
                x = P[up][pop][i] + off * s
                for t in tang:
                    st = self.vanleer((P[up][pop][i] - P[self.at(up, t, -1)][pop][i]) / self.sp[t],
                                      (P[self.at(up, t, 1)][pop][i] - P[up][pop][i]) / self.sp[t])
                    x += -v[i, t] * h * st
                val[i] = x
            out.append(val)
        return out

    def step(self, passes=300):
        D, h = self.D, None
        # 1. every cell in its own frame
        for k in self.cells():
            rho, u, T = self.moments(self.f[k], self.g[k], self.u[k], self.T[k])
            self.f[k] = self.transform(self.f[k], self.u[k], self.T[k], u, T, 3)
            self.g[k] = self.transform(self.g[k], self.u[k], self.T[k], u, T, 2)
            self.u[k], self.T[k] = u, T
        rate = max(((abs(self.u[k]) + np.sqrt(self.T[k]) * LD(self.cmax)) / self.sp).max() for k in self.cells())
        dt = self.cfl / rate
        h, tau = dt / 2, self.tau
        cp, ce = (2 * tau - h) / (2 * tau + dt), 3 * h / (2 * tau + dt)
        fp, gp = {}, {}
        for k in self.cells():
            feq, geq = self.equilibria(self.f[k].sum(), self.T[k])
            fp[k], gp[k] = cp * self.f[k] + ce * feq, cp * self.g[k] + ce * geq
        # 2. faces to their fixed points
        faces, self.residual = {}, 0.0
        for key, (lu, lT) in self.face.items():
            cell, a = key
            for _ in range(passes):
                fb, gb = self.face_pass(cell, a, fp, gp, lu, lT, h)
                rho, nu, nT = self.moments(fb, gb, lu, lT)
                moved = max(abs(nu - lu).max() / np.sqrt(lT), abs(nT - lT) / lT)
                lu_prev, lT_prev = lu, lT
                lu, lT = nu, nT
                if moved < LD(1e-17):
                    break
            # populations of the last pass in the frame of their own moments, Eq. (FluxTransf)
            fb2 = self.transform(fb, lu_prev, lT_prev, lu, lT, 3)
            gb2 = self.transform(gb, lu_prev, lT_prev, lu, lT, 2)
            feq, geq = self.equilibria(rho, lT)
            faces[key] = ((2 * tau * fb2 + h * feq) / (2 * tau + h), (2 * tau * gb2 + h * geq) / (2 * tau + h), lu, lT)
            self.face[key] = (lu, lT)
            # fixed-point residual: one more pass from the converged frame
            fb3, gb3 = self.face_pass(cell, a, fp, gp, lu, lT, h)
            _, ru, rT = self.moments(fb3, gb3, lu, lT)
            self.residual = max(self.residual, float(max(abs(ru - lu).max() / np.sqrt(lT), abs(rT - lT) / lT)))
        # 3. fluxes into each cell's frame and the update
        ca, cb = (2 * tau - dt) / (2 * tau + dt), 2 * dt / (2 * tau + dt)
        newf, newg = {}, {}
        for k in self.cells():
            Ff, Fg = np.zeros(self.Q, dtype=LD), np.zeros(self.Q, dtype=LD)
            vk = np.sqrt(self.T[k]) * self.c + self.u[k][None, :]
            for a in range(D):
                for side, key in ((-1, (k, a)), (+1, (self.at(k, a, 1), a))):
                    ff, gg, lu, lT = faces[key]
                    pf = self.transform(ff, lu, lT, self.u[k], self.T[k], 3)
                    pg = self.transform(gg, lu, lT, self.u[k], self.T[k], 2)
                    Ff += side * vk[:, a] * pf / self.sp[a]
                    Fg += side * vk[:, a] * pg / self.sp[a]
            feq, geq = self.equilibria(self.f[k].sum(), self.T[k])
            newf[k] = ca * self.f[k] + cb * feq - dt * Ff
            newg[k] = ca * self.g[k] + cb * geq - dt * Fg
        self.f, self.g = newf, newg
        return dt

    def conserved(self):
        out = []
        for k in self.cells():
            rho, u, T = self.moments(self.f[k], self.g[k], self.u[k], self.T[k])
            out.append([rho, *(rho * u), rho * (self.Cv * T + 0.5 * (u * u).sum())])
        return np.array(out, dtype=float)


def random_state(D, shape, seed):
    rng = np.random.default_rng(seed)
    c, W = lattice(D)
    n = int(np.prod(shape))
    f = [W * (LD(1.0 + 0.3 * rng.uniform(-1, 1)) * (1 + LD(0.05) * rng.uniform(-1, 1, len(W)).astype(LD))) for _ in range(n)]
    g = [W * LD(1.5 + 0.3 * rng.uniform(-1, 1)) * (1 + LD(0.05) * rng.uniform(-1, 1, len(W)).astype(LD)) for _ in range(n)]
    u = [rng.uniform(-0.5, 0.5, D).astype(LD) for _ in range(n)]
    T = [LD(np.exp(rng.uniform(-0.3, 0.3))) for _ in range(n)]
    return f, g, u, T


@pytest.mark.parametrize("D,shape,seed,steps,minmod", [(1, (3,), 1, 2, False), (1, (5,), 2, 2, False),
                                                       (1, (8,), 3, 2, False), (2, (3, 3), 4, 2, False),
                                                       (1, (5,), 10, 2, True), (2, (3, 3), 11, 2, True),
                                                       (2, (3, 4), 12, 2, False), (3, (3, 3, 4), 5, 1, False)],
                         ids=["1d_3", "1d_5", "1d_8", "2d_3x3", "1d_5_minmod", "2d_3x3_minmod", "2d_3x4_nonsquare",
                              "3d_3x3x4"])
def test_oracle_step_equals_brute_force(D, shape, seed, steps, minmod):
    """The D3Q64 case (one step, about 40 s) pins the three-dimensional stencil: the normal
    and both tangential slopes of every face, and the fluxes of the three axes.  The 3 x 4
    field has non-square cells (1/3 x 1/4), which pins the spacing used along each axis."""
    gamma, tau, cfl = 1.4, 1e-3, 0.3
    sp = [1.0 / n for n in shape]   # unit box: non-square cells where the sides differ
    f, g, u, T = random_state(D, shape, seed)
    bf = Brute(D, shape, sp, gamma, tau, cfl)
    bf.minmod = minmod
    cells = bf.cells()
    # the brute force keys cells as (i,), (i, j) or (i, j, k); the oracle's order is x fastest
    order = sorted(cells, key=lambda k: tuple(reversed(k)))
    bf.set_state({k: f[n] for n, k in enumerate(order)}, {k: g[n] for n, k in enumerate(order)},
                 {k: u[n] for n, k in enumerate(order)}, {k: T[n] for n, k in enumerate(order)})
    bf.init_faces()
    nx, ny, nz = (tuple(shape) + (1, 1))[:3]
    n = nx * ny * nz
    sp3 = (sp + [1.0, 1.0])[:3]
    s = O.make_solver(D, nx, ny, nz, dx=sp3[0], dy=sp3[1], dz=sp3[2], gamma=gamma, tau=tau, cfl=cfl, bc=(1,) * (2 * max(D, 2)),
                      tol=1e-15, max_iter=300, limiter=O.MINMOD if minmod else O.VANLEER)
    if D == 3:
        s.set_primitive3(np.ones(n), np.zeros(n), np.zeros(n), np.zeros(n), np.ones(n))
    else:
        s.set_primitive(np.ones(n), np.zeros(n), np.zeros(n) if D == 2 else None, np.ones(n))
    s.set_state(np.array([np.asarray(x, dtype=float) for x in f]), np.array([np.asarray(x, dtype=float) for x in g]),
                np.array([np.asarray(x, dtype=float) for x in u]), np.array([float(x) for x in T]))
    # oracle columns (rho, m..., E) holding the brute force's (rho, m_1..m_D, E)
    cols = {1: [0, 1, 3], 2: [0, 1, 2, 3], 3: [0, 1, 2, 3, 4]}[D]
    for _ in range(steps):
        dt_b = bf.step()
        s.step(1)
        assert s.stats()["dt"] == pytest.approx(float(dt_b), rel=1e-13)
        assert s.stats()["nonconverged"] == 0
        assert bf.residual <= 1e-14
        want = bf.conserved()[[cells.index(k) for k in order]]
        got = np.stack(s.conserved(), 1)
        for j, col in enumerate(cols):
            if 0 < j <= D:   # momentum: absolute, on the scale of the energy
                scale = max(np.abs(want[:, -1]).max(), 1.0)
                assert np.abs(got[:, col] - want[:, j]).max() <= 1e-12 * scale, (col, got[:, col], want[:, j])
            else:
                assert max_rel(got[:, col], want[:, j]) <= 1e-12, (col, got[:, col], want[:, j])


# ---------------------------------------------------------------- semi-Lagrangian step

def neville(xs, ys, x):
    """Value at x of the polynomial through the points (xs, ys), by Neville's recursion."""
    p = list(ys)
    n = len(xs)
    for k in range(1, n):
        for i in range(n - k):
            p[i] = ((x - xs[i + k]) * p[i] + (xs[i] - x) * p[i + 1]) / (xs[i] - xs[i + k])
    return p[0]


class BruteSL(Brute):
    """The semi-Lagrangian step (Sec. III.A) on the same periodic grids: every node iterates
    its own frame; a pass re-expresses the 5 (or 5 x 5) surrounding nodes in the pass's frame
    and takes each population at its departure point x - v_i dt from the cubic through the
    four nearest nodes along each axis (the tensor product in 2D), replaced by the linear
    (bilinear) interpolant of the bracketing nodes when it leaves their range (the reading
    for the thesis-only limiter); BGK collision with beta = dt / (2 tau + dt)."""

    def interp(self, vals, theta):
        """vals over offsets -1..2 along x (1D) or [y][x] (2D); theta = fractions in [0, 1)."""
        xs = [LD(-1), LD(0), LD(1), LD(2)]
        if self.D == 1:
            p = neville(xs, vals, theta[0])
            lo, hi = min(vals[1], vals[2]), max(vals[1], vals[2])
            if p < lo or p > hi:
                p = vals[1] + theta[0] * (vals[2] - vals[1])
            return p
        rows = [neville(xs, vals[r], theta[0]) for r in range(4)]
        p = neville(xs, rows, theta[1])
        br = [vals[1][1], vals[1][2], vals[2][1], vals[2][2]]
        if p < min(br) or p > max(br):
            a = vals[1][1] + theta[0] * (vals[1][2] - vals[1][1])
            b = vals[2][1] + theta[0] * (vals[2][2] - vals[2][1])
            p = a + theta[1] * (b - a)
        return p

    def node_pass(self, k, lam_u, lam_T, dt):
        near = {}
        for off in itertools.product(range(-2, 3), repeat=self.D):
            cell = k
            for a in range(self.D):
                cell = self.at(cell, a, off[a])
            near[off] = (self.transform(self.f[cell], self.u[cell], self.T[cell], lam_u, lam_T, 3),
                         self.transform(self.g[cell], self.u[cell], self.T[cell], lam_u, lam_T, 2))
        v = np.sqrt(lam_T) * self.c + lam_u[None, :]
        out = [np.zeros(self.Q, dtype=LD), np.zeros(self.Q, dtype=LD)]
        for i in range(self.Q):
            base, theta = [], []
            for a in range(self.D):
                xd = -v[i, a] * dt / self.sp[a]       # departure point in node units
                b = int(np.floor(xd))
                base.append(b)
                theta.append(xd - b)
            for pop in range(2):
                if self.D == 1:
                    vals = [near[(base[0] + m,)][pop][i] for m in (-1, 0, 1, 2)]
                else:
                    vals = [[near[(base[0] + m, base[1] + r)][pop][i] for m in (-1, 0, 1, 2)] for r in (-1, 0, 1, 2)]
                out[pop][i] = self.interp(vals, theta)
        return out

    def step(self, passes=300):
        rate = max(((abs(self.u[k]) + np.sqrt(self.T[k]) * LD(self.cmax)) / self.sp).max() for k in self.cells())
        dt = self.cfl / rate
        beta = dt / (2 * self.tau + dt)
        new, self.residual = {}, 0.0
        for k in self.cells():
            lu, lT = self.u[k], self.T[k]
            for _ in range(passes):
                fb, gb = self.node_pass(k, lu, lT, dt)
                rho, nu, nT = self.moments(fb, gb, lu, lT)
                moved = max(abs(nu - lu).max() / np.sqrt(lT), abs(nT - lT) / lT)
                lu_prev, lT_prev, lu, lT = lu, lT, nu, nT
                if moved < LD(1e-17):
                    break
            fl = self.transform(fb, lu_prev, lT_prev, lu, lT, 3)
            gl = self.transform(gb, lu_prev, lT_prev, lu, lT, 2)
            feq, geq = self.equilibria(rho, lT)
            new[k] = (fl + 2 * beta * (feq - fl), gl + 2 * beta * (geq - gl), lu, lT)
            fb3, gb3 = self.node_pass(k, lu, lT, dt)
            _, ru, rT = self.moments(fb3, gb3, lu, lT)
            self.residual = max(self.residual, float(max(abs(ru - lu).max() / np.sqrt(lT), abs(rT - lT) / lT)))
        for k, (f, g, u, T) in new.items():
            self.f[k], self.g[k], self.u[k], self.T[k] = f, g, u, T
        return dt


@pytest.mark.parametrize("D,shape,seed", [(1, (5,), 6), (1, (7,), 9), (2, (5, 4), 13)], ids=["1d_5", "1d_7", "2d_5x4"])
def test_oracle_sl_step_equals_brute_force(D, shape, seed):
    """Two semi-Lagrangian steps of the oracle (tol 1e-15) against the brute force: the
    conserved fields to 1e-12 and the time steps to 1e-13; every node frame the brute force
    converged to is a fixed point of its corrector map.  The 2D field has non-square cells
    (1/5 x 1/4).  (On the 7-node tube with seed 7, and on this field with seed 8, one node's
    corrector cycles without converging in both implementations, in long double too: the
    limiter's switch to the linear interpolant makes the corrector map discontinuous.  The
    two still agree to 1e-15 there.)"""
    gamma, tau, cfl = 1.4, 1e-3, 0.3
    sp = [1.0 / n for n in shape]
    f, g, u, T = random_state(D, shape, seed)
    bf = BruteSL(D, shape, sp, gamma, tau, cfl)
    cells = bf.cells()
    order = sorted(cells, key=lambda k: tuple(reversed(k)))
    bf.set_state({k: f[n] for n, k in enumerate(order)}, {k: g[n] for n, k in enumerate(order)},
                 {k: u[n] for n, k in enumerate(order)}, {k: T[n] for n, k in enumerate(order)})
    nx, ny = (tuple(shape) + (1,))[:2]
    n = nx * ny
    s = O.make_solver(D, nx, ny, dx=sp[0], dy=(sp + [1.0])[1], gamma=gamma, tau=tau, cfl=cfl, bc=(1, 1, 1, 1), tol=1e-15,
                      max_iter=300)
    s.set_primitive(np.ones(n), np.zeros(n), np.zeros(n) if D == 2 else None, np.ones(n))
    s.set_state(np.array([np.asarray(x, dtype=float) for x in f]), np.array([np.asarray(x, dtype=float) for x in g]),
                np.array([np.asarray(x, dtype=float) for x in u]), np.array([float(x) for x in T]))
    cols = [0, 1, 3] if D == 1 else [0, 1, 2, 3]
    for _ in range(2):
        dt_b = bf.step()
        s.sl_step(1)
        assert s.stats()["dt"] == pytest.approx(float(dt_b), rel=1e-13)
        assert s.stats()["nonconverged"] == 0 and s.stats()["fallbacks"] == 0
        assert bf.residual <= 1e-14
        want = bf.conserved()[[cells.index(k) for k in order]]
        got = np.stack(s.conserved(), 1)
        for j, col in enumerate(cols):
            if 0 < j <= D:
                scale = max(np.abs(want[:, -1]).max(), 1.0)
                assert np.abs(got[:, col] - want[:, j]).max() <= 1e-12 * scale, (col, got[:, col], want[:, j])
            else:
                assert max_rel(got[:, col], want[:, j]) <= 1e-12, (col, got[:, col], want[:, j])
