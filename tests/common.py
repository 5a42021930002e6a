"""Helpers shared by the tests (problem -> oracle solver, error norms)."""
import numpy as np

import oracle as O


def oracle_for(problem, *, tau, cfl, t_end=0.0, tol=1e-10, max_iter=16, fixed_iters=0, limiter=0):
    if problem.dim == 3:
        s = O.make_solver(3, problem.nx, problem.ny, problem.nz, dx=problem.dx, dy=problem.dy, dz=problem.dz,
                          gamma=problem.gamma, tau=tau, cfl=cfl, t_end=t_end, bc=problem.bc, limiter=limiter,
                          tol=tol, max_iter=max_iter, fixed_iters=fixed_iters)
        s.set_primitive3(problem.rho, problem.ux, problem.uy, problem.uz, problem.p)
        return s
    s = O.make_solver(problem.dim, problem.nx, problem.ny, dx=problem.dx, dy=problem.dy,
                      gamma=problem.gamma, tau=tau, cfl=cfl, t_end=t_end, bc=problem.bc,
                      inflow=problem.inflow, inflow_range=problem.inflow_range, limiter=limiter,
                      tol=tol, max_iter=max_iter, fixed_iters=fixed_iters)
    s.set_primitive(problem.rho, problem.ux, problem.uy if problem.dim == 2 else None, problem.p)
    return s


def rel_l1(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).sum() / max(np.abs(np.asarray(b)).sum(), 1e-300))


def hermite_coeffs_1d(f, c):
    """Hermite moments a_k = sum_i f_i He_k(c_i), k = 0..3 (probabilists' Hermite)."""
    He = [np.ones_like(c), c, c * c - 1.0, c ** 3 - 3.0 * c]
    return np.array([np.dot(f, h) for h in He])


def hermite_of_pops(f, D):
    """Hermite moments of populations f [cells, Q] on D1Q4 / D2Q16 in the library's packed
    order (1D: a0..a3; 2D: 00 10 01 20 11 02 30 21 12 03), all orders up to 3."""
    c, W, _ = O.lattice(D)
    He = lambda k, x: [np.ones_like(x), x, x * x - 1.0, x ** 3 - 3.0 * x][k]
    if D == 1:
        return np.stack([f @ He(k, c[:, 0]) for k in range(4)], 1)
    cols = []
    for n in range(4):
        for s in range(n + 1):
            r = n - s
            cols.append(f @ (He(r, c[:, 0]) * He(s, c[:, 1])))
    return np.stack(cols, 1)


def max_rel(a, b):
    """max |a - b| / max |b| (field-wise relative error)."""
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def gpu_primitive(s):
    """Primitive fields of a GPU solver's grid from the conserved fields it returns (test
    helper; the library itself never converts): rho, ux, uy, p on 1D/2D grids and rho, ux,
    uy, uz, p on D3Q64 grids, with p = rho T and E = rho (Cv T + |u|^2 / 2), Cv = 1/(gamma - 1)."""
    out, _ = s.moments(totals=False)
    cv = 1.0 / (s.problem.gamma - 1.0)
    rho, E = out[0], out[-1]
    mom = out[1:-1]
    T = (E - 0.5 * sum(m * m for m in mom) / rho) / (cv * rho)
    return (rho, *[m / rho for m in mom], rho * T)


def gpu_primitive_tube(s, k, gamma):
    """rho, u, p of tube k of a batched GPU solver (test helper, as gpu_primitive)."""
    (rho, mx, _, E), _ = s.moments(totals=False)
    a, b = s.offsets[k], s.offsets[k + 1]
    r, m, e = rho[a:b], mx[a:b], E[a:b]
    cv = 1.0 / (gamma - 1.0)
    T = (e - 0.5 * m * m / r) / (cv * r)
    return r, m / r, r * T
