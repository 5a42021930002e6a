"""The oracle's corrector when a pass defines no frame (reading of Sec. III.B.3, which only
says to iterate until convergence): restart once from the frame of the pooled conserved
moments of the whole face stencil (4 cells in 1D, 8 in 2D), otherwise stop and keep the
frame defined by the moments of the last pass that did define one.

Pinned against the independent long-double brute force of the step
(tests/test_oracle_bruteforce.py): periodic grids with strong contrasts, and a face whose
predictor is set far from its stencil so that its passes follow a chosen sequence of valid
(v) and frame-less (X) passes.  The expected face frame is computed here: the passes by the
brute force, the restart frame from the stencil cells' conserved moments (rho = sum f,
rho u = sum v f, rho E = sum |v|^2/2 f + sum g, Sec. II.B), pooled as plain means.  Each
case also checks that the plausible misreadings -- pooling only the two cells next to the
face, averaging the cells' frames instead of their conserved moments, keeping the frame a
pass ran in instead of the frame its moments define -- give a different face frame, so a
mistake of that kind in the oracle would fail here."""
import numpy as np
import pytest

import oracle as O
from tests.test_oracle_bruteforce import LD, Brute, lattice


def state(D, shape, seed):
    """Cells with densities over e^[-2,2], temperatures over e^[-3,3], velocities up to 2 and
    5% non-equilibrium noise (populations in the cell's frame (u, T))."""
    rng = np.random.default_rng(seed)
    c, W = lattice(D)
    f, g, u, T = [], [], [], []
    for _ in range(int(np.prod(shape))):
        rho = LD(np.exp(rng.uniform(-2, 2)))
        Tk = LD(np.exp(rng.uniform(-3, 3)))
        f.append(W * rho * (1 + LD(0.05) * rng.uniform(-1, 1, len(W)).astype(LD)))
        g.append(W * rho * Tk * LD(1.5) * (1 + LD(0.05) * rng.uniform(-1, 1, len(W)).astype(LD)))
        u.append(rng.uniform(-2.0, 2.0, D).astype(LD))
        T.append(Tk)
    return f, g, u, T


def regauge_and_stage(bf):
    """Step 1 of the algorithm (every cell in its own frame), the CFL time step and
    phi-bar-plus (Eq. Fbarplus), as the brute force's step does."""
    for k in bf.cells():
        rho, u, T = bf.moments(bf.f[k], bf.g[k], bf.u[k], bf.T[k])
        bf.f[k] = bf.transform(bf.f[k], bf.u[k], bf.T[k], u, T, 3)
        bf.g[k] = bf.transform(bf.g[k], bf.u[k], bf.T[k], u, T, 2)
        bf.u[k], bf.T[k] = u, T
    rate = max(((abs(bf.u[k]) + np.sqrt(bf.T[k]) * LD(bf.cmax)) / bf.sp).max() for k in bf.cells())
    dt = bf.cfl / rate
    h, tau = dt / 2, bf.tau
    cp, ce = (2 * tau - h) / (2 * tau + dt), 3 * h / (2 * tau + dt)
    fp, gp = {}, {}
    for k in bf.cells():
        feq, geq = bf.equilibria(bf.f[k].sum(), bf.T[k])
        fp[k], gp[k] = cp * bf.f[k] + ce * feq, cp * bf.g[k] + ce * geq
    return fp, gp, h


def stencil(bf, cell, a):
    """LL, L, R, RR along axis a, then (2D) the tangential neighbours of L and R."""
    L = bf.at(cell, a, -1)
    out = [bf.at(cell, a, -2), L, cell, bf.at(cell, a, 1)]
    for t in range(bf.D):
        if t != a:
            out += [bf.at(L, t, -1), bf.at(L, t, 1), bf.at(cell, t, -1), bf.at(cell, t, 1)]
    return out


def pooled_frame(bf, cells):
    """Frame of the mean conserved moments (rho, rho u, rho E) of the given cells."""
    r, m, e = LD(0), np.zeros(bf.D, dtype=LD), LD(0)
    for k in cells:
        c = bf.c
        v = np.sqrt(bf.T[k]) * c + bf.u[k][None, :]
        r += bf.f[k].sum()
        m += (bf.f[k][:, None] * v).sum(0)
        e += (0.5 * (v * v).sum(1) * bf.f[k]).sum() + bf.g[k].sum()
    r, m, e = r / len(cells), m / len(cells), e / len(cells)
    return m / r, (e - 0.5 * (m * m).sum() / r) / (bf.Cv * r)


def frame_average(bf, cells):
    return sum(bf.u[k] for k in cells) / len(cells), sum(bf.T[k] for k in cells) / len(cells)


def defines_frame(u, T):
    return T > 0 and np.isfinite(float(T)) and np.all(np.isfinite(u.astype(float)))


def corrector(bf, cell, a, fp, gp, h, lu, lT, passes, restart, keep_input=False, max_iter=8):
    """The corrector with the given restart frame: returns the pass sequence and the kept
    frame (the frame of the last valid pass's moments, or with keep_input the frame that
    pass ran in)."""
    seq, restarted, keep = "", False, None
    for k in range(max_iter):
        fb, gb = bf.face_pass(cell, a, fp, gp, lu, lT, h)
        _, u1, T1 = bf.moments(fb, gb, lu, lT)
        if not defines_frame(u1, T1):
            seq += "X"
            if not restarted:
                restarted = True
                lu, lT = restart
                continue
            break
        seq += "v"
        keep = (lu, lT) if keep_input else (u1, T1)
        if k + 1 >= passes:
            break
        lu, lT = u1, T1
    return seq, keep


# (D, shape, state seed, predictor velocity offset in units of sqrt(T), predictor T factor,
#  expected pass sequence with 3 passes)
CASES = [
    (1, (6,), 0, -8, 100.0, "Xvv"),    # restart, then two passes from the restart frame
    (1, (6,), 17, -5, 100.0, "XvX"),   # restart; the pass after the valid one defines no frame
    (1, (6,), 3, 8, 100.0, "vXX"),     # the restart's pass defines no frame: keep pass 1
    (1, (6,), 4, -8, 0.01, "vXv"),     # a valid pass, then a restart
    (2, (4, 4), 0, -3, 0.01, "Xvv"),
    (2, (4, 4), 14, -8, 0.01, "XvX"),
    (2, (4, 4), 13, 5, 1.0, "vXX"),
    (2, (4, 4), 1, -8, 1.0, "vXv"),
]


@pytest.mark.parametrize("D,shape,seed,d,s,seq", CASES, ids=["%dd_%s_seed%d" % (c[0], c[5], c[2]) for c in CASES])
def test_restart_and_last_valid_pass(D, shape, seed, d, s, seq):
    gamma, tau, cfl = 1.4, 1e-3, 0.3
    sp = [1.0 / n for n in shape]
    f, g, u, T = state(D, shape, seed)
    bf = Brute(D, shape, sp, gamma, tau, cfl)
    cells = bf.cells()
    order = sorted(cells, key=lambda k: tuple(reversed(k)))  # the oracle's order: x fastest
    bf.set_state({k: f[n] for n, k in enumerate(order)}, {k: g[n] for n, k in enumerate(order)},
                 {k: u[n] for n, k in enumerate(order)}, {k: T[n] for n, k in enumerate(order)})
    fp, gp, h = regauge_and_stage(bf)
    cell, a = cells[len(cells) // 2], 0
    st = stencil(bf, cell, a)
    Tm = np.mean([float(bf.T[k]) for k in st])
    lu = np.mean([bf.u[k] for k in st], axis=0)
    lu[0] += LD(d * np.sqrt(Tm))
    lT = LD(s * Tm)
    got_seq, keep = corrector(bf, cell, a, fp, gp, h, lu, lT, 3, pooled_frame(bf, st))
    assert got_seq == seq   # the case still exercises the branch it is meant for

    # the oracle: the same populations, the predictor at this face, three passes
    nx, ny = (tuple(shape) + (1,))[:2]
    n = nx * ny
    o = O.make_solver(D, nx, ny, dx=sp[0], dy=sp[1] if D == 2 else None, gamma=gamma, tau=tau, cfl=cfl,
                      bc=(1, 1, 1, 1), fixed_iters=3, max_iter=8)
    o.set_primitive(np.ones(n), np.zeros(n), np.zeros(n) if D == 2 else None, np.ones(n))
    o.set_state(np.array([np.asarray(x, dtype=float) for x in f]), np.array([np.asarray(x, dtype=float) for x in g]),
                np.array([np.asarray(x, dtype=float) for x in u]), np.array([float(x) for x in T]))
    xg, yg = o.face_gauges()
    fidx = cell[1] * (nx + 1) + cell[0] if D == 2 else cell[0]
    xg[fidx, :D] = np.asarray(lu, dtype=float)
    xg[fidx, D] = float(lT)
    o.set_face_gauges(xg, yg)
    o.step(1)
    got = o.face_gauges()[0][fidx]
    want_u, want_T = np.asarray(keep[0], dtype=float), float(keep[1])
    scale_u = np.sqrt(want_T)

    def err(fr):
        return max(np.abs(got[:D] - np.asarray(fr[0], dtype=float)).max() / scale_u,
                   abs(got[D] - float(fr[1])) / want_T)

    assert err((want_u, want_T)) <= 1e-11, (got, want_u, want_T)
    # the misreadings give other frames
    L, R = bf.at(cell, a, -1), cell
    alternatives = []
    if seq != "vXX":   # the restart frame decides the result
        alternatives += [corrector(bf, cell, a, fp, gp, h, lu, lT, 3, pooled_frame(bf, [L, R]))[1],
                         corrector(bf, cell, a, fp, gp, h, lu, lT, 3, frame_average(bf, st))[1]]
    alternatives.append(corrector(bf, cell, a, fp, gp, h, lu, lT, 3, pooled_frame(bf, st), keep_input=True)[1])
    for alt in alternatives:
        if alt is not None and defines_frame(np.asarray(alt[0]), alt[1]):
            assert err(alt) > 1e-6, alt
