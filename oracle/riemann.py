"""Exact solution of the Riemann problem for the ideal-gas Euler equations.

TEST INFRASTRUCTURE ONLY.  The paper compares its 1D shock tubes (Sod, Lax, strong
shock, double rarefaction, 1D jet; Sec. IV.A-IV.C) against an exact Riemann solver;
this module is that yardstick, written from the gas dynamics: the star pressure is
the root of f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is the shock (Rankine-
Hugoniot) branch for p > p_K and the isentropic rarefaction branch for p <= p_K;
the wave pattern is then sampled at x/t.  Vacuum generation (two receding
rarefactions whose Riemann invariants do not overlap) is handled explicitly.
"""
from __future__ import annotations

import math

import numpy as np


def _fk(p, rho, pk, a, g):
    """Velocity change across the K-wave as a function of the star pressure, and its derivative."""
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        q = math.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (p + B))
    # rarefaction
    e = (g - 1.0) / (2.0 * g)
    return (2.0 * a / (g - 1.0)) * ((p / pk) ** e - 1.0), (1.0 / (rho * a)) * (p / pk) ** (-(g + 1.0) / (2.0 * g))


class RiemannSolution:
    """Exact solution for left/right states (rho, u, p) and ratio of specific heats g."""

    def __init__(self, left, right, gamma):
        self.rl, self.ul, self.pl = map(float, left)
        self.rr, self.ur, self.pr = map(float, right)
        self.g = float(gamma)
        g = self.g
        self.al = math.sqrt(g * self.pl / self.rl)
        self.ar = math.sqrt(g * self.pr / self.rr)
        self.vacuum = (2.0 / (g - 1.0)) * (self.al + self.ar) <= self.ur - self.ul
        if self.vacuum:
            self.pstar = 0.0
            self.ustar = float("nan")
            return
        self.pstar = self._solve_pstar()
        fl, _ = _fk(self.pstar, self.rl, self.pl, self.al, g)
        fr, _ = _fk(self.pstar, self.rr, self.pr, self.ar, g)
        self.ustar = 0.5 * (self.ul + self.ur) + 0.5 * (fr - fl)
        self.rstar_l = self._rho_star(self.rl, self.pl)
        self.rstar_r = self._rho_star(self.rr, self.pr)

    def _f(self, p):
        fl, dl = _fk(p, self.rl, self.pl, self.al, self.g)
        fr, dr = _fk(p, self.rr, self.pr, self.ar, self.g)
        return fl + fr + (self.ur - self.ul), dl + dr

    def _solve_pstar(self):
        g = self.g
        # two-rarefaction estimate as starting value, then safeguarded Newton on [lo, hi]
        e = (g - 1.0) / (2.0 * g)
        num = self.al + self.ar - 0.5 * (g - 1.0) * (self.ur - self.ul)
        den = self.al / self.pl ** e + self.ar / self.pr ** e
        p = max((num / den) ** (1.0 / e), 1e-300) if num > 0 else 1e-12 * min(self.pl, self.pr)
        lo, hi = 0.0, max(self.pl, self.pr, p)
        while self._f(hi)[0] < 0.0:
            hi *= 2.0
        for _ in range(200):
            fv, dv = self._f(p)
            if fv > 0.0:
                hi = min(hi, p)
            else:
                lo = max(lo, p)
            pn = p - fv / dv if dv > 0 else 0.5 * (lo + hi)
            if not (lo < pn < hi):
                pn = 0.5 * (lo + hi)
            if abs(pn - p) <= 1e-15 * max(p, 1e-300) or hi - lo <= 1e-15 * hi:
                p = pn
                break
            p = pn
        return p

    def _rho_star(self, rk, pk):
        g, p = self.g, self.pstar
        if p > pk:
            r = p / pk
            gm = (g - 1.0) / (g + 1.0)
            return rk * (r + gm) / (gm * r + 1.0)
        return rk * (p / pk) ** (1.0 / g)

    def shock_speed(self, side):
        """Speed of the shock on side 'L' or 'R' (None if that wave is a rarefaction)."""
        g = self.g
        if side == "L":
            if self.pstar <= self.pl:
                return None
            return self.ul - self.al * math.sqrt((g + 1.0) / (2.0 * g) * self.pstar / self.pl + (g - 1.0) / (2.0 * g))
        if self.pstar <= self.pr:
            return None
        return self.ur + self.ar * math.sqrt((g + 1.0) / (2.0 * g) * self.pstar / self.pr + (g - 1.0) / (2.0 * g))

    def sample(self, s):
        """(rho, u, p) at similarity coordinate s = (x - x0)/t; s may be an array."""
        s = np.atleast_1d(np.asarray(s, dtype=np.float64))
        out = np.array([self._sample1(float(v)) for v in s])
        return out[:, 0], out[:, 1], out[:, 2]

    def _sample1(self, s):
        g = self.g
        rl, ul, pl, al = self.rl, self.ul, self.pl, self.al
        rr, ur, pr, ar = self.rr, self.ur, self.pr, self.ar
        if self.vacuum:
            sl_tail = ul + 2.0 * al / (g - 1.0)
            sr_tail = ur - 2.0 * ar / (g - 1.0)
            if s <= ul - al:
                return rl, ul, pl
            if s < sl_tail:
                return self._fan_left(s)
            if s <= sr_tail:
                return 0.0, 0.5 * (sl_tail + sr_tail), 0.0
            if s < ur + ar:
                return self._fan_right(s)
            return rr, ur, pr
        ps, us = self.pstar, self.ustar
        if s <= us:  # left of the contact
            if ps > pl:
                S = self.shock_speed("L")
                return (rl, ul, pl) if s <= S else (self.rstar_l, us, ps)
            head = ul - al
            a_star = al * (ps / pl) ** ((g - 1.0) / (2.0 * g))
            tail = us - a_star
            if s <= head:
                return rl, ul, pl
            if s >= tail:
                return self.rstar_l, us, ps
            return self._fan_left(s)
        if ps > pr:
            S = self.shock_speed("R")
            return (rr, ur, pr) if s >= S else (self.rstar_r, us, ps)
        head = ur + ar
        a_star = ar * (ps / pr) ** ((g - 1.0) / (2.0 * g))
        tail = us + a_star
        if s >= head:
            return rr, ur, pr
        if s <= tail:
            return self.rstar_r, us, ps
        return self._fan_right(s)

    def _fan_left(self, s):
        g, rl, ul, pl, al = self.g, self.rl, self.ul, self.pl, self.al
        # left-facing fan: u - a = s, u + 2a/(g-1) constant, p rho^-g constant
        c = 2.0 / (g + 1.0) + (g - 1.0) / ((g + 1.0) * al) * (ul - s)
        c = max(c, 0.0)
        return rl * c ** (2.0 / (g - 1.0)), 2.0 / (g + 1.0) * (al + 0.5 * (g - 1.0) * ul + s), pl * c ** (2.0 * g / (g - 1.0))

    def _fan_right(self, s):
        g, rr, ur, pr, ar = self.g, self.rr, self.ur, self.pr, self.ar
        c = 2.0 / (g + 1.0) - (g - 1.0) / ((g + 1.0) * ar) * (ur - s)
        c = max(c, 0.0)
        return rr * c ** (2.0 / (g - 1.0)), 2.0 / (g + 1.0) * (-ar + 0.5 * (g - 1.0) * ur + s), pr * c ** (2.0 * g / (g - 1.0))


def exact_profile(left, right, gamma, x, x0, t):
    """(rho, u, p) of the exact solution at positions x and time t > 0 for a split at x0."""
    sol = RiemannSolution(left, right, gamma)
    return sol.sample((np.asarray(x) - x0) / t)


def cell_averaged_profile(left, right, gamma, x_edges, x0, t, sub=16):
    """Exact solution averaged over each cell [x_edges[k], x_edges[k+1]] with `sub` midpoint samples."""
    x_edges = np.asarray(x_edges, dtype=np.float64)
    n = x_edges.size - 1
    frac = (np.arange(sub) + 0.5) / sub
    xs = (x_edges[:-1, None] + (x_edges[1:] - x_edges[:-1])[:, None] * frac[None, :]).ravel()
    r, u, p = exact_profile(left, right, gamma, xs, x0, t)
    return r.reshape(n, sub).mean(1), u.reshape(n, sub).mean(1), p.reshape(n, sub).mean(1)
