"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds only problem definitions: primitive fields (rho, u, p), grids,
boundary conditions and random draws.  It contains none of the method's arithmetic,
so both the CUDA library and the CPU oracle can be fed from it.

Workloads (paper Sec. IV; sizes of the benchmark configurations):
  - ``shock_tube``      two-state 1D Riemann problems (Sod, Lax, strong shock, jet ...)
  - ``quadrants_2d``    2D four-quadrant Riemann problem with seeded quadrant states
  - ``tube_batch``      thousands of 1D tubes of uneven length with seeded states
  - ``shocked_interface_2d``  planar shock hitting a perturbed density interface
  - ``jet_2d``          high-Mach jet entering a light ambient through a left inflow band
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

TRANSMISSIVE, PERIODIC, INFLOW, REFLECTIVE = 0, 1, 2, 3


@dataclass
class Problem:
    dim: int
    nx: int
    ny: int
    x0: float
    x1: float
    y0: float
    y1: float
    gamma: float
    rho: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    p: np.ndarray
    bc: tuple = (TRANSMISSIVE,) * 4
    inflow: np.ndarray = field(default_factory=lambda: np.zeros((4, 4)))
    inflow_range: np.ndarray = field(default_factory=lambda: np.zeros((4, 2), dtype=np.int64))
    name: str = ""

    @property
    def dx(self):
        return (self.x1 - self.x0) / self.nx

    @property
    def dy(self):
        return (self.y1 - self.y0) / self.ny if self.dim == 2 else 1.0

    @property
    def ncell(self):
        return self.nx * self.ny


def cell_centres(n, a, b):
    return a + (np.arange(n) + 0.5) * (b - a) / n


# Two-state tubes of the paper (Sec. IV.A-C): (left, right, gamma, x0, x1, x_split, t_end)
PAPER_TUBES = {
    "sod_classic": ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4, 0.0, 1.0, 0.5, 0.2),
    "sod_paper": ((1.0, 0.0, 0.15), (0.125, 0.0, 0.015), 1.4, 0.0, 1.0, 0.5, 0.2),
    "lax": ((0.445, 0.698, 3.528), (0.5, 0.0, 0.571), 1.4, 0.0, 1.0, 0.5, 0.14),
    "strong_shock": ((1.0, 0.0, 1000.0), (1.0, 0.0, 0.01), 1.4, 0.0, 1.0, 0.5, 0.012),
    "double_rarefaction": ((1.0, -2.0, 0.1), (1.0, 2.0, 0.1), 1.4, 0.0, 1.0, 0.5, 0.1),
    "jet_1d": ((5.0, 30.0, 0.4127), (0.5, 0.0, 0.4127), 5.0 / 3.0, 0.0, 2.0, 0.1, 0.06),
}


def shock_tube(left, right, gamma, n, x0=0.0, x1=1.0, x_split=0.5, name=""):
    """1D two-state Riemann problem; the left state holds where the cell centre < x_split."""
    x = cell_centres(n, x0, x1)
    L = x < x_split
    rho = np.where(L, left[0], right[0]).astype(np.float64)
    ux = np.where(L, left[1], right[1]).astype(np.float64)
    p = np.where(L, left[2], right[2]).astype(np.float64)
    return Problem(1, n, 1, x0, x1, 0.0, 1.0, float(gamma), rho, ux, np.zeros(n), p, name=name)


def paper_tube(name, n):
    left, right, g, x0, x1, xs, t_end = PAPER_TUBES[name]
    return shock_tube(left, right, g, n, x0, x1, xs, name=name), t_end


def sod_400():
    """Shock tube on [0,1]: (1, 0, 1) | (0.125, 0, 0.1) at x = 0.5, gamma 1.4, 400 cells."""
    return shock_tube((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4, 400, name="sod_400")


def quadrants_2d(n, seed, gamma=1.4, mach_max=3.0, direction="centre"):
    """2D four-quadrant Riemann problem on the unit square (n x n cells).

    Each quadrant draws rho and p log-uniform in [0.1, 10] and a Mach number uniform in
    [0, mach_max].  direction "centre" (the workload): its velocity points towards the
    domain centre within +-45 degrees, so that neighbouring quadrants meet in shocks,
    contacts and slip lines.  direction "any": uniform in [0, 2 pi), which also makes
    quadrants recede from one another."""
    rng = np.random.default_rng(seed)
    r4 = np.exp(rng.uniform(np.log(0.1), np.log(10.0), 4))
    p4 = np.exp(rng.uniform(np.log(0.1), np.log(10.0), 4))
    M = rng.uniform(0.0, mach_max, 4)
    cx = np.array([0.25, 0.75, 0.25, 0.75])
    cy = np.array([0.25, 0.25, 0.75, 0.75])
    if direction == "centre":
        th = np.arctan2(0.5 - cy, 0.5 - cx) + rng.uniform(-np.pi / 4, np.pi / 4, 4)
    elif direction == "any":
        th = rng.uniform(0.0, 2.0 * np.pi, 4)
    else:
        raise ValueError(direction)
    c = np.sqrt(gamma * p4 / r4)
    u4, v4 = M * c * np.cos(th), M * c * np.sin(th)
    x = cell_centres(n, 0.0, 1.0)
    X, Y = np.meshgrid(x, x)  # rows are y
    q = ((X > 0.5).astype(np.int64) + 2 * (Y > 0.5).astype(np.int64)).ravel()
    return Problem(2, n, n, 0.0, 1.0, 0.0, 1.0, gamma, r4[q], u4[q], v4[q], p4[q],
                   name="quadrants_%d_seed%d" % (n, seed))


def lax_liu_2d(n):
    """The 2D Riemann configuration of Sec. IV.C (symmetric under x <-> y)."""
    x = cell_centres(n, 0.0, 1.0)
    X, Y = np.meshgrid(x, x)
    rho = np.select([(X > 0.5) & (Y > 0.5), (X <= 0.5) & (Y > 0.5), (X <= 0.5) & (Y <= 0.5)],
                    [0.5313, 1.0, 0.8], 1.0).ravel()
    ux = np.where((X <= 0.5) & (Y > 0.5), 0.7276, 0.0).ravel()
    uy = np.where((X > 0.5) & (Y <= 0.5), 0.7276, 0.0).ravel()
    p = np.where((X > 0.5) & (Y > 0.5), 0.4, 1.0).ravel()
    return Problem(2, n, n, 0.0, 1.0, 0.0, 1.0, 1.4, rho, ux, uy, p, name="lax_liu_%d" % n)


def smooth_periodic(dim, nx, ny, seed, amp=0.1, gamma=1.4, modes=3):
    """Smooth random periodic fields (a few Fourier modes of relative amplitude amp)."""
    rng = np.random.default_rng(seed)
    x = cell_centres(nx, 0.0, 1.0)
    y = cell_centres(ny, 0.0, 1.0) if dim == 2 else np.array([0.5])
    X, Y = np.meshgrid(x, y)

    def field_(scale):
        f = np.zeros_like(X)
        for _ in range(modes):
            kx, ky = rng.integers(1, 3), (rng.integers(0, 3) if dim == 2 else 0)
            ph = rng.uniform(0, 2 * np.pi)
            f += rng.uniform(-1, 1) * np.sin(2 * np.pi * (kx * X + ky * Y) + ph)
        return scale * f / modes

    rho = np.exp(field_(amp)).ravel()
    p = np.exp(field_(amp)).ravel()
    ux = (rng.uniform(-1, 1) + field_(amp)).ravel()
    uy = ((rng.uniform(-1, 1) + field_(amp)) if dim == 2 else np.zeros_like(X)).ravel()
    return Problem(dim, nx, ny if dim == 2 else 1, 0.0, 1.0, 0.0, 1.0, gamma, rho, ux, uy, p,
                   bc=(PERIODIC,) * 4, name="smooth_periodic")


@dataclass
class TubeBatch:
    lengths: np.ndarray   # cells per tube
    gammas: np.ndarray
    left: np.ndarray      # (n, 3) rho, u, p
    right: np.ndarray

    @property
    def total_cells(self):
        return int(self.lengths.sum())


def tube_batch(n_tubes, seed, len_min=200, len_max=8000, ratio_max=1e5, mach_max=20.0):
    """Independent 1D shock tubes: lengths log-uniform in [len_min, len_max]; rho_L, p_L
    log-uniform in [0.1, 10]; density and pressure ratios log-uniform in [1, ratio_max];
    sides swapped with probability 1/2; a velocity jump of Mach up to mach_max (with
    respect to the left sound speed), split symmetrically or put on one side; gamma in
    {1.4, 5/3}.  Each tube spans [0, 1] with the split at its middle."""
    rng = np.random.default_rng(seed)
    lengths = np.rint(np.exp(rng.uniform(np.log(len_min), np.log(len_max), n_tubes))).astype(np.int64)
    gam = np.where(rng.integers(0, 2, n_tubes) == 0, 1.4, 5.0 / 3.0)
    rl = np.exp(rng.uniform(np.log(0.1), np.log(10.0), n_tubes))
    pl = np.exp(rng.uniform(np.log(0.1), np.log(10.0), n_tubes))
    rr = rl / np.exp(rng.uniform(0.0, np.log(ratio_max), n_tubes))
    pr = pl / np.exp(rng.uniform(0.0, np.log(ratio_max), n_tubes))
    du = rng.uniform(0.0, mach_max, n_tubes) * np.sqrt(gam * pl / rl)
    split = rng.integers(0, 3, n_tubes)  # 0 symmetric, 1 left moves, 2 right moves
    ul = np.where(split == 0, 0.5 * du, np.where(split == 1, du, 0.0))
    ur = np.where(split == 0, -0.5 * du, np.where(split == 2, -du, 0.0))
    swap = rng.integers(0, 2, n_tubes) == 1
    left = np.stack([np.where(swap, rr, rl), np.where(swap, -ur, ul), np.where(swap, pr, pl)], 1)
    right = np.stack([np.where(swap, rl, rr), np.where(swap, -ul, ur), np.where(swap, pl, pr)], 1)
    return TubeBatch(lengths, gam, left, right)


def tube_batch_fields(batch: TubeBatch):
    """Concatenated primitive fields of a tube batch (tube-major, x fastest)."""
    rho, ux, p = [], [], []
    for k in range(len(batch.lengths)):
        n = int(batch.lengths[k])
        x = cell_centres(n, 0.0, 1.0)
        L = x < 0.5
        rho.append(np.where(L, batch.left[k, 0], batch.right[k, 0]))
        ux.append(np.where(L, batch.left[k, 1], batch.right[k, 1]))
        p.append(np.where(L, batch.left[k, 2], batch.right[k, 2]))
    return np.concatenate(rho), np.concatenate(ux), np.concatenate(p)


def shocked_interface_2d(nx, ny, seed, gamma=1.4):
    """Planar shock (Mach in [1.5, 3]) moving +x through light gas (rho 1, p 1) towards a
    heavy-gas interface (Atwood number in [0.5, 0.9]) at x = 1 + 0.05 sin(2 pi m y),
    m in {2..8}; domain [0, 4] x [0, 1]; left inflow at the post-shock state, right
    transmissive, periodic in y.  The post-shock state is the Rankine-Hugoniot one."""
    rng = np.random.default_rng(seed)
    M = rng.uniform(1.5, 3.0)
    A = rng.uniform(0.5, 0.9)
    m = int(rng.integers(2, 9))
    rho1, p1 = 1.0, 1.0
    rho_h = (1.0 + A) / (1.0 - A)
    g = gamma
    c1 = np.sqrt(g * p1 / rho1)
    p2 = p1 * (2.0 * g * M * M - (g - 1.0)) / (g + 1.0)
    rho2 = rho1 * (g + 1.0) * M * M / ((g - 1.0) * M * M + 2.0)
    u2 = M * c1 * (1.0 - rho1 / rho2)
    x = cell_centres(nx, 0.0, 4.0)
    y = cell_centres(ny, 0.0, 1.0)
    X, Y = np.meshgrid(x, y)
    xi = 1.0 + 0.05 * np.sin(2.0 * np.pi * m * Y)
    post = X < 0.5
    heavy = X >= xi
    rho = np.where(post, rho2, np.where(heavy, rho_h, rho1)).ravel()
    ux = np.where(post, u2, 0.0).ravel()
    p = np.where(post, p2, p1).ravel()
    inflow = np.zeros((4, 4))
    inflow[0] = (rho2, u2, 0.0, p2)
    rngs = np.zeros((4, 2), dtype=np.int64)
    rngs[0] = (0, ny)
    return Problem(2, nx, ny, 0.0, 4.0, 0.0, 1.0, gamma, rho, ux, np.zeros_like(ux), p,
                   bc=(INFLOW, TRANSMISSIVE, PERIODIC, PERIODIC), inflow=inflow,
                   inflow_range=rngs, name="shocked_interface_%dx%d_seed%d" % (nx, ny, seed))


def jet_2d(n, seed, gamma=5.0 / 3.0, mach=80.0, density_ratio=10.0):
    """Jet of Mach 80 and density 10 x ambient entering [0,1] x [-0.5,0.5] (n x n cells)
    through a left inflow band |y| <= 0.05; ambient rho 1 at rest with p drawn uniform in
    [0.1, 1]; jet temperature = r x ambient temperature with r log-uniform in [0.01, 1];
    transmissive elsewhere."""
    rng = np.random.default_rng(seed)
    p_amb = rng.uniform(0.1, 1.0)
    r = np.exp(rng.uniform(np.log(0.01), 0.0))
    rho_amb = 1.0
    T_amb = p_amb / rho_amb
    rho_j = density_ratio * rho_amb
    T_j = r * T_amb
    p_j = rho_j * T_j
    u_j = mach * np.sqrt(gamma * T_j)
    N = n * n
    inflow = np.zeros((4, 4))
    inflow[0] = (rho_j, u_j, 0.0, p_j)
    y = cell_centres(n, -0.5, 0.5)
    band = np.nonzero(np.abs(y) <= 0.05)[0]
    rngs = np.zeros((4, 2), dtype=np.int64)
    rngs[0] = (band.min(), band.max() + 1)
    return Problem(2, n, n, 0.0, 1.0, -0.5, 0.5, gamma, np.full(N, rho_amb), np.zeros(N),
                   np.zeros(N), np.full(N, p_amb), bc=(INFLOW, TRANSMISSIVE, TRANSMISSIVE, TRANSMISSIVE),
                   inflow=inflow, inflow_range=rngs, name="jet_%d_seed%d" % (n, seed))


# ------------------------------------------------------------------ reflective walls

def two_blast_1d(n, gamma=1.4):
    """Two interacting blast waves (Sec. IV, Woodward-Colella): rho = 1, u = 0 and p = 1000 on
    [0, 0.1), 0.01 on [0.1, 0.9), 100 on [0.9, 1]; reflective walls at x = 0 and x = 1
    (the paper runs 1600 cells to t = 0.038)."""
    x = cell_centres(n, 0.0, 1.0)
    p = np.where(x < 0.1, 1000.0, np.where(x < 0.9, 0.01, 100.0))
    return Problem(1, n, 1, 0.0, 1.0, 0.0, 1.0, gamma, np.ones(n), np.zeros(n), np.zeros(n), p,
                   bc=(REFLECTIVE, REFLECTIVE, TRANSMISSIVE, TRANSMISSIVE), name="two_blast_%d" % n)


def explosion_box_2d(n, gamma=1.4):
    """Explosion in a box (Sec. IV): the unit square with reflective walls; (rho, u, v, p) =
    (5, 0, 0, 5) inside the circle of radius 0.3 about (0.4, 0.4), (1, 0, 0, 1) elsewhere,
    sampled at cell centres (the paper runs 256 x 256 to t = 0.5)."""
    x = cell_centres(n, 0.0, 1.0)
    X, Y = np.meshgrid(x, x)
    inside = ((X - 0.4) ** 2 + (Y - 0.4) ** 2 < 0.09).ravel()
    rho = np.where(inside, 5.0, 1.0)
    return Problem(2, n, n, 0.0, 1.0, 0.0, 1.0, gamma, rho, np.zeros(n * n), np.zeros(n * n), rho.copy(),
                   bc=(REFLECTIVE,) * 4, name="explosion_box_%d" % n)


def wall_reflection_1d(n, rho=1.0, u=-1.0, p=1.0, gamma=1.4):
    """Uniform gas moving into a reflective wall at x = 0 (transmissive at x = 1).  By
    symmetry it is the Riemann problem (rho, -u, p) | (rho, u, p) about x = 0, whose exact
    solution on x > 0 is a reflected shock leaving the wall with the gas at rest behind it."""
    return Problem(1, n, 1, 0.0, 1.0, 0.0, 1.0, gamma, np.full(n, rho), np.full(n, u), np.zeros(n), np.full(n, p),
                   bc=(REFLECTIVE, TRANSMISSIVE, TRANSMISSIVE, TRANSMISSIVE), name="wall_reflection_%d" % n)


def mirror_extend(pb: Problem) -> Problem:
    """The reflective problem pb unfolded into a periodic one: every reflective axis is
    doubled with the mirror image (the normal velocity reversed) placed across the wall.
    Its copy of pb's cells evolves exactly as pb does (both sides of each wall see the
    same ghost values)."""
    nx, ny = pb.nx, pb.ny
    rho, ux, uy, p = (a.reshape(ny, nx) for a in (pb.rho, pb.ux, pb.uy, pb.p))
    x0, x1, y0, y1 = pb.x0, pb.x1, pb.y0, pb.y1
    bc = list(pb.bc)
    if pb.bc[0] == REFLECTIVE:
        assert pb.bc[1] == REFLECTIVE
        rho, ux, uy, p = (np.concatenate([a[:, ::-1] * s, a], axis=1) for a, s in ((rho, 1), (ux, -1), (uy, 1), (p, 1)))
        x0 = x0 - (x1 - x0)
        bc[0] = bc[1] = PERIODIC
    if pb.dim == 2 and pb.bc[2] == REFLECTIVE:
        assert pb.bc[3] == REFLECTIVE
        rho, ux, uy, p = (np.concatenate([a[::-1, :] * s, a], axis=0) for a, s in ((rho, 1), (ux, 1), (uy, -1), (p, 1)))
        y0 = y0 - (y1 - y0)
        bc[2] = bc[3] = PERIODIC
    NY, NX = rho.shape
    return Problem(pb.dim, NX, NY if pb.dim == 2 else 1, x0, x1, y0, y1, pb.gamma, rho.ravel(), ux.ravel(),
                   uy.ravel(), p.ravel(), bc=tuple(bc), name=pb.name + "_unfolded")


def rankine_hugoniot(mach, rho1, p1, gamma):
    """(rho2, u2, p2) behind a shock of Mach number `mach` running into gas at rest
    (rho1, p1): the normal-shock relations of ideal-gas dynamics."""
    m2 = mach * mach
    rho2 = rho1 * (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    p2 = p1 * (1.0 + 2.0 * gamma / (gamma + 1.0) * (m2 - 1.0))
    vs = mach * np.sqrt(gamma * p1 / rho1)
    return rho2, vs * (1.0 - rho1 / rho2), p2


def rmi_2d(kind, nx=600, ny=100):
    """Richtmyer-Meshkov instability of Sec. IV on [0, 0.6] x [0, 0.1] (the paper runs
    600 x 100).  kind 1: a Mach-1.2 shock from the light gas into the heavy one (post-shock,
    light and heavy states split at x = 1/6 and x = 1/4); kind 2: a Mach-2.5 shock from the
    heavy gas into the light one (split at 1/12 and 1/6).  The interface carries a
    sinusoidal perturbation of amplitude 0.008; the paper gives no wavelength, and the
    reading is one cosine period over the height, x_I(y) = x_I + 0.008 cos(2 pi y / 0.1),
    symmetric about mid-height.  Inflow of the post-shock state on the left side,
    transmissive elsewhere; gamma = 1.4."""
    # the post-shock state is the Rankine-Hugoniot state of the shock running into
    # (1, 0, 0, 1); it reproduces the printed (rho, u) of both types and the printed p of
    # type 2, while type 1 prints p = 0.151332 for 1.51332 (see rankine_hugoniot)
    if kind == 1:
        post = rankine_hugoniot(1.2, 1.0, 1.0, 1.4)
        states = ((post[0], post[1], 0.0, post[2]), (1.0, 0.0, 0.0, 1.0), (5.04, 0.0, 0.0, 1.0))
        x_shock, x_int = 1.0 / 6.0, 0.25
    else:
        post = rankine_hugoniot(2.5, 1.0, 1.0, 1.4)
        states = ((post[0], post[1], 0.0, post[2]), (1.0, 0.0, 0.0, 1.0), (0.138, 0.0, 0.0, 1.0))
        x_shock, x_int = 1.0 / 12.0, 1.0 / 6.0
    x = cell_centres(nx, 0.0, 0.6)
    y = cell_centres(ny, 0.0, 0.1)
    X, Y = np.meshgrid(x, y)
    xi = x_int + 0.008 * np.cos(2.0 * np.pi * Y / 0.1)
    region = np.where(X < x_shock, 0, np.where(X < xi, 1, 2)).ravel()
    S = np.array(states)
    inflow = np.zeros((4, 4))
    inflow[0] = states[0]
    rng = np.zeros((4, 2), dtype=np.int64)
    rng[0] = (0, ny)
    return Problem(2, nx, ny, 0.0, 0.6, 0.0, 0.1, 1.4, S[region, 0], S[region, 1], S[region, 2], S[region, 3],
                   bc=(INFLOW, TRANSMISSIVE, TRANSMISSIVE, TRANSMISSIVE), inflow=inflow, inflow_range=rng,
                   name="rmi%d_%dx%d" % (kind, nx, ny))



# ------------------------------------------------------------------ 3D (D3Q64) problems

@dataclass
class Problem3:
    """A D3Q64 problem on a box of nx x ny x nz cells; fields are flat, x fastest, then y."""
    nx: int
    ny: int
    nz: int
    x0: float
    x1: float
    y0: float
    y1: float
    z0: float
    z1: float
    gamma: float
    rho: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    uz: np.ndarray
    p: np.ndarray
    bc: tuple = (TRANSMISSIVE,) * 6   # x-lo, x-hi, y-lo, y-hi, z-lo, z-hi
    name: str = ""
    dim: int = 3

    @property
    def dx(self):
        return (self.x1 - self.x0) / self.nx

    @property
    def dy(self):
        return (self.y1 - self.y0) / self.ny

    @property
    def dz(self):
        return (self.z1 - self.z0) / self.nz

    @property
    def ncell(self):
        return self.nx * self.ny * self.nz


def _grid3(nx, ny, nz, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    x = cell_centres(nx, lo[0], hi[0])
    y = cell_centres(ny, lo[1], hi[1])
    z = cell_centres(nz, lo[2], hi[2])
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")   # [z][y][x]: x fastest when flattened
    return X, Y, Z


def smooth_periodic_3d(nx, ny, nz, seed, amp=0.1, gamma=1.4, modes=3):
    """Smooth random periodic fields on the unit cube (a few Fourier modes of relative
    amplitude amp; a random mean velocity)."""
    rng = np.random.default_rng(seed)
    X, Y, Z = _grid3(nx, ny, nz)

    def field_(scale):
        f = np.zeros_like(X)
        for _ in range(modes):
            k = rng.integers(0, 3, 3)
            k[0] = max(k[0], 1)
            ph = rng.uniform(0, 2 * np.pi)
            f += rng.uniform(-1, 1) * np.sin(2 * np.pi * (k[0] * X + k[1] * Y + k[2] * Z) + ph)
        return scale * f / modes

    rho = np.exp(field_(amp)).ravel()
    p = np.exp(field_(amp)).ravel()
    u = [(rng.uniform(-1, 1) + field_(amp)).ravel() for _ in range(3)]
    return Problem3(nx, ny, nz, 0, 1, 0, 1, 0, 1, gamma, rho, u[0], u[1], u[2], p, bc=(PERIODIC,) * 6,
                    name="smooth_periodic_3d_%dx%dx%d" % (nx, ny, nz))


def shock_tube_3d(left, right, gamma, n, axis, nt=1, x_split=0.5):
    """A two-state Riemann problem along one axis of the unit box (n cells along it, nt
    along the others, periodic across it, transmissive along it); left = (rho, u_n, p)."""
    shape = [nt, nt, nt]
    shape[axis] = n
    X, Y, Z = _grid3(*shape)
    s = (X, Y, Z)[axis].ravel()
    L = s < x_split
    rho = np.where(L, left[0], right[0]).astype(np.float64)
    un = np.where(L, left[1], right[1]).astype(np.float64)
    p = np.where(L, left[2], right[2]).astype(np.float64)
    u = [np.zeros_like(rho) for _ in range(3)]
    u[axis] = un
    bc = [PERIODIC] * 6
    bc[2 * axis] = bc[2 * axis + 1] = TRANSMISSIVE
    return Problem3(shape[0], shape[1], shape[2], 0, 1, 0, 1, 0, 1, float(gamma), rho, u[0], u[1], u[2], p,
                    bc=tuple(bc), name="tube3d_axis%d_%d" % (axis, n))


def spherical_blast_3d(n, r0=0.4, inner=(1.0, 1.0), outer=(0.125, 0.1), gamma=1.4):
    """The spherical explosion in a box: gas at rest, (rho, p) = inner inside a sphere of
    radius r0 about the centre of [-1, 1]^3 and outer outside; transmissive sides."""
    X, Y, Z = _grid3(n, n, n, (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0))
    inside = (X * X + Y * Y + Z * Z < r0 * r0).ravel()
    rho = np.where(inside, inner[0], outer[0]).astype(np.float64)
    p = np.where(inside, inner[1], outer[1]).astype(np.float64)
    z = np.zeros_like(rho)
    return Problem3(n, n, n, -1, 1, -1, 1, -1, 1, gamma, rho, z, z.copy(), z.copy(), p,
                    name="spherical_blast_%d" % n)


def octants_3d(n, seed, gamma=1.4, mach_max=2.0):
    """Eight-octant Riemann problem on the unit cube: each octant draws rho and p
    log-uniform in [0.1, 10] and a velocity of Mach number uniform in [0, mach_max] pointing
    towards the centre within a cone of half-angle 45 degrees; transmissive sides."""
    rng = np.random.default_rng(seed)
    r8 = np.exp(rng.uniform(np.log(0.1), np.log(10.0), 8))
    p8 = np.exp(rng.uniform(np.log(0.1), np.log(10.0), 8))
    M = rng.uniform(0.0, mach_max, 8)
    u8 = np.zeros((8, 3))
    for q in range(8):
        centre = np.array([0.25 + 0.5 * (q & 1), 0.25 + 0.5 * ((q >> 1) & 1), 0.25 + 0.5 * ((q >> 2) & 1)])
        d = 0.5 - centre
        d = d / np.linalg.norm(d)
        w = rng.normal(size=3)
        w -= (w @ d) * d
        w /= np.linalg.norm(w)
        th = rng.uniform(0.0, np.pi / 4)
        u8[q] = M[q] * np.sqrt(gamma * p8[q] / r8[q]) * (np.cos(th) * d + np.sin(th) * w)
    X, Y, Z = _grid3(n, n, n)
    q = ((X > 0.5).astype(np.int64) + 2 * (Y > 0.5).astype(np.int64) + 4 * (Z > 0.5).astype(np.int64)).ravel()
    return Problem3(n, n, n, 0, 1, 0, 1, 0, 1, gamma, r8[q], u8[q, 0], u8[q, 1], u8[q, 2], p8[q],
                    name="octants_%d_seed%d" % (n, seed))


def permute_3d(pb, perm):
    """The same problem with the axes relabelled: new axis a is old axis perm[a]."""
    shape = (pb.nz, pb.ny, pb.nx)                     # array axes [z][y][x]
    arr = lambda a: np.asarray(a).reshape(shape)
    # array axis of old spatial axis k is 2 - k; new array axis 2 - a holds old 2 - perm[a]
    order = [2 - perm[2 - ax] for ax in range(3)]
    rho, p = (np.transpose(arr(a), order).ravel() for a in (pb.rho, pb.p))
    uo = [pb.ux, pb.uy, pb.uz]
    u = [np.transpose(arr(uo[perm[a]]), order).ravel() for a in range(3)]
    n = (pb.nx, pb.ny, pb.nz)
    lo, hi = (pb.x0, pb.y0, pb.z0), (pb.x1, pb.y1, pb.z1)
    bc = []
    for a in range(3):
        bc += [pb.bc[2 * perm[a]], pb.bc[2 * perm[a] + 1]]
    return Problem3(n[perm[0]], n[perm[1]], n[perm[2]], lo[perm[0]], hi[perm[0]], lo[perm[1]], hi[perm[1]],
                    lo[perm[2]], hi[perm[2]], pb.gamma, rho, u[0], u[1], u[2], p, bc=tuple(bc),
                    name=pb.name + "_perm%d%d%d" % tuple(perm))


def mirror_extend_3d(pb):
    """A box with reflective walls on both sides of an axis unfolded into the periodic box
    of twice the length along that axis (the mirror image, normal velocity reversed)."""
    shape = (pb.nz, pb.ny, pb.nx)
    f = {k: np.asarray(getattr(pb, k)).reshape(shape) for k in ("rho", "ux", "uy", "uz", "p")}
    n = [pb.nx, pb.ny, pb.nz]
    lo, hi = [pb.x0, pb.y0, pb.z0], [pb.x1, pb.y1, pb.z1]
    bc = list(pb.bc)
    for axis in range(3):
        if pb.bc[2 * axis] != REFLECTIVE:
            continue
        assert pb.bc[2 * axis + 1] == REFLECTIVE
        ax = 2 - axis
        for k in f:
            s = -1.0 if k == "u" + "xyz"[axis] else 1.0
            f[k] = np.concatenate([np.flip(f[k], ax) * s, f[k]], axis=ax)
        lo[axis] -= hi[axis] - lo[axis]
        n[axis] *= 2
        bc[2 * axis] = bc[2 * axis + 1] = PERIODIC
    return Problem3(n[0], n[1], n[2], lo[0], hi[0], lo[1], hi[1], lo[2], hi[2], pb.gamma,
                    *(f[k].ravel() for k in ("rho", "ux", "uy", "uz", "p")), bc=tuple(bc), name=pb.name + "_unfolded")
