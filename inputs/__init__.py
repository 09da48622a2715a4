"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests
and the benchmark.

This module only builds problem descriptions (grid, bed, node-type mask,
edge kinds, Dirichlet data, initial state).  It holds none of the
MacLABSWE arithmetic: both the oracle and the CUDA library receive the same
``Case`` and compute the update on their own.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) evaluated on a counter, so a
case is a pure function of its seed.

Workloads (stand-ins for the paper's Section 4 tests; all synthetic):
  * ``tidal_strip``   -- Section 4.1, the 1D tidal flow over the irregular bed
                         of Table tidal-irre.zb, run as a 2D strip.
  * ``paper_lake``    -- Section 4.2, Eq. wind_bed dish, 5 m/s SW->NE wind.
  * ``dish_lake``     -- a seeded paraboloid dish (Section 4.2 family).
  * ``paper_hump``    -- Section 4.3, Eqs. 2D sand bed / 2D sand bedAdd.
  * ``bump_channel``  -- a seeded Gaussian bump channel (Section 4.3 family).
  * ``random_case``   -- small random grids exercising every node type and
                         edge kind, for parity tests.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# node types of the uint8 mask and the edge kinds (same coding as the C ABI)
SOLID, FLUID, NOSLIP, DIR_H, DIR_Q, DIR_HU = 0, 1, 2, 3, 4, 5
BOUNCEBACK, SPECULAR, PERIODIC = 0, 1, 2
W, E, S, N = 0, 1, 2, 3

G = 9.81          # Section 2
RHO_A = 1.293     # Eq. wind_u-stress
CW = 0.0026       # Eq. wind_u-stress
RHO_W = 1000.0    # not given in the paper; fresh water

# Table tidal-irre.zb: bed elevation of the 1D tidal test (x in m, z_b in m)
TIDAL_BED_X = (0, 50, 100, 150, 250, 300, 350, 400, 425, 435, 450, 475, 500, 505,
               530, 550, 565, 575, 600, 650, 700, 750, 800, 820, 900, 950, 1000, 1500)
TIDAL_BED_Z = (0, 0, 2.5, 5, 5, 3, 5, 5, 7.5, 8, 9, 9, 9.1, 9,
               9, 6, 5.5, 5.5, 5, 4, 3, 3, 2.3, 2, 1.2, 0.4, 0, 0)
TIDAL_LENGTH = 1500.0
TIDAL_PERIOD = 43200.0   # 2*pi / omega with omega = 4*pi/86400 (Eq. veri-Ini-Bc.3r)


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """SplitMix64 output for each uint64 counter value."""
    z = counter.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


class Rng:
    """Counter-based uniform doubles: stream ``k`` of ``seed`` is
    splitmix64(seed * 2^32 + k * 2^20 + i) for i = 0, 1, ..."""

    def __init__(self, seed: int):
        self.seed = int(seed)
        self.stream = 0

    def uniform(self, n: int = 1, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        base = (self.seed << 32) + (self.stream << 20)
        self.stream += max(1, (n + (1 << 20) - 1) >> 20)
        with np.errstate(over="ignore"):
            bits = splitmix64(np.arange(n, dtype=np.uint64) + np.uint64(base))
        u = (bits >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
        return lo + (hi - lo) * u

    def scalar(self, lo: float, hi: float) -> float:
        return float(self.uniform(1, lo, hi)[0])


@dataclasses.dataclass
class Case:
    """One shallow-water problem: everything the update needs, in SI units.

    Arrays are row-major [ny][nx] (x fastest).  ``bc[edge, var]`` holds the
    Dirichlet data (mean, amp, omega, phase) of var 0 = h, 1 = q_x = h u,
    2 = q_y = h v, giving value(t) = mean + amp * sin(omega * t + phase).
    ``h_ref`` is the still-water level about which the FP32 path stores h.
    """
    name: str
    nx: int
    ny: int
    dx: float
    nu: float
    zb: np.ndarray
    mask: np.ndarray
    h0: np.ndarray
    u0: np.ndarray
    v0: np.ndarray
    edges: tuple = (BOUNCEBACK, BOUNCEBACK, BOUNCEBACK, BOUNCEBACK)
    bc: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((4, 3, 4)))
    g: float = G
    rho_w: float = RHO_W
    rho_a: float = RHO_A
    cw: float = CW
    wind_u: float = 0.0
    wind_v: float = 0.0
    cb: float = 0.0
    omega: float = 0.0
    h_ref: float = 0.0

    @property
    def e(self) -> float:
        """Particle speed of Eq. mlb-viscosity."""
        return 6.0 * self.nu / self.dx

    @property
    def dt(self) -> float:
        return self.dx / self.e

    @property
    def nodes(self) -> int:
        return self.nx * self.ny

    def copy(self) -> "Case":
        c = dataclasses.replace(self)
        for f in ("zb", "mask", "h0", "u0", "v0", "bc"):
            setattr(c, f, getattr(self, f).copy())
        return c


def _ring(fluid: np.ndarray) -> np.ndarray:
    """Fluid nodes with a non-fluid node among their 8 neighbours."""
    ny, nx = fluid.shape
    pad = np.pad(fluid, 1, constant_values=False)
    allnb = np.ones_like(fluid)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            allnb &= pad[1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
    return fluid & ~allnb


def tidal_strip(nx: int = 400, ny: int = 3) -> Case:
    """Section 4.1: 1500 m channel, bed from Table tidal-irre.zb (linear
    interpolation between the listed points), h(x,0) = 16 - z_b, u = 0,
    h(0,t) = 20 - 4 sin(pi (4t/86400 + 1/2)) at the west column, u = 0 at
    x = 1500 (no-slip east column), nu = 31.25 m^2/s, free-slip side walls."""
    dx = TIDAL_LENGTH / (nx - 1)
    x = np.arange(nx) * dx
    zb1 = np.interp(x, TIDAL_BED_X, TIDAL_BED_Z)
    zb = np.tile(zb1, (ny, 1))
    mask = np.full((ny, nx), FLUID, np.uint8)
    mask[:, 0] = DIR_H
    mask[:, -1] = NOSLIP
    bc = np.zeros((4, 3, 4))
    bc[W, 0] = (20.0, -4.0, 4.0 * math.pi / 86400.0, math.pi / 2)
    h0 = 16.0 - zb
    z = np.zeros((ny, nx))
    return Case("tidal_strip_%dx%d" % (nx, ny), nx, ny, dx, 31.25, zb, mask, h0, z, z.copy(),
                edges=(BOUNCEBACK, BOUNCEBACK, SPECULAR, SPECULAR), bc=bc, h_ref=16.0)


def paper_lake(n: int = 201) -> Case:
    """Section 4.2 with the paper's own parameters: Eq. wind_bed dish on
    [-200,200]^2, dx = 2, nu = 5.33, 5 m/s wind from south-west, still
    water at rest.  Fluid where the square-root argument of Eq. wind_bed is
    non-negative; the outermost fluid ring is a no-slip wall."""
    dx = 2.0
    c = (np.arange(n) - (n - 1) / 2) * dx
    X, Y = np.meshgrid(c, c)
    r = np.sqrt(X * X + Y * Y)
    arg = 0.5 - r / 386.4
    fluid = arg >= 0.0
    H = np.where(fluid, (1.0 / 1.3) * (0.5 + np.sqrt(np.maximum(arg, 0.0))), 0.0)
    H00 = (1.0 / 1.3) * (0.5 + math.sqrt(0.5))
    zb = H00 - H
    mask = np.where(fluid, FLUID, SOLID).astype(np.uint8)
    mask[_ring(fluid)] = NOSLIP
    h0 = np.where(fluid, H, 0.0)
    z = np.zeros((n, n))
    w = 5.0 / math.sqrt(2.0)
    return Case("paper_lake_%d" % n, n, n, dx, 5.33, zb, mask, h0, z, z.copy(),
                wind_u=w, wind_v=w, h_ref=H00)


def dish_lake(n: int = 256, seed: int = 0) -> Case:
    """Seeded paraboloid dish: still-water depth D = h0 (1 - r^2/R^2) with
    R ~ U[150,250] m and h0 ~ U[0.8,1.5] m on [-R,R]^2, fluid where
    D >= 0.415 h0 (the edge/centre depth ratio of Eq. wind_bed), no-slip ring,
    nu = 8 dx / 3 (e = 16 m/s as in the paper's lake), 5 m/s wind at a seeded
    angle, Chezy C_z ~ U[40,80]."""
    rng = Rng(seed)
    R = rng.scalar(150.0, 250.0)
    hc = rng.scalar(0.8, 1.5)
    theta = rng.scalar(0.0, 2 * math.pi)
    cz = rng.scalar(40.0, 80.0)
    dx = 2 * R / (n - 1)
    c = np.linspace(-R, R, n)
    X, Y = np.meshgrid(c, c)
    D = hc * (1.0 - (X * X + Y * Y) / (R * R))
    fluid = D >= 0.415 * hc
    mask = np.where(fluid, FLUID, SOLID).astype(np.uint8)
    mask[_ring(fluid)] = NOSLIP
    zb = hc - D
    h0 = np.where(fluid, D, 0.0)
    z = np.zeros((n, n))
    return Case("dish_lake_%d_s%d" % (n, seed), n, n, dx, 8.0 * dx / 3.0, zb, mask, h0, z,
                z.copy(), wind_u=5.0 * math.cos(theta), wind_v=5.0 * math.sin(theta),
                cb=G / (cz * cz), h_ref=hc)


def _channel(name, nx, ny, dx, nu, zb, depth, q, cb):
    mask = np.full((ny, nx), FLUID, np.uint8)
    mask[:, 0] = DIR_Q
    mask[:, -1] = DIR_H
    bc = np.zeros((4, 3, 4))
    bc[W, 1] = (q, 0.0, 0.0, 0.0)
    bc[E, 0] = (depth, 0.0, 0.0, 0.0)
    h0 = depth - zb
    u0 = q / h0
    return Case(name, nx, ny, dx, nu, zb, mask, h0, u0, np.zeros((ny, nx)),
                edges=(BOUNCEBACK, BOUNCEBACK, SPECULAR, SPECULAR), bc=bc, cb=cb, h_ref=depth)


def paper_hump(n: int = 201) -> Case:
    """Section 4.3: 1000 m x 1000 m channel, dx = 5, hump of Eqs. 2D sand
    bed / 2D sand bedAdd on [300,500] x [400,600], q = 10 m^2/s inflow,
    h = 10 m outflow.  nu is not given in the paper: 10 m^2/s."""
    dx = 1000.0 / (n - 1)
    c = np.arange(n) * dx
    X, Y = np.meshgrid(c, c)
    inside = (X >= 300) & (X <= 500) & (Y >= 400) & (Y <= 600)
    psi = np.sin(math.pi * (X - 300) / 200) ** 2 * np.sin(math.pi * (Y - 400) / 200) ** 2
    zb = np.where(inside, psi, 0.0)
    return _channel("paper_hump_%d" % n, n, n, dx, 10.0, zb, 10.0, 10.0, 0.0)


def bump_channel(nx: int = 8192, ny: int = 2048, seed: int = 0) -> Case:
    """Seeded channel over a Gaussian bump: dx = 5 m, nu = 10 m^2/s, still
    depth 10 m, bump height A ~ U[0.1,0.4] x 10 m, width sigma ~
    U[0.02,0.05] x ny dx, centred at (nx/4, ny/2); inflow q = 10 m^2/s,
    outflow h = 10 m, free-slip side walls, Chezy C_z ~ U[30,60]."""
    rng = Rng(seed)
    A = rng.scalar(0.1, 0.4) * 10.0
    sigma = rng.scalar(0.02, 0.05) * ny * 5.0
    cz = rng.scalar(30.0, 60.0)
    dx = 5.0
    xs = np.arange(nx) * dx
    ys = np.arange(ny) * dx
    x0, y0 = nx / 4 * dx, ny / 2 * dx
    gx = np.exp(-((xs - x0) ** 2) / (2 * sigma * sigma))
    gy = np.exp(-((ys - y0) ** 2) / (2 * sigma * sigma))
    zb = A * np.outer(gy, gx)
    return _channel("bump_channel_%dx%d_s%d" % (nx, ny, seed), nx, ny, dx, 10.0, zb, 10.0,
                    10.0, G / (cz * cz))


def random_case(nx: int, ny: int, seed: int, edges=(BOUNCEBACK, BOUNCEBACK, SPECULAR, SPECULAR),
                solids: bool = True, dirichlet: bool = True, forcing: bool = True,
                amp: float = 0.15, dirichlet_sn: bool = False) -> Case:
    """Small random problem for parity tests: smooth random bed, random
    solid blocks (with no-slip borders), Dirichlet columns on non-periodic
    W/E edges (DIR_H west, DIR_Q east, DIR_HU on the first and last rows of
    the west column when ny > 6), random smooth initial state, random wind,
    friction and Coriolis.  With dirichlet_sn, Dirichlet rows on
    non-periodic S/N edges too (DIR_Q south, DIR_H north, columns 2 ..
    nx - 3, so that no corner's inward node is a Dirichlet node).  Speeds
    stay well inside the stability condition of Section 3
    (R_le = U dx / nu < 1)."""
    rng = Rng(seed)
    dx = 1.0
    nu = rng.scalar(3.0, 4.5)            # e = 6 nu / dx in [18, 27] m/s
    href = 1.0
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)

    def smooth_field(scale):
        f = np.zeros((ny, nx))
        for _ in range(3):
            kx, ky, ph = rng.uniform(3, 0.0, 1.0)
            kx = 2 * math.pi * (1 + int(kx * 3)) / max(nx, 1)
            ky = 2 * math.pi * (1 + int(ky * 3)) / max(ny, 1)
            f += math.sin(2 * math.pi * ph) * np.cos(kx * xx + ky * yy + 2 * math.pi * ph)
        return scale * f / 3.0 + 0.02 * scale * (rng.uniform(nx * ny, -1, 1).reshape(ny, nx))

    zb = 0.2 + smooth_field(0.15)
    mask = np.full((ny, nx), FLUID, np.uint8)
    if solids and nx >= 12 and ny >= 12:
        nblk = 1 + int(rng.scalar(0, 3))
        for _ in range(nblk):
            w, hgt = 1 + int(rng.scalar(0, min(6, nx // 4))), 1 + int(rng.scalar(0, min(6, ny // 4)))
            i0 = int(rng.scalar(4, nx - 4 - w))
            j0 = int(rng.scalar(3, ny - 3 - hgt))
            mask[j0:j0 + hgt, i0:i0 + w] = SOLID
        fluid = mask != SOLID
        # a no-slip border around each block
        pad = np.pad(~fluid, 1, constant_values=False)
        near = np.zeros_like(fluid)
        for dy in (-1, 0, 1):
            for ddx in (-1, 0, 1):
                near |= pad[1 + dy:1 + dy + ny, 1 + ddx:1 + ddx + nx]
        mask[fluid & near] = NOSLIP
    bc = np.zeros((4, 3, 4))
    if dirichlet and edges[W] != PERIODIC and nx >= 8:
        mask[:, 0] = DIR_H
        mask[:, -1] = DIR_Q
        if ny > 6:
            mask[0, 0] = DIR_HU
            mask[-1, 0] = DIR_HU
        bc[W, 0] = (href + 0.01, 0.01, 2 * math.pi / 40.0, 0.3)
        bc[W, 1] = (0.08, 0.02, 2 * math.pi / 30.0, 0.0)
        bc[W, 2] = (0.0, 0.01, 2 * math.pi / 50.0, 1.0)
        bc[E, 1] = (0.08, 0.0, 0.0, 0.0)
        bc[E, 2] = (0.005, 0.0, 0.0, 0.0)
    if dirichlet_sn and edges[S] != PERIODIC and ny >= 8 and nx >= 8:
        mask[0, 2:nx - 2] = DIR_Q
        mask[-1, 2:nx - 2] = DIR_H
        bc[S, 1] = (0.1, 0.01, 2 * math.pi / 45.0, 0.2)
        bc[S, 2] = (0.0, 0.005, 2 * math.pi / 35.0, 0.0)
        bc[N, 0] = (href + 0.005, 0.005, 2 * math.pi / 60.0, 0.7)
    h0 = (href - zb) + smooth_field(0.05)
    u0 = 0.1 + smooth_field(amp)
    v0 = smooth_field(amp)
    solid = mask == SOLID
    h0[solid] = 0.0
    u0[solid] = 0.0
    v0[solid] = 0.0
    u0[mask == NOSLIP] = 0.0
    v0[mask == NOSLIP] = 0.0
    wind = rng.uniform(2, -8.0, 8.0) if forcing else (0.0, 0.0)
    cb = rng.scalar(0.002, 0.01) if forcing else 0.0
    om = rng.scalar(-1e-3, 1e-3) if forcing else 0.0
    return Case("random_%dx%d_s%d" % (nx, ny, seed), nx, ny, dx, nu, zb, mask, h0, u0, v0,
                edges=tuple(edges), bc=bc, wind_u=float(wind[0]), wind_v=float(wind[1]),
                cb=cb, omega=om, h_ref=href)


def ensemble(count: int = 512, seed: int = 0):
    """A batch of uneven problems: sizes nx, ny ~ U{64..512} drawn per
    instance; even instances are seeded dish lakes (n = nx, square), odd
    ones seeded bump channels (nx x ny), each with its own wind, bump height
    and Chezy coefficient from the instance seed."""
    rng = Rng(10_000 + seed)
    sizes = rng.uniform(2 * count, 64, 513).astype(int)
    out = []
    for i in range(count):
        nx, ny = int(sizes[2 * i]), int(sizes[2 * i + 1])
        sub = 1_000 * (seed + 1) + i
        out.append(dish_lake(nx, seed=sub) if i % 2 == 0 else bump_channel(nx, ny, seed=sub))
    return out
