"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
checks.  Pure numpy; holds none of the method's arithmetic (no equilibria,
no interpolation, no refinement criterion): only initial fields, fixed flag
patterns and boundary profiles, in the shapes of the paper's test problems.

Units: dx = 1, T_L = 1, so the athermal sound speed is 1 and a Mach number is
a speed.  Fields are (ny, nx) arrays, x fastest, cell centres at integers.
"""
from __future__ import annotations

import math

import numpy as np


def convected_vortex(L: int = 64, U0: float = 0.1, eps: float = 0.05, R: float | None = None,
                     disc_r: float | None = None, rho0: float = 1.0):
    """Athermal convected vortex of Sec. IV.A (its initial fields), at the
    64 x 64 size: uniform advection U0 along x plus the Gaussian vortex
    u' = eps (-(y - yc), x - xc) / R exp(-r^2 / 2R^2), R = L/10, and the
    isothermal radial-equilibrium density rho0 exp(-Ma_v^2/2 exp(-r^2/R^2))
    with Ma_v = eps.  Flags: a fixed disc of radius L/4 on the high-order
    lattice.  Returns rho, ux, uy, flags."""
    R = L / 10.0 if R is None else R
    disc_r = L / 4.0 if disc_r is None else disc_r
    xc = yc = L / 2.0
    x = np.arange(L, dtype=np.float64)
    X, Y = np.meshgrid(x, x)
    r2 = (X - xc) ** 2 + (Y - yc) ** 2
    g = np.exp(-r2 / (2.0 * R * R))
    ux = U0 - eps * (Y - yc) / R * g
    uy = eps * (X - xc) / R * g
    rho = rho0 * np.exp(-0.5 * eps * eps * np.exp(-r2 / (R * R)))
    flags = (r2 < disc_r * disc_r).astype(np.uint8)
    return rho, ux, uy, flags


def uniform(nx: int, ny: int, rho: float = 1.0, ux: float = 0.0, uy: float = 0.0):
    return (np.full((ny, nx), rho), np.full((ny, nx), ux), np.full((ny, nx), uy))


def perturbed(nx: int, ny: int, seed: int, amp_rho: float = 0.02, amp_u: float = 0.05,
              U: tuple[float, float] = (0.05, -0.03)):
    """Smooth random field: a few random Fourier modes on top of a uniform
    flow (seeded), for parity tests on generic states."""
    rng = np.random.default_rng(seed)
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    X, Y = np.meshgrid(x, y)
    rho = np.ones((ny, nx))
    ux = np.full((ny, nx), U[0])
    uy = np.full((ny, nx), U[1])
    for _ in range(4):
        kx, ky = rng.integers(1, 3, size=2)
        ph = rng.uniform(0, 2 * math.pi, size=3)
        a = rng.uniform(0.5, 1.0, size=3)
        arg = 2 * math.pi * (kx * X / nx + ky * Y / ny)
        rho += amp_rho * a[0] * np.sin(arg + ph[0]) / 4
        ux += amp_u * a[1] * np.sin(arg + ph[1]) / 4
        uy += amp_u * a[2] * np.cos(arg + ph[2]) / 4
    return rho, ux, uy


def perturbed_T(nx: int, ny: int, seed: int, amp: float = 0.05, T0: float = 1.0):
    """Smooth random temperature field (a few seeded Fourier modes around T0),
    for the thermal co-moving frame."""
    rng = np.random.default_rng(seed)
    X, Y = np.meshgrid(np.arange(nx, dtype=np.float64), np.arange(ny, dtype=np.float64))
    T = np.full((ny, nx), T0)
    for _ in range(3):
        kx, ky = rng.integers(1, 3, size=2)
        ph, a = rng.uniform(0, 2 * math.pi), rng.uniform(0.5, 1.0)
        T += amp * a * np.sin(2 * math.pi * (kx * X / nx + ky * Y / ny) + ph) / 3
    return T


def random_flags(nx: int, ny: int, seed: int, blobs: int = 3, rmin: float = 3.0, rmax: float = 8.0):
    """A few random discs (periodic distance) of high-order cells."""
    rng = np.random.default_rng(seed)
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    X, Y = np.meshgrid(x, y)
    fl = np.zeros((ny, nx), dtype=np.uint8)
    for _ in range(blobs):
        cx, cy = rng.uniform(0, nx), rng.uniform(0, ny)
        r = rng.uniform(rmin, rmax)
        dx = np.abs(X - cx); dx = np.minimum(dx, nx - dx)
        dy = np.abs(Y - cy); dy = np.minimum(dy, ny - dy)
        fl |= ((dx * dx + dy * dy) < r * r).astype(np.uint8)
    return fl


def strip_flags(N: int, frac: float = 0.1):
    """The paper's efficiency study (Sec. IV.C): an N x N domain split into two
    rectangular zones, a left strip of `frac` of the columns high-order."""
    fl = np.zeros((N, N), dtype=np.uint8)
    fl[:, : int(round(frac * N))] = 1
    return fl


def free_jet(nx: int = 1024, ny: int = 512, slot: int = 32, ma_jet: float = 0.5,
             ma_co: float = 0.05, pert: float = 0.01, seed: int = 1, edge: float = 1.5,
             developed: bool = True, spread: float = 0.1, core: float = 6.0):
    """2-D free jet of Sec. IV.A at the 1024 x 512 size: an inlet slot `slot`
    cells wide at Mach ma_jet in a co-flow of Mach ma_co, with a seeded `pert`
    relative random perturbation of the inlet velocity (both components).

    Returns a dict with the initial fields rho, ux, uy (ny, nx) and the inlet
    profile in_ux, in_uy (ny,).  The slot edges are smoothed by a tanh of
    width `edge` cells.  With developed=True the interior starts from a
    planar-jet similarity profile (half-width growing by `spread` per cell
    after a potential core of `core` slot widths, centreline excess velocity
    decaying like sqrt(x_core / x)), so a timed window sees a jet already
    spread through the domain; otherwise the interior starts at co-flow."""
    rng = np.random.default_rng(seed)
    y = np.arange(ny, dtype=np.float64)
    yc = (ny - 1) / 2.0
    half = slot / 2.0
    prof = 0.5 * (np.tanh((y - yc + half) / edge) - np.tanh((y - yc - half) / edge))
    in_ux = ma_co + (ma_jet - ma_co) * prof
    in_ux = in_ux * (1.0 + pert * rng.uniform(-1.0, 1.0, size=ny))
    in_uy = pert * (ma_jet - ma_co) * prof * rng.uniform(-1.0, 1.0, size=ny)
    x = np.arange(nx, dtype=np.float64)
    X, Y = np.meshgrid(x, y)
    if developed:
        xcore = core * slot
        b = half + spread * np.maximum(X - xcore, 0.0)
        decay = np.sqrt(xcore / np.maximum(X, xcore))
        # top-hat of half-width b smoothed over `edge` cells, scaled by the decay
        shape = 0.5 * (np.tanh((Y - yc + b) / edge) - np.tanh((Y - yc - b) / edge))
        excess = (ma_jet - ma_co) * decay * shape
        ux = ma_co + excess
    else:
        ux = np.full((ny, nx), ma_co)
    uy = np.zeros((ny, nx))
    rho = np.ones((ny, nx))
    return dict(rho=rho, ux=ux, uy=uy, in_ux=in_ux, in_uy=in_uy,
                fs_rho=1.0, fs_ux=ma_co, fs_uy=0.0)


def random_vortex_field(N: int = 4096, count: int = 512, seed: int = 4, rmin: float = 8.0,
                        rmax: float = 64.0, umax: float = 0.9):
    """Large periodic random-vortex field: `count` Gaussian vortices with
    random centres, radii in [rmin, rmax] and random signs, summed with
    periodic images and rescaled so max |u| = umax; rho = 1."""
    rng = np.random.default_rng(seed)
    ux = np.zeros((N, N))
    uy = np.zeros((N, N))
    xs = np.arange(N, dtype=np.float64)
    for _ in range(count):
        cx, cy = rng.uniform(0, N, size=2)
        R = rng.uniform(rmin, rmax)
        s = rng.choice([-1.0, 1.0]) * rng.uniform(0.5, 1.0)
        w = int(min(N // 2, math.ceil(4 * R)))
        ix = (np.arange(int(cx) - w, int(cx) + w + 1)) % N
        iy = (np.arange(int(cy) - w, int(cy) + w + 1)) % N
        dx = (xs[ix] - cx + N / 2) % N - N / 2
        dy = (xs[iy] - cy + N / 2) % N - N / 2
        DX, DY = np.meshgrid(dx, dy)
        g = s * np.exp(-(DX * DX + DY * DY) / (2 * R * R)) / R
        ux[np.ix_(iy, ix)] += -DY * g
        uy[np.ix_(iy, ix)] += DX * g
    m = np.sqrt(ux * ux + uy * uy).max()
    ux *= umax / m
    uy *= umax / m
    return np.ones((N, N)), ux, uy


def taylor_green(N: int, U0: float = 0.02, rho0: float = 1.0):
    """Taylor-Green vortex (App. A) on an N x N periodic grid, k = 2 pi / N:
    u_x = U0 sin(kx) cos(ky), u_y = -U0 cos(kx) sin(ky)."""
    k = 2 * math.pi / N
    x = np.arange(N, dtype=np.float64)
    X, Y = np.meshgrid(x, x)
    ux = U0 * np.sin(k * X) * np.cos(k * Y)
    uy = -U0 * np.cos(k * X) * np.sin(k * Y)
    rho = rho0 - rho0 * U0 * U0 / 4.0 * (np.cos(2 * k * X) + np.cos(2 * k * Y))
    return rho, ux, uy


def disc_flags(N: int, r: float):
    x = np.arange(N, dtype=np.float64)
    X, Y = np.meshgrid(x, x)
    c = N / 2.0
    return (((X - c) ** 2 + (Y - c) ** 2) < r * r).astype(np.uint8)


def rankine_hugoniot(mach: float, gamma: float = 5.0 / 3.0, rho1: float = 1.0, T1: float = 1.0):
    """Upstream and downstream states {rho, u, T} of a stationary normal shock
    of an ideal gas (R = 1) with upstream Mach number `mach` relative to the
    upstream sound speed sqrt(gamma T1), from the Rankine-Hugoniot jump
    relations (the initial and end states of the shock structure problem)."""
    m2 = mach * mach
    r = (gamma + 1) * m2 / ((gamma - 1) * m2 + 2)            # rho2 / rho1
    pr = 1 + 2 * gamma / (gamma + 1) * (m2 - 1)               # p2 / p1
    u1 = mach * math.sqrt(gamma * T1)
    return (rho1, u1, T1), (rho1 * r, u1 / r, T1 * pr / r)


def shock_batch(count: int = 256, seed: int = 2, mach_range=(1.2, 4.0), len_range=(1024, 8192),
                gamma: float = 5.0 / 3.0, width: float = 20.0, cells_per_mfp: float = 50.0):
    """A batch of independent quasi-one-dimensional shock instances: upstream
    Mach numbers uniform in mach_range, lengths uniform in len_range (cells),
    Rankine-Hugoniot states joined by a tanh ramp of `width` cells at the
    middle.  The upstream mean free path of hard spheres,
    lambda_1 = 16 / (5 sqrt(2 pi gamma)) mu_1 a_1 / p_1, is `cells_per_mfp`
    cells (the paper resolves it with 50), which fixes mu_1.  Returns per
    instance: length, Mach, the two end states and mu_1, T_1, and a function
    giving the initial rho, u, T of an instance on its cells."""
    rng = np.random.default_rng(seed)
    mach = rng.uniform(*mach_range, count)
    lens = rng.integers(len_range[0], len_range[1] + 1, count)
    out = []
    for M, L in zip(mach, lens):
        s1, s2 = rankine_hugoniot(float(M), gamma)
        a1 = math.sqrt(gamma * s1[2])
        p1 = s1[0] * s1[2]
        mu1 = cells_per_mfp * p1 * 5 * math.sqrt(2 * math.pi * gamma) / (16 * a1)
        out.append({"len": int(L), "mach": float(M), "left": s1, "right": s2, "mu1": mu1,
                    "T1": s1[2]})
    return out


def couette_batch(count: int = 128, seed: int = 3, h_range=(64, 512), kn_range=(0.01, 1.0),
                  wall_speed: float = 0.1):
    """A batch of independent Couette channels: heights H uniform in h_range
    (cells between the walls), Knudsen numbers Kn = lambda / H log-uniform in
    kn_range, walls moving at -wall_speed (y = 0) and +wall_speed (y = H - 1)
    along the streamwise axis.  Returns per channel H, Kn and the two wall
    speeds."""
    rng = np.random.default_rng(seed)
    hs = rng.integers(h_range[0], h_range[1] + 1, count)
    kn = np.exp(rng.uniform(math.log(kn_range[0]), math.log(kn_range[1]), count))
    return [{"H": int(h), "kn": float(k), "uw_lo": -wall_speed, "uw_hi": wall_speed}
            for h, k in zip(hs, kn)]


def channel_layout(widths, G: int):
    """Columns of channels placed side by side along x with 2 G gap columns
    between neighbours and G before the first / after the last: returns the
    first column of every channel and the grid width."""
    x0, x = [], G
    for w in widths:
        x0.append(x)
        x += int(w) + 2 * G
    return x0, x - G


def shock_profile(inst: dict, nx: int, width: float = 20.0):
    """rho, u, T of one instance on nx cells (cells beyond its length hold the
    downstream state): the tanh ramp between the end states at the middle."""
    L = inst["len"]
    x = np.arange(nx, dtype=np.float64)
    w = 0.5 * (1 + np.tanh((x - 0.5 * L) / width))
    w[L:] = 1.0
    (r1, u1, t1), (r2, u2, t2) = inst["left"], inst["right"]
    return r1 + (r2 - r1) * w, u1 + (u2 - u1) * w, t1 + (t2 - t1) * w
