"""Seeded synthetic workloads shaped like the paper's cases.

This module holds the initial states and the parameter sets only: none of the
method's arithmetic lives here.  It is the single input source shared by the
CUDA path and the CPU oracle, and it imports neither.

A parameter set is a plain ``dict`` with the physical names of the method
(Sec. 2 and the parameter paragraph of Sec. 4):

``dim, nx, ny, nz, dx, dt, cs, rhoL, rhoG, etaL, etaG, rho_ref, sigma, M, W,
g (3-tuple), bc (3-tuple of "periodic" | "noslip" | "freeslip"),
ch_scheme (2 | 4), iso (9 | 15 | 19 | 27), bulk_visc, p_average, ch_advection``

and a field set is a ``dict`` of float64 numpy arrays ``phi, p, u, v[, w]``
of shape ``(ny, nx)`` or ``(nz, ny, nx)``.  The velocity component along an
axis lives on the low face of each cell along that axis.

Uniform noise is drawn from SplitMix64 (Steele, Lea & Flood 2014) of
``seed * 2**32 + cell index``, mapped to ``[-amp, amp]`` with 53-bit mantissas,
so the same cell gets the same number at any grid decomposition.
"""
from __future__ import annotations

import math

import numpy as np

_M64 = (1 << 64) - 1


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser of the uint64 counters ``x`` (published constants)."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & np.uint64(_M64)
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & np.uint64(_M64)
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & np.uint64(_M64)
        return z ^ (z >> np.uint64(31))


def uniform_noise(seed: int, shape, amp: float) -> np.ndarray:
    """Uniform numbers in [-amp, amp], one per cell, from SplitMix64(seed, index)."""
    n = int(np.prod(shape))
    ctr = np.arange(n, dtype=np.uint64) + np.uint64((int(seed) & 0xFFFFFFFF) << 32)
    r = splitmix64(ctr)
    u01 = (r >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return (amp * (2.0 * u01 - 1.0)).reshape(shape)


def base_params(dim: int, nx: int, ny: int, nz: int = 1, **kw) -> dict:
    prm = dict(dim=dim, nx=nx, ny=ny, nz=nz if dim == 3 else 1, dx=1.0, dt=0.1, cs=1.0,
               rhoL=1.0, rhoG=0.1, etaL=0.1, etaG=0.01, rho_ref=0.0, sigma=0.01, M=0.02, W=4.0,
               g=(0.0, 0.0, 0.0), bc=("periodic",) * 3, ch_scheme=2 if dim == 2 else 4,
               iso=9 if dim == 2 else 15, bulk_visc=1, p_average=1, ch_advection=0)
    prm.update(kw)
    return prm


def shape_of(prm: dict):
    if prm["dim"] == 3:
        return (prm["nz"], prm["ny"], prm["nx"])
    return (prm["ny"], prm["nx"])


def zero_fields(prm: dict) -> dict:
    shp = shape_of(prm)
    f = {k: np.zeros(shp) for k in ("phi", "p", "u", "v")}
    if prm["dim"] == 3:
        f["w"] = np.zeros(shp)
    return f


def cell_centres(prm: dict):
    """Coordinates of the cell centres, one array per axis (x, y[, z])."""
    dx = prm["dx"]
    if prm["dim"] == 3:
        z, y, x = np.meshgrid((np.arange(prm["nz"]) + 0.5) * dx, (np.arange(prm["ny"]) + 0.5) * dx,
                              (np.arange(prm["nx"]) + 0.5) * dx, indexing="ij")
        return x, y, z
    y, x = np.meshgrid((np.arange(prm["ny"]) + 0.5) * dx, (np.arange(prm["nx"]) + 0.5) * dx,
                       indexing="ij")
    return x, y


# ---------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------

def static_drop(n: int = 64, R: float = 16.0, W_cfg: float = 2.0, noise: float = 1e-3, seed: int = 1,
                steps: int = 2000):
    """2D static drop, periodic n x n, dx = 1, drop of radius R centred in the box.

    phi = tanh((R - r) / (sqrt(2) W_cfg)) + U[-noise, noise]; u = v = p = 0.
    Density ratio 10, viscosity ratio 10 (heavy inside), sigma = 0.01,
    M = 0.02, Mach 0.1, acoustic CFL 0.3.  With U_c = sigma / eta_L (Sec. 4)
    and eta_L = 0.1 this gives c_s = 1, dt = 0.3.  The model width W is the
    one whose equilibrium profile tanh(2d/W) equals the prescribed initial
    profile: W = 2 sqrt(2) W_cfg.
    """
    etaL, sigma, Ma, cfl = 0.1, 0.01, 0.1, 0.3
    Uc = sigma / etaL
    cs = Uc / Ma
    prm = base_params(2, n, n, dx=1.0, cs=cs, dt=cfl * 1.0 / cs, rhoL=1.0, rhoG=0.1, etaL=etaL,
                      etaG=etaL / 10.0, sigma=sigma, M=0.02, W=2.0 * math.sqrt(2.0) * W_cfg,
                      bc=("periodic", "periodic", "periodic"))
    prm["steps"] = steps
    f = zero_fields(prm)
    x, y = cell_centres(prm)
    r = np.sqrt((x - n / 2.0) ** 2 + (y - n / 2.0) ** 2)
    f["phi"] = np.tanh((R - r) / (math.sqrt(2.0) * W_cfg)) + uniform_noise(seed, f["phi"].shape, noise)
    return prm, f


def rayleigh_taylor(nx: int = 256, ny: int = 1024, variant: str = "pe1000"):
    """2D Rayleigh-Taylor, width 1, height 4, periodic in x, free-slip walls in y.

    Heavy fluid (phi = +1, rho_L = 1) over light (rho_G = 1/3, Atwood 0.5),
    equal viscosity, Re = sqrt(g lambda^3)/nu_L = 3000 with g = lambda = 1,
    sigma = 0, rho_ref = rho_G, W = 4 cells, interface y = 2 + 0.1 cos(2 pi x).
    The sound speed follows the paper's RT runs, c = dx/dt_paper = 200 U_c
    (c_s = c / sqrt 3).  ``variant="pe1000"``: Pe = 1000 (M = 1e-3) and
    dt = 1.2e-6, about half the explicit CH limit; ``variant="paper"``:
    Pe = 8e4 and N_t = 51200 steps per unit time.
    """
    dx = 1.0 / nx
    cs = 200.0 / math.sqrt(3.0)
    if variant == "paper":
        M, dt = 1.0 / 8e4, 1.0 / 51200.0
    else:
        M, dt = 1.0e-3, 1.2e-6
    eta = 1.0 / 3000.0
    prm = base_params(2, nx, ny, dx=dx, dt=dt, cs=cs, rhoL=1.0, rhoG=1.0 / 3.0, etaL=eta, etaG=eta,
                      rho_ref=1.0 / 3.0, sigma=0.0, M=M, W=4.0 * dx, g=(0.0, -1.0, 0.0),
                      bc=("periodic", "freeslip", "periodic"))
    f = zero_fields(prm)
    x, y = cell_centres(prm)
    h = 2.0 + 0.1 * np.cos(2.0 * math.pi * x)
    f["phi"] = np.tanh(2.0 * (y - h) / prm["W"])
    return prm, f


def bubble3d(nx: int = 256, ny: int = 256, nz: int = 512, R: float = 32.0, gap: float = 64.0,
             W: float = 3.0):
    """3D buoyant bubble in a closed box (no-slip walls on all sides), dx = dt = 1.

    Liquid outside (phi = +1, rho_L = 1), gas bubble inside (rho_G = 0.1),
    viscosity ratio 10, Eotvos g drho D^2/sigma = 10 and Morton
    g eta_L^4 drho/(rho_L^2 sigma^3) = 1e-4 with D = 2R and g = 1e-5 along -z;
    c_s = 1/sqrt 3 (the paper's tie to dx/dt), M = 0.01, rho_ref = rho_L,
    D3Q15 isotropic stencils and RK4 for the CH equation.  The bubble centre
    sits ``gap + R`` cells above the bottom wall, centred in x and y.
    """
    rhoL, rhoG, g = 1.0, 0.1, 1e-5
    D = 2.0 * R
    sigma = g * (rhoL - rhoG) * D * D / 10.0
    etaL = (1e-4 * rhoL * rhoL * sigma ** 3 / (g * (rhoL - rhoG))) ** 0.25
    prm = base_params(3, nx, ny, nz, dx=1.0, dt=1.0, cs=1.0 / math.sqrt(3.0), rhoL=rhoL, rhoG=rhoG,
                      etaL=etaL, etaG=etaL / 10.0, rho_ref=rhoL, sigma=sigma, M=0.01, W=W,
                      g=(0.0, 0.0, -g), bc=("noslip", "noslip", "noslip"), ch_scheme=4, iso=15)
    f = zero_fields(prm)
    x, y, z = cell_centres(prm)
    r = np.sqrt((x - nx / 2.0) ** 2 + (y - ny / 2.0) ** 2 + (z - (gap + R)) ** 2)
    f["phi"] = -np.tanh(2.0 * (R - r) / W)
    return prm, f


def random_fields(prm: dict, seed: int, amp_u: float = 0.05, amp_p: float = 0.01) -> dict:
    """A rough synthetic state for operator-level parity: phi in (-1, 1) with
    interfaces of a few cells, velocities and pressure of the given amplitudes.
    Wall faces of the normal velocity are zeroed."""
    shp = shape_of(prm)
    f = {}
    base = uniform_noise(seed, shp, 1.0)
    # a smooth-ish phi: tanh of a low-pass of the noise
    sm = base.copy()
    for ax in range(len(shp)):
        sm = (np.roll(sm, 1, ax) + 2.0 * sm + np.roll(sm, -1, ax)) / 4.0
    f["phi"] = np.tanh(4.0 * sm)
    f["p"] = uniform_noise(seed + 101, shp, amp_p)
    names = ["u", "v", "w"][: prm["dim"]]
    for a, nm in enumerate(names):
        vel = uniform_noise(seed + 202 + a, shp, amp_u)
        if prm["bc"][a] != "periodic":
            ax = len(shp) - 1 - a
            sl = [slice(None)] * len(shp)
            sl[ax] = 0
            vel[tuple(sl)] = 0.0
        f[nm] = vel
    return f


def batch_instances(n: int = 96, seed: int = 0, sides=(64, 128, 192, 256, 384, 512), precision: int = 32):
    """The batched 2D workload: n drops and bubbles on periodic boxes.

    Per instance (seeded): side from ``sides``; density ratio log-uniform in
    [2, 100] (rho_L = 1); viscosity ratio log-uniform in [1, 50]
    (eta_L = 0.1); radius uniform in [0.15, 0.3] x side, centred; sigma
    uniform in [1e-3, 1e-2]; M uniform in [5e-3, 2e-2]; W = 4 cells.  Even
    instances are drops (phi = +1 inside, g = 0), odd ones bubbles (phi = -1
    inside, |g| uniform in [0, 1e-5] along -y, rho_ref the mean density of
    the initial state, so that the periodic box does not accelerate).  The
    sound speed is U_c / Ma with U_c = sigma / eta_L and Ma = 0.1; dt is the
    acoustic CFL 0.3 step, reduced where needed to dx^2 / (16 nu_max) (0.6 of
    the RK3 viscous limit 2.51 dx^2 / (24 nu_max) of a 2D grid with bulk
    viscosity) and to 0.4 of the CH bound 2 / (M lam (8a + kappa lam)),
    lam = 16/3 dx^-2.  Returns (list of params, list of field dicts)."""
    rng = np.random.default_rng(seed)
    prms, fields = [], []
    for k in range(n):
        side = int(rng.choice(sides))
        r_rho = float(np.exp(rng.uniform(np.log(2.0), np.log(100.0))))
        r_eta = float(np.exp(rng.uniform(np.log(1.0), np.log(50.0))))
        frac = float(rng.uniform(0.15, 0.3))
        sigma = float(rng.uniform(1e-3, 1e-2))
        M = float(rng.uniform(5e-3, 2e-2))
        gmag = float(rng.uniform(0.0, 1e-5)) if k % 2 else 0.0
        etaL, W, dx = 0.1, 4.0, 1.0
        rhoL, rhoG, etaG = 1.0, 1.0 / r_rho, etaL / r_eta
        cs = (sigma / etaL) / 0.1
        nu_max = max(etaL / rhoL, etaG / rhoG)
        lam = 16.0 / 3.0 / (dx * dx)
        a, kappa = 3.0 / (4.0 * W), 3.0 * W / 8.0
        dt = min(0.3 * dx / cs, 0.4 * 2.5 * dx * dx / (16.0 * nu_max), 0.4 * 2.0 / (M * lam * (8.0 * a + kappa * lam)))
        prm = base_params(2, side, side, dx=dx, dt=dt, cs=cs, rhoL=rhoL, rhoG=rhoG, etaL=etaL, etaG=etaG,
                          sigma=sigma, M=M, W=W, g=(0.0, -gmag, 0.0), bc=("periodic", "periodic", "periodic"),
                          ch_scheme=2, iso=9)
        prm["precision"] = precision
        f = zero_fields(prm)
        x, y = cell_centres(prm)
        r = np.sqrt((x - side / 2.0) ** 2 + (y - side / 2.0) ** 2)
        sign = 1.0 if k % 2 == 0 else -1.0
        f["phi"] = sign * np.tanh(2.0 * (frac * side - r) / W)
        rho0 = 0.5 * (rhoL * (1.0 + f["phi"]) + rhoG * (1.0 - f["phi"]))
        prm["rho_ref"] = float(np.mean(rho0)) if gmag > 0 else 0.0
        prms.append(prm)
        fields.append(f)
    return prms, fields


def two_drops(seed: int, n: int = 256, gap=(2.0, 8.0), precision: int = 32):
    """Two drops on a periodic n x n box: the surrogate's training and test case.

    Seeded draws: radii R1, R2 uniform in [20, 50] cells (scaled by n / 256
    on other boxes); density ratio
    log-uniform in [2, 20] (rho_L = 1) with the viscosity ratio equal to it
    (eta_L = 0.1, so both phases have the kinematic viscosity 0.1); the
    first centre uniform on the box, the second at the distance
    R1 + R2 + gap in a uniform direction, gap uniform in ``gap`` cells, so
    that the drops are separate but close enough to coalesce within a few
    thousand steps.  phi is the larger of the two profiles
    tanh(2 (R - d) / W), d the periodic distance to the centre.
    sigma = 0.01, M = 0.02, W = 4, Mach 0.1 with U_c = sigma / eta_L
    (c_s = 1) and acoustic CFL 0.3 (dt = 0.3; the viscous and CH bounds of
    ``batch_instances`` are looser here).  u = v = p = 0.
    Returns (params, fields)."""
    rng = np.random.default_rng([seed, 20110814])
    R1, R2 = (float(r) * n / 256.0 for r in rng.uniform(20.0, 50.0, size=2))
    r_rho = float(np.exp(rng.uniform(np.log(2.0), np.log(20.0))))
    c1 = rng.uniform(0.0, n, size=2)
    ang = float(rng.uniform(0.0, 2.0 * math.pi))
    dist = R1 + R2 + float(rng.uniform(*gap))
    c2 = (c1 + dist * np.array([math.cos(ang), math.sin(ang)])) % n
    etaL, sigma, M, W, dx = 0.1, 0.01, 0.02, 4.0, 1.0
    rhoL, rhoG, etaG = 1.0, 1.0 / r_rho, etaL / r_rho
    cs = (sigma / etaL) / 0.1
    nu_max = max(etaL / rhoL, etaG / rhoG)
    lam = 16.0 / 3.0 / (dx * dx)
    a, kappa = 3.0 / (4.0 * W), 3.0 * W / 8.0
    dt = min(0.3 * dx / cs, 0.4 * 2.5 * dx * dx / (16.0 * nu_max), 0.4 * 2.0 / (M * lam * (8.0 * a + kappa * lam)))
    prm = base_params(2, n, n, dx=dx, dt=dt, cs=cs, rhoL=rhoL, rhoG=rhoG, etaL=etaL, etaG=etaG, sigma=sigma, M=M,
                      W=W, bc=("periodic", "periodic", "periodic"), ch_scheme=2, iso=9)
    prm["precision"] = precision
    prm["r_rho"] = r_rho
    f = zero_fields(prm)
    x, y = cell_centres(prm)

    def pdist(c):
        dxp = np.abs(x - c[0])
        dyp = np.abs(y - c[1])
        dxp = np.minimum(dxp, n - dxp)
        dyp = np.minimum(dyp, n - dyp)
        return np.sqrt(dxp ** 2 + dyp ** 2)

    f["phi"] = np.maximum(np.tanh(2.0 * (R1 - pdist(c1)) / W), np.tanh(2.0 * (R2 - pdist(c2)) / W))
    return prm, f


def capillary_wave(n: int = 64, nt: int = 384, cn: float = 0.0625, pe: float = 2.0e4, precision: int = 64):
    """The 2D capillary wave of Sec. "Capillary wave in 2D", on the lower half
    of the unit square (the wave is symmetric about y = 1/2).

    L_c = 1 and U_c = sigma / eta_L = 1, so T_c = 1; Re = rho_L U_c L_c /
    eta_L = 1000 gives eta_L = sigma = 10^-3; r_rho = r_eta = 20 (rho_L = 1,
    equal kinematic viscosities); Cn = W / L_c = 0.0625; Pe = U_c L_c^2 / (M
    sigma_ref) = 2 10^4 with the reference surface tension sigma_ref = 1 of
    the chemical potential gives M = 5 10^-5.  dx = 1/n, dt = T_c / nt and c_s = nt /
    (sqrt(3) n) U_c (the paper's N_L = 64, N_t = 384, c = 6).  x in [0, 1]
    between no-slip walls; y in [0, 1/2] between symmetry planes (free-slip
    walls).  Gas on the left, liquid on the right: phi = tanh(2 (x - h(y)) /
    Cn), h(y) = 1/2 + 0.01 cos(2 pi (y + 1/2)).  u = v = p = 0.  The fine
    mesh of the paper's refinement study is n = 128, nt = 1920, cn = 0.03125,
    pe = 4 10^4.  Returns (params, fields)."""
    Re, r, Cn, Pe, Ap = 1000.0, 20.0, cn, pe, 0.01
    sigma = 1.0 / Re
    etaL = sigma
    M = 1.0 / Pe
    dx, dt = 1.0 / n, 1.0 / nt
    cs = nt / (math.sqrt(3.0) * n)
    prm = base_params(2, n, n // 2, dx=dx, dt=dt, cs=cs, rhoL=1.0, rhoG=1.0 / r, etaL=etaL, etaG=etaL / r,
                      sigma=sigma, M=M, W=Cn, bc=("noslip", "freeslip", "periodic"), ch_scheme=2, iso=9)
    prm["precision"] = precision
    prm["amplitude"] = Ap
    f = zero_fields(prm)
    x, y = cell_centres(prm)
    h = 0.5 + Ap * np.cos(2.0 * math.pi * (y + 0.5))
    f["phi"] = np.tanh(2.0 * (x - h) / Cn)
    return prm, f


# ---------------------------------------------------------------------------
# axisymmetric workloads (x = r with the axis at x = 0, y = z; "axisym": 1)
# ---------------------------------------------------------------------------

def _axisym_drop(prm: dict, zc: float, R: float, cn: float, noise: float, seed: int) -> dict:
    f = zero_fields(prm)
    r, z = cell_centres(prm)
    rdc = np.sqrt((z - zc) ** 2 + r**2)
    f["phi"] = -np.tanh(2.0 * (rdc - R) / cn)
    if noise > 0:
        f["phi"] = f["phi"] + uniform_noise(seed, f["phi"].shape, noise)
    return f


def falling_drop(n_l: int = 50, n_t: int = 4000, cn: float = 0.06, pe: float = 1000.0, precision: int = 64,
                 noise: float = 0.0, seed: int = 0):
    """The axisymmetric falling drop of Sec. "Falling drop": L_c = R = 1 with
    n_l cells per R, domain r in [0, 8], z in [0, 24] (at n_l = 50: 400 x 1200
    cells), axis at r = 0, no-slip walls elsewhere.  r_rho = 1.15, r_eta = 1,
    Eo = g (rho_L - rho_G) D^2 / sigma = 144, Oh = eta_L / sqrt(rho_L D sigma)
    = 0.0466 (D = 2R), rho_ref = rho_G, gravity along +z; the drop starts at
    (z, r) = (2, 0).  U_c = sigma / eta_L = 1 and T_c = L_c / U_c = 1, so
    sigma = eta_L = 2 Oh^2 and g = Eo sigma / ((rho_L - rho_G) D^2);
    dx = 1/n_l, dt = 1/n_t, c_s = (dx / dt) / sqrt 3 (the paper's N_L = 50,
    N_t = 4000, c = 80), W = Cn, M = 1/Pe (Pe with the chemical potential's
    sigma_ref = 1).  One T'_c = sqrt(D/g) is about 1.29 T_c.  Returns
    (params, fields)."""
    R, D, rhoL, r_rho, Eo, Oh = 1.0, 2.0, 1.0, 1.15, 144.0, 0.0466
    rhoG = rhoL / r_rho
    etaL = 2.0 * Oh * Oh * rhoL
    sigma = etaL  # U_c = sigma / eta_L = 1
    g = Eo * sigma / ((rhoL - rhoG) * D * D)
    dx, dt = R / n_l, 1.0 / n_t
    prm = base_params(2, 8 * n_l, 24 * n_l, dx=dx, dt=dt, cs=(dx / dt) / math.sqrt(3.0), rhoL=rhoL,
                      rhoG=rhoG, etaL=etaL, etaG=etaL, rho_ref=rhoG, sigma=sigma, M=1.0 / pe, W=cn * R,
                      g=(0.0, g, 0.0), bc=("noslip", "noslip", "periodic"), ch_scheme=2, iso=9, axisym=1)
    prm["precision"] = precision
    return prm, _axisym_drop(prm, 2.0 * R, R, cn * R, noise, seed)


def drop_coalescence(oh: float = 0.119, n_l: int = 40, n_t: int = None, cn: float = 0.1, pe: float = 8.0e3,
                     precision: int = 64, noise: float = 0.0, seed: int = 0):
    """The axisymmetric coalescence of two equal drops of Sec. "Drop
    coalescence (axisymmetric)": the quarter r in [0, 3], z in [0, 3] with
    symmetric boundaries on every side (the plane z = 0 mirrors the second
    drop), L_c = R = 1 with n_l cells per R (120 x 120 at n_l = 40), the drop
    centred at (z, r) = (1, 0).  r_rho = 50, r_eta = 58.8, Oh = eta_L /
    sqrt(rho_L sigma R) in {0.037, 0.119, 0.3}; U_c = sigma / eta_L = 1, so
    sigma = eta_L = Oh^2.  n_t defaults to the paper's 400 (c = 10), or 2000
    (c = 50) at Oh = 0.3.  Returns (params, fields)."""
    R, rhoL = 1.0, 1.0
    if n_t is None:
        n_t = 2000 if oh >= 0.3 else 400
    etaL = oh * oh * rhoL
    dx, dt = R / n_l, 1.0 / n_t
    prm = base_params(2, 3 * n_l, 3 * n_l, dx=dx, dt=dt, cs=(dx / dt) / math.sqrt(3.0), rhoL=rhoL,
                      rhoG=rhoL / 50.0, etaL=etaL, etaG=etaL / 58.8, rho_ref=0.0, sigma=etaL, M=1.0 / pe,
                      W=cn * R, bc=("freeslip", "freeslip", "periodic"), ch_scheme=2, iso=9, axisym=1)
    prm["precision"] = precision
    return prm, _axisym_drop(prm, 1.0 * R, R, cn * R, noise, seed)
