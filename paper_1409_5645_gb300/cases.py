"""Seeded synthetic inputs for the free-surface LBM step.

This module only builds *inputs*: cell flags, densities, velocities, fill
levels, seeded noise and wall link fractions, from the geometry of each
workload.  It holds none of the method's arithmetic (no equilibrium, no
collision, no closure): both the CUDA library and the CPU oracle turn these
arrays into populations themselves.

Layout conventions (shared with the C interface):
  * cell index ``i = x + nx*(y + ny*z)`` (x fastest),
  * per-link arrays are ``[19][N]`` in the library's population order,
  * cell flags: LIQUID=1, INTERFACE=2, GAS=4, WALL=8,
  * node (x, y, z) sits at the physical point (x+1/2, y+1/2, z+1/2); a
    non-periodic face is a half-way wall on the domain boundary.

Workloads follow the paper's test cases (Sec. 4.3 film flows, Sec. 4.4 dam
break) and the standing wave; sizes are parameters.
"""
from __future__ import annotations

import math

import numpy as np

LIQUID, INTERFACE, GAS, WALL = 1, 2, 4, 8

# D3Q19 link directions in the public population order (an interface
# convention of the C ABI: rest, 6 axis links, 12 diagonals, each followed by
# its opposite).  Used here only to place wall link fractions.
LINKS = np.array(
    [[0, 0, 0],
     [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
     [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0],
     [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1],
     [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]], dtype=np.int64)

SEED = 1409

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Counter-based SplitMix64 (Steele, Lea, Flood 2014): output k is the
    finaliser applied to ``seed + (offset + k + 1) * golden``."""
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, amp: float, offset: int = 0) -> np.ndarray:
    """Uniform numbers in [-amp, amp) from the top 53 bits of SplitMix64."""
    u = (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return amp * (2.0 * u - 1.0)


def default_params(**kw) -> dict:
    p = dict(tau=0.8, magic=3.0 / 16.0, g=(0.0, 0.0, 0.0), rho_G=1.0, sigma=0.0,
             rule=1, compressible=0, linear_eq=0, eps=1e-3,
             periodic=(0, 0, 0), zshift=0, freeze=0, cleanup=3, delta_min=0.0, stress=0)
    p.update(kw)
    return p


class Case(dict):
    """dict with keys dims, params, flags, rho, u, phi, noise, wall_delta."""

    @property
    def N(self) -> int:
        nx, ny, nz = self["dims"]
        return nx * ny * nz


def _neighbour_index(dims, periodic, zshift, i, c):
    """Index of cell i + c (arrays), -1 beyond a non-periodic face."""
    nx, ny, nz = dims
    x = i % nx
    y = (i // nx) % ny
    z = i // (nx * ny)
    X, Y, Z = x + c[0], y + c[1], z + c[2]
    ok = np.ones_like(i, dtype=bool)
    if periodic[0]:
        lo, hi = X < 0, X >= nx
        Z = Z + np.where(lo, zshift, 0) - np.where(hi, zshift, 0)
        X = np.where(lo, X + nx, np.where(hi, X - nx, X))
    else:
        ok &= (X >= 0) & (X < nx)
    if periodic[1]:
        Y = np.mod(Y, ny)
    else:
        ok &= (Y >= 0) & (Y < ny)
    if periodic[2]:
        Z = np.mod(Z, nz)
    ok &= (X >= 0) & (X < nx) & (Y >= 0) & (Y < ny) & (Z >= 0) & (Z < nz)
    out = X + nx * (Y + ny * Z)
    return np.where(ok, out, -1)


def classify(dims, periodic, zshift, phi, solid=None, sharp=False) -> np.ndarray:
    """Flags from fill levels: phi == 0 -> GAS, a cell with phi > 0 that has a
    gas cell along one of the 18 links -> INTERFACE, else LIQUID; solid cells
    -> WALL.  ``sharp=True`` (frozen-interface test geometries) takes a cell as
    liquid only when its node lies inside the liquid, i.e. phi >= 1/2 for a
    planar cut, so that every boundary node has its surface ahead of it."""
    N = int(np.prod(dims))
    thresh = (phi >= 0.5) if sharp else (phi > 0.0)
    flags = np.where(thresh, LIQUID, GAS).astype(np.uint8)
    if solid is not None:
        flags[solid] = WALL
    i = np.arange(N, dtype=np.int64)
    gas = flags == GAS
    near_gas = np.zeros(N, dtype=bool)
    for q in range(1, 19):
        j = _neighbour_index(dims, periodic, zshift, i, LINKS[q])
        near_gas |= (j >= 0) & gas[np.maximum(j, 0)]
    flags[(flags == LIQUID) & near_gas] = INTERFACE
    return flags


def _clamped_linear_mean(z0, z1):
    """Exact mean over t in [0,1] of clamp(z0 + (z1-z0) t, 0, 1) (vectorised)."""
    z0 = np.asarray(z0, dtype=np.float64)
    z1 = np.asarray(z1, dtype=np.float64)
    lo = np.minimum(z0, z1)
    hi = np.maximum(z0, z1)
    span = hi - lo
    out = np.empty(np.broadcast(lo, hi).shape)
    flat = span <= 1e-300
    # integral of clamp(s,0,1) ds over [lo,hi] divided by the span
    def G(s):  # antiderivative of clamp(s, 0, 1)
        return np.where(s <= 0.0, 0.0, np.where(s >= 1.0, s - 0.5, 0.5 * s * s))
    with np.errstate(divide="ignore", invalid="ignore"):
        out = (G(hi) - G(lo)) / np.where(flat, 1.0, span)
    return np.where(flat, np.clip(lo, 0.0, 1.0), out)


def film(nx=4, ny=4, nz=32, h=20.0, tau=0.8, gx=1e-6, rule=1, noise_amp=1e-8,
         magic=3.0 / 16.0, seed=SEED, **kw) -> Case:
    """Gravity-driven film on a half-way bounce-back wall at z=0 (Sec. 4.3):
    x, y periodic, liquid depth h (fill 1 below the surface plane z = h, the
    exact cut fraction in the cut cell, 0 above), rho = rho_G = 1, u = 0,
    populations at equilibrium plus seeded uniform noise."""
    dims = (nx, ny, nz)
    N = nx * ny * nz
    z = np.arange(N) // (nx * ny)
    phi = np.clip(h - z, 0.0, 1.0).astype(np.float64)
    params = default_params(tau=tau, magic=magic, g=(gx, 0.0, 0.0), rule=rule,
                            periodic=(1, 1, 0))
    params.update(kw)
    sharp = bool(params["freeze"])
    flags = classify(dims, params["periodic"], 0, phi, sharp=sharp)
    noise = uniform(seed, 19 * N, noise_amp) if noise_amp else None
    keep = (flags == INTERFACE) | ((flags == GAS) & sharp)
    return Case(dims=dims, params=params, flags=flags, rho=np.ones(N),
                u=np.zeros((N, 3)), phi=np.where(keep, phi, 0.0),
                noise=noise, wall_delta=None, h=h)


def film_profile(z, h, g, nu):
    """Steady half-Poiseuille film u(z) = g/(2 nu) (2 h z - z^2)."""
    return g / (2.0 * nu) * (2.0 * h * z - z * z)


def film_transient(z, t, h, g, nu, terms=200):
    """Film started from rest: u(z,t) = u_s(z) - sum_n b_n sin(l_n z) exp(-nu l_n^2 t),
    l_n = (2n+1) pi / (2h), b_n = 2 g / (nu h l_n^3) (separation of variables for
    u_t = nu u_zz + g, u(0) = 0, u_z(h) = 0, u(z, 0) = 0)."""
    z = np.asarray(z, dtype=np.float64)
    out = film_profile(z, h, g, nu)
    for n in range(terms):
        ln = (2 * n + 1) * math.pi / (2.0 * h)
        bn = 2.0 * g / (nu * h * ln ** 3)
        out = out - bn * np.sin(ln * z) * math.exp(-nu * ln * ln * t)
    return out


def inclined_film(h=8, tau=0.8, rule=1, magic=0.25, wall_offset=0.1, peak=None,
                  headroom=4, init_exact=True, **kw) -> Case:
    """Film on an inclined wall, slope 1/2 (Sec. 4.3, rotated film): ny = 1,
    period nx = 2h with a z-shift of h on the x wrap, wall plane
    z = x/2 + wall_offset (explicit WALL cells below it, link fractions from the
    exact plane), free surface h cells higher (vertical depth h), exact cut
    fill levels, gravity along the slope with g = 2 nu peak / H^2
    (H = 2h/sqrt5 the normal depth), frozen interface.

    ``peak=None`` keeps the Reynolds number fixed across depths as the paper's
    refinement does (g ~ dx^-3 at fixed tau): peak velocity 0.05 at h = 8,
    scaled as 8/h."""
    if peak is None:
        peak = 0.05 * 8.0 / h
    nx, ny, nz = 2 * h, 1, 2 * h + headroom
    dims = (nx, ny, nz)
    N = nx * ny * nz
    i = np.arange(N)
    x = (i % nx) + 0.5
    z = (i // (nx * ny)) + 0.5
    zw = x / 2.0 + wall_offset
    solid = z < zw
    # fill: mean over the cell's x-extent of clamp(z_s(x) - k, 0, 1)
    k = z - 0.5
    xl = x - 0.5
    zs0 = xl / 2.0 + wall_offset + h - k
    zs1 = zs0 + 0.5
    phi = _clamped_linear_mean(zs0, zs1)
    phi = np.where(solid, 0.0, phi)
    params = default_params(tau=tau, magic=magic, rule=rule, periodic=(1, 1, 0),
                            zshift=h, freeze=1)
    params.update(kw)
    nu = (params["tau"] - 0.5) / 3.0
    H = 2.0 * h / math.sqrt(5.0)
    g = 2.0 * nu * peak / (H * H)
    t_hat = np.array([2.0, 0.0, 1.0]) / math.sqrt(5.0)
    params["g"] = tuple(g * t_hat)
    flags = classify(dims, params["periodic"], params["zshift"], phi, solid=solid,
                     sharp=bool(params["freeze"]))
    # wall link fractions: x_b + s c_q crosses the plane z - x/2 - off = 0
    wd = np.full((19, N), -1.0)
    fluid = (flags == LIQUID) | (flags == INTERFACE)
    for q in range(1, 19):
        c = LINKS[q]
        j = _neighbour_index(dims, params["periodic"], params["zshift"], i, c)
        hit = fluid & ((j < 0) | (flags[np.maximum(j, 0)] == WALL))
        denom = c[0] / 2.0 - c[2]
        with np.errstate(divide="ignore", invalid="ignore"):
            s = (z - x / 2.0 - wall_offset) / denom
        good = hit & (denom > 0)
        wd[q, good] = s[good]
    ncoord = (z - zw) * (2.0 / math.sqrt(5.0))
    ut = np.where(fluid, g / (2 * nu) * (2 * H * np.minimum(ncoord, H) - np.minimum(ncoord, H) ** 2), 0.0)
    u = np.zeros((N, 3))
    if init_exact:
        u = ut[:, None] * t_hat[None, :]
    keep = (flags == INTERFACE) | ((flags == GAS) & bool(params["freeze"]))
    return Case(dims=dims, params=params, flags=flags, rho=np.ones(N), u=u,
                phi=np.where(keep, phi, 0.0), noise=None,
                wall_delta=wd.reshape(-1), h=h, H=H, nu=nu, gmag=g,
                ncoord=ncoord, t_hat=t_hat)


def skew_couette(h=8, slope=0.25, period=1, shear=1e-3, tau=1.1, rule=1, magic=0.25,
                 wall_offset=0.1, headroom=4, init_exact=True, **kw) -> Case:
    """Linear Couette flow in a channel inclined with slope dz/dx (Sec. 6,
    rotated Couette flow): ny = 1, period nx = period/slope with a z-shift of
    ``period`` on the x wrap; wall plane z = slope x + wall_offset (WALL cells
    below it, CLI link fractions from the exact plane); free surface at
    vertical height h above the wall plane, exact cut fill levels, frozen;
    the surface shear rate du_t/dn = shear is prescribed through
    S^b = shear/2 (t n^T + n t^T) (stress = 2); steady u = shear d t with d the
    distance from the wall plane and t the unit tangent (1, 0, slope)/L."""
    nx = int(round(period / slope))
    assert abs(nx * slope - period) < 1e-12, "period / slope must be an integer"
    nz = h + period + headroom
    dims = (nx, 1, nz)
    N = nx * nz
    i = np.arange(N)
    x = (i % nx) + 0.5
    z = (i // nx) + 0.5
    L = math.sqrt(1.0 + slope * slope)
    zw = slope * x + wall_offset
    solid = z < zw
    k = z - 0.5
    zs0 = slope * (x - 0.5) + wall_offset + h - k
    phi = np.where(solid, 0.0, _clamped_linear_mean(zs0, zs0 + slope))
    t_hat = np.array([1.0, 0.0, slope]) / L
    n_hat = np.array([-slope, 0.0, 1.0]) / L
    Sb = 0.5 * shear * (np.outer(t_hat, n_hat) + np.outer(n_hat, t_hat))
    params = default_params(tau=tau, magic=magic, rule=rule, periodic=(1, 1, 0), zshift=period,
                            freeze=1, stress=2,
                            shear_b=(Sb[0, 0], Sb[1, 1], Sb[2, 2], Sb[0, 1], Sb[0, 2], Sb[1, 2]))
    params.update(kw)
    flags = classify(dims, params["periodic"], params["zshift"], phi, solid=solid, sharp=True)
    wd = np.full((19, N), -1.0)
    fluid = (flags == LIQUID) | (flags == INTERFACE)
    for q in range(1, 19):
        c = LINKS[q]
        j = _neighbour_index(dims, params["periodic"], params["zshift"], i, c)
        hit = fluid & ((j < 0) | (flags[np.maximum(j, 0)] == WALL))
        denom = slope * c[0] - c[2]
        with np.errstate(divide="ignore", invalid="ignore"):
            s = (z - slope * x - wall_offset) / denom
        good = hit & (denom > 0)
        wd[q, good] = s[good]
    d = (z - zw) / L
    u_exact = np.where(fluid, shear * d, 0.0)[:, None] * t_hat[None, :]
    keep = (flags == INTERFACE) | (flags == GAS)
    return Case(dims=dims, params=params, flags=flags, rho=np.ones(N),
                u=u_exact.copy() if init_exact else np.zeros((N, 3)),
                phi=np.where(keep, phi, 0.0), noise=None, wall_delta=wd.reshape(-1),
                h=h, shear=shear, u_exact=u_exact, d=d, t_hat=t_hat)


def droplet(n=24, R=6.0, centre=None, sigma=1e-3, tau=0.8, rule=1, sub=16, **kw) -> Case:
    """Spherical liquid droplet of radius R at rest in gas (fully periodic
    n^3 box, no gravity), frozen interface, surface tension sigma: the static
    Laplace test (Sec. 2.3, Laplace pressure).  Fill levels are the liquid
    fraction of each cell, sampled on sub^3 points (cells away from the
    surface are exactly 0 or 1)."""
    dims = (n, n, n)
    N = n ** 3
    if centre is None:
        centre = (n / 2 + 0.13, n / 2 - 0.21, n / 2 + 0.07)  # off the lattice symmetry
    i = np.arange(N)
    x, y, z = i % n + 0.5, (i // n) % n + 0.5, i // (n * n) + 0.5
    r = np.sqrt((x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2)
    phi = np.where(r < R, 1.0, 0.0)
    near = np.abs(r - R) < 1.0
    o = (np.arange(sub) + 0.5) / sub - 0.5
    ox, oy, oz = np.meshgrid(o, o, o, indexing="ij")
    ox, oy, oz = ox.ravel(), oy.ravel(), oz.ravel()
    for j in np.where(near)[0]:
        rr = np.sqrt((x[j] + ox - centre[0]) ** 2 + (y[j] + oy - centre[1]) ** 2 + (z[j] + oz - centre[2]) ** 2)
        phi[j] = np.mean(rr < R)
    params = default_params(tau=tau, rule=rule, sigma=sigma, periodic=(1, 1, 1), freeze=1)
    params.update(kw)
    flags = classify(dims, params["periodic"], 0, phi, sharp=True)
    keep = (flags == INTERFACE) | (flags == GAS)
    return Case(dims=dims, params=params, flags=flags, rho=np.ones(N), u=np.zeros((N, 3)),
                phi=np.where(keep, phi, 0.0), noise=None, wall_delta=None, R=R, centre=centre, r=r)


def standing_wave(n=128, depth=64.0, amp=2.0, tau=0.55, g=2e-5, sigma=1e-4,
                  phi_noise=1e-4, seed=SEED, quad=8, rule=1, **kw) -> Case:
    """Standing gravity-capillary wave in an n^3 box with walls on all faces:
    surface z = depth + amp cos(2 pi x / n) cos(2 pi y / n); fill levels from
    the exact cut volume (quad x quad Gauss quadrature of clamp(s - k, 0, 1)
    over the cell's x-y square), seeded fill noise on interface cells,
    hydrostatic density."""
    dims = (n, n, n)
    N = n ** 3
    gx, gw = np.polynomial.legendre.leggauss(quad)
    gx = 0.5 * (gx + 1.0)
    gw = 0.5 * gw
    xs = np.arange(n)
    # surface heights at quadrature points, per column
    X = xs[:, None] + gx[None, :]  # (n, quad)
    cx = np.cos(2 * math.pi * X / n)
    phi = np.empty((n, n, n))
    for k in range(n):
        s = depth + amp * cx[None, :, None, :] * cx[:, None, :, None] - k  # (y, x, qy, qx)
        v = np.clip(s, 0.0, 1.0)
        phi[k] = np.einsum("yxab,a,b->yx", v, gw, gw)
    phi = phi.reshape(-1)
    phi[np.abs(phi) < 1e-15] = 0.0
    phi[np.abs(phi - 1.0) < 1e-15] = 1.0
    params = default_params(tau=tau, g=(0.0, 0.0, -g), sigma=sigma, rule=rule)
    params.update(kw)
    flags = classify(dims, params["periodic"], 0, phi)
    i = np.arange(N)
    x = (i % n) + 0.5
    y = ((i // n) % n) + 0.5
    z = (i // (n * n)) + 0.5
    surf = depth + amp * np.cos(2 * math.pi * x / n) * np.cos(2 * math.pi * y / n)
    rho = params["rho_G"] + 3.0 * g * np.maximum(surf - z, 0.0)
    ifc = flags == INTERFACE
    phi = np.where(ifc, phi, 0.0)
    phi[ifc] += uniform(seed, int(ifc.sum()), phi_noise, offset=19 * N)
    return Case(dims=dims, params=params, flags=flags, rho=rho, u=np.zeros((N, 3)),
                phi=phi, noise=None, wall_delta=None, depth=depth, amp=amp)


def dam_break(nx=512, ny=256, nz=256, col_x=128, col_z=192, tau=0.51, g=1e-5,
              phi_noise=1e-3, seed=SEED, rule=1, **kw) -> Case:
    """Dam break (Sec. 4.4) at throughput scale: walls on all faces, liquid
    column x < col_x, z < col_z at rest with hydrostatic density from the
    surface, rest gas; seeded fill perturbation on the interface layer."""
    dims = (nx, ny, nz)
    N = nx * ny * nz
    i = np.arange(N, dtype=np.int64)
    x = i % nx
    z = i // (nx * ny)
    inside = (x < col_x) & (z < col_z)
    phi = inside.astype(np.float64)
    params = default_params(tau=tau, g=(0.0, 0.0, -g), rule=rule)
    params.update(kw)
    if any(params["periodic"]) or col_x >= nx or col_z >= nz:
        flags = classify(dims, params["periodic"], 0, phi)
    else:
        # walled box: the column's cells on its two open faces touch gas
        flags = np.where(inside, LIQUID, GAS).astype(np.uint8)
        flags[inside & ((x == col_x - 1) | (z == col_z - 1))] = INTERFACE
    rho = np.where(inside, params["rho_G"] + 3.0 * g * (col_z - (z + 0.5)), params["rho_G"])
    ifc = flags == INTERFACE
    phi = np.where(ifc, 1.0, 0.0)
    phi[ifc] += uniform(seed, int(ifc.sum()), phi_noise, offset=19 * N)
    return Case(dims=dims, params=params, flags=flags, rho=rho, u=np.zeros((N, 3)),
                phi=phi, noise=None, wall_delta=None)


def adjoint_film(**kw) -> Case:
    """Film of the differentiation workload: 8 x 4 x 64, depth 40."""
    args = dict(nx=8, ny=4, nz=64, h=40.0)
    args.update(kw)
    return film(**args)


def plate_flow(h=8, tau=1.0, rule=0, u_wall=1e-3, magic=0.25, headroom=3, **kw) -> Case:
    """Plate-driven planar flow (Sec. 6, transient): x, y periodic, the wall at
    the bottom face moves along x with u_wall, a flat free surface h cells
    above it (interface layer z = h - 1 with fill 1, frozen), at rest at t = 0.
    (The paper puts the surface below and the wall above; the mirror image.)"""
    nx, ny, nz = 2, 2, h + headroom
    dims = (nx, ny, nz)
    N = nx * ny * nz
    z = np.arange(N) // (nx * ny)
    phi = np.where(z < h, 1.0, 0.0)
    params = default_params(tau=tau, magic=magic, rule=rule, periodic=(1, 1, 0), freeze=1,
                            wall_u=(u_wall, 0.0, 0.0))
    params.update(kw)
    flags = np.where(z < h - 1, LIQUID, np.where(z == h - 1, INTERFACE, GAS)).astype(np.uint8)
    return Case(dims=dims, params=params, flags=flags, rho=np.ones(N), u=np.zeros((N, 3)),
                phi=np.where(flags == INTERFACE, 1.0, 0.0), noise=None, wall_delta=None, h=h, u_wall=u_wall)


def plate_flow_exact(zc, t, h, nu, u_wall, terms=400):
    """Fourier series of the plate-driven flow (the paper's transient formula):
    u / u_wall = 1 - sum_k 4 (-1)^k / ((2k+1) pi) exp(-(2k+1)^2 pi^2 nu t / (4 h^2))
    cos((2k+1) pi s / (2h)), s the distance from the free surface."""
    s = h - np.asarray(zc, dtype=np.float64)
    out = np.ones_like(s)
    for k in range(terms):
        m = 2 * k + 1
        out -= 4.0 * (-1) ** k / (m * math.pi) * math.exp(-(m * math.pi) ** 2 * nu * t / (4.0 * h * h)) * \
            np.cos(m * math.pi * s / (2.0 * h))
    return u_wall * out


def couette(h=8, tau=1.1, rule=1, shear=1e-3, headroom=3, **kw) -> Case:
    """Linear Couette flow driven by a prescribed shear rate at the free surface
    (Sec. 6): x, y periodic, resting bounce-back wall at the bottom face, flat
    surface h cells above (interface layer z = h - 1, fill 1, frozen), S^b_xz =
    shear prescribed, at rest at t = 0; steady u_x = 2 shear (z + 1/2)."""
    nx, ny, nz = 2, 2, h + headroom
    dims = (nx, ny, nz)
    N = nx * ny * nz
    z = np.arange(N) // (nx * ny)
    params = default_params(tau=tau, rule=rule, periodic=(1, 1, 0), freeze=1, stress=2,
                            shear_b=(0.0, 0.0, 0.0, 0.0, shear, 0.0))
    params.update(kw)
    flags = np.where(z < h - 1, LIQUID, np.where(z == h - 1, INTERFACE, GAS)).astype(np.uint8)
    return Case(dims=dims, params=params, flags=flags, rho=np.ones(N), u=np.zeros((N, 3)),
                phi=np.where(flags == INTERFACE, 1.0, 0.0), noise=None, wall_delta=None, h=h, shear=shear)


def churn(nx=3, ny=3, nz=6, seed=SEED, u_amp=0.04, g=(2e-3, 0.0, -4e-3), tau=0.7, rule=0,
          plant=True, base=2.5, periodic=(1, 1, 0), **kw) -> Case:
    """A tiny lattice whose interface converts every few steps (pins of the
    conversion rules): x and y periodic, walls at the z faces; column heights
    between base - 1 and base + 1 cells over the footprint; seeded velocities of
    amplitude u_amp and density noise 1e-2 on the fluid cells; strong gravity.
    ``plant`` sets two diagonal neighbours of the interface layer over- and
    under-full (fill levels 1.3 and -0.3), so that the first step has a cell
    that fills next to one that empties.  The strong gravity accelerates cells
    past the library's stability guard on |u| within a few hundred steps, so
    the guard is off here (u_max = 0): these lattices test the bookkeeping,
    not the flow."""
    dims = (nx, ny, nz)
    N = nx * ny * nz
    i = np.arange(N, dtype=np.int64)
    x, y, z = i % nx, (i // nx) % ny, i // (nx * ny)
    heights = base + uniform(seed, nx * ny, 1.0)
    h = heights[x + nx * y]
    phi = np.clip(h - z, 0.0, 1.0)
    params = default_params(tau=tau, g=tuple(g), rule=rule, periodic=tuple(periodic), u_max=0.0)
    params.update(kw)
    flags = classify(dims, params["periodic"], 0, phi)
    fluid = (flags == LIQUID) | (flags == INTERFACE)
    ifc = flags == INTERFACE
    phi = np.where(ifc, np.clip(phi, 0.05, 1.0), np.where(flags == LIQUID, 1.0, 0.0))
    if plant:
        cand = np.nonzero(ifc)[0]
        for a in cand:
            ax, ay, az = a % nx, (a // nx) % ny, a // (nx * ny)
            b = ((ax + 1) % nx) + nx * (((ay + 1) % ny) + ny * az)
            if ifc[b]:
                phi[a], phi[b] = 1.3, -0.3
                break
    u = np.zeros((N, 3))
    u[fluid] = uniform(seed, 3 * int(fluid.sum()), u_amp, offset=N).reshape(-1, 3)
    rho = np.where(fluid, 1.0 + uniform(seed, N, 1e-2, offset=4 * N), params["rho_G"])
    return Case(dims=dims, params=params, flags=flags, rho=rho, u=u, phi=phi, noise=None, wall_delta=None)
