"""Seeded synthetic inputs for the generalized Poisson / Poisson-Boltzmann solver.

This module builds the *inputs* of a solve -- a charge density rho and a
dielectric function eps (and, for Poisson-Boltzmann, the electrolyte) on a
uniform orthorhombic grid -- from seeded random draws.  It contains none of the
solver's arithmetic: no Green's function, no stencil, no PCG.  Both the CPU
oracle (tests, CPU baseline) and the CUDA path (tests, bench) consume these
arrays, so neither side depends on the other.

Conventions (atomic units: bohr, Hartree, e = 1):
  * grid points x_i = origin + i*h, i in [0, n); arrays have numpy shape
    (nz, ny, nx), i.e. x is the fastest index: flat = i + nx*(j + ny*k);
  * a Gaussian charge q at c with width sigma has density
    q (2 pi sigma^2)^(-3/2) exp(-|x-c|^2 / (2 sigma^2));
  * the cavity switching function is h(d0, Delta; r) = (1 + erf((r-d0)/Delta))/2
    (Sec. "Numerical results", Eq. hfunc) and the rigid cavity is
    eps = (eps0 - 1) prod_i h(d_i, Delta; |r - R_i|) + 1 (Sec. "Rigid cavity",
    Eq. RigCav).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import os

import numpy as np
from scipy.special import erf

BC_FREE, BC_PERIODIC, BC_SURFACE, BC_WIRE = 0, 1, 2, 3
BC_NAMES = {BC_FREE: "free", BC_PERIODIC: "periodic", BC_SURFACE: "surface", BC_WIRE: "wire"}
EPS_WATER = 78.36


@dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    hx: float
    hy: float
    hz: float
    bc: int
    origin: tuple = (0.0, 0.0, 0.0)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def npts(self):
        return self.nx * self.ny * self.nz

    def periodic_axes(self):
        """Axes (x, y, z order) along which the grid wraps."""
        if self.bc == BC_PERIODIC:
            return (True, True, True)
        if self.bc == BC_SURFACE:
            return (True, True, False)
        if self.bc == BC_WIRE:
            return (False, False, True)
        return (False, False, False)

    def lengths(self):
        return (self.nx * self.hx, self.ny * self.hy, self.nz * self.hz)

    def axes(self):
        ox, oy, oz = self.origin
        return (ox + self.hx * np.arange(self.nx), oy + self.hy * np.arange(self.ny),
                oz + self.hz * np.arange(self.nz))


@dataclass
class Electrolyte:
    """Mobile ion species: valences z_i and bulk concentrations c_i (mol/L);
    with effective radii R_i (angstrom) and a packing coefficient p > 0 the
    steric (modified PB) distribution applies."""
    z: tuple = (1, -1)
    c_molar: tuple = (0.1, 0.1)
    temperature: float = 300.0
    radius_angstrom: tuple = None
    packing: float = 0.0


@dataclass
class Problem:
    name: str
    grid: Grid
    rho: np.ndarray
    eps: np.ndarray
    kind: str = "gpe"              # "gpe", "lpb", "nlpb"
    electrolyte: Electrolyte | None = None
    eps0: float = EPS_WATER
    tol_abs: float = 1e-10
    charges: list = field(default_factory=list)   # (q, sigma, (cx, cy, cz))
    spheres: list = field(default_factory=list)   # (d, (cx, cy, cz))


def _axis_windows(grid: Grid, center, cutoff):
    """Per-axis index arrays and signed offsets within `cutoff` of `center`.

    Periodic axes use the minimum image; free axes are clipped to the grid."""
    out = []
    for ax, (n, h, o, per) in enumerate(zip((grid.nx, grid.ny, grid.nz),
                                           (grid.hx, grid.hy, grid.hz),
                                           grid.origin, grid.periodic_axes())):
        c = center[ax]
        if per:
            L = n * h
            span = min(n, int(np.ceil(2 * cutoff / h)) + 1)
            i0 = int(np.floor((c - o - cutoff) / h))
            idx = np.arange(i0, i0 + span)
            d = (o + idx * h) - c
            idx = np.mod(idx, n)
            d = d - L * np.round(d / L)
            if span == n:          # whole axis: offsets by minimum image
                idx = np.arange(n)
                d = (o + idx * h) - c
                d = d - L * np.round(d / L)
        else:
            i0 = max(0, int(np.floor((c - o - cutoff) / h)))
            i1 = min(n, int(np.ceil((c - o + cutoff) / h)) + 1)
            idx = np.arange(i0, i1)
            d = (o + idx * h) - c
        out.append((idx, d))
    return out


def _window(iz, iy, ix):
    """Index of a box given by per-axis index arrays: plain slices when every
    array is a contiguous ascending range (the same elements, without the
    gather and scatter of fancy indexing), else np.ix_."""
    sl = []
    for idx in (iz, iy, ix):
        if len(idx) and idx[-1] - idx[0] + 1 == len(idx) and np.all(np.diff(idx) == 1):
            sl.append(slice(int(idx[0]), int(idx[-1]) + 1))
        else:
            return np.ix_(iz, iy, ix)
    return tuple(sl)


def _gauss_profile(n, h, o, per, c, sigma, cutoff):
    """Index array and 1D Gaussian factor exp(-d^2/(2 sigma^2)) along one axis.

    Periodic axes cover the whole axis and sum every image within `cutoff`
    (the periodized Gaussian); free axes keep the window within `cutoff`."""
    if per:
        L = n * h
        idx = np.arange(n)
        x = o + idx * h
        m = int(np.ceil(cutoff / L)) + 1
        prof = np.zeros(n)
        for k in range(-m, m + 1):
            d = x - c - k * L
            prof += np.exp(-d * d / (2 * sigma * sigma))
        return idx, prof
    i0 = max(0, int(np.floor((c - o - cutoff) / h)))
    i1 = min(n, int(np.ceil((c - o + cutoff) / h)) + 1)
    idx = np.arange(i0, i1)
    d = (o + idx * h) - c
    return idx, np.exp(-d * d / (2 * sigma * sigma))


def add_gaussian(grid: Grid, field_: np.ndarray, q, sigma, center, cutoff_sigmas=10.0, zrange=None):
    """Add a normalized Gaussian charge (total q) to `field_` in place; along
    periodic axes the Gaussian is periodized (sum over images).  zrange =
    (z0, z1): only the planes z0 <= k < z1 (the same values there)."""
    prof = [_gauss_profile(n, h, o, per, center[a], sigma, cutoff_sigmas * sigma)
            for a, (n, h, o, per) in enumerate(zip((grid.nx, grid.ny, grid.nz),
                                                   (grid.hx, grid.hy, grid.hz),
                                                   grid.origin, grid.periodic_axes()))]
    (ix, gx), (iy, gy), (iz, gz) = prof
    if zrange is not None:
        keep = (iz >= zrange[0]) & (iz < zrange[1])
        iz, gz = iz[keep], gz[keep]
        if not len(iz):
            return
    norm = q * (2.0 * np.pi * sigma * sigma) ** -1.5
    field_[_window(iz, iy, ix)] += norm * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]


def switch_h(r, d0, delta):
    """Cavity switching function h(d0, Delta; r) = (1 + erf((r - d0)/Delta)) / 2."""
    return 0.5 * (1.0 + erf((r - d0) / delta))


def rigid_cavity(grid: Grid, spheres, delta, eps0=EPS_WATER):
    """eps = (eps0-1) prod_i h(d_i, Delta; |r - R_i|) + 1 on the grid."""
    prod = np.ones(grid.shape)
    for d, c in spheres:
        cutoff = d + 8.0 * delta         # h = 1 to double precision beyond
        (ix, dx), (iy, dy), (iz, dz) = _axis_windows(grid, c, cutoff)
        r = np.sqrt(dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2)
        prod[_window(iz, iy, ix)] *= switch_h(r, d, delta)
    return (eps0 - 1.0) * prod + 1.0


def planar_cavity(grid: Grid, z0, delta, eps0=EPS_WATER):
    """eps(z) = 1 + (eps0 - 1) h(z0, Delta; z): vacuum below z0, solvent above."""
    z = grid.axes()[2]
    prof = 1.0 + (eps0 - 1.0) * switch_h(z, z0, delta)
    return np.broadcast_to(prof[:, None, None], grid.shape).copy()


def _min_dist(p, others, grid: Grid):
    if not others:
        return np.inf
    o = np.asarray(others)
    d = o - np.asarray(p)[None, :]
    for ax, per in enumerate(grid.periodic_axes()):
        if per:
            L = grid.lengths()[ax]
            d[:, ax] -= L * np.round(d[:, ax] / L)
    return float(np.sqrt((d * d).sum(1)).min())


def _neutral_charges(rng, count, values):
    """Draw count-1 charges from `values` and set the last so the sum is zero;
    redraw until the last one also lies in `values`."""
    values = list(values)
    while True:
        qs = [int(v) for v in rng.choice(values, size=count - 1)]
        last = -sum(qs)
        if last in values:
            return qs + [last]


def _place(rng, grid, count, lo, hi, min_dist, max_tries=200000):
    pos = []
    tries = 0
    while len(pos) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place charges with the requested spacing")
        p = [rng.uniform(lo[a], hi[a]) for a in range(3)]
        if _min_dist(p, pos, grid) >= min_dist:
            pos.append(p)
    return pos


def gaussian_charges(grid, charges):
    """Sum of the Gaussian charges on the grid.  Large grids are filled by
    threads over slabs of z planes; every point receives the same additions
    in the same order as in a single pass, so the result does not depend on
    the number of threads."""
    rho = np.zeros(grid.shape)
    nthreads = min(os.cpu_count() or 1, 16, grid.nz)
    if grid.npts < (1 << 20) or nthreads < 2 or len(charges) < 2:
        for q, sigma, c in charges:
            add_gaussian(grid, rho, q, sigma, c)
        return rho
    from concurrent.futures import ThreadPoolExecutor
    bounds = np.linspace(0, grid.nz, nthreads + 1).astype(int)

    def slab(k):
        for q, sigma, c in charges:
            add_gaussian(grid, rho, q, sigma, c, zrange=(bounds[k], bounds[k + 1]))

    with ThreadPoolExecutor(max_workers=nthreads) as ex:
        list(ex.map(slab, range(nthreads)))
    return rho


# --------------------------------------------------------------------------
# The five workloads.  Seeds default to 1000 + workload index.
# --------------------------------------------------------------------------

def gpe_free_single(n=64, h=0.3, seed=1001):
    """Generalized Poisson, free BC: one Gaussian (q=1, sigma=1) at the grid
    centre (n/2)h, eps = 1 + (eps0-1) h(3, 0.5; r)."""
    grid = Grid(n, n, n, h, h, h, BC_FREE)
    c = (n // 2 * h,) * 3
    charges = [(1.0, 1.0, c)]
    eps = rigid_cavity(grid, [(3.0, c)], 0.5)
    return Problem("gpe_free_%d" % n, grid, gaussian_charges(grid, charges), eps,
                   charges=charges, spheres=[(3.0, c)], tol_abs=1e-10)


def gpe_periodic_cluster(n=128, h=0.3, count=20, seed=1002):
    """Generalized Poisson, periodic BC: `count` Gaussians, sigma ~ U[0.8, 1.5],
    q in {+-1, +-2} with zero sum, minimum-image spacing >= 2.5 bohr; eps from
    the product of erf spheres with d_i = 1.2 * U[2.5, 3.5], Delta = 0.5."""
    rng = np.random.default_rng(seed)
    grid = Grid(n, n, n, h, h, h, BC_PERIODIC)
    L = n * h
    pos = _place(rng, grid, count, (0, 0, 0), (L, L, L), 2.5)
    qs = _neutral_charges(rng, count, (-2, -1, 1, 2))
    sig = rng.uniform(0.8, 1.5, size=count)
    radii = 1.2 * rng.uniform(2.5, 3.5, size=count)
    charges = [(float(qs[i]), float(sig[i]), tuple(pos[i])) for i in range(count)]
    spheres = [(float(radii[i]), tuple(pos[i])) for i in range(count)]
    eps = rigid_cavity(grid, spheres, 0.5)
    return Problem("gpe_periodic_%d" % n, grid, gaussian_charges(grid, charges), eps,
                   charges=charges, spheres=spheres, tol_abs=1e-10)


def surface_slab(nxy=160, nz=256, h=0.3, count=64, kind="lpb", conc=0.1, seed=1003):
    """Surface BC (periodic x, y; free z): `count` Gaussians (q = +-1, neutral,
    sigma ~ U[0.8, 1.5]) with x, y uniform and z in U[0, 8]; grid z origin at
    -12 bohr; planar interface eps(z) = 1 + (eps0-1) h(10, 0.5; z).  1:1
    electrolyte at `conc` mol/L and 300 K."""
    rng = np.random.default_rng(seed)
    grid = Grid(nxy, nxy, nz, h, h, h, BC_SURFACE, origin=(0.0, 0.0, -12.0))
    L = nxy * h
    pos = [(rng.uniform(0, L), rng.uniform(0, L), rng.uniform(0, 8.0)) for _ in range(count)]
    qs = [1.0] * (count // 2) + [-1.0] * (count - count // 2)
    rng.shuffle(qs)
    sig = rng.uniform(0.8, 1.5, size=count)
    charges = [(float(qs[i]), float(sig[i]), tuple(pos[i])) for i in range(count)]
    eps = planar_cavity(grid, 10.0, 0.5)
    return Problem("surface_%s_%dx%dx%d" % (kind, nxy, nxy, nz), grid,
                   gaussian_charges(grid, charges), eps, kind=kind,
                   electrolyte=Electrolyte((1, -1), (conc, conc), 300.0),
                   charges=charges, tol_abs=1e-10)


def free_union(n=256, h=0.3, count=200, margin=10.0, kind="nlpb", conc=0.5, seed=1004):
    """Free BC: `count` Gaussians (config-2 charge rules) in the central cube
    leaving `margin` bohr to each face, eps from the union of erf spheres
    (d_i = 1.2 * U[2.5, 3.5], Delta = 0.5); 1:1 electrolyte at `conc` mol/L."""
    rng = np.random.default_rng(seed)
    grid = Grid(n, n, n, h, h, h, BC_FREE)
    L = n * h
    pos = _place(rng, grid, count, (margin,) * 3, (L - margin,) * 3, 2.5)
    qs = _neutral_charges(rng, count, (-2, -1, 1, 2))
    sig = rng.uniform(0.8, 1.5, size=count)
    radii = 1.2 * rng.uniform(2.5, 3.5, size=count)
    charges = [(float(qs[i]), float(sig[i]), tuple(pos[i])) for i in range(count)]
    spheres = [(float(radii[i]), tuple(pos[i])) for i in range(count)]
    eps = rigid_cavity(grid, spheres, 0.5)
    return Problem("free_%s_%d" % (kind, n), grid, gaussian_charges(grid, charges), eps,
                   kind=kind, electrolyte=Electrolyte((1, -1), (conc, conc), 300.0),
                   charges=charges, spheres=spheres, tol_abs=1e-10)


def manufactured(n=300, L=10.0, bc=BC_FREE, sigma=0.5, d0=1.7, delta=0.3, eps0=EPS_WATER):
    """The paper's GPe test (Sec. "Numerical results"): a cubic box of edge L
    with n points per side, phi a normalized Gaussian of width sigma at the
    centre, eps = 1 + (eps0 - 1) h(d0, delta; r), and rho = -(1/4 pi) div eps
    grad phi in closed form (radial functions).  The Gaussian is negligible
    at the faces (exp(-L^2 / 8 sigma^2)), so the same fields serve every BC.
    Returns the Problem with the exact potential in `phi_exact`."""
    from scipy.special import erf
    h = L / n
    grid = Grid(n, n, n, h, h, h, bc)
    c = n // 2 * h
    x = h * np.arange(n)
    r = np.sqrt((x[:, None, None] - c) ** 2 + (x[None, :, None] - c) ** 2 + (x[None, None, :] - c) ** 2)
    phi = np.exp(-r * r / (2 * sigma * sigma)) / (2 * np.pi * sigma * sigma) ** 1.5
    lap = (r * r / sigma ** 4 - 3.0 / sigma ** 2) * phi
    dphi = -(r / sigma ** 2) * phi
    eps = 1.0 + (eps0 - 1.0) * 0.5 * (1.0 + erf((r - d0) / delta))
    deps = (eps0 - 1.0) / (delta * np.sqrt(np.pi)) * np.exp(-((r - d0) / delta) ** 2)
    rho = -(eps * lap + deps * dphi) / (4.0 * np.pi)
    prob = Problem("manufactured_%s_%d" % (BC_NAMES[bc], n), grid, rho, eps, eps0=eps0, tol_abs=1e-10)
    prob.phi_exact = phi
    return prob


def wire_chain(n=32, nz=48, h=0.35, count=3, radius=2.4, conc=0.3, kind="lpb"):
    """Wire BC (periodic z, free x and y): `count` cavities of radius `radius`
    (Delta = 0.5) evenly spaced along z on the box axis, each holding a pair
    of Gaussians, q = +-1 (sigma 0.9) and -q/2 (sigma 0.8), offset from the
    centre; the cavities end well inside the free faces.  1:1 electrolyte at
    `conc` mol/L and 300 K."""
    g = Grid(n, n, nz, h, h, h, BC_WIRE)
    c = n // 2 * h
    L = nz * h
    zs = [(2 * i + 1) * L / (2 * count) for i in range(count)]
    eps = rigid_cavity(g, [(radius, (c, c, z)) for z in zs], 0.5)
    charges = []
    for i, z in enumerate(zs):
        q = 1.0 if i % 2 == 0 else -1.0
        charges += [(q, 0.9, (c - 0.6, c, z)), (-0.5 * q, 0.8, (c + 0.7, c + 0.3, z + 0.4))]
    return Problem("wire_%s_%dx%dx%d" % (kind, n, n, nz), g, gaussian_charges(g, charges), eps, kind=kind,
                   electrolyte=Electrolyte((1, -1), (conc, conc), 300.0), charges=charges,
                   spheres=[(radius, (c, c, z)) for z in zs], tol_abs=1e-10)


def serving_request(rng, edge, bc, kind, h=0.3):
    """One serving request: cubic grid of `edge` points, 2-80 charges placed
    by the periodic-cluster rules, 1:1 electrolyte with c ~ log-U[0.01, 1]
    mol/L.  On a free axis every cavity ends 3 Delta inside the faces (the
    sphere radius is clipped to 0.45 (n-1) h - 3 Delta in small boxes), so that eps
    is flat across the free boundary; the spheres fill about a third of the
    box at most, so that there is solvent around the solute."""
    delta = 0.5
    if bc == BC_SURFACE:
        grid = Grid(edge, edge, edge, h, h, h, bc, origin=(0.0, 0.0, 0.0))
    else:
        grid = Grid(edge, edge, edge, h, h, h, bc)
    L = edge * h
    span = (edge - 1) * h            # first to last grid point of a free axis
    per = grid.periodic_axes()
    dmax = 1.2 * 3.5
    if not all(per):
        dmax = min(dmax, 0.45 * span - 3.0 * delta)
    lo = [0.0, 0.0, 0.0]
    hi = [L, L, L]
    for a in range(3):
        if not per[a]:
            lo[a], hi[a] = dmax + 3.0 * delta, span - dmax - 3.0 * delta
    width = [hi[a] - lo[a] for a in range(3)]
    rmean = min(1.2 * 3.0, dmax)
    fill = int(0.35 * L ** 3 / (4.0 / 3.0 * np.pi * rmean ** 3))
    count = int(rng.integers(5, 81))
    count = max(2, min(count, fill, int(np.prod(width) / 25.0)))
    pos = _place(rng, grid, count, lo, hi, min(2.5, 0.5 * min(width)))
    qs = _neutral_charges(rng, count, (-2, -1, 1, 2))
    sig = rng.uniform(0.8, 1.5, size=count)
    radii = np.minimum(1.2 * rng.uniform(2.5, 3.5, size=count), dmax)
    charges = [(float(qs[i]), float(sig[i]), tuple(pos[i])) for i in range(count)]
    spheres = [(float(radii[i]), tuple(pos[i])) for i in range(count)]
    eps = rigid_cavity(grid, spheres, delta)
    conc = float(np.exp(rng.uniform(np.log(0.01), np.log(1.0))))
    return Problem("req_%s_%d_%s" % (BC_NAMES[bc], edge, kind), grid,
                   gaussian_charges(grid, charges), eps, kind=kind,
                   electrolyte=Electrolyte((1, -1), (conc, conc), 300.0),
                   charges=charges, spheres=spheres, tol_abs=1e-10)


def serving_stream(count=512, seed=1005, edges=(48, 64, 96, 128, 192)):
    """Request descriptors of the serving workload (drawn lazily: the grids are
    built by `serving_request`).  Returns a list of (edge, bc, kind, seed)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        edge = int(rng.choice(edges))
        bc = int(rng.integers(0, 3))
        kind = ("gpe", "lpb", "nlpb")[int(rng.integers(0, 3))]
        out.append((edge, bc, kind, seed * 100003 + i))
    return out


WORKLOADS = {
    1: gpe_free_single,
    2: gpe_periodic_cluster,
    3: surface_slab,
    4: free_union,
}


def workload(index, **kw):
    """Seeded workload `index` (1..4); keyword arguments shrink it for tests."""
    kw.setdefault("seed", 1000 + index)
    return WORKLOADS[index](**kw)
