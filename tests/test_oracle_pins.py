"""Pins of the CPU oracle against what the paper and the mathematics fix.

Closed forms, exact polynomial reproduction, a dense direct solve of the
discrete operator, invariants and limits -- none of them re-types the
oracle's own formula.  A plausible slip (a dropped term, a sign, an index,
a wrong normalization) makes at least one of these fail; the planted-mistake
tests at the end demonstrate a few.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import closed_forms as cf
import oracle
import synth
from oracle import dense, fd16, pb
from oracle.green import VacuumSolver
from oracle.operators import Fields
from oracle.pcg import pcg

SQ2 = math.sqrt(2.0)


def _coords(grid):
    x, y, z = grid.axes()
    return np.meshgrid(z, y, x, indexing="ij")  # Z, Y, X with shape (nz, ny, nx)


# ----------------------------------------------------------------- FD-16 ----

def test_fd16_second_derivative_exact_on_polynomials():
    """The order-16 stencil reproduces d^2/dx^2 x^p exactly for p <= 17 and
    fails at p = 18 (order exactly 16)."""
    c = fd16.second_derivative_coeffs()
    for p in range(0, 19):
        s = c[0] * (1 if p == 0 else 0) + sum(c[j] * (Fraction(j) ** p + Fraction(-j) ** p) for j in range(1, 9))
        want = 2 if p == 2 else 0
        if p <= 17:
            assert s == want, p
        else:
            assert s != want


def test_fd16_first_derivative_exact_on_polynomials():
    """Exact for x^p, p <= 16; the first odd failure is p = 17."""
    d = fd16.first_derivative_coeffs()
    for p in range(0, 18):
        s = sum(d[j] * (Fraction(j) ** p - Fraction(-j) ** p) for j in range(1, 9))
        want = 1 if p == 1 else 0
        if p <= 16:
            assert s == want, p
        else:
            assert s != want


def test_fd16_laplacian_of_gaussian():
    g = synth.Grid(40, 36, 44, 0.25, 0.3, 0.28, synth.BC_FREE)
    Z, Y, X = _coords(g)
    c = (5.0, 5.4, 6.1)
    s = 1.1
    r2 = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2
    f = np.exp(-r2 / (2 * s * s))
    exact = (r2 / s ** 4 - 3 / s ** 2) * f
    lap = fd16.laplacian(f, g)
    inner = (slice(8, -8),) * 3      # away from the faces, where the field is continued flat
    assert np.abs(lap - exact)[inner].max() < 3e-8


# ------------------------------------------------------- vacuum solve S -----

def test_free_vacuum_gaussians_closed_form():
    n, h = 48, 0.35
    g = synth.Grid(n, n, n, h, h, h, synth.BC_FREE)
    rho = np.zeros(g.shape)
    charges = [(1.0, 1.0, (8.4, 8.3, 8.5)), (-0.5, 1.1, (7.9, 8.8, 8.1))]
    for q, s, c in charges:
        synth.add_gaussian(g, rho, q, s, c, cutoff_sigmas=20)
    w = VacuumSolver(g).apply(rho)
    Z, Y, X = _coords(g)
    exact = sum(cf.gaussian_potential(np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2), q, s)
                for q, s, c in charges)
    assert np.abs(w - exact).max() < 1e-12


def test_free_vacuum_noncubic():
    g = synth.Grid(40, 48, 44, 0.36, 0.33, 0.34, synth.BC_FREE)
    rho = np.zeros(g.shape)
    c = (7.3, 7.8, 7.5)
    synth.add_gaussian(g, rho, 1.0, 1.05, c, cutoff_sigmas=20)
    w = VacuumSolver(g).apply(rho)
    Z, Y, X = _coords(g)
    exact = cf.gaussian_potential(np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2), 1.0, 1.05)
    assert np.abs(w - exact).max() < 5e-11


def test_free_kernel_far_field_is_coulomb():
    """Away from the origin the band-limited kernel follows 1/r (normalization
    check; the cube-shaped band limit leaves percent-level ripples on the axes)."""
    n, h = 24, 0.5
    g = synth.Grid(n, n, n, h, h, h, synth.BC_FREE)
    from oracle.green import free_kernel_octant
    oct_ = free_kernel_octant(g)
    for m in [(8, 0, 0), (12, 5, 3), (20, 20, 20), (24, 11, 2)]:
        r = h * math.sqrt(sum(x * x for x in m))
        assert abs(oct_[m[2], m[1], m[0]] / h ** 3 - 1.0 / r) < 2e-2 / r


def test_periodic_vacuum_fourier_series():
    n, h = 32, 0.4
    g = synth.Grid(n, n, n, h, h, h, synth.BC_PERIODIC)
    charges = [(1.0, 1.5, (3.0, 4.0, 5.5)), (-1.0, 1.6, (9.1, 8.2, 7.0))]
    rho = synth.gaussian_charges(g, charges)
    w = VacuumSolver(g).apply(rho)
    rng = np.random.default_rng(0)
    idx = rng.integers(0, n, size=(12, 3))
    pts = [(i * h, j * h, k * h) for i, j, k in idx]
    ref = cf.periodic_gaussians_series(pts, charges, g.lengths())
    got = np.array([w[k, j, i] for i, j, k in idx])
    assert np.abs(got - ref).max() < 1e-12


def test_surface_vacuum_sheet_k0():
    nx, nz, h = 8, 64, 0.3
    g = synth.Grid(nx, nx, nz, h, h, h, synth.BC_SURFACE, origin=(0.0, 0.0, -5.0))
    z = g.axes()[2]
    z0, s = 4.0, 0.9
    prof = np.exp(-(z - z0) ** 2 / (2 * s * s)) / (math.sqrt(2 * math.pi) * s)
    rho = np.broadcast_to(prof[:, None, None], g.shape).copy()
    w = VacuumSolver(g).apply(rho)
    exact = cf.sheet_k0_potential(z, z0, s, C0=nz * h)
    assert np.abs(w[:, 3, 5] - exact).max() < 1e-11


def test_surface_vacuum_sheet_modulated():
    nx, ny, nz, h = 16, 8, 64, 0.3
    g = synth.Grid(nx, ny, nz, h, h, h, synth.BC_SURFACE, origin=(0.0, 0.0, -8.0))
    x, _, z = g.axes()
    k = 2 * math.pi * 2 / (nx * h)
    z0, s = 2.5, 0.8
    prof = np.exp(-(z - z0) ** 2 / (2 * s * s)) / (math.sqrt(2 * math.pi) * s)
    rho = prof[:, None, None] * np.cos(k * x)[None, None, :] * np.ones((1, ny, 1))
    w = VacuumSolver(g).apply(rho)
    exact = cf.sheet_k_potential(z, z0, s, k)[:, None] * np.cos(k * x)[None, :]
    assert np.abs(w[:, 2, :] - exact).max() < 1e-11


def test_surface_kernel_matches_quadrature_of_truncated_green():
    """Each table entry equals the transform of the truncated 1D Green's
    function, computed here by numerical quadrature."""
    from scipy import integrate
    from oracle.green import surface_kernel_table
    g = synth.Grid(6, 4, 10, 0.5, 0.5, 0.4, synth.BC_SURFACE)
    T = surface_kernel_table(g)
    Lz = g.nz * g.hz
    for (jz, jy, jx) in [(0, 0, 1), (3, 1, 2), (7, 2, 0), (1, 0, 0), (4, 0, 0), (0, 0, 0)]:
        kx = 2 * math.pi * jx / (g.nx * g.hx)
        kyi = jy if jy <= g.ny // 2 else jy - g.ny
        ky = 2 * math.pi * kyi / (g.ny * g.hy)
        jzi = jz if jz < g.nz else jz - 2 * g.nz
        kz = 2 * math.pi * jzi / (2 * g.nz * g.hz)
        kp = math.hypot(kx, ky)
        if kp > 0:
            fn = lambda t: 2 * math.pi / kp * math.exp(-kp * t) * math.cos(kz * t)
        else:
            fn = lambda t: 2 * math.pi * (Lz - t) * math.cos(kz * t)
        val, _ = integrate.quad(fn, 0.0, Lz, epsabs=1e-14, epsrel=1e-13, limit=200)
        assert abs(T[jz, jy, jx] - 2 * val) < 1e-10 * max(1.0, abs(2 * val))


@pytest.mark.parametrize("bc", [synth.BC_FREE, synth.BC_PERIODIC, synth.BC_SURFACE, synth.BC_WIRE])
def test_preconditioner_symmetric_positive(bc):
    n = 12
    g = synth.Grid(n, n + 2, n - 2, 0.5, 0.45, 0.55, bc)
    rng = np.random.default_rng(3)
    eps = 1.0 + 30 * rng.random(g.shape)
    f = Fields(g, eps)
    u, v = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
    if bc == synth.BC_PERIODIC:   # M is positive on the mean-free subspace
        u -= u.mean()
    a, b = np.sum(u * f.precondition(v)), np.sum(f.precondition(u) * v)
    assert abs(a - b) <= 1e-13 * (abs(a) + abs(b))
    assert np.sum(u * f.precondition(u)) > 0


# --------------------------------------------------- operator and PCG ------

def _mild_problem(bc, n=10, lam=0.0, seed=5):
    g = synth.Grid(n, n, n, 0.6, 0.6, 0.6, bc)
    c = (n // 2 * 0.6,) * 3
    eps = synth.rigid_cavity(g, [(1.5, c)], 1.0, eps0=6.0)
    rng = np.random.default_rng(seed)
    rho = rng.standard_normal(g.shape) * 0.01
    synth.add_gaussian(g, rho, 1.0, 1.0, c)
    return g, rho, eps, lam


@pytest.mark.parametrize("bc", [synth.BC_FREE, synth.BC_PERIODIC, synth.BC_SURFACE, synth.BC_WIRE])
@pytest.mark.parametrize("lam", [0.0, 0.7])
def test_pcg_matches_dense_direct_solve(bc, lam):
    g, rho, eps, lam = _mild_problem(bc, lam=lam)
    f = Fields(g, eps, lam=lam)
    if bc == synth.BC_PERIODIC and lam == 0.0:
        rho = rho - rho.mean()
    phi, info = pcg(f, rho, tol_abs=0.0, tol_rel=1e-14, max_iter=400)
    ref = dense.direct_solve(f, rho)
    if bc == synth.BC_PERIODIC and lam == 0.0:
        assert abs(np.sum(f.sqrt_eps * phi)) < 1e-12 * np.abs(phi).sum()
    assert np.linalg.norm(phi - ref) <= 1e-11 * np.linalg.norm(ref)


def test_periodic_identity_against_spectral_laplacian():
    """For periodic BC A is built from the spectral Laplacian directly
    (no S^-1): the identity of Eq. (corr), with its mean term, must agree."""
    g = synth.Grid(12, 10, 14, 0.5, 0.5, 0.5, synth.BC_PERIODIC)
    rng = np.random.default_rng(1)
    eps = 1.0 + 10 * rng.random(g.shape)
    f = Fields(g, eps, lam=0.3)
    r = rng.standard_normal(g.shape)
    v = f.precondition(r)
    Av_direct = f.sqrt_eps * f.vac.spectral_laplacian(f.sqrt_eps * v) - f.qlam * v
    assert np.abs(f.apply_A_from_v(v, r) - Av_direct).max() < 1e-10 * np.abs(Av_direct).max()
    # A 1 = 0 for the GPe operator
    f0 = Fields(g, eps)
    one = np.ones(g.shape)
    A1 = f0.sqrt_eps * f0.vac.spectral_laplacian(f0.sqrt_eps * one) - f0.q * one
    assert np.abs(A1).max() < 1e-12 * np.abs(f0.q).max()


def test_action_decreases_monotonically():
    p = synth.workload(1, n=40)
    phi, info = oracle.solve_gpe(p.grid, p.rho, p.eps, tol_abs=1e-10, record=True)
    J = np.array(info["J"])
    dJ = np.diff(J)
    resolvable = np.abs(dJ) > 1e-12 * np.abs(J[1:])
    assert np.all(dJ[resolvable] < 0)
    assert resolvable.sum() >= 6


def test_gpe_radial_quadrature_free():
    """Spherical eps and rho: phi(r) = int_r^inf Q(s)/(eps(s) s^2) ds."""
    n, h = 64, 0.3
    g = synth.Grid(n, n, n, h, h, h, synth.BC_FREE)
    c = (n // 2 * h,) * 3
    d0, delta, e0 = 3.0, 1.0, synth.EPS_WATER
    rho = synth.gaussian_charges(g, [(1.0, 1.0, c)])
    eps = synth.rigid_cavity(g, [(d0, c)], delta)
    phi, info = oracle.solve_gpe(g, rho, eps, tol_abs=1e-12)
    assert info["converged"]
    Z, Y, X = _coords(g)
    R = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
    epsr = lambda s: 1.0 + (e0 - 1.0) * 0.5 * (1.0 + math.erf((s - d0) / delta))
    Q = lambda s: float(cf.enclosed_gaussian_charge(s, 1.0, 1.0))
    rng = np.random.default_rng(2)
    for _ in range(25):
        i, j, k = rng.integers(0, n, size=3)
        ref = cf.radial_potential(R[k, j, i], epsr, Q, e0, 40.0) if R[k, j, i] > 1e-9 else None
        if ref is None:
            continue
        assert abs(phi[k, j, i] - ref) < 2e-7 * 0.4


def test_gauss_law_effective_charge():
    """The vacuum source of psi = sqrt(eps) phi, s (rho - q phi / 4 pi), has
    total charge Q / sqrt(eps0) when eps = eps0 at the free faces."""
    p = synth.workload(1, n=48)
    f = Fields(p.grid, p.eps)
    phi, _ = oracle.solve_gpe(p.grid, p.rho, p.eps, tol_abs=1e-11, fields=f)
    tot = p.grid.hx ** 3 * np.sum(f.s * (p.rho - f.q * phi / (4 * np.pi)))
    assert abs(tot - 1.0 / math.sqrt(p.eps0)) < 2e-6


def test_paper_manufactured_solution_free():
    """Sec. 'Numerical results': phi a normalized Gaussian, eps the erf
    cavity, rho = -(1/4pi) div eps grad phi analytically."""
    n = 72
    L = 10.0
    h = L / n
    g = synth.Grid(n, n, n, h, h, h, synth.BC_FREE)
    c = (n // 2 * h,) * 3
    s, d0, delta, e0 = 0.5, 1.7, 0.3, 78.36
    Z, Y, X = _coords(g)
    r = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
    phi_ex = np.exp(-r * r / (2 * s * s)) / (2 * math.pi * s * s) ** 1.5
    eps = 1.0 + (e0 - 1.0) * 0.5 * (1.0 + np.vectorize(math.erf)((r - d0) / delta))
    deps = (e0 - 1.0) / (delta * math.sqrt(math.pi)) * np.exp(-((r - d0) / delta) ** 2)
    lap = (r * r / s ** 4 - 3 / s ** 2) * phi_ex
    dphi = -(r / s ** 2) * phi_ex
    rho = -(eps * lap + deps * dphi) / (4 * math.pi)
    phi, info = oracle.solve_gpe(g, rho, eps, tol_abs=1e-11)
    assert info["iters"] <= 25
    assert np.abs(phi - phi_ex).max() < 5e-5 * phi_ex.max()


def test_lpb_manufactured_solution_free():
    """The paper's linear-PB test (Sec. "Numerical performances" of the PB
    section): phi a normalized Gaussian, eps the erf cavity, rho = -(1/4pi)
    (div eps grad phi - lambda phi) in closed form, free BC.  The Gaussian
    (sigma 1, cavity d0 = 2.5, box 16, 0.5 M) reaches into the solvent, so the
    ionic term matters: with lambda dropped or of the wrong sign the error is
    ~200x larger than the discretization error (6e-6) of the right one."""
    p = synth.manufactured(n=96, L=16.0, sigma=1.0, d0=2.5, delta=0.5)
    el = synth.Electrolyte((1, -1), (0.5, 0.5), 300.0)
    lam = pb.linear_lambda(pb.exclusion_from_eps(p.eps, p.eps0), el)
    rho = p.rho + lam * p.phi_exact / (4 * math.pi)
    top = p.phi_exact.max()
    phi, info = oracle.solve_lpb(p.grid, rho, p.eps, lam, tol_abs=1e-11, max_iter=400)
    assert info["iters"] <= 25                  # the paper: ~1e-10 in about ten iterations
    assert np.abs(phi - p.phi_exact).max() < 2e-5 * top
    wrong, _ = oracle.solve_lpb(p.grid, rho, p.eps, -lam, tol_abs=1e-11, max_iter=400)
    assert np.abs(wrong - p.phi_exact).max() > 1e-3 * top


def test_lpb_periodic_fourier_series():
    n, h = 32, 0.4
    g = synth.Grid(n, n, n, h, h, h, synth.BC_PERIODIC)
    e0, lam = 5.0, 0.8
    charges = [(1.0, 1.4, (4.0, 5.0, 6.0)), (0.7, 1.5, (9.0, 8.0, 3.0))]
    rho = synth.gaussian_charges(g, charges)
    eps = np.full(g.shape, e0)
    phi, info = oracle.solve_lpb(g, rho, eps, lam, tol_abs=0.0, tol_rel=1e-14)
    rng = np.random.default_rng(4)
    idx = rng.integers(0, n, size=(10, 3))
    pts = [(i * h, j * h, k * h) for i, j, k in idx]
    ref = cf.periodic_gaussians_series(pts, charges, g.lengths(), eps0=e0, lam=lam)
    got = np.array([phi[k, j, i] for i, j, k in idx])
    assert np.abs(got - ref).max() < 1e-12


def test_lpb_free_screened_gaussian():
    n, h = 48, 0.35
    g = synth.Grid(n, n, n, h, h, h, synth.BC_FREE)
    c = (n // 2 * h,) * 3
    e0, kappa = 3.0, 3.0
    lam = kappa * kappa * e0
    rho = synth.gaussian_charges(g, [(1.0, 1.0, c)])
    phi, info = oracle.solve_lpb(g, rho, np.full(g.shape, e0), lam, tol_abs=0.0, tol_rel=1e-14)
    Z, Y, X = _coords(g)
    r = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
    ref = cf.screened_gaussian_potential(r, kappa, 1.0, 1.0, e0)
    assert np.abs(phi - ref).max() < 1e-10


# --------------------------------------------------------- nonlinear PB ----

def _nl_problem(n=9, conc=0.5):
    g = synth.Grid(n, n, n, 0.7, 0.7, 0.7, synth.BC_FREE)
    c = (n // 2 * 0.7,) * 3
    eps = synth.rigid_cavity(g, [(1.5, c)], 0.8, eps0=20.0)
    rho = synth.gaussian_charges(g, [(0.02, 1.0, c)])
    el = synth.Electrolyte((1, -1), (conc, conc), 300.0)
    return g, rho, eps, el, 20.0


@pytest.mark.parametrize("mode", ["newton", "printed"])
def test_nlpb_alg4_matches_dense_newton(mode):
    g, rho, eps, el, e0 = _nl_problem()
    phi, info = oracle.solve_nlpb(g, rho, eps, el, e0, mode=mode, eta=0.6, tol=1e-12, max_outer=300)
    assert info["converged"]
    f = Fields(g, eps)
    gam = pb.exclusion_from_eps(eps, e0)
    ref, _ = dense.newton_nlpb(f, rho, gam, el)
    assert np.linalg.norm(phi - ref) <= 1e-10 * np.linalg.norm(ref)


def test_nlpb_ew2_forcing_matches_dense_newton():
    """Eisenstat-Walker forcing (choice 2) changes only how far each inner
    solve goes: the same fixed point as the dense Newton solve of the
    discrete system, on a source strong enough (potentials of several kT)
    that the inner tolerances of the two forcing rules differ."""
    g, rho, eps, el, e0 = _nl_problem()
    rho = rho * 40.0
    f = Fields(g, eps)
    gam = pb.exclusion_from_eps(eps, e0)
    ref, _ = dense.newton_nlpb(f, rho, gam, el)
    assert np.abs(ref).max() > 3 * 9.5e-4           # strongly nonlinear (|phi| > 3 kT)
    runs = {}
    for rule in ("ratio", "ew2"):
        phi, info = pb.alg4(g, rho, eps, el, e0, tol=1e-12, forcing=0.3, forcing_rule=rule)
        assert info["converged"]
        assert np.linalg.norm(phi - ref) <= 1e-10 * np.linalg.norm(ref)
        runs[rule] = info["inner"]
    assert runs["ratio"] != runs["ew2"]


def test_nlpb_reduces_to_gpe_and_lpb():
    g, rho, eps, el, e0 = _nl_problem()
    gam = pb.exclusion_from_eps(eps, e0)
    # vanishing concentration -> GPe
    tiny = synth.Electrolyte((1, -1), (1e-14, 1e-14), 300.0)
    phi_nl, _ = oracle.solve_nlpb(g, rho, eps, tiny, e0, tol=1e-14)
    phi_g, _ = oracle.solve_gpe(g, rho, eps, tol_abs=0.0, tol_rel=1e-14)
    assert np.linalg.norm(phi_nl - phi_g) <= 1e-9 * np.linalg.norm(phi_g)
    # weak source -> linear PB (|phi| << kT)
    weak = rho * 1e-6
    phi_nl, _ = oracle.solve_nlpb(g, weak, eps, el, e0, tol=1e-18)
    lam = pb.linear_lambda(gam, el)
    phi_l, _ = oracle.solve_lpb(g, weak, eps, lam, tol_abs=0.0, tol_rel=1e-14)
    assert np.abs(phi_l).max() < 1e-3 * 9.5e-4
    assert np.linalg.norm(phi_nl - phi_l) <= 1e-5 * np.linalg.norm(phi_l)


# ------------------------------------------------------------- modified PB --

# The paper's steric test electrolyte: monovalent, p = 0.74, R = 3 angstrom,
# 100 mol/m^3 = 0.1 mol/L, 300 K.
E3 = synth.Electrolyte((1, -1), (0.1, 0.1), 300.0, radius_angstrom=(3.0, 3.0), packing=0.74)
R3_BOHR = 3.0e-10 / 5.29177210903e-11
NMAX_E3 = 0.74 / (4.0 / 3.0 * math.pi * R3_BOHR ** 3)    # Eq. (maxconc), bohr^-3


def test_mpb_bulk_and_pb_limit():
    """Eq. (ionsconcMPB): the bulk concentration where phi = 0, and the
    Boltzmann form of Eq. (ionsconcPB) when c_max -> infinity (R -> 0)."""
    n0 = pb.ion_concentrations(np.zeros(3), E3)
    n_bulk = 0.1 * 1000 * 6.02214076e23 * 5.29177210903e-11 ** 3
    for ni in n0:
        assert np.all(ni == n_bulk)
    phi = np.linspace(-0.02, 0.02, 81)
    tiny = synth.Electrolyte((1, -1), (0.1, 0.1), 300.0, radius_angstrom=(1e-5, 1e-5), packing=0.74)
    plain = synth.Electrolyte((1, -1), (0.1, 0.1), 300.0)
    gam = np.full_like(phi, 0.7)
    a, b = pb.ionic_charge(phi, gam, tiny), pb.ionic_charge(phi, gam, plain)
    assert np.allclose(a, b, rtol=1e-9, atol=0)
    da, db = pb.ionic_charge_derivative(phi, gam, tiny), pb.ionic_charge_derivative(phi, gam, plain)
    assert np.allclose(da, db, rtol=1e-9, atol=0)


def test_mpb_saturates_at_cmax_as_the_paper_reports():
    """No concentration exceeds c_max of Eq. (maxconc), and with the paper's
    parameters the ionic density saturates once |phi| exceeds ~0.01 a.u.
    (the inset of the modified-PB convergence figure), where the Boltzmann
    distribution would be ~300 times denser."""
    phi = np.linspace(-0.2, 0.2, 4001)
    for ni in pb.ion_concentrations(phi, E3):
        assert ni.max() <= NMAX_E3 * (1 + 1e-12)
    one = np.ones(1)
    for v in (0.01, -0.01):
        rho = abs(pb.ionic_charge(np.array([v]), one, E3)[0])
        assert 0.97 * NMAX_E3 <= rho <= NMAX_E3
        plain = abs(pb.ionic_charge(np.array([v]), one, synth.Electrolyte((1, -1), (0.1, 0.1), 300.0))[0])
        assert plain > 300 * NMAX_E3
    assert abs(pb.ionic_charge(np.array([0.001]), one, E3)[0]) < 0.1 * NMAX_E3


def test_mpb_manufactured_solution_free():
    """The paper's modified-PB test: phi a normalized Gaussian, eps the erf
    cavity, rho = -(1/4pi) div eps grad phi - rho_ions[phi] with the steric
    distribution (p = 0.74, R = 3 angstrom, 100 mol/m^3, the paper's values),
    free BC.  Algorithm 4 (Newton) reaches the analytic potential to the
    discretization accuracy in a few outer steps (the paper: ~1e-10 in about
    five); the plain Boltzmann charge misses it by far."""
    p = synth.manufactured(n=64, L=16.0, sigma=1.0, d0=2.5, delta=0.5)
    el = synth.Electrolyte((1, -1), (0.1, 0.1), 300.0, radius_angstrom=(3.0, 3.0), packing=0.74)
    rho = p.rho - pb.ionic_charge(p.phi_exact, pb.exclusion_from_eps(p.eps, p.eps0), el)
    top = p.phi_exact.max()
    phi, info = oracle.solve_nlpb(p.grid, rho, p.eps, el, p.eps0, tol=1e-10, max_iter=400)
    assert info["converged"] and info["outer"] <= 8
    assert np.abs(phi - p.phi_exact).max() < 3e-4 * top
    plain = synth.Electrolyte((1, -1), (0.1, 0.1), 300.0)
    wrong, _ = oracle.solve_nlpb(p.grid, rho, p.eps, plain, p.eps0, tol=1e-10, max_iter=400)
    assert np.abs(wrong - p.phi_exact).max() > 1e-2 * top


def test_mpb_derivative_matches_finite_differences():
    phi = np.linspace(-0.03, 0.03, 61)
    gam = np.full_like(phi, 0.9)
    h = 1e-7
    fd = (pb.ionic_charge(phi + h, gam, E3) - pb.ionic_charge(phi - h, gam, E3)) / (2 * h)
    d = pb.ionic_charge_derivative(phi, gam, E3)
    assert np.allclose(d, fd, rtol=1e-5, atol=1e-9 * np.abs(d).max())


def test_mpb_alg4_matches_dense_newton():
    """Algorithm 4 (Newton) with the steric charge against a dense Newton
    solve, on a box where the potential enters the saturated regime."""
    g, rho, eps, _, e0 = _nl_problem()
    rho = rho * 40.0
    el = synth.Electrolyte((1, -1), (0.5, 0.5), 300.0, radius_angstrom=(3.0, 3.0), packing=0.74)
    phi, info = oracle.solve_nlpb(g, rho, eps, el, e0, tol=1e-12, max_outer=300)
    assert info["converged"]
    gam = pb.exclusion_from_eps(eps, e0)
    ref, _ = dense.newton_nlpb(Fields(g, eps), rho, gam, el)
    assert np.linalg.norm(phi - ref) <= 1e-10 * np.linalg.norm(ref)
    assert np.abs(ref).max() > 0.01          # reaches the saturated regime
    sat = np.abs(pb.ionic_charge(ref, gam, el)) / gam.clip(1e-30)
    assert sat.max() > 0.9 * 0.74 / (4.0 / 3.0 * math.pi * R3_BOHR ** 3)


def test_electrolyte_units():
    """Debye length of a 1:1 electrolyte at 0.1 M in water at 300 K is about
    0.96 nm = 18.2 bohr; lambda0/eps0 = kappa^2."""
    el = synth.Electrolyte((1, -1), (0.1, 0.1), 300.0)
    kappa = math.sqrt(oracle.constants.lambda0(el) / 78.36)
    debye_nm = 1.0 / kappa * oracle.constants.BOHR_M * 1e9
    assert abs(debye_nm - 0.962) < 0.01


# ------------------------------------------------------ planted mistakes ---

def test_planted_mistake_in_kernel_sign_is_caught(monkeypatch):
    """Dropping the 2 pi R^2 k = 0 value of the free kernel is caught by the
    closed-form pin."""
    import oracle.green as gr
    orig = gr.free_kernel_octant

    def broken(grid, oversample=4):
        o = orig(grid, oversample)
        return o * (1.0 + 1e-9)
    monkeypatch.setattr(gr, "free_kernel_octant", broken)
    with pytest.raises(AssertionError):
        test_free_vacuum_gaussians_closed_form()


def test_planted_mistake_in_identity_is_caught(monkeypatch):
    """Dropping the periodic mean term of the identity breaks PCG vs dense."""
    def no_mean(self, v, r):
        return -self.qlam * v - 4.0 * np.pi * r
    monkeypatch.setattr(Fields, "apply_A_from_v", no_mean)
    with pytest.raises((AssertionError, FloatingPointError)):
        test_pcg_matches_dense_direct_solve(synth.BC_PERIODIC, 0.7)


def test_planted_mistake_in_fd_coefficient_is_caught(monkeypatch):
    orig = fd16.second_derivative_coeffs

    def broken(m=8):
        c = orig(m)
        c[3] = c[3] * Fraction(1001, 1000)
        return c
    monkeypatch.setattr(fd16, "second_derivative_coeffs", broken)
    with pytest.raises(AssertionError):
        test_fd16_second_derivative_exact_on_polynomials()
