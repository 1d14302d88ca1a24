"""Pins of the oracle's DFT-facing quantities: the sccs dielectric (Eq. sccs),
the polarization charge (Eqs. remap, rhopol), v_eps (Eq. veps) and the two
forms of the electrostatic energy.

The pins use the limits and special values of the sccs function, finite
differences for its derivative, closed forms (uniform dielectric), Gauss's
law, and the paper's manufactured test (analytic phi, eps and rho, hence
analytic rho_pol, |grad phi|^2 and energy integrals by radial quadrature).
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle
import synth
from oracle import dft

RMAX, RMIN, E0 = 5e-3, 1e-4, 78.36


def test_sccs_limits_midpoint_and_monotonicity():
    rho = np.array([1.0, RMAX * 1.0001, RMAX, RMIN, RMIN * 0.9999, 1e-9])
    eps, deps = dft.sccs_eps(rho, RMAX, RMIN, E0)
    assert np.array_equal(eps, [1.0, 1.0, 1.0, E0, E0, E0]) and not deps.any()
    mid = math.sqrt(RMAX * RMIN)              # z = pi, w = 1/2
    assert abs(dft.sccs_eps(np.array([mid]), RMAX, RMIN, E0)[0][0] - math.sqrt(E0)) < 1e-12 * E0
    q = RMAX * (RMIN / RMAX) ** 0.25          # z = pi/2, w = (pi/2 - 1)/(2 pi)
    want = E0 ** ((math.pi / 2 - 1) / (2 * math.pi))
    assert abs(dft.sccs_eps(np.array([q]), RMAX, RMIN, E0)[0][0] - want) < 1e-12 * want
    r = np.geomspace(RMIN, RMAX, 2001)
    e, d = dft.sccs_eps(r, RMAX, RMIN, E0)
    assert np.all(np.diff(e) < 0) and np.all(d[1:-1] < 0)
    # continuous at both thresholds
    e_in, _ = dft.sccs_eps(np.array([RMAX * (1 - 1e-9), RMIN * (1 + 1e-9)]), RMAX, RMIN, E0)
    assert abs(e_in[0] - 1.0) < 1e-12 and abs(e_in[1] - E0) < 1e-9


def test_sccs_derivative_matches_finite_differences():
    r = np.geomspace(RMIN * 1.05, RMAX * 0.95, 37)
    _, d = dft.sccs_eps(r, RMAX, RMIN, E0)
    hstep = r * 1e-6
    ep, _ = dft.sccs_eps(r + hstep, RMAX, RMIN, E0)
    em, _ = dft.sccs_eps(r - hstep, RMAX, RMIN, E0)
    fd = (ep - em) / (2 * hstep)
    assert np.abs(fd - d).max() < 1e-7 * np.abs(d).max()


def test_printed_sccs_form_is_discontinuous():
    """The printed middle branch eps0 exp(w) jumps at both thresholds, which is
    why the reading eps0^w is taken (the pins above fail for it)."""
    def printed(rho):
        z = 2 * math.pi * math.log(RMAX / rho) / math.log(RMAX / RMIN)
        return E0 * math.exp((z - math.sin(z)) / (2 * math.pi))
    assert abs(printed(RMAX * (1 - 1e-12)) - 1.0) > 10
    assert abs(printed(RMIN * (1 + 1e-12)) - E0) > 10


def test_polarization_charge_uniform_eps():
    """eps = e0 everywhere: grad ln eps = 0, rho_pol = -((e0 - 1)/e0) rho."""
    g = synth.Grid(20, 20, 20, 0.4, 0.4, 0.4, synth.BC_FREE)
    rng = np.random.default_rng(5)
    rho, phi = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
    e0 = 7.5
    pol = dft.polarization_charge(g, rho, np.full(g.shape, e0), phi)
    assert np.array_equal(pol, -((e0 - 1.0) / e0) * rho)


def test_polarization_charge_gauss_law():
    """Free BC, solute inside the cavity and the box: the total charge seen
    outside, sum (rho + rho_pol) h^3, is Q / eps0, to discretization error that
    falls fast with h (the cavity wall, Delta = 0.5, is resolved by more
    points): 7.7e-4 Q at h = 0.3, 3.6e-5 Q at h = 0.2 (a 14.4 bohr box)."""
    errs = []
    for n, h in ((48, 0.3), (72, 0.2)):
        p = synth.workload(1, n=n, h=h)
        phi, info = oracle.solve_gpe(p.grid, p.rho, p.eps, tol_abs=1e-11)
        dv = h ** 3
        Q = float(np.sum(p.rho)) * dv
        tot = float(np.sum(p.rho + dft.polarization_charge(p.grid, p.rho, p.eps, phi))) * dv
        errs.append(abs(tot - Q / p.eps0) / Q)
    assert errs[0] < 2e-3 and errs[1] < 1e-4 and errs[1] < errs[0] / 10


def _manufactured(n=72, L=10.0, s=0.5, d0=1.7, delta=0.3):
    """Sec. 'Numerical results': phi a normalized Gaussian (sigma 0.5), eps the
    erf cavity (d0 1.7, Delta 0.3, eps0 78.36), box 10 (the defaults); radial
    functions."""
    h = L / n
    g = synth.Grid(n, n, n, h, h, h, synth.BC_FREE)
    c = n // 2 * h
    x = h * np.arange(n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    r = np.sqrt((X - c) ** 2 + (Y - c) ** 2 + (Z - c) ** 2)

    def phi_r(r):
        return np.exp(-r * r / (2 * s * s)) / (2 * math.pi * s * s) ** 1.5

    def dphi_r(r):
        return -(r / s ** 2) * phi_r(r)

    def lap_r(r):
        return (r * r / s ** 4 - 3 / s ** 2) * phi_r(r)

    def eps_r(r):
        return 1.0 + (E0 - 1.0) * 0.5 * (1.0 + special.erf((r - d0) / delta))

    def deps_r(r):
        return (E0 - 1.0) / (delta * math.sqrt(math.pi)) * np.exp(-((r - d0) / delta) ** 2)

    def rho_r(r):
        return -(eps_r(r) * lap_r(r) + deps_r(r) * dphi_r(r)) / (4 * math.pi)

    return g, r, dict(phi=phi_r, dphi=dphi_r, lap=lap_r, eps=eps_r, deps=deps_r, rho=rho_r)


def _pol_error(**kw):
    g, r, f = _manufactured(**kw)
    pol = dft.polarization_charge(g, f["rho"](r), f["eps"](r), f["phi"](r))
    exact = ((f["eps"](r) - 1.0) * f["lap"](r) + f["deps"](r) * f["dphi"](r)) / (4 * math.pi)
    return np.abs(pol - exact).max() / np.abs(exact).max()


def test_polarization_charge_manufactured():
    """Analytic rho_pol = -lap phi / 4pi - rho = ((eps - 1) lap phi + eps' phi') / 4pi.
    With a wall the order-16 differences resolve (Delta = 0.8, 5 points) the
    error is 7e-5 of the peak; with the paper's steep wall (Delta = 0.3) it
    falls from 1e-2 (n = 72) to 4e-4 (n = 120), which is why the paper ran
    this test at n = 300."""
    assert _pol_error(n=64, L=12.0, s=0.8, d0=2.5, delta=0.8) < 2e-4
    assert _pol_error(n=120) < _pol_error(n=72) / 10


def test_v_eps_against_analytic_gradient():
    """v_eps from a smooth phi with known gradient (a Gaussian of width 1.6,
    5 grid points: the order-16 gradient is then accurate to ~1e-10) and an
    electron density spanning the sccs transition."""
    g = synth.Grid(56, 56, 56, 0.3, 0.3, 0.3, synth.BC_FREE)
    c = 28 * 0.3
    x = 0.3 * np.arange(56)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    r = np.sqrt((X - c) ** 2 + (Y - c) ** 2 + (Z - c) ** 2)
    rho_e = 0.2 * np.exp(-r * r / (2 * 1.3 ** 2))         # 0.2 at the centre, < 1e-4 beyond 5 bohr
    _, deps = dft.sccs_eps(rho_e, RMAX, RMIN, E0)
    s = 1.6
    phi = np.exp(-r * r / (2 * s * s))
    grad2 = (r / s ** 2) ** 2 * phi ** 2
    v = dft.v_eps(g, deps, phi)
    exact = -deps * grad2 / (8 * math.pi)
    assert np.abs(exact).max() > 0
    assert np.abs(v - exact).max() < 1e-8 * np.abs(exact).max()


def test_energy_forms_against_radial_quadrature():
    """E_es = 1/2 int rho phi = 1/(8 pi) int eps |grad phi|^2 for the
    manufactured test (phi decays far inside the box); both grid sums against
    the radial integral."""
    g, r, f = _manufactured(n=96)
    e1, e2 = dft.electrostatic_energy(g, f["rho"](r), f["eps"](r), f["phi"](r))
    ref, _ = integrate.quad(lambda t: 0.5 * f["rho"](t) * f["phi"](t) * 4 * math.pi * t * t, 0.0, 6.0,
                            epsabs=1e-15, epsrel=1e-13, limit=400)
    ref2, _ = integrate.quad(lambda t: f["eps"](t) * f["dphi"](t) ** 2 * t * t / 2.0, 0.0, 6.0,
                             epsabs=1e-15, epsrel=1e-13, limit=400)
    assert abs(ref - ref2) < 1e-10 * abs(ref)
    assert abs(e1 - ref) < 1e-8 * abs(ref)
    assert abs(e2 - ref) < 1e-6 * abs(ref)
