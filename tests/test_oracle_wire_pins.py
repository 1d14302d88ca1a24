"""Pins of the oracle's wire boundary condition (periodic in z, free in x and y).

The vacuum solve is checked against closed forms that do not use the
kernel's formula: the 2D potential of a neutral pair of Gaussian lines
(the kz = 0 slice), the Hankel-transform quadrature of a line modulated along
z (kz != 0), and the transverse kernel against direct quadrature of the
truncated Green's function.  The dense symmetric-positive and direct-solve
pins of tests/test_oracle_pins.py include the wire BC as well.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

import synth
from oracle import green
from oracle.green import VacuumSolver


def _line_profile(g, centers, lams, sigma):
    x, y, _ = g.axes()
    Y, X = np.meshgrid(y, x, indexing="ij")
    out = np.zeros((g.ny, g.nx))
    for (cx, cy), lam in zip(centers, lams):
        out += lam / (2 * math.pi * sigma ** 2) * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * sigma ** 2))
    return X, Y, out


def _line_potential(d, sigma):
    """Potential of a unit Gaussian line charge, -2 ln d - E1(d^2 / 2 sigma^2),
    up to a constant (limit gamma - ln(2 sigma^2) at d = 0)."""
    d = np.asarray(d, dtype=float)
    with np.errstate(divide="ignore", invalid="ignore"):
        v = -2.0 * np.log(d) - special.exp1(d * d / (2 * sigma ** 2))
    return np.where(d == 0.0, np.euler_gamma - math.log(2 * sigma ** 2), v)


def test_wire_neutral_line_pair_closed_form():
    """Two opposite Gaussian lines along z (uniform in z): the kz = 0 slice of
    the kernel, against the exact 2D potential (the gauge cancels)."""
    h, sigma = 0.3, 0.8
    g = synth.Grid(48, 48, 8, h, h, 0.5, synth.BC_WIRE)
    centers, lams = [(6.2, 7.2), (8.2, 7.0)], [1.0, -1.0]
    X, Y, prof = _line_profile(g, centers, lams, sigma)
    rho = np.broadcast_to(prof[None], g.shape).copy()
    w = VacuumSolver(g).apply(rho)
    exact = sum(lam * _line_potential(np.hypot(X - cx, Y - cy), sigma) for (cx, cy), lam in zip(centers, lams))
    for k in (0, 5):
        assert np.abs(w[k] - exact).max() < 1e-11 * np.abs(exact).max()


@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
@pytest.mark.parametrize("m", [1, 3])
def test_wire_modulated_line_quadrature(m):
    """A Gaussian line modulated by cos(kz z): the potential is cos(kz z) Phi(d)
    with Phi(d) = 2 int_0^inf exp(-k^2 sigma^2 / 2) J0(k d) k / (k^2 + kz^2) dk."""
    sigma = 0.8
    g = synth.Grid(40, 40, 16, 0.3, 0.3, 0.4, synth.BC_WIRE)
    kz = 2 * math.pi * m / (g.nz * g.hz)
    c = (6.0, 6.1)
    X, Y, prof = _line_profile(g, [c], [1.0], sigma)
    z = g.axes()[2]
    rho = np.cos(kz * z)[:, None, None] * prof[None]
    w = VacuumSolver(g).apply(rho)
    rng = np.random.default_rng(11)
    for _ in range(8):
        i, j, k = rng.integers(0, g.nx), rng.integers(0, g.ny), rng.integers(0, g.nz)
        d = math.hypot(X[j, i] - c[0], Y[j, i] - c[1])
        val, _ = integrate.quad(lambda t: math.exp(-t * t * sigma * sigma / 2) * special.j0(t * d) * t / (t * t + kz * kz),
                                0.0, 14.0 / sigma, epsabs=1e-15, epsrel=1e-13, limit=400)
        assert abs(w[k, j, i] - math.cos(kz * z[k]) * 2 * val) < 1e-11


def test_wire_transverse_kernel_matches_quadrature():
    """The closed-form transform of the truncated transverse Green's function
    against direct quadrature of int_0^R g(rho) J0(k rho) 2 pi rho d rho."""
    R = 7.3
    for kz in (0.0, 0.4, 2.1):
        for k in (0.0, 0.37, 1.9, 5.5):
            if kz == 0.0:
                gf = lambda r: 2 * math.log(R / r)
            else:
                gf = lambda r, kz=kz: 2 * special.k0(kz * r)
            val, _ = integrate.quad(lambda r: gf(r) * special.j0(k * r) * 2 * math.pi * r, 0.0, R,
                                    epsabs=1e-13, epsrel=1e-12, limit=400)
            got = float(green.wire_transverse_hat(np.array([k]), kz, R)[0])
            assert abs(got - val) < 1e-9 * max(1.0, abs(val))


def test_wire_grid_rejects_large_transverse_aspect():
    g = synth.Grid(40, 8, 8, 0.3, 0.3, 0.3, synth.BC_WIRE)
    with pytest.raises(ValueError):
        green.wire_kernel_table(g)


def test_planted_mistakes_in_wire_kernel_are_caught(monkeypatch):
    """Dropping the K0 term of the kz != 0 kernel fails the quadrature pin (the
    term is of order exp(-|kz| R) and changes potentials inside the box only
    slightly); J1 in place of J0 in the kz = 0 kernel fails the line-pair pin."""
    good = green.wire_transverse_hat

    def no_k0(kperp, kz, R):
        if kz == 0.0:
            return good(kperp, kz, R)
        a, x = abs(kz) * R, np.asarray(kperp, dtype=float) * R
        return 4 * np.pi / (np.asarray(kperp) ** 2 + kz * kz) * (1.0 - a * special.j0(x) * special.k1(a))

    def j1_for_j0(kperp, kz, R):
        if kz != 0.0:
            return good(kperp, kz, R)
        kperp = np.asarray(kperp, dtype=float)
        with np.errstate(divide="ignore", invalid="ignore"):
            out = 4 * np.pi * (1.0 - special.j1(kperp * R)) / (kperp * kperp)
        return np.where(kperp == 0.0, np.pi * R * R, out)

    monkeypatch.setattr(green, "wire_transverse_hat", no_k0)
    with pytest.raises(AssertionError):
        test_wire_transverse_kernel_matches_quadrature()
    monkeypatch.setattr(green, "wire_transverse_hat", j1_for_j0)
    with pytest.raises(AssertionError):
        test_wire_neutral_line_pair_closed_form()
