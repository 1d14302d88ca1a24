"""DFT-facing quantities around the generalized Poisson solve, oracle side:
the charge-dependent (sccs) dielectric, the polarization charge, the
Kohn-Sham potential correction v_eps and the electrostatic energy.

Test infrastructure only (see the package docstring).

sccs cavity (Sec. "Charge-dependent cavity", Eq. sccs): eps = 1 where
rho_elec > rho_max, eps0 where rho_elec < rho_min, and in between
    eps = eps0^w = exp(w ln eps0),  w = (z - sin z) / (2 pi),
    z = 2 pi ln(rho_max / rho) / ln(rho_max / rho_min).
Reading: the paper prints the middle branch as eps0 exp(w); that form is 1 at
neither threshold (eps0 at rho_max, eps0 e at rho_min), while eps0^w is
continuous with both outer branches (w = 0 at rho_max, 1 at rho_min) and is
the sccs function of the work the paper cites.  Its derivative is
    d eps / d rho = -eps ln(eps0) (1 - cos z) / (rho ln(rho_max / rho_min))
inside the transition and 0 outside (the one-sided derivatives vanish at
both thresholds).

Polarization charge (Eqs. remap, rhopol): rho_pol = rho_iter - ((eps-1)/eps) rho
with rho_iter = grad ln eps . grad phi / 4 pi (order-16 central differences).
Reading: the paper prints "+ ((eps-1)/eps) rho"; Eq. (remap) requires "-".

v_eps (Eq. veps) = -(1/8 pi) (d eps / d rho_elec) |grad phi|^2, the gradient by
order-16 central differences.

Electrostatic energy (Sec. "Charge-dependent cavity"): E_es = (1/2) int rho
phi = (1/8 pi) int eps |grad phi|^2; both forms as grid sums (h^3 per point),
equal up to discretization error for a converged phi with no flux through
the box faces.
"""
import math

import numpy as np

from . import fd16


def sccs_eps(rho_elec, rho_max=5e-3, rho_min=1e-4, eps0=78.36):
    """(eps, d eps / d rho) of Eq. (sccs) (reading in the module docstring)."""
    rho_elec = np.asarray(rho_elec, dtype=float)
    lnr = math.log(rho_max / rho_min)
    lne = math.log(eps0)
    mid = (rho_elec > rho_min) & (rho_elec < rho_max)
    safe = np.where(mid, rho_elec, rho_max)
    z = 2.0 * np.pi * np.log(rho_max / safe) / lnr
    w = (z - np.sin(z)) / (2.0 * np.pi)
    eps_mid = np.exp(w * lne)
    eps = np.where(rho_elec >= rho_max, 1.0, np.where(rho_elec <= rho_min, eps0, eps_mid))
    deps = np.where(mid, -eps_mid * lne * (1.0 - np.cos(z)) / (safe * lnr), 0.0)
    return eps, deps


def grad_dot(a, b, grid):
    """grad a . grad b, order-16 central differences."""
    ga = fd16.gradient(a, grid)
    gb = fd16.gradient(b, grid)
    return ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2]


def polarization_charge(grid, rho, eps, phi):
    """rho_pol = grad ln eps . grad phi / 4 pi - ((eps - 1)/eps) rho."""
    return grad_dot(np.log(eps), phi, grid) / (4.0 * np.pi) - (eps - 1.0) / eps * rho


def v_eps(grid, deps, phi):
    """-(1/8 pi) (d eps / d rho_elec) |grad phi|^2 (Eq. veps)."""
    return -deps * grad_dot(phi, phi, grid) / (8.0 * np.pi)


def electrostatic_energy(grid, rho, eps, phi):
    """(1/2 sum rho phi h^3, 1/(8 pi) sum eps |grad phi|^2 h^3)."""
    dv = grid.hx * grid.hy * grid.hz
    return (0.5 * float(np.sum(rho * phi)) * dv,
            float(np.sum(eps * grad_dot(phi, phi, grid))) * dv / (8.0 * np.pi))
