"""Closed-form potentials that pin the oracle (no solver code here).

Each is an exact solution of a continuous problem whose discrete counterpart
the method solves spectrally accurately:
  * Gaussian charge in vacuum / uniform eps0:  phi = q erf(r / (sqrt2 sigma)) / (eps0 r)
  * screened Gaussian (uniform eps0, uniform lambda; linear PB, Eq. corrPB):
        phi = q/(eps0 r) * 1/2 e^(k^2 s^2/2) [e^(-k r) erfc((k s^2 - r)/(sqrt2 s))
                                             - e^(k r) erfc((k s^2 + r)/(sqrt2 s))],
    k = sqrt(lambda/eps0)
  * Gaussian sheets for the surface BC (1D Green's functions 2 pi (C0 - |z|)
    and (2 pi / k) e^(-k |z|))
  * spherically symmetric eps and rho:  phi(r) = int_r^inf Q(s) / (eps(s) s^2) ds
  * Fourier series of periodized Gaussians on a periodic cell.
"""
import math

import numpy as np
from scipy import integrate
from scipy.special import erf, erfc, erfcx

SQRT2 = math.sqrt(2.0)


def gaussian_potential(r, q=1.0, sigma=1.0, eps0=1.0):
    r = np.asarray(r, dtype=float)
    out = np.empty_like(r)
    small = r < 1e-8
    out[~small] = q * erf(r[~small] / (SQRT2 * sigma)) / (eps0 * r[~small])
    out[small] = q * math.sqrt(2.0 / math.pi) / (sigma * eps0)
    return out


def screened_gaussian_potential(r, kappa, q=1.0, sigma=1.0, eps0=1.0):
    """Potential of a Gaussian charge in a uniform screening medium.

    Uses erfcx to stay finite: e^(a^2) erfc(a) = erfcx(a)."""
    r = np.asarray(r, dtype=float)
    s = sigma
    a1 = (kappa * s * s - r) / (SQRT2 * s)
    a2 = (kappa * s * s + r) / (SQRT2 * s)
    # 1/2 e^(k^2 s^2 / 2) e^(-k r) erfc(a1) = 1/2 e^(-r^2 / (2 s^2)) erfcx(a1) when a1 >= 0
    ex = -r * r / (2 * s * s)
    t1 = np.where(a1 >= 0, 0.5 * np.exp(ex) * erfcx(np.maximum(a1, 0)),
                  0.5 * np.exp(0.5 * kappa ** 2 * s ** 2 - kappa * r) * erfc(a1))
    t2 = 0.5 * np.exp(ex) * erfcx(a2)
    with np.errstate(invalid="ignore", divide="ignore"):
        out = q * (t1 - t2) / (eps0 * r)
    # r -> 0 limit: derivative of the bracket
    small = r < 1e-6
    if np.any(small):
        lim = q / eps0 * (math.sqrt(2.0 / math.pi) / s - kappa * erfcx(kappa * s / SQRT2))
        out = np.where(small, lim, out)
    return out


def sheet_k0_potential(z, z0, sigma, C0, areal_charge=1.0):
    """lap w = -4 pi sigma_A g(z - z0), g a unit Gaussian in z, with the 1D
    Green's function 2 pi (C0 - |z|):  w = 2 pi sigma_A (C0 - E|z - z'|)."""
    d = np.asarray(z) - z0
    mean_abs = d * erf(d / (SQRT2 * sigma)) + sigma * math.sqrt(2.0 / math.pi) * np.exp(-d * d / (2 * sigma ** 2))
    return 2.0 * math.pi * areal_charge * (C0 - mean_abs)


def sheet_k_potential(z, z0, sigma, k):
    """Profile f(z) of w = cos(k x) f(z) for the source cos(k x) g(z - z0):
    f = (2 pi / k) E[e^(-k |z - z'|)]."""
    d = np.asarray(z) - z0
    s = sigma
    ex = -d * d / (2 * s * s)
    t1 = 0.5 * np.exp(ex) * erfcx((k * s * s - d) / (SQRT2 * s))
    t2 = 0.5 * np.exp(ex) * erfcx((k * s * s + d) / (SQRT2 * s))
    return 2.0 * math.pi / k * (t1 + t2)


def enclosed_gaussian_charge(s, q=1.0, sigma=1.0):
    x = s / sigma
    return q * (erf(x / SQRT2) - math.sqrt(2.0 / math.pi) * x * np.exp(-x * x / 2))


def radial_potential(r, eps_of_r, Qfun, eps_inf, r_max):
    """phi(r) = int_r^inf Q(s)/(eps(s) s^2) ds, with Q and eps constant
    beyond r_max (tail q_tot / (eps_inf r_max))."""
    q_tot = Qfun(r_max)
    tail = q_tot / (eps_inf * r_max)
    val, _ = integrate.quad(lambda s: Qfun(s) / (eps_of_r(s) * s * s), r, r_max,
                            epsabs=1e-15, epsrel=1e-13, limit=400)
    return val + tail


def periodic_gaussians_series(points, charges, lengths, kmax_sigma=9.0, eps0=1.0, lam=0.0):
    """Sum over reciprocal-lattice vectors of 4 pi rho^(k) / (eps0 k^2 + lam)
    e^(i k.x) for periodized Gaussians (k = 0 dropped when lam = 0).

    points: (m, 3) xyz; charges: [(q, sigma, (cx, cy, cz))]."""
    Lx, Ly, Lz = lengths
    smin = min(c[1] for c in charges)
    kmax = kmax_sigma / smin
    mx = int(kmax * Lx / (2 * math.pi)) + 1
    my = int(kmax * Ly / (2 * math.pi)) + 1
    mz = int(kmax * Lz / (2 * math.pi)) + 1
    kx = 2 * math.pi * np.arange(-mx, mx + 1) / Lx
    ky = 2 * math.pi * np.arange(-my, my + 1) / Ly
    kz = 2 * math.pi * np.arange(-mz, mz + 1) / Lz
    KX, KY, KZ = np.meshgrid(kx, ky, kz, indexing="ij")
    KX, KY, KZ = KX.ravel(), KY.ravel(), KZ.ravel()
    K2 = KX ** 2 + KY ** 2 + KZ ** 2
    keep = K2 <= kmax * kmax
    if lam == 0.0:
        keep &= K2 > 0
    KX, KY, KZ, K2 = KX[keep], KY[keep], KZ[keep], K2[keep]
    V = Lx * Ly * Lz
    rhohat = np.zeros(K2.shape, dtype=complex)
    for q, s, c in charges:
        rhohat += q * np.exp(-0.5 * K2 * s * s) * np.exp(-1j * (KX * c[0] + KY * c[1] + KZ * c[2])) / V
    coef = 4 * math.pi * rhohat / (eps0 * K2 + lam)
    pts = np.asarray(points)
    out = np.empty(len(pts))
    for i, (x, y, z) in enumerate(pts):
        out[i] = np.real(np.sum(coef * np.exp(1j * (KX * x + KY * y + KZ * z))))
    return out
