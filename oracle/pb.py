"""Poisson-Boltzmann pieces of the oracle: ionic charge, Algorithms 3 and 4.

Test infrastructure only (see the package docstring).

Ionic charge (Eqs. rhoions, ionsconcPB; with ion radii and a packing
coefficient the steric Eq. ionsconcMPB, see ion_concentrations), atomic units:
    rho_ions[phi] = gamma(r) sum_i Z_i n_i exp(-Z_i phi / kT),
with n_i the bulk number densities and gamma the ion-exclusion function, here
the cavity function gamma = (eps - 1)/(eps0 - 1) (so ions live only in the
solvent).  The exponent is capped at +EXP_CAP (reading of the overflow that
the paper does not discuss).  Its linearization at phi = 0 gives the linear
PB term of Eq. (corrPB): lambda(r) = gamma(r) * 4 pi sum_i Z_i^2 n_i / kT.

Algorithm 3 solves the full GPe with rho + rho_ions_k every outer step.
Algorithm 4 solves only for the correction phi' whose source is the previous
inner residual (as a charge) plus the change of the ionic charge, and
accumulates phi.  Both mix the ionic charge linearly with eta and stop on the
Euclidean norm of its change.

Reading: Algorithm 4 as printed (linear mixing, GPe inner operator)
diverges once the box exceeds the Debye length and the solvent potential
exceeds a few kT (the paper's own test box was 10 bohr).  The default outer
step therefore linearizes the ionic charge inside the PCG operator -- the
linear PB operator of Eq. (corrPB) with lambda taken at the current potential
-- which turns the same loop into a damped Newton iteration; the printed
algorithm remains available as mode="printed".
"""
import numpy as np

from .constants import EXP_CAP, kT, lambda0, max_number_density, number_density
from .operators import Fields
from .pcg import pcg


def exclusion_from_eps(eps, eps0):
    return (eps - 1.0) / (eps0 - 1.0)


def steric_ratios(electrolyte):
    """a_j = c_j^inf / c_j^max of Eq. (ionsconcMPB), or None for the plain
    Boltzmann distribution of Eq. (ionsconcPB) (no packing coefficient)."""
    packing = getattr(electrolyte, "packing", 0.0) or 0.0
    radii = getattr(electrolyte, "radius_angstrom", None)
    if packing <= 0.0 or radii is None:
        return None
    return [number_density(c) / max_number_density(r, packing)
            for c, r in zip(electrolyte.c_molar, radii)]


def ion_concentrations(phi, electrolyte):
    """Number densities n_i[phi] of Eq. (ionsconcPB), or of Eq. (ionsconcMPB)
    when the electrolyte has ion radii and a packing coefficient:
        n_i = n_i^inf e_i / (1 + sum_j a_j (e_j - 1)),  e_i = exp(-Z_i phi / kT).
    Reading: the paper prints the bracket as (e_j + 1); with "+ 1" the bulk
    concentration is not recovered where phi = 0, so it is read as the
    Bikerman form "- 1" (both forms give Eq. (ionsconcPB) as c_max -> inf)."""
    kt = kT(electrolyte.temperature)
    e = [np.exp(np.minimum(-z * phi / kt, EXP_CAP)) for z in electrolyte.z]
    a = steric_ratios(electrolyte)
    den = 1.0
    if a is not None:
        den = 1.0 + sum(aj * (ej - 1.0) for aj, ej in zip(a, e))
    return [number_density(c) * ei / den for c, ei in zip(electrolyte.c_molar, e)]


def ionic_charge(phi, gamma, electrolyte):
    """rho_ions[phi] = gamma sum_i Z_i n_i[phi] (Eq. rhoions)."""
    n = ion_concentrations(phi, electrolyte)
    return gamma * sum(z * ni for z, ni in zip(electrolyte.z, n))


def ionic_charge_derivative(phi, gamma, electrolyte):
    """d rho_ions / d phi (a species' exponential counts as constant where
    its cap is active)."""
    kt = kT(electrolyte.temperature)
    us = [-z * phi / kt for z in electrolyte.z]
    e = [np.exp(np.minimum(u, EXP_CAP)) for u in us]
    de = [np.where(u < EXP_CAP, -z / kt * ei, 0.0) for u, z, ei in zip(us, electrolyte.z, e)]
    num = sum(z * number_density(c) * ei for z, c, ei in zip(electrolyte.z, electrolyte.c_molar, e))
    dnum = sum(z * number_density(c) * dei for z, c, dei in zip(electrolyte.z, electrolyte.c_molar, de))
    a = steric_ratios(electrolyte)
    if a is None:
        return gamma * dnum
    den = 1.0 + sum(aj * (ej - 1.0) for aj, ej in zip(a, e))
    dden = sum(aj * dej for aj, dej in zip(a, de))
    return gamma * (dnum * den - num * dden) / (den * den)


def linear_lambda(gamma, electrolyte):
    """lambda(r) of Eq. (corrPB) with the exclusion function."""
    return gamma * lambda0(electrolyte)


def alg3(grid, rho, eps, electrolyte, eps0, eta=0.6, tol=1e-10, max_outer=200,
         inner_tol=1e-10, gamma=None):
    """Algorithm 3: full GPe solve (Algorithm 2) with rho + rho_ions_k each step."""
    gamma = exclusion_from_eps(eps, eps0) if gamma is None else gamma
    fields = Fields(grid, eps)
    rions = np.zeros_like(rho)                 # rho_ions_0
    hist = []
    phi = np.zeros_like(rho)
    for k in range(max_outer):
        phi, _ = pcg(fields, rho + rions, tol_abs=inner_tol)
        new = eta * ionic_charge(phi, gamma, electrolyte) + (1.0 - eta) * rions
        hist.append(float(np.sqrt(np.sum((new - rions) ** 2))))
        rions = new
        if hist[-1] <= tol:
            break
    return phi, {"outer": len(hist), "res": hist, "converged": hist[-1] <= tol}


def alg4(grid, rho, eps, electrolyte, eps0, mode="newton", eta=0.6, tol=1e-10,
         max_outer=100, gamma=None, max_iter=2000, loose_rel=1e-4, loose_steps=2,
         forcing=1e-2, forcing_rule="ratio", record=False):
    """Algorithm 4 with an optionally linearized inner operator.

    State after each outer step: phi, the effective ionic charge rho_ions and
    the inner solve's unresolved charge r', with the bookkeeping invariant
        A phi = -4 pi (rho + rho_ions - r')        (A = div eps grad).
    One outer step:
        fresh = rho_ions[phi]                         (Eqs. rhoions, ionsconcPB)
        mix   = eta fresh + (1 - eta) rho_ions        (Algorithm 4, mixing)
        solve (A - lambda) phi' = -4 pi (r' + mix - rho_ions) from phi' = 0
              with Algorithm 2; its final residual gives the new r''
        phi   += t phi';  rho_ions += t (mix - rho_ions - lambda phi'/4pi);
        r'    = (1-t) r' + t r''
    mode "printed": lambda = 0, t = 1 -- Algorithm 4 as printed (first two
      inner solves loose, then the outer criterion in residual units).
    mode "newton": eta = 1, lambda = -4 pi d rho_ions/d phi at phi (the
      linear PB term of Eq. corrPB at the current potential) and t halved
      until the nonlinear residual decreases; inner tolerance relative to the
      inner solve's initial residual, floored at the outer one:
        forcing_rule "ratio": eta_k = min(forcing, ||F_k|| / ||F_0||);
        forcing_rule "ew2":   Eisenstat & Walker's choice 2 (SIAM J. Sci.
          Comput. 17 (1996)), eta_0 = forcing, eta_k = 0.9 (||F_k|| /
          ||F_(k-1)||)^2, raised to 0.9 eta_(k-1)^2 when that exceeds 0.1,
          capped at forcing.
      Both leave the fixed point unchanged; they differ in how far each
      inner solve is taken.
    Outer residual: ||rho_ions[phi] - rho_ions + r'||_2 (the charge-unit
    residual of A phi + 4 pi (rho + rho_ions[phi]) = 0)."""
    gamma = exclusion_from_eps(eps, eps0) if gamma is None else gamma
    zero = np.zeros_like(rho)
    phi = zero.copy()
    rions = ionic_charge(phi, gamma, electrolyte)      # rho_ions_1 = rho_ions[phi = 0]
    rp = rho.copy()                                    # r'_0 = rho
    hist, inner, steps = [], [], []
    vac = None
    F0 = None
    F_prev = eta_prev = None
    for k in range(max_outer):
        fresh = ionic_charge(phi, gamma, electrolyte)
        F = float(np.sqrt(np.sum((fresh - rions + rp) ** 2)))
        hist.append(F)
        F0 = F if F0 is None else F0
        if F <= tol:
            break
        if mode == "printed":
            lam, e = zero, eta
        else:
            lam, e = -4.0 * np.pi * ionic_charge_derivative(phi, gamma, electrolyte), 1.0
        mix = e * fresh + (1.0 - e) * rions
        src = rp + mix - rions
        fields = Fields(grid, eps, lam=lam, vac=vac)
        vac = fields.vac
        if mode == "printed":
            if k < loose_steps:
                kw = dict(tol_abs=0.0, tol_rel=loose_rel)
            else:
                kw = dict(tol_abs=4.0 * np.pi * tol)
        else:
            if forcing_rule == "ew2" and F_prev is not None:
                eta_k = 0.9 * (F / F_prev) ** 2
                if 0.9 * eta_prev ** 2 > 0.1:
                    eta_k = max(eta_k, 0.9 * eta_prev ** 2)
                eta_k = min(eta_k, forcing)
            elif forcing_rule == "ew2":
                eta_k = forcing
            else:
                eta_k = min(forcing, F / F0)
            F_prev, eta_prev = F, eta_k
            kw = dict(tol_abs=4.0 * np.pi * tol * 0.1, tol_rel=eta_k)
        dphi, info = pcg(fields, src, max_iter=max_iter, **kw)
        inner.append(info["iters"])
        rpp = -info["r"] / (4.0 * np.pi)
        lin = mix - rions - lam * dphi / (4.0 * np.pi)
        t = 1.0
        while True:
            phit = phi + t * dphi
            rit = rions + t * lin
            rpt = (1.0 - t) * rp + t * rpp
            if mode == "printed" or t < 1e-4:
                break
            Ft = float(np.sqrt(np.sum((ionic_charge(phit, gamma, electrolyte) - rit + rpt) ** 2)))
            if Ft < F:
                break
            t *= 0.5
        steps.append(t)
        phi, rions, rp = phit, rit, rpt
    out = {"outer": len(inner), "res": hist, "inner": inner, "steps": steps,
           "converged": hist[-1] <= tol}
    if record:
        out["rions"], out["rprime"] = rions, rp
    return phi, out


def solve_nlpb(grid, rho, eps, electrolyte, eps0, mode="newton", eta=0.6, tol=1e-10,
               max_outer=100, gamma=None, **kw):
    """Nonlinear PB (Eqs. PBe, rhoions, ionsconcPB) by Algorithm 4."""
    return alg4(grid, rho, eps, electrolyte, eps0, mode=mode, eta=eta, tol=tol,
                max_outer=max_outer, gamma=gamma, **kw)
