"""Algorithm 2 (preconditioned conjugate gradient), oracle side.

Test infrastructure only (see the package docstring).

Algorithm 2 (Sec. "Preconditioned conjugate gradient"), with phi_0 = 0 so
that r_0 = -4 pi rho:
    v_k = P^-1 r_k                                  (Eq. PCGdef; operators.Fields)
    p_k = v_k + beta_k p_(k-1),  beta_k = (v_k, r_k)/(v_(k-1), r_(k-1)), beta_0 = 0
    alpha_k = (v_k, r_k)/(p_k, A p_k)
    phi_(k+1) = phi_k + alpha_k p_k
    r_(k+1) = r_k - alpha_k A p_k
A p_k is obtained without any derivative: A p_k = A v_k + beta_k A p_(k-1)
with A v_k from the identity of Eq. (corr) [Eq. (corrPB) for linear PB].
Convergence is tested on the Euclidean norm of r (Sec. "Preconditioned
conjugate gradient"): stop once ||r_(k+1)||_2 <= max(tol_abs, tol_rel ||r_0||_2).

The discrete action J_k = (1/2) phi_k . (r_k + b), b = -4 pi rho, is the
quantity CG minimizes (Eq. AIntegral up to the grid measure and sign); it is
recorded for the monotonicity invariant.
"""
import numpy as np

from .green import BC_PERIODIC
from .operators import Fields


def pcg(fields: Fields, rho, tol_abs=1e-10, tol_rel=0.0, max_iter=200, record=False):
    """Solve A phi = -4 pi rho (A = div eps grad [- lambda]) from phi_0 = 0.

    Returns (phi, info); info has iters, res (||r_k||, k = 0..iters),
    converged, and J (if record)."""
    b = -4.0 * np.pi * rho
    phi = np.zeros_like(rho)
    r = b.copy()
    p = np.zeros_like(rho)
    Ap = np.zeros_like(rho)
    vr_prev = None
    res = [float(np.sqrt(np.sum(r * r)))]
    J = [0.0]
    tol = max(tol_abs, tol_rel * res[0])
    converged = res[0] <= tol
    k = 0
    while not converged and k < max_iter:
        v = fields.precondition(r)
        vr = float(np.sum(v * r))
        beta = 0.0 if vr_prev is None else vr / vr_prev
        p = v + beta * p
        Ap = fields.apply_A_from_v(v, r) + beta * Ap
        pAp = float(np.sum(p * Ap))
        if not np.isfinite(pAp) or pAp >= 0.0:
            raise FloatingPointError("PCG breakdown: (p, A p) = %r" % pAp)
        alpha = vr / pAp
        phi = phi + alpha * p
        r = r - alpha * Ap
        vr_prev = vr
        k += 1
        res.append(float(np.sqrt(np.sum(r * r))))
        if record:
            J.append(0.5 * float(np.sum(phi * (r + b))))
        converged = res[-1] <= tol
    info = {"iters": k, "res": res, "converged": converged, "r": r}
    if record:
        info["J"] = J
    return phi, info


def neutralize(rho, grid):
    """Periodic BC admits a solution only for a neutral cell (A 1 = 0): the
    grid mean of rho is removed (a uniform neutralizing background)."""
    if grid.bc == BC_PERIODIC:
        return rho - np.mean(rho), float(np.mean(rho))
    return rho, 0.0


def solve_gpe(grid, rho, eps, tol_abs=1e-10, tol_rel=0.0, max_iter=200, record=False, fields=None):
    """Generalized Poisson equation (Eq. GPe) by Algorithm 2."""
    f = fields if fields is not None else Fields(grid, eps)
    rho, _ = neutralize(rho, grid)
    return pcg(f, rho, tol_abs, tol_rel, max_iter, record)


def solve_lpb(grid, rho, eps, lam, tol_abs=1e-10, tol_rel=0.0, max_iter=200, record=False, fields=None):
    """Linear Poisson-Boltzmann (Eq. corrPB): A = div eps grad - lambda(r)."""
    f = fields if fields is not None else Fields(grid, eps, lam=lam)
    return pcg(f, rho, tol_abs, tol_rel, max_iter, record)
