"""Dense assembly of the discrete operator and direct solves (oracle side).

Test infrastructure only (see the package docstring).

The method's PCG reaches the solution of one discrete linear system.  With
D = diag(sqrt(eps)) and S the vacuum solve of the BC, the preconditioner of
Eq. (PCGdef) is M = D^-1 S D^-1 and the identity of Eq. (corr) fixes the
operator (free and surface BC, S invertible):
    A = -4 pi D S^-1 D - diag(q + lambda).
For periodic BC the vacuum solve inverts the spectral Laplacian L on
mean-free sources and A = D L D - diag(q + lambda).  Assembling these for
8^3..12^3 grids and solving with LAPACK gives the exact discrete solution the
PCG must reach.  Nonlinear PB is solved by damped Newton on
F(phi) = A phi + 4 pi (rho + rho_ions[phi]).
"""
import numpy as np

from .green import BC_PERIODIC
from .operators import Fields
from .pb import ionic_charge, ionic_charge_derivative


def columns(apply, n, shape):
    """Dense matrix of a linear map given on arrays of `shape`."""
    out = np.empty((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[j] = 1.0
        out[:, j] = apply(e.reshape(shape)).ravel()
        e[j] = 0.0
    return out


def vacuum_matrix(fields: Fields):
    g = fields.grid
    return columns(fields.vac.apply, g.npts, g.shape)


def operator_matrix(fields: Fields):
    g = fields.grid
    n = g.npts
    d = fields.sqrt_eps.ravel()
    if g.bc == BC_PERIODIC:
        L = columns(fields.vac.spectral_laplacian, n, g.shape)
        A = d[:, None] * L * d[None, :]
    else:
        S = vacuum_matrix(fields)
        A = -4.0 * np.pi * d[:, None] * np.linalg.inv(S) * d[None, :]
    A -= np.diag(fields.qlam.ravel())
    return 0.5 * (A + A.T)


def direct_solve(fields: Fields, rho):
    """phi with A phi = -4 pi rho; periodic GPe in the gauge sum sqrt(eps) phi = 0."""
    g = fields.grid
    A = operator_matrix(fields)
    b = -4.0 * np.pi * rho.ravel()
    if g.bc == BC_PERIODIC and not np.any(fields.lam):
        d = fields.sqrt_eps.ravel()
        n = g.npts
        K = np.zeros((n + 1, n + 1))
        K[:n, :n] = A
        K[:n, n] = d
        K[n, :n] = d
        rhs = np.concatenate([b - np.mean(b), [0.0]])
        return np.linalg.solve(K, rhs)[:n].reshape(g.shape)
    return np.linalg.solve(A, b).reshape(g.shape)


def newton_nlpb(fields: Fields, rho, gamma, electrolyte, tol=1e-13, max_iter=100):
    """Damped Newton for A phi + 4 pi (rho + rho_ions[phi]) = 0 (dense)."""
    g = fields.grid
    A = operator_matrix(fields)
    phi = np.zeros(g.npts)
    rho_f = rho.ravel()
    gam = gamma.ravel()

    def F(x):
        return A @ x + 4.0 * np.pi * (rho_f + ionic_charge(x, gam, electrolyte))

    f = F(phi)
    for it in range(max_iter):
        J = A + 4.0 * np.pi * np.diag(ionic_charge_derivative(phi, gam, electrolyte))
        step = np.linalg.solve(J, -f)
        t = 1.0
        nf = np.linalg.norm(f)
        while True:
            trial = phi + t * step
            ft = F(trial)
            if np.linalg.norm(ft) < (1 - 1e-4 * t) * nf or t < 1e-6:
                break
            t *= 0.5
        phi, f = trial, ft
        if np.linalg.norm(t * step) <= tol * max(1.0, np.linalg.norm(phi)):
            break
    return phi.reshape(g.shape), {"iters": it + 1, "res": float(np.linalg.norm(f))}
