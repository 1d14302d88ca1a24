"""Comparison solvers for the generalized Poisson equation, oracle side:
Algorithm 1 (self-consistent iteration, SC) and preconditioned steepest
descent (PSD, Algorithm 2 with beta = 0) with optional DIIS.

Test infrastructure only (see the package docstring).

Discretization (Sec. "Self-consistent iterative procedure", Eqs. remap and
rhoiter): the nabla of Eq. (rhoiter) is the order-16 central first
derivative (fd16.gradient; Sec. "Numerical results"), the Laplacian is the
one the vacuum solve S inverts (Eq. SPe).  With g = grad ln eps the discrete
operator of both solvers is
    A_sc phi = eps (lap_S phi + g . grad phi),
a different discretization of Eq. (GPe) from the q-identity of Algorithm 2
(Eq. corr); the two agree to discretization error.

Residual, in Algorithm 2's units: r = -4 pi rho - A_sc phi.  For periodic BC,
S drops the grid mean of its source, so the component of r along eps
(r / eps constant) is out of reach of every iteration (at the level of
discretization error the FD-16 gradient and the spectral Laplacian do not
make sum A_sc phi vanish); the residual is measured modulo it:
r -> r - eps <r / eps>.  Both solvers stop once
||r_k||_2 <= max(tol_abs, tol_rel ||r_0||_2).

Algorithm 1: rho_iter_0 = 0; for k = 0, 1, ...:
    phi_k = S(rho / eps + rho_iter_k)
    rho~ = g . grad phi_k / (4 pi)                       (Eq. rhoiter)
    residual of phi_k: r_k = -4 pi eps (rho~ - rho_iter_k)
    rho_iter_(k+1) = eta rho~ + (1 - eta) rho_iter_k      (linear mixing)
The paper's r_(k+1) = rho_iter_(k+1) - rho_iter_k is eta (rho~ - rho_iter_k):
the same vector up to the factor -4 pi eps / eta; the stopping test uses r_k
so that every method shares one residual.

PSD (Sec. "Preconditioned conjugate gradient", Eq. PrePSD): the
preconditioner solves eps lap v = r, i.e. v = S(-r / (4 pi eps)) (the -4 pi
of Eq. PrePSD absorbed in the scale of v, so that alpha = 1 is a full SC
step), and the operator acts on v through the identity
    A_sc v = r + eps g . grad v        [periodic: - eps <r / eps>]
Steps: phi += alpha v, r -= alpha A_sc v, with alpha = (v, r) / (v, A_sc v)
(steepest descent) or fixed.  With alpha_0 = 1 and alpha_k = eta after that
the iterates are those of Algorithm 1: PSD's phi_(k+1) is SC's phi_k.

DIIS (Pulay's direct inversion in the iterative subspace; the paper only
says it was integrated in the PSD loop): keep the last m triples
(phi_i, r_i, v_i = P^-1 r_i); choose c minimizing ||sum c_i v_i||_2 with
sum c_i = 1; combine phi, r, v with c (exact by linearity); take one PSD
step from the combination.  One vacuum solve per iteration; m = 1 is PSD.
"""
import numpy as np

from . import fd16
from .green import BC_PERIODIC, VacuumSolver


class ScFields:
    """eps-dependent quantities of the comparison solvers (computed once)."""

    def __init__(self, grid, eps, vac=None):
        if np.any(eps <= 0):
            raise ValueError("eps must be positive")
        self.grid = grid
        self.eps = eps
        self.vac = vac if vac is not None else VacuumSolver(grid)
        self.g = fd16.gradient(np.log(eps), grid)     # grad ln eps (Eq. rhoiter)
        self.periodic = grid.bc == BC_PERIODIC

    def g_dot_grad(self, f):
        gx, gy, gz = fd16.gradient(f, self.grid)
        return self.g[0] * gx + self.g[1] * gy + self.g[2] * gz

    def project(self, r):
        """Periodic BC: drop the component of r along eps (see the module
        docstring); other BCs: r unchanged."""
        if self.periodic:
            return r - self.eps * np.mean(r / self.eps)
        return r

    def precondition(self, r):
        """v with eps lap_S v = r (Eq. PrePSD, scaled): v = S(-r / (4 pi eps))."""
        return self.vac.apply(-r / (4.0 * np.pi * self.eps))

    def apply_A_from_v(self, v, r):
        """A_sc v for v = precondition(r)."""
        Av = r + self.eps * self.g_dot_grad(v)
        if self.periodic:
            Av = Av - self.eps * np.mean(r / self.eps)
        return Av


def _norm(x):
    return float(np.sqrt(np.sum(x * x)))


def sc(grid, rho, eps, eta=0.6, tol_abs=1e-10, tol_rel=0.0, max_iter=500, fields=None, history=False):
    """Algorithm 1.  Returns (phi_k, info): phi_k is the last potential
    solved, the one whose residual met the tolerance; info has iters (the
    number of vacuum solves), res (||r_k||, k = 0.., with r_0 the residual
    of phi = 0), converged, and phis (every phi_k) if history."""
    f = fields if fields is not None else ScFields(grid, eps)
    r0 = f.project(-4.0 * np.pi * rho)
    res = [_norm(r0)]
    tol = max(tol_abs, tol_rel * res[0])
    rho_eps = rho / eps
    rho_iter = np.zeros_like(rho)
    phi = np.zeros_like(rho)
    phis = []
    converged = res[0] <= tol
    k = 0
    while not converged and k < max_iter:
        phi = f.vac.apply(rho_eps + rho_iter)
        k += 1
        if history:
            phis.append(phi)
        rho_new = f.g_dot_grad(phi) / (4.0 * np.pi)
        r = f.project(-4.0 * np.pi * eps * (rho_new - rho_iter))
        res.append(_norm(r))
        converged = res[-1] <= tol
        rho_iter = eta * rho_new + (1.0 - eta) * rho_iter
    info = {"iters": k, "res": res, "converged": converged}
    if history:
        info["phis"] = phis
    return phi, info


def psd(grid, rho, eps, alpha=None, alpha0=None, diis=0, tol_abs=1e-10, tol_rel=0.0, max_iter=500,
        fields=None, history=False):
    """PSD (Algorithm 2 with beta = 0 and the preconditioner of Eq. PrePSD),
    with DIIS over the last `diis` iterates if diis > 1.  alpha None: the
    steepest-descent step (v, r) / (v, A v); else that fixed step (alpha0,
    if given, for the first step).  Returns (phi, info) like sc()."""
    f = fields if fields is not None else ScFields(grid, eps)
    phi = np.zeros_like(rho)
    r = f.project(-4.0 * np.pi * rho)
    v = f.precondition(r)
    res = [_norm(r)]
    tol = max(tol_abs, tol_rel * res[0])
    hist = [(phi, r, v)]
    phis = []
    converged = res[0] <= tol
    k = 0
    while not converged and k < max_iter:
        if diis > 1 and len(hist) > 1:
            c = diis_coefficients([h[2] for h in hist])
            phi = sum(ci * h[0] for ci, h in zip(c, hist))
            r = sum(ci * h[1] for ci, h in zip(c, hist))
            v = sum(ci * h[2] for ci, h in zip(c, hist))
        Av = f.apply_A_from_v(v, r)
        if alpha is None:
            vAv = float(np.sum(v * Av))
            if not np.isfinite(vAv) or vAv >= 0.0:
                raise FloatingPointError("PSD breakdown: (v, A v) = %r" % vAv)
            a = float(np.sum(v * r)) / vAv
        else:
            a = alpha0 if (k == 0 and alpha0 is not None) else alpha
        phi = phi + a * v
        r = f.project(r - a * Av)
        k += 1
        res.append(_norm(r))
        if history:
            phis.append(phi)
        converged = res[-1] <= tol
        if not converged:
            v = f.precondition(r)
            hist = (hist + [(phi, r, v)])[-max(diis, 1):]
    info = {"iters": k, "res": res, "converged": converged}
    if history:
        info["phis"] = phis
    return phi, info


def diis_coefficients(vs):
    """c minimizing ||sum_i c_i v_i||_2 subject to sum_i c_i = 1 (Pulay):
    the bordered system [[B, 1], [1^T, 0]] [c, mu] = [0, 1], B_ij = (v_i, v_j)."""
    m = len(vs)
    B = np.empty((m + 1, m + 1))
    for i in range(m):
        for j in range(m):
            B[i, j] = float(np.sum(vs[i] * vs[j]))
    B[m, :m] = 1.0
    B[:m, m] = 1.0
    B[m, m] = 0.0
    rhs = np.zeros(m + 1)
    rhs[m] = 1.0
    return np.linalg.solve(B, rhs)[:m]


def solve_sc(grid, rho, eps, method="sc", **kw):
    """Dispatch: method "sc" (Algorithm 1), "psd" (steepest descent),
    "diis" (PSD with DIIS, history kw['diis'], default 6)."""
    if method == "sc":
        return sc(grid, rho, eps, **kw)
    if method == "psd":
        return psd(grid, rho, eps, **kw)
    if method == "diis":
        kw.setdefault("diis", 6)
        return psd(grid, rho, eps, **kw)
    raise ValueError("unknown method %r" % method)
