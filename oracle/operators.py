"""Fields and operators of the PCG (oracle side).

Test infrastructure only (see the package docstring).

Sec. "Preconditioned conjugate gradient":
  * the preconditioner of Eq. (PCGdef), sqrt(eps) lap[sqrt(eps) v] = -4 pi r,
    is solved with one vacuum Poisson solve:  v = M r = s S(s r), s = eps^-1/2;
  * q = sqrt(eps) lap sqrt(eps) is computed once (Eq. corr), here with the
    order-16 Laplacian for free/surface BC and, for periodic BC, with the
    spectral Laplacian that S inverts (so that A 1 = 0 holds exactly);
  * the operator identity of Eq. (corr) [Eq. (corrPB) with the linear PB term
    lambda]:  A v = -(q + lambda) v - 4 pi r  for v = M r.
    For periodic BC the vacuum solve drops the mean of its source, so the
    exact discrete identity gains 4 pi <s r> sqrt(eps), <.> the grid mean
    (whatever value S^(0) takes, since the Laplacian annihilates k = 0).
"""
import numpy as np

from . import fd16
from .green import BC_PERIODIC, VacuumSolver


class Fields:
    """Everything that depends on eps only, computed once per solve (S1)."""

    def __init__(self, grid, eps, lam=None, vac=None):
        if np.any(eps <= 0):
            raise ValueError("eps must be positive")
        self.grid = grid
        self.vac = vac if vac is not None else VacuumSolver(grid)
        self.sqrt_eps = np.sqrt(eps)
        self.s = 1.0 / self.sqrt_eps
        if grid.bc == BC_PERIODIC:
            lap = self.vac.spectral_laplacian(self.sqrt_eps)
        else:
            lap = fd16.laplacian(self.sqrt_eps, grid)
        self.q = self.sqrt_eps * lap
        self.lam = np.zeros_like(eps) if lam is None else np.broadcast_to(lam, eps.shape).copy()
        # periodic linear PB: finite k = 0 value of the vacuum kernel (see green)
        self.k0 = 0.0
        if grid.bc == BC_PERIODIC and np.mean(self.lam) > 0:
            self.k0 = 4.0 * np.pi * float(np.mean(eps)) / float(np.mean(self.lam))

    @property
    def qlam(self):
        return self.q + self.lam

    def precondition(self, r):
        """v = P^-1 r of Eq. (PCGdef): v = s S(s r)."""
        return self.s * self.vac.apply(self.s * r, self.k0)

    def apply_A_from_v(self, v, r):
        """A v via the identity of Eq. (corr)/(corrPB), valid for v = M r."""
        Av = -self.qlam * v - 4.0 * np.pi * r
        if self.grid.bc == BC_PERIODIC:
            Av = Av + 4.0 * np.pi * np.mean(self.s * r) * self.sqrt_eps
        return Av
