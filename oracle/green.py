"""Vacuum Poisson solve w = S(sigma), i.e. lap w = -4 pi sigma (Eq. SPe), oracle side.

Test infrastructure only (see the package docstring).

The paper delegates this step to the ISF Poisson solver of BigDFT (Sec.
"Numerical results"; free, wire, surface and periodic BC in O(N log N)) and
does not print its kernel.  The oracle uses spectrally accurate kernels with a
plain definition each:

periodic  S^(k) = 4 pi / |k|^2 on the DFT wavevectors; S^(0) = 0 (the mean
          of the source is dropped) for the GPe.  For linear PB the k = 0
          value is set to 4 pi <eps>/<lambda> (the exact inverse of a uniform
          screened medium at k = 0), which keeps M nonsingular; the operator
          identity is unaffected because the Laplacian annihilates k = 0.

free      Truncated Coulomb kernel (Vico, Greengard & Ferrando, J. Comput.
          Phys. 323 (2016)): G_R(x) = 1/|x| for |x| <= R, R = box diagonal
          sqrt(sum_d (n_d h_d)^2), whose transform 8 pi sin^2(R|k|/2)/|k|^2
          (2 pi R^2 at k = 0) is sampled on a grid 4x oversampled on every
          axis.  Its inverse DFT gives the real-space kernel h^3 g_m, kept for
          |m_d| <= n_d; the aperiodic convolution sum_j h^3 g_(i-j) sigma_j is
          then done as a cyclic convolution on the 2n-padded grid.  The inverse
          DFT of the (even) oversampled table is taken as a DCT-I per axis.

surface   Periodic in x and y, free in z.  For each in-plane wavevector the
          1D Green's function (2 pi / k) exp(-k |z|) (k > 0), or 2 pi (L_z - |z|)
          (k = 0, gauge C0 = L_z), is truncated at |z| <= R = L_z = n_z h_z and
          transformed in closed form on the 2n_z-padded z grid
          (kz_j = 2 pi j / (2 n_z h_z)):
              S^ = 4 pi (1 - (-1)^j exp(-k L_z)) / (k^2 + kz_j^2),
          and S^ = 2 pi L_z^2 at k = kz = 0.

wire      Periodic in z, free in x and y.  For each z wavevector kz the 2D
          Green's function of the transverse problem, truncated at
          rho = |(x, y)| <= R = sqrt((n_x h_x)^2 + (n_y h_y)^2), has the closed-form
          transform (cylindrical truncation of Rozzi et al., Phys. Rev. B 73,
          205119 (2006)):
              kz != 0: g = 2 K0(|kz| rho),
                  S^ = 4 pi / (k^2 + kz^2) [1 + k R J1(k R) K0(|kz| R) - |kz| R J0(k R) K1(|kz| R)]
              kz = 0:  g = 2 ln(R / rho) (gauge: zero at rho = R),
                  S^ = 4 pi (1 - J0(k R)) / k^2,  pi R^2 at k = 0,
          with k = |(kx, ky)|.  As for the free kernel, S^ is sampled on a
          grid 4x oversampled in x and y, taken to real space by a DCT-I per
          axis (h_x h_y g_m, |m_d| <= n_d), and the aperiodic transverse
          convolution is done cyclically on the 2n-padded x, y grid; along z
          the source is used at its DFT wavevectors (no padding).
"""
import math

import numpy as np
import scipy.fft as sfft

BC_FREE, BC_PERIODIC, BC_SURFACE, BC_WIRE = 0, 1, 2, 3

_WORKERS = -1   # scipy.fft: use every host core


def _rfftn(a):
    return sfft.rfftn(a, workers=_WORKERS)


def _irfftn(a, shape):
    return sfft.irfftn(a, s=shape, workers=_WORKERS)


def wavevectors_periodic(n, h):
    """Angular DFT wavevectors 2 pi m / (n h), m in fftfreq order."""
    return 2.0 * np.pi * np.fft.fftfreq(n, d=h)


def free_kernel_octant(grid, oversample=4):
    """h^3 g_m for 0 <= m_d <= n_d: the real-space truncated-Coulomb kernel.

    Returns an array of shape (nz+1, ny+1, nx+1)."""
    ns = (grid.nz, grid.ny, grid.nx)
    hs = (grid.hz, grid.hy, grid.hx)
    R = math.sqrt(sum((n * h) ** 2 for n, h in zip(ns, hs)))
    Ms = [oversample * n for n in ns]
    for n, h, M in zip(ns, hs, Ms):
        if M * h < n * h + R:
            raise ValueError("box aspect ratio too large for %dx oversampling" % oversample)
    k1 = [2.0 * np.pi * np.arange(M // 2 + 1) / (M * h) for M, h in zip(Ms, hs)]
    K = np.sqrt(k1[0][:, None, None] ** 2 + k1[1][None, :, None] ** 2 + k1[2][None, None, :] ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        Ghat = 8.0 * np.pi * np.sin(0.5 * R * K) ** 2 / (K * K)
    Ghat[0, 0, 0] = 2.0 * np.pi * R * R
    y = sfft.dct(Ghat, type=1, axis=0, workers=_WORKERS)
    y = sfft.dct(y, type=1, axis=1, workers=_WORKERS)
    y = sfft.dct(y, type=1, axis=2, workers=_WORKERS)
    return y[:ns[0] + 1, :ns[1] + 1, :ns[2] + 1] / float(Ms[0] * Ms[1] * Ms[2])


def free_kernel_table(grid):
    """Transform of the 2n-periodic even extension of h^3 g (real).

    Shape (2nz, 2ny, nx+1), matching numpy's rfftn of the padded grid."""
    g = free_kernel_octant(grid)
    idx = [np.minimum(np.arange(2 * n), 2 * n - np.arange(2 * n)) for n in (grid.nz, grid.ny, grid.nx)]
    gfull = g[np.ix_(idx[0], idx[1], idx[2])]
    return _rfftn(gfull).real


def wire_transverse_hat(kperp, kz, R):
    """Transform of the truncated transverse Green's function at |kz| (see the
    module docstring); kperp an array."""
    from scipy import special
    kperp = np.asarray(kperp, dtype=float)
    if kz == 0.0:
        with np.errstate(divide="ignore", invalid="ignore"):
            out = 4.0 * np.pi * (1.0 - special.j0(kperp * R)) / (kperp * kperp)
        return np.where(kperp == 0.0, np.pi * R * R, out)
    a = abs(kz) * R
    x = kperp * R
    return 4.0 * np.pi / (kperp * kperp + kz * kz) * (
        1.0 + x * special.j1(x) * special.k0(a) - a * special.j0(x) * special.k1(a))


def wire_kernel_table(grid, oversample=4):
    """Wire kernel on the rfftn layout (nz, 2ny, nx+1) of the grid padded to
    (nz, 2ny, 2nx)."""
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    hx, hy, hz = grid.hx, grid.hy, grid.hz
    R = math.sqrt((nx * hx) ** 2 + (ny * hy) ** 2)
    Mx, My = oversample * nx, oversample * ny
    for n, h, M in ((nx, hx, Mx), (ny, hy, My)):
        if M * h < n * h + R:
            raise ValueError("box aspect ratio too large for %dx oversampling" % oversample)
    kx = 2.0 * np.pi * np.arange(Mx // 2 + 1) / (Mx * hx)
    ky = 2.0 * np.pi * np.arange(My // 2 + 1) / (My * hy)
    kperp = np.sqrt(ky[:, None] ** 2 + kx[None, :] ** 2)
    kz = 2.0 * np.pi * np.fft.fftfreq(nz, d=hz)
    idx = [np.minimum(np.arange(2 * n), 2 * n - np.arange(2 * n)) for n in (ny, nx)]
    T = np.empty((nz, 2 * ny, nx + 1))
    cache = {}
    for j in range(nz):
        key = abs(int(round(np.fft.fftfreq(nz)[j] * nz)))
        if key not in cache:
            Ghat = wire_transverse_hat(kperp, abs(kz[j]), R)
            y = sfft.dct(Ghat, type=1, axis=0, workers=_WORKERS)
            y = sfft.dct(y, type=1, axis=1, workers=_WORKERS)
            g = y[:ny + 1, :nx + 1] / float(Mx * My)          # h_x h_y g_m
            cache[key] = sfft.rfft2(g[np.ix_(idx[0], idx[1])], workers=_WORKERS).real
        T[j] = cache[key]
    return T


def periodic_kernel_table(grid):
    """4 pi / |k|^2 (0 at k = 0) on the rfftn layout (nz, ny, nx//2+1)."""
    kx = 2.0 * np.pi * np.fft.rfftfreq(grid.nx, d=grid.hx)
    ky = wavevectors_periodic(grid.ny, grid.hy)
    kz = wavevectors_periodic(grid.nz, grid.hz)
    K2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    with np.errstate(divide="ignore"):
        T = 4.0 * np.pi / K2
    T[0, 0, 0] = 0.0
    return T, K2


def surface_kernel_table(grid):
    """Surface kernel on the rfftn layout (2nz, ny, nx//2+1)."""
    kx = 2.0 * np.pi * np.fft.rfftfreq(grid.nx, d=grid.hx)
    ky = wavevectors_periodic(grid.ny, grid.hy)
    j = np.rint(np.fft.fftfreq(2 * grid.nz) * 2 * grid.nz).astype(np.int64)
    kz = 2.0 * np.pi * j / (2 * grid.nz * grid.hz)
    Lz = grid.nz * grid.hz
    kpar = np.sqrt(ky[:, None] ** 2 + kx[None, :] ** 2)[None, :, :]
    sign = np.where(j % 2 == 0, 1.0, -1.0)[:, None, None]
    denom = kpar ** 2 + kz[:, None, None] ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        T = 4.0 * np.pi * (1.0 - sign * np.exp(-kpar * Lz)) / denom
    T[0, 0, 0] = 2.0 * np.pi * Lz * Lz
    return T


class VacuumSolver:
    """w = S(sigma) for one grid and BC (Eq. SPe: lap w = -4 pi sigma)."""

    def __init__(self, grid):
        self.grid = grid
        self.bc = grid.bc
        n = (grid.nz, grid.ny, grid.nx)
        if self.bc == BC_PERIODIC:
            self.table, self.K2 = periodic_kernel_table(grid)
            self.pshape = n
        elif self.bc == BC_FREE:
            self.table = free_kernel_table(grid)
            self.pshape = (2 * n[0], 2 * n[1], 2 * n[2])
        elif self.bc == BC_SURFACE:
            self.table = surface_kernel_table(grid)
            self.pshape = (2 * n[0], n[1], n[2])
        elif self.bc == BC_WIRE:
            self.table = wire_kernel_table(grid)
            self.pshape = (n[0], 2 * n[1], 2 * n[2])
        else:
            raise ValueError("unknown boundary condition %r" % self.bc)

    def apply(self, sigma, k0_value=0.0):
        """S sigma; `k0_value` replaces S^(0) for periodic BC."""
        g = self.grid
        if self.bc == BC_PERIODIC:
            sh = self.table * _rfftn(sigma)
            if k0_value:
                sh[0, 0, 0] = k0_value * _rfftn(sigma)[0, 0, 0]
            return _irfftn(sh, self.pshape)
        pad = np.zeros(self.pshape)
        pad[:g.nz, :g.ny, :g.nx] = sigma
        w = _irfftn(self.table * _rfftn(pad), self.pshape)
        return np.ascontiguousarray(w[:g.nz, :g.ny, :g.nx])

    def spectral_laplacian(self, f):
        """-|k|^2 multiplier on the periodic grid (periodic BC only): the
        Laplacian that S inverts, lap S sigma = -4 pi (sigma - mean sigma)."""
        if self.bc != BC_PERIODIC:
            raise ValueError("spectral Laplacian is defined for periodic BC only")
        return _irfftn(-self.K2 * _rfftn(f), self.pshape)
