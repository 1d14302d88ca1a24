"""Order-16 central finite differences (oracle side).

Test infrastructure only (see the package docstring).

Sec. "Numerical results" uses finite-difference filters of order 16 for the
derivatives of eps.  The Laplacian needed for q = sqrt(eps) lap sqrt(eps)
(Eq. corr) is taken here as the sum over axes of the order-16 central second
derivative (8 points on each side):

    f''(x) ~ (1/h^2) sum_{j=-8..8} c_|j| f(x + j h),
    c_j = 2 (-1)^(j+1) (8!)^2 / (j^2 (8-j)! (8+j)!),   c_0 = -2 sum_{j>=1} c_j.

Beyond a free face the field is continued by its face value (every cavity of
the method is flat there); periodic axes wrap.  The coefficients are built
from exact rationals.
"""
from fractions import Fraction
from math import factorial

import numpy as np

HALF_WIDTH = 8


def second_derivative_coeffs(m=HALF_WIDTH):
    """Exact coefficients c_0..c_m of the order-2m central second derivative."""
    c = [Fraction(0)] * (m + 1)
    for j in range(1, m + 1):
        c[j] = Fraction(2 * (-1) ** (j + 1) * factorial(m) ** 2,
                        j * j * factorial(m - j) * factorial(m + j))
    c[0] = -2 * sum(c[1:])
    return c


def first_derivative_coeffs(m=HALF_WIDTH):
    """Exact antisymmetric coefficients d_1..d_m of the order-2m central first
    derivative, f'(x) ~ (1/h) sum_j d_j (f(x+jh) - f(x-jh))."""
    return [Fraction(0)] + [Fraction((-1) ** (j + 1) * factorial(m) ** 2,
                                     j * factorial(m - j) * factorial(m + j))
                            for j in range(1, m + 1)]


def _shifted(f, axis, j, periodic):
    """f evaluated at index i + j along `axis` (numpy axis), wrapping or clamping."""
    n = f.shape[axis]
    idx = np.arange(n) + j
    idx = np.mod(idx, n) if periodic else np.clip(idx, 0, n - 1)
    return np.take(f, idx, axis=axis)


def second_derivative(f, h, axis, periodic):
    c = [float(x) for x in second_derivative_coeffs()]
    out = c[0] * f
    for j in range(1, HALF_WIDTH + 1):
        out = out + c[j] * (_shifted(f, axis, j, periodic) + _shifted(f, axis, -j, periodic))
    return out / (h * h)


def first_derivative(f, h, axis, periodic):
    d = [float(x) for x in first_derivative_coeffs()]
    out = np.zeros_like(f)
    for j in range(1, HALF_WIDTH + 1):
        out = out + d[j] * (_shifted(f, axis, j, periodic) - _shifted(f, axis, -j, periodic))
    return out / h


def laplacian(f, grid):
    """Order-16 Laplacian of f (numpy shape (nz, ny, nx)) on `grid`."""
    per = grid.periodic_axes()                       # x, y, z
    return (second_derivative(f, grid.hx, 2, per[0]) +
            second_derivative(f, grid.hy, 1, per[1]) +
            second_derivative(f, grid.hz, 0, per[2]))


def gradient(f, grid):
    per = grid.periodic_axes()
    return (first_derivative(f, grid.hx, 2, per[0]),
            first_derivative(f, grid.hy, 1, per[1]),
            first_derivative(f, grid.hz, 0, per[2]))
