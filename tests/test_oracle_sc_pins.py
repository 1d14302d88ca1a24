"""Pins of the oracle's comparison solvers (Algorithm 1, PSD, PSD + DIIS).

Each pin rests on something other than the iteration itself: a dense direct
solve of the discrete equations (Eqs. remap, rhoiter), the closed form of a
Gaussian in a uniform dielectric, the analytic potential of the paper's
manufactured test, the SC <-> PSD equivalence the paper states, and brute
force for the DIIS coefficients.  A planted sign error in the polarization
term is caught.
"""
import math

import numpy as np
import pytest

import closed_forms as cf
import oracle
import synth
from oracle import sc as S


def _coords(grid):
    x, y, z = grid.axes()
    return np.meshgrid(z, y, x, indexing="ij")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _small_cavity(bc, n=10, h=0.6):
    g = synth.Grid(n, n, n, h, h, h, bc)
    c = (n // 2 * h,) * 3
    eps = synth.rigid_cavity(g, [(1.6, c)], 0.6, eps0=10.0)
    rho = synth.gaussian_charges(g, [(1.0, 0.9, (c[0] - 0.4, c[1], c[2])), (-0.6, 0.8, (c[0] + 0.6, c[1], c[2]))])
    return g, rho, eps


def _manufactured(n=48):
    """The paper's GPe test (Sec. 'Numerical results'): phi a normalized
    Gaussian (sigma 0.5), eps the erf cavity (d0 1.7, Delta 0.3, eps0
    78.36) in a box of edge 10, rho = -(1/4pi) div eps grad phi analytically."""
    L = 10.0
    h = L / n
    g = synth.Grid(n, n, n, h, h, h, synth.BC_FREE)
    c = (n // 2 * h,) * 3
    s, d0, delta, e0 = 0.5, 1.7, 0.3, 78.36
    Z, Y, X = _coords(g)
    r = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
    phi_ex = np.exp(-r * r / (2 * s * s)) / (2 * math.pi * s * s) ** 1.5
    erf = np.vectorize(math.erf)
    eps = 1.0 + (e0 - 1.0) * 0.5 * (1.0 + erf((r - d0) / delta))
    deps = (e0 - 1.0) / (delta * math.sqrt(math.pi)) * np.exp(-((r - d0) / delta) ** 2)
    lap = (r * r / s ** 4 - 3 / s ** 2) * phi_ex
    dphi = -(r / s ** 2) * phi_ex
    rho = -(eps * lap + deps * dphi) / (4 * math.pi)
    return g, rho, eps, phi_ex


@pytest.mark.parametrize("bc", [synth.BC_FREE, synth.BC_SURFACE])
def test_sc_and_diis_reach_the_dense_solution(bc):
    """The fixed point of Algorithm 1 solves phi = S(rho/eps + g.grad phi/4pi)
    (Eqs. remap, rhoiter): assembled densely on a 10^3 grid and solved
    directly, it equals converged SC, PSD + DIIS and fixed-step PSD."""
    g, rho, eps = _small_cavity(bc)
    f = S.ScFields(g, eps)
    n = rho.size
    Smat = np.empty((n, n))
    Gmat = np.empty((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[j] = 1.0
        u = e.reshape(rho.shape)
        Smat[:, j] = f.vac.apply(u).ravel()
        Gmat[:, j] = f.g_dot_grad(u).ravel()
        e[j] = 0.0
    M = np.eye(n) - Smat @ Gmat / (4 * math.pi)
    ref = np.linalg.solve(M, Smat @ (rho / eps).ravel()).reshape(rho.shape)
    phi_sc, i1 = S.sc(g, rho, eps, eta=0.6, tol_abs=0.0, tol_rel=1e-14, max_iter=400, fields=f)
    phi_di, i2 = S.psd(g, rho, eps, diis=5, tol_abs=0.0, tol_rel=1e-14, max_iter=400, fields=f)
    phi_fx, i3 = S.psd(g, rho, eps, alpha=0.6, tol_abs=0.0, tol_rel=1e-14, max_iter=400, fields=f)
    assert i1["converged"] and i2["converged"] and i3["converged"]
    assert _rel(phi_sc, ref) < 1e-11
    assert _rel(phi_di, ref) < 1e-11
    assert _rel(phi_fx, ref) < 1e-11
    assert i2["iters"] < i1["iters"]          # DIIS lowers the iteration count


@pytest.mark.parametrize("bc", [synth.BC_FREE, synth.BC_PERIODIC])
def test_sc_is_psd_with_alpha_eta(bc):
    """Sec. 'Preconditioned conjugate gradient': PSD with alpha = 1 is the SC
    procedure; with mixing eta, SC's phi_k is PSD's phi_(k+1) for steps
    alpha_0 = 1, alpha_k = eta."""
    g, rho, eps = _small_cavity(bc, n=12, h=0.55)
    if bc == synth.BC_PERIODIC:
        rho = rho - rho.mean()
    f = S.ScFields(g, eps)
    _, i_sc = S.sc(g, rho, eps, eta=0.6, tol_abs=0.0, max_iter=10, fields=f, history=True)
    _, i_pd = S.psd(g, rho, eps, alpha=0.6, alpha0=1.0, tol_abs=0.0, max_iter=10, fields=f, history=True)
    for k in range(10):     # psd's phis[k] is phi after step k + 1
        assert _rel(i_pd["phis"][k], i_sc["phis"][k]) < 1e-12


def test_uniform_eps_single_step_is_the_gaussian_potential():
    """eps = e0 everywhere: grad ln eps = 0, so SC ends after one vacuum
    solve and PSD after one step of length 1, both at the closed-form
    potential of a Gaussian in a dielectric e0 (free BC)."""
    n, h, e0 = 40, 0.35, 4.0
    g = synth.Grid(n, n, n, h, h, h, synth.BC_FREE)
    c = (n // 2 * h,) * 3
    rho = synth.gaussian_charges(g, [(1.0, 1.0, c)])
    eps = np.full(g.shape, e0)
    phi_sc, i1 = S.sc(g, rho, eps, tol_abs=1e-9)
    phi_pd, i2 = S.psd(g, rho, eps, tol_abs=1e-9)
    assert i1["iters"] == 1 and i2["iters"] == 1
    Z, Y, X = _coords(g)
    r = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
    ref = cf.gaussian_potential(r, 1.0, 1.0, e0)
    assert np.abs(phi_sc - ref).max() < 1e-10
    assert np.abs(phi_pd - ref).max() < 1e-10


def test_paper_manufactured_solution_sc_psd_diis():
    """The paper's GPe test: SC (eta = 0.6) and PSD + DIIS reach the analytic
    potential to the order-16 discretization's accuracy, agree with the
    Algorithm-2 solution to that accuracy, and DIIS needs fewer iterations
    than SC (Sec. 'Numerical results')."""
    g, rho, eps, phi_ex = _manufactured()
    f = S.ScFields(g, eps)
    phi_sc, i1 = S.sc(g, rho, eps, eta=0.6, tol_abs=1e-10, max_iter=200, fields=f)
    phi_di, i2 = S.psd(g, rho, eps, diis=6, tol_abs=1e-10, max_iter=200, fields=f)
    phi_cg, _ = oracle.solve_gpe(g, rho, eps, tol_abs=1e-10)
    top = phi_ex.max()
    assert i1["converged"] and i2["converged"]
    assert np.abs(phi_sc - phi_ex).max() < 1e-3 * top
    assert np.abs(phi_di - phi_sc).max() < 1e-9 * top
    assert np.abs(phi_sc - phi_cg).max() < 1e-3 * top
    assert i2["iters"] < i1["iters"]


def test_diis_coefficients_brute_force():
    """Pulay coefficients: the minimum of ||sum c_i v_i|| on sum c_i = 1,
    against a fine scan of the constraint line (two vectors) and against
    random points of the constraint plane (three vectors)."""
    rng = np.random.default_rng(3)
    v = [rng.standard_normal(50) for _ in range(3)]
    c2 = S.diis_coefficients(v[:2])
    t = np.linspace(-5, 5, 200001)
    vals = [np.linalg.norm(ti * v[0] + (1 - ti) * v[1]) for ti in t[::100]]
    best = t[::100][int(np.argmin(vals))]
    assert abs(c2.sum() - 1.0) < 1e-14 and abs(c2[0] - best) < 5e-3
    c3 = S.diis_coefficients(v)
    f3 = np.linalg.norm(sum(ci * vi for ci, vi in zip(c3, v)))
    for _ in range(2000):
        a, b = rng.standard_normal(2) * 2
        cc = c3 + np.array([a, b, -a - b]) * 0.05
        assert np.linalg.norm(sum(ci * vi for ci, vi in zip(cc, v))) >= f3 - 1e-12
    assert abs(c3.sum() - 1.0) < 1e-14


def test_diis_history_one_is_plain_psd():
    g, rho, eps = _small_cavity(synth.BC_FREE)
    f = S.ScFields(g, eps)
    a, ia = S.psd(g, rho, eps, alpha=0.6, tol_abs=0.0, max_iter=15, fields=f)
    b, ib = S.psd(g, rho, eps, alpha=0.6, diis=1, tol_abs=0.0, max_iter=15, fields=f)
    assert np.array_equal(a, b) and ia["res"] == ib["res"]


def test_steepest_descent_step_is_the_energy_minimum():
    """Periodic BC (no boundary terms): the steepest-descent step
    (v, r) / (v, A v) equals 1 + int v grad eps . grad v / int eps |grad v|^2,
    the exact minimizer of the energy along v for A = div eps grad."""
    g, rho, eps = _small_cavity(synth.BC_PERIODIC, n=16, h=0.5)
    rho = rho - rho.mean()
    f = S.ScFields(g, eps)
    r = f.project(-4 * math.pi * rho)
    v = f.precondition(r)
    Av = f.apply_A_from_v(v, r)
    vx, vy, vz = oracle.fd16.gradient(v, g)
    ex, ey, ez = oracle.fd16.gradient(eps, g)
    E = np.sum(eps * (vx * vx + vy * vy + vz * vz))
    C = np.sum(v * (ex * vx + ey * vy + ez * vz))
    assert abs(np.sum(v * r) / np.sum(v * Av) - (1 + C / E)) < 1e-3


def test_planted_sign_error_in_rho_iter_is_caught(monkeypatch):
    """rho_iter with the wrong sign (Eq. rhoiter) misses the analytic
    potential of the manufactured test by far more than its accuracy."""
    g, rho, eps, phi_ex = _manufactured(n=40)
    good = S.ScFields.g_dot_grad
    monkeypatch.setattr(S.ScFields, "g_dot_grad", lambda self, u: -good(self, u))
    phi, info = S.sc(g, rho, eps, eta=0.3, tol_abs=1e-8, max_iter=200)
    assert not info["converged"] or np.abs(phi - phi_ex).max() > 1e-2 * phi_ex.max()
