"""GPU parity of the comparison solvers (Algorithm 1 / SC, PSD, PSD + DIIS)
against the oracle, element by element on the same seeded inputs.

Fixed iteration counts compare the iterates themselves (each method's
arithmetic step by step, DIIS ring wrap-around included); converged runs
compare the solutions and the iteration counts.  At full size the oracle is
too slow, so the properties checked there hold at any size: DIIS and SC
reach the same discrete fixed point, and both agree with Algorithm 2's
solution to discretization error.
"""
import numpy as np
import pytest

import synth
from oracle import sc as S

pytestmark = pytest.mark.gpu

# FP64 throughout; the two sides differ by summation order only.  A few
# dozen iterations of a contraction amplify that by a small factor.
TOL_ITER = 1e-11
TOL_CONV = 1e-10


@pytest.fixture(scope="module")
def gps():
    from paper_1509_00680_gb300 import build
    build.build()
    from paper_1509_00680_gb300 import gps as g
    return g


@pytest.fixture(scope="module")
def ctx(gps):
    c = gps.Context(0)
    yield c
    c.close()


def T(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def N(t, shape):
    return t.cpu().numpy().reshape(shape)


def rel2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _gauge(a, periodic):
    return a - a.mean() if periodic else a


CASES = {
    "free": lambda: synth.workload(1, n=32),
    "free_ragged": lambda: _ragged_free(),
    "periodic": lambda: _neutral(synth.workload(2, n=32, count=4)),
    "surface": lambda: synth.workload(3, nxy=24, nz=96, count=4),
    "wire": lambda: _wire(),
}


def _wire():
    """Wire BC (periodic z, free x and y): two cavities along z."""
    g = synth.Grid(24, 24, 32, 0.4, 0.4, 0.35, synth.BC_WIRE)
    c = 12 * 0.4
    eps = synth.rigid_cavity(g, [(2.2, (c, c, 2.8)), (2.2, (c, c, 8.4))], 0.5)
    rho = synth.gaussian_charges(g, [(1.0, 0.9, (c - 0.5, c, 2.8)), (-1.0, 0.8, (c + 0.5, c, 8.4))])
    return synth.Problem("wire", g, rho, eps)


def _neutral(p):
    p.rho = p.rho - p.rho.mean()
    return p


def _ragged_free():
    """Unequal, non-power-of-two sides (padded lengths 2 x {18, 20, 24})."""
    g = synth.Grid(18, 20, 24, 0.4, 0.4, 0.35, synth.BC_FREE)
    c = (9 * 0.4, 10 * 0.4, 12 * 0.35)
    eps = synth.rigid_cavity(g, [(2.2, c)], 0.5)
    rho = synth.gaussian_charges(g, [(1.0, 0.9, (c[0] - 0.5, c[1], c[2])), (-1.0, 0.8, (c[0] + 0.6, c[1], c[2]))])
    return synth.Problem("ragged", g, rho, eps)


def _run(gps, ctx, p, method, max_iter, tol_rel=0.0, tol_abs=0.0, allow=None, **kw):
    phi = T(np.zeros(p.grid.shape))
    o = gps.default_opts(method=gps.METHOD[method], tol_abs=tol_abs, tol_rel=tol_rel, max_iter=max_iter, **kw)
    rep = ctx.gpe_solve(gps.grid_from(p.grid), T(p.rho), T(p.eps), phi, o,
                        allow=allow or (gps.GPS_OK, gps.GPS_ERR_NOT_CONVERGED))
    return N(phi, p.grid.shape), rep


@pytest.mark.parametrize("case", list(CASES))
def test_sc_iterates(gps, ctx, case):
    """Six SC steps (eta = 0.6): phi_5 and the residual history."""
    p = CASES[case]()
    got, rep = _run(gps, ctx, p, "sc", 6, eta=0.6)
    ref, info = S.sc(p.grid, p.rho, p.eps, eta=0.6, tol_abs=0.0, max_iter=6)
    assert rep.iters == 6 and rep.status == gps.GPS_ERR_NOT_CONVERGED
    assert rel2(got, ref) < TOL_ITER
    assert abs(rep.res0 - info["res"][0]) <= 1e-13 * info["res"][0]
    assert abs(rep.res - info["res"][-1]) <= 1e-9 * info["res"][-1]


@pytest.mark.parametrize("case", list(CASES))
def test_sc_converged(gps, ctx, case):
    p = CASES[case]()
    got, rep = _run(gps, ctx, p, "sc", 500, tol_rel=1e-11, allow=(gps.GPS_OK,), eta=0.6)
    ref, info = S.sc(p.grid, p.rho, p.eps, eta=0.6, tol_abs=0.0, tol_rel=1e-11, max_iter=500)
    assert info["converged"]
    assert abs(rep.iters - info["iters"]) <= 1
    per = p.grid.bc == synth.BC_PERIODIC
    assert rel2(_gauge(got, per), _gauge(ref, per)) < TOL_CONV


@pytest.mark.parametrize("case", ["free", "periodic", "surface"])
@pytest.mark.parametrize("alpha", [0.6, 0.0])
def test_psd_iterates(gps, ctx, case, alpha):
    """Seven PSD steps with a fixed step and with the steepest-descent step."""
    p = CASES[case]()
    got, rep = _run(gps, ctx, p, "psd", 7, alpha=alpha)
    ref, info = S.psd(p.grid, p.rho, p.eps, alpha=alpha or None, tol_abs=0.0, max_iter=7)
    assert rep.iters == 7
    assert rel2(got, ref) < TOL_ITER
    assert abs(rep.res - info["res"][-1]) <= 1e-9 * info["res"][-1]


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("m", [3, 6])
def test_diis_iterates(gps, ctx, case, m):
    """Ten PSD + DIIS steps: with m = 3 the ring wraps three times."""
    p = CASES[case]()
    got, rep = _run(gps, ctx, p, "psd", 10, diis=m)
    ref, info = S.psd(p.grid, p.rho, p.eps, diis=m, tol_abs=0.0, max_iter=10)
    assert rep.iters == 10
    assert rel2(got, ref) < 1e-10
    assert abs(rep.res - info["res"][-1]) <= 1e-8 * info["res"][-1]


@pytest.mark.parametrize("case", list(CASES))
def test_diis_converged(gps, ctx, case):
    p = CASES[case]()
    got, rep = _run(gps, ctx, p, "psd", 300, tol_rel=1e-11, allow=(gps.GPS_OK,), diis=6)
    ref, info = S.psd(p.grid, p.rho, p.eps, diis=6, tol_abs=0.0, tol_rel=1e-11, max_iter=300)
    assert info["converged"]
    # near convergence the Pulay matrix is ill-conditioned: rounding may move
    # the path by an iteration or two, not the solution
    assert abs(rep.iters - info["iters"]) <= 2
    per = p.grid.bc == synth.BC_PERIODIC
    assert rel2(_gauge(got, per), _gauge(ref, per)) < TOL_CONV


def test_psd_fixed_step_alpha_one_uniform_eps(gps, ctx):
    """Uniform eps: one step of length 1 ends the solve (grad ln eps = 0)."""
    g = synth.Grid(24, 24, 24, 0.4, 0.4, 0.4, synth.BC_FREE)
    c = (12 * 0.4,) * 3
    p = synth.Problem("uniform", g, synth.gaussian_charges(g, [(1.0, 1.0, c)]), np.full(g.shape, 5.0))
    for method, kw in (("sc", dict(eta=0.6)), ("psd", dict(alpha=0.0)), ("psd", dict(diis=4))):
        got, rep = _run(gps, ctx, p, method, 20, tol_abs=1e-9, allow=(gps.GPS_OK,), **kw)
        ref, info = S.solve_sc(g, p.rho, p.eps, method="sc", tol_abs=1e-9, max_iter=20)
        assert rep.iters == 1 and info["iters"] == 1
        assert rel2(got, ref) < 1e-13


def test_zero_source_returns_zero(gps, ctx):
    p = CASES["free"]()
    p.rho = np.zeros_like(p.rho)
    for method in ("sc", "psd"):
        got, rep = _run(gps, ctx, p, method, 10, tol_abs=1e-12, allow=(gps.GPS_OK,))
        assert rep.iters == 0 and not got.any()


def test_full_size_periodic_sc_diis_and_pcg(gps, ctx):
    """The 128^3 periodic workload (20 Gaussians, union-of-spheres eps): SC
    and PSD + DIIS converge to the same discrete solution; Algorithm 2's
    solution (a different discretization of Eq. GPe) agrees with it to
    discretization error; DIIS needs fewer iterations than SC."""
    p = synth.workload(2)
    got_sc, rep_sc = _run(gps, ctx, p, "sc", 2000, tol_rel=1e-9, allow=(gps.GPS_OK,), eta=0.6)
    got_di, rep_di = _run(gps, ctx, p, "psd", 2000, tol_rel=1e-9, allow=(gps.GPS_OK,), diis=6)
    phi = T(np.zeros(p.grid.shape))
    ctx.gpe_solve(gps.grid_from(p.grid), T(p.rho), T(p.eps), phi, gps.default_opts(tol_abs=1e-10))
    got_cg = N(phi, p.grid.shape)
    assert rep_sc.res <= 1e-9 * rep_sc.res0 and rep_di.res <= 1e-9 * rep_di.res0
    assert rel2(_gauge(got_di, True), _gauge(got_sc, True)) < 1e-7
    assert rel2(_gauge(got_cg, True), _gauge(got_sc, True)) < 5e-3
    assert rep_di.iters < rep_sc.iters


def test_paper_manufactured_test_accuracy(gps, ctx):
    """The paper's GPe test (Gaussian potential, erf cavity d0 = 1.7,
    Delta = 0.3, eps0 = 78.36, box 10): SC and DIIS reach the analytic
    potential to the order-16 discretization's accuracy at 96^3."""
    import math
    n, L = 96, 10.0
    h = L / n
    g = synth.Grid(n, n, n, h, h, h, synth.BC_FREE)
    c = n // 2 * h
    x = h * np.arange(n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    r = np.sqrt((X - c) ** 2 + (Y - c) ** 2 + (Z - c) ** 2)
    s, d0, delta, e0 = 0.5, 1.7, 0.3, 78.36
    phi_ex = np.exp(-r * r / (2 * s * s)) / (2 * math.pi * s * s) ** 1.5
    from scipy.special import erf
    eps = 1.0 + (e0 - 1.0) * 0.5 * (1.0 + erf((r - d0) / delta))
    deps = (e0 - 1.0) / (delta * math.sqrt(math.pi)) * np.exp(-((r - d0) / delta) ** 2)
    rho = -(eps * (r * r / s ** 4 - 3 / s ** 2) * phi_ex + deps * (-(r / s ** 2) * phi_ex)) / (4 * math.pi)
    p = synth.Problem("manufactured", g, rho, eps)
    for method, kw in (("sc", dict(eta=0.6)), ("psd", dict(diis=6))):
        got, rep = _run(gps, ctx, p, method, 300, tol_rel=1e-10, allow=(gps.GPS_OK,), **kw)
        assert np.abs(got - phi_ex).max() < 2e-4 * phi_ex.max()


def test_invalid_method_arguments(gps, ctx):
    p = CASES["free"]()
    gr = gps.grid_from(p.grid)
    phi = T(np.zeros(p.grid.shape))
    bad = [dict(method=3), dict(method=gps.GPS_SC, precision=gps.GPS_MIXED),
           dict(method=gps.GPS_SC, warm_start=1), dict(method=gps.GPS_SC, eta=0.0),
           dict(method=gps.GPS_PSD, diis=gps.GPS_MAX_DIIS + 1), dict(method=gps.GPS_PSD, alpha=-1.0)]
    for kw in bad:
        with pytest.raises(gps.GpsError) as e:
            ctx.gpe_solve(gr, T(p.rho), T(p.eps), phi, gps.default_opts(**kw))
        assert e.value.status == gps.GPS_ERR_INVALID
    el = gps.make_electrolyte((1, -1), (0.1, 0.1), 300.0, synth.EPS_WATER)
    with pytest.raises(gps.GpsError):
        ctx.pb_solve(gr, T(p.rho), T(p.eps), el, "lpb", phi, gps.default_opts(method=gps.GPS_SC))
    gs = synth.Grid(16, 6, 16, 0.5, 0.5, 0.5, synth.BC_PERIODIC)   # a periodic axis < 8 points
    with pytest.raises(gps.GpsError):
        ctx.gpe_solve(gps.grid_from(gs), T(np.zeros(gs.shape)), T(np.ones(gs.shape)), T(np.zeros(gs.shape)),
                      gps.default_opts(method=gps.GPS_SC))
    rho = np.ascontiguousarray(p.rho.ravel())
    eps = np.ascontiguousarray(p.eps.ravel())
    out = np.zeros(p.grid.npts)
    req = gps.make_request(gr, "gpe", rho, eps, out, opts=gps.default_opts(method=gps.GPS_SC))
    reps = gps.batch_solve(ctx, [req], allow=(gps.GPS_OK, gps.GPS_ERR_INVALID))
    assert reps[0].status == gps.GPS_ERR_INVALID


def test_host_entry_point_matches_device(gps, ctx):
    p = CASES["surface"]()
    got, rep = _run(gps, ctx, p, "psd", 200, tol_rel=1e-10, allow=(gps.GPS_OK,), diis=5)
    out = np.zeros(p.grid.npts)
    o = gps.default_opts(method=gps.GPS_PSD, diis=5, tol_abs=0.0, tol_rel=1e-10, max_iter=200)
    rep_h = ctx.gpe_solve_host(gps.grid_from(p.grid), np.ascontiguousarray(p.rho.ravel()),
                               np.ascontiguousarray(p.eps.ravel()), out, o)
    assert rep_h.iters == rep.iters
    assert np.array_equal(out.reshape(p.grid.shape), got)
