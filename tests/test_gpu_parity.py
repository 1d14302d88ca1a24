"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Small grids that span several FFT tiles with ragged edges are compared
element by element; the full-size workloads are checked through properties
that hold at any size (the oracle's own discrete fixed-point residual of the
GPU result) plus sampled comparisons.  Tolerances:
  * vacuum solve / preconditioner, FP64: 1e-12 relative (max norm) -- two
    FFTs of different factorization order differ by O(eps log N);
  * s = eps^-1/2: bit-exact (correctly rounded sqrt and division on both sides);
  * q by FD-16: 1e-13 relative (different summation order);
  * potentials phi of converged solves: relative L2 <= 1e-10 (the target
    stated for the FP64 path), both sides converged to ||r|| <= 1e-13 ||r0||.
"""
import importlib.util
import os

import numpy as np
import pytest

import oracle
import synth
from oracle.green import VacuumSolver
from oracle.operators import Fields

pytestmark = pytest.mark.gpu


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


def relmax(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def rel2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


SMALL = [
    (synth.BC_FREE, (12, 10, 16), (0.5, 0.45, 0.4)),
    (synth.BC_FREE, (20, 18, 15), (0.4, 0.4, 0.4)),
    (synth.BC_PERIODIC, (16, 12, 10), (0.5, 0.5, 0.6)),
    (synth.BC_PERIODIC, (30, 24, 20), (0.4, 0.45, 0.5)),
    (synth.BC_SURFACE, (16, 12, 10), (0.5, 0.5, 0.5)),
    (synth.BC_SURFACE, (20, 18, 24), (0.4, 0.4, 0.35)),
    (synth.BC_WIRE, (12, 10, 16), (0.5, 0.45, 0.4)),
    (synth.BC_WIRE, (20, 18, 24), (0.4, 0.4, 0.35)),
]


def _grid(bc, n, h):
    return synth.Grid(n[0], n[1], n[2], h[0], h[1], h[2], bc)


@pytest.mark.parametrize("bc,n,h", SMALL)
def test_vacuum_solve(gps, ctx, bc, n, h):
    g = _grid(bc, n, h)
    rng = np.random.default_rng(11)
    sigma = rng.standard_normal(g.shape)
    w = T(np.zeros(g.shape))
    ctx.vacuum_solve(gps.grid_from(g), T(sigma), w)
    ref = VacuumSolver(g).apply(sigma)
    assert relmax(N(w, g.shape), ref) < 1e-12


@pytest.mark.parametrize("bc,n,h", SMALL)
def test_setup_fields(gps, ctx, bc, n, h):
    g = _grid(bc, n, h)
    rng = np.random.default_rng(12)
    eps = 1.0 + 20.0 * rng.random(g.shape)
    s, q = T(np.zeros(g.shape)), T(np.zeros(g.shape))
    ctx.setup_fields(gps.grid_from(g), T(eps), s, q)
    f = Fields(g, eps)
    assert np.array_equal(N(s, g.shape), f.s)
    assert relmax(N(q, g.shape), f.q) < 1e-12


@pytest.mark.parametrize("bc,n,h", SMALL)
def test_precondition_fp64(gps, ctx, bc, n, h):
    g = _grid(bc, n, h)
    rng = np.random.default_rng(13)
    eps = 1.0 + 30.0 * rng.random(g.shape)
    r = rng.standard_normal(g.shape)
    f = Fields(g, eps)
    v = T(np.zeros(g.shape))
    ctx.precondition(gps.grid_from(g), T(f.s), T(r), v)
    assert relmax(N(v, g.shape), f.precondition(r)) < 1e-12


@pytest.mark.parametrize("bc,n,h", SMALL[::2])
def test_precondition_fp32_spectrum(gps, ctx, bc, n, h):
    g = _grid(bc, n, h)
    rng = np.random.default_rng(14)
    eps = 1.0 + 30.0 * rng.random(g.shape)
    r = rng.standard_normal(g.shape)
    f = Fields(g, eps)
    v = T(np.zeros(g.shape))
    ctx.precondition(gps.grid_from(g), T(f.s), T(r), v, precision=gps.GPS_MIXED)
    assert relmax(N(v, g.shape), f.precondition(r)) < 2e-5


# Grids whose padded lengths are multiples of 16 on most axes, so that the
# radix-16 order (FP64 only) applies: 16, 32, 48, 64, 2048.
RADIX = [
    (synth.BC_PERIODIC, (32, 48, 64), (0.3, 0.3, 0.3)),
    (synth.BC_FREE, (16, 24, 32), (0.5, 0.45, 0.4)),
    (synth.BC_SURFACE, (32, 16, 24), (0.4, 0.45, 0.5)),
    (synth.BC_WIRE, (24, 16, 40), (0.4, 0.5, 0.35)),
    (synth.BC_PERIODIC, (8, 8, 2048), (0.5, 0.5, 0.01)),
]


@pytest.mark.parametrize("order", [0, 1, 2, 3])
def test_fft_radix_orders(gps, order):
    """Every radix order of the shared-memory FFT passes (gps_set_radix_order):
    FP64 vacuum solve and preconditioner against the oracle; order 3 takes the
    radix-16 kernels wherever a length has a factor 16."""
    gps.set_radix_order(order)
    c = gps.Context(0)
    try:
        for bc, n, h in RADIX:
            g = _grid(bc, n, h)
            rng = np.random.default_rng(21)
            sigma = rng.standard_normal(g.shape)
            w = T(np.zeros(g.shape))
            c.vacuum_solve(gps.grid_from(g), T(sigma), w)
            assert relmax(N(w, g.shape), VacuumSolver(g).apply(sigma)) < 1e-12
            eps = 1.0 + 30.0 * rng.random(g.shape)
            r = rng.standard_normal(g.shape)
            f = Fields(g, eps)
            v = T(np.zeros(g.shape))
            c.precondition(gps.grid_from(g), T(f.s), T(r), v)
            assert relmax(N(v, g.shape), f.precondition(r)) < 1e-12
        if order == 3:
            p = synth.workload(2, n=64, count=8)
            phi = T(np.zeros(p.grid.shape))
            rep = c.gpe_solve(gps.grid_from(p.grid), T(p.rho), T(p.eps), phi,
                              gps.default_opts(tol_abs=0.0, tol_rel=1e-13, max_iter=2000))
            ref, info = oracle.solve_gpe(p.grid, p.rho, p.eps, tol_abs=0.0, tol_rel=1e-13, max_iter=2000)
            assert abs(rep.iters - info["iters"]) <= 2
            assert rel2(N(phi, p.grid.shape), ref) <= 1e-10
    finally:
        c.close()
        gps.set_radix_order(-1)


# Grids whose padded x / y / z lengths are the powers of two 64 .. 1024 handled
# by the register-resident kernels, with column tiles that end ragged
# (Hx not a multiple of the columns per CTA); free-BC boxes are cubic in
# length, as the oversampled free kernel requires.
COLUMN = [
    (synth.BC_PERIODIC, (20, 64, 128), (0.4, 0.4, 0.3)),    # y 64, z 128
    (synth.BC_FREE, (16, 32, 64), (0.8, 0.4, 0.2)),         # y 64, z 128 (zero padded)
    (synth.BC_FREE, (16, 128, 20), (0.8, 0.1, 0.64)),       # y 256
    (synth.BC_PERIODIC, (12, 256, 512), (0.5, 0.3, 0.2)),   # y 256, z 512
    (synth.BC_SURFACE, (8, 6, 512), (0.5, 0.5, 0.1)),       # z 1024
    (synth.BC_WIRE, (16, 32, 128), (0.8, 0.4, 0.3)),        # y 64 (zero padded), z 128 (periodic)
    # x passes (row pairs; odd row counts leave a last pair with one row)
    (synth.BC_PERIODIC, (64, 6, 6), (0.3, 0.5, 0.6)),       # x 64
    (synth.BC_FREE, (32, 5, 9), (0.4, 2.56, 1.42)),         # x 64 (zero padded), 45 rows
    (synth.BC_PERIODIC, (128, 12, 10), (0.3, 0.4, 0.5)),    # x 128
    (synth.BC_FREE, (128, 16, 20), (0.1, 0.8, 0.64)),       # x 256
    (synth.BC_PERIODIC, (512, 6, 8), (0.05, 0.5, 0.5)),     # x 512
    (synth.BC_SURFACE, (1024, 4, 6), (0.05, 0.5, 0.5)),     # x 1024
]


@pytest.mark.parametrize("bc,n,h", COLUMN)
def test_vacuum_solve_column_kernels(gps, ctx, bc, n, h):
    g = _grid(bc, n, h)
    rng = np.random.default_rng(21)
    sigma = rng.standard_normal(g.shape)
    w = T(np.zeros(g.shape))
    ctx.vacuum_solve(gps.grid_from(g), T(sigma), w)
    ref = VacuumSolver(g).apply(sigma)
    assert relmax(N(w, g.shape), ref) < 1e-12


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("df64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("bc,n,h", COLUMN)
def test_precondition_column_kernels(gps, ctx, bc, n, h, prec, tol):
    g = _grid(bc, n, h)
    rng = np.random.default_rng(22)
    eps = 1.0 + 30.0 * rng.random(g.shape)
    r = rng.standard_normal(g.shape)
    f = Fields(g, eps)
    v = T(np.zeros(g.shape))
    code = {"fp64": gps.GPS_FP64, "df64": gps.GPS_DF64, "fp32": gps.GPS_MIXED}[prec]
    ctx.precondition(gps.grid_from(g), T(f.s), T(r), v, precision=code)
    assert relmax(N(v, g.shape), f.precondition(r)) < tol


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("bc,n,h", [c for c in COLUMN if c[1][0] >= 32])
def test_precondition_fp32_x_kernels(gps, bc, n, h, kind):
    """FP32 x passes by the shared-memory (0) and the register-resident (1)
    kernels, whichever the tuner would pick: the preconditioner against the
    oracle at the FP32 spectrum's tolerance."""
    g = _grid(bc, n, h)
    rng = np.random.default_rng(23)
    eps = 1.0 + 30.0 * rng.random(g.shape)
    r = rng.standard_normal(g.shape)
    f = Fields(g, eps)
    gps.set_x_kernel(kind)
    c = gps.Context(0)
    try:
        v = T(np.zeros(g.shape))
        c.precondition(gps.grid_from(g), T(f.s), T(r), v, precision=gps.GPS_MIXED)
        assert relmax(N(v, g.shape), f.precondition(r)) < 2e-5
    finally:
        c.close()
        gps.set_x_kernel(-1)


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-5), ("df64", 1e-12)])
@pytest.mark.parametrize("bc,n,h", COLUMN[:6])
def test_precondition_tma_z_pass(gps, bc, n, h, prec, tol):
    """The z pass of the FP32 and double-float spectra in its TMA-staged form
    (tensor loads and stores of column tiles, persistent CTAs), forced: the
    preconditioner against the oracle at each spectrum's tolerance, for the
    column lengths 128-1024, zero-padded and periodic."""
    g = _grid(bc, n, h)
    rng = np.random.default_rng(24)
    eps = 1.0 + 30.0 * rng.random(g.shape)
    r = rng.standard_normal(g.shape)
    f = Fields(g, eps)
    gps.set_z_kernel(1)
    c = gps.Context(0)
    try:
        v = T(np.zeros(g.shape))
        code = gps.GPS_MIXED if prec == "fp32" else gps.GPS_DF64
        c.precondition(gps.grid_from(g), T(f.s), T(r), v, precision=code)
        assert relmax(N(v, g.shape), f.precondition(r)) < tol
    finally:
        c.close()
        gps.set_z_kernel(-1)


def test_mixed_solve_tma_z_pass(gps):
    """A mixed-precision solve (df64 then FP32 spectrum) with the TMA-staged
    z pass forced, against the oracle at the mixed bar."""
    p = synth.workload(4, n=64, count=12, margin=6.0, kind="gpe")
    gps.set_z_kernel(1)
    c = gps.Context(0)
    try:
        phi = T(np.zeros(p.grid.shape))
        rep = c.gpe_solve(gps.grid_from(p.grid), T(p.rho), T(p.eps), phi,
                          gps.default_opts(tol_abs=1e-10, precision=gps.GPS_MIXED_DF64, max_iter=2000))
        ref, _ = oracle.solve_gpe(p.grid, p.rho, p.eps, tol_abs=0.0, tol_rel=1e-13, max_iter=2000)
        assert rep.status == 0 and 0 < rep.fp64_iters < rep.iters
        assert 0 <= rep.fixed_point_res < 1e-8
        err = rel2(N(phi, p.grid.shape), ref)
        assert err <= 1e-8, err
    finally:
        c.close()
        gps.set_z_kernel(-1)


def _has_solvent(p):
    """A slab test box must reach above the interface (z = 10 bohr): below it
    eps = 1 and the problem is vacuum Poisson."""
    return oracle.pb.exclusion_from_eps(p.eps, p.eps0).max() > 0.99


def _solve_pair(gps, ctx, p, kind="gpe", tol_rel=1e-13, **okw):
    g = p.grid
    phi = T(np.zeros(g.shape))
    opts = gps.default_opts(tol_abs=0.0, tol_rel=tol_rel, max_iter=2000, **okw)
    if kind == "gpe":
        rep = ctx.gpe_solve(gps.grid_from(g), T(p.rho), T(p.eps), phi, opts)
        ref, info = oracle.solve_gpe(g, p.rho, p.eps, tol_abs=0.0, tol_rel=tol_rel, max_iter=2000)
    elif kind == "lpb":
        el = gps.make_electrolyte(p.electrolyte.z, p.electrolyte.c_molar, p.electrolyte.temperature, p.eps0)
        rep = ctx.pb_solve(gps.grid_from(g), T(p.rho), T(p.eps), el, "lpb", phi, opts)
        gam = oracle.pb.exclusion_from_eps(p.eps, p.eps0)
        lam = oracle.pb.linear_lambda(gam, p.electrolyte)
        ref, info = oracle.solve_lpb(g, p.rho, p.eps, lam, tol_abs=0.0, tol_rel=tol_rel, max_iter=2000)
    return N(phi, g.shape), ref, rep, info


def _wire_chain(n=32, nz=48):
    return synth.wire_chain(n=n, nz=nz)


@pytest.mark.parametrize("kind", ["gpe", "lpb"])
def test_wire_solves(gps, ctx, kind):
    p = _wire_chain()
    got, ref, rep, info = _solve_pair(gps, ctx, p, kind=kind)
    assert rep.status == 0
    assert abs(rep.iters - info["iters"]) <= 2
    assert rel2(got, ref) <= 1e-10


def test_wire_nlpb(gps, ctx):
    p = _wire_chain(n=24, nz=32)
    el = gps.make_electrolyte(p.electrolyte.z, p.electrolyte.c_molar, p.electrolyte.temperature, p.eps0)
    phi = T(np.zeros(p.grid.shape))
    rep = ctx.pb_solve(gps.grid_from(p.grid), T(p.rho), T(p.eps), el, "nlpb", phi,
                       gps.default_opts(tol_outer=1e-11, max_iter=3000))
    ref, info = oracle.solve_nlpb(p.grid, p.rho, p.eps, p.electrolyte, p.eps0, tol=1e-11, max_iter=3000)
    assert info["converged"] and rep.status == 0
    err = rel2(N(phi, p.grid.shape), ref)
    assert err <= 1e-10, err


def test_lpb_manufactured_solution(gps, ctx):
    """The paper's linear-PB test on the GPU (free BC, the library's own
    lambda from the electrolyte): the analytic potential to the
    discretization accuracy the oracle reaches (6e-6 of the peak at 96^3)."""
    import math
    p = synth.manufactured(n=96, L=16.0, sigma=1.0, d0=2.5, delta=0.5)
    e = synth.Electrolyte((1, -1), (0.5, 0.5), 300.0)
    lam = oracle.pb.linear_lambda(oracle.pb.exclusion_from_eps(p.eps, p.eps0), e)
    rho = p.rho + lam * p.phi_exact / (4 * math.pi)
    el = gps.make_electrolyte(e.z, e.c_molar, e.temperature, p.eps0)
    phi = T(np.zeros(p.grid.shape))
    rep = ctx.pb_solve(gps.grid_from(p.grid), T(rho), T(p.eps), el, "lpb", phi, gps.default_opts(tol_abs=1e-11))
    assert rep.status == 0 and rep.iters <= 25
    assert np.abs(N(phi, p.grid.shape) - p.phi_exact).max() < 2e-5 * p.phi_exact.max()


def test_mpb_manufactured_solution(gps, ctx):
    """The paper's modified-PB test on the GPU (p = 0.74, R = 3 angstrom,
    100 mol/m^3, free BC, FP64 Newton outer loop): the analytic potential to
    the discretization accuracy of 96^3 in a few outer steps."""
    p = synth.manufactured(n=96, L=16.0, sigma=1.0, d0=2.5, delta=0.5)
    e = synth.Electrolyte((1, -1), (0.1, 0.1), 300.0, radius_angstrom=(3.0, 3.0), packing=0.74)
    rho = p.rho - oracle.pb.ionic_charge(p.phi_exact, oracle.pb.exclusion_from_eps(p.eps, p.eps0), e)
    el = gps.make_electrolyte(e.z, e.c_molar, e.temperature, p.eps0, radius_angstrom=e.radius_angstrom,
                              packing=e.packing)
    phi = T(np.zeros(p.grid.shape))
    rep = ctx.pb_solve(gps.grid_from(p.grid), T(rho), T(p.eps), el, "mpb", phi,
                       gps.default_opts(tol_outer=1e-10, max_iter=500))
    assert rep.status == 0 and rep.outer_iters <= 8
    assert np.abs(N(phi, p.grid.shape) - p.phi_exact).max() < 2e-5 * p.phi_exact.max()


def _custom_gamma(p):
    """An ion-exclusion function other than the cavity function: its square
    (ions kept further from the solute)."""
    return oracle.pb.exclusion_from_eps(p.eps, p.eps0) ** 2


def test_exclusion_function_lpb_and_host(gps, ctx):
    p = synth.workload(3, nxy=32, nz=96, count=6, kind="lpb")
    assert _has_solvent(p)
    gam = np.ascontiguousarray(_custom_gamma(p))
    e = p.electrolyte
    gr = gps.grid_from(p.grid)
    g_dev = T(gam)
    el = gps.make_electrolyte(e.z, e.c_molar, e.temperature, p.eps0, exclusion=g_dev)
    phi = T(np.zeros(p.grid.shape))
    opts = gps.default_opts(tol_abs=0.0, tol_rel=1e-13, max_iter=2000, warm_start=1)
    rep = ctx.pb_solve(gr, T(p.rho), T(p.eps), el, "lpb", phi, opts)
    lam = oracle.pb.linear_lambda(gam, e)
    ref, info = oracle.solve_lpb(p.grid, p.rho, p.eps, lam, tol_abs=0.0, tol_rel=1e-13, max_iter=2000)
    got = N(phi, p.grid.shape)
    assert rep.status == 0 and rep.warm == 0
    assert rel2(got, ref) <= 1e-10
    plain, _ = oracle.solve_lpb(p.grid, p.rho, p.eps, oracle.pb.linear_lambda(
        oracle.pb.exclusion_from_eps(p.eps, p.eps0), e), tol_abs=0.0, tol_rel=1e-13, max_iter=2000)
    assert rel2(got, plain) > 1e-6                 # the exclusion array was used
    out = np.zeros(p.grid.npts)
    el_h = gps.make_electrolyte(e.z, e.c_molar, e.temperature, p.eps0, exclusion=gam.ravel())
    ctx.pb_solve_host(gr, np.ascontiguousarray(p.rho.ravel()), np.ascontiguousarray(p.eps.ravel()), el_h,
                      "lpb", out, gps.default_opts(tol_abs=0.0, tol_rel=1e-13, max_iter=2000))
    assert np.array_equal(out.reshape(p.grid.shape), got)
    req = gps.make_request(gr, "lpb", np.ascontiguousarray(p.rho.ravel()), np.ascontiguousarray(p.eps.ravel()),
                           np.zeros(p.grid.npts), el_h)
    assert gps.batch_solve(ctx, [req], allow=(gps.GPS_OK, gps.GPS_ERR_INVALID))[0].status == gps.GPS_ERR_INVALID


def test_exclusion_function_nlpb_and_ionic_charge(gps, ctx):
    p = synth.workload(4, n=48, count=6, margin=5.0, kind="nlpb", conc=0.5)
    gam = np.ascontiguousarray(_custom_gamma(p))
    e = p.electrolyte
    gr = gps.grid_from(p.grid)
    g_dev = T(gam)                       # kept alive: the electrolyte holds its address only
    el = gps.make_electrolyte(e.z, e.c_molar, e.temperature, p.eps0, exclusion=g_dev)
    phi = T(np.zeros(p.grid.shape))
    rep = ctx.pb_solve(gr, T(p.rho), T(p.eps), el, "nlpb", phi, gps.default_opts(tol_outer=1e-11, max_iter=3000))
    ref, info = oracle.solve_nlpb(p.grid, p.rho, p.eps, e, p.eps0, tol=1e-11, max_iter=3000, gamma=gam)
    assert info["converged"] and rep.status == 0
    err = rel2(N(phi, p.grid.shape), ref)
    assert err <= 1e-10, err
    out = T(np.zeros(p.grid.shape))
    ctx.ionic_charge(gr, T(ref), T(p.eps), el, out)
    assert relmax(N(out, p.grid.shape), oracle.pb.ionic_charge(ref, gam, e)) < 1e-13


def test_gpe_free_single_cavity(gps, ctx):
    p = synth.workload(1)          # 64^3, h = 0.3, the free-BC workload itself
    got, ref, rep, info = _solve_pair(gps, ctx, p)
    assert rep.status == 0
    assert abs(rep.iters - info["iters"]) <= 2
    assert rel2(got, ref) <= 1e-10


def test_gpe_free_default_tolerance(gps, ctx):
    """The workload's own stopping rule, ||r|| <= 1e-10."""
    p = synth.workload(1)
    phi = T(np.zeros(p.grid.shape))
    rep = ctx.gpe_solve(gps.grid_from(p.grid), T(p.rho), T(p.eps), phi, gps.default_opts(tol_abs=1e-10))
    ref, info = oracle.solve_gpe(p.grid, p.rho, p.eps, tol_abs=1e-10)
    assert rep.res <= 1e-10 and rep.iters <= 25
    assert rel2(N(phi, p.grid.shape), ref) <= 1e-10


def test_gpe_periodic_cluster_small(gps, ctx):
    p = synth.workload(2, n=48, count=8)
    got, ref, rep, info = _solve_pair(gps, ctx, p)
    assert rep.status == 0
    assert rel2(got, ref) <= 1e-10
    assert abs(np.sum(np.sqrt(p.eps) * got)) <= 1e-10 * np.abs(got).sum()


def test_gpe_surface_small(gps, ctx):
    p = synth.workload(3, nxy=40, nz=96, count=8)
    assert _has_solvent(p)
    got, ref, rep, info = _solve_pair(gps, ctx, p)
    assert rel2(got, ref) <= 1e-10


@pytest.mark.parametrize("wl,kw", [(1, dict(n=40)), (2, dict(n=36, count=6)),
                                   (3, dict(nxy=32, nz=96, count=6))])
def test_lpb(gps, ctx, wl, kw):
    p = synth.workload(wl, **kw)
    assert _has_solvent(p)
    if p.electrolyte is None:
        p.electrolyte = synth.Electrolyte((1, -1), (0.3, 0.3), 300.0)
    got, ref, rep, info = _solve_pair(gps, ctx, p, kind="lpb")
    assert rep.status == 0
    assert rel2(got, ref) <= 1e-10


def test_nlpb_newton_surface_small(gps, ctx):
    # nz = 96 puts the top of the box (z = 16.8 bohr) above the interface at
    # z = 10, so part of the grid is solvent and carries ionic charge.
    p = synth.workload(3, nxy=32, nz=96, count=8, kind="nlpb")
    assert _has_solvent(p)
    el = gps.make_electrolyte(p.electrolyte.z, p.electrolyte.c_molar, p.electrolyte.temperature, p.eps0)
    phi = T(np.zeros(p.grid.shape))
    opts = gps.default_opts(tol_outer=1e-11, max_iter=3000)
    rep = ctx.pb_solve(gps.grid_from(p.grid), T(p.rho), T(p.eps), el, "nlpb", phi, opts)
    ref, info = oracle.solve_nlpb(p.grid, p.rho, p.eps, p.electrolyte, p.eps0, tol=1e-11, max_iter=3000)
    assert info["converged"] and rep.status == 0
    err = rel2(N(phi, p.grid.shape), ref)
    assert err <= 1e-10, err


def test_nlpb_forcing_rules(gps, ctx):
    """Both inner-tolerance rules of the Newton outer loop (Eisenstat-Walker
    choice 2, the default, and min(forcing, F/F0)) reach the oracle's
    solution at the FP64 bar; they take different inner iterations."""
    p = synth.workload(4, n=48, count=6, margin=5.0, kind="nlpb", conc=0.5)
    el = gps.make_electrolyte(p.electrolyte.z, p.electrolyte.c_molar, p.electrolyte.temperature, p.eps0)
    ref, info = oracle.solve_nlpb(p.grid, p.rho, p.eps, p.electrolyte, p.eps0, tol=1e-11, max_iter=3000)
    assert info["converged"]
    iters = {}
    for rule in (gps.GPS_FORCING_EW2, gps.GPS_FORCING_RATIO):
        phi = T(np.zeros(p.grid.shape))
        rep = ctx.pb_solve(gps.grid_from(p.grid), T(p.rho), T(p.eps), el, "nlpb", phi,
                           gps.default_opts(tol_outer=1e-11, max_iter=3000, forcing_rule=rule))
        assert rep.status == 0
        err = rel2(N(phi, p.grid.shape), ref)
        assert err <= 1e-10, (rule, err)
        iters[rule] = rep.iters
    assert iters[gps.GPS_FORCING_EW2] != iters[gps.GPS_FORCING_RATIO]


def test_nlpb_printed_small_box(gps, ctx):
    """Algorithm 4 as printed (linear mixing) where it converges: a box
    smaller than the Debye length, weak source."""
    g = synth.Grid(16, 16, 16, 0.6, 0.6, 0.6, synth.BC_FREE)
    c = (8 * 0.6,) * 3
    eps = synth.rigid_cavity(g, [(2.0, c)], 0.6)
    rho = synth.gaussian_charges(g, [(0.002, 1.0, c)])
    el_o = synth.Electrolyte((1, -1), (0.1, 0.1), 300.0)
    el = gps.make_electrolyte((1, -1), (0.1, 0.1), 300.0, synth.EPS_WATER)
    phi = T(np.zeros(g.shape))
    opts = gps.default_opts(tol_outer=1e-13, outer_mode=gps.GPS_OUTER_PRINTED, eta=0.6, max_outer=200)
    rep = ctx.pb_solve(gps.grid_from(g), T(rho), T(eps), el, "nlpb", phi, opts)
    ref, info = oracle.solve_nlpb(g, rho, eps, el_o, synth.EPS_WATER, mode="printed", eta=0.6,
                                  tol=1e-13, max_outer=200)
    assert info["converged"] and rep.status == 0
    err = rel2(N(phi, g.shape), ref)
    assert err <= 1e-10, err


def test_ionic_charge(gps, ctx):
    g = synth.Grid(10, 12, 14, 0.5, 0.5, 0.5, synth.BC_FREE)
    rng = np.random.default_rng(15)
    phi = 0.02 * rng.standard_normal(g.shape)
    phi[0, 0, :3] = [1.0, -1.0, 0.5]      # exponent cap active
    eps = 1.0 + 77.36 * rng.random(g.shape)
    el_o = synth.Electrolyte((1, -1, 2), (0.1, 0.1, 0.05), 310.0)
    el = gps.make_electrolyte((1, -1, 2), (0.1, 0.1, 0.05), 310.0, synth.EPS_WATER)
    out = T(np.zeros(g.shape))
    ctx.ionic_charge(gps.grid_from(g), T(phi), T(eps), el, out)
    ref = oracle.pb.ionic_charge(phi, oracle.pb.exclusion_from_eps(eps, synth.EPS_WATER), el_o)
    assert relmax(N(out, g.shape), ref) < 1e-13


# ------------------------------------------------------------ modified PB --

def _steric(el, radius=3.0, packing=0.74):
    """The paper's steric parameters (p = 0.74, R = 3 angstrom) on an electrolyte."""
    return synth.Electrolyte(el.z, el.c_molar, el.temperature, radius_angstrom=(radius,) * len(el.z),
                             packing=packing)


def _gps_el(gps, el, eps0):
    return gps.make_electrolyte(el.z, el.c_molar, el.temperature, eps0,
                                radius_angstrom=el.radius_angstrom, packing=el.packing)


@pytest.mark.parametrize("wl,kw,scale", [
    (3, dict(nxy=32, nz=96, count=8, kind="nlpb"), 1.0),
    (4, dict(n=48, count=6, margin=5.0, kind="nlpb", conc=0.5), 1.0),
])
def test_mpb_against_oracle(gps, ctx, wl, kw, scale):
    """Modified PB (Eq. ionsconcMPB) by the Newton outer loop, FP64, against
    the oracle; the steric term changes the potential (it is not plain PB)."""
    p = synth.workload(wl, **kw)
    el_o = _steric(p.electrolyte)
    el = _gps_el(gps, el_o, p.eps0)
    rho = p.rho * scale
    phi = T(np.zeros(p.grid.shape))
    opts = gps.default_opts(tol_outer=1e-11, max_iter=3000)
    rep = ctx.pb_solve(gps.grid_from(p.grid), T(rho), T(p.eps), el, "mpb", phi, opts)
    ref, info = oracle.solve_nlpb(p.grid, rho, p.eps, el_o, p.eps0, tol=1e-11, max_iter=3000)
    assert info["converged"] and rep.status == 0
    if p.grid.bc == synth.BC_FREE:
        assert rep.outer_iters <= 8          # the paper reports about five (free BC)
    got = N(phi, p.grid.shape)
    err = rel2(got, ref)
    assert err <= 1e-10, err
    plain, _ = oracle.solve_nlpb(p.grid, rho, p.eps, p.electrolyte, p.eps0, tol=1e-11, max_iter=3000)
    assert rel2(got, plain) > 1e-6


def test_mpb_mixed_df64(gps, ctx):
    p = synth.workload(4, n=48, count=6, margin=5.0, kind="nlpb", conc=0.5)
    el_o = _steric(p.electrolyte)
    phi = T(np.zeros(p.grid.shape))
    opts = gps.default_opts(tol_outer=1e-10, max_iter=3000, precision=gps.GPS_MIXED_DF64)
    rep = ctx.pb_solve(gps.grid_from(p.grid), T(p.rho), T(p.eps), _gps_el(gps, el_o, p.eps0), "mpb", phi, opts)
    ref, info = oracle.solve_nlpb(p.grid, p.rho, p.eps, el_o, p.eps0, tol=1e-11, max_iter=3000)
    assert rep.status == 0 and info["converged"]
    assert 0 <= rep.fixed_point_res < 1e-8
    assert rel2(N(phi, p.grid.shape), ref) <= 1e-8


def test_ionic_charge_steric(gps, ctx):
    g = synth.Grid(10, 12, 14, 0.5, 0.5, 0.5, synth.BC_FREE)
    rng = np.random.default_rng(16)
    phi = 0.03 * rng.standard_normal(g.shape)
    phi[0, 0, :3] = [1.0, -1.0, 0.5]      # exponent cap active
    eps = 1.0 + 77.36 * rng.random(g.shape)
    el_o = synth.Electrolyte((1, -1, 2), (0.1, 0.1, 0.05), 310.0, radius_angstrom=(3.0, 2.5, 3.5),
                             packing=0.74)
    out = T(np.zeros(g.shape))
    ctx.ionic_charge(gps.grid_from(g), T(phi), T(eps), _gps_el(gps, el_o, synth.EPS_WATER), out)
    ref = oracle.pb.ionic_charge(phi, oracle.pb.exclusion_from_eps(eps, synth.EPS_WATER), el_o)
    assert relmax(N(out, g.shape), ref) < 1e-13


def test_mpb_requires_steric_parameters(gps, ctx):
    p = synth.workload(4, n=32, count=2, margin=3.0, kind="nlpb")
    el = gps.make_electrolyte(p.electrolyte.z, p.electrolyte.c_molar, p.electrolyte.temperature, p.eps0)
    with pytest.raises(gps.GpsError) as e:
        ctx.pb_solve(gps.grid_from(p.grid), T(p.rho), T(p.eps), el, "mpb", T(np.zeros(p.grid.shape)))
    assert e.value.status == gps.GPS_ERR_INVALID


def test_full_surface_mpb(gps, ctx):
    """Config-3 slab with the steric ionic charge (0.1 M, p = 0.74,
    R = 3 angstrom), FP64 at full size: the oracle's fixed-point residual of
    the full modified-PB equation at the GPU potential."""
    p = synth.workload(3, kind="nlpb")
    el_o = _steric(p.electrolyte)
    phi = T(np.zeros(p.grid.shape))
    rep = ctx.pb_solve(gps.grid_from(p.grid), T(p.rho), T(p.eps), _gps_el(gps, el_o, p.eps0), "mpb", phi,
                       gps.default_opts(tol_outer=1e-10, max_iter=2000))
    assert rep.status == 0 and rep.outer_iters > 1
    ph = N(phi, p.grid.shape)
    gam = oracle.pb.exclusion_from_eps(p.eps, p.eps0)
    rions = oracle.pb.ionic_charge(ph, gam, el_o)
    assert _fixed_point_residual(p, ph, rions=rions) < 1e-9


# ---------------------------------------------------------------- edge cases

def test_invalid_inputs(gps, ctx):
    g = synth.Grid(16, 16, 16, 0.5, 0.5, 0.5, synth.BC_FREE)
    rho, phi = T(np.zeros(g.shape)), T(np.zeros(g.shape))
    bad_eps = np.ones(g.shape)
    bad_eps[3, 4, 5] = -1.0
    with pytest.raises(gps.GpsError) as e:
        ctx.gpe_solve(gps.grid_from(g), rho, T(bad_eps), phi)
    assert e.value.status == gps.GPS_ERR_INVALID
    for dims, bc in [((7, 16, 16), synth.BC_PERIODIC), ((14, 16, 16), synth.BC_PERIODIC),
                     ((2, 16, 16), synth.BC_FREE)]:
        g2 = synth.Grid(dims[0], dims[1], dims[2], 0.5, 0.5, 0.5, bc)
        z = T(np.ones(g2.shape))
        with pytest.raises(gps.GpsError) as e:
            ctx.gpe_solve(gps.grid_from(g2), z, z, T(np.zeros(g2.shape)))
        assert e.value.status == gps.GPS_ERR_INVALID


def test_not_converged_and_zero_source(gps, ctx):
    p = synth.workload(1, n=24)
    phi = T(np.zeros(p.grid.shape))
    rep = ctx.gpe_solve(gps.grid_from(p.grid), T(p.rho), T(p.eps), phi,
                        gps.default_opts(max_iter=2), allow=(gps.GPS_ERR_NOT_CONVERGED,))
    assert rep.status == gps.GPS_ERR_NOT_CONVERGED and rep.iters == 2
    rep = ctx.gpe_solve(gps.grid_from(p.grid), T(np.zeros(p.grid.shape)), T(p.eps), phi)
    assert rep.iters == 0 and np.all(N(phi, p.grid.shape) == 0)


@pytest.mark.parametrize("bc", [synth.BC_FREE, synth.BC_SURFACE, synth.BC_PERIODIC])
def test_uniform_eps_converges_in_one_iteration(gps, ctx, bc):
    """eps = 1 everywhere: q = 0, so A M r = -4 pi r exactly (Eq. corr) and
    Algorithm 2 lands on the vacuum solution phi = S (rho - mean) in one
    iteration; phi equals the oracle's vacuum solve."""
    g = synth.Grid(24, 20, 16, 0.4, 0.45, 0.5, bc)
    rng = np.random.default_rng(31)
    rho = rng.standard_normal(g.shape)
    eps = np.ones(g.shape)
    phi = T(np.zeros(g.shape))
    rep = ctx.gpe_solve(gps.grid_from(g), T(rho), T(eps), phi, gps.default_opts(tol_abs=1e-10))
    assert rep.status == 0 and rep.iters == 1
    src = rho - rho.mean() if bc == synth.BC_PERIODIC else rho
    ref = VacuumSolver(g).apply(src)
    assert relmax(N(phi, g.shape), ref) < 1e-12


@pytest.mark.parametrize("dims", [(4096, 4, 4), (4, 4096, 4), (4, 4, 4096)])
def test_maximum_transform_length(gps, ctx, dims):
    """The longest transform the library accepts (4096 points on an axis) in
    the shared-memory kernels, one line per CTA, in the three spectrum
    precisions; one point more is rejected."""
    g = synth.Grid(dims[0], dims[1], dims[2], 0.3, 0.3, 0.3, synth.BC_PERIODIC)
    rng = np.random.default_rng(32)
    sigma = rng.standard_normal(g.shape)
    w = T(np.zeros(g.shape))
    ctx.vacuum_solve(gps.grid_from(g), T(sigma), w)
    assert relmax(N(w, g.shape), VacuumSolver(g).apply(sigma)) < 1e-12
    eps = 1.0 + 30.0 * rng.random(g.shape)
    r = rng.standard_normal(g.shape)
    f = Fields(g, eps)
    ref = f.precondition(r)
    for code, tol in ((gps.GPS_FP64, 1e-12), (gps.GPS_DF64, 1e-12), (gps.GPS_MIXED, 2e-5)):
        v = T(np.zeros(g.shape))
        ctx.precondition(gps.grid_from(g), T(f.s), T(r), v, precision=code)
        assert relmax(N(v, g.shape), ref) < tol
    big = [d * 2 if d == 4096 else d for d in dims]
    g2 = synth.Grid(big[0], big[1], big[2], 0.3, 0.3, 0.3, synth.BC_PERIODIC)
    z = T(np.zeros(g2.shape))
    with pytest.raises(gps.GpsError) as e:
        ctx.vacuum_solve(gps.grid_from(g2), z, T(np.zeros(g2.shape)))
    assert e.value.status == gps.GPS_ERR_INVALID


@pytest.mark.parametrize("bc,kind", [(synth.BC_FREE, "gpe"), (synth.BC_PERIODIC, "gpe"),
                                     (synth.BC_SURFACE, "lpb")])
def test_warm_start(gps, bc, kind):
    """opts.warm_start: after a solve with the same eps, a solve for a nearby
    rho starts from its potential and its final residual (reported warm),
    needs fewer iterations than a cold start and reaches the cold solve's
    potential (relative L2 <= 1e-10, both to ||r|| <= 1e-12 ||b||); eps
    changed anywhere gives a cold start."""
    rng = np.random.default_rng(41 + bc)
    p = synth.serving_request(rng, 32, bc, kind, h=0.45)
    g = gps.grid_from(p.grid)
    el = gps.make_electrolyte(p.electrolyte.z, p.electrolyte.c_molar, p.electrolyte.temperature, p.eps0)
    rho1 = p.rho
    rho2 = p.rho + 0.02 * np.roll(p.rho, 3, axis=2)
    tol = 1e-12 * 4 * np.pi * np.linalg.norm(rho2)
    c = gps.Context(0)
    try:
        def solve(rho, eps, warm):
            phi = T(np.zeros(p.grid.shape))
            o = gps.default_opts(tol_abs=tol, max_iter=2000, warm_start=warm)
            rep = c.pb_solve(g, T(rho), T(eps), el, kind, phi, o)
            assert rep.status == 0
            return N(phi, p.grid.shape), rep
        _, r1 = solve(rho1, p.eps, 1)
        assert r1.warm == 0
        phi_w, r2 = solve(rho2, p.eps, 1)
        assert r2.warm == 1
        phi_c, r3 = solve(rho2, p.eps, 0)
        assert r3.warm == 0
        assert r2.iters < r3.iters
        assert rel2(phi_w, phi_c) <= 1e-10
        eps3 = p.eps.copy()
        eps3.flat[123] *= 1.0 + 1e-9
        _, r4 = solve(rho2, eps3, 1)
        assert r4.warm == 0
    finally:
        c.close()


def test_deterministic_and_host_entry_point(gps, ctx):
    p = synth.workload(2, n=32, count=5)
    g = gps.grid_from(p.grid)
    a, b = T(np.zeros(p.grid.shape)), T(np.zeros(p.grid.shape))
    ctx.gpe_solve(g, T(p.rho), T(p.eps), a)
    ctx.gpe_solve(g, T(p.rho), T(p.eps), b)
    assert np.array_equal(N(a, p.grid.shape), N(b, p.grid.shape))
    h = np.zeros(p.grid.shape)
    ctx.gpe_solve_host(g, np.ascontiguousarray(p.rho), np.ascontiguousarray(p.eps), h)
    assert np.array_equal(h, N(a, p.grid.shape))


# ------------------------------------------------ full-size workloads -------

def _fixed_point_residual(p, phi, lam=None, rions=None):
    """|| M(rho [+ rho_ions] - (q + lam) phi / 4pi) - phi || / ||phi|| with the
    oracle's own operators (free and surface BC, where S is invertible): zero
    for the exact discrete solution, Eq. (corr) rearranged."""
    assert p.grid.bc != synth.BC_PERIODIC
    f = Fields(p.grid, p.eps, lam=lam)
    src = p.rho if rions is None else p.rho + rions
    g = f.precondition(src - f.qlam * phi / (4 * np.pi)) - phi
    return np.linalg.norm(g) / np.linalg.norm(phi)


def test_full_periodic_cluster_128(gps, ctx):
    """The 128^3 periodic workload timed by the benchmark, FP64: element-wise
    against the oracle."""
    p = synth.workload(2)
    phi = T(np.zeros(p.grid.shape))
    rep = ctx.gpe_solve(gps.grid_from(p.grid), T(p.rho), T(p.eps), phi, gps.default_opts(tol_abs=1e-10))
    ref, info = oracle.solve_gpe(p.grid, p.rho, p.eps, tol_abs=1e-10, max_iter=500)
    assert rep.status == 0 and abs(rep.iters - info["iters"]) <= 3
    assert rel2(N(phi, p.grid.shape), ref) <= 1e-10


def test_full_surface_lpb(gps, ctx):
    """Config-3 slab (surface BC, 160 x 160 x 256) with the linear PB term
    (0.1 M), FP64 at full size: element-wise against the oracle's Algorithm 2,
    both sides to ||r|| <= 1e-13 ||r0||; and the oracle's fixed-point residual
    of the GPU potential."""
    p = synth.workload(3, kind="lpb")
    got, ref, rep, info = _solve_pair(gps, ctx, p, kind="lpb")
    assert rep.status == 0 and abs(rep.iters - info["iters"]) <= 3
    err = rel2(got, ref)
    assert err <= 1e-10, err
    gam = oracle.pb.exclusion_from_eps(p.eps, p.eps0)
    lam = oracle.pb.linear_lambda(gam, p.electrolyte)
    assert _fixed_point_residual(p, got, lam=lam) < 1e-10


def test_full_free_union_gpe(gps, ctx):
    """Config 4's generalized Poisson problem at full size (free 256^3, the
    same 200 charges and union-of-spheres eps), FP64: element-wise against the
    oracle's Algorithm 2, both sides to ||r|| <= 1e-13 ||r0||."""
    p = synth.workload(4, kind="gpe")
    got, ref, rep, info = _solve_pair(gps, ctx, p, kind="gpe")
    assert rep.status == 0 and abs(rep.iters - info["iters"]) <= 3
    err = rel2(got, ref)
    assert err <= 1e-10, err


def _golden_nlpb(fname):
    """Oracle samples of a full-size nonlinear PB potential, written by
    tests/golden/make_full_nlpb_samples.py (oracle only)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "make_full_nlpb_samples.py")
    spec = importlib.util.spec_from_file_location("make_full_nlpb_samples", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.load(fname)


def _check_golden(ph, fname, bar):
    """Sampled values and whole-field norms of `ph` against the fixture:
    max sampled error relative to the field's largest magnitude, and the L2
    norm and largest magnitude relative to the oracle's, all <= bar."""
    shape, stats, idx, val = _golden_nlpb(fname)
    assert ph.shape == shape and idx.size > 2000
    flat = ph.ravel()
    err = float(np.max(np.abs(flat[idx] - val))) / stats["maxabs"]
    l2 = abs(float(np.sqrt(np.sum(flat * flat))) - stats["l2"]) / stats["l2"]
    mx = abs(float(np.max(np.abs(flat))) - stats["maxabs"]) / stats["maxabs"]
    assert err <= bar and l2 <= bar and mx <= bar, (err, l2, mx)


def test_full_surface_nlpb(gps, ctx):
    """Config-3 slab (surface BC, 160 x 160 x 256) with the nonlinear PB term
    (0.1 M, Newton outer loop), FP64 at full size to an outer residual of
    1e-11: element-wise at 2049 sampled points, and in L2 norm and largest
    magnitude, against the oracle's Algorithm 4 on the same inputs (stored
    samples; same forcing rule, same outer residual); and the oracle's
    fixed-point residual of the full nonlinear equation at the GPU
    potential."""
    p = synth.workload(3, kind="nlpb")
    el = gps.make_electrolyte(p.electrolyte.z, p.electrolyte.c_molar, p.electrolyte.temperature, p.eps0)
    phi = T(np.zeros(p.grid.shape))
    rep = ctx.pb_solve(gps.grid_from(p.grid), T(p.rho), T(p.eps), el, "nlpb", phi,
                       gps.default_opts(tol_outer=1e-11, max_iter=3000))
    assert rep.status == 0 and rep.outer_iters > 1
    ph = N(phi, p.grid.shape)
    _check_golden(ph, "surface_nlpb_160x160x256.txt", 1e-10)
    gam = oracle.pb.exclusion_from_eps(p.eps, p.eps0)
    rions = oracle.pb.ionic_charge(ph, gam, p.electrolyte)
    assert _fixed_point_residual(p, ph, rions=rions) < 1e-10


def test_full_free_union_nlpb_fp64(gps, ctx):
    """Config 4 at full size (free 256^3, 200 charges in a union-of-spheres
    cavity, nonlinear PB at 0.5 M), plain FP64 to an outer residual of 1e-11:
    element-wise at 2049 sampled points, and in L2 norm and largest
    magnitude, against the oracle's Algorithm 4 on the same inputs (stored
    samples; same forcing rule, same outer residual)."""
    p = synth.workload(4)
    el = gps.make_electrolyte(p.electrolyte.z, p.electrolyte.c_molar, p.electrolyte.temperature, p.eps0)
    phi = T(np.zeros(p.grid.shape))
    rep = ctx.pb_solve(gps.grid_from(p.grid), T(p.rho), T(p.eps), el, "nlpb", phi,
                       gps.default_opts(tol_outer=1e-11, max_iter=4000, precision=gps.GPS_FP64))
    assert rep.status == 0 and rep.outer_iters > 1
    _check_golden(N(phi, p.grid.shape), "free_nlpb_256.txt", 1e-10)


def test_full_free_union_nlpb_mixed(gps, ctx):
    """Config 4 at full size: free 256^3, 200 charges in a union-of-spheres
    cavity, nonlinear PB at 0.5 M, FP32 spectrum after the switch with the
    double-float spectrum as the high-precision side.  The FP64 certificate
    and the oracle's fixed-point residual of the full nonlinear equation are
    below 1e-8, and the result agrees with the plain FP64 solve (FP64
    spectrum throughout) of the same problem to 1e-8, and with the oracle's
    stored samples of the same problem to 1e-8."""
    p = synth.workload(4)
    el = gps.make_electrolyte(p.electrolyte.z, p.electrolyte.c_molar, p.electrolyte.temperature, p.eps0)
    g = gps.grid_from(p.grid)
    rho, eps = T(p.rho), T(p.eps)
    phi = T(np.zeros(p.grid.shape))
    rep = ctx.pb_solve(g, rho, eps, el, "nlpb", phi,
                       gps.default_opts(tol_outer=1e-10, max_iter=3000, precision=gps.GPS_MIXED_DF64))
    assert rep.status == 0
    assert 0 <= rep.fixed_point_res < 1e-8
    ref = T(np.zeros(p.grid.shape))
    rep_ref = ctx.pb_solve(g, rho, eps, el, "nlpb", ref,
                           gps.default_opts(tol_outer=1e-10, max_iter=3000, precision=gps.GPS_FP64))
    assert rep_ref.status == 0 and rep_ref.fp64_iters == rep_ref.iters
    ph, ph_ref = N(phi, p.grid.shape), N(ref, p.grid.shape)
    err = rel2(ph, ph_ref)
    assert err <= 1e-8, err
    _check_golden(ph, "free_nlpb_256.txt", 1e-8)
    gam = oracle.pb.exclusion_from_eps(p.eps, p.eps0)
    rions = oracle.pb.ionic_charge(ph, gam, p.electrolyte)
    assert _fixed_point_residual(p, ph, rions=rions) < 1e-8


# ------------------------------------------------------ mixed precision -----

@pytest.mark.parametrize("wl,kw,kind", [
    (4, dict(n=64, count=12, margin=6.0, kind="gpe"), "gpe"),
    (2, dict(n=48, count=8), "gpe"),
    (3, dict(nxy=32, nz=96, count=6), "lpb"),
    (2, dict(n=96, count=12), "gpe"),
])
def test_mixed_precision_error(gps, ctx, wl, kw, kind):
    """FP32 spectrum inside the FP64 PCG: relative L2 error against the FP64
    oracle <= 1e-8, with the FP64 certificate of each result below 1e-8."""
    p = synth.workload(wl, **kw)
    g = p.grid
    phi = T(np.zeros(g.shape))
    opts = gps.default_opts(tol_abs=1e-10, precision=gps.GPS_MIXED, max_iter=2000)
    if kind == "gpe":
        rep = ctx.gpe_solve(gps.grid_from(g), T(p.rho), T(p.eps), phi, opts)
        ref, _ = oracle.solve_gpe(g, p.rho, p.eps, tol_abs=0.0, tol_rel=1e-13, max_iter=2000)
    else:
        el = gps.make_electrolyte(p.electrolyte.z, p.electrolyte.c_molar, p.electrolyte.temperature, p.eps0)
        rep = ctx.pb_solve(gps.grid_from(g), T(p.rho), T(p.eps), el, "lpb", phi, opts)
        lam = oracle.pb.linear_lambda(oracle.pb.exclusion_from_eps(p.eps, p.eps0), p.electrolyte)
        ref, _ = oracle.solve_lpb(g, p.rho, p.eps, lam, tol_abs=0.0, tol_rel=1e-13, max_iter=2000)
    err = rel2(N(phi, g.shape), ref)
    assert rep.status == 0
    assert 0 < rep.fp64_iters < rep.iters
    assert 0 <= rep.fixed_point_res < 1e-8
    assert err <= 1e-8


def test_mixed_precision_nlpb(gps, ctx):
    p = synth.workload(4, n=48, count=6, margin=5.0, kind="nlpb", conc=0.5)
    el = gps.make_electrolyte(p.electrolyte.z, p.electrolyte.c_molar, p.electrolyte.temperature, p.eps0)
    phi = T(np.zeros(p.grid.shape))
    opts = gps.default_opts(tol_outer=1e-10, precision=gps.GPS_MIXED, max_iter=3000)
    rep = ctx.pb_solve(gps.grid_from(p.grid), T(p.rho), T(p.eps), el, "nlpb", phi, opts)
    ref, info = oracle.solve_nlpb(p.grid, p.rho, p.eps, p.electrolyte, p.eps0, tol=1e-11, max_iter=3000)
    assert rep.status == 0 and info["converged"]
    assert 0 <= rep.fixed_point_res < 1e-8
    assert rel2(N(phi, p.grid.shape), ref) <= 1e-8


def test_fp64_certificate(gps, ctx):
    p = synth.workload(1, n=40)
    phi = T(np.zeros(p.grid.shape))
    rep = ctx.gpe_solve(gps.grid_from(p.grid), T(p.rho), T(p.eps), phi,
                        gps.default_opts(tol_abs=0.0, tol_rel=1e-13, certify=1))
    assert 0 <= rep.fixed_point_res < 1e-12
    p2 = synth.workload(2, n=32, count=5)
    rep = ctx.gpe_solve(gps.grid_from(p2.grid), T(p2.rho), T(p2.eps), T(np.zeros(p2.grid.shape)),
                        gps.default_opts(tol_abs=0.0, tol_rel=1e-13, certify=1))
    assert 0 <= rep.fixed_point_res < 1e-12


# ----------------------------------------------------- double-float spectrum

@pytest.mark.parametrize("bc,n,h", SMALL)
def test_precondition_df64(gps, ctx, bc, n, h):
    """Spectrum passes in double-float (two floats, ~48 bits) on the FP32 pipe."""
    g = _grid(bc, n, h)
    rng = np.random.default_rng(16)
    eps = 1.0 + 30.0 * rng.random(g.shape)
    r = rng.standard_normal(g.shape)
    f = Fields(g, eps)
    v = T(np.zeros(g.shape))
    ctx.precondition(gps.grid_from(g), T(f.s), T(r), v, precision=gps.GPS_DF64)
    assert relmax(N(v, g.shape), f.precondition(r)) < 1e-12


@pytest.mark.parametrize("wl,kw,kind", [
    (1, dict(), "gpe"),
    (2, dict(n=48, count=8), "gpe"),
    (3, dict(nxy=32, nz=96, count=6), "lpb"),
])
def test_df64_solves(gps, ctx, wl, kw, kind):
    p = synth.workload(wl, **kw)
    if p.electrolyte is None:
        p.electrolyte = synth.Electrolyte((1, -1), (0.3, 0.3), 300.0)
    got, ref, rep, info = _solve_pair(gps, ctx, p, kind=kind, precision=gps.GPS_DF64)
    assert rep.status == 0
    assert rep.fp64_iters == rep.iters
    assert rel2(got, ref) <= 1e-10


def test_df64_nlpb(gps, ctx):
    p = synth.workload(3, nxy=32, nz=96, count=8, kind="nlpb")
    assert _has_solvent(p)
    el = gps.make_electrolyte(p.electrolyte.z, p.electrolyte.c_molar, p.electrolyte.temperature, p.eps0)
    phi = T(np.zeros(p.grid.shape))
    opts = gps.default_opts(tol_outer=1e-11, max_iter=3000, precision=gps.GPS_DF64)
    rep = ctx.pb_solve(gps.grid_from(p.grid), T(p.rho), T(p.eps), el, "nlpb", phi, opts)
    ref, info = oracle.solve_nlpb(p.grid, p.rho, p.eps, p.electrolyte, p.eps0, tol=1e-11, max_iter=3000)
    assert rep.status == 0
    err = rel2(N(phi, p.grid.shape), ref)
    assert err <= 1e-10, err


def test_mixed_df64(gps, ctx):
    p = synth.workload(4, n=64, count=12, margin=6.0, kind="gpe")
    phi = T(np.zeros(p.grid.shape))
    opts = gps.default_opts(tol_abs=1e-10, precision=gps.GPS_MIXED_DF64, max_iter=2000)
    rep = ctx.gpe_solve(gps.grid_from(p.grid), T(p.rho), T(p.eps), phi, opts)
    ref, _ = oracle.solve_gpe(p.grid, p.rho, p.eps, tol_abs=0.0, tol_rel=1e-13, max_iter=2000)
    assert rep.status == 0 and 0 < rep.fp64_iters < rep.iters
    assert 0 <= rep.fixed_point_res < 1e-8
    assert rel2(N(phi, p.grid.shape), ref) <= 1e-8
