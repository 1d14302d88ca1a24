"""GPU parity of the DFT-facing quantities (sccs dielectric, polarization
charge, v_eps, electrostatic energy) against the oracle, element by element on
the same seeded inputs, on every boundary condition; and Gauss's law for the
polarization charge of a full-size GPU solution."""
import numpy as np
import pytest

import oracle
import synth
from oracle import dft

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


GRIDS = [
    synth.Grid(12, 10, 16, 0.5, 0.45, 0.4, synth.BC_FREE),
    synth.Grid(16, 12, 10, 0.5, 0.5, 0.6, synth.BC_PERIODIC),
    synth.Grid(16, 12, 10, 0.5, 0.5, 0.5, synth.BC_SURFACE),
    synth.Grid(12, 10, 16, 0.5, 0.45, 0.4, synth.BC_WIRE),
    synth.Grid(30, 15, 20, 0.3, 0.4, 0.35, synth.BC_FREE),    # ragged, odd ny
]


def _fields(g, seed):
    rng = np.random.default_rng(seed)
    eps = 1.0 + 40.0 * rng.random(g.shape)
    return rng.standard_normal(g.shape), eps, rng.standard_normal(g.shape)


def test_sccs_eps(gps, ctx):
    rng = np.random.default_rng(3)
    rho_e = 10.0 ** rng.uniform(-6, 0, size=20000)
    rho_e[:4] = [5e-3, 1e-4, 5e-3 * (1 - 1e-12), 1e-4 * (1 + 1e-12)]
    eps, deps = T(np.zeros_like(rho_e)), T(np.zeros_like(rho_e))
    ctx.sccs_eps(T(rho_e), eps, deps)
    e_ref, d_ref = dft.sccs_eps(rho_e)
    assert relmax(N(eps, rho_e.shape), e_ref) < 1e-14
    assert relmax(N(deps, rho_e.shape), d_ref) < 1e-13
    only = T(np.zeros_like(rho_e))
    ctx.sccs_eps(T(rho_e), only, None, rho_max=1e-2, rho_min=1e-5, eps0=35.7)
    assert relmax(N(only, rho_e.shape), dft.sccs_eps(rho_e, 1e-2, 1e-5, 35.7)[0]) < 1e-14


@pytest.mark.parametrize("g", GRIDS, ids=lambda g: "%s_%dx%dx%d" % (synth.BC_NAMES[g.bc], g.nx, g.ny, g.nz))
def test_polarization_charge(gps, ctx, g):
    rho, eps, phi = _fields(g, 7)
    out = T(np.zeros(g.shape))
    ctx.polarization_charge(gps.grid_from(g), T(rho), T(eps), T(phi), out)
    assert relmax(N(out, g.shape), dft.polarization_charge(g, rho, eps, phi)) < 1e-12


@pytest.mark.parametrize("g", GRIDS, ids=lambda g: "%s_%dx%dx%d" % (synth.BC_NAMES[g.bc], g.nx, g.ny, g.nz))
def test_v_eps_and_energy(gps, ctx, g):
    rho, eps, phi = _fields(g, 8)
    deps = np.where(np.random.default_rng(9).random(g.shape) < 0.5, 0.0, -np.abs(rho))
    out = T(np.zeros(g.shape))
    ctx.v_eps(gps.grid_from(g), T(deps), T(phi), out)
    assert relmax(N(out, g.shape), dft.v_eps(g, deps, phi)) < 1e-12
    e1, e2 = ctx.electrostatic_energy(gps.grid_from(g), T(rho), T(eps), T(phi))
    r1, r2 = dft.electrostatic_energy(g, rho, eps, phi)
    assert abs(e1 - r1) < 1e-12 * abs(r1) and abs(e2 - r2) < 1e-12 * abs(r2)


def test_gauss_law_of_gpu_solution(gps, ctx):
    """The free-BC single-cavity workload (64^3, Q = 1 at the centre of a
    19.2 bohr box): the GPU potential's polarization charge makes the total
    charge Q / eps0 (to the discretization error of h = 0.3, 7.7e-4 Q; see the
    oracle pins).  The two energy forms differ by the field energy outside
    the box, which (1/8 pi) sum eps |grad phi|^2 does not see: positive and
    below Q^2 / (2 eps0 R), R = 9.6 bohr to the nearest face (the energy
    outside the inscribed sphere), up to discretization (1e-3 of E)."""
    p = synth.workload(1)
    gr = gps.grid_from(p.grid)
    phi = T(np.zeros(p.grid.shape))
    ctx.gpe_solve(gr, T(p.rho), T(p.eps), phi, gps.default_opts(tol_abs=1e-11))
    pol = T(np.zeros(p.grid.shape))
    ctx.polarization_charge(gr, T(p.rho), T(p.eps), phi, pol)
    dv = p.grid.hx ** 3
    Q = float(np.sum(p.rho)) * dv
    tot = (float(np.sum(p.rho)) + float(N(pol, p.grid.shape).sum())) * dv
    assert abs(tot - Q / p.eps0) < 2e-3 * Q
    e1, e2 = ctx.electrostatic_energy(gr, T(p.rho), T(p.eps), phi)
    R = p.grid.nx // 2 * p.grid.hx
    assert 0.0 < e1 - e2 < Q * Q / (2 * p.eps0 * R) + 1e-3 * e1


def test_invalid_arguments(gps, ctx):
    x = T(np.full(10, 1e-3))
    for kw in (dict(rho_max=1e-4, rho_min=1e-3), dict(rho_min=0.0), dict(eps0=1.0)):
        with pytest.raises(gps.GpsError):
            ctx.sccs_eps(x, T(np.zeros(10)), None, **kw)
    g = synth.Grid(16, 6, 16, 0.5, 0.5, 0.5, synth.BC_PERIODIC)   # a periodic axis < 8 points
    z = T(np.zeros(g.shape))
    with pytest.raises(gps.GpsError):
        ctx.polarization_charge(gps.grid_from(g), z, T(np.ones(g.shape)), z, T(np.zeros(g.shape)))
