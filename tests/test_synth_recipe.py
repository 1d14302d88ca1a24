"""The serving-request recipe yields well-posed problems: on every free axis
eps is flat (equal to the solvent value) across the faces, so the flat
continuation of eps used for q is exact there, and solvent surrounds the
solute.  A small surface-BC request, the smallest box of the serving tests,
converges in the oracle's PCG."""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("edge,bc", [(24, synth.BC_FREE), (24, synth.BC_SURFACE), (32, synth.BC_SURFACE),
                                     (24, synth.BC_PERIODIC), (48, synth.BC_FREE)])
def test_request_eps_flat_on_free_faces(edge, bc):
    rng = np.random.default_rng(100 + edge + bc)
    for _ in range(3):
        p = synth.serving_request(rng, edge, bc, "gpe", h=0.45)
        per = p.grid.periodic_axes()
        # array axes are (z, y, x); grid axes (x, y, z)
        for a in range(3):
            if per[a]:
                continue
            ax = 2 - a
            for face in (0, -1):
                f = np.take(p.eps, face, axis=ax)
                assert np.allclose(f, p.eps0, rtol=0, atol=1e-3 * p.eps0)
        gam = oracle.pb.exclusion_from_eps(p.eps, p.eps0)
        assert (gam > 0.5).mean() >= 0.5
        assert abs(sum(q for q, _, _ in p.charges)) == 0


def test_small_surface_request_converges():
    rng = np.random.default_rng(7)
    p = synth.serving_request(rng, 24, synth.BC_SURFACE, "gpe", h=0.45)
    phi, info = oracle.solve_gpe(p.grid, p.rho, p.eps, tol_abs=1e-10, max_iter=500)
    assert info["converged"]


@pytest.mark.parametrize("n,nz", [(24, 32), (32, 48), (128, 256)])
def test_wire_chain_recipe(n, nz):
    """The wire chain keeps eps at the solvent value on the free x and y faces,
    places its cavities on the box axis evenly along the periodic z axis, and
    carries q/2 per cavity with q alternating in sign along the chain (a net
    0.5 per cell for an odd number of cavities, 0 for an even one)."""
    p = synth.wire_chain(n=n, nz=nz, count=8 if n == 128 else 3)
    assert p.grid.bc == synth.BC_WIRE and p.grid.periodic_axes() == (False, False, True)
    for ax in (1, 2):                      # array axes y and x (the free ones)
        for face in (0, -1):
            assert np.allclose(np.take(p.eps, face, axis=ax), p.eps0, rtol=0, atol=1e-3 * p.eps0)
    zs = [c[2] for _, c in p.spheres]
    L = p.grid.nz * p.grid.hz
    assert np.allclose(np.diff(zs), L / len(zs))
    assert abs(sum(q for q, _, _ in p.charges) - (0.5 if len(zs) % 2 else 0.0)) < 1e-12


def test_manufactured_recipe_matches_its_definition():
    """rho of the manufactured test is -(1/4pi) div eps grad phi: checked with
    order-16 differences of the stored phi and eps away from the box faces
    (discretization error only), and phi_exact is the normalized Gaussian."""
    import math
    p = synth.manufactured(n=64, L=10.0)
    g = p.grid
    phi, eps = p.phi_exact, p.eps
    gx, gy, gz = oracle.fd16.gradient(phi, g)
    div = (oracle.fd16.gradient(eps * gx, g)[0] + oracle.fd16.gradient(eps * gy, g)[1]
           + oracle.fd16.gradient(eps * gz, g)[2])
    inner = (slice(10, -10),) * 3
    err = np.abs(-div[inner] / (4 * math.pi) - p.rho[inner]).max()
    assert err < 2e-3 * np.abs(p.rho).max()
    assert abs(phi.max() - (2 * math.pi * 0.25) ** -1.5) < 1e-12
