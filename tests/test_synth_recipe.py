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
