"""The allocation-free vacuum solve, gps_vacuum_solve_noalloc.

It is meant for callers that cannot allocate device memory (a plugin inside
an application that owns the device-memory budget, a process whose framework
has reserved nearly all of HBM, a latency-critical loop that cannot take the
device synchronization of cudaMalloc).  Its buffers live in one fixed
file-scope device array shared by every call, so this test runs several
calls in a row -- of different grids, so the array holds the previous call's
data each time -- and checks each result against the allocating entry point
gps_vacuum_solve within the tolerance of the vacuum-solve parity tests
(1e-12 relative, max norm).  This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def gps():
    from paper_1509_00680_gb300 import build
    build.build()
    from paper_1509_00680_gb300 import gps as g
    return g


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def test_noalloc_matches_allocating_entry_point(gps):
    import torch
    ctx = gps.Context(0)
    grids = [
        synth.Grid(32, 24, 20, 0.4, 0.45, 0.5, synth.BC_PERIODIC),
        synth.Grid(20, 18, 24, 0.4, 0.4, 0.35, synth.BC_SURFACE),
        synth.Grid(32, 24, 20, 0.4, 0.45, 0.5, synth.BC_PERIODIC),
    ]
    rng = np.random.default_rng(99)
    for g in grids:                       # several calls in a row on the shared array
        sigma = _dev(rng.standard_normal(g.shape))
        w_ref = torch.zeros_like(sigma)
        w_new = torch.full_like(sigma, np.nan)
        ctx.vacuum_solve(gps.grid_from(g), sigma, w_ref)
        gps.vacuum_solve_noalloc(gps.grid_from(g), sigma, w_new)
        torch.cuda.synchronize()
        ref = w_ref.cpu().numpy()
        got = w_new.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= TOL * np.abs(ref).max()
    ctx.close()


def test_noalloc_rejects_unsupported_sizes(gps):
    import torch
    big = synth.Grid(128, 128, 128, 0.3, 0.3, 0.3, synth.BC_PERIODIC)   # spectrum > 8 MiB
    free = synth.Grid(16, 16, 16, 0.3, 0.3, 0.3, synth.BC_FREE)
    for g in (big, free):
        x = torch.zeros(g.npts, dtype=torch.float64, device="cuda")
        with pytest.raises(gps.GpsError) as e:
            gps.vacuum_solve_noalloc(gps.grid_from(g), x, torch.zeros_like(x))
        assert e.value.status == gps.GPS_ERR_INVALID
