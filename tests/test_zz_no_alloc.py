"""The allocation-free vacuum solve, gps_vacuum_solve_noalloc.

It is meant for callers that cannot allocate device memory (a plugin inside
an application that owns the device-memory budget, a process whose framework
has reserved nearly all of HBM, a latency-critical loop that cannot take the
device synchronization of cudaMalloc).  Its buffers live in one fixed
file-scope device array shared by every call, so these tests run several
calls in a row -- of different grids, so the array holds the previous call's
data each time -- and check each result against the allocating entry point
gps_vacuum_solve and against the CPU oracle's vacuum solve, within the
tolerance of the vacuum-solve parity tests (1e-12 relative, max norm).
The grids include the largest documented one (periodic 96^3), a grid with
short rows and many of them (8 x 256 x 256: the untuned line count of the
x passes would exceed the kernels' supported range without its clamp) and
one with a length-4 y axis (480 x 4 x 360: likewise for the y columns).
This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth
from oracle.green import VacuumSolver

TOL = 1e-12
SCRATCH_BYTES = 8 << 20


@pytest.fixture(scope="module")
def gps():
    from paper_1509_00680_gb300 import build
    build.build()
    from paper_1509_00680_gb300 import gps as g
    return g


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def _relmax(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def scratch_need(g):
    """Bytes of the fixed array a grid needs, by the layout the header
    states (twiddles, octant table, spectrum; 256-byte aligned parts)."""
    al = lambda b: (b + 255) // 256 * 256
    Px, Py = g.nx, g.ny
    Pz = 2 * g.nz if g.bc == synth.BC_SURFACE else g.nz
    Hx = Px // 2 + 1
    Hp = Hx + Hx % 2                  # even row pitch of the spectrum
    return (al(16 * Px) + al(16 * Py) + al(16 * Pz) + al(8 * Hx * (Py // 2 + 1) * (Pz // 2 + 1))
            + 16 * Hp * Py * g.nz)


GRIDS = [
    synth.Grid(32, 24, 20, 0.4, 0.45, 0.5, synth.BC_PERIODIC),
    synth.Grid(20, 18, 24, 0.4, 0.4, 0.35, synth.BC_SURFACE),
    synth.Grid(96, 96, 96, 0.3, 0.3, 0.3, synth.BC_PERIODIC),      # the documented maximum
    synth.Grid(8, 256, 256, 0.3, 0.3, 0.3, synth.BC_PERIODIC),     # short rows, many of them
    synth.Grid(480, 4, 360, 0.3, 0.3, 0.3, synth.BC_PERIODIC),     # length-4 y columns
    synth.Grid(32, 24, 20, 0.4, 0.45, 0.5, synth.BC_PERIODIC),
]


def test_layout_sizes():
    assert scratch_need(synth.Grid(96, 96, 96, 0.3, 0.3, 0.3, synth.BC_PERIODIC)) == 8318720
    for g in GRIDS:
        assert scratch_need(g) <= SCRATCH_BYTES


@pytest.mark.gpu
def test_noalloc_matches_allocating_entry_point_and_oracle(gps):
    import torch
    ctx = gps.Context(0)
    rng = np.random.default_rng(99)
    for g in GRIDS:                       # several calls in a row on the shared array
        sig = rng.standard_normal(g.shape)
        sigma = _dev(sig)
        w_ref = torch.zeros_like(sigma)
        w_new = torch.full_like(sigma, np.nan)
        ctx.vacuum_solve(gps.grid_from(g), sigma, w_ref)
        gps.vacuum_solve_noalloc(gps.grid_from(g), sigma, w_new)
        torch.cuda.synchronize()
        ref = w_ref.cpu().numpy().reshape(g.shape)
        got = w_new.cpu().numpy().reshape(g.shape)
        assert np.all(np.isfinite(got))
        assert _relmax(got, ref) <= TOL
        assert _relmax(got, VacuumSolver(g).apply(sig)) <= TOL
    ctx.close()


@pytest.mark.gpu
def test_noalloc_allocates_no_device_memory(gps):
    """Free device memory is the same before and after a sequence of calls
    of different grids (after one warm-up call, which may load the module)."""
    import torch
    rng = np.random.default_rng(7)
    bufs = []
    for g in GRIDS:
        sigma = _dev(rng.standard_normal(g.shape))
        bufs.append((g, sigma, torch.empty_like(sigma)))
    g0, s0, w0 = bufs[0]
    gps.vacuum_solve_noalloc(gps.grid_from(g0), s0, w0)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        for g, sigma, w in bufs:
            gps.vacuum_solve_noalloc(gps.grid_from(g), sigma, w)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


@pytest.mark.gpu
def test_noalloc_rejects_unsupported_sizes(gps):
    import torch
    over = [
        synth.Grid(96, 96, 100, 0.3, 0.3, 0.3, synth.BC_PERIODIC),    # just above the maximum
        synth.Grid(100, 100, 100, 0.3, 0.3, 0.3, synth.BC_PERIODIC),
        synth.Grid(128, 128, 128, 0.3, 0.3, 0.3, synth.BC_PERIODIC),
    ]
    for g in over:
        assert scratch_need(g) > SCRATCH_BYTES
    free = synth.Grid(16, 16, 16, 0.3, 0.3, 0.3, synth.BC_FREE)
    odd = synth.Grid(16, 14, 16, 0.3, 0.3, 0.3, synth.BC_PERIODIC)  # 14 = 2 x 7 does not factor
    for g in over + [free, odd]:
        x = torch.zeros(g.npts, dtype=torch.float64, device="cuda")
        with pytest.raises(gps.GpsError) as e:
            gps.vacuum_solve_noalloc(gps.grid_from(g), x, torch.zeros_like(x))
        assert e.value.status == gps.GPS_ERR_INVALID
