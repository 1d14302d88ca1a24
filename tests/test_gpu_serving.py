"""Batched and served solves (continuous batching over pools of slots).

Each request reduces in a fixed order inside its own slot, so its potential
must be bitwise identical whether it is solved alone (gps_pb_solve_host) or
together with other requests of other sizes, boundary conditions, problems
and precisions (gps_batch_solve, gps_server_*).  One request of each kind is
also checked against the CPU oracle.
"""
import threading
import time

import numpy as np
import pytest

import oracle
import synth

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


def _requests(gps, count=10, seed=7):
    """Small requests drawn like the serving workload (edges 24/32/36)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        edge = int(rng.choice([24, 32, 36]))
        bc = int(rng.integers(0, 3))
        kind = ("gpe", "lpb", "nlpb")[int(rng.integers(0, 3))]
        p = synth.serving_request(rng, edge, bc, kind, h=0.45)
        mixed = bool(rng.integers(0, 2)) and kind != "nlpb"
        # the GPe request runs to 1e-13 relative so that it can be compared
        # with the oracle at the FP64 parity bar
        tol = dict(tol_abs=0.0, tol_rel=1e-13) if kind == "gpe" else dict(tol_abs=1e-10)
        opts = gps.default_opts(max_iter=2000, tol_outer=1e-10,
                                precision=gps.GPS_MIXED if mixed else gps.GPS_FP64, **tol)
        el = gps.make_electrolyte(p.electrolyte.z, p.electrolyte.c_molar,
                                  p.electrolyte.temperature, p.eps0)
        out.append((p, kind, opts, el))
    return out


def _alone(gps, ctx, reqs):
    res = []
    for p, kind, opts, el in reqs:
        phi = np.zeros(p.grid.npts)
        rep = ctx.pb_solve_host(gps.grid_from(p.grid), np.ascontiguousarray(p.rho.ravel()),
                                np.ascontiguousarray(p.eps.ravel()), el, kind, phi, opts)
        res.append((phi, rep))
    return res


def test_batch_identical_to_alone(gps, ctx):
    reqs = _requests(gps)
    alone = _alone(gps, ctx, reqs)
    keep, rs = [], []
    for p, kind, opts, el in reqs:
        rho = np.ascontiguousarray(p.rho.ravel())
        eps = np.ascontiguousarray(p.eps.ravel())
        phi = np.full(p.grid.npts, np.nan)
        keep.append((rho, eps, phi))
        rs.append(gps.make_request(gps.grid_from(p.grid), kind, rho, eps, phi, el, opts))
    reps = gps.batch_solve(ctx, rs)
    for (phi_a, rep_a), (_, _, phi_b), rep_b in zip(alone, keep, reps):
        assert rep_b.status == 0 and rep_a.status == 0
        assert rep_a.iters == rep_b.iters
        assert np.array_equal(phi_a, phi_b)


def test_batch_against_oracle(gps, ctx):
    g = synth.Grid(32, 32, 32, 0.45, 0.45, 0.45, synth.BC_PERIODIC)
    rng = np.random.default_rng(3)
    p = synth.serving_request(rng, 32, synth.BC_PERIODIC, "gpe", h=0.45)
    q = synth.serving_request(rng, 24, synth.BC_FREE, "lpb", h=0.45)
    keep, rs = [], []
    for pr, kind in ((p, "gpe"), (q, "lpb")):
        rho = np.ascontiguousarray(pr.rho.ravel())
        eps = np.ascontiguousarray(pr.eps.ravel())
        phi = np.zeros(pr.grid.npts)
        keep.append(phi)
        el = gps.make_electrolyte(pr.electrolyte.z, pr.electrolyte.c_molar, 300.0, pr.eps0)
        rs.append(gps.make_request(gps.grid_from(pr.grid), kind, rho, eps, phi, el,
                                   gps.default_opts(tol_abs=0.0, tol_rel=1e-13, max_iter=3000)))
    gps.batch_solve(ctx, rs)
    ref_p, _ = oracle.solve_gpe(p.grid, p.rho, p.eps, tol_abs=0.0, tol_rel=1e-13, max_iter=3000)
    lam = oracle.pb.linear_lambda(oracle.pb.exclusion_from_eps(q.eps, q.eps0), q.electrolyte)
    ref_q, _ = oracle.solve_lpb(q.grid, q.rho, q.eps, lam, tol_abs=0.0, tol_rel=1e-13, max_iter=3000)
    for got, ref in ((keep[0], ref_p), (keep[1], ref_q)):
        got = got.reshape(ref.shape)
        assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_batch_with_wire_requests(gps, ctx):
    """Wire-BC requests (three of one grid, so their pool holds several slots)
    batched with a periodic and a free request: each potential bitwise equal
    to its single solve; the wire GPe one also against the oracle."""
    rng = np.random.default_rng(12)
    reqs = []
    for kind, mixed in (("gpe", False), ("lpb", True), ("nlpb", False)):
        p = synth.wire_chain(n=24, nz=32, kind=kind)
        # the GPe request runs to 1e-13 relative so that it can be compared
        # with the oracle at the FP64 parity bar
        tol = dict(tol_abs=0.0, tol_rel=1e-13) if kind == "gpe" else dict(tol_abs=1e-10)
        opts = gps.default_opts(max_iter=2000, tol_outer=1e-10,
                                precision=gps.GPS_MIXED if mixed else gps.GPS_FP64, **tol)
        el = gps.make_electrolyte(p.electrolyte.z, p.electrolyte.c_molar, p.electrolyte.temperature, p.eps0)
        reqs.append((p, kind, opts, el))
    for bc, kind in ((synth.BC_PERIODIC, "gpe"), (synth.BC_FREE, "lpb")):
        p = synth.serving_request(rng, 32, bc, kind, h=0.45)
        el = gps.make_electrolyte(p.electrolyte.z, p.electrolyte.c_molar, p.electrolyte.temperature, p.eps0)
        reqs.append((p, kind, gps.default_opts(tol_abs=1e-10, max_iter=2000), el))
    alone = _alone(gps, ctx, reqs)
    keep, rs = [], []
    for p, kind, opts, el in reqs:
        rho = np.ascontiguousarray(p.rho.ravel())
        eps = np.ascontiguousarray(p.eps.ravel())
        phi = np.full(p.grid.npts, np.nan)
        keep.append((rho, eps, phi))
        rs.append(gps.make_request(gps.grid_from(p.grid), kind, rho, eps, phi, el, opts))
    reps = gps.batch_solve(ctx, rs)
    for (phi_a, rep_a), (_, _, phi_b), rep_b in zip(alone, keep, reps):
        assert rep_b.status == 0 and rep_a.status == 0 and rep_a.iters == rep_b.iters
        assert np.array_equal(phi_a, phi_b)
    p = reqs[0][0]
    ref, _ = oracle.solve_gpe(p.grid, p.rho, p.eps, tol_abs=0.0, tol_rel=1e-13, max_iter=2000)
    got = keep[0][2].reshape(ref.shape)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= 1e-10, err


def test_server_stream_identical_to_alone(gps, ctx):
    reqs = _requests(gps, count=12, seed=11)
    alone = _alone(gps, ctx, reqs)
    srv = gps.Server(0, hbm_budget_bytes=8 << 30)
    rng = np.random.default_rng(5)
    tickets, keep = [], []

    def producer():
        for p, kind, opts, el in reqs:
            rho = np.ascontiguousarray(p.rho.ravel())
            eps = np.ascontiguousarray(p.eps.ravel())
            phi = np.full(p.grid.npts, np.nan)
            keep.append((rho, eps, phi))
            r = gps.make_request(gps.grid_from(p.grid), kind, rho, eps, phi, el, opts)
            tickets.append(srv.submit(r, keep=keep[-1]))
            time.sleep(float(rng.exponential(0.003)))   # Poisson arrivals

    th = threading.Thread(target=producer)
    th.start()
    th.join()
    results = [srv.wait(t, timeout=300) for t in tickets]
    stats = srv.stats()
    srv.close()
    for (phi_a, rep_a), (_, _, phi_b), (status, rep_b) in zip(alone, keep, results):
        assert status == 0
        assert rep_b.time_ms > 0
        assert np.array_equal(phi_a, phi_b)
    assert stats["max_concurrent"] >= 2


def _bench_requests(gps, count=9, seed=1005):
    """Requests drawn like the benchmark's serving stream (h = 0.3, edges 48,
    64 and 96, every BC and problem), all on the mixed-precision path the
    benchmark serves: double-float spectrum, FP32 after the switch, FP64
    certificate; nonlinear PB included."""
    rng = np.random.default_rng(seed)
    out = []
    kinds = ("gpe", "lpb", "nlpb")
    for i in range(count):
        edge = (48, 64, 96)[i % 3]
        bc = int(rng.integers(0, 3))
        kind = kinds[(i // 3) % 3]
        p = synth.serving_request(rng, edge, bc, kind)
        opts = gps.default_opts(tol_abs=1e-10, tol_outer=1e-10, max_iter=3000,
                                precision=gps.GPS_MIXED_DF64)
        el = gps.make_electrolyte(p.electrolyte.z, p.electrolyte.c_molar, 300.0, p.eps0)
        out.append((p, kind, opts, el))
    return out


def test_server_mixed_df64_stream_identical_to_alone(gps, ctx):
    """The benchmark's serving configuration: every request (GPe, linear and
    nonlinear PB, edges 48-96) on GPS_MIXED_DF64, arriving while others are on
    the GPU, gives the bitwise result of its single solve, carries an FP64
    certificate below 1e-8, and the smallest nonlinear one matches the
    oracle's FP64 solution to 1e-8."""
    reqs = _bench_requests(gps)
    alone = _alone(gps, ctx, reqs)
    srv = gps.Server(0, hbm_budget_bytes=16 << 30)
    rng = np.random.default_rng(6)
    tickets, keep = [], []

    def producer():
        for p, kind, opts, el in reqs:
            rho = np.ascontiguousarray(p.rho.ravel())
            eps = np.ascontiguousarray(p.eps.ravel())
            phi = np.full(p.grid.npts, np.nan)
            keep.append((rho, eps, phi))
            r = gps.make_request(gps.grid_from(p.grid), kind, rho, eps, phi, el, opts)
            tickets.append(srv.submit(r, keep=keep[-1]))
            time.sleep(float(rng.exponential(0.02)))

    th = threading.Thread(target=producer)
    th.start()
    th.join()
    results = [srv.wait(t, timeout=300) for t in tickets]
    stats = srv.stats()
    srv.close()
    for (phi_a, rep_a), (_, _, phi_b), (status, rep_b) in zip(alone, keep, results):
        assert status == 0 and rep_a.status == 0
        assert rep_a.iters == rep_b.iters
        assert 0 <= rep_b.fixed_point_res < 1e-8
        assert np.array_equal(phi_a, phi_b)
    assert stats["max_concurrent"] >= 2
    nl = [i for i, r in enumerate(reqs) if r[1] == "nlpb"]
    i = min(nl, key=lambda k: reqs[k][0].grid.npts)
    p = reqs[i][0]
    ref, info = oracle.solve_nlpb(p.grid, p.rho, p.eps, p.electrolyte, p.eps0, tol=1e-11, max_iter=3000)
    assert info["converged"]
    got = keep[i][2].reshape(ref.shape)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= 1e-8, err


def test_server_admission_under_budget(gps):
    """A budget that holds one small pool at a time still completes every
    request (pools are evicted when idle); a budget below one pool fails the
    request with GPS_ERR_NOMEM instead of hanging."""
    rng = np.random.default_rng(9)
    a = synth.serving_request(rng, 24, synth.BC_PERIODIC, "gpe", h=0.45)
    b = synth.serving_request(rng, 32, synth.BC_FREE, "gpe", h=0.45)
    srv = gps.Server(0, hbm_budget_bytes=64 << 20, max_slots=2)
    keep, tickets = [], []
    for p in (a, b, a, b):
        rho = np.ascontiguousarray(p.rho.ravel())
        eps = np.ascontiguousarray(p.eps.ravel())
        phi = np.zeros(p.grid.npts)
        keep.append(phi)
        tickets.append(srv.submit(gps.make_request(gps.grid_from(p.grid), "gpe", rho, eps, phi),
                                  keep=(rho, eps, phi)))
    out = [srv.wait(t, timeout=300) for t in tickets]
    srv.close()
    assert all(s == 0 for s, _ in out)
    assert np.array_equal(keep[0], keep[2]) and np.array_equal(keep[1], keep[3])
    tiny = gps.Server(0, hbm_budget_bytes=1 << 20)
    rho = np.ascontiguousarray(a.rho.ravel())
    eps = np.ascontiguousarray(a.eps.ravel())
    phi = np.zeros(a.grid.npts)
    t = tiny.submit(gps.make_request(gps.grid_from(a.grid), "gpe", rho, eps, phi), keep=(rho, eps, phi))
    status, _ = tiny.wait(t, timeout=300)
    tiny.close()
    assert status == gps.GPS_ERR_NOMEM


@pytest.mark.parametrize("bc,kind", [(1, "gpe"), (2, "lpb"), (0, "gpe")])
def test_server_warm_start(gps, bc, kind):
    """opts.warm_start on served requests (GPe and linear PB): a request whose
    eps equals, value by value, that of the last warm-start request completed
    in its pool starts from that request's potential and final residual
    (reported warm), needs fewer iterations than the same request served
    cold, and reaches the cold result (relative L2 <= 1e-10, both to
    ||r|| <= 1e-12 ||b||); a request that does not ask, and one with eps
    changed anywhere, start cold."""
    rng = np.random.default_rng(61 + bc)
    p = synth.serving_request(rng, 32, bc, kind, h=0.45)
    g = gps.grid_from(p.grid)
    el = gps.make_electrolyte(p.electrolyte.z, p.electrolyte.c_molar, p.electrolyte.temperature, p.eps0)
    rho1 = p.rho
    rho2 = p.rho + 0.02 * np.roll(p.rho, 3, axis=2)
    tol = 1e-12 * 4 * np.pi * np.linalg.norm(rho2)
    srv = gps.Server(0, hbm_budget_bytes=4 << 30)
    try:
        def serve(rho, eps, warm):
            rho_h = np.ascontiguousarray(rho.ravel())
            eps_h = np.ascontiguousarray(eps.ravel())
            phi = np.full(p.grid.npts, np.nan)
            o = gps.default_opts(tol_abs=tol, max_iter=2000, warm_start=warm)
            t = srv.submit(gps.make_request(g, kind, rho_h, eps_h, phi, el, o), keep=(rho_h, eps_h, phi))
            status, rep = srv.wait(t, timeout=120)
            assert status == 0
            return phi, rep
        _, r1 = serve(rho1, p.eps, 1)
        assert r1.warm == 0
        phi_w, r2 = serve(rho2, p.eps, 1)
        assert r2.warm == 1
        phi_c, r3 = serve(rho2, p.eps, 0)
        assert r3.warm == 0
        assert r2.iters < r3.iters
        err = np.linalg.norm(phi_w - phi_c) / np.linalg.norm(phi_c)
        assert err <= 1e-10, err
        eps3 = p.eps.copy()
        eps3.flat[123] *= 1.0 + 1e-9
        _, r4 = serve(rho2, eps3, 1)
        assert r4.warm == 0
    finally:
        srv.close()
