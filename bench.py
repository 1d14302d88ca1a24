"""Benchmark: nonlinear Poisson-Boltzmann solve of the free-BC 256^3 workload.

One step = one complete solve through the C ABI (gps_pb_solve, kind NLPB):
setup of s, sqrt(eps) and q, then the Newton outer loop of Algorithm 4 with
Algorithm 2 inside, to an outer residual <= 1e-10, on the mixed-precision
path (double-float spectrum, FP32 spectrum once ||r|| <= 1e-2 ||r_ref||,
FP64 vectors, dot products and ionic term, FP64 certificate of the result),
inputs resident in HBM.  Workload: free BC, 256^3 points at h = 0.3 bohr,
200 Gaussian charges in a union-of-spheres cavity, 1:1 electrolyte at 0.5 M.
The value is PCG grid-point iterations per second (grid points x PCG
iterations / solve time) aggregated over ranks; solves/s, the plain FP64
solve of the same problem (solves/s and the error of the mixed result
against it) and the end-to-end rate through gps_pb_solve_host go beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the reference implementation of the
method written for the tests) on the host cores, each step a bounded sample
of the same workload: setup plus a fixed number of PCG iterations of the
first Newton step's inner solve.

Under torchrun each rank solves its own replica of the workload on its own
GPU (the solve does not shard; "replicas only"), timing is the max over
ranks, and the value is the total over ranks.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "free_nlpb_256"
METRIC = ("PCG grid-pt*iter/s, nonlinear PB (free 256^3, 200 charges, union of spheres, 0.5 M), "
          "mixed precision certified <= 1e-8 (solves/s and the plain FP64 path beside it)")
UNIT = "grid-pt*iter/s"
L2_FLUSH_BYTES = 512 << 20
TOL_OUTER = 1e-10


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# How the GPU arm computes the headline (a property of the arm, not of the
# workload: it is reported beside `config`, which both arms share).
PRECISION = ("mixed: df64 spectrum, FP32 spectrum once ||r|| <= 1e-2 ||r_ref||; FP64 vectors, "
             "dots, alpha/beta and ionic term; FP64 certificate")


def config_dict():
    """The headline workload, identical in both arms' lines."""
    return {"workload": WORKLOAD, "grid": [256, 256, 256], "h_bohr": 0.3, "bc": "free",
            "charges": 200, "eps0": 78.36, "cavity": "union of erf spheres (d_i = 1.2 U[2.5, 3.5], Delta 0.5)",
            "problem": "nonlinear PB (Eq. PBe), Newton outer loop of Algorithm 4 around Algorithm 2",
            "electrolyte": "1:1, 0.5 mol/L, 300 K, ion exclusion = cavity function",
            "tol_outer": TOL_OUTER,
            "l2_flush": "inputs larger than L2 (each FP64 field 134 MB) and a 512 MiB buffer written "
                        "between timed steps",
            "parallelism": "replicas"}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index, path=None):
        self.dev = device_index
        self.proc = None
        self.path = path or os.path.join(tempfile.gettempdir(), "gps_bench_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# FP64 FMA units: 152 SMs x 2 DFMA/clk (measured 600 GFMA/s on this GPU, see
# --fp64-peak) at the 2070 MHz maximum SM clock, 2 flop per FMA.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# FP32 issue rate: 152 SMs x 128 FP32 lanes x 2.07 GHz (an FMA is one instruction).
FP32_PEAK_TINST = 152 * 128 * 2.070e9 / 1e12
# FP32 instructions per double-float operation as the spectrum passes implement
# them: an addition is the TwoSum of the high parts plus the sum of the low
# parts (8), a product the TwoProd of the high parts by FMA plus the two cross
# terms (4).
DF64_ADD_INST, DF64_MUL_INST = 8, 4

# dram__bytes_read.sum + dram__bytes_write.sum per launch of a kernel from one
# ncu capture, valid only for the kernel source it was taken with (the SHA-256
# of the listed files, first 16 hex digits); otherwise the line reports null.
NCU_TRAFFIC = {
    # k_col<dfc, 512, 2, 1>, free 256^3: 796.9 MB read + 505.3 MB written per launch
    "z_df64": {"bytes": 1302184960, "files": ['fft_col.cu', 'fft_common.cuh', 'device_util.cuh', 'gps_internal.h'], "sha": '1076a7d09e65df31'},
}


def source_sha(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1509_00680_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kind):
    rec = NCU_TRAFFIC.get(kind)
    if not rec:
        return None
    try:
        return rec["bytes"] if source_sha(rec["files"]) == rec["sha"] else None
    except OSError:
        return None


def pass_geometry(grid):
    free = grid.bc == 0
    fz = grid.bc != 1
    Px = 2 * grid.nx if free else grid.nx
    Py = 2 * grid.ny if free else grid.ny
    Pz = 2 * grid.nz if fz else grid.nz
    return {"Px": Px, "Py": Py, "Pz": Pz, "Hx": Px // 2 + 1, "nx": grid.nx, "ny": grid.ny,
            "nz": grid.nz, "npairs": (grid.ny * grid.nz + 1) // 2}


def kernel_flops(kind, P):
    """Algorithmic flops of one launch: the conventional 5 L log2 L per complex
    FFT of length L (two real rows per complex x transform), plus 2 per point
    for the real Green's-table multiply in the z pass."""
    import math
    f = lambda L: 5.0 * L * math.log2(L)
    if kind in ("x_fwd", "x_inv"):
        return P["npairs"] * f(P["Px"])
    if kind in ("y_fwd", "y_inv"):
        return P["Hx"] * P["nz"] * f(P["Py"])
    if kind == "z":
        return P["Hx"] * P["Py"] * (2 * f(P["Pz"]) + 2 * P["Pz"])
    n = P["nx"] * P["ny"] * P["nz"]
    return {"update_p": 10.0, "update_r": 6.0}.get(kind, 0.0) * n


def reduce_over_ranks(total_ms, units, device=None):
    """Whole-job numbers of a replica run: the slowest rank's timed region
    (max over ranks) and the units every rank processed (sum over ranks).
    The identity on a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return total_ms, units
    tmax = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    usum = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(usum, op=dist.ReduceOp.SUM)
    return float(tmax.item()), float(usum.item())


def timed_call(stream, flush, fn):
    """One call bracketed by CUDA events on `stream` after an L2 flush."""
    import torch
    flush.fill_(1.0)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    e1.synchronize()
    return out, e0.elapsed_time(e1)


def run_ours(args, ws, rank, local):
    import torch
    from paper_1509_00680_gb300 import build
    import synth

    build.build()
    from paper_1509_00680_gb300 import gps

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    p = synth.workload(4)
    g = gps.grid_from(p.grid)
    npts = p.grid.npts
    e = p.electrolyte
    el = gps.make_electrolyte(e.z, e.c_molar, e.temperature, p.eps0)
    rho = torch.from_numpy(p.rho.ravel()).to(dev)
    eps = torch.from_numpy(p.eps.ravel()).to(dev)
    phi = torch.zeros_like(rho)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ctx = gps.Context(local)
    opts = gps.default_opts(tol_outer=TOL_OUTER, max_iter=3000, precision=gps.GPS_MIXED_DF64)
    stream = torch.cuda.current_stream()
    P = pass_geometry(p.grid)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def solve(o, out):
        out.zero_()
        return ctx.pb_solve(g, rho, eps, el, "nlpb", out, o)

    for _ in range(args.warmup):
        solve(opts, phi)
    barrier()
    clocks = ClockSampler(local, args.clocks_log)
    clocks.start()
    launches0 = gps.kernel_launches()
    t_steps, reps = [], []
    torch.cuda.profiler.start()               # ncu --profile-from-start off: timed steps only
    for _ in range(args.steps):
        rep, ms = timed_call(stream, flush, lambda: solve(opts, phi))
        t_steps.append(ms)
        reps.append(rep)
    torch.cuda.profiler.stop()
    barrier()
    launches = gps.kernel_launches() - launches0
    clk = clocks.stop()
    iters = [r.iters for r in reps]
    total_ms, units = reduce_over_ranks(sum(t_steps), npts * sum(iters), dev)
    _, solves = reduce_over_ranks(sum(t_steps), len(t_steps), dev)
    value = units / (total_ms / 1e3)
    last = reps[-1]
    headline = {"solves_per_s": solves / (total_ms / 1e3), "ms_per_solve": total_ms / args.steps,
                "pcg_iters": int(statistics.median(iters)), "outer_iters": last.outer_iters,
                "high_precision_iters": last.fp64_iters, "certificate": last.fixed_point_res,
                "outer_res": last.outer_res, "status": last.status}

    # the plain FP64 GPU path on the same problem (FP64 spectrum throughout)
    fp64 = None
    if not args.no_fp64:
        phi64 = torch.zeros_like(rho)
        o64 = gps.default_opts(tol_outer=TOL_OUTER, max_iter=3000, precision=gps.GPS_FP64)
        rep64, ms64 = timed_call(stream, flush, lambda: solve(o64, phi64))
        err = (torch.linalg.norm(phi - phi64) / torch.linalg.norm(phi64)).item()
        fp64 = {"solves_per_s": 1e3 / ms64, "ms_per_solve": ms64, "pcg_iters": rep64.iters,
                "outer_iters": rep64.outer_iters, "grid_pt_iter_per_s": npts * rep64.iters / (ms64 / 1e3),
                "status": rep64.status, "timed_solves": 1,
                "mixed_rel_l2_err_vs_fp64": err,
                "mixed_speedup_solves_per_s": (1e3 / ms64) and headline["solves_per_s"] / (1e3 / ms64)}
        del phi64

    # kernel times: one more mixed solve, untimed, every kernel kind event-timed
    ctx.set_profiling("all")
    ctx.get_profile(reset=True)
    solve(opts, torch.zeros_like(rho))
    torch.cuda.synchronize()
    prof = {k: v for k, v in ctx.get_profile(reset=True).items() if v[0] > 0}
    ctx.set_profiling(None)
    ktot = sum(v[1] for v in prof.values())
    shares = {k: {"launches": v[0], "ms": round(v[1], 3), "share": round(v[1] / ktot, 4)}
              for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    dom = max(prof, key=lambda k: prof[k][1])
    roof = kernel_roofline(dom, prof[dom][1] / prof[dom][0], P, peaks())
    roof["kernel_time_shares"] = shares
    roof["measured_in"] = "one untimed mixed solve after the timed steps, every kernel kind event-timed"
    runner_up = {}
    for k in sorted(prof, key=lambda k: -prof[k][1])[1:4]:
        runner_up[k] = kernel_roofline(k, prof[k][1] / prof[k][0], P, peaks())
    roof["next_kernels"] = runner_up

    e2e = None if args.no_e2e else run_e2e(ctx, g, p, el, npts, opts, args)
    ctx.close()
    del phi
    torch.cuda.empty_cache()
    # the other workloads' sections run on a single GPU only: under torchrun
    # every rank solves the headline replica and nothing else
    single = ws == 1
    periodic128 = run_periodic128(gps, local, flush, args) if single and not args.no_periodic128 else None
    configs13 = run_configs13(gps, local, flush) if single and not args.no_configs13 else None
    nonlinear = run_nonlinear(gps, local, flush) if single and not args.no_nonlinear else None
    comparison = run_comparison(gps, local, flush) if single and not args.no_comparison else None
    wire = run_wire(gps, local, flush) if single and not args.no_wire else None
    dft = run_dft(gps, local, flush) if single and not args.no_dft else None
    serving = run_serving(gps, local, args) if single and not args.no_serving else None

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+df64+f32", "data": "synthetic",
        "config": config_dict(), "precision": PRECISION,
        "solves_per_s": headline["solves_per_s"],
        "headline": headline,
        "fp64": fp64,
        "e2e": e2e,
        "periodic128": periodic128,
        "configs13": configs13,
        "nonlinear": nonlinear,
        "comparison": comparison,
        "wire": wire,
        "dft": dft,
        "serving": serving,
        "roofline": roof,
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(p)
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_configs13(gps, device, flush):
    """Configurations 1 and 3: the free 64^3 single-cavity GPe (||r|| <= 1e-10)
    and the surface-BC 160 x 160 x 256 slab with the linear and the nonlinear PB
    term (1:1 electrolyte at 0.1 M, outer residual <= 1e-10), each on the plain
    FP64 path and the mixed path (df64 spectrum, FP32 after the switch):
    time of one solve after an untimed one, iterations, certificate, and the
    mixed result's relative L2 difference from the FP64 one."""
    import torch
    import synth
    out = {}
    cases = (("1 gpe_free_64", synth.workload(1), "gpe"),
             ("3 surface_lpb_160x160x256", synth.workload(3, kind="lpb"), "lpb"),
             ("3 surface_nlpb_160x160x256", synth.workload(3, kind="nlpb"), "nlpb"))
    ctx = gps.Context(device)
    stream = torch.cuda.current_stream()
    for name, p, kind in cases:
        g = gps.grid_from(p.grid)
        rho = torch.from_numpy(p.rho.ravel()).to(device)
        eps = torch.from_numpy(p.eps.ravel()).to(device)
        el = None
        if kind != "gpe":
            e = p.electrolyte
            el = gps.make_electrolyte(e.z, e.c_molar, e.temperature, p.eps0)
        row, phis = {}, {}
        for prec_name, prec in (("fp64", gps.GPS_FP64), ("mixed_df64", gps.GPS_MIXED_DF64)):
            o = gps.default_opts(tol_abs=1e-10, tol_outer=1e-10, max_iter=3000, precision=prec)
            phi = torch.zeros_like(rho)

            def solve():
                phi.zero_()
                if kind == "gpe":
                    return ctx.gpe_solve(g, rho, eps, phi, o)
                return ctx.pb_solve(g, rho, eps, el, kind, phi, o)

            solve()
            rep, ms = timed_call(stream, flush, solve)
            phis[prec_name] = phi
            row[prec_name] = {"ms": ms, "solves_per_s": 1e3 / ms, "pcg_iters": rep.iters,
                              "outer_iters": rep.outer_iters, "status": rep.status,
                              "grid_pt_iter_per_s": p.grid.npts * rep.iters / (ms / 1e3),
                              "certificate": rep.fixed_point_res}
        row["mixed_rel_l2_vs_fp64"] = (torch.linalg.norm(phis["mixed_df64"] - phis["fp64"]) /
                                      torch.linalg.norm(phis["fp64"])).item()
        row["speedup"] = row["fp64"]["ms"] / row["mixed_df64"]["ms"]
        out[name] = row
        del rho, eps, phis
    ctx.close()
    return out


def run_periodic128(gps, device, flush, args):
    """The 128^3 periodic GPe workload (20 charges, ||r|| <= 1e-10): the plain
    FP64 PCG timed over `steps` solves (no profiling in the timed region),
    then the other spectrum precisions, the warm start and the roofline of
    the FP64 path's dominant kernel from one more, untimed, profiled solve."""
    import torch
    import synth
    p = synth.workload(2)
    g = gps.grid_from(p.grid)
    npts = p.grid.npts
    rho = torch.from_numpy(p.rho.ravel()).to(device)
    eps = torch.from_numpy(p.eps.ravel()).to(device)
    phi = torch.empty_like(rho)
    ctx = gps.Context(device)
    opts = gps.default_opts(tol_abs=1e-10)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        ctx.gpe_solve(g, rho, eps, phi, opts)
    ts, its = [], []
    for _ in range(args.steps):
        rep, ms = timed_call(stream, flush, lambda: ctx.gpe_solve(g, rho, eps, phi, opts))
        ts.append(ms)
        its.append(rep.iters)
    fp64_ms = sum(ts) / len(ts)
    ctx.set_profiling("all")
    ctx.get_profile(reset=True)
    ctx.gpe_solve(g, rho, eps, torch.empty_like(rho), opts)
    torch.cuda.synchronize()
    prof = {k: v for k, v in ctx.get_profile(reset=True).items() if v[0] > 0}
    ctx.set_profiling(None)
    dom = max(prof, key=lambda k: prof[k][1])
    out = {"workload": p.name, "grid": [128, 128, 128], "bc": "periodic", "tol_abs": 1e-10,
           "grid_pt_iter_per_s": npts * sum(its) / (sum(ts) / 1e3), "solves_per_s": 1e3 / fp64_ms,
           "ms_per_solve": fp64_ms, "pcg_iters": int(statistics.median(its)),
           "roofline": kernel_roofline(dom, prof[dom][1] / prof[dom][0], pass_geometry(p.grid), peaks(),
                                       periodic=True)}
    out["roofline"]["kernel_time_shares"] = {k: round(v[1] / sum(w[1] for w in prof.values()), 4)
                                             for k, v in prof.items()}
    if not args.no_mixed:
        out["mixed"] = run_mixed(ctx, g, rho, eps, phi, flush, args, gps, fp64_ms)
        out["df64"] = run_mixed(ctx, g, rho, eps, phi, flush, args, gps, fp64_ms, precision=gps.GPS_DF64)
        out["mixed_df64"] = run_mixed(ctx, g, rho, eps, phi, flush, args, gps, fp64_ms,
                                      precision=gps.GPS_MIXED_DF64)
        out["warm_start"] = run_warm(gps, device, p, g, rho, eps, flush)
    ctx.close()
    return out


def run_mixed(ctx, g, rho, eps, phi64, flush, args, gps, fp64_ms, precision=None):
    """The same workload with another spectrum precision inside the FP64 PCG
    (default: FP32 after the switch; GPS_DF64: double-float throughout):
    solves/s, relative L2 error against the FP64 GPU result, FP64
    certificate."""
    import torch
    stream = torch.cuda.current_stream()
    phi = torch.empty_like(phi64)
    prec = gps.GPS_MIXED if precision is None else precision
    o = gps.default_opts(tol_abs=1e-10, precision=prec)
    ctx.gpe_solve(g, rho, eps, phi, o)
    ms, reps = 0.0, []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        reps.append(ctx.gpe_solve(g, rho, eps, phi, o))
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
    err = (torch.linalg.norm(phi - phi64) / torch.linalg.norm(phi64)).item()
    return {"solves_per_s": args.steps / (ms / 1e3), "ms_per_solve": ms / args.steps,
            "speedup_vs_fp64": fp64_ms / (ms / args.steps), "rel_l2_err_vs_fp64": err,
            "certificate": reps[-1].fixed_point_res, "pcg_iters": reps[-1].iters,
            "fp64_iters": reps[-1].fp64_iters,
            "spectrum": {gps.GPS_MIXED: "fp32 after ||r|| <= 1e-2 ||r0||, fp64 before",
                         gps.GPS_DF64: "df64",
                         gps.GPS_MIXED_DF64: "fp32 after ||r|| <= 1e-2 ||r0||, df64 before"}.get(prec, prec)}


def run_warm(gps, device, p, g, rho, eps, flush):
    """Warm start (opts.warm_start) on the same workload: after a solve, the
    solve for a nearby charge density (rho + 2% of itself shifted by 3 grid
    points along z, eps unchanged) from the previous potential, against the
    same solve from zero; FP64, ||r|| <= 1e-10."""
    import torch
    ctx = gps.Context(device)
    rho2 = rho + 0.02 * torch.roll(rho.view(p.grid.shape), 3, dims=0).reshape(-1)
    stream = torch.cuda.current_stream()

    def timed(r, warm):
        phi = torch.zeros_like(rho)
        o = gps.default_opts(tol_abs=1e-10, warm_start=warm)
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rep = ctx.gpe_solve(g, r, eps, phi, o)
        e1.record(stream)
        e1.synchronize()
        return phi, rep, e0.elapsed_time(e1)

    timed(rho2, 0)                         # plans and tuning
    timed(rho, 1)                          # state for the warm start
    phi_w, rep_w, ms_w = timed(rho2, 1)
    phi_c, rep_c, ms_c = timed(rho2, 0)
    ctx.close()
    return {"cold_iters": rep_c.iters, "warm_iters": rep_w.iters, "cold_ms": ms_c, "warm_ms": ms_w,
            "warm": rep_w.warm, "rel_l2_warm_vs_cold": (torch.linalg.norm(phi_w - phi_c) /
                                                        torch.linalg.norm(phi_c)).item(),
            "perturbation": "rho + 0.02 * rho shifted by 3 points along z, same eps"}


def run_nonlinear(gps, device, flush):
    """Modified (steric) PB on the headline workload (free 256^3, 200
    Gaussians, 1:1 electrolyte at 0.5 M, 300 K, p = 0.74 and R = 3 angstrom
    for both species), by the Newton outer loop around Algorithm 2 on the
    same mixed-precision path, outer tolerance 1e-10.  One untimed solve
    first (plans, tuning)."""
    import torch
    import synth
    p = synth.workload(4)
    g = gps.grid_from(p.grid)
    rho = torch.from_numpy(p.rho.ravel()).to(device)
    eps = torch.from_numpy(p.eps.ravel()).to(device)
    e = p.electrolyte
    el = gps.make_electrolyte(e.z, e.c_molar, e.temperature, p.eps0, radius_angstrom=(3.0,) * len(e.z),
                              packing=0.74)
    ctx = gps.Context(device)
    stream = torch.cuda.current_stream()
    opts = gps.default_opts(tol_outer=TOL_OUTER, max_iter=3000, precision=gps.GPS_MIXED_DF64)
    phi = torch.zeros_like(rho)
    ctx.pb_solve(g, rho, eps, el, "mpb", phi, opts)
    phi.zero_()
    rep, ms = timed_call(stream, flush, lambda: ctx.pb_solve(g, rho, eps, el, "mpb", phi, opts))
    ctx.close()
    return {"workload": p.name, "problem": "modified PB (steric, p = 0.74, R = 3 angstrom)",
            "precision": "mixed_df64", "mpb": {"ms": ms, "status": rep.status, "outer_iters": rep.outer_iters,
                                               "pcg_iters": rep.iters, "high_precision_iters": rep.fp64_iters,
                                               "outer_res": rep.outer_res, "fixed_point_res": rep.fixed_point_res}}


# FP64 pipe operations per grid point of the stencil kernels (gps_opts.method
# GPS_SC / GPS_PSD): 3 axes x 8 pairs x (subtract + FMA) = 48 for the
# order-16 derivatives, 8 for grad ln eps . grad u, the rest for the
# method's own update and the three residual sums (SC step: 66; PSD A v: 62).
STENCIL_OPS = {"sc": 66, "psd": 62}
FP64_PIPE_GOPS = 152 * 2 * 2.07   # 2 FP64 operations per clock per SM at 2.07 GHz


def run_comparison(gps, device, flush):
    """Algorithm 1 (SC, eta = 0.6), PSD + DIIS (m = 6) and Algorithm 2 on
    the 128^3 periodic workload, each to ||r|| <= 1e-10 ||r_0|| in its own
    discretization (FP64).  Per method: time per solve, iterations, time per
    iteration, and the order-16 stencil kernel's time per launch against the
    FP64-pipe peak (the kernel is FP64-pipe bound on GB300)."""
    import torch
    import synth
    p = synth.workload(2)
    g = gps.grid_from(p.grid)
    rho = torch.from_numpy(p.rho.ravel()).to(device)
    eps = torch.from_numpy(p.eps.ravel()).to(device)
    ctx = gps.Context(device)
    stream = torch.cuda.current_stream()
    out = {"workload": p.name, "tol_rel": 1e-10}
    methods = {"pcg": dict(method=gps.GPS_PCG), "sc": dict(method=gps.GPS_SC, eta=0.6),
               "psd_diis6": dict(method=gps.GPS_PSD, diis=6)}
    for name, kw in methods.items():
        o = gps.default_opts(tol_abs=0.0, tol_rel=1e-10, max_iter=3000, **kw)
        phi = torch.zeros_like(rho)
        ctx.gpe_solve(g, rho, eps, phi, o)          # plans, tuning, work arrays
        ctx.set_profiling(["stencil"] if name != "pcg" else None)
        ctx.get_profile(reset=True)
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.profiler.start()           # ncu --profile-from-start off: the timed solves
        e0.record(stream)
        rep = ctx.gpe_solve(g, rho, eps, phi, o)
        e1.record(stream)
        e1.synchronize()
        torch.cuda.profiler.stop()
        ms = e0.elapsed_time(e1)
        prof = ctx.get_profile(reset=True)
        ctx.set_profiling(None)
        row = {"ms": ms, "iters": rep.iters, "ms_per_iter": ms / max(rep.iters, 1), "status": rep.status,
               "res_rel": rep.res / rep.res0 if rep.res0 else 0.0}
        if name != "pcg":
            n_l, t_l = prof["stencil"]
            avg = t_l / max(n_l, 1)
            ops = STENCIL_OPS["sc" if name == "sc" else "psd"] * p.grid.npts
            row["stencil"] = {"launches": n_l, "avg_ms": avg, "fp64_gops": ops / (avg / 1e3) / 1e9,
                              "frac_of_fp64_pipe": ops / (avg / 1e3) / 1e9 / FP64_PIPE_GOPS}
        out[name] = row
    ctx.close()
    return out


def run_wire(gps, device, flush):
    """Wire BC (periodic z, free x and y): GPe on a 128 x 128 x 256 chain of 8
    cavities (radius 2.4 bohr, a pair of Gaussians in each), ||r|| <= 1e-10,
    FP64 and mixed df64 spectra; one untimed solve first (table, tuning)."""
    import torch
    import synth
    p = synth.wire_chain(n=128, nz=256, count=8, kind="gpe")
    g = gps.grid_from(p.grid)
    rho = torch.from_numpy(p.rho.ravel()).to(device)
    eps = torch.from_numpy(p.eps.ravel()).to(device)
    ctx = gps.Context(device)
    stream = torch.cuda.current_stream()
    out = {"workload": p.name, "grid": list(p.grid.shape), "padded": [2 * p.grid.nx, 2 * p.grid.ny, p.grid.nz]}
    for name, prec in (("fp64", gps.GPS_FP64), ("mixed_df64", gps.GPS_MIXED_DF64)):
        o = gps.default_opts(tol_abs=1e-10, max_iter=2000, precision=prec)
        phi = torch.zeros_like(rho)
        ctx.gpe_solve(g, rho, eps, phi, o)
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rep = ctx.gpe_solve(g, rho, eps, phi, o)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        out[name] = {"ms": ms, "iters": rep.iters, "status": rep.status,
                     "grid_pt_iter_per_s": p.grid.npts * rep.iters / (ms / 1e3),
                     "certificate": rep.fixed_point_res}
    ctx.close()
    return out


def run_dft(gps, device, flush):
    """DFT-facing passes on the 128^3 periodic workload's GPU potential: the
    sccs dielectric of a synthetic electron density (a Gaussian of peak 0.2
    and width 1.2 bohr on every solute charge, spanning the sccs transition
    rho_max = 5e-3, rho_min = 1e-4), the polarization charge, v_eps and the
    electrostatic energy; CUDA-event time per call (mean of 5 after one
    warm-up), L2 flushed before each."""
    import torch
    import synth
    p = synth.workload(2)
    g = gps.grid_from(p.grid)
    rho = torch.from_numpy(p.rho.ravel()).to(device)
    eps = torch.from_numpy(p.eps.ravel()).to(device)
    norm = 0.2 * (2 * np.pi * 1.2 ** 2) ** 1.5
    rho_e_h = synth.gaussian_charges(p.grid, [(norm, 1.2, c) for _, _, c in p.charges])
    rho_e = torch.from_numpy(rho_e_h.ravel()).to(device)
    ctx = gps.Context(device)
    phi = torch.zeros_like(rho)
    ctx.gpe_solve(g, rho, eps, phi, gps.default_opts(tol_abs=1e-10))
    e_s, d_s, out = torch.empty_like(rho), torch.empty_like(rho), torch.empty_like(rho)
    stream = torch.cuda.current_stream()
    calls = {"sccs_eps": lambda: ctx.sccs_eps(rho_e, e_s, d_s),
             "polarization_charge": lambda: ctx.polarization_charge(g, rho, eps, phi, out),
             "v_eps": lambda: ctx.v_eps(g, d_s, phi, out),
             "electrostatic_energy": lambda: ctx.electrostatic_energy(g, rho, eps, phi)}
    res = {"workload": p.name, "npts": p.grid.npts}
    for name, fn in calls.items():
        fn()
        ts = []
        for _ in range(5):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = float(np.mean(ts))
        res[name] = {"ms": ms, "grid_pts_per_s": p.grid.npts / (ms / 1e3)}
    res["transition_fraction"] = float(((rho_e_h > 1e-4) & (rho_e_h < 5e-3)).mean())
    e1_, e2_ = ctx.electrostatic_energy(g, rho, eps, phi)
    res["energy"] = {"rho_phi": e1_, "eps_grad2": e2_}
    ctx.close()
    return res


def run_experiments(args):
    """The paper's GPe experiment (Sec. "Numerical results", Fig. NormrAcc) at
    its own size: box 10, 300^3, phi a normalized Gaussian (sigma 0.5), eps the
    erf cavity (d0 1.7, Delta 0.3, eps0 78.36), free, surface and periodic BC.
    Accuracy (max |phi - phi_exact|, for periodic BC in the solver's gauge)
    after k iterations of Algorithm 2 (PCG) and of Algorithm 1 (SC, eta =
    0.6), FP64; one JSON line."""
    import torch
    from paper_1509_00680_gb300 import build
    import synth
    build.build()
    from paper_1509_00680_gb300 import gps
    dev = torch.device("cuda", 0)
    ctx = gps.Context(0)
    stream = torch.cuda.current_stream()
    out = {"experiment": "E1 (Fig. NormrAcc)", "n": args.exp_n, "box": 10.0, "bcs": {}}
    pcg_ks, sc_ks = (1, 2, 3, 4, 5, 6, 8, 10, 12, 15, 20), (5, 10, 20, 40, 80)
    for bc in (synth.BC_FREE, synth.BC_SURFACE, synth.BC_PERIODIC):
        p = synth.manufactured(n=args.exp_n, bc=bc)
        g = gps.grid_from(p.grid)
        rho = torch.from_numpy(p.rho.ravel()).to(dev)
        eps = torch.from_numpy(p.eps.ravel()).to(dev)
        ex = torch.from_numpy(p.phi_exact.ravel()).to(dev)
        periodic = bc == synth.BC_PERIODIC
        sq = torch.sqrt(eps)
        ex_g = ex - (sq * ex).sum() / sq.sum() if periodic else ex     # the solver's gauge
        row = {}
        for name, ks, kw in (("pcg", pcg_ks, {}), ("sc", sc_ks, dict(method=gps.GPS_SC, eta=0.6))):
            pts = []
            for k in ks:
                phi = torch.zeros_like(rho)
                o = gps.default_opts(tol_abs=0.0, max_iter=k, **kw)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rep = ctx.gpe_solve(g, rho, eps, phi, o, allow=(gps.GPS_OK, gps.GPS_ERR_NOT_CONVERGED))
                e1.record(stream)
                e1.synchronize()
                ref = ex_g if not (periodic and name == "sc") else ex - ex.mean()
                got = phi if not (periodic and name == "sc") else phi - phi.mean()
                pts.append({"iters": rep.iters, "res": rep.res, "accuracy": (got - ref).abs().max().item(),
                            "ms": e0.elapsed_time(e1)})
            row[name] = pts
        out["bcs"][synth.BC_NAMES[bc]] = row
        del rho, eps, ex, ex_g, sq
        torch.cuda.empty_cache()
    ctx.close()
    print(json.dumps(out))


def run_serving(gps, device, args):
    """The serving workload: `--serving-count` requests (default the 512 of
    the configuration) drawn like the request stream (edges {48,64,96,128,
    192}, BC and problem mixed, 5-80 charges, 0.01-1 M), 120 GB admission
    budget, every request on the mixed-precision path (df64 spectrum, FP32
    once ||r|| <= 1e-2 ||r_ref||, FP64 certificate).
      capacity      one batch solve of the first `--serving-capacity-count`
                    requests (after one untimed batch of one request per
                    distinct grid and problem: plans, tuning, graphs);
      saturated     Poisson arrivals at 1.5x that capacity through the server:
                    throughput and latency (queueing included);
      low load      the first `--serving-low-count` requests at 0.5x capacity:
                    latency of a sustainable load;
      fp64 / mixed  the plain FP64 path (FP64 spectrum, one solve per call
      sequential    through the host-array entry points, as a served request
                    arrives) on every request of the stream, and the mixed
                    path the same way on a uniform sample
                    (`--serving-mixed-sample` requests)."""
    import threading
    import synth
    count = args.serving_count
    desc = synth.serving_stream(count=count, seed=1005)
    reqs = []
    for edge, bc, kind, seed in desc:
        rng = np.random.default_rng(seed)
        p = synth.serving_request(rng, edge, bc, kind)
        el = gps.make_electrolyte(p.electrolyte.z, p.electrolyte.c_molar, 300.0, p.eps0)
        reqs.append((p, kind, el))
    mixed_opts = lambda: gps.default_opts(tol_abs=1e-10, tol_outer=1e-10, max_iter=3000,
                                          precision=gps.GPS_MIXED_DF64)

    def make(i, opts):
        p, kind, el = reqs[i]
        rho = np.ascontiguousarray(p.rho.ravel())
        eps = np.ascontiguousarray(p.eps.ravel())
        phi = np.zeros(p.grid.npts)
        r = gps.make_request(gps.grid_from(p.grid), kind, rho, eps, phi, el, opts)
        return r, (rho, eps, phi)

    secs = {}

    def note(name, value):
        secs[name] = value
        print("serving: %s %.2f s" % (name, value), file=sys.stderr, flush=True)

    tw0 = time.perf_counter()
    made = [make(i, mixed_opts()) for i in range(count)]
    note("inputs", time.perf_counter() - tw0)
    first = {}
    for i, (edge, bc, kind, _) in enumerate(desc):
        first.setdefault((edge, bc, kind), i)
    budget = 120 << 30
    ctx = gps.Context(device, budget)
    tw0 = time.perf_counter()
    gps.batch_solve(ctx, [made[i][0] for i in first.values()], allow=(0, 3))    # plans, graphs
    note("warmup", time.perf_counter() - tw0)
    ncap = min(count, args.serving_capacity_count)
    t0 = time.perf_counter()
    reps_b = gps.batch_solve(ctx, [m[0] for m in made[:ncap]], allow=(0, 3))
    note("capacity", time.perf_counter() - t0)
    capacity = ncap / secs["capacity"]
    ctx.close()

    # one server for both streams, warmed (untimed) with one request per
    # distinct grid and problem: tables, plans and graphs are in place, as in
    # a server that has been running
    srv = gps.Server(device, hbm_budget_bytes=budget)
    tw0 = time.perf_counter()
    for st_, _ in [srv.wait(t, timeout=1800) for t in [srv.submit(made[i][0], keep=made[i][1]) for i in first.values()]]:
        pass
    note("server_warmup", time.perf_counter() - tw0)

    def stream(n, rate, seed):
        rng = np.random.default_rng(seed)
        tickets, keep = [], []
        start = time.perf_counter()

        def producer():
            for i in range(n):
                r, hold = made[i]
                keep.append(hold)
                tickets.append(srv.submit(r, keep=hold))
                time.sleep(float(rng.exponential(1.0 / rate)))

        th = threading.Thread(target=producer)
        th.start()
        th.join()
        results = [srv.wait(t, timeout=1800) for t in tickets]
        wall = time.perf_counter() - start
        return results, wall, srv.stats()

    rate = 1.5 * capacity
    results, wall, stats = stream(count, rate, 77)
    note("saturated", wall)
    lat = sorted(rep.time_ms for _, rep in results)
    ok = sum(1 for st_, _ in results if st_ == 0)
    nlow = min(count, args.serving_low_count)
    res_l, wall_l, _ = stream(nlow, 0.5 * capacity, 78)
    note("low_load", wall_l)
    srv.close()
    lat_l = sorted(rep.time_ms for _, rep in res_l)

    # sequential single solves: plain FP64 on every request of the stream,
    # mixed on a uniform sample
    k = max(1, count // max(1, args.serving_mixed_sample))
    samples = {"fp64": list(range(count)), "mixed_df64": list(range(0, count, k))}
    seq = {}
    ctx = gps.Context(device, budget)
    for name, prec in (("fp64", gps.GPS_FP64), ("mixed_df64", gps.GPS_MIXED_DF64)):
        sample = samples[name]
        for i in sorted({(desc[j][0], desc[j][1], desc[j][2]): j for j in sample}.values()):
            run_single(gps, ctx, reqs[i], prec)                      # plans and tuning, untimed
        t0 = time.perf_counter()
        st_ok = 0
        for i in sample:
            st_ok += run_single(gps, ctx, reqs[i], prec) == 0
        dt = time.perf_counter() - t0
        note("sequential_" + name, dt)
        seq[name] = {"solves_per_s": len(sample) / dt, "ok": st_ok}
    ctx.close()
    served = count / wall
    return {"requests": count, "ok": ok, "hbm_budget_bytes": budget,
            "arrival_rate_per_s": rate, "batch_capacity_solves_per_s": capacity,
            "batch_capacity_requests": ncap, "batch_ok": sum(1 for r in reps_b if r.status == 0),
            "solves_per_s": served, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)),
            "at_0.5x_capacity": {"requests": nlow, "arrival_rate_per_s": 0.5 * capacity,
                                 "solves_per_s": nlow / wall_l,
                                 "p50_ms": float(np.percentile(lat_l, 50)),
                                 "p99_ms": float(np.percentile(lat_l, 99)),
                                 "ok": sum(1 for st_, _ in res_l if st_ == 0)},
            "sequential": {"how": "one solve per call through the host-array entry points; FP64 on all %d "
                                  "requests of the stream, mixed df64 on every %d-th (%d)"
                                  % (count, k, len(samples["mixed_df64"])),
                           "fp64_solves_per_s": seq["fp64"]["solves_per_s"],
                           "mixed_df64_solves_per_s": seq["mixed_df64"]["solves_per_s"],
                           "ok": {n: v["ok"] for n, v in seq.items()}},
            "served_vs_fp64_sequential": served / seq["fp64"]["solves_per_s"],
            "max_concurrent": stats["max_concurrent"],
            "pool_bytes": stats["bytes_in_use"],
            "precision": "mixed_df64 (FP32 spectrum after the switch, df64 before, FP64 certificate)",
            "max_certificate": float(max(rep.fixed_point_res for _, rep in results)),
            "seconds": {k: round(v, 2) for k, v in secs.items()}}


def run_single(gps, ctx, req, precision):
    """One serving request solved alone through the host-array entry point."""
    p, kind, el = req
    rho = np.ascontiguousarray(p.rho.ravel())
    eps = np.ascontiguousarray(p.eps.ravel())
    phi = np.zeros(p.grid.npts)
    o = gps.default_opts(tol_abs=1e-10, tol_outer=1e-10, max_iter=3000, precision=precision)
    g = gps.grid_from(p.grid)
    if kind == "gpe":
        return ctx.gpe_solve_host(g, rho, eps, phi, o).status
    return ctx.pb_solve_host(g, rho, eps, el, kind, phi, o, allow=(0, 3)).status


def run_e2e(ctx, g, p, el, npts, opts, args):
    """Same metric through the host-pointer entry point gps_pb_solve_host:
    the H2D copy of rho and eps from pinned memory and the D2H copy of phi
    are inside the timed region of every step (wall clock around the call,
    which returns after its stream synchronizes)."""
    import torch
    rho_h = torch.from_numpy(p.rho.ravel().copy()).pin_memory().numpy()
    eps_h = torch.from_numpy(p.eps.ravel().copy()).pin_memory().numpy()
    phi_h = torch.empty(npts, dtype=torch.float64).pin_memory().numpy()
    e2e_ms, e2e_iters, n = 0.0, 0, max(2, args.e2e_steps)
    for _ in range(n):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = ctx.pb_solve_host(g, rho_h, eps_h, el, "nlpb", phi_h, opts)
        e2e_ms += (time.perf_counter() - t0) * 1e3
        e2e_iters += rep.iters
    return {"value": npts * e2e_iters / (e2e_ms / 1e3), "unit": UNIT, "steps": n,
            "solves_per_s": n / (e2e_ms / 1e3),
            "h2d_bytes_per_step": 2 * npts * 8, "d2h_bytes_per_step": npts * 8}


def oracle_sample(p, iters):
    """Setup plus `iters` PCG iterations of the oracle on the headline
    workload: the first Newton step of Algorithm 4 (ionic charge and its
    derivative at phi = 0, the linearized operator, Algorithm 2 on the
    outer residual); returns (seconds, iterations)."""
    import oracle
    from oracle.operators import Fields
    from oracle.pcg import pcg
    t0 = time.perf_counter()
    e = p.electrolyte
    gam = oracle.pb.exclusion_from_eps(p.eps, p.eps0)
    phi = np.zeros_like(p.rho)
    lam = -4.0 * np.pi * oracle.pb.ionic_charge_derivative(phi, gam, e)
    f = Fields(p.grid, p.eps, lam=lam)
    # first outer step: rho_ions = rho_ions[0] = fresh, r' = rho, so the inner
    # source rho + fresh - rho_ions is rho itself (free BC: no background)
    _, info = pcg(f, p.rho, tol_abs=0.0, tol_rel=1e-13, max_iter=iters)
    return time.perf_counter() - t0, info["iters"]


def cpu_baseline(p, iters=8):
    secs, it = oracle_sample(p, iters)
    return {"value": p.grid.npts * it / secs, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": "oracle setup (Green's table, s, q, ionic terms) + %d PCG iterations of the first "
                      "Newton step of the free 256^3 nonlinear-PB workload (%.1f s)" % (it, secs)}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import synth
    p = synth.workload(4)
    iters = 4
    for _ in range(args.warmup):
        oracle_sample(p, 1)
    secs, its = 0.0, 0
    for _ in range(args.steps):
        sec, i = oracle_sample(p, iters)
        secs += sec
        its += i
    value = p.grid.npts * its / secs
    sample = ("per step: oracle setup + %d PCG iterations of the first Newton step of the free 256^3 "
              "nonlinear-PB workload" % iters)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": config_dict(), "precision": "FP64 (oracle)",
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_cpu_configs(args):
    """The CPU oracle on each configuration's workload, median of 5 timed runs
    after 1 warm-up: setup plus a fixed number of PCG iterations (configs 3
    and 4: of the first Newton step of the nonlinear problem), as grid-pt*iter/s
    and the implied seconds per PCG iteration."""
    import synth
    cases = [("1 gpe_free_64", synth.workload(1), 10, False),
             ("2 gpe_periodic_128", synth.workload(2), 10, False),
             ("3 surface_nlpb_160x160x256", synth.workload(3, kind="nlpb"), 6, True),
             ("4 free_nlpb_256", synth.workload(4), 4, True)]
    out = {"cores": os.cpu_count(), "kind": "oracle", "configs": {}}
    for name, p, iters, nl in cases:
        fn = (lambda: oracle_sample(p, iters)) if nl else (lambda: gpe_oracle_sample(p, iters))
        fn()
        runs = [fn() for _ in range(5)]
        secs = statistics.median(r[0] for r in runs)
        its = runs[0][1]
        out["configs"][name] = {"grid_pt_iter_per_s": p.grid.npts * its / secs, "seconds": secs,
                                "iters": its, "sample": "setup + %d PCG iterations" % its}
    print(json.dumps(out))


def gpe_oracle_sample(p, iters):
    from oracle.operators import Fields
    from oracle.pcg import neutralize, pcg
    t0 = time.perf_counter()
    f = Fields(p.grid, p.eps)
    rho, _ = neutralize(p.rho, p.grid)
    _, info = pcg(f, rho, tol_abs=0.0, tol_rel=1e-13, max_iter=iters)
    return time.perf_counter() - t0, info["iters"]


def run_fp64_peak(args):
    """Measured FP64 rate of this GPU: a cuBLAS DGEMM (torch.matmul, FP64,
    8192^3, 2 N^3 flops, best of 5 after 2 warm-ups), for comparison with
    the derived FP64-pipe peak used by the roofline."""
    import torch
    n = 8192
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    for _ in range(2):
        torch.matmul(a, b)
    best = 1e30
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    print(json.dumps({"fp64_dgemm_tflops": 2 * n ** 3 / (best / 1e3) / 1e12, "n": n, "best_ms": best,
                      "derived_fp64_pipe_tflops": FP64_PEAK_TFLOPS}))


PASS_CASES = {
    # name: (nx, ny, nz, bc) at h = 0.3 bohr
    "free256": (256, 256, 256, 0),
    "periodic128": (128, 128, 128, 1),
    "periodic256": (256, 256, 256, 1),
    "surface160": (160, 160, 256, 2),
}


def pass_bytes(P, e):
    """Algorithmic HBM bytes of each spectrum pass of one preconditioner
    application with spectrum elements of e bytes (8 FP32, 16 FP64 or df64):
    the x forward pass reads r (FP64) and s (FP32 copy on the FP32 path,
    FP64 otherwise) and writes the half spectrum (only the planes and rows
    that hold data); y and z passes read and write spectrum elements (z also
    the octant Green's table, FP32 or FP64); the x inverse pass reads the half
    spectrum, s and r (for (v, r)) and writes v (FP64)."""
    n = P["nx"] * P["ny"] * P["nz"]
    se = 4 if e == 8 else 8
    half = P["nz"] * P["ny"] * P["Hx"] * e
    full = P["nz"] * P["Py"] * P["Hx"] * e
    table = P["Hx"] * (P["Py"] // 2 + 1) * (P["Pz"] // 2 + 1) * (4 if e == 8 else 8)
    return {"x_fwd": (8 + se) * n + half, "y_fwd": half + full, "z": 2 * full + table,
            "y_inv": full + half, "x_inv": half + (16 + se) * n}


def vector_bytes(P, periodic=False):
    """Algorithmic bytes of the PCG vector updates per launch (FP64 fields):
    update_p reads v, r, q + lambda, p, A p and writes p, A p (periodic: also
    sqrt(eps) and s); update_r reads phi, r, p, A p and writes phi, r."""
    n = P["nx"] * P["ny"] * P["nz"]
    return {"update_p": (72 if periodic else 56) * n, "update_r": 48 * n}


def df64_alu_view(base, ms, P):
    """FP32-pipe view of a double-float spectrum pass, the bound its counters
    show (issue-bound, FMA pipe the busiest): the conventional FFT flops of
    kernel_flops split as in a radix-2 butterfly (6 additions and 4 products
    per 10 flops) and the Green's-table products of the z pass, each costed
    at the FP32 instructions of its double-float operation, over the launch
    time, against the FP32 issue rate.  The conventional count exceeds what
    radix-8 butterflies and the pruned zero half execute, so this is an upper
    estimate of the pass's FP32 work rate."""
    fl = kernel_flops(base, P)
    table = 2.0 * P["Hx"] * P["Py"] * P["Pz"] if base == "z" else 0.0
    inst = (fl - table) * (0.6 * DF64_ADD_INST + 0.4 * DF64_MUL_INST) + table * DF64_MUL_INST
    ach = inst / (ms / 1e3) / 1e12
    return {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TINST, "unit": "T FP32 instructions/s",
            "frac": ach / FP32_PEAK_TINST, "fp32_instructions": inst,
            "peak_source": "derived: 152 SM x 128 FP32 lanes x 2.07 GHz",
            "model": "5 L log2 L flops per complex FFT, 0.6 x 8 + 0.4 x 4 FP32 instructions per flop; "
                     "4 per Green's-table product"}


def kernel_roofline(kind, ms, P, peaks_, periodic=False):
    """Roofline entry of one kernel kind from its average launch time."""
    hbm = peaks_.get("hbm_gbs")
    prec = "fp64"
    base = kind
    for suf in ("_df64", "_fp32"):
        if kind.endswith(suf):
            base, prec = kind[:-len(suf)], suf[1:]
    if base in ("x_fwd", "y_fwd", "z", "y_inv", "x_inv") and prec == "fp64":
        fl = kernel_flops(base, P)
        ach = fl / (ms / 1e3) / 1e12
        return {"kernel": kind, "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS, "traffic": ncu_traffic(kind),
                "avg_launch_ms": ms,
                "peak_source": "derived: 152 SM x 2 DFMA/clk x 2 flop x 2.07 GHz (FP64 pipe, measured by --fp64-peak)",
                "flops_model": "5 L log2 L per complex FFT of length L (+2 per point for the table)"}
    if base in ("x_fwd", "y_fwd", "z", "y_inv", "x_inv"):
        byt = pass_bytes(P, 8 if prec == "fp32" else 16)[base]
    else:
        byt = vector_bytes(P, periodic).get(base)
    if byt is None or not hbm:
        return {"kernel": kind, "avg_launch_ms": ms}
    ach = byt / (ms / 1e3) / 1e9
    out = {"kernel": kind, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
           "frac": ach / hbm, "traffic": ncu_traffic(kind), "avg_launch_ms": ms,
           "algorithmic_bytes": byt, "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy), burst"}
    if prec == "df64" and base in ("x_fwd", "y_fwd", "z", "y_inv", "x_inv"):
        out["alu_view"] = df64_alu_view(base, ms, P)
    return out


def run_passes(args):
    """Per-pass device time and achieved HBM GB/s of one preconditioner
    application v = s S(s r) in each spectrum precision, with random r and s;
    one more application per precision runs inside a profiler region for ncu
    (--profile-from-start off)."""
    import torch
    from paper_1509_00680_gb300 import build
    import synth
    build.build()
    from paper_1509_00680_gb300 import gps
    nx, ny, nz, bc = PASS_CASES[args.passes]
    gps.set_x_kernel(args.x_kernel)
    gps.set_z_kernel(args.z_kernel)
    origin = (0.0, 0.0, 0.0)
    grid = synth.Grid(nx, ny, nz, 0.3, 0.3, 0.3, bc, origin=origin)
    g = gps.grid_from(grid)
    n = grid.npts
    rng = np.random.default_rng(0)
    s = torch.from_numpy(rng.uniform(0.1, 1.0, n)).cuda()
    r = torch.from_numpy(rng.standard_normal(n)).cuda()
    v = torch.zeros_like(r)
    ctx = gps.Context(0)
    P = pass_geometry(grid)
    peak = peaks().get("hbm_gbs")
    codes = {"fp64": (gps.GPS_FP64, 16), "fp32": (gps.GPS_MIXED, 8), "df64": (gps.GPS_DF64, 16)}
    out = {"passes": args.passes, "grid": [nx, ny, nz], "bc": bc, "P": [P["Px"], P["Py"], P["Pz"]],
           "hbm_peak_gbs": peak, "x_kernel": args.x_kernel, "z_kernel": args.z_kernel}
    for name in args.precisions.split(","):
        code, e = codes[name]
        for _ in range(3):
            ctx.precondition(g, s, r, v, code)
        ctx.set_profiling("all")
        ctx.get_profile(reset=True)
        for _ in range(args.steps):
            ctx.precondition(g, s, r, v, code)
        torch.cuda.synchronize()
        prof = ctx.get_profile(reset=True)
        ctx.set_profiling(None)
        byt = pass_bytes(P, e)
        res, tot = {}, 0.0
        suf = "" if name == "fp64" else "_" + name
        for k, (cnt, ms) in prof.items():
            if not cnt:
                continue
            if suf and k.endswith(suf):
                k = k[:-len(suf)]
            t = ms / cnt
            tot += t
            res[k] = {"us": round(t * 1e3, 2), "bytes": byt.get(k)}
            if k in byt:
                res[k]["GBs"] = round(byt[k] / (t * 1e-3) / 1e9, 1)
                if peak:
                    res[k]["frac_hbm"] = round(byt[k] / (t * 1e-3) / 1e9 / peak, 3)
        res["total_us"] = round(tot * 1e3, 2)
        out[name] = res
        torch.cuda.profiler.start()
        ctx.precondition(g, s, r, v, code)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    out["cufft"] = cufft_comparison(torch, grid, P, args.steps)
    print(json.dumps(out))
    ctx.close()


def cufft_comparison(torch, grid, P, steps):
    """Timed comparison only (not part of any solve): cuFFT through torch.fft on
    the same application, v = s irfftn(G rfftn(pad(s r))), in FP64 and FP32.
    cuFFT transforms the full padded box (it cannot skip the zero padding);
    the Green's function is a random real array of the half-spectrum shape."""
    res = {}
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    shp = (P["Pz"], P["Py"], P["Px"])
    for name, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
        try:
            s = torch.rand((nz, ny, nx), dtype=torch.float64, device="cuda") + 0.1
            r = torch.randn((nz, ny, nx), dtype=torch.float64, device="cuda")
            G = torch.rand((P["Pz"], P["Py"], P["Hx"]), dtype=dt, device="cuda")
            pad = torch.zeros(shp, dtype=dt, device="cuda")

            def apply():
                pad[:nz, :ny, :nx] = (s * r).to(dt)
                w = torch.fft.irfftn(torch.fft.rfftn(pad) * G, s=shp)
                return s * w[:nz, :ny, :nx].to(torch.float64)

            for _ in range(3):
                apply()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                apply()
            e1.record()
            e1.synchronize()
            res[name] = {"us": round(e0.elapsed_time(e1) / steps * 1e3, 1)}
            del s, r, G, pad
            torch.cuda.empty_cache()
        except Exception as exc:   # e.g. out of memory on a very large box
            res[name] = {"error": str(exc)[:120]}
    return res


def run_warm_serving(args):
    """Served warm starts (opts.warm_start): per BC and problem (GPe, linear
    PB) at edge 64, h = 0.3, a sequence of requests that share eps while rho
    drifts (rho_k = rho + 0.01 k roll(rho, 1 along z), as successive steps of
    a fixed-cavity calculation), each submitted once the previous one has
    completed, served cold and then with warm_start (from the pool's retained
    eps, phi and b - r of the previous request).  Reports the mean PCG
    iterations and latency of requests 1 .. K-1 both ways and the largest
    relative L2 difference of a warm result from the cold one."""
    from paper_1509_00680_gb300 import build
    import synth

    build.build()
    from paper_1509_00680_gb300 import gps

    K = max(2, args.warm_count)
    srv = gps.Server(0, hbm_budget_bytes=8 << 30)
    cases = {}
    try:
        for bc in (0, 1, 2):
            for kind in ("gpe", "lpb"):
                rng = np.random.default_rng(1200 + 2 * bc + (kind == "lpb"))
                p = synth.serving_request(rng, 64, bc, kind)
                e = p.electrolyte
                el = gps.make_electrolyte(e.z, e.c_molar, e.temperature, p.eps0)
                g = gps.grid_from(p.grid)
                eps_h = np.ascontiguousarray(p.eps.ravel())
                shifted = np.roll(p.rho, 1, axis=2)
                rhos = [np.ascontiguousarray((p.rho + 0.01 * k * shifted).ravel()) for k in range(K)]
                runs = {}
                for warm in (0, 1):
                    iters, ms, nwarm, phis = [], [], 0, []
                    for k in range(K):
                        phi = np.full(p.grid.npts, np.nan)
                        o = gps.default_opts(tol_abs=1e-10, max_iter=2000, warm_start=warm)
                        t = srv.submit(gps.make_request(g, kind, rhos[k], eps_h, phi, el, o),
                                       keep=(rhos[k], eps_h, phi))
                        status, rep = srv.wait(t, timeout=300)
                        if status != 0:
                            raise RuntimeError("warm-serving request failed with status %d" % status)
                        if k > 0:
                            iters.append(rep.iters)
                            ms.append(rep.time_ms)
                            nwarm += rep.warm
                        phis.append(phi)
                    runs[warm] = (iters, ms, nwarm, phis)
                diff = max(float(np.linalg.norm(a - b) / np.linalg.norm(b))
                           for a, b in zip(runs[1][3], runs[0][3]))
                name = "%s_%s_64" % (("free", "periodic", "surface")[bc], kind)
                cases[name] = {
                    "cold": {"iters": statistics.mean(runs[0][0]), "ms": statistics.mean(runs[0][1])},
                    "warm": {"iters": statistics.mean(runs[1][0]), "ms": statistics.mean(runs[1][1]),
                             "started_warm": runs[1][2]},
                    "max_rel_l2_warm_vs_cold": diff,
                }
                print("warm serving %s: cold %.1f iterations, warm %.1f" % (
                    name, cases[name]["cold"]["iters"], cases[name]["warm"]["iters"]), file=sys.stderr, flush=True)
    finally:
        srv.close()
    print(json.dumps({"mode": "warm_serving", "requests_per_sequence": K,
                      "tol_abs": 1e-10, "cases": cases}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-nonlinear", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 solve of the headline")
    ap.add_argument("--no-periodic128", action="store_true")
    ap.add_argument("--no-configs13", action="store_true", help="skip the configuration 1 and 3 section")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-comparison", action="store_true")
    ap.add_argument("--no-wire", action="store_true")
    ap.add_argument("--no-dft", action="store_true")
    ap.add_argument("--clocks-log", default=None, help="keep the nvidia-smi samples of the timed region here")
    ap.add_argument("--serving-count", type=int, default=512)
    ap.add_argument("--serving-capacity-count", type=int, default=128)
    ap.add_argument("--serving-low-count", type=int, default=48)
    ap.add_argument("--serving-mixed-sample", type=int, default=64)
    ap.add_argument("--passes", default=None, choices=sorted(PASS_CASES),
                    help="per-pass times of one preconditioner application instead of the bench")
    ap.add_argument("--precisions", default="fp64,df64,fp32")
    ap.add_argument("--x-kernel", type=int, default=-1, choices=(-1, 0, 1),
                    help="--passes: FP32 x-pass kernels (-1 tuned, 0 shared-memory, 1 register-resident)")
    ap.add_argument("--z-kernel", type=int, default=-1, choices=(-1, 0, 1),
                    help="--passes: FP32 / df64 z-pass kernel (-1 tuned, 0 plain, 1 TMA-staged)")
    ap.add_argument("--experiments", action="store_true",
                    help="the paper's GPe convergence experiment (accuracy vs iterations) instead of the bench")
    ap.add_argument("--exp-n", type=int, default=300, help="grid points per side of --experiments")
    ap.add_argument("--fp64-peak", action="store_true", help="measure the FP64 rate (cuBLAS DGEMM)")
    ap.add_argument("--cpu-configs", action="store_true",
                    help="time the CPU oracle on every configuration (median of 5)")
    ap.add_argument("--warm-serving", action="store_true",
                    help="served warm starts: sequences of requests sharing eps, cold against warm")
    ap.add_argument("--warm-count", type=int, default=8, help="--warm-serving: requests per sequence")
    args = ap.parse_args()
    if args.fp64_peak:
        run_fp64_peak(args)
        return
    if args.cpu_configs:
        run_cpu_configs(args)
        return
    if args.warm_serving:
        run_warm_serving(args)
        return
    if args.passes:
        run_passes(args)
        return
    if args.experiments:
        run_experiments(args)
        return
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
