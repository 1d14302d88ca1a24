"""Thin ctypes binding of libgps.so (include/gps.h).

Argument marshalling only: every step of a solve runs in the library's CUDA
kernels.  Device arrays are torch CUDA tensors (contiguous float64 on the
context's device); the *_host entry points take contiguous float64 numpy
arrays.  The library must have been built (``build.build()``); importing
this module without it raises -- there is no fallback.
"""
import ctypes
import os

import numpy as np

from .build import LIB

GPS_OK, GPS_ERR_INVALID, GPS_ERR_NOMEM, GPS_ERR_NOT_CONVERGED = 0, 1, 2, 3
GPS_ERR_BREAKDOWN, GPS_ERR_TIMEOUT, GPS_ERR_CUDA, GPS_PENDING = 4, 5, 6, 7
GPS_BC_FREE, GPS_BC_PERIODIC, GPS_BC_SURFACE, GPS_BC_WIRE = 0, 1, 2, 3
GPS_FP64, GPS_MIXED, GPS_DF64, GPS_MIXED_DF64 = 0, 1, 2, 3
GPS_GPE, GPS_LPB, GPS_NLPB, GPS_MPB = 0, 1, 2, 3
GPS_OUTER_NEWTON, GPS_OUTER_PRINTED = 0, 1
GPS_FORCING_EW2, GPS_FORCING_RATIO = 0, 1
GPS_PCG, GPS_SC, GPS_PSD = 0, 1, 2
GPS_MAX_DIIS = 8
METHOD = {"pcg": GPS_PCG, "sc": GPS_SC, "psd": GPS_PSD}
GPS_MAX_SPECIES = 8
KIND = {"gpe": GPS_GPE, "lpb": GPS_LPB, "nlpb": GPS_NLPB, "mpb": GPS_MPB}


class gps_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("hx", ctypes.c_double), ("hy", ctypes.c_double), ("hz", ctypes.c_double),
                ("bc", ctypes.c_int)]


class gps_electrolyte(ctypes.Structure):
    _fields_ = [("nspecies", ctypes.c_int), ("z", ctypes.c_int * GPS_MAX_SPECIES),
                ("c_molar", ctypes.c_double * GPS_MAX_SPECIES),
                ("temperature", ctypes.c_double), ("eps0", ctypes.c_double),
                ("radius_angstrom", ctypes.c_double * GPS_MAX_SPECIES), ("packing", ctypes.c_double),
                ("exclusion", ctypes.c_void_p)]


class gps_opts(ctypes.Structure):
    _fields_ = [("tol_abs", ctypes.c_double), ("tol_rel", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("max_outer", ctypes.c_int),
                ("tol_outer", ctypes.c_double), ("eta", ctypes.c_double),
                ("outer_mode", ctypes.c_int), ("forcing", ctypes.c_double),
                ("precision", ctypes.c_int), ("mixed_switch", ctypes.c_double),
                ("certify", ctypes.c_int), ("warm_start", ctypes.c_int),
                ("method", ctypes.c_int), ("alpha", ctypes.c_double), ("diis", ctypes.c_int),
                ("forcing_rule", ctypes.c_int)]


class gps_report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("outer_iters", ctypes.c_int),
                ("fp64_iters", ctypes.c_int), ("res0", ctypes.c_double), ("res", ctypes.c_double),
                ("outer_res", ctypes.c_double), ("background", ctypes.c_double),
                ("fixed_point_res", ctypes.c_double), ("time_ms", ctypes.c_double),
                ("warm", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class gps_request(ctypes.Structure):
    _fields_ = [("grid", gps_grid), ("kind", ctypes.c_int), ("el", gps_electrolyte),
                ("opts", gps_opts), ("rho_host", ctypes.c_void_p), ("eps_host", ctypes.c_void_p),
                ("phi_host", ctypes.c_void_p)]


_P = ctypes.c_void_p
_SIGS = {
    "gps_default_opts": (None, [ctypes.POINTER(gps_opts)]),
    "gps_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "gps_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_size_t]),
    "gps_destroy": (None, [_P]),
    "gps_bytes_in_use": (ctypes.c_size_t, [_P]),
    "gps_gpe_solve": (ctypes.c_int, [_P, ctypes.POINTER(gps_grid), _P, _P, _P,
                                     ctypes.POINTER(gps_opts), ctypes.POINTER(gps_report), _P]),
    "gps_pb_solve": (ctypes.c_int, [_P, ctypes.POINTER(gps_grid), _P, _P,
                                    ctypes.POINTER(gps_electrolyte), ctypes.c_int, _P,
                                    ctypes.POINTER(gps_opts), ctypes.POINTER(gps_report), _P]),
    "gps_gpe_solve_host": (ctypes.c_int, [_P, ctypes.POINTER(gps_grid), _P, _P, _P,
                                          ctypes.POINTER(gps_opts), ctypes.POINTER(gps_report), _P]),
    "gps_pb_solve_host": (ctypes.c_int, [_P, ctypes.POINTER(gps_grid), _P, _P,
                                         ctypes.POINTER(gps_electrolyte), ctypes.c_int, _P,
                                         ctypes.POINTER(gps_opts), ctypes.POINTER(gps_report), _P]),
    "gps_setup_fields": (ctypes.c_int, [_P, ctypes.POINTER(gps_grid), _P, _P, _P, _P]),
    "gps_vacuum_solve": (ctypes.c_int, [_P, ctypes.POINTER(gps_grid), _P, _P, _P]),
    "gps_precondition": (ctypes.c_int, [_P, ctypes.POINTER(gps_grid), _P, _P, _P, ctypes.c_int, _P]),
    "gps_ionic_charge": (ctypes.c_int, [_P, ctypes.POINTER(gps_grid), _P, _P,
                                        ctypes.POINTER(gps_electrolyte), _P, _P]),
    "gps_vacuum_solve_noalloc": (ctypes.c_int, [ctypes.POINTER(gps_grid), _P, _P, _P]),
    "gps_set_radix_order": (ctypes.c_int, [ctypes.c_int]),
    "gps_set_x_kernel": (ctypes.c_int, [ctypes.c_int]),
    "gps_set_z_kernel": (ctypes.c_int, [ctypes.c_int]),
    "gps_set_engine_mode": (ctypes.c_int, [ctypes.c_int]),
    "gps_sccs_eps": (ctypes.c_int, [_P, ctypes.c_size_t, _P, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, _P, _P, _P]),
    "gps_polarization_charge": (ctypes.c_int, [_P, ctypes.POINTER(gps_grid), _P, _P, _P, _P, _P]),
    "gps_v_eps": (ctypes.c_int, [_P, ctypes.POINTER(gps_grid), _P, _P, _P, _P]),
    "gps_electrostatic_energy": (ctypes.c_int, [_P, ctypes.POINTER(gps_grid), _P, _P, _P,
                                                ctypes.POINTER(ctypes.c_double),
                                                ctypes.POINTER(ctypes.c_double), _P]),
    "gps_batch_solve": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(gps_request),
                                       ctypes.POINTER(gps_report)]),
    "gps_server_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_size_t, ctypes.c_int]),
    "gps_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(gps_request), ctypes.POINTER(ctypes.c_ulonglong)]),
    "gps_server_poll": (ctypes.c_int, [_P, ctypes.c_ulonglong, ctypes.POINTER(gps_report)]),
    "gps_server_wait": (ctypes.c_int, [_P, ctypes.c_ulonglong, ctypes.POINTER(gps_report)]),
    "gps_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_int)]),
    "gps_server_destroy": (None, [_P]),
    "gps_set_profiling": (ctypes.c_int, [_P, ctypes.c_int]),
    "gps_get_profile": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    "gps_kernel_launches": (ctypes.c_ulonglong, []),
}
GPS_PROFILE_KINDS = 20
_PASSES = ["x_fwd", "y_fwd", "z", "y_inv", "x_inv"]
# kinds 0-4: passes of the FP64 spectrum; 10-14 double-float; 15-19 FP32
PROFILE_KINDS = (_PASSES + ["update_p", "update_r", "other", "stencil", "sc_vector"]
                 + [k + "_df64" for k in _PASSES] + [k + "_fp32" for k in _PASSES])

_lib = None


def load():
    """Load libgps.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError("libgps.so is not built; run paper_1509_00680_gb300.build.build()")
        lib = ctypes.CDLL(LIB)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


class GpsError(RuntimeError):
    def __init__(self, status, where):
        msg = load().gps_status_string(status).decode()
        super().__init__("%s: %s (status %d)" % (where, msg, status))
        self.status = status


def _check(status, where, allow=(GPS_OK,)):
    if status not in allow:
        raise GpsError(status, where)
    return status


def make_grid(nx, ny, nz, hx, hy, hz, bc):
    return gps_grid(int(nx), int(ny), int(nz), float(hx), float(hy), float(hz), int(bc))


def grid_from(g):
    """gps_grid from any object with nx..hz and bc attributes."""
    return make_grid(g.nx, g.ny, g.nz, g.hx, g.hy, g.hz, g.bc)


def make_electrolyte(z, c_molar, temperature=300.0, eps0=78.36, radius_angstrom=None, packing=0.0,
                     exclusion=None):
    """Electrolyte description; radius_angstrom (per species) and packing > 0
    select the steric distribution of the modified PB problem ("mpb").
    exclusion: the ion-exclusion function gamma on the grid, a float64 CUDA
    tensor (device entry points) or a C-contiguous float64 numpy array
    (host entry points); the caller keeps it alive while it is in use."""
    el = gps_electrolyte()
    el.nspecies = len(z)
    for i, (zi, ci) in enumerate(zip(z, c_molar)):
        el.z[i] = int(zi)
        el.c_molar[i] = float(ci)
        if radius_angstrom is not None:
            el.radius_angstrom[i] = float(radius_angstrom[i])
    el.temperature = float(temperature)
    el.eps0 = float(eps0)
    el.packing = float(packing)
    if exclusion is not None:
        el.exclusion = _dev(exclusion) if hasattr(exclusion, "is_cuda") else _host(exclusion)
    return el


def default_opts(**kw):
    o = gps_opts()
    load().gps_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _dev(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _host(a):
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise TypeError("expected a C-contiguous float64 numpy array")
    return ctypes.c_void_p(a.ctypes.data)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(int(stream))


class Context:
    """Owns one gps_ctx (plans, workspaces) on a CUDA device."""

    def __init__(self, device=0, hbm_budget_bytes=0):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.gps_create(ctypes.byref(h), int(device), int(hbm_budget_bytes)), "gps_create")
        self.handle = h

    def close(self):
        if self.handle:
            load().gps_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bytes_in_use(self):
        return int(load().gps_bytes_in_use(self.handle))

    def set_profiling(self, kinds=None):
        """Time the kernels of the given kinds (names of PROFILE_KINDS); None or
        an empty list turns profiling off, "all" times every kind."""
        if kinds == "all":
            mask = (1 << GPS_PROFILE_KINDS) - 1
        else:
            mask = 0
            for k in (kinds or []):
                mask |= 1 << PROFILE_KINDS.index(k)
        _check(load().gps_set_profiling(self.handle, mask), "gps_set_profiling")

    def get_profile(self, reset=False):
        """{kind: (launches, total_ms)} of the kernels timed since the last reset."""
        n = (ctypes.c_longlong * GPS_PROFILE_KINDS)()
        t = (ctypes.c_double * GPS_PROFILE_KINDS)()
        _check(load().gps_get_profile(self.handle, n, t, int(bool(reset))), "gps_get_profile")
        return {k: (int(n[i]), float(t[i])) for i, k in enumerate(PROFILE_KINDS)}

    # --- device arrays -------------------------------------------------
    def gpe_solve(self, grid, rho, eps, phi, opts=None, stream=None, allow=(GPS_OK,)):
        rep = gps_report()
        o = opts if opts is not None else default_opts()
        s = load().gps_gpe_solve(self.handle, ctypes.byref(grid), _dev(rho), _dev(eps), _dev(phi),
                                 ctypes.byref(o), ctypes.byref(rep), _stream(stream))
        _check(s, "gps_gpe_solve", allow)
        return rep

    def pb_solve(self, grid, rho, eps, electrolyte, kind, phi, opts=None, stream=None, allow=(GPS_OK,)):
        rep = gps_report()
        o = opts if opts is not None else default_opts()
        s = load().gps_pb_solve(self.handle, ctypes.byref(grid), _dev(rho), _dev(eps),
                                ctypes.byref(electrolyte), int(KIND.get(kind, kind)), _dev(phi),
                                ctypes.byref(o), ctypes.byref(rep), _stream(stream))
        _check(s, "gps_pb_solve", allow)
        return rep

    # --- host arrays ---------------------------------------------------
    def gpe_solve_host(self, grid, rho, eps, phi, opts=None, stream=None):
        rep = gps_report()
        o = opts if opts is not None else default_opts()
        s = load().gps_gpe_solve_host(self.handle, ctypes.byref(grid), _host(rho), _host(eps),
                                      _host(phi), ctypes.byref(o), ctypes.byref(rep), _stream(stream))
        _check(s, "gps_gpe_solve_host")
        return rep

    def pb_solve_host(self, grid, rho, eps, electrolyte, kind, phi, opts=None, stream=None,
                      allow=(GPS_OK,)):
        rep = gps_report()
        o = opts if opts is not None else default_opts()
        s = load().gps_pb_solve_host(self.handle, ctypes.byref(grid), _host(rho), _host(eps),
                                     ctypes.byref(electrolyte), int(KIND.get(kind, kind)),
                                     _host(phi), ctypes.byref(o), ctypes.byref(rep), _stream(stream))
        _check(s, "gps_pb_solve_host", allow)
        return rep

    # --- steps -----------------------------------------------------------
    def setup_fields(self, grid, eps, s, q, stream=None):
        _check(load().gps_setup_fields(self.handle, ctypes.byref(grid), _dev(eps), _dev(s), _dev(q),
                                       _stream(stream)), "gps_setup_fields")

    def vacuum_solve(self, grid, sigma, w, stream=None):
        _check(load().gps_vacuum_solve(self.handle, ctypes.byref(grid), _dev(sigma), _dev(w),
                                       _stream(stream)), "gps_vacuum_solve")

    def precondition(self, grid, s, r, v, precision=GPS_FP64, stream=None):
        _check(load().gps_precondition(self.handle, ctypes.byref(grid), _dev(s), _dev(r), _dev(v),
                                       int(precision), _stream(stream)), "gps_precondition")

    def ionic_charge(self, grid, phi, eps, electrolyte, out, stream=None):
        _check(load().gps_ionic_charge(self.handle, ctypes.byref(grid), _dev(phi), _dev(eps),
                                       ctypes.byref(electrolyte), _dev(out), _stream(stream)),
               "gps_ionic_charge")

    # --- DFT-facing quantities ------------------------------------------
    def sccs_eps(self, rho_elec, eps, deps=None, rho_max=5e-3, rho_min=1e-4, eps0=78.36, stream=None):
        _check(load().gps_sccs_eps(self.handle, rho_elec.numel(), _dev(rho_elec), rho_max, rho_min, eps0,
                                   _dev(eps), _dev(deps) if deps is not None else None, _stream(stream)),
               "gps_sccs_eps")

    def polarization_charge(self, grid, rho, eps, phi, out, stream=None):
        _check(load().gps_polarization_charge(self.handle, ctypes.byref(grid), _dev(rho), _dev(eps),
                                              _dev(phi), _dev(out), _stream(stream)),
               "gps_polarization_charge")

    def v_eps(self, grid, deps, phi, out, stream=None):
        _check(load().gps_v_eps(self.handle, ctypes.byref(grid), _dev(deps), _dev(phi), _dev(out),
                                _stream(stream)), "gps_v_eps")

    def electrostatic_energy(self, grid, rho, eps, phi, stream=None):
        """(1/2 sum rho phi h^3, 1/(8 pi) sum eps |grad phi|^2 h^3)."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(load().gps_electrostatic_energy(self.handle, ctypes.byref(grid), _dev(rho), _dev(eps),
                                               _dev(phi), ctypes.byref(a), ctypes.byref(b),
                                               _stream(stream)), "gps_electrostatic_energy")
        return a.value, b.value


def set_radix_order(order):
    """-1: tune the FFT radix order (default); 0..3: use that order for new plans."""
    _check(load().gps_set_radix_order(int(order)), "gps_set_radix_order")


def set_x_kernel(kind):
    """FP32 x passes: -1 tuned (default), 0 shared-memory kernels, 1 register-resident."""
    _check(load().gps_set_x_kernel(int(kind)), "gps_set_x_kernel")


def set_z_kernel(kind):
    """FP32 / df64 z pass: -1 tuned (default), 0 plain column kernel, 1 TMA-staged."""
    _check(load().gps_set_z_kernel(int(kind)), "gps_set_z_kernel")


def set_engine_mode(asynchronous):
    """Batching engine: True pools advance independently (default), False lockstep."""
    _check(load().gps_set_engine_mode(1 if asynchronous else 0), "gps_set_engine_mode")


def make_request(grid, kind, rho, eps, phi, electrolyte=None, opts=None):
    """A gps_request over host arrays (C-contiguous float64 numpy arrays that
    must stay alive until the request completes)."""
    r = gps_request()
    r.grid = grid
    r.kind = int(KIND.get(kind, kind))
    if electrolyte is not None:
        r.el = electrolyte
    r.opts = opts if opts is not None else default_opts()
    r.rho_host = _host(rho)
    r.eps_host = _host(eps)
    r.phi_host = _host(phi)
    return r


def batch_solve(ctx, requests, allow=(GPS_OK,)):
    """Solve gps_requests together (continuous batching); returns the reports."""
    n = len(requests)
    arr = (gps_request * n)(*requests)
    reps = (gps_report * n)()
    s = load().gps_batch_solve(ctx.handle, n, arr, reps)
    _check(s, "gps_batch_solve", allow)
    return list(reps)


class Server:
    """Asynchronous serving loop (gps_server_*)."""

    def __init__(self, device=0, hbm_budget_bytes=0, max_slots=0):
        h = ctypes.c_void_p()
        _check(load().gps_server_create(ctypes.byref(h), int(device), int(hbm_budget_bytes),
                                        int(max_slots)), "gps_server_create")
        self.handle = h
        self._keep = {}

    def submit(self, request, keep=None):
        t = ctypes.c_ulonglong()
        _check(load().gps_server_submit(self.handle, ctypes.byref(request), ctypes.byref(t)),
               "gps_server_submit")
        self._keep[t.value] = (request, keep)
        return t.value

    def poll(self, ticket):
        rep = gps_report()
        s = load().gps_server_poll(self.handle, ctypes.c_ulonglong(ticket), ctypes.byref(rep))
        if s == GPS_PENDING:
            return None
        self._keep.pop(ticket, None)
        return s, rep

    def wait(self, ticket, timeout=None):
        """(status, report) of a ticket once it is done.  timeout (seconds):
        poll instead of blocking, and raise TimeoutError past the deadline."""
        rep = gps_report()
        if timeout is None:
            s = load().gps_server_wait(self.handle, ctypes.c_ulonglong(ticket), ctypes.byref(rep))
        else:
            import time
            deadline = time.monotonic() + timeout
            while True:
                s = load().gps_server_poll(self.handle, ctypes.c_ulonglong(ticket), ctypes.byref(rep))
                if s != GPS_PENDING:
                    break
                if time.monotonic() > deadline:
                    raise TimeoutError("server ticket %d not done after %.0f s" % (ticket, timeout))
                time.sleep(0.002)
        self._keep.pop(ticket, None)
        return s, rep

    def stats(self):
        b = ctypes.c_size_t()
        m = ctypes.c_int()
        _check(load().gps_server_stats(self.handle, ctypes.byref(b), ctypes.byref(m)), "gps_server_stats")
        return {"bytes_in_use": b.value, "max_concurrent": m.value}

    def close(self):
        if self.handle:
            load().gps_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def vacuum_solve_noalloc(grid, sigma, w, stream=None):
    """w = S(sigma) without any device allocation (periodic / surface BC,
    sizes bounded by the library's fixed 8 MiB scratch array).  Calls that
    overlap on the GPU share that array and race; serialize them."""
    _check(load().gps_vacuum_solve_noalloc(ctypes.byref(grid), _dev(sigma), _dev(w), _stream(stream)),
           "gps_vacuum_solve_noalloc")


gps_vacuum_solve_noalloc = vacuum_solve_noalloc


def kernel_launches():
    return int(load().gps_kernel_launches())


# C-ABI names, for callers that prefer the flat interface.
def gps_create(device=0, hbm_budget_bytes=0):
    return Context(device, hbm_budget_bytes)


def gps_destroy(ctx):
    ctx.close()


def gps_gpe_solve(ctx, grid, rho, eps, phi, opts=None, stream=None):
    return ctx.gpe_solve(grid, rho, eps, phi, opts, stream)


def gps_pb_solve(ctx, grid, rho, eps, electrolyte, kind, phi, opts=None, stream=None):
    return ctx.pb_solve(grid, rho, eps, electrolyte, kind, phi, opts, stream)


def gps_gpe_solve_host(ctx, grid, rho, eps, phi, opts=None, stream=None):
    return ctx.gpe_solve_host(grid, rho, eps, phi, opts, stream)


def gps_pb_solve_host(ctx, grid, rho, eps, electrolyte, kind, phi, opts=None, stream=None):
    return ctx.pb_solve_host(grid, rho, eps, electrolyte, kind, phi, opts, stream)


def gps_setup_fields(ctx, grid, eps, s, q, stream=None):
    return ctx.setup_fields(grid, eps, s, q, stream)


def gps_vacuum_solve(ctx, grid, sigma, w, stream=None):
    return ctx.vacuum_solve(grid, sigma, w, stream)


def gps_precondition(ctx, grid, s, r, v, precision=GPS_FP64, stream=None):
    return ctx.precondition(grid, s, r, v, precision, stream)


def gps_ionic_charge(ctx, grid, phi, eps, electrolyte, out, stream=None):
    return ctx.ionic_charge(grid, phi, eps, electrolyte, out, stream)
