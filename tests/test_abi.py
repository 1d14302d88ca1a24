"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/gps.h declares; the ctypes structures match the header's layout.
No compute call is made (no GPU needed)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gps.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gps_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1509_00680_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["gps_create", "gps_destroy", "gps_gpe_solve", "gps_pb_solve",
                     "gps_gpe_solve_host", "gps_pb_solve_host", "gps_setup_fields",
                     "gps_vacuum_solve", "gps_precondition", "gps_ionic_charge"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1509_00680_gb300 import gps
    assert set(declared_functions()) <= set(gps._SIGS)


def test_struct_layout_matches_header(tmp_path):
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_1509_00680_gb300 import gps
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "gps.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(gps_grid),'
                    ' sizeof(gps_electrolyte), sizeof(gps_opts), sizeof(gps_report),'
                    ' offsetof(gps_opts, precision), offsetof(gps_report, time_ms),'
                    ' sizeof(gps_request), offsetof(gps_request, phi_host));'
                    ' printf("%zu %zu %zu\\n", offsetof(gps_opts, diis), offsetof(gps_electrolyte, exclusion),'
                    ' offsetof(gps_request, opts)); return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    want = [ctypes.sizeof(gps.gps_grid), ctypes.sizeof(gps.gps_electrolyte),
            ctypes.sizeof(gps.gps_opts), ctypes.sizeof(gps.gps_report),
            gps.gps_opts.precision.offset, gps.gps_report.time_ms.offset,
            ctypes.sizeof(gps.gps_request), gps.gps_request.phi_host.offset,
            gps.gps_opts.diis.offset, gps.gps_electrolyte.exclusion.offset, gps.gps_request.opts.offset]
    assert [int(x) for x in out] == want


def test_default_opts_and_status_strings(lib):
    from paper_1509_00680_gb300 import gps
    o = gps.default_opts()
    assert o.tol_abs == 1e-10 and o.max_iter == 500 and o.precision == gps.GPS_FP64
    assert gps.load().gps_status_string(gps.GPS_ERR_BREAKDOWN) == b"PCG breakdown"
    assert gps.load().gps_create(None, 0, 0) == gps.GPS_ERR_INVALID


def test_new_defaults_and_host_side_argument_checks(lib):
    """Defaults of the solver options and argument checks that return before
    any CUDA call (NULL context or pointers, option ranges)."""
    from paper_1509_00680_gb300 import gps
    o = gps.default_opts()
    assert o.forcing == 0.3 and o.eta == 0.6 and o.method == gps.GPS_PCG
    assert o.forcing_rule == 0            # GPS_FORCING_EW2
    assert o.alpha == 0.0 and o.diis == 0 and o.warm_start == 0 and o.mixed_switch == 1e-2
    L = gps.load()
    assert L.gps_set_radix_order(4) == gps.GPS_ERR_INVALID
    assert L.gps_set_radix_order(-2) == gps.GPS_ERR_INVALID
    assert L.gps_set_radix_order(-1) == gps.GPS_OK
    assert L.gps_set_x_kernel(2) == gps.GPS_ERR_INVALID
    assert L.gps_set_x_kernel(-2) == gps.GPS_ERR_INVALID
    assert L.gps_set_x_kernel(-1) == gps.GPS_OK
    assert L.gps_set_z_kernel(2) == gps.GPS_ERR_INVALID
    assert L.gps_set_z_kernel(-1) == gps.GPS_OK
    g = gps.gps_grid()
    rep = gps.gps_report()
    assert L.gps_gpe_solve(None, ctypes.byref(g), None, None, None, ctypes.byref(o), ctypes.byref(rep),
                           None) == gps.GPS_ERR_INVALID
    assert L.gps_sccs_eps(None, 10, None, 5e-3, 1e-4, 78.36, None, None, None) == gps.GPS_ERR_INVALID
    assert L.gps_polarization_charge(None, ctypes.byref(g), None, None, None, None, None) == gps.GPS_ERR_INVALID
    assert L.gps_v_eps(None, ctypes.byref(g), None, None, None, None) == gps.GPS_ERR_INVALID
    e1, e2 = ctypes.c_double(), ctypes.c_double()
    assert L.gps_electrostatic_energy(None, ctypes.byref(g), None, None, None, ctypes.byref(e1), ctypes.byref(e2),
                                      None) == gps.GPS_ERR_INVALID


def test_product_path_has_no_oracle_dependency():
    """The package never imports the oracle (it is test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_1509_00680_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
