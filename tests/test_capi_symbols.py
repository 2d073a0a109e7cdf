"""The C-ABI library builds, loads without a GPU and exports every entry
point declared in include/*.h (no compute calls here)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(amr_[a-z_0-9]+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_1812_03689_gb300 import build
    return build.build()


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("amr_create_hierarchy", "amr_deposit", "amr_solve", "amr_gather", "amr_destroy", "amr_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert declared_functions() <= exported


def test_binding_loads_and_host_only_calls_work(lib_path):
    from paper_1812_03689_gb300 import amrmg
    assert amrmg.last_error() == ""
    b = amrmg.hierarchy_bytes(64, 2, fill=0.05)
    assert b > 64 ** 3 * 8
    d, _keep = amrmg.make_desc(64, 0)
    assert d.n0 == 64 and d.brick == 8


def test_invalid_arguments_fail_before_device_work(lib_path):
    from paper_1812_03689_gb300 import amrmg
    d, _keep = amrmg.make_desc(5, 0)  # n0 < 8
    h = ctypes.c_void_p()
    rc = amrmg._lib.amr_create_hierarchy(ctypes.byref(d), None, None, None, None, 0, None, ctypes.byref(h))
    assert rc == amrmg.AMR_EINVAL and not h.value
    assert "invalid descriptor" in amrmg.last_error()
    assert amrmg._lib.amr_solve(None, None, None) == amrmg.AMR_EINVAL


def test_new_entry_points_reject_bad_arguments_before_device_work(lib_path):
    """Boundary conditions, regrid, gather buffer and the particle-side calls
    validate their arguments on the host (no GPU needed)."""
    from paper_1812_03689_gb300 import amrmg
    L = amrmg._lib
    h = ctypes.c_void_p()
    for kw in (dict(robin_d=0.0), dict(robin_d=-1.0), dict(robin_d=float("inf"))):
        d, _keep = amrmg.make_desc(16, 0, **kw)
        assert L.amr_create_hierarchy(ctypes.byref(d), None, None, None, None, 0, None, ctypes.byref(h)) \
            == amrmg.AMR_EINVAL
        assert "boundary condition" in amrmg.last_error()
    d, _keep = amrmg.make_desc(16, 0)
    d.bc = 7
    assert L.amr_create_hierarchy(ctypes.byref(d), None, None, None, None, 0, None, ctypes.byref(h)) \
        == amrmg.AMR_EINVAL
    n = ctypes.c_int(0)
    assert L.amr_regrid_boxes(None, 3, 0.5, 1, 2, None, 0, ctypes.byref(n)) == amrmg.AMR_EINVAL
    assert L.amr_transfer_phi(None, None) == amrmg.AMR_EINVAL
    assert L.amr_set_gather_buffer(None, 1) == amrmg.AMR_EINVAL
    assert L.amr_rescale_fields(None, 2.0) == amrmg.AMR_EINVAL
    c = (ctypes.c_double * 3)()
    S = ctypes.c_double()
    assert L.amr_domain_transform(None, None, None, 0, c, -0.5, None, None, None, ctypes.byref(S), None) \
        == amrmg.AMR_EINVAL
    assert L.amr_push(*([None] * 9), -1, 1.0, 0.1, None) == amrmg.AMR_EINVAL
    out = (ctypes.c_double * 9)()
    assert L.amr_moments(None, None, None, 0, out, None) == amrmg.AMR_EINVAL
    assert L.amr_solve_many(None, 0, None, 16, None) == amrmg.AMR_EINVAL
    arr = (ctypes.c_void_p * 2)(None, None)
    assert L.amr_solve_many(arr, 2, None, 16, None) == amrmg.AMR_EINVAL
