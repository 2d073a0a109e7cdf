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
