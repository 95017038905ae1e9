"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
symbol that include/ec3r.h declares (no compute calls: this host has no GPU)."""
import ctypes
import os
import re

from paper_2510_02080_b300 import build, ec3r

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "ec3r.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ec3r_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    build.build()
    lib = ctypes.CDLL(ec3r.LIB_PATH)
    names = declared_symbols()
    assert "ec3r_align_submaps" in names and "ec3r_fuse_points" in names
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(ec3r.EXPORTS) == sorted(n for n in names if n in ec3r.EXPORTS)
    assert set(names) <= set(ec3r.EXPORTS), set(names) - set(ec3r.EXPORTS)


def test_version_and_status_strings():
    l = ec3r.lib()
    assert l.ec3r_version().decode().endswith("sm_103a")
    assert l.ec3r_status_string(0) == b"ok"
    assert l.ec3r_status_string(4) == b"output capacity exceeded"


def test_struct_layouts_match_header():
    assert ctypes.sizeof(ec3r.Sim3) == 13 * 8
    assert ctypes.sizeof(ec3r.AlignOpts) == 24
    o = ec3r.AlignOpts()
    ec3r.lib().ec3r_align_opts_default(ctypes.byref(o))
    assert abs(o.huber_delta - 0.02) < 1e-9 and o.iters == 10 and o.precision == 0
