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


def test_noalloc_limits_are_enforced_before_any_device_work():
    """ec3r_align_submaps_noalloc checks its sizes against the fixed scratch
    before touching the device, so each limit the header states can be checked
    on the host: the pointers below are placeholders that are never used."""
    l = ec3r.lib()
    f = l.ec3r_align_submaps_noalloc
    P, I64 = ctypes.c_void_p, ctypes.c_int64
    f.argtypes = [P, P, I64, I64, ctypes.c_int, I64, P, P, P, P,
                  ctypes.POINTER(ec3r.AlignOpts), P, P, P, P]
    f.restype = ctypes.c_int
    text = open(os.path.join(ROOT, "include", "ec3r.h")).read()
    lim = {k: int(v) for k, v in re.findall(r"#define EC3R_NOALLOC_(MAX_\w+) (\d+)", text)}
    assert set(lim) == {"MAX_PAIRS", "MAX_LINKS", "MAX_TILES"}
    o = ec3r.AlignOpts()
    l.ec3r_align_opts_default(ctypes.byref(o))
    x = P(256)

    def call(n_pairs, n_links, hw, opts=o):
        return f(x, x, 4, hw, n_pairs, n_links, x, x, x, None, ctypes.byref(opts), x, x, None,
                 None)

    assert call(0, 0, 64) == 0                                     # nothing to do
    assert call(lim["MAX_PAIRS"] + 1, 1, 64) == 1
    assert call(1, lim["MAX_LINKS"] + 1, 64) == 1
    tiles_per_link = lim["MAX_TILES"] // lim["MAX_LINKS"] + 1     # one link more than fits
    assert call(1, lim["MAX_LINKS"], tiles_per_link * 8192) == 1
    bad = ec3r.AlignOpts()
    l.ec3r_align_opts_default(ctypes.byref(bad))
    bad.iters = 0
    assert call(1, 1, 64, bad) == 1
    bad.iters, bad.want_cost = 10, 1                               # cost wanted, no buffer
    assert call(1, 1, 64, bad) == 1


def test_context_settings_reject_bad_arguments_on_the_host():
    """The context settings and the variant table validate their arguments
    before any device work: a NULL context is EC3R_ERR_INVALID_ARG (1) for
    every setter, the token of a NULL context is 0, and the variant table
    answers every index in range and rejects the rest."""
    l = ec3r.lib()
    assert l.ec3r_set_wait_limit(None, 1.0) == 1
    assert l.ec3r_inject(None, 0) == 1
    assert l.ec3r_align_set_variant(None, 0) == 1
    assert l.ec3r_align_backward_set_ctas_per_sm(None, 0) == 1
    assert l.ec3r_align_token(None) == 0
    n = l.ec3r_align_variant_count()
    assert n >= 2
    t, c, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    persistent = []
    for v in range(n):
        assert l.ec3r_align_variant_info(v, ctypes.byref(t), ctypes.byref(c), ctypes.byref(p)) == 0
        assert t.value % 4096 == 0 and 1 <= c.value <= 4 and p.value in (0, 1)
        persistent.append(p.value)
    assert 0 in persistent and 1 in persistent
    for v in (-1, n):
        assert l.ec3r_align_variant_info(v, ctypes.byref(t), ctypes.byref(c), ctypes.byref(p)) == 1
