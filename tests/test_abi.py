"""The C ABI library builds, loads and exports every entry point that
include/dash.h declares; host-side argument checks run without a GPU."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def _declared():
    names = set()
    for fn in os.listdir(HEADER_DIR):
        if fn.endswith(".h"):
            src = open(os.path.join(HEADER_DIR, fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(dash_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2305_18376_gb300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
    from paper_2305_18376_gb300 import _native
    return _native.load()


def test_header_declares_the_problem_statement_calls():
    names = _declared()
    for n in ["dash_init", "dash_append_rows", "dash_append_slices", "dash_update",
              "dash_factors", "dash_fitness", "dash_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2305_18376_gb300 import build as B
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (dash_[a-z0-9_]+)\b", out))
    missing = _declared() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_binding_covers_every_declared_symbol(lib):
    from paper_2305_18376_gb300 import _native
    bound = {n for n, _, _ in _native.SIGNATURES}
    assert _declared() <= bound


def test_status_strings_and_default_config(lib):
    from paper_2305_18376_gb300 import _native
    assert lib.dash_status_string(0) == b"ok"
    assert lib.dash_status_string(1) == b"invalid argument"
    cfg = _native.Config()
    lib.dash_config_default(C.byref(cfg), 88, 10, 0.98)
    assert (cfg.J, cfg.R, cfg.n_sweeps) == (88, 10, 1)
    assert abs(cfg.lambda_ - 0.98) < 1e-15


def test_init_rejects_bad_arguments_before_touching_the_device(lib):
    from paper_2305_18376_gb300 import _native
    for field, value in [("J", 0), ("R", 65), ("R", 0), ("lambda_", 0.0), ("lambda_", 1.5),
                         ("n_sweeps", 0), ("n_sweeps", 65), ("mode", 7), ("precision", 9)]:
        cfg = _native.Config()
        lib.dash_config_default(C.byref(cfg), 8, 3, 0.9)
        setattr(cfg, field, value)
        h = C.c_void_p()
        assert lib.dash_init(C.byref(cfg), C.byref(h)) == 1, field
        assert not h.value


def test_config_bytes_counts_the_allocation_list_without_a_device(lib):
    """dash_config_bytes runs dash_init's allocation list in a counting mode:
    no device is touched, bad configs are rejected like dash_init rejects
    them, and the count grows with the capacities as the per-slice and
    per-row buffers say (D_k, c_k, W(k,:) in 8-byte words; staged X in the
    input dtype, twice for the double staging)."""
    from paper_2305_18376_gb300 import _native

    def count(**kw):
        cfg = _native._config(lib, **{"J": 64, "R": 8, "lam": 0.9, "precision": "f16x3", **kw})
        dev, host = C.c_int64(), C.c_int64()
        assert lib.dash_config_bytes(C.byref(cfg), C.byref(dev), C.byref(host)) == 0
        return dev.value, host.value

    base = dict(max_slices=4096, max_rows=8192, max_segments=4096)
    d0, h0 = count(**base)
    assert d0 > 0 and h0 > 0
    # 4096 more slices: D (R·R), c (R), W (R) in 8 bytes, plus small per-slice words
    d1, _ = count(**{**base, "max_slices": 8192})
    per_slice = (d1 - d0) / 4096
    assert 8 * (8 * 8 + 2 * 8) <= per_slice < 8 * (8 * 8 + 2 * 8) + 128
    # 8192 more rows: at least the two staging buffers of J FP32 values a row
    d2, _ = count(**{**base, "max_rows": 16384})
    assert (d2 - d0) / 8192 >= 2 * 64 * 4
    # FP64 input doubles the two staging buffers and nothing else (FP64 products)
    d4, _ = count(**base, precision="fp64", input_dtype="f32")
    d5, _ = count(**base, precision="fp64", input_dtype="f64")
    assert d5 - d4 == 2 * 8192 * 64 * 4
    cfg = _native._config(lib, J=64, R=65, lam=0.9)
    assert lib.dash_config_bytes(C.byref(cfg), None, None) == 1
