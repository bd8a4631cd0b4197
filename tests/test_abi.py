"""C-ABI checks that need no GPU: the library loads, exports every declared entry point, and its
host-side argument validation and sizing behave as include/irls.h states."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "irls.h")


@pytest.fixture(scope="module")
def L():
    from paper_2401_09961_gb300 import _binding
    if not os.path.exists(_binding.LIB_PATH):
        from paper_2401_09961_gb300 import build
        build.build()
    return _binding.lib()


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(irls_[a-z0-9_]+)\s*\(",
                       txt, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("irls_unwrap", "irls_unwrap_ex", "irls_plan_create", "irls_plan_destroy",
                 "irls_workspace_bytes", "irls_opts_default", "irls_status_string"):
        assert must in names


def test_every_declared_symbol_is_exported(L):
    from paper_2401_09961_gb300 import _binding
    names = declared_functions()
    for n in names:
        assert hasattr(L, n), f"{n} declared in irls.h but not exported"
        assert n in _binding.SIGNATURES, f"{n} has no Python signature"


def test_opts_default(L):
    from paper_2401_09961_gb300 import _binding
    o = _binding.default_opts()
    assert abs(o.tau - 1e-2) < 1e-9 and abs(o.delta - 1e-6) < 1e-12
    assert o.outer_iters == 20 and o.cg_max_iter == 1000 and o.precision == 0
    assert o.warm_start == 1
    assert L.irls_opts_default(None) == -1


def test_workspace_bytes_and_validation(L):
    from paper_2401_09961_gb300 import _binding
    o = _binding.default_opts()
    n1 = L.irls_workspace_bytes(256, 256, ctypes.byref(o))
    n2 = L.irls_workspace_bytes(512, 512, ctypes.byref(o))
    assert 0 < n1 < n2
    # 21 float32 planes at least
    assert n2 >= 21 * 512 * 512 * 4
    assert L.irls_workspace_bytes(0, 10, ctypes.byref(o)) == 0
    assert L.irls_workspace_bytes(10, -1, ctypes.byref(o)) == 0
    bad = _binding.default_opts(tau=-1.0)
    assert L.irls_workspace_bytes(10, 10, ctypes.byref(bad)) == 0


def test_plan_create_rejects_bad_arguments_before_device_work(L):
    from paper_2401_09961_gb300 import _binding
    h = ctypes.c_void_p()
    o = _binding.default_opts()
    assert L.irls_plan_create(0, 5, ctypes.byref(o), ctypes.byref(h)) == -2
    assert L.irls_plan_create(5, 0, ctypes.byref(o), ctypes.byref(h)) == -2
    assert L.irls_plan_create(5, 5, ctypes.byref(o), None) == -1
    for kw in (dict(tau=0.0), dict(delta=-1.0), dict(cg_tol=-1.0), dict(outer_iters=300),
               dict(cg_max_iter=-2), dict(precision=7)):
        bad = _binding.default_opts(**kw)
        assert L.irls_plan_create(5, 5, ctypes.byref(bad), ctypes.byref(h)) == -1, kw
    assert L.irls_unwrap(None, None, 4, 4, 1e-3, 2, 1e-5, None, None) == -1
    assert L.irls_unwrap_ex(None, None, None, None, None, None, None, None, None, None, None) == -1
    assert L.irls_plan_destroy(None) == 0


def test_status_strings(L):
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7, -8):
        s = L.irls_status_string(code)
        assert isinstance(s, bytes) and len(s) > 0
    assert L.irls_status_string(12345) == b"unknown status"


def test_product_path_does_not_import_the_oracle():
    """The package (the CUDA path's binding) never imports oracle/: only tests, smoke() and
    bench.py's CPU legs may."""
    pkg = os.path.join(ROOT, "paper_2401_09961_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, flags=re.M), f
                assert "synthetic" not in re.findall(r"^\s*(?:from|import)\s+(\w+)", txt,
                                                     flags=re.M), f


def test_workspace_by_precision(L):
    """Host-side sizing: the float16 plan holds the single-part direct buffers plus the folded
    form's; split bf16 holds two parts of the direct buffers plus the folded form's."""
    from paper_2401_09961_gb300 import _binding
    n = {p: L.irls_workspace_bytes(512, 512, ctypes.byref(_binding.default_opts(precision=p)))
         for p in ("fp32", "bf16", "fp16", "bf16x3")}
    assert 0 < n["fp32"] < n["bf16"] < n["fp16"] < n["bf16x3"], n
    bad = _binding.default_opts(precision=4)
    assert L.irls_workspace_bytes(512, 512, ctypes.byref(bad)) == 0


def test_new_entry_points_reject_null_handles(L):
    from paper_2401_09961_gb300 import _binding
    d, u = ctypes.c_int(), ctypes.c_int()
    assert L.irls_plan_set_tiles(None, 8, 8) == -1
    assert L.irls_plan_get_tiles(None, ctypes.byref(d), ctypes.byref(u)) == -1
    assert L.irls_plan_autotune(None, None, None) == -1
    assert L.irls_batch_set_tiles(None, 8, 8) == -1
    assert L.irls_batch_get_tiles(None, ctypes.byref(d), ctypes.byref(u)) == -1
    assert L.irls_batch_autotune(None, None, None) == -1
    assert L.irls_batch_dct_form(None) == -1
    assert L.irls_debug_stall_fold(None, 1) == -1
    # float16 batches are refused before any device work
    H = (ctypes.c_int * 1)(256)
    W = (ctypes.c_int * 1)(256)
    h = ctypes.c_void_p()
    o = _binding.default_opts(precision="fp16")
    assert L.irls_batch_create(1, H, W, ctypes.byref(o), ctypes.byref(h)) == -8
    # fast-transform plans of a shape or precision the form does not take are refused first too
    for (Hh, Ww, prec) in ((100, 128, "fp32"), (128, 100, "fp32"), (16384, 64, "fp32"),
                           (64, 32768, "fp32"), (3000, 2000, "fp32"), (256, 256, "bf16x3")):
        o = _binding.default_opts(precision=prec, dct_form="fft")
        assert L.irls_plan_create(Hh, Ww, ctypes.byref(o), ctypes.byref(h)) == -8, (Hh, Ww, prec)
    # and so are fast-transform batches (single-image plans only), in either precision
    for prec in ("bf16x3", "fp32"):
        o = _binding.default_opts(precision=prec, dct_form="fft")
        assert L.irls_batch_create(1, H, W, ctypes.byref(o), ctypes.byref(h)) == -8, prec


def test_header_constants_match_the_binding():
    """The IRLS_DCT_* / IRLS_PREC_* / IRLS_SYS_* / IRLS_CG_* values of include/irls.h are the
    ones the Python binding passes."""
    from paper_2401_09961_gb300 import _binding
    txt = open(HEADER).read()
    consts = {k: int(v) for k, v in re.findall(r"#define\s+(IRLS_[A-Z0-9_]+)\s+(-?\d+)", txt)}
    for name, v in _binding.DCT_FORMS.items():
        assert consts[f"IRLS_DCT_{name.upper()}"] == v
    for name, v in _binding.PRECISIONS.items():
        assert consts[f"IRLS_PREC_{name.upper()}"] == v
    assert consts["IRLS_SYS_FULL"] == _binding.SYSTEMS["full"]
    assert consts["IRLS_SYS_SCHUR"] == _binding.SYSTEMS["schur"]
    assert consts["IRLS_CG_FIXED"] == _binding.CG_SCHEDULES["fixed"]
    assert consts["IRLS_CG_PAPER"] == _binding.CG_SCHEDULES["paper"]


def test_fft_form_is_validated(L):
    """dct_form beyond IRLS_DCT_FFT is an invalid argument (no device work needed to say so)."""
    from paper_2401_09961_gb300 import _binding
    ok = _binding.default_opts(dct_form=3)
    bad = _binding.default_opts(dct_form=4)
    assert L.irls_workspace_bytes(256, 256, ctypes.byref(ok)) > 0
    assert L.irls_workspace_bytes(256, 256, ctypes.byref(bad)) == 0
