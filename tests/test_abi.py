"""The C ABI library builds for sm_103a, loads, and exports every entry point that
include/emfuse.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1506_02079_gb300 import api, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "emfuse.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(emfuse_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("emfuse_smooth_z", "emfuse_screened_poisson", "emfuse_correct_stack",
                 "emfuse_backward", "emfuse_last_error"):
        assert name in syms


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    for name in declared_symbols():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(emfuse_[a-z0-9_]+)\b", out))
    assert set(declared_symbols()) <= exported
    assert set(api.EXPORTED_SYMBOLS) <= exported


def test_library_is_built_for_sm103a_only():
    """The build compiles every translation unit for sm_103a and nothing else (the device code's
    binary version is checked at run time by a GPU test)."""
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert "sm_103a" in api.emfuse_version()


def test_host_side_calls_without_gpu(libpath):
    """Calls that touch no device: defaults, version, and argument validation (which runs
    before any CUDA call and must report EINVAL, not crash)."""
    o = api.default_opts()
    assert o.tol == 1e-6 and o.nu_pre == 2 and o.nu_post == 2 and o.precision == api.PREC_MIXED
    assert "sm_103a" in api.emfuse_version()
    L = api.lib()
    assert L.emfuse_smooth_z(None, 1, None, 4, 4, 4, 4, 0, 4, 1.0, 3.0, None) == 1
    assert b"null" in L.emfuse_last_error()
    one = (ctypes.c_int64 * 1)(4)
    off = (ctypes.c_int64 * 1)(0)
    fake = ctypes.c_void_p(16)
    assert L.emfuse_screened_poisson(fake, ctypes.c_void_p(32), ctypes.c_void_p(48), 1, one, one,
                                     off, 0.0, None, None, None) == 1
    assert b"alpha" in L.emfuse_last_error()
    assert L.emfuse_correct_stack(fake, 7, 0, fake, 4, 4, 4, 1.0, 3.0, 1e-3, None, None, None) == 1
    assert L.emfuse_correct_stack(fake, 1, 0, fake, 4, 4, 4, -1.0, 3.0, 1e-3, None, None, None) == 1
    bad = api.default_opts(nu_pre=0, nu_post=0)
    assert L.emfuse_screened_poisson(fake, ctypes.c_void_p(32), ctypes.c_void_p(48), 1, one, one,
                                     off, 1e-3, ctypes.byref(bad), None, None) == 1
    # 3-D gradient-domain smoothing: aliasing, precision, alpha and size checks
    assert L.emfuse_smooth_gradient_domain(fake, 1, fake, 4, 4, 4, 1e-3, api.PREC_FP32, None) == 1
    assert b"alias" in L.emfuse_last_error()
    assert L.emfuse_smooth_gradient_domain(fake, 1, ctypes.c_void_p(32), 4, 4, 4, 1e-3, api.PREC_MIXED, None) == 1
    assert L.emfuse_smooth_gradient_domain(fake, 1, ctypes.c_void_p(32), 4, 4, 4, 0.0, api.PREC_FP32, None) == 1
    assert L.emfuse_smooth_gradient_domain(fake, 1, ctypes.c_void_p(32), 1 << 20, 1 << 20, 4, 1e-3,
                                           api.PREC_FP32, None) == 1
    assert L.emfuse_smooth_gradient_domain(fake, 3, ctypes.c_void_p(32), 4, 4, 4, 1e-3, api.PREC_FP32, None) == 1
    # 3-D gradient-domain multigrid: aliasing, dtype, alpha, size and option checks
    mg = L.emfuse_smooth_gradient_domain_mg
    assert mg(fake, 1, fake, 4, 4, 4, 1e-3, None, None, None) == 1
    assert b"alias" in L.emfuse_last_error()
    assert mg(fake, 3, ctypes.c_void_p(32), 4, 4, 4, 1e-3, None, None, None) == 1
    assert mg(fake, 1, ctypes.c_void_p(32), 4, 4, 4, -1.0, None, None, None) == 1
    assert mg(fake, 1, ctypes.c_void_p(32), 0, 4, 4, 1e-3, None, None, None) == 1
    assert mg(fake, 1, ctypes.c_void_p(32), 1 << 20, 1 << 20, 4, 1e-3, None, None, None) == 1
    assert mg(fake, 1, ctypes.c_void_p(32), 4, 4, 4, 1e-3, ctypes.byref(bad), None, None) == 1
    # the bounded-wait self-test validates its limit before any CUDA call
    assert L.emfuse_selftest_wait_timeout(0, None) == 1
    assert L.emfuse_selftest_wait_timeout((1 << 20) + 1, None) == 1
