"""The C-ABI library builds, loads without a GPU, exports every symbol that
include/lens.h declares, and reports host-side faults (no GPU needed)."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lens.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lens_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2211_00354_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path_calls():
    syms = declared_symbols()
    for name in ("lens_fmm_build", "lens_deflect", "lens_deflect_grid", "lens_ipm_map",
                 "lens_deflect_adjoint", "lens_plan_destroy", "lens_last_error"):
        assert name in syms


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    from paper_2211_00354_gb300 import lens
    assert sorted(lens.EXPORTED) == declared_symbols()


def test_version_and_error_string(lib):
    lib.lens_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.lens_version()
    lib.lens_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.lens_last_error(), bytes)


# The argument checks below pass a made-up device address.  They run in a
# child process that sees no CUDA device (CUDA_VISIBLE_DEVICES=""), so even a
# check that regressed could reach no GPU: the call would fail on the missing
# device instead of launching a kernel on that address.
def run_without_device(body, **extra_env):
    code = "import ctypes, sys\nsys.path.insert(0, %r)\n" % ROOT + body
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", **extra_env)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    return out.stdout


ARGS_CHILD = r"""
from paper_2211_00354_gb300 import lens
L = lens.load()
opts = lens.lens_build_opts()
opts.p, opts.leaf_size, opts.prec = 0, 16, 1
h = ctypes.c_void_p()
fake = ctypes.c_void_p(0x1000)
st = L.lens_fmm_build(fake, fake, 10, 0.0, 0.0, ctypes.byref(opts), None, None, ctypes.byref(h))
assert st == lens.LENS_EINVAL, st
assert b"p must be" in L.lens_last_error()
opts.p, opts.leaf_size = 8, 0
assert L.lens_fmm_build(fake, fake, 10, 0.0, 0.0, ctypes.byref(opts), None, None,
                        ctypes.byref(h)) == lens.LENS_EINVAL
opts.leaf_size = 16
assert L.lens_fmm_build(fake, fake, 0, 0.0, 0.0, ctypes.byref(opts), None, None,
                        ctypes.byref(h)) == lens.LENS_EINVAL
assert L.lens_fmm_build(fake, fake, 5, float("nan"), 0.0, ctypes.byref(opts), None, None,
                        ctypes.byref(h)) == lens.LENS_EINVAL
assert L.lens_direct_deflect(fake, fake, 4, 0.0, 0.0, fake, 4, 7, fake, None, None,
                             None) == lens.LENS_EINVAL
assert L.lens_direct_deflect_noalloc(fake, fake, 262145, 0.0, 0.0, fake, 4, fake, None,
                                     None) == lens.LENS_EINVAL
assert b"262144" in L.lens_last_error()
n = ctypes.c_int64(-1)
g = lens.lens_grid(0.0, 0.0, 0.1, 10, 10)
assert L.lens_find_images(None, ctypes.byref(g), 0.0, 0.0, 4, fake, fake, ctypes.byref(n),
                          None) == lens.LENS_EINVAL
assert L.lens_find_images(fake, ctypes.byref(g), 0.0, 0.0, -1, fake, fake, ctypes.byref(n),
                          None) == lens.LENS_EINVAL
assert L.lens_find_images(fake, ctypes.byref(g), float("nan"), 0.0, 4, fake, fake,
                          ctypes.byref(n), None) == lens.LENS_EINVAL
bad = lens.lens_grid(0.0, 0.0, 0.0, 10, 10)
assert L.lens_find_images(fake, ctypes.byref(bad), 0.0, 0.0, 4, fake, fake, ctypes.byref(n),
                          None) == lens.LENS_EINVAL
assert b"h > 0" in L.lens_last_error()
assert n.value == -1  # untouched on failure
assert L.lens_source_image(fake, 4, 0.0, 0.0, 0.0, fake, None) == lens.LENS_EINVAL
assert L.lens_source_image(fake, -1, 0.0, 0.0, 0.1, fake, None) == lens.LENS_EINVAL
assert L.lens_source_image(None, 0, 0.0, 0.0, 0.1, None, None) == lens.LENS_OK  # empty
assert L.lens_potential(None, fake, 4, fake, None) == lens.LENS_EINVAL
print("ok")
"""


def test_invalid_arguments_rejected_before_any_device_work(lib):
    assert run_without_device(ARGS_CHILD).strip() == "ok"


FAULT_CHILD = r"""
from paper_2211_00354_gb300 import lens
L = lens.load()
fake = ctypes.c_void_p(0x1000)
st = L.lens_direct_deflect(fake, fake, 16, 0.0, 0.0, fake, 16, lens.FP32_BULK, fake, None, None, None)
print(st, L.lens_last_error().decode())
"""


def test_allocation_fault_injection_on_host(lib):
    out = run_without_device(FAULT_CHILD, LENS_FAULT="alloc@1")
    st, msg = out.strip().split(" ", 1)
    assert int(st) == 7 and "injected" in msg
