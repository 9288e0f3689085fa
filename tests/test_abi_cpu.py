"""CPU-side checks of the C ABI: the library loads without a GPU, exports every entry point
include/se2ot.h declares, and rejects invalid descriptors before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2402_15322_gb300 import build, se2ot

HEADER = os.path.join(build.ROOT, "include", "se2ot.h")


def declared_functions(path):
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(se2ot_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return se2ot.lib()


def test_header_declares_the_entry_points():
    names = declared_functions(HEADER)
    for want in ("se2ot_kernel_build", "se2ot_kernel_destroy", "se2ot_apply", "se2ot_apply_log",
                 "se2ot_barycenter", "se2ot_interpolate", "se2ot_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions(HEADER):
        assert hasattr(lib, name), name
    # nothing but the C ABI is visible
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", se2ot.LIB_PATH], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert exported == set(declared_functions(HEADER)), exported ^ set(declared_functions(HEADER))


def test_version_and_empty_error(lib):
    assert "sm_103a" in se2ot.se2ot_version()


@pytest.mark.parametrize("bad", [
    dict(nx=4, ny=16, ntheta=8, radius=3),      # grid smaller than the window
    dict(nx=16, ny=16, ntheta=65, radius=3),    # unsupported ntheta
    dict(nx=16, ny=16, ntheta=8, radius=-1),
    dict(nx=16, ny=16, ntheta=8, radius=3, eps=0.0),
    dict(nx=16, ny=16, ntheta=8, radius=3, w=(1.0, -3.0, 0.5)),
    dict(nx=256, ny=256, ntheta=32, radius=17),  # radius beyond the instantiated kernels
])
def test_invalid_descriptor_is_rejected_on_the_host(lib, bad):
    args = dict(w=(1.0, 3.0, 0.5), eps=1e-3)
    args.update(bad)
    desc = se2ot.make_desc(args["nx"], args["ny"], args["ntheta"], args["radius"], args["w"], args["eps"])
    h = ctypes.c_void_p()
    st = lib.se2ot_kernel_build(ctypes.byref(desc), None, ctypes.byref(h))
    assert st == se2ot.SE2OT_EINVAL
    assert h.value is None
    assert se2ot.se2ot_last_error()


def test_unknown_boundary_or_distance_is_rejected_on_the_host(lib):
    for field, value in (("boundary", 5), ("distance", 3)):
        desc = se2ot.make_desc(16, 16, 8, 3)
        setattr(desc, field, value)
        h = ctypes.c_void_p()
        assert lib.se2ot_kernel_build(ctypes.byref(desc), None, ctypes.byref(h)) == se2ot.SE2OT_EINVAL
        assert h.value is None and field in se2ot.se2ot_last_error()


def test_null_arguments_are_rejected(lib):
    assert lib.se2ot_kernel_build(None, None, None) == se2ot.SE2OT_EINVAL
    assert lib.se2ot_apply(None, None, None, 1, 0, None) == se2ot.SE2OT_EINVAL
    assert lib.se2ot_barycenter(None, 2, None, None, None, None, None, None) == se2ot.SE2OT_EINVAL
    assert lib.se2ot_w2(None, None, None, None, None, None) == se2ot.SE2OT_EINVAL
    assert lib.se2ot_project(None, None, 1, 4, 4, 4, None) == se2ot.SE2OT_EINVAL
    assert lib.se2ot_jko(None, None, 0.1, 5.0, 1, None, None, None, None) == se2ot.SE2OT_EINVAL
    assert lib.se2ot_lift_field(None, None, 4, 4, 4, None) == se2ot.SE2OT_EINVAL
    assert lib.se2ot_reconstruct_field(None, None, 4, 4, 4, None) == se2ot.SE2OT_EINVAL
    assert lib.se2ot_interpolate_signed(None, None, None, 0.5, None, None, None, None) == se2ot.SE2OT_EINVAL
    assert lib.se2ot_kernel_destroy(None) == se2ot.SE2OT_OK


def test_missing_library_fails_loudly(monkeypatch):
    """No CPU fallback: without libse2ot.so every entry point raises instead of computing."""
    monkeypatch.setattr(se2ot, "_LIB", None)
    monkeypatch.setattr(se2ot, "LIB_PATH", os.path.join(build.ROOT, "no_such_dir", "libse2ot.so"))
    with pytest.raises(ImportError):
        se2ot.lib()
    with pytest.raises(ImportError):
        se2ot.se2ot_kernel_build(se2ot.make_desc(16, 16, 4, 2, (1.0, 3.0, 0.5), 1e-2))
