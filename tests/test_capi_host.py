"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/mpdata.h declares, and rejects bad arguments with
status codes before touching a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpdata.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"MPDATA_API[^;(]*?\b(mpdata_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def capi():
    from paper_1908_06094_b300 import build
    build.build()
    from paper_1908_06094_b300 import _capi
    return _capi


def test_every_declared_symbol_is_exported_and_bound(capi):
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(capi.lib, n), n
        assert n in capi.SIGNATURES, f"{n} declared but not bound in _capi"
    assert sorted(capi.SIGNATURES) == names


def test_strerror_and_version(capi):
    for code in range(0, -7, -1):
        assert capi.mpdata_strerror(code)
    assert capi.mpdata_strerror(-99) == "unknown status"
    assert capi.mpdata_version() >= 10000


@pytest.mark.parametrize("args", [
    (0, 4, 4, 2, 2, 1, 0, 0),     # nx < 1
    (4, 0, 4, 2, 2, 1, 0, 0),     # ny < 1
    (4, 4, 0, 2, 2, 1, 0, 0),     # nz < 1
    (4, 4, 4, 1, 2, 1, 0, 0),     # halo 1 with a corrective pass
    (4, 4, 4, 0, 1, 0, 0, 0),     # halo 0
    (4, 4, 4, 2, 0, 1, 0, 0),     # iord 0
    (4, 4, 4, 2, 9, 1, 0, 0),     # iord too large
    (4, 4, 4, 2, 2, 2, 0, 0),     # nonoscillatory not 0/1
    (4, 4, 4, 2, 2, 1, 7, 0),     # unknown dtype
    (4, 4, 4, 2, 2, 1, 0, 3),     # unknown vertical boundary
])
def test_init_rejects_bad_arguments(capi, args):
    out = ctypes.c_void_p(1234)
    rc = capi.lib.mpdata_init(ctypes.byref(out), *args, None)
    assert rc == capi.MPDATA_EINVAL
    assert out.value is None


def test_init_rejects_null_out_and_oversize(capi):
    assert capi.lib.mpdata_init(None, 4, 4, 4, 2, 2, 1, 0, 0, None) == capi.MPDATA_EINVAL
    out = ctypes.c_void_p()
    assert capi.lib.mpdata_init(ctypes.byref(out), 4, 4, 70000, 2, 2, 1, 0, 0,
                                None) == capi.MPDATA_ERANGE


def test_row_bound_of_the_mass_reduction(capi):
    """ny*nz one past the mass reduction's row bound is refused before any
    device call, by the context and by the allocation-free entry point (whose
    argument checks all run before it touches a device, so fake aligned
    pointers are never dereferenced)."""
    bound = 2147483647 - 16 * 1184
    ny, nz = 65534, bound // 65534 + 1          # ny * nz = bound + a few
    assert ny * nz > bound and nz <= 65535
    out = ctypes.c_void_p()
    assert capi.lib.mpdata_init(ctypes.byref(out), 1, ny, nz, 2, 2, 1, 0, 0,
                                None) == capi.MPDATA_ERANGE
    fake = 1 << 20                               # 16-byte aligned, never read
    for dt in (0, 1):
        assert capi.lib.mpdata_mass_noalloc(fake, fake, 1, ny, nz, 2, dt, fake,
                                            None) == capi.MPDATA_ERANGE


def test_later_calls_reject_bad_arguments_without_a_device(capi):
    """The pipelined host calls, the slab calls and the FP64 probe check
    their arguments before any device call."""
    L = capi.lib
    fake = 1 << 20
    assert L.mpdata_step_host_async(None, fake, fake, fake, fake, fake, fake, 1) == \
        capi.MPDATA_EINVAL
    assert L.mpdata_step_host_interior_async(None, fake, fake, fake, fake, fake, fake, 1) == \
        capi.MPDATA_EINVAL
    assert L.mpdata_host_wait(None) == capi.MPDATA_EINVAL
    assert L.mpdata_set_ij_boundary(None, capi.MPDATA_IJ_HALO) == capi.MPDATA_EINVAL
    n = ctypes.c_longlong()
    assert L.mpdata_halo_strip_elems(None, 0, ctypes.byref(n)) == capi.MPDATA_EINVAL
    assert L.mpdata_halo_pack(None, fake, 0, fake) == capi.MPDATA_EINVAL
    assert L.mpdata_halo_unpack(None, fake, 0, fake) == capi.MPDATA_EINVAL
    fl = ctypes.c_double()
    assert L.mpdata_probe_fp64_fma(None, 1, 1, None, ctypes.byref(fl)) == capi.MPDATA_EINVAL
    assert L.mpdata_probe_fp64_fma(fake, 0, 1, None, ctypes.byref(fl)) == capi.MPDATA_EINVAL
    assert L.mpdata_probe_fp64_fma(fake, 1, 1, None, None) == capi.MPDATA_EINVAL


def test_calls_reject_null_context(capi):
    L = capi.lib
    assert L.mpdata_step(None, None, None, None, None, None, 1) == capi.MPDATA_EINVAL
    assert L.mpdata_fill_halo(None, None, 0) == capi.MPDATA_EINVAL
    assert L.mpdata_mass(None, None, None, None) == capi.MPDATA_EINVAL
    assert L.mpdata_set_stream(None, None) == capi.MPDATA_EINVAL
    assert L.mpdata_set_variant(None, 0) == capi.MPDATA_EINVAL
    assert L.mpdata_profile(None, 1) == capi.MPDATA_EINVAL
    assert L.mpdata_launch_count(None) == -1
    L.mpdata_destroy(None)


def test_valid_init_without_a_device_reports_edevice(capi):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    out = ctypes.c_void_p()
    assert capi.lib.mpdata_init(ctypes.byref(out), 8, 8, 4, 2, 2, 1, 0, 0,
                                None) == capi.MPDATA_EDEVICE


def test_python_front_end_fails_loudly_without_library(tmp_path, monkeypatch):
    """No silent fallback: a missing library is an ImportError."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "capi_probe", os.path.join(ROOT, "paper_1908_06094_b300", "_capi.py"))
    mod = importlib.util.module_from_spec(spec)
    monkeypatch.setattr(os.path, "exists", lambda p: False)
    with pytest.raises(ImportError):
        spec.loader.exec_module(mod)
