"""The C ABI library builds, loads and exports every entry point that include/sphbuf.h declares."""
import os
import re

import numpy as np
import pytest

from oracle import frames
from paper_2406_16786_gb300 import _ffi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "sphbuf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"\b(sphbuf_[a-z_]+)\s*\(", text))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_ffi.LIB_PATH):
        from paper_2406_16786_gb300 import build

        build.build()
    return _ffi.load()


def test_every_declared_symbol_is_exported_and_bound(lib):
    names = _declared()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert names == set(_ffi.SIGNATURES), names ^ set(_ffi.SIGNATURES)


def test_status_strings(lib):
    for s in range(8):
        assert lib.sphbuf_status_string(s)


def test_rotation_helper_matches_the_oracle_frame(lib):
    # host-only helper (no device work): Eq. (14) under the sign reading, plus a roll
    from paper_2406_16786_gb300.domain import rotation_from_normal

    rng = np.random.default_rng(12)
    for _ in range(20):
        d = rng.standard_normal(3)
        psi = rng.uniform(0, 6.3)
        R = rotation_from_normal(d, psi)
        want = frames.roll_about_x(frames.rotation_3d(d), psi)
        assert np.allclose(R, want, atol=1e-13)
    assert np.allclose(rotation_from_normal([-2.0, 0, 0]), np.diag([-1.0, -1.0, 1.0]))


def test_header_and_c_example_compile_as_c99(tmp_path):
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = os.path.join(ROOT, "tests", "c", "channel.c")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), "-c", src,
                        "-o", str(tmp_path / "channel.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """No fallback: without the built library the binding raises instead of computing."""
    monkeypatch.setattr(_ffi, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        _ffi.load(str(tmp_path / "libsphbuf.so"))


# ------------------------------------------------------------------ host-side error behaviour
_HOST_ONLY = {"sphbuf_status_string", "sphbuf_error_message", "sphbuf_create_domain", "sphbuf_rotation_from_normal",
              "sphbuf_cell_list_build", "sphbuf_cell_list_build_noalloc"}


def _zero_args(argtypes):
    import ctypes

    ints = (ctypes.c_int, ctypes.c_uint, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_longlong)
    return [0 if a in ints else 0.0 if a is ctypes.c_double else None for a in argtypes]


def test_every_handle_call_rejects_a_null_handle(lib):
    # every entry point that takes a domain or batch handle returns SPHBUF_ERR_INVALID_ARG
    # for a NULL handle (and NULL / zero for the rest), before any CUDA call: no crash, no trap
    names = sorted(set(_ffi.SIGNATURES) - _HOST_ONLY)
    assert len(names) >= 35
    for name in names:
        _, argtypes = _ffi.SIGNATURES[name]
        assert getattr(lib, name)(*_zero_args(argtypes)) == 1, name


def _desc(**kw):
    d = _ffi.DomainDesc(dim=3, dp=0.01, h_over_dp=1.3, rho0=1000.0, c0=10.0, nu=1e-3, dt=1e-4, capacity=1000)
    for x in range(3):
        d.lo[x], d.hi[x] = 0.0, 1.0
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("bad", [dict(dim=1), dict(dim=4), dict(dp=0.0), dict(dp=float("nan")),
                                 dict(h_over_dp=-1.0), dict(rho0=0.0), dict(c0=0.0), dict(dt=0.0),
                                 dict(nu=-1.0), dict(capacity=0), dict(capacity=1 << 25), "empty_box"])
def test_create_domain_validates_its_descriptor(lib, bad):
    import ctypes

    d = _desc() if bad == "empty_box" else _desc(**bad)
    if bad == "empty_box":
        d.hi[1] = d.lo[1]
    h = ctypes.c_void_p(1)
    assert lib.sphbuf_create_domain(ctypes.byref(d), None, ctypes.byref(h)) == 1
    assert h.value is None  # *out is cleared
    assert lib.sphbuf_create_domain(None, None, ctypes.byref(h)) == 1


def test_create_domain_without_a_gpu_reports_a_cuda_error(lib):
    import ctypes

    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    d = _desc()
    h = ctypes.c_void_p(1)
    assert lib.sphbuf_create_domain(ctypes.byref(d), None, ctypes.byref(h)) == 4  # SPHBUF_ERR_CUDA
    assert h.value is None


def test_host_helpers_reject_bad_input(lib):
    import ctypes

    R = (ctypes.c_double * 9)()
    for n in ((0.0, 0.0, 0.0), (float("nan"), 0.0, 0.0), (float("inf"), 1.0, 0.0)):
        assert lib.sphbuf_rotation_from_normal((ctypes.c_double * 3)(*n), 0.0, R) == 1, n
    assert lib.sphbuf_rotation_from_normal((ctypes.c_double * 3)(1.0, 0.0, 0.0), 0.0, None) == 1
    assert lib.sphbuf_cell_list_build(None, None, None, 0, 0, None, None, None) == 1
    assert lib.sphbuf_cell_list_build_noalloc(None, None, None, 0, 0, None, None, None) == 1
    names = [lib.sphbuf_status_string(s) for s in range(9)]
    assert len(set(names)) == 9 and all(names)
    assert lib.sphbuf_status_string(9) == lib.sphbuf_status_string(-1) == b"unknown status"


def test_binding_raises_instead_of_falling_back(lib):
    # without a GPU the Python binding raises the library's status; nothing runs on the CPU
    import torch

    from paper_2406_16786_gb300 import workloads as wl
    from paper_2406_16786_gb300.domain import Domain, SphbufError, rotation_from_normal

    with pytest.raises(SphbufError) as e:
        rotation_from_normal([0.0, 0.0, 0.0])
    assert e.value.status == 1
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(SphbufError) as e:
        Domain.from_case(wl.config1())
    assert e.value.status == 4 and "CUDA error" in str(e.value)
