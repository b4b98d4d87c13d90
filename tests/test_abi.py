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
