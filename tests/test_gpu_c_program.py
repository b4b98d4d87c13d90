"""The C ABI used from C alone: tests/c/channel.c (a 2-D channel with a velocity inlet and a
pressure outlet, 200 steps) is compiled, linked against libsphbuf.so and run; it checks the
count invariant and that both buffers acted."""
import os
import shutil
import subprocess

import pytest

from paper_2406_16786_gb300 import _ffi

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program_steps_a_channel(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    _ffi.load()  # the library is built
    libdir = os.path.dirname(_ffi.LIB_PATH)
    exe = str(tmp_path / "channel")
    r = subprocess.run([cc, "-std=c99", "-O2", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "c", "channel.c"), "-L", libdir, "-lsphbuf",
                        "-Wl,-rpath," + libdir, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("ok"), r.stdout
