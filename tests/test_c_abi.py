"""The C-ABI from C: tests/c/abi_host.c, a C99 program that includes
include/glbe.h and include/glbe2d.h and links the in-tree libglbe.so, is
compiled with gcc (as C, -Wall -Werror) and run.  It calls only host-side
entry points (defaults, validation, workspace sizing, error reporting,
NULL-context handling), so no GPU is needed."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT


def test_headers_compile_as_c_and_host_calls_work(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    from paper_0809_4730_gb300 import glbe
    lib = glbe.load()            # builds libglbe.so if it is missing or stale
    libpath = lib._name
    exe = tmp_path / "abi_host"
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c", "abi_host.c"), libpath, "-o", str(exe),
           "-Wl,-rpath," + os.path.dirname(libpath)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 failure(s)" in r.stdout
    assert "FAIL" not in r.stdout
