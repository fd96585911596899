"""The C ABI from plain C: tests/c_abi_host.c includes include/dte.h under a
strict C99 compiler (-pedantic -Werror), links the built library and checks
host-side construction, commit, attributes, iov queries and error codes
against closed forms.  No GPU is needed."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIBDIR = os.path.join(ROOT, "paper_2402_12274_gb300")


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not found")
def test_c_client_of_the_abi(tmp_path):
    exe = str(tmp_path / "c_abi_host")
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_abi_host.c"), "-o", exe, "-L", LIBDIR, "-ldte", f"-Wl,-rpath,{LIBDIR}"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
