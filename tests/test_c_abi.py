"""The C ABI from plain C: tests/c/abi_client.c, compiled by gcc against
include/hfav.h and linked to libhfav.so, plans a DAG of rule bodies (analysis,
footprints, schedule, emitted source, a too-small buffer, a refused body)
without a device."""
import os
import shutil
import subprocess

import pytest

from paper_1710_08774_gb300 import hfav as H

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plain_c_client(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    lib = H.load()._name
    exe = tmp_path / "abi_client"
    subprocess.check_call(["gcc", "-std=c99", "-O1", "-o", str(exe), os.path.join(ROOT, "tests", "c", "abi_client.c"),
                           "-I", os.path.join(ROOT, "include"), lib, "-Wl,-rpath," + os.path.dirname(lib)])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    assert r.stdout.startswith("ok ")
