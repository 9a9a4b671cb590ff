"""The C ABI from plain C: tests/c_abi_host.c is compiled as C99 (gcc,
-pedantic) against include/opf_admm.h, linked to libopf_admm.so and run.
It calls only host entry points (create, dims, operators, the row
reduction, error paths), so it needs no GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_dir():
    from paper_2501_08293_b300 import build
    return os.path.dirname(build.build())


def test_header_compiles_as_c99_and_cxx17():
    cc, cxx = shutil.which("gcc"), shutil.which("g++")
    if not cc or not cxx:
        pytest.skip("gcc / g++ not installed")
    hdr = os.path.join(ROOT, "include", "opf_admm.h")
    for cmd in ([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-x", "c", hdr],
                [cxx, "-std=c++17", "-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-x", "c++", hdr]):
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_host_entry_points_from_c(lib_dir, tmp_path):
    cc = shutil.which("gcc")
    if not cc:
        pytest.skip("gcc not installed")
    exe = str(tmp_path / "c_abi_host")
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_abi_host.c"), "-L", lib_dir, "-lopf_admm",
           "-Wl,-rpath," + lib_dir, "-lm", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith("c abi ok"), r.stdout + r.stderr
