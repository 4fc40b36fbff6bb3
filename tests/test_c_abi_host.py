"""The boundary as a C caller sees it: tests/host/c_abi_main.c includes include/sp.h
and include/sp_fno.h, is compiled as strict C11 (-pedantic, warnings as errors),
links libsp_gb300.so and calls the entry points that need no GPU: struct sizes
against sp_abi_size, default options, nested-dissection level sizes against their
closed forms, sp_setup's argument and resonance checks, status strings.  CPU only."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_caller(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    from paper_1409_0297_gb300 import build as bld
    if not os.path.exists(bld.LIB):
        bld.build()
    libdir = os.path.dirname(bld.LIB)
    exe = tmp_path / "c_abi_main"
    p = subprocess.run([cc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic",
                        "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "host", "c_abi_main.c"), "-o", str(exe),
                        "-L", libdir, "-lsp_gb300", f"-Wl,-rpath,{libdir}"],
                       capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-4000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "c abi ok", r.stdout + r.stderr
