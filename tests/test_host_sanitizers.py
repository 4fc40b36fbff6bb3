"""The library's host set-up code (csrc/sp_host.cpp: Green's kernels by the host FFT,
stencil tables by both routes and both stencil kinds, the nested-dissection structure,
their worker threads) built with AddressSanitizer and UndefinedBehaviorSanitizer and run
on small grids of one and two problems (tests/host/sanitize_main.cpp).  Any
out-of-bounds access, use after free or undefined operation fails the test.  CPU only;
skipped where the compiler has no sanitizer runtimes."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FLAGS = ["-O1", "-g", "-std=c++17", "-fsanitize=address,undefined",
         "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer"]


def test_host_setup_clean_under_sanitizers(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    probe = tmp_path / "probe.cpp"
    probe.write_text("int main() { return 0; }\n")
    if subprocess.run([cxx, *FLAGS, str(probe), "-o", str(tmp_path / "probe")],
                      capture_output=True).returncode != 0:
        pytest.skip("compiler has no sanitizer runtimes")
    exe = tmp_path / "sanitize_main"
    build = subprocess.run(
        [cxx, *FLAGS, "-I", os.path.join(ROOT, "paper_1409_0297_gb300", "csrc"),
         os.path.join(ROOT, "tests", "host", "sanitize_main.cpp"),
         os.path.join(ROOT, "paper_1409_0297_gb300", "csrc", "sp_host.cpp"),
         "-o", str(exe), "-lpthread"], capture_output=True, text=True, timeout=600)
    assert build.returncode == 0, build.stderr[-4000:]
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=0:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1")
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600, env=env)
    out = run.stdout + run.stderr
    assert run.returncode == 0, out[-4000:]
    assert "runtime error" not in out and "Sanitizer" not in out, out[-4000:]
    assert out.count(": ok") == 40, out[-4000:]
