"""Host AddressSanitizer / UndefinedBehaviorSanitizer runs: the CPU oracle
and the input generators (tests/sanitize_driver.c: every oracle routine on
generated and hand-made graphs, the CSR check on malformed ones), and the
paper's OpenMP form gc_host_color (tests/host_sanitize_driver.cpp)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_and_generators_under_asan_ubsan(tmp_path):
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no gcc")
    exe = str(tmp_path / "sanitize_driver")
    cmd = [cc, "-std=gnu11", "-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=all", "-I", os.path.join(ROOT, "oracle"),
           os.path.join(ROOT, "tests", "sanitize_driver.c"),
           os.path.join(ROOT, "paper_1505_04086_gb300", "inputs", "gen.c"), "-lm", "-lpthread", "-o", exe]
    build = subprocess.run(cmd, capture_output=True, text=True)
    if build.returncode != 0:
        probe = subprocess.run([cc, "-x", "c", "-", "-fsanitize=address,undefined", "-o", str(tmp_path / "probe")],
                               input="int main(void) { return 0; }\n", capture_output=True, text=True)
        if probe.returncode != 0:
            pytest.skip("sanitizer runtime not available")
    assert build.returncode == 0, build.stderr[-2000:]
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    run = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=600)
    assert run.returncode == 0, run.stderr[-4000:]
    assert "all expectations met" in run.stderr


def test_host_openmp_form_under_asan_ubsan(tmp_path):
    cxx, cc = shutil.which("g++"), shutil.which("gcc")
    if cxx is None or cc is None:
        pytest.skip("no host compiler")
    exe = str(tmp_path / "host_sanitize_driver")
    san = ["-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined", "-fno-sanitize-recover=all"]
    gen_o = str(tmp_path / "gen.o")
    b1 = subprocess.run([cc, "-std=gnu11", *san, "-c", os.path.join(ROOT, "paper_1505_04086_gb300", "inputs", "gen.c"),
                         "-o", gen_o], capture_output=True, text=True)
    assert b1.returncode == 0, b1.stderr[-2000:]
    b2 = subprocess.run([cxx, "-std=c++17", *san, "-fopenmp", "-I", os.path.join(ROOT, "include"),
                         os.path.join(ROOT, "tests", "host_sanitize_driver.cpp"),
                         os.path.join(ROOT, "paper_1505_04086_gb300", "csrc", "gc_host.cpp"), gen_o,
                         "-lm", "-lpthread", "-o", exe], capture_output=True, text=True)
    if b2.returncode != 0:
        probe = subprocess.run([cxx, "-x", "c++", "-", *san, "-fopenmp", "-o", str(tmp_path / "probe")],
                               input="int main() { return 0; }\n", capture_output=True, text=True)
        if probe.returncode != 0:
            pytest.skip("sanitizer or OpenMP runtime not available")
    assert b2.returncode == 0, b2.stderr[-2000:]
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    run = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=600)
    assert run.returncode == 0, run.stderr[-4000:]
    assert "all expectations met" in run.stderr
