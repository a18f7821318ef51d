"""Host code under the address and undefined-behaviour sanitizers (no GPU):
the C oracle, running its pins, and libcia's host-only community detection
and graph validation, driven by tests/sanitize/detect_main.cpp."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SAN = ["-fsanitize=address,undefined", "-fno-omit-frame-pointer", "-fno-sanitize-recover=undefined", "-g", "-O1"]
ENV = {"ASAN_OPTIONS": "detect_leaks=0:halt_on_error=1", "UBSAN_OPTIONS": "halt_on_error=1:print_stacktrace=1"}


def _runtime(compiler, name):
    path = subprocess.run([compiler, "-print-file-name=" + name], capture_output=True, text=True).stdout.strip()
    return path if os.path.isabs(path) and os.path.exists(path) else None


@pytest.fixture(scope="module")
def gcc():
    cc = shutil.which("gcc")
    if not cc or not _runtime(cc, "libasan.so") or not _runtime(cc, "libubsan.so"):
        pytest.skip("gcc with the address and undefined-behaviour sanitizer runtimes is needed")
    return cc


def test_oracle_pins_under_sanitizers(gcc, tmp_path):
    lib = str(tmp_path / "libcia_oracle_san.so")
    subprocess.check_call([gcc, *SAN, "-fopenmp", "-fPIC", "-shared", "-std=c11", "-fno-fast-math", "-o", lib,
                           os.path.join(ROOT, "oracle", "cia_oracle.c"), "-lm"])
    env = dict(os.environ, **ENV, CIA_ORACLE_LIB=lib,
               LD_PRELOAD=_runtime(gcc, "libasan.so") + ":" + _runtime(gcc, "libubsan.so"))
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-q",
                        "-x", "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]


def test_community_detection_under_sanitizers(tmp_path):
    cxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if not cxx or not _runtime(cxx, "libasan.so") or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("g++ with sanitizer runtimes and the CUDA headers are needed")
    exe = str(tmp_path / "detect_san")
    csrc = os.path.join(ROOT, "paper_2203_16657_gb300", "csrc")
    subprocess.check_call([cxx, *SAN, "-fopenmp", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", csrc,
                           "-I", cuda_inc, "-o", exe, os.path.join(ROOT, "tests", "sanitize", "detect_main.cpp"),
                           os.path.join(csrc, "detect.cpp"), os.path.join(csrc, "graph.cpp")])
    r = subprocess.run([exe], env=dict(os.environ, **ENV), capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout[-3000:] + r.stderr[-3000:]
