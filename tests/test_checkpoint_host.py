"""The setup checkpoint's file logic (save, bit-exact restore, chunked copies,
checksum, .part handling, every refusal) without a GPU: checkpoint.cu built as
plain C++ against host stand-ins for its copies (tests/host/checkpoint_host.cpp)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")


def test_checkpoint_file_logic_on_the_host(tmp_path):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = tmp_path / "checkpoint_host"
    cmd = ["g++", "-std=c++17", "-O1", "-g", "-Wall", "-I", CUDA_INC, "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(ROOT, "paper_1601_03184_gb300", "csrc"),
           "-x", "c++", os.path.join(ROOT, "paper_1601_03184_gb300", "csrc", "checkpoint.cu"),
           "-x", "c++", os.path.join(ROOT, "tests", "host", "checkpoint_host.cpp"), "-o", str(exe)]
    # under AddressSanitizer and UBSan where the toolchain has them (memory
    # errors and leaks in the file logic fail the run), else plain
    sanitized = subprocess.call(cmd[:1] + ["-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
                                           "-fno-omit-frame-pointer"] + cmd[1:],
                                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL) == 0
    if not sanitized:
        subprocess.check_call(cmd)
    work = tmp_path / "files"
    work.mkdir()
    out = subprocess.run([str(exe), str(work)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip().endswith("ok (0 failed checks)")
