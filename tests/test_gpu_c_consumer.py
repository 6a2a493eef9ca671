"""GPU: a plain C program (tests/abi_c_consumer.c) uses the gather through the C ABI alone, with
CUDA runtime allocations and no Python or PyTorch in the loop."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_c_program_uses_the_abi(tmp_path):
    import paper_2301_11376_gb300 as ssilvb
    lib = ssilvb.build()
    nvcc = shutil.which("nvcc")
    assert nvcc, "nvcc is needed to build the C consumer"
    cuda = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    exe = tmp_path / "abi_c_consumer"
    libdir = os.path.dirname(lib)
    subprocess.run(["gcc", "-std=c11", "-O1", os.path.join(HERE, "abi_c_consumer.c"), "-I", ssilvb.INCLUDE,
                    "-I", os.path.join(cuda, "include"), "-L", libdir, "-lssilvb", "-L", os.path.join(cuda, "lib64"),
                    "-lcudart", f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{os.path.join(cuda, 'lib64')}", "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "OK"
