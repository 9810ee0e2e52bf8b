"""The ERI device code's single-ket-component path evaluates in a relabelled
frame (the ket direction moved to axis 0, the Kronecker-delta terms of the
Obara-Saika / Head-Gordon-Pople recurrences fixed at compile time).  Built as
host C++ with g++, it must give the same integrals as the general path for
every bra class and ket component, and execute no more FP64 operations; the
saving it books in the kernel's executed-operation counter must be the one an
operation-counting build of the source finds."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CUDA_INC = "/usr/local/cuda/include"


@pytest.mark.skipif(shutil.which("g++") is None or not os.path.isfile(os.path.join(CUDA_INC, "cuda_runtime.h")),
                    reason="needs g++ and the CUDA runtime headers")
def test_relabelled_ket_path_equals_general_path(tmp_path):
    exe = str(tmp_path / "eri_relabel")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-w", "-I" + CUDA_INC, "-o", exe,
                           os.path.join(HERE, "eri_relabel_host.cpp")])
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert "worst relative difference" in r.stdout


@pytest.mark.skipif(shutil.which("g++") is None or not os.path.isfile(os.path.join(CUDA_INC, "cuda_runtime.h")),
                    reason="needs g++ and the CUDA runtime headers")
def test_relabelled_path_savings_match_the_operation_counter(tmp_path):
    # the executed-operation counter of the roofline books the same saving per
    # primitive quartet as an operation-counting build of the source finds
    exe = str(tmp_path / "eri_opcount")
    subprocess.check_call(["g++", "-O0", "-std=c++17", "-w", "-I" + CUDA_INC, "-o", exe,
                           os.path.join(HERE, "eri_opcount_host.cpp")])
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert "all savings agree" in r.stdout
