"""Host-side checks of library code that needs no GPU (compiled as host code with nvcc): the
exact 8 -> 27 cell derivation against brute-force counting, the bit extraction of the sample
compaction against a plain bit loop, and the compacted scan's derived first-SNP genotype
(counted-genotype slots, relabelled pair tables and marginals, cell order restored) against
brute-force tables."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_derive27_matches_bruteforce(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "derive27_check"
    subprocess.check_call([nvcc, "-std=c++17", "-o", str(exe),
                           os.path.join(HERE, "host", "derive27_check.cu")])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and "derive27 ok" in out.stdout, out.stdout + out.stderr


def test_bit_compress_matches_bit_loop(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "bit_compress_check"
    subprocess.check_call([nvcc, "-std=c++17", "-o", str(exe),
                           os.path.join(HERE, "host", "bit_compress_check.cu")])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and "bit compress ok" in out.stdout, out.stdout + out.stderr


def test_derived_genotype_relabelling_matches_bruteforce(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "relabel_check"
    subprocess.check_call([nvcc, "-std=c++17", "-o", str(exe),
                           os.path.join(HERE, "host", "relabel_check.cu")])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and "relabel ok" in out.stdout, out.stdout + out.stderr
