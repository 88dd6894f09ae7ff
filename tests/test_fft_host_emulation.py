"""The device FFT's source run on the host (CPU only).

tests/fft_host_emu.cpp compiles csrc/fft.cuh with the host compiler and runs fft2_forward /
fft2_inverse with one std::thread per CUDA thread of the tile and a barrier for __syncthreads, for
the tile sizes and lines per thread the kernels use (fused kernels and generator: M = 8 ... 64 with
one line per thread, M = 128 with two) and two more splits. The forward transform (COL layout) is
compared with a direct 2-D DFT in double precision, the inverse with M^2 times the input: the
index arithmetic, twiddles, swaps and transposes of the kernel source, checked without a GPU.
"""
import os
import pathlib
import shutil
import subprocess

import pytest

HERE = pathlib.Path(__file__).resolve().parent
CSRC = HERE.parent / "paper_2406_06640_gb300" / "csrc"
CUDA_INC = pathlib.Path(os.environ.get("CUDA_HOME", "/usr/local/cuda")) / "include"


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    cxx = shutil.which("g++")
    if not cxx or not (CUDA_INC / "cuda_runtime.h").exists():
        pytest.skip("g++ and the CUDA headers are needed to compile the FFT source for the host")
    exe = tmp_path_factory.mktemp("fftemu") / "fft_host_emu"
    r = subprocess.run([cxx, "-std=c++20", "-O2", f"-I{CUDA_INC}", f"-I{CSRC}", str(HERE / "fft_host_emu.cpp"),
                        "-o", str(exe), "-lpthread"], stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    assert r.returncode == 0, r.stdout
    return exe


@pytest.mark.parametrize("M,V", [(8, 1), (16, 1), (32, 1), (64, 1), (64, 2), (128, 2), (128, 4)])
def test_device_fft_source_matches_a_direct_dft(emu, M, V):
    r = subprocess.run([str(emu), str(M), str(V)], stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout
    _, fwd, _, rt = r.stdout.split()
    # FP32 butterflies and twiddles: ~1e-7 relative per transform (log2(M^2) stages)
    assert float(fwd) < 5e-6 and float(rt) < 5e-6, r.stdout


@pytest.mark.parametrize("BL", [256, 512])
def test_staged_line_transform_source_matches_a_direct_dft(emu, BL):
    """line_fft of the staged passes (big_line.cuh): one BL-point line on 16 threads, frequencies by
    line_freq, and the inverse back to x = t + 16 j."""
    r = subprocess.run([str(emu), "line", str(BL)], stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout
    _, fwd, _, rt = r.stdout.split()
    assert float(fwd) < 5e-6 and float(rt) < 5e-6, r.stdout
