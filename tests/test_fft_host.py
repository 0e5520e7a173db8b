"""The register line FFTs of the CUDA path (prime-factor split for coprime lengths,
Cooley-Tukey with exact quarter-turn twiddles otherwise), compiled for the host through
their __host__ paths and checked against the direct DFT in long double: every supported
line length, both directions, FP64 and FP32."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_line_ffts_match_the_direct_dft(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "fft_lines"
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-O2",
                    "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "paper_1611_06797_gb300", "csrc"), "-x", "cu",
                    os.path.join(ROOT, "tests", "native", "fft_lines.cu"), "-o", str(exe)],
                   check=True, capture_output=True, timeout=600)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout
    rows = [line.split() for line in out.strip().splitlines()]
    sizes = {int(r[0]) for r in rows}
    assert sizes == {8, 10, 12, 16, 18, 20, 24, 25, 27, 30, 32, 36, 40}
    assert len(rows) == 4 * len(sizes)
    for n, d, prec, err in rows:
        bound = 1e-15 if prec == "f64" else 5e-7
        assert float(err) < bound, (n, d, prec, err)
