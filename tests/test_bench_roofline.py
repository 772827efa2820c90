"""The benchmark's roofline accounting on CPU: the algorithmic bytes and flops it divides
by each kernel's time are the per-launch figures of the in-vivo workload (256^2 x 128,
36 angles, 128 x 512 x 128 samples per line, harmonics 1..16 at +-4 bins), worked out
here from the shapes: the projector pair reads the volume once and the projections once
(33.5 MB + 4.7 MB), its taps are two 4-byte reads per sample (2.42 GB), the interleave
pass reads and writes the volume once, and a line-stage GEMM is 3 products of 2 M N K
flops."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

bench = pytest.importorskip("bench")

N, NZ, M, S, P, K, W = 256, 128, 36, 128, 512, 16, 9
NVOX = N * N * NZ
NPROJ = M * NZ * N
NSEG = M * NZ
NB = K * W
Q = 8
NE = (N - 1) * Q + 2 * 48 + 1  # fine cells of a line: (N - 1) Q + 2 ceil(A Q) + 1 with A = 6


def _dims(path):
    return {"N": N, "M": M, "nvox": NVOX, "nproj": NPROJ, "nfine": NSEG * NE, "nsig": NSEG * S * P,
            "ndata": NSEG * 2 * NB, "path": path}


def test_projector_pair_bytes_are_the_volume_and_projections_once():
    d = _dims("full_gemm")
    assert bench.ALGO_BYTES["project"](d) == 4 * (NVOX + NPROJ)
    assert abs(bench.ALGO_BYTES["project"](d) / 1e6 - 38.27) < 0.01  # 33.55 MB + 4.72 MB
    assert bench.ALGO_BYTES["backproject"](d) == bench.ALGO_BYTES["project"](d)
    assert bench.SMEM_BYTES["project"](d) == 2 * 4 * M * NVOX  # two taps per sample
    assert abs(bench.SMEM_BYTES["project"](d) / 1e9 - 2.416) < 0.001
    assert bench.ALGO_BYTES["transpose"](d) == 2 * 4 * NVOX  # read once, one copy written


def test_fractions_divide_the_algorithmic_figures_by_the_measured_time():
    d = _dims("full_gemm")
    hbm, smem = 6762.6, 40000.0
    prof = {"project": (0.1 * 20, 20), "gemm_fwd": (0.012 * 20, 20), "unknown": (1.0, 4), "idle": (0.0, 0)}
    out = bench.kernel_rooflines(prof, d, hbm, smem)
    assert set(out) == {"project", "gemm_fwd"}
    sec = 0.1e-3
    assert out["project"]["ms_per_launch"] == pytest.approx(0.1)
    assert out["project"]["hbm_frac"] == pytest.approx(4 * (NVOX + NPROJ) / sec / 1e9 / hbm, rel=1e-4)
    assert out["project"]["smem_frac"] == pytest.approx(8 * M * NVOX / sec / 1e9 / smem, rel=1e-4)
    flops = 3 * 2 * NSEG * (2 * NB) * N  # rows = lines, N = 2 n_b, K = detector bins
    peak, _ = bench.bf16_peak_tflops()
    assert out["gemm_fwd"]["tensor_tflops"] == pytest.approx(flops / 0.012e-3 / 1e12, rel=1e-4)
    assert out["gemm_fwd"]["tensor_frac"] == pytest.approx(flops / 0.012e-3 / 1e12 / peak, rel=1e-4)
    assert out["gemm_fwd"]["method_tensor_frac"] == pytest.approx(out["gemm_fwd"]["tensor_frac"] / 3, rel=1e-3)


def test_tf32_gemm_is_held_to_the_tf32_peak():
    d = _dims("full_gemm_tf32")
    prof = {"gemm_adj": (0.015, 1)}
    out = bench.kernel_rooflines(prof, d, 6762.6, 40000.0)
    peak, _ = bench.bf16_peak_tflops()
    assert out["gemm_adj"]["tensor_frac"] == pytest.approx(
        out["gemm_adj"]["tensor_tflops"] / (peak * 1.1 / 2.25), rel=1e-3)
