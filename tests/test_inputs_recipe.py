"""The seeded input generators (``synth.py``) follow the recipe the tests and the benchmark
state: the spectra of Sec. 4.1 and of the workloads, exact low-rank factors, the noise level
read as a spectral norm (a per-entry std of level * sigma_1 / (sqrt(m) + sqrt(n))), column
means, reproducibility from the seed, and the storage forms (BF16 rounding, FP8 E4M3 with a
per-block scale max|a| / 448). CPU only, small sizes.
"""
import math

import numpy as np
import pytest
import torch

from paper_1704_07669_gb300 import synth


def test_spectra_of_section_4_1_and_of_the_workloads():
    i = np.arange(1, 101, dtype=np.float64)
    t1 = synth.spectrum("type1", 100)
    assert t1[0] == 1.0 and t1[19] == pytest.approx(1e-4, rel=1e-14)          # 10^-4 at i = 20
    assert t1[9] == pytest.approx(10.0 ** (-4.0 * 9 / 19), rel=1e-14)
    assert t1[20] == pytest.approx(1e-4, rel=1e-14)                            # 1e-4 / 1^0.1 at i = 21
    assert t1[99] == pytest.approx(1e-4 / 80.0 ** 0.1, rel=1e-14)
    assert np.allclose(synth.spectrum("type2", 100), i ** -2.0, rtol=1e-15)
    assert np.allclose(synth.spectrum("type3", 100), i ** -3.0, rtol=1e-15)
    assert np.allclose(synth.spectrum("type4", 100), np.exp(-i / 7.0), rtol=1e-15)
    assert synth.spectrum("type5", 100)[49] == pytest.approx(1e-5, rel=1e-14)   # 10^(-50/10)
    assert synth.spectrum("dec20", 200)[199] == pytest.approx(1e-10, rel=1e-14)
    assert synth.spectrum("pow1.5", 1000)[999] == pytest.approx(1000.0 ** -1.5, rel=1e-14)
    assert np.all(np.diff(synth.spectrum("type1", 100)) <= 0)


def test_low_rank_part_has_the_prescribed_singular_values_and_orthonormal_factors():
    sig = synth.spectrum("type4", 20)
    A = synth.low_rank_plus_noise(300, 200, sig, seed=5).numpy()
    s = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(s[:20], sig, rtol=1e-12, atol=1e-14)
    assert np.all(s[20:] < 1e-13)
    A2, U, sig2, V = synth.exact_rank(150, 90, 12, seed=3)
    assert np.allclose(U.T @ U, np.eye(12), atol=1e-13) and np.allclose(V.T @ V, np.eye(12), atol=1e-13)
    assert np.allclose(A2, (U * sig2) @ V.T, atol=1e-14)
    assert np.allclose(sig2, 1.0 / np.arange(1, 13))


def test_noise_level_reads_as_a_spectral_norm():
    m, n = 2000, 1000
    std = synth.noise_std_for(1e-3, 2.0, m, n)
    assert std == pytest.approx(2e-3 / (math.sqrt(m) + math.sqrt(n)))
    A = synth.low_rank_plus_noise(m, n, np.zeros(1), noise_std=std, seed=11).numpy()
    # the largest singular value of an m x n Gaussian matrix is std (sqrt(m) + sqrt(n)) to
    # within a few percent at this size (Marchenko-Pastur edge, Tracy-Widom fluctuations)
    assert np.linalg.norm(A, 2) == pytest.approx(1e-3 * 2.0, rel=0.03)
    assert A.std() == pytest.approx(std, rel=0.01)


def test_column_means_and_reproducibility():
    m, n = 4000, 50
    A = synth.low_rank_plus_noise(m, n, synth.spectrum("inv", 5), noise_std=1e-3, mean_std=0.7, seed=9)
    B = synth.low_rank_plus_noise(m, n, synth.spectrum("inv", 5), noise_std=1e-3, mean_std=0.7, seed=9)
    C = synth.low_rank_plus_noise(m, n, synth.spectrum("inv", 5), noise_std=1e-3, mean_std=0.7, seed=10)
    assert torch.equal(A, B) and not torch.equal(A, C)
    mu = A.numpy().mean(axis=0)
    # the low-rank part has columns of norm <= sigma_1 = 1: its column mean is at most 1/sqrt(m)
    assert 0.3 < mu.std() < 1.2
    assert np.abs(mu - A[:1000].numpy().mean(axis=0)).max() < 0.05
    # the factors and the means come from the seed in FP64 whatever the output type (the noise
    # is drawn in the working type, so only the noise-free part is compared)
    D64 = synth.low_rank_plus_noise(m, n, synth.spectrum("inv", 5), mean_std=0.7, seed=9)
    D32 = synth.low_rank_plus_noise(m, n, synth.spectrum("inv", 5), mean_std=0.7, seed=9, dtype=torch.float32)
    assert D32.dtype == torch.float32 and np.abs(D32.double().numpy() - D64.numpy()).max() < 1e-6


def test_storage_forms():
    g = torch.Generator().manual_seed(4)
    a = torch.randn(64, 96, generator=g) * 3.0
    b, s = synth.store_rows(a, "bf16")
    assert s is None and b.dtype == torch.bfloat16
    assert torch.equal(b, a.to(torch.bfloat16))
    f8, s8 = synth.store_rows(a, "f8e4m3")
    assert f8.dtype == torch.float8_e4m3fn
    assert s8 == pytest.approx(float(a.abs().max()) / 448.0, rel=1e-7)
    dec = f8.float() * s8
    assert float(f8.float().abs().max()) <= 448.0
    # E4M3 keeps 3 fraction bits: relative rounding error <= 2^-4 for normal values
    big = a.abs() > 2.0 ** -6 * s8
    assert float(((dec - a).abs()[big] / a.abs()[big]).max()) <= 2.0 ** -4 + 1e-7
    same, none = synth.store_rows(a, "f32")
    assert same is a and none is None
