"""Pins of the oracle's Omega generator (Philox4x32-10 + Box-Muller) to things other than itself.

* the integer stream is compared with cuRAND's host-side Philox4_32_10 generator,
  an independent implementation of the same published function (its output
  group g comes from counter (g div 65536, 0, g mod 65536, 0) under the key
  (seed mod 2^32, seed div 2^32));
* the normals are checked against the standard normal law (moments, a
  Kolmogorov-Smirnov test, pair independence, the tail bound that the 32-bit
  uniforms imply);
* the reduced-precision roundings are checked against torch's own casts.
"""
import ctypes
import ctypes.util
import glob
import os

import numpy as np
import pytest
import scipy.stats
import torch

from oracle import philox
from oracle import spca as O


def _load_curand():
    cands = []
    for base in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if base:
            cands += sorted(glob.glob(os.path.join(base, "lib64", "libcurand.so*")))
            cands += sorted(glob.glob(os.path.join(base, "targets", "*", "lib", "libcurand.so*")))
    found = ctypes.util.find_library("curand")
    if found:
        cands.append(found)
    for c in cands:
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand_host_words(lib, seed, offset, count):
    gen = ctypes.c_void_p()
    st = lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10)
    if st != 0:
        pytest.skip(f"cuRAND host generator unavailable (status {st})")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(count, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(count)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 1, 17040769, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host_generator(seed):
    lib = _load_curand()
    if lib is None:
        pytest.skip("libcurand not found")
    groups = 1 << 18                      # ctr word 0 in [0, 4), word 2 in [0, 65536)
    got = _curand_host_words(lib, seed, 0, 4 * groups).reshape(groups, 4)
    g = np.arange(groups, dtype=np.uint64)
    k0, k1 = philox.seed_key(seed)
    ref = np.stack(philox.philox4x32_10(g // np.uint64(65536), 0, g % np.uint64(65536), 0, k0, k1), -1)
    assert np.array_equal(got, ref)


def test_philox_matches_curand_far_counters():
    lib = _load_curand()
    if lib is None:
        pytest.skip("libcurand not found")
    seed = 987654321
    start = 65536 * 123457 + 11            # counter word 0 = 123457
    got = _curand_host_words(lib, seed, 4 * start, 4 * 4096).reshape(-1, 4)
    g = np.arange(start, start + 4096, dtype=np.uint64)
    k0, k1 = philox.seed_key(seed)
    ref = np.stack(philox.philox4x32_10(g // np.uint64(65536), 0, g % np.uint64(65536), 0, k0, k1), -1)
    assert np.array_equal(got, ref)


def test_philox_avalanche_on_every_input_bit():
    # Flipping any single bit of the counter or key changes about half the output bits.
    rng = np.random.default_rng(5)
    base = rng.integers(0, 2**32, size=(6, 512), dtype=np.uint64)
    ref = np.stack(philox.philox4x32_10(base[0], base[1], base[2], base[3], 77, 99), -1)
    for word in range(6):
        for bit in (0, 13, 31):
            x = base.copy()
            x[word] ^= np.uint64(1 << bit)
            if word < 4:
                out = np.stack(philox.philox4x32_10(x[0], x[1], x[2], x[3], 77, 99), -1)
            else:
                k = [77, 99]
                k[word - 4] ^= 1 << bit
                out = np.stack(philox.philox4x32_10(base[0], base[1], base[2], base[3], k[0], k[1]), -1)
            flips = np.unpackbits((out ^ ref).view(np.uint8)).mean()
            assert 0.45 < flips < 0.55


def test_uniforms_strictly_inside_unit_interval():
    w = np.array([0, 1, 2**31, 2**32 - 1], dtype=np.uint32)
    u = philox.uniforms(w)
    assert np.all(u > 0) and np.all(u < 1)
    assert u[0] == 2.0 ** -33 and u[-1] == 1.0 - 2.0 ** -33


def test_box_muller_normal_law():
    z = O.omega(262144, 16, seed=2024).ravel()       # 4.2M draws
    N = z.size
    assert abs(z.mean()) < 5.0 / np.sqrt(N)
    assert abs(z.var() - 1.0) < 5.0 * np.sqrt(2.0 / N)
    kurt = np.mean(z ** 4) / np.mean(z ** 2) ** 2
    assert abs(kurt - 3.0) < 5.0 * np.sqrt(24.0 / N)
    assert abs(np.mean(z ** 3)) < 5.0 * np.sqrt(15.0 / N)
    assert scipy.stats.kstest(z[:1_000_000], "norm").pvalue > 1e-4
    # 32-bit uniforms bound the radius: |z| <= sqrt(-2 ln(2^-33))
    assert np.abs(z).max() <= np.sqrt(-2.0 * np.log(2.0 ** -33))


def test_box_muller_pairs_and_columns_uncorrelated():
    W = O.omega(200000, 12, seed=7)
    C = np.corrcoef(W.T)
    off = C - np.diag(np.diag(C))
    assert np.abs(off).max() < 5.0 / np.sqrt(W.shape[0])


def test_omega_does_not_depend_on_padding_or_other_seeds():
    a = O.omega(300, 13, seed=11)
    b = O.omega(300, 64, seed=11)
    assert np.array_equal(a, b[:, :13])
    c = O.omega(300, 13, seed=12)
    assert not np.allclose(a, c)
    # rows are independent of n
    d = O.omega(100, 13, seed=11)
    assert np.array_equal(a[:100], d)


def test_round_bf16_matches_torch_cast():
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(100000) * 10.0 ** rng.integers(-20, 20, 100000),
                        [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -1.0 - 2.0 ** -8, 0.0, -0.0]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(O.round_bf16(x), ref)
    assert O.round_bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0           # tie to even
    assert O.round_bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6


def test_round_f16_matches_torch_cast():
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.standard_normal(100000) * 10.0 ** rng.integers(-9, 6, 100000),
                        [1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, 65504.0, 65520.0, 2.0 ** -24, 0.0]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.float16).to(torch.float64).numpy()
    assert np.array_equal(O.round_f16(x), ref)
    assert O.round_f16(np.array([1.0 + 2.0 ** -11]))[0] == 1.0           # tie to even
    assert O.round_f16(np.array([1.0 + 3 * 2.0 ** -11]))[0] == 1.0 + 2.0 ** -9
    assert np.isinf(O.round_f16(np.array([65520.0]))[0])                 # rounds past the largest finite


def test_decode_e4m3_matches_torch_float8():
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8_e4m3fn")
    codes = np.arange(256, dtype=np.uint8)
    ref = torch.from_numpy(codes).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    got = O.decode_e4m3(codes)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan], ref[~nan])
    assert got[0x7E] == 448.0 and got[0x01] == 2.0 ** -9
