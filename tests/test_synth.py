"""The seeded input generators: shapes, storage forms and the recipes the GPU tests rely on
(CPU, small sizes)."""
import math

import numpy as np
import torch

from paper_1704_07669_gb300 import synth


def test_store_rows_forms():
    a = torch.randn(64, 48, generator=torch.Generator().manual_seed(3)) * 1e-5
    same, s = synth.store_rows(a, "f32")
    assert same is a and s is None
    b, s = synth.store_rows(a, "bf16")
    assert b.dtype == torch.bfloat16 and s is None
    assert torch.equal(b, a.to(torch.bfloat16))
    q, s = synth.store_rows(a, "f8e4m3")
    assert q.dtype == torch.float8_e4m3fn
    # one FP32 scale per block, max |a| / 448: the largest code is +-448 (no NaN codes)
    assert s == float(np.float32(float(a.abs().max()) / 448.0))
    codes = q.float()
    assert torch.isfinite(codes).all() and codes.abs().max() == 448.0
    # the stored values approximate the block to FP8's relative precision (3 mantissa bits)
    err = (codes.double() * s - a.double()).abs().max() / a.abs().max()
    assert err <= 2.0 ** -4


def test_workload_c3_blocks_on_a_small_grid():
    w = synth.workload_c3(m=2500, n=300, device="cpu", block_rows=1024, r=50)
    assert (w["k"], w["p"], w["block_rows"]) == (100, 20, 1024)
    blocks = list(w["blocks"]())
    assert [r0 for r0, _ in blocks] == [0, 1024, 2048]
    assert [a.shape for _, a in blocks] == [(1024, 300), (1024, 300), (452, 300)]
    A = torch.cat([a for _, a in blocks]).double()
    # sigma_i = i^-1.5 plus noise of spectral norm ~1e-3 sigma_1: the leading values follow the law
    s = torch.linalg.svdvals(A).numpy()
    law = synth.spectrum("pow1.5", 50)
    assert np.max(np.abs(s[:10] - law[:10]) / law[:10]) < 0.05
    # regenerating gives the same rows (each block has its own seed)
    again = torch.cat([a for _, a in w["blocks"]()]).double()
    assert torch.equal(A, again)


def test_noise_std_gives_the_stated_spectral_norm():
    m, n = 3000, 400
    std = synth.noise_std_for(1e-3, 2.0, m, n)
    assert math.isclose(std, 2e-3 / (math.sqrt(m) + math.sqrt(n)))
    E = torch.randn(m, n, generator=torch.Generator().manual_seed(5), dtype=torch.float64) * std
    top = float(torch.linalg.svdvals(E)[0])
    assert 0.9 * 2e-3 < top < 1.05 * 2e-3
