"""BF16- and FP8-stored rows on the tensor-core pass (Alg. 4 steps 5-7 on stored values).

The grouped tensor-core kernel reads rows in their storage format: BF16, or FP8 E4M3
codes with one FP32 scale per block (a stored value is code x scale). Per operand
format (BF16, scaled FP16) and storage format:

* equivalence: a session fed the stored rows and a session fed the same values as FP32
  produce the same state. For BF16 the decoded values are exact in FP32 and every later
  step is the same, so H_bar, the Gram matrix and the column sums agree bit for bit. For
  FP8 the kernel rounds (code x scale - c) s once, while the FP32 copy rounds code x scale
  first: about one element in 2^16 then lands on the other side of an operand rounding
  boundary and moves by one operand ulp (2^-8 for BF16, 2^-11 for FP16), so the states
  agree within FP8_TOL[math] relative (Frobenius), sqrt(2^-16) times that ulp with margin;
* against the FP64 oracle on the decoded values (Omega in the operand format): the
  singular values no further from it than those of the FP32 copy (x 1.2), and within the
  tensor-core gate (assert_sigma) except for BF16 operands on FP8 data: E4M3 quantisation
  noise (about 2^-4 of each entry) raises the Frobenius norm that BF16 rounding scales
  with, and the values near sigma_1 / 10 then move by about 2e-3 relative whatever the
  storage format of the same values; the leading directions within 5e-2;
* a block whose rows are not a multiple of 16 bytes apart (BF16 with ld = n + 3) goes
  through the session's staging copy and gives the state of aligned blocks (to the order
  of FP32 additions: staged blocks launch one at a time);
* a session that mixes storage formats across updates equals one fed FP32 values (within
  the FP8 tolerance: half of its blocks are FP8).
"""
import numpy as np
import pytest
import torch

import paper_1704_07669_gb300 as spca
from oracle import spca as O
from paper_1704_07669_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
TOL_SIGMA_TC = 1e-3
OMEGA_FORM = {"bf16": "bf16", "fp16": "f16"}
M, N, K, P, SEED, ROWS = 9000, 10000, 50, 10, 23, 2048
FP8_TOL = {"bf16": 1e-4, "fp16": 1e-5}


@pytest.fixture(scope="module")
def data():
    if DEV is None:
        pytest.fail("GPU tests need CUDA")
    spca.build.build()
    spca.lib()
    A = synth.low_rank_plus_noise(M, N, synth.spectrum("dec20", 200), noise_std=synth.noise_std_for(1e-4, 1.0, M, N),
                                  mean_std=1.0, seed=SEED, device=DEV, dtype=torch.float32)
    blocks = {}
    for st in ("bf16", "f8e4m3"):
        parts = []
        for r0 in range(0, M, ROWS):
            stored, scale = synth.store_rows(A[r0:r0 + ROWS], st)
            dec = stored.float() * scale if scale is not None else stored.float()
            parts.append((stored.contiguous(), scale, dec.contiguous()))
        blocks[st] = parts
    return A, blocks


def assert_sigma(sigma, ref_sigma, math):
    rel = np.abs(sigma - ref_sigma) / ref_sigma
    if math == "fp16":
        assert rel.max() <= TOL_SIGMA_TC, rel
    else:
        lead = ref_sigma >= 0.1 * ref_sigma[0]
        assert rel[lead].max() <= TOL_SIGMA_TC, rel
        assert (np.abs(sigma - ref_sigma) / ref_sigma[0]).max() <= TOL_SIGMA_TC, rel
    return rel


def _run(math, feed):
    with spca.Session(N, K, P, SEED, math=math) as s:
        assert "kernel=grouped" in spca.spca_describe(s.handle)
        for rows, scale in feed:
            s.update(rows, block_scale=scale)
        sigma, V = s.finalize()
        st = s.state()
    return sigma, V, st


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _close(st_a, st_b, tol):
    """H_bar and the Gram matrix are shift-invariant; the column sums are of the shifted
    rows, so they are compared with the shift added back (the two sessions' shifts can
    differ in the last place when one reads FP8 codes and the other their rounded values)."""
    for key in ("H_bar", "gram_bar"):
        assert _rel(st_a[key], st_b[key]) <= tol, key
    sa = st_a["colsum"] + st_a["m"] * st_a["shift"].astype(np.float64)
    sb = st_b["colsum"] + st_b["m"] * st_b["shift"].astype(np.float64)
    assert _rel(sa, sb) <= tol, "column sums"


@pytest.mark.parametrize("store", ["bf16", "f8e4m3"])
@pytest.mark.parametrize("math", ["bf16", "fp16"])
def test_stored_rows_equal_their_fp32_values_and_the_oracle(math, store, data):
    A, blocks = data
    parts = blocks[store]
    sig_s, V_s, st_s = _run(math, [(b, sc) for b, sc, _ in parts])
    sig_f, V_f, st_f = _run(math, [(d, None) for _, _, d in parts])
    keys = ("H_bar", "gram_bar", "colsum")
    if store == "bf16":
        for key in keys:
            assert np.array_equal(st_s[key], st_f[key]), key
        assert np.array_equal(sig_s, sig_f)
    else:
        _close(st_s, st_f, FP8_TOL[math])
    # the oracle on the decoded values, Omega in the operand format
    A64 = torch.cat([d for _, _, d in parts]).cpu().double().numpy()
    ref = O.single_pass_pca(A64, K, P, SEED, ROWS, finalize="blocked", omega_form=OMEGA_FORM[math])
    rel = np.abs(sig_s - ref["sigma"]) / ref["sigma"]
    rel_f = np.abs(sig_f - ref["sigma"]) / ref["sigma"]
    sine = O.max_principal_sine(V_s[:, :10], ref["V"][:, :10])
    print(f"{math} on {store} rows: sigma rel max {rel.max():.2e} (FP32 copy {rel_f.max():.2e}), "
          f"leading 10 {rel[:10].max():.2e}, sin theta (10) {sine:.2e}")
    assert rel.max() <= 1.2 * rel_f.max() + 1e-6
    if store == "bf16" or math == "fp16":
        assert_sigma(sig_s, ref["sigma"], math)
    assert sine <= 5e-2


@pytest.mark.parametrize("math", ["bf16", "fp16"])
def test_bf16_rows_with_an_unaligned_leading_dimension_are_restaged(math, data):
    _, blocks = data
    parts = blocks["bf16"]
    wide = []
    for b, _, _ in parts:
        w = torch.zeros((b.shape[0], N + 3), device=DEV, dtype=torch.bfloat16)
        w[:, :N] = b
        wide.append(w[:, :N])   # ld = N + 3: rows 2 (N + 3) bytes apart, not a multiple of 16
    _, _, st_w = _run(math, [(v, None) for v in wide])
    _, _, st_a = _run(math, [(b, None) for b, _, _ in parts])
    # the staged blocks launch one at a time, the aligned ones in one batch: the FP32 sums of
    # H then add in another order
    _close(st_w, st_a, 1e-6)


@pytest.mark.parametrize("math", ["bf16", "fp16"])
def test_mixed_storage_formats_in_one_session(math, data):
    _, blocks = data
    feed, dec = [], []
    for i, ((b16, _, d16), (b8, s8, d8)) in enumerate(zip(blocks["bf16"], blocks["f8e4m3"])):
        if i % 2 == 0:
            feed.append((b16, None))
            dec.append((d16, None))
        else:
            feed.append((b8, s8))
            dec.append((d8, None))
    _, _, st_m = _run(math, feed)
    _, _, st_d = _run(math, dec)
    _close(st_m, st_d, FP8_TOL[math])
