"""GPU parity of the tensor-core (BF16 tcgen05) form of the pass with the FP64 oracle.

The oracle runs the method in FP64 on the same stored rows with Omega defined as its
BF16 value (the tensor-core form rounds Omega once, by definition). The remaining
differences are the BF16 rounding of the shifted rows and of G, and FP32
accumulation. Gate (the stated target of the tensor-core form): leading singular
values within 1e-3 relative; the largest principal-angle sine of V and the G rows
are reported and bounded.
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    if DEV is None:
        pytest.fail("GPU tests need CUDA")
    spca.build.build()
    spca.lib()


def run_tc(A, k, p, seed, update_rows, *, center=True, want_G=False, math="bf16"):
    m, n = A.shape
    src = A.to(DEV, torch.float32)
    G = torch.zeros((m, k + p), device=DEV, dtype=torch.float32) if want_G else None
    with spca.Session(n, k, p, seed, math=math, center=center) as s:
        for r0 in range(0, m, update_rows):
            s.update(src[r0:r0 + update_rows], G_out=None if G is None else G[r0:r0 + update_rows])
        sigma, V = s.finalize()
        st = s.state()
    return {"sigma": sigma, "V": V, "state": st, "G": None if G is None else G.cpu().double().numpy()}


def oracle_tc(A, k, p, seed, block_rows, center=True):
    fin = "blocked" if (k + p) % 10 == 0 else "gram"
    return O.single_pass_pca(A.double().numpy(), k, p, seed, block_rows, center_columns=center, finalize=fin,
                             omega_form="bf16")


def sigma_rel(res, ref):
    return np.abs(res["sigma"] - ref["sigma"]) / ref["sigma"]


def test_tc_small_workload_sigma_and_directions():
    w = synth.workload_small()
    A = w["A"].to(torch.float32)
    k, p, seed = w["k"], w["p"], w["seed"]
    res = run_tc(A, k, p, seed, w["block_rows"], want_G=True)
    ref = oracle_tc(A, k, p, seed, w["block_rows"])
    rel = sigma_rel(res, ref)
    assert rel.max() <= TOL_SIGMA_TC, rel
    assert O.max_principal_sine(res["V"][:, :5], ref["V"][:, :5]) <= 3e-2
    # G rows: BF16 of the FP32 sketch of the BF16 shifted rows
    A64 = A.double().numpy()
    c = res["state"]["shift"].astype(np.float64)
    Om = O.omega(A64.shape[1], k + p, seed, "bf16")
    G_ref = O.round_bf16(A64 - c[None, :]) @ Om
    assert O.rel_fro(res["G"], G_ref) <= 5e-3


def test_tc_agrees_with_fp32_path():
    w = synth.workload_small()
    A = w["A"].to(torch.float32)
    tc = run_tc(A, 10, 10, 5, 500)
    f32 = run_tc(A, 10, 10, 5, 500, math="fp32")
    assert np.max(np.abs(tc["sigma"] - f32["sigma"]) / f32["sigma"]) <= TOL_SIGMA_TC


TC_SHAPES = [
    # (m, n, k, p, update_rows, note)
    (1000, 1001, 10, 6, 1000, "n not a multiple of 8, ragged last tile"),
    (777, 640, 50, 14, 300, "l = 64, updates not multiples of 128 rows"),
    (300, 129, 4, 4, 300, "l = 8 (L = 16), n just over one 128-feature tile"),
    (5000, 6000, 40, 10, 4096, "cluster of 16, w = 384"),
]


@pytest.mark.parametrize("m,n,k,p,rows,note", TC_SHAPES, ids=[s[-1] for s in TC_SHAPES])
def test_tc_shapes(m, n, k, p, rows, note):
    A = synth.low_rank_plus_noise(m, n, synth.spectrum("type4", min(m, n, 120)), noise_std=1e-4, mean_std=0.5,
                                  seed=m + 3 * n, dtype=torch.float32)
    res = run_tc(A, k, p, 40 + m, rows)
    ref = oracle_tc(A, k, p, 40 + m, rows)
    rel = sigma_rel(res, ref)
    assert rel.max() <= TOL_SIGMA_TC, rel


def test_tc_batched_updates_match_one_update():
    A = synth.workload_small()["A"].to(torch.float32)
    one = run_tc(A, 10, 10, 8, 2000)
    many = run_tc(A, 10, 10, 8, 64)
    assert np.max(np.abs(one["sigma"] - many["sigma"]) / one["sigma"]) <= 2e-4


def test_tc_reset_is_a_fresh_pass():
    A = synth.workload_small()["A"].to(DEV, torch.float32)
    with spca.Session(1000, 10, 10, 3, math="bf16") as s:
        s.update(torch.randn(512, 1000, device=DEV))
        s.reset(3)
        s.update(A)
        a = s.finalize()
    with spca.Session(1000, 10, 10, 3, math="bf16") as s:
        s.update(A)
        b = s.finalize()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_tc_rejects_shapes_it_cannot_take():
    with pytest.raises(spca.SpcaError) as ei:
        spca.Session(40000, 100, 20, 1, math="bf16")
    assert ei.value.status == 7
    with pytest.raises(spca.SpcaError) as ei:
        spca.Session(20000, 50, 10, 1, math="bf16")
    assert ei.value.status == 7


def test_tc_non_finite_input_is_reported():
    A = torch.randn(256, 300, device=DEV)
    A[100, 7] = float("inf")
    with spca.Session(300, 8, 8, 1, math="bf16") as s:
        s.update(A)
        with pytest.raises(spca.SpcaError) as ei:
            s.finalize()
        assert ei.value.status == 5


def test_tc_full_size_100000x10000_against_oracle():
    w = synth.workload_c2(device=DEV)
    A = w["A"]
    k, p, seed, mb = w["k"], w["p"], w["seed"], w["block_rows"]
    m, n = A.shape
    with spca.Session(n, k, p, seed, math="bf16") as s:
        for r0 in range(0, m, mb):
            s.update(A[r0:r0 + mb])
        sigma, V = s.finalize()
    ref = O.single_pass_pca(A.cpu().double().numpy(), k, p, seed, mb, finalize="blocked", omega_form="bf16")
    rel = np.abs(sigma - ref["sigma"]) / ref["sigma"]
    assert rel.max() <= TOL_SIGMA_TC, rel
    assert O.max_principal_sine(V[:, :10], ref["V"][:, :10]) <= 5e-2
