"""GPU parity of the tensor-core (tcgen05) forms of the pass with the FP64 oracle.

Two operand formats: BF16, and FP16 on rows and G scaled by one power of two. The
oracle runs the method in FP64 on the same stored rows with Omega defined as its
value in the operand format (the tensor-core forms round Omega once, by
definition). The remaining differences are the rounding of the shifted rows and of
G to the operand format, and FP32 accumulation. Gate (the stated target of the
tensor-core forms): FP16 holds every singular value within 1e-3 relative; BF16,
whose 8-bit significand costs about 8x more, holds the values above sigma_1 / 10
within 1e-3 relative and every value within 1e-3 sigma_1 (assert_sigma).
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
TC_MATHS = ["bf16", "fp16"]
OMEGA_FORM = {"bf16": "bf16", "fp16": "f16"}
ROUND_OP = {"bf16": O.round_bf16, "fp16": O.round_f16}


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


def oracle_tc(A, k, p, seed, block_rows, center=True, math="bf16"):
    fin = "blocked" if (k + p) % 10 == 0 else "gram"
    return O.single_pass_pca(A.double().numpy(), k, p, seed, block_rows, center_columns=center, finalize=fin,
                             omega_form=OMEGA_FORM[math])


def sigma_rel(res, ref):
    return np.abs(res["sigma"] - ref["sigma"]) / ref["sigma"]


def assert_sigma(sigma, ref_sigma, math):
    """FP16: every value within TOL_SIGMA_TC relative. BF16: a perturbation of the
    operands of relative size u = 2^-9 moves each singular value by about u times
    the largest one, so BF16 is held to TOL_SIGMA_TC relative on the values above
    sigma_1 / 10 and to TOL_SIGMA_TC * sigma_1 absolute on the rest."""
    rel = np.abs(sigma - ref_sigma) / ref_sigma
    if math == "fp16":
        assert rel.max() <= TOL_SIGMA_TC, rel
    else:
        lead = ref_sigma >= 0.1 * ref_sigma[0]
        assert rel[lead].max() <= TOL_SIGMA_TC, rel
        assert (np.abs(sigma - ref_sigma) / ref_sigma[0]).max() <= TOL_SIGMA_TC, rel
    return rel


@pytest.mark.parametrize("math", TC_MATHS)
def test_tc_small_workload_sigma_and_directions(math):
    w = synth.workload_small()
    A = w["A"].to(torch.float32)
    k, p, seed = w["k"], w["p"], w["seed"]
    res = run_tc(A, k, p, seed, w["block_rows"], want_G=True, math=math)
    ref = oracle_tc(A, k, p, seed, w["block_rows"], math=math)
    assert_sigma(res["sigma"], ref["sigma"], math)
    assert O.max_principal_sine(res["V"][:, :5], ref["V"][:, :5]) <= 3e-2
    # G rows: the FP32 sketch of the shifted rows rounded to the operand format
    # (a power-of-two scale does not change a rounding in the normal range)
    A64 = A.double().numpy()
    c = res["state"]["shift"].astype(np.float64)
    Om = O.omega(A64.shape[1], k + p, seed, OMEGA_FORM[math])
    G_ref = ROUND_OP[math](A64 - c[None, :]) @ Om
    assert O.rel_fro(res["G"], G_ref) <= (5e-3 if math == "bf16" else 1e-3)


@pytest.mark.parametrize("math", TC_MATHS)
def test_tc_agrees_with_fp32_path(math):
    w = synth.workload_small()
    A = w["A"].to(torch.float32)
    tc = run_tc(A, 10, 10, 5, 500, math=math)
    f32 = run_tc(A, 10, 10, 5, 500, math="fp32")
    assert_sigma(tc["sigma"], f32["sigma"], math)


TC_SHAPES = [
    # (m, n, k, p, update_rows, note)
    (1000, 1001, 10, 6, 1000, "n not a multiple of 8, ragged last tile"),
    (777, 640, 50, 13, 300, "l = 63 (L = 64), updates not multiples of 128 rows"),
    (300, 129, 4, 4, 300, "l = 8 (L = 16), n just over one 128-feature tile"),
    (5000, 6000, 40, 10, 4096, "cluster of 16, w = 384"),
]


@pytest.mark.parametrize("math", TC_MATHS)
@pytest.mark.parametrize("m,n,k,p,rows,note", TC_SHAPES, ids=[s[-1] for s in TC_SHAPES])
def test_tc_shapes(m, n, k, p, rows, note, math):
    A = synth.low_rank_plus_noise(m, n, synth.spectrum("type4", min(m, n, 120)), noise_std=1e-4, mean_std=0.5,
                                  seed=m + 3 * n, dtype=torch.float32)
    res = run_tc(A, k, p, 40 + m, rows, math=math)
    ref = oracle_tc(A, k, p, 40 + m, rows, math=math)
    assert_sigma(res["sigma"], ref["sigma"], math)


@pytest.mark.parametrize("math", TC_MATHS)
def test_tc_batched_updates_match_one_update(math):
    A = synth.workload_small()["A"].to(torch.float32)
    one = run_tc(A, 10, 10, 8, 2000, math=math)
    many = run_tc(A, 10, 10, 8, 64, math=math)
    assert np.max(np.abs(one["sigma"] - many["sigma"]) / one["sigma"]) <= 2e-4


@pytest.mark.parametrize("math", TC_MATHS)
def test_tc_reset_is_a_fresh_pass(math):
    A = synth.workload_small()["A"].to(DEV, torch.float32)
    with spca.Session(1000, 10, 10, 3, math=math) as s:
        s.update(30.0 * torch.randn(512, 1000, device=DEV))   # also a different FP16 operand scale
        s.reset(3)
        s.update(A)
        a = s.finalize()
    with spca.Session(1000, 10, 10, 3, math=math) as s:
        s.update(A)
        b = s.finalize()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("math", TC_MATHS)
def test_tc_repeated_sessions_at_padded_l_32(math):
    """l + 1 = 17 pads to L = 32, where H drains through staged TMA copies: the staging must stay
    inside its own buffer. Sessions created one after another (reusing freed device memory)
    and a reset session must all give the Gram matrix and sigma of the FP32 path."""
    n, k, p, seed = 300, 8, 8, 900
    A = synth.low_rank_plus_noise(2917, n, synth.spectrum("dec20", 46), noise_std=1e-4, mean_std=0.5, seed=500,
                                  device=DEV, dtype=torch.float32)
    torch.cuda.synchronize()
    cuts = [0, 587, 1223, 2037, 2585, 2917]

    def run(math_, reps=1):
        out = []
        with spca.Session(n, k, p, seed, math=math_, max_block_rows=4096) as s:
            for r in range(reps):
                if r:
                    s.reset(seed)
                for a, b in zip(cuts[:-1], cuts[1:]):
                    s.update(A[a:b])
                sigma, _ = s.finalize()
                out.append((sigma, s.state()["gram_bar"]))
        return out

    sig32, gram32 = run("fp32")[0]
    results = [run(math)[0] for _ in range(3)] + run(math, reps=3)
    sig0, gram0 = results[0]
    tol_gram = 1e-3 if math == "fp16" else 4e-3   # BF16 rounds G' to 2^-9 relative
    for sigma, gram in results:
        # the same launches on the same rows: equal up to the order of FP32 partial sums
        assert np.abs(gram - gram0).max() <= 1e-6 * np.abs(gram0).max()
        assert np.abs(sigma - sig0).max() <= 1e-6 * sig0[0]
        assert np.abs(gram - gram32).max() <= tol_gram * np.abs(gram32).max()
        assert_sigma(sigma, sig32, math)


@pytest.mark.parametrize("math", TC_MATHS)
def test_tc_left_vectors_from_kept_sketch_rows(math):
    """U of the tensor-core forms from their own G_out rows against the oracle's U (Omega in
    the operand format): the leading columns agree, with the same signs, and U^T U = I."""
    A = synth.low_rank_plus_noise(3000, 700, synth.spectrum("dec20", 80), noise_std=1e-4, mean_std=0.5, seed=31,
                                  device=DEV, dtype=torch.float32)
    torch.cuda.synchronize()
    k, p = 20, 10
    G = torch.zeros((3000, k + p), device=DEV, dtype=torch.float32)
    with spca.Session(700, k, p, 77, math=math) as s:
        for r0 in range(0, 3000, 512):
            s.update(A[r0:r0 + 512], G_out=G[r0:r0 + 512])
        sigma, V = s.finalize()
        U = s.left_vectors(G)
    ref = O.single_pass_pca(A.cpu().double().numpy(), k, p, 77, 512, finalize="blocked",
                            omega_form=OMEGA_FORM[math], keep_U=True)
    assert np.abs(U.T @ U - np.eye(k)).max() <= 1e-3
    lead = ref["sigma"] >= 0.1 * ref["sigma"][0]
    cos = np.sum(U[:, lead] * ref["U"][:, lead], axis=0)
    assert np.all(cos >= 1 - 1e-3), cos


@pytest.mark.parametrize("math", TC_MATHS)
def test_tc_checkpoint_resume(math):
    """Save after half of the blocks, resume in a new session: the result of one session
    whose pending blocks were launched at the same point (the FP16 operand scale travels
    with the checkpoint)."""
    A = synth.low_rank_plus_noise(3000, 700, synth.spectrum("dec20", 80), noise_std=1e-4, mean_std=0.5, seed=43,
                                  device=DEV, dtype=torch.float32)
    torch.cuda.synchronize()
    k, p = 20, 10
    with spca.Session(700, k, p, 79, math=math) as one:
        for r0 in range(0, 1536, 512):
            one.update(A[r0:r0 + 512])
        one.sync()
        for r0 in range(1536, 3000, 512):
            one.update(A[r0:r0 + 512])
        s_one, V_one = one.finalize()
    with spca.Session(700, k, p, 79, math=math) as a:
        for r0 in range(0, 1536, 512):
            a.update(A[r0:r0 + 512])
        ck = a.save_state()
    with spca.Session(700, k, p, 79, math=math) as b:
        b.load_state(ck)
        for r0 in range(1536, 3000, 512):
            b.update(A[r0:r0 + 512])
        s_b, V_b = b.finalize()
    assert np.allclose(s_b, s_one, rtol=1e-6, atol=0)
    assert O.max_principal_sine(V_b[:, :10], V_one[:, :10]) <= 1e-5


@pytest.mark.parametrize("math", TC_MATHS)
def test_tc_power_scheme_pass(math):
    """The power step on the tensor-core forms: Omega <- orth(H_bar) in the operand format,
    one more pass, against the oracle's twice-run while loop with Omega in that format."""
    A = synth.low_rank_plus_noise(3000, 700, synth.spectrum("inv", 300), noise_std=1e-3, mean_std=0.5, seed=41,
                                  device=DEV, dtype=torch.float32)
    torch.cuda.synchronize()
    k, p = 20, 10
    with spca.Session(700, k, p, 78, math=math) as s:
        for _ in range(2):
            for r0 in range(0, 3000, 512):
                s.update(A[r0:r0 + 512])
            if _ == 0:
                s.power_step()
        sigma, V = s.finalize()
    ref = O.single_pass_pca(A.cpu().double().numpy(), k, p, 78, 512, finalize="blocked",
                            omega_form=OMEGA_FORM[math], power=1)
    assert_sigma(sigma, ref["sigma"], math)
    lead = ref["sigma"] >= 0.1 * ref["sigma"][0]
    assert O.max_principal_sine(V[:, lead], ref["V"][:, lead]) <= 5e-2


@pytest.mark.parametrize("math", TC_MATHS)
def test_tc_rejects_shapes_it_cannot_take(math):
    # l + 1 (the column sums' column) padded to 144 > 128: beyond the tensor-core tiles
    with pytest.raises(spca.SpcaError) as ei:
        spca.Session(20000, 130, 10, 1, math=math)
    assert ei.value.status == 7
    for n, k, p in [(20000, 50, 10), (20000, 90, 10), (40000, 100, 20)]:   # the grouped kernel takes these
        with spca.Session(n, k, p, 1, math=math) as s:
            assert "kernel=grouped" in spca.spca_describe(s.handle)


@pytest.mark.parametrize("math", TC_MATHS)
def test_tc_non_finite_input_is_reported(math):
    A = torch.randn(256, 300, device=DEV)
    A[100, 7] = float("inf")
    with spca.Session(300, 8, 8, 1, math=math) as s:
        s.update(A)
        with pytest.raises(spca.SpcaError) as ei:
            s.finalize()
        assert ei.value.status == 5


def test_fp16_rows_far_above_the_first_ones_are_reported():
    """The FP16 operand scale comes from the first rows; rows whose sketch would
    overflow FP16 under it make finalize report a numeric failure instead of
    returning a wrong answer."""
    A = torch.randn(512, 300, device=DEV)
    with spca.Session(300, 8, 8, 1, math="fp16") as s:
        s.update(A[:256])
        s.update(1e4 * A[256:])
        with pytest.raises(spca.SpcaError) as ei:
            s.finalize()
        assert ei.value.status == 5


@pytest.fixture(scope="module")
def c2_oracle():
    """Oracle results on the 100000 x 10000 workload for both operand formats."""
    w = synth.workload_c2(device=DEV)
    A64 = w["A"].cpu().double().numpy()
    refs = {math: O.single_pass_pca(A64, w["k"], w["p"], w["seed"], w["block_rows"], finalize="blocked",
                                    omega_form=OMEGA_FORM[math]) for math in TC_MATHS}
    return w, refs


@pytest.mark.parametrize("math", TC_MATHS)
def test_tc_full_size_100000x10000_against_oracle(math, c2_oracle):
    w, refs = c2_oracle
    A = w["A"]
    k, p, seed, mb = w["k"], w["p"], w["seed"], w["block_rows"]
    m, n = A.shape
    with spca.Session(n, k, p, seed, math=math) as s:
        for r0 in range(0, m, mb):
            s.update(A[r0:r0 + mb])
        sigma, V = s.finalize()
    ref = refs[math]
    rel = np.abs(sigma - ref["sigma"]) / ref["sigma"]
    print(f"{math}: sigma rel max {rel.max():.3e}, leading 10 {rel[:10].max():.3e}")
    assert_sigma(sigma, ref["sigma"], math)
    assert O.max_principal_sine(V[:, :10], ref["V"][:, :10]) <= 5e-2


@pytest.mark.parametrize("math", TC_MATHS)
def test_tc_rows_no_tensor_map_describes_at_large_n(math):
    """n = 15205 (odd) is taken by the grouped kernel only, which reads rows through tensor maps:
    device rows with ld = n and host rows go through the session's staging buffers, laid out
    with a leading dimension padded to 16 bytes; the result equals the oracle's."""
    A = synth.low_rank_plus_noise(1500, 15205, synth.spectrum("type4", 80), noise_std=1e-4, mean_std=0.5,
                                  seed=77, dtype=torch.float32)
    Ad = A.to(DEV)
    ref = oracle_tc(A, 20, 10, 5, 500, math=math)
    with spca.Session(15205, 20, 10, 5, math=math) as s:
        assert "kernel=grouped" in spca.spca_describe(s.handle)
        s.update(Ad[:500])
        s.update(A[500:1000].numpy())            # host rows
        s.update(Ad[1000:])
        sigma, V = s.finalize()
    assert_sigma(sigma, ref["sigma"], math)
