"""GPU checks of spca_merge with the shift rebase: the sketch is a sum over rows (Eq. 11), so
sessions that each saw a disjoint share of the rows - and each centred on the mean of its own
first rows - must merge into the session that saw all of them. The reference is the FP64
oracle on the whole matrix (Alg. 4, same Omega), and a single session over all rows."""
import numpy as np
import pytest
import torch

import paper_1704_07669_gb300 as spca
from oracle import spca as O
from paper_1704_07669_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
TOL_STATE = 1e-5
TOL_SIGMA = 1e-4
OMEGA_FORM = {"fp32": "f32", "bf16": "bf16", "fp16": "f16"}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if DEV is None:
        pytest.fail("GPU tests need CUDA")
    spca.build.build()
    spca.lib()


def shard_sessions(A, k, p, seed, cuts, block, math):
    """One session per row shard [cuts[i], cuts[i+1]), each fed in blocks of `block` rows."""
    m, n = A.shape
    out = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        s = spca.Session(n, k, p, seed, math=math)
        for r0 in range(a, b, block):
            s.update(A[r0:min(r0 + block, b)])
        out.append(s)
    return out


def oracle_centred(A64, k, p, seed, form):
    Om = O.omega(A64.shape[1], k + p, seed, form)
    Gb = O.center(A64) @ Om
    return O.center(A64).T @ Gb, Gb.T @ Gb


@pytest.mark.parametrize("cuts", [(0, 700, 1300, 2000), (0, 100, 2000), (0, 1999, 2000)],
                         ids=["three-shards", "short-first", "one-row-last"])
def test_fp32_shards_merge_to_the_whole(cuts):
    w = synth.workload_small()
    A = w["A"].to(torch.float32)
    k, p, seed = w["k"], w["p"], w["seed"]
    sess = shard_sessions(A.to(DEV), k, p, seed, list(cuts), 100, "fp32")
    try:
        for s in sess[1:]:
            spca.spca_merge(sess[0].handle, s.handle)
        st = sess[0].state()
        sigma, V = sess[0].finalize()
    finally:
        for s in sess:
            s.close()
    A64 = A.double().numpy()
    H_ref, gram_ref = oracle_centred(A64, k, p, seed, "f32")
    assert st["m"] == A.shape[0]
    assert O.rel_fro(st["H_bar"], H_ref) <= TOL_STATE
    assert O.rel_fro(st["gram_bar"], gram_ref) <= TOL_STATE
    ref = O.single_pass_pca(A64, k, p, seed, 100, finalize="blocked", omega_form="f32")
    rel = np.abs(sigma - ref["sigma"]) / ref["sigma"]
    assert rel.max() <= TOL_SIGMA, rel
    cos = np.abs(np.sum(V * ref["V"], axis=0))
    assert cos.min() >= 1 - 1e-6, cos


def test_merge_into_an_empty_session_takes_the_source_shift():
    w = synth.workload_small()
    A = w["A"].to(torch.float32).to(DEV)
    k, p, seed = w["k"], w["p"], w["seed"]
    with spca.Session(A.shape[1], k, p, seed) as empty, spca.Session(A.shape[1], k, p, seed) as full:
        full.update(A)
        spca.spca_merge(empty.handle, full.handle)
        a, b = empty.state(), full.state()
        assert a["m"] == b["m"]
        assert np.array_equal(a["shift"], b["shift"])
        assert np.array_equal(a["H_bar"], b["H_bar"]) and np.array_equal(a["gram_bar"], b["gram_bar"])


@pytest.mark.parametrize("math", ["fp16", "bf16"])
def test_tensor_core_shards_merge_to_the_whole(math):
    w = synth.workload_small()
    A = w["A"].to(torch.float32)
    k, p, seed = w["k"], w["p"], w["seed"]
    Ad = A.to(DEV)
    sess = shard_sessions(Ad, k, p, seed, [0, 900, 2000], 100, math)
    try:
        spca.spca_merge(sess[0].handle, sess[1].handle)
        sigma, _ = sess[0].finalize()
    finally:
        for s in sess:
            s.close()
    with spca.Session(A.shape[1], k, p, seed, math=math) as one:
        for r0 in range(0, A.shape[0], 100):
            one.update(Ad[r0:r0 + 100])
        sigma_one, _ = one.finalize()
    ref = O.single_pass_pca(A.double().numpy(), k, p, seed, 100, finalize="blocked", omega_form=OMEGA_FORM[math])
    for s_ in (sigma, sigma_one):
        assert (np.abs(s_ - ref["sigma"]) / ref["sigma"]).max() <= 1e-3
    assert (np.abs(sigma - sigma_one) / sigma_one).max() <= 1e-3


def test_merge_rejects_mismatched_sessions():
    with spca.Session(300, 4, 4, 1) as a, spca.Session(300, 4, 4, 2) as b, \
            spca.Session(300, 4, 4, 1, math="bf16") as c:
        for other in (b, c):
            with pytest.raises(spca.SpcaError) as ei:
                spca.spca_merge(a.handle, other.handle)
            assert ei.value.status == 1
