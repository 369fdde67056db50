"""The row-sharded pass's exchange step on one GPU: ranks emulated in sequence.

Each emulated rank runs a session over its share of the rows (``shard.row_shard``) and
centres on the mean of its own first rows; the root receives the other ranks' checkpoints
in rank order and merges them through one scratch session (``shard.merge_blobs``, the
root's half of ``shard.merge_across_ranks``). The merged session must equal one session
over all rows (Eq. 11): state within 1e-5 (FP32) or 1e-4 (FP16 operands) relative, and the
singular values of both against the FP64 oracle on the whole matrix.
"""
import numpy as np
import pytest
import torch

import paper_1704_07669_gb300 as spca
from oracle import spca as O
from paper_1704_07669_gb300 import shard, synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
OMEGA_FORM = {"fp32": "f32", "fp16": "f16"}
TOL_STATE = {"fp32": 1e-5, "fp16": 1e-4}
TOL_SIGMA = {"fp32": 1e-4, "fp16": 1e-3}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if DEV is None:
        pytest.fail("GPU tests need CUDA")
    spca.build.build()
    spca.lib()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("math", ["fp32", "fp16"])
def test_shards_merged_on_the_root_equal_one_session(math, world):
    m, n, k, p, seed, block = 6000, 12000, 20, 10, 11, 512
    A = synth.low_rank_plus_noise(m, n, synth.spectrum("dec20", 80), noise_std=synth.noise_std_for(1e-4, 1.0, m, n),
                                  mean_std=0.5, seed=3, device=DEV, dtype=torch.float32)
    sessions = []
    for r in range(world):
        r0, r1 = shard.row_shard(m, world, r, block)
        s = spca.Session(n, k, p, seed, math=math)
        for b0 in range(r0, r1, block):
            s.update(A[b0:min(b0 + block, r1)])
        sessions.append(s)
    blobs = [s.save_state() for s in sessions]
    root = sessions[0]
    with shard.scratch_like(root) as scratch:
        shard.merge_blobs(root, blobs, scratch=scratch)
    sig_m, V_m = root.finalize()
    st_m = root.state()
    with spca.Session(n, k, p, seed, math=math) as one:
        for b0 in range(0, m, block):
            one.update(A[b0:b0 + block])
        sig_1, V_1 = one.finalize()
        st_1 = one.state()
    for s in sessions:
        s.close()
    assert st_m["m"] == m
    for key in ("H_bar", "gram_bar"):
        assert O.rel_fro(st_m[key], st_1[key]) <= TOL_STATE[math], key
    ref = O.single_pass_pca(A.double().cpu().numpy(), k, p, seed, block, finalize="gram",
                            omega_form=OMEGA_FORM[math])
    rel_m = np.abs(sig_m - ref["sigma"]) / ref["sigma"]
    rel_1 = np.abs(sig_1 - ref["sigma"]) / ref["sigma"]
    print(f"{math}, {world} shards: sigma rel max merged {rel_m.max():.2e}, one session {rel_1.max():.2e}")
    assert rel_m.max() <= TOL_SIGMA[math]
    assert O.max_principal_sine(V_m[:, :10], V_1[:, :10]) <= 1e-3
