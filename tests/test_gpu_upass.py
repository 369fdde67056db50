"""U by a second pass over the rows (spca_left_vectors_pass), against the FP64 oracle.

After a finalize, U = A_bar V diag(sigma)^-1 of any rows (``left_vectors_second_pass``).
The oracle takes the library's own sigma and V, so only the second pass's arithmetic is
tested: FP32 products of (a - c) and W = V Sigma^-1, slices summed and the centring term
subtracted in FP64; held to 1e-5 relative Frobenius. Cases: the FP32 path on a
low-rank-plus-noise matrix with column means, rows passed block by block and all at once
(same result); a tensor-core session reading BF16 rows (the pass reads the same stored
values); and an exactly rank-r matrix sketched with l = r, where U has orthonormal columns and
equals the U that spca_left_vectors forms from the kept sketch rows (Alg. 4 step 18).
"""
import numpy as np
import pytest
import torch

import paper_1704_07669_gb300 as spca
from oracle import spca as O
from paper_1704_07669_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if DEV is None:
        pytest.fail("GPU tests need CUDA")
    spca.build.build()
    spca.lib()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("math,store", [("fp32", "f32"), ("fp16", "bf16")])
def test_second_pass_matches_the_oracle(math, store):
    m, n, k, p, seed, block = 7000, 3000, 20, 10, 5, 1024
    A = synth.low_rank_plus_noise(m, n, synth.spectrum("dec20", 60), noise_std=synth.noise_std_for(1e-3, 1.0, m, n),
                                  mean_std=0.7, seed=21, device=DEV, dtype=torch.float32)
    rows = A if store == "f32" else A.to(torch.bfloat16)
    with spca.Session(n, k, p, seed, math=math) as s:
        for r0 in range(0, m, block):
            s.update(rows[r0:r0 + block])
        sigma, V = s.finalize()
        parts = [s.left_vectors_pass(rows[r0:r0 + block]) for r0 in range(0, m, block)]
        U_all = s.left_vectors_pass(rows)
        s.sync()   # the results are written on the session stream: read them after it
        U_blocks = torch.cat(parts).cpu().numpy()
        U_all = U_all.cpu().numpy()
    A64 = rows.double().cpu().numpy()
    ref = O.left_vectors_second_pass(A64, V, sigma)
    e = _rel(U_all, ref)
    print(f"{math} on {store} rows: U second pass rel {e:.2e}")
    assert e <= TOL
    assert _rel(U_blocks, ref) <= TOL


def test_exact_rank_second_pass_equals_the_kept_sketch_route():
    # l = rank(A) = 8: the sketch has full column rank (with l > rank, the sketch of FP32-rounded
    # rows has directions at rounding level that the FP32 products of H cannot resolve)
    A, U, sig, Vt = synth.exact_rank(4000, 1500, 8, seed=4)
    Ad = torch.from_numpy(A).to(DEV, torch.float32)
    k, p = 6, 2
    G = torch.empty((4000, k + p), device=DEV, dtype=torch.float32)
    with spca.Session(1500, k, p, 3, center=False) as s:
        for r0 in range(0, 4000, 1000):
            s.update(Ad[r0:r0 + 1000], G_out=G[r0:r0 + 1000])
        sigma, V = s.finalize()
        U_keep = s.left_vectors(G)
        U_pass = s.left_vectors_pass(Ad)
        s.sync()
        U_pass = U_pass.cpu().numpy()
    r = 6
    assert np.max(np.abs(U_pass[:, :r].T @ U_pass[:, :r] - np.eye(r))) <= 1e-5
    assert np.max(np.abs(U_pass[:, :r] - U_keep[:, :r])) <= 1e-5
