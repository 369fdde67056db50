"""Pins of the FP64 oracle of the method to facts the paper and the mathematics fix.

* Eq. 11: H accumulated row block by row block equals A^T (A Omega) = (A^T A) Omega,
  row by row, for any block size.
* Centering algebra: the shift-corrected accumulators equal those of the
  two-pass column-centred matrix, for any shift.
* Thm 1: the blocked QB of Alg. 4 gives Q^T Q = I and B = Q^T A.
* Alg. 4 = Alg. 1 (two passes) = the Gram/Cholesky reading, in exact arithmetic.
* Exactness: rank(A) = r <= l recovers sigma and V exactly; l >= n gives sigma(A).
* Brute force: the one-sided Jacobi SVD against LAPACK on tiny inputs.
* Eq. 7: the expected-error bound holds on average over seeds.
* Power scheme (P = 1): the QB of (A A^T) A, and the Sec. 4 error reduction on Type 1.
* Sec. 4.1: the Type 1 3000 x 3000 worked example (golden fixture).
* Mutations: plausible slips planted in the oracle's own source make a pin fail.
"""
import inspect
import json
import os
import textwrap

import numpy as np
import pytest

from oracle import philox
from oracle import spca as O
from paper_1704_07669_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand(m, n, seed):
    return np.random.default_rng(seed).standard_normal((m, n))


# ---------------------------------------------------------------- Eq. 11

def test_sketch_pass_closed_form_and_block_invariance():
    A = _rand(37, 23, 1)
    Om = O.omega(23, 7, seed=3)
    G, H = O.sketch_pass(O.row_blocks(A, 37), Om)
    assert np.allclose(G, A @ Om, rtol=0, atol=1e-12)
    assert np.allclose(H, (A.T @ A) @ Om, rtol=0, atol=1e-11)
    # Eq. 11 literally: sum over rows of a_i^T g_i
    Hrow = np.zeros_like(H)
    for i in range(A.shape[0]):
        Hrow += np.outer(A[i], A[i] @ Om)
    assert np.allclose(H, Hrow, rtol=0, atol=1e-11)
    for mb in (1, 5, 8, 36):
        G2, H2 = O.sketch_pass(O.row_blocks(A, mb), Om)
        assert np.allclose(G2, G, atol=1e-12) and np.allclose(H2, H, atol=1e-11)


def test_centering_correction_matches_two_pass_centering():
    A = _rand(120, 30, 2) * 0.1 + 5.0 * _rand(1, 30, 3)
    Om = O.omega(30, 8, seed=4)
    A_bar = O.center(A)
    G_bar = A_bar @ Om
    for c in (np.zeros(30), _rand(1, 30, 9)[0] * 3.0, O.first_block_shift(A[:17])):
        st = O.shifted_state(O.row_blocks(A, 17), Om, c)
        H_bar, gram_bar = O.centering_correction(st["H"], st["gram"], st["s"], st["sG"], st["m"])
        assert np.allclose(H_bar, A_bar.T @ G_bar, atol=1e-10)
        assert np.allclose(gram_bar, G_bar.T @ G_bar, atol=1e-10)
    assert np.allclose(O.column_means(A_bar), 0.0, atol=1e-13)


def test_block_fed_pass_matches_two_pass_centering_and_the_whole_method():
    A = _rand(150, 40, 12) * 0.2 + 4.0 * _rand(1, 40, 13) + _rand(150, 5, 14) @ _rand(5, 40, 15)
    Om = O.omega(40, 9, seed=16)
    acc = O.ShiftedPass(Om)
    for a in O.row_blocks(A, 23):          # ragged tail of 12 rows
        acc.add(a)
    st = acc.state()
    assert np.array_equal(acc.c, O.first_block_shift(A[:23]))
    A_bar = O.center(A)
    G_bar = A_bar @ Om
    H_bar, gram_bar = O.centering_correction(st["H"], st["gram"], st["s"], st["sG"], st["m"])
    assert np.allclose(H_bar, A_bar.T @ G_bar, atol=1e-10)
    assert np.allclose(gram_bar, G_bar.T @ G_bar, atol=1e-10)
    assert np.allclose(st["G"] - st["sG"][None, :] / st["m"], G_bar, atol=1e-12)
    sigma, V = O.finalize_centred(st["G"], st["H"], st["s"], st["sG"], st["m"], Om, 6, b=3)
    ref = O.single_pass_pca(A, 6, 3, 16, 23, b=3)
    assert np.allclose(sigma, ref["sigma"], rtol=1e-12)
    assert np.allclose(V, ref["V"], atol=1e-10)
    # a repeated block folded in once with its multiplicity = the literal stream
    B = A[:40]
    lit = O.ShiftedPass(Om)
    for a in [B, B, B, A[40:51]]:
        lit.add(a)
    rep = O.ShiftedPass(Om)
    rep.add(B.copy(), overwrite=True, times=3)
    rep.add(A[40:51])
    s1, s2 = lit.state(), rep.state()
    assert s1["m"] == s2["m"] == 131
    for key in ("G", "H", "gram", "s", "sG"):
        assert np.allclose(s1[key], s2[key], rtol=1e-13, atol=1e-12), key


# ---------------------------------------------------------------- Thm 1, Alg. 4 = Alg. 1

@pytest.mark.parametrize("b", [1, 4, 12])
def test_thm1_q_orthonormal_and_b_equals_qt_a(b):
    A = _rand(200, 90, 5) @ np.diag(0.9 ** np.arange(90))
    Om = O.omega(90, 12, seed=6)
    G, H = O.sketch_pass(O.row_blocks(A, 33), Om)
    Q, B = O.blocked_qb(G, H, Om, b)
    assert np.abs(Q.T @ Q - np.eye(12)).max() < 1e-13
    assert np.abs(B - Q.T @ A).max() < 1e-12 * np.abs(B).max()


def test_alg4_equals_alg1_equals_gram_reading():
    w = synth.workload_small()
    A = w["A"].numpy()
    r4 = O.single_pass_pca(A, 10, 10, w["seed"], 100, finalize="blocked")
    rg = O.single_pass_pca(A, 10, 10, w["seed"], 100, finalize="gram")
    Q1, B1 = O.randqb_two_pass(O.center(A), r4["Omega"])
    _, s1, V1 = O.svd_truncate(None, B1, 10)
    V1, _ = O.sign_fix(V1)
    for s, V in ((rg["sigma"], rg["V"]), (s1, V1)):
        assert np.max(np.abs(s - r4["sigma"]) / r4["sigma"]) < 1e-12
        assert np.abs(V - r4["V"]).max() < 1e-10


# ---------------------------------------------------------------- power scheme (Sec. 3.2, Sec. 4)

def test_power_scheme_is_the_qb_of_a_at_a_times_omega():
    """P = 1: the while loop once more with Omega <- orth(H) gives the randomized QB of
    (A A^T) A (Sec. 3.2): Q = orth(A orth(A^T A Omega)), B = Q^T A, written out with
    numpy's QR and SVD."""
    A = _rand(300, 200, 21) @ np.diag(0.97 ** np.arange(200))
    k, p = 8, 4
    r = O.single_pass_pca(A, k, p, 22, 37, b=4, power=1)
    A_bar = O.center(A)
    Om = O.omega(200, k + p, 22)
    Om2, _ = np.linalg.qr(A_bar.T @ (A_bar @ Om))
    Q, _ = np.linalg.qr(A_bar @ Om2)
    _, s, Vt = np.linalg.svd(Q.T @ A_bar, full_matrices=False)
    V, _ = O.sign_fix(Vt[:k].T)
    assert np.max(np.abs(r["sigma"] - s[:k]) / s[:k]) < 1e-11
    assert np.abs(r["V"] - V).max() < 1e-9


def test_two_power_passes_are_the_qb_of_a_at_a_squared_times_omega():
    """P = 2: Omega <- orth(H) twice gives Q = orth((A A^T)^2 A Omega) (Sec. 3.2)."""
    A = _rand(250, 160, 23) @ np.diag(0.96 ** np.arange(160))
    k, p = 6, 4
    r = O.single_pass_pca(A, k, p, 24, 41, b=5, power=2, center_columns=False)
    Om = O.omega(160, k + p, 24)
    Y = A @ Om
    for _ in range(2):
        W, _ = np.linalg.qr(A.T @ Y)
        Y = A @ W
    Q, _ = np.linalg.qr(Y)
    _, s, Vt = np.linalg.svd(Q.T @ A, full_matrices=False)
    V, _ = O.sign_fix(Vt[:k].T)
    assert np.max(np.abs(r["sigma"] - s[:k]) / s[:k]) < 1e-11
    assert np.abs(r["V"] - V).max() < 1e-9


def test_power_scheme_shrinks_the_sigma_error_on_a_slow_decay():
    """Sec. 4: one more pass 'dramatically reduces max_err' for the Type 1 spectrum."""
    m, n, k = 1500, 1000, 16
    sig = synth.spectrum("type1", n)
    A = (synth.haar(m, n, 5).numpy() * sig) @ synth.haar(n, n, 6).numpy().T
    e0 = np.max(np.abs(O.single_pass_pca(A, k, 4, 7, 100, center_columns=False)["sigma"] - sig[:k]))
    e1 = np.max(np.abs(O.single_pass_pca(A, k, 4, 7, 100, center_columns=False, power=1)["sigma"] - sig[:k]))
    assert e1 <= e0 / 100 and e1 <= 1e-6, (e0, e1)


# ---------------------------------------------------------------- exactness

@pytest.mark.parametrize("finalize", ["blocked", "gram"])
def test_exact_rank_recovered_exactly(finalize):
    # rank(A) = l: range(A Omega) = range(A), so Q Q^T A = A and the sigma are exact
    # (Thm 1 needs full column rank of every Y_i, hence r = l for the blocked route).
    A, U, sig, V = synth.exact_rank(150, 80, 12, seed=7)
    r = O.single_pass_pca(A, 8, 4, 11, 25, center_columns=False, b=4, finalize=finalize)
    assert np.max(np.abs(r["sigma"] - sig[:8]) / sig[:8]) < 1e-12
    assert O.max_principal_sine(r["V"], V[:, :8]) < 1e-11


def test_second_pass_left_vectors_of_an_exact_rank_matrix():
    # rank(A) = r <= k: A = U_r S V_r^T exactly, so A V S^-1 with the method's V and sigma is
    # U_r up to the sign each v_i carries, and equals Alg. 4 step 18's Q U~
    A, U, sig, V = synth.exact_rank(150, 80, 6, seed=9)
    r = O.single_pass_pca(A, 8, 4, 14, 25, center_columns=False, finalize="gram", keep_U=True)
    U2 = O.left_vectors_second_pass(A, r["V"], r["sigma"], center_columns=False)
    signs = np.sign(np.sum(r["V"][:, :6] * V, axis=0))
    assert np.max(np.abs(U2[:, :6] - U * signs[None, :])) < 1e-10
    assert np.all(U2[:, 6:] == 0.0)          # sigma_7.. = 0: no direction
    assert np.max(np.abs(U2[:, :6] - r["U"][:, :6])) < 1e-10
    # with centering the column means come off first: a rank-r matrix plus 1 mu^T
    mu = np.linspace(-1.0, 2.0, 80)
    rc = O.single_pass_pca(A + mu[None, :], 8, 4, 14, 25, center_columns=True, finalize="gram")
    U3 = O.left_vectors_second_pass(A + mu[None, :], rc["V"], rc["sigma"])
    Ub = O.center(A) @ rc["V"][:, :5] / rc["sigma"][None, :5]
    assert np.max(np.abs(U3[:, :5] - Ub)) < 1e-12
    assert np.max(np.abs(U3[:, :5].T @ U3[:, :5] - np.eye(5))) < 1e-9


def test_rank_below_l_uses_eigen_route_and_pads_zero_sigma():
    A, U, sig, V = synth.exact_rank(150, 80, 5, seed=8)
    Om = O.omega(80, 12, seed=12)
    G, H = O.sketch_pass([A], Om)
    res = O.gram_qb(G.T @ G, H)
    assert res["route"] == "eigen" and res["rank"] == 5
    r = O.single_pass_pca(A, 8, 4, 12, 30, center_columns=False, finalize="gram")
    assert np.max(np.abs(r["sigma"][:5] - sig) / sig) < 1e-10
    assert np.all(r["sigma"][5:] == 0.0)
    assert O.max_principal_sine(r["V"][:, :5], V) < 1e-10


def test_l_at_least_n_gives_the_exact_singular_values():
    A = _rand(60, 20, 9)
    r = O.single_pass_pca(A, 15, 5, 13, 7, center_columns=False, b=5)
    s = np.linalg.svd(A, compute_uv=False)
    assert np.max(np.abs(r["sigma"] - s[:15]) / s[:15]) < 1e-12


# ---------------------------------------------------------------- brute force

@pytest.mark.parametrize("shape", [(12, 7), (7, 12), (9, 9)])
def test_jacobi_svd_matches_lapack(shape):
    A = _rand(*shape, 10)
    U, s, V = O.jacobi_svd(A)
    assert np.allclose(s, np.linalg.svd(A, compute_uv=False), rtol=1e-13, atol=1e-14)
    assert np.allclose((U * s) @ V.T, A, atol=1e-13)
    assert np.allclose(V.T @ V, np.eye(V.shape[1]), atol=1e-13)


def test_alg4_matches_jacobi_svd_on_tiny_exact_rank_input():
    A, _, _, _ = synth.exact_rank(60, 40, 10, seed=14, sigma_kind="type2")
    r = O.single_pass_pca(A, 6, 4, 15, 9, center_columns=False, b=5)
    U, s, V = O.jacobi_svd(A)
    assert np.max(np.abs(r["sigma"] - s[:6]) / s[:6]) < 1e-11
    Vj, _ = O.sign_fix(V[:, :6])
    assert np.abs(r["V"] - Vj).max() < 1e-9


# ---------------------------------------------------------------- Eq. 7

def test_expected_error_bound_eq7():
    m, n, k, s_over = 400, 300, 10, 5
    sig = synth.spectrum("type2", n)
    U = synth.haar(m, n, 21).numpy()
    V = synth.haar(n, n, 22).numpy()
    A = (U * sig) @ V.T
    errs = []
    for seed in range(20):
        Om = O.omega(n, k + s_over, seed=100 + seed)
        G, H = O.sketch_pass(O.row_blocks(A, 64), Om)
        Q, B = O.blocked_qb(G, H, Om, 5)
        errs.append(np.linalg.norm(A - Q @ B))
    bound = np.sqrt(1.0 + k / (s_over - 1.0)) * np.sqrt(np.sum(sig[k:] ** 2))
    assert np.mean(errs) <= bound
    # and no better than optimal: ||A - QB|| >= (sum_{j>l} sigma_j^2)^1/2
    assert min(errs) >= np.sqrt(np.sum(sig[k + s_over:] ** 2)) * (1 - 1e-12)


# ---------------------------------------------------------------- Sec. 4.1 worked example

def test_section41_type1_accuracy_matches_printed_orders():
    gold = json.load(open(os.path.join(GOLDEN, "sec41_type1_accuracy.json")))
    n = 3000
    sig = synth.spectrum("type1", n)
    U = synth.haar(n, n, 101).numpy()
    V = synth.haar(n, n, 102).numpy()
    A = (U * sig) @ V.T
    k, l, b = gold["k"], gold["l"], gold["b"]
    r = O.single_pass_pca(A, k, l - k, 1, l, center_columns=False, b=b)
    err = np.abs(r["sigma"] - sig[:k]).max()
    # same order as the printed 1.3e-4 (depends on the draw), far below Alg. 2's 1.2e-2
    assert gold["alg4_max_abs_sigma_error"] / 4 < err < gold["alg4_max_abs_sigma_error"] * 4
    assert err < gold["alg2_max_abs_sigma_error"] / 20
    Vt, _ = O.sign_fix(V[:, :10])
    assert np.abs(r["V"][:, 0] - Vt[:, 0]).max() <= gold["v1_linf_difference"]
    corr = [abs(np.corrcoef(r["V"][:, i], V[:, i])[0, 1]) for i in range(10)]
    assert min(corr) >= gold["worst_pc_correlation_first10"]
    assert int(np.argmin(corr)) + 1 == gold["worst_pc_index_first10"]


# ---------------------------------------------------------------- planted mistakes

def _mutant(func, old, new):
    """Recompile ``func`` from its own source with one textual change."""
    src = textwrap.dedent(inspect.getsource(func))
    assert src.count(old) == 1, (func.__name__, old)
    ns = dict(func.__globals__)
    exec(compile(src.replace(old, new), f"<mutant {func.__name__}>", "exec"), ns)
    return ns[func.__name__]


def _alg4_vs_alg1_gap(blocked):
    A = O.center(synth.workload_small()["A"].numpy()[:600, :300])
    Om = O.omega(300, 20, seed=3)
    G, H = O.sketch_pass(O.row_blocks(A, 64), Om)
    Q, B = blocked(G, H, Om, 10)
    s = np.linalg.svd(B, compute_uv=False)
    _, B1 = O.randqb_two_pass(A, Om)
    s1 = np.linalg.svd(B1, compute_uv=False)
    return max(np.max(np.abs(s - s1) / s1), np.abs(B - Q.T @ A).max() / np.abs(B).max())


BLOCKED_MUTATIONS = [
    ("- (Om_i.T @ B.T) @ B", ""),                       # dropped term of step 15
    ("Y_i = G[:, cols] - Q", "Y_i = G[:, cols] + Q"),    # wrong sign in step 11
    ("H[:, cols].T", "H[:, cols][::-1].T"),             # wrong index of H block
    ("Y_i = G[:, cols]", "Y_i = G[::-1, cols]"),         # wrong rows of the G block
]


def test_unmutated_blocked_qb_passes_the_pin():
    assert _alg4_vs_alg1_gap(O.blocked_qb) < 1e-12


def _orthonormality_loss_fast_decay(blocked):
    # Type 5 spectrum, l = 80: later blocks of G are tiny, so without the
    # re-orthogonalisation of Eq. 8 the columns of Q lose orthogonality.
    n = 600
    sig = synth.spectrum("type5", n)
    A = (synth.haar(800, n, 1).numpy() * sig) @ synth.haar(n, n, 2).numpy().T
    Om = O.omega(n, 80, seed=3)
    G, H = O.sketch_pass(O.row_blocks(A, 100), Om)
    Q, _ = blocked(G, H, Om, 10)
    return np.abs(Q.T @ Q - np.eye(80)).max()


def test_reorthogonalisation_keeps_q_orthonormal_on_fast_decay():
    assert _orthonormality_loss_fast_decay(O.blocked_qb) < 1e-13


def test_planted_dropped_reorthogonalisation_is_caught():
    bad = _mutant(O.blocked_qb, "Q_i, Rt_i = qr(Q_i - Q @ (Q.T @ Q_i))",
                  "Rt_i = np.eye(Q_i.shape[1])")
    assert _orthonormality_loss_fast_decay(bad) > 1e-3


@pytest.mark.parametrize("old,new", BLOCKED_MUTATIONS)
def test_planted_mistake_in_blocked_qb_is_caught(old, new):
    assert _alg4_vs_alg1_gap(_mutant(O.blocked_qb, old, new)) > 1e-6


def test_planted_sign_error_in_centering_correction_is_caught():
    bad = _mutant(O.centering_correction, "H_hat - np.outer", "H_hat + np.outer")
    A = _rand(50, 10, 2) + 3.0
    Om = O.omega(10, 4, seed=4)
    A_bar = O.center(A)
    st = O.shifted_state([A], Om, np.zeros(10))
    H_bar, _ = bad(st["H"], st["gram"], st["s"], st["sG"], st["m"])
    assert not np.allclose(H_bar, A_bar.T @ (A_bar @ Om), atol=1e-6)


def test_planted_mistakes_in_omega_generator_are_caught(monkeypatch):
    z_ok = O.omega(20000, 8, seed=1).ravel()
    assert abs(z_ok.var() - 1.0) < 0.05
    bad_bm = _mutant(philox.box_muller, "-2.0 * np.log(u0)", "-np.log(u0)")
    monkeypatch.setattr(philox, "box_muller", bad_bm)
    z_bad = philox.omega(20000, 8, seed=1).ravel()
    assert abs(z_bad.var() - 1.0) > 0.2
    monkeypatch.undo()
    # a Philox key schedule without the Weyl increment no longer matches itself
    w_ok = philox.omega_words(4, 4, seed=5)
    monkeypatch.setattr(philox, "PHILOX_W0", np.uint64(0))
    assert not np.array_equal(philox.omega_words(4, 4, seed=5), w_ok)
