"""Pins of the oracle's comparison measures: the subspace measure ``max_principal_sine``
and, at the end, the relative Frobenius error ``rel_fro``.

The sine of the largest principal angle between two k-dimensional subspaces is
fixed by construction here: with V1 = [e_1 .. e_k] and the columns of V2 equal to
cos(t_i) e_i + sin(t_i) e_{k+i}, the k planes span(e_i, e_{k+i}) are mutually
orthogonal, so the principal angles are exactly t_1 .. t_k (Bjorck and Golub,
1973: the cosines are the singular values of Q1^T Q2). An orthogonal change of
coordinates of the whole space and any invertible mixing of each basis leave the
angles unchanged. Planted mistakes (the smallest angle instead of the largest, a
Frobenius norm instead of the spectral norm, a basis not made orthonormal) fail.
"""
import inspect
import textwrap

import numpy as np
import pytest

from oracle import spca as O
from paper_1704_07669_gb300 import synth


def _pair(n, thetas, seed, rotate=True, mix=True):
    k = len(thetas)
    V1 = np.zeros((n, k))
    V2 = np.zeros((n, k))
    for i, t in enumerate(thetas):
        V1[i, i] = 1.0
        V2[i, i] = np.cos(t)
        V2[k + i, i] = np.sin(t)
    rng = np.random.default_rng(seed)
    if rotate:
        Q = synth.haar(n, n, seed).numpy()
        V1, V2 = Q @ V1, Q @ V2
    if mix:   # a non-orthogonal basis of each subspace
        V1 = V1 @ (np.eye(k) + 0.5 * rng.standard_normal((k, k)))
        V2 = V2 @ (np.eye(k) + 0.5 * rng.standard_normal((k, k)))
    return V1, V2


THETAS = np.array([1e-9, 3e-6, 1e-3, 0.2, 1.0])


def _check(f, V1, V2, thetas, atol):
    want = np.sin(np.max(thetas))
    got = f(V1, V2)
    assert abs(got - want) <= 1e-12 * want + atol, (got, want)
    return got


@pytest.mark.parametrize("which", range(len(THETAS)))
def test_axis_aligned_angles_exactly(which):
    # the largest angle is THETAS[which]; the others are smaller
    th = np.minimum(THETAS, THETAS[which])
    V1, V2 = _pair(12, th, 3, rotate=False, mix=False)
    _check(O.max_principal_sine, V1, V2, th, atol=0.0)


@pytest.mark.parametrize("which", range(len(THETAS)))
def test_rotated_and_mixed_bases(which):
    th = np.minimum(THETAS, THETAS[which])
    V1, V2 = _pair(40, th, 5 + which)
    # rounding of the rotation and mixing: a few units of eps in absolute terms
    _check(O.max_principal_sine, V1, V2, th, atol=2e-14)


def test_symmetric_in_its_arguments():
    th = np.array([0.01, 0.3, 0.05])
    V1, V2 = _pair(30, th, 9)
    a, b = O.max_principal_sine(V1, V2), O.max_principal_sine(V2, V1)
    assert abs(a - b) <= 1e-14 and abs(a - np.sin(0.3)) <= 1e-13


def test_same_subspace_and_orthogonal_subspaces():
    V1, _ = _pair(20, np.zeros(4), 2)
    assert O.max_principal_sine(V1, V1 @ np.diag([2.0, -1.0, 0.5, 3.0])) <= 1e-14
    E = np.eye(20)
    assert abs(O.max_principal_sine(E[:, :4], E[:, 4:8]) - 1.0) <= 1e-15


def _mutant(old, new):
    src = textwrap.dedent(inspect.getsource(O.max_principal_sine))
    assert src.count(old) == 1, old
    ns = dict(O.max_principal_sine.__globals__)
    exec(compile(src.replace(old, new), "<mutant max_principal_sine>", "exec"), ns)
    return ns["max_principal_sine"]


MUTANTS = [
    ("np.linalg.norm(resid, 2)", "np.linalg.norm(resid, -2)"),       # smallest angle
    ("np.linalg.norm(resid, 2)", "np.linalg.norm(resid)"),           # Frobenius norm
    ("Q1, _ = np.linalg.qr(np.asarray(V1, dtype=np.float64))",
     "Q1 = np.asarray(V1, dtype=np.float64)"),                      # basis not orthonormal
    ("resid = Q2 - Q1 @ (Q1.T @ Q2)", "resid = Q2 - Q1 @ (Q2.T @ Q1)"),   # transposed operand
]


@pytest.mark.parametrize("old,new", MUTANTS)
def test_planted_mistakes_are_caught(old, new):
    bad = _mutant(old, new)
    th = np.array([1e-3, 0.2, 0.05, 0.6])
    V1, V2 = _pair(30, th, 11)
    want = np.sin(0.6)
    assert abs(bad(V1, V2) - want) > 1e-3


# ---------------------------------------------------------------- the relative Frobenius error

def test_rel_fro_is_the_relative_frobenius_norm_of_the_difference():
    """``rel_fro`` is the measure of every state comparison (H, Gram, sums, U): pinned to
    values fixed by construction, so that a helper returning 0, a max-abs norm, or a
    denominator taken from the wrong argument fails."""
    ref = np.array([[3.0, 0.0], [0.0, 4.0]])            # ||ref||_F = 5
    assert O.rel_fro(ref, ref) == 0.0
    assert O.rel_fro(2.0 * ref, ref) == pytest.approx(1.0, rel=1e-15)
    # one entry off by 1: ||diff||_F / ||ref||_F = 1 / 5
    x = ref.copy()
    x[0, 1] = 1.0
    assert O.rel_fro(x, ref) == pytest.approx(0.2, rel=1e-15)
    # Frobenius, not the largest entry: two entries off by 3 and 4 -> 5 / 5
    y = ref.copy()
    y[0, 1], y[1, 0] = 3.0, 4.0
    assert O.rel_fro(y, ref) == pytest.approx(1.0, rel=1e-15)
    # the denominator is the reference's norm: not symmetric in its arguments
    assert O.rel_fro(ref, 2.0 * ref) == pytest.approx(0.5, rel=1e-15)
    # scale invariance and shape independence (a flat view gives the same value)
    rng = np.random.default_rng(0)
    a, b = rng.standard_normal((7, 5)), rng.standard_normal((7, 5))
    assert O.rel_fro(1e-30 * a, 1e-30 * b) == pytest.approx(O.rel_fro(a, b), rel=1e-12)
    assert O.rel_fro(a.ravel(), b.ravel()) == pytest.approx(O.rel_fro(a, b), rel=1e-15)
    assert O.rel_fro(a, b) == pytest.approx(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()), rel=1e-12)
