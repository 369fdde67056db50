"""Oracle (test infrastructure only): single-pass randomized PCA, step by step in FP64.

Plain numpy/scipy in float64. Library routines serve only as single steps the
paper itself names (a matrix product, ``qr``, ``svd``, a triangular solve, a
Cholesky factorisation); nothing is blocked, fused or reordered beyond what the
paper's algorithms state. Section, equation and algorithm numbers refer to
Yu, Gu, Li, Liu, Li, "Single-Pass PCA of Large High-Dimensional Data",
IJCAI 2017 (arXiv 1704.07669).

Readings where the paper is silent (each one is also listed in the design notes):

* centering: PCA assumes a column-centred matrix (Sec. 2.1). ``center`` is the
  plain two-pass definition. The streaming library subtracts a shift c (the FP32
  column mean of the first row block) and corrects exactly at the end;
  ``shifted_state`` and ``centering_correction`` restate that algebra so that a
  test can pin it to the two-pass definition.
* R from the Gram matrix: with G not stored, the QB factor R of G = QR is the
  Cholesky factor of G^T G (upper triangular with positive diagonal, hence the
  same R as a QR with positive diagonal), followed by one refinement step in
  Gram space; see ``gram_qb``. Thm 1 makes this equal to Alg. 4 in exact
  arithmetic.
* rank deficiency: when the Gram matrix is numerically singular (Thm 1 assumes
  full column rank), ``gram_qb`` falls back to its eigendecomposition and keeps
  the eigenvalues above l * eps * lambda_max.
* signs and order: singular values descending; each right singular vector is
  scaled by +-1 so that its entry of largest magnitude (lowest index on ties) is
  positive.
* power scheme (Sec. 3.2, Sec. 4): "orth" is the Q factor of the QR of H; the
  new Omega is, like the Gaussian one, defined as its value in the operand
  format (``power_omega``). Only range(Omega) matters to the result, so any
  orthonormal basis of H gives the same sigma and V.
* streams too large to hold in FP64 are fed block by block (``ShiftedPass``);
  a block repeated in a stream may be folded in once with its multiplicity,
  the same sum as Eq. 11 over the stream.
"""
import numpy as np
import scipy.linalg as sla

from . import philox

EPS64 = np.finfo(np.float64).eps


# --------------------------------------------------------------------------
# Stored-value rounding (the data the library reads, and the reduced-precision
# forms of Omega and G). Round-to-nearest-even throughout.
# --------------------------------------------------------------------------

def round_f32(x):
    """Round to IEEE binary32 (RNE) and return as float64."""
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def round_bf16(x):
    """Round to bfloat16 (RNE on the binary32 bit pattern) and return as float64.

    The value is first rounded to binary32, then the low 16 bits of its bit
    pattern are rounded off to nearest, ties to an even upper half.
    """
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> np.uint64(16)) & np.uint64(1)
    rounded = ((bits + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def decode_e4m3(codes):
    """Value of FP8 E4M3 (OCP 'fn' variant: no infinities, 0x7F/0xFF are NaN) codes.

    Layout: sign bit, 4 exponent bits (bias 7), 3 mantissa bits; exponent field 0
    encodes subnormals m * 2^-9.
    """
    c = np.asarray(codes, dtype=np.uint8).astype(np.int64)
    sign = np.where(c & 0x80, -1.0, 1.0)
    e = (c >> 3) & 0xF
    m = c & 0x7
    normal = (1.0 + m / 8.0) * np.exp2(e - 7.0)
    sub = (m / 8.0) * np.exp2(-6.0)
    val = np.where(e == 0, sub, normal)
    val = np.where((c & 0x7F) == 0x7F, np.nan, val)
    return sign * val


# --------------------------------------------------------------------------
# Omega (Alg. 4 step 3) in the forms the library uses.
# --------------------------------------------------------------------------

def round_f16(x):
    """Round to IEEE binary16 and return as float64: first to binary32, then
    to binary16, each to nearest with ties to even (numpy's conversions)."""
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float16).astype(np.float64)


def omega(n, l, seed, form="f64"):
    """Omega = randn(n, l): FP64 draw, optionally defined as its FP32, BF16 or FP16 value."""
    z = philox.omega(n, l, seed)
    if form == "f64":
        return z
    if form == "f32":
        return round_f32(z)
    if form == "bf16":
        return round_bf16(z)
    if form == "f16":
        return round_f16(z)
    raise ValueError(form)


# --------------------------------------------------------------------------
# Centering (Sec. 2.1: rows are observations, columns must have zero mean).
# --------------------------------------------------------------------------

def column_means(A):
    """mu_j = (1/m) sum_i A_ij in FP64."""
    A = np.asarray(A, dtype=np.float64)
    return A.sum(axis=0) / A.shape[0]


def center(A):
    """Plain two-pass centering: A_bar = A - 1 mu^T."""
    A = np.asarray(A, dtype=np.float64)
    return A - column_means(A)[None, :]


def row_blocks(A, block_rows):
    """The stream of row blocks 'read next few rows of A' (Alg. 4 step 5)."""
    m = A.shape[0]
    return [A[i:i + block_rows] for i in range(0, m, block_rows)]


# --------------------------------------------------------------------------
# The one pass (Alg. 4 steps 3-8; Eq. 11).
# --------------------------------------------------------------------------

def sketch_pass(blocks, Omega):
    """Alg. 4 while loop: for each block a, g = a Omega; G = [G; g]; H = H + a^T g.

    Returns (G, H) with G of shape (m, l) and H of shape (n, l).
    """
    n, l = Omega.shape
    H = np.zeros((n, l))
    G_parts = []
    for a in blocks:
        a = np.asarray(a, dtype=np.float64)
        g = a @ Omega            # step 6
        G_parts.append(g)        # step 6: G = [G; g]
        H = H + a.T @ g          # step 7, Eq. 11
    G = np.vstack(G_parts) if G_parts else np.zeros((0, l))
    return G, H


def first_block_shift(first_block):
    """The shift c: FP64 column mean of the first row block, stored as FP32."""
    return round_f32(column_means(first_block))


def shifted_state(blocks, Omega, c):
    """Accumulators of the pass on A_hat = A - 1 c^T, by their plain definitions.

    Returns dict with G_hat = A_hat Omega (m x l), H_hat = A_hat^T G_hat (n x l),
    gram = G_hat^T G_hat (l x l), s = A_hat^T 1 (n), sG = G_hat^T 1 (l), m.
    """
    A_hat = np.vstack([np.asarray(a, dtype=np.float64) for a in blocks]) - np.asarray(c)[None, :]
    G_hat = A_hat @ Omega
    return {
        "G": G_hat,
        "H": A_hat.T @ G_hat,
        "gram": G_hat.T @ G_hat,
        "s": A_hat.sum(axis=0),
        "sG": G_hat.sum(axis=0),
        "m": A_hat.shape[0],
    }


def centering_correction(H_hat, gram, s, sG, m):
    """From shifted accumulators to those of the column-centred matrix.

    With A_bar = A_hat - (1/m) 1 s^T and G_bar = A_bar Omega = G_hat - (1/m) 1 sG^T:
      H_bar    = A_bar^T G_bar = H_hat - (1/m) s sG^T
      gram_bar = G_bar^T G_bar = gram  - (1/m) sG sG^T
    """
    s = np.asarray(s, dtype=np.float64)
    sG = np.asarray(sG, dtype=np.float64)
    return H_hat - np.outer(s, sG) / m, gram - np.outer(sG, sG) / m


class ShiftedPass:
    """The accumulators of ``shifted_state``, fed one row block at a time.

    For matrices too large to hold in FP64 at once: each block a is shifted,
    g = a_hat Omega is formed (Alg. 4 step 6) and H, the Gram matrix and the sums
    are increased by that block's terms (step 7, Eq. 11). The shift c is the
    ``first_block_shift`` of the first block added unless one is given.
    """

    def __init__(self, Omega, c=None, keep_G=True):
        self.Omega = np.asarray(Omega, dtype=np.float64)
        n, l = self.Omega.shape
        self.c = None if c is None else np.asarray(c, dtype=np.float64)
        self.H = np.zeros((n, l))
        self.gram = np.zeros((l, l))
        self.s = np.zeros(n)
        self.sG = np.zeros(l)
        self.m = 0
        self.G_parts = [] if keep_G else None

    def add(self, a, overwrite=False, times=1):
        """Fold block a in; with ``overwrite`` the shifted rows replace a's values.

        ``times`` > 1 folds in that many consecutive copies of the same block (a
        stream that repeats a block): each sum gains ``times`` equal terms.
        """
        a = np.asarray(a, dtype=np.float64)
        if self.c is None:
            self.c = first_block_shift(a)
        if overwrite:
            a_hat = a
            np.subtract(a, self.c[None, :], out=a_hat)
        else:
            a_hat = a - self.c[None, :]
        g = a_hat @ self.Omega
        self.H += times * (a_hat.T @ g)
        self.gram += times * (g.T @ g)
        self.s += times * a_hat.sum(axis=0)
        self.sG += times * g.sum(axis=0)
        self.m += times * a_hat.shape[0]
        if self.G_parts is not None:
            self.G_parts.extend([g] * times)
        return g

    def state(self):
        """Same keys as ``shifted_state`` (G only when kept)."""
        G = np.vstack(self.G_parts) if self.G_parts else None
        return {"G": G, "H": self.H, "gram": self.gram, "s": self.s, "sG": self.sG, "m": self.m}


def finalize_centred(G_hat, H_hat, s, sG, m, Omega, k, b=10):
    """sigma_1..k and V of the column-centred rows from the shifted pass (FP64).

    The centring correction, then Alg. 4 steps 9-19 on G_bar = G_hat - (1/m) 1 sG^T
    and H_bar, with the same sign convention as ``single_pass_pca``.
    """
    H_bar, _ = centering_correction(H_hat, np.zeros((len(sG), len(sG))), s, sG, m)
    G_bar = np.asarray(G_hat, dtype=np.float64) - np.asarray(sG, dtype=np.float64)[None, :] / m
    Q, B = blocked_qb(G_bar, H_bar, Omega, b)
    _, sigma, V = svd_truncate(None, B, k)
    V, _ = sign_fix(V)
    return sigma, V


# --------------------------------------------------------------------------
# Finalisation: blocked QB with re-orthogonalisation (Alg. 4 steps 9-16).
# --------------------------------------------------------------------------

def qr(Y):
    """Unpivoted Householder QR, economy size (the paper's qr / qr(X, 0))."""
    Q, R = np.linalg.qr(Y, mode="reduced")
    return Q, R


def blocked_qb(G, H, Omega, b):
    """Alg. 4 steps 9-16: Q (m x l) and B (l x n) from G, H and Omega, block size b.

    For i = 1..t:
      Omega_i = Omega(:, block i)
      Y_i = G(:, block i) - Q (B Omega_i)                         (step 11)
      [Q_i, R_i] = qr(Y_i)                                        (step 12)
      [Q_i, R~_i] = qr(Q_i - Q (Q^T Q_i))                         (step 13, Eq. 8)
      R_i = R~_i R_i                                              (step 14)
      B_i = R_i^-T (H(:, block i)^T - Y_i^T Q B - Omega_i^T B^T B) (step 15, Eq. 10)
      Q = [Q, Q_i];  B = [B; B_i]                                 (step 16)
    In the first iteration Q and B are empty and their terms vanish.
    """
    m, l = G.shape
    n = H.shape[0]
    if l % b:
        raise ValueError("l must be a multiple of b (Alg. 4 step 2: l = t b)")
    Q = np.zeros((m, 0))
    B = np.zeros((0, n))
    for i in range(l // b):
        cols = slice(i * b, (i + 1) * b)
        Om_i = Omega[:, cols]
        Y_i = G[:, cols] - Q @ (B @ Om_i)
        Q_i, R_i = qr(Y_i)
        Q_i, Rt_i = qr(Q_i - Q @ (Q.T @ Q_i))
        R_i = Rt_i @ R_i
        rhs = H[:, cols].T - (Y_i.T @ Q) @ B - (Om_i.T @ B.T) @ B
        B_i = sla.solve_triangular(R_i, rhs, trans="T", lower=False)
        Q = np.hstack([Q, Q_i])
        B = np.vstack([B, B_i])
    return Q, B


def svd_truncate(Q, B, k):
    """Alg. 4 steps 17-19: [U~, S, V] = svd(B); U = Q U~; keep the leading k.

    Q may be None when only S and V are wanted. Returns (U or None, sigma, V).
    """
    U_t, S, Vt = np.linalg.svd(B, full_matrices=False)
    V = Vt.T
    U = None if Q is None else Q @ U_t[:, :k]
    return U, S[:k].copy(), V[:, :k].copy()


def left_vectors_second_pass(A, V, sigma, center_columns=True):
    """U = A_bar V diag(sigma)^-1 (FP64): the left singular vectors from a second pass over
    the rows, for a caller that kept no sketch rows. The truncated SVD A_bar ~ U diag(sigma)
    V^T of Alg. 4 step 19 with V^T V = I gives U = A_bar V diag(sigma)^-1 when A_bar lies in
    the span of V (exactly for a rank-r matrix, r <= k); otherwise it is the projection the
    second pass computes, where step 18's U = Q U~ projects onto range(Q) instead. Columns for
    zero sigma are 0."""
    A_bar = center(A) if center_columns else np.asarray(A, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    inv = np.where(sigma > 0, 1.0 / np.where(sigma > 0, sigma, 1.0), 0.0)
    return (A_bar @ np.asarray(V, dtype=np.float64)) * inv[None, :]


def sign_fix(V, U=None):
    """Scale each column of V by +-1 so its largest-|.| entry (lowest index on ties) is > 0."""
    V = np.array(V, dtype=np.float64, copy=True)
    U = None if U is None else np.array(U, dtype=np.float64, copy=True)
    for i in range(V.shape[1]):
        j = int(np.argmax(np.abs(V[:, i])))
        if V[j, i] < 0:
            V[:, i] = -V[:, i]
            if U is not None:
                U[:, i] = -U[:, i]
    return V, U


# --------------------------------------------------------------------------
# Gram reading of the same QB factorisation (G not stored).
# --------------------------------------------------------------------------

def gram_qb(gram, H, refine=True):
    """R from the Gram matrix and B = R^-T H^T.

    Full rank: R1 = chol(gram) (upper), then one refinement in Gram space,
    R2 = chol(R1^-T gram R1^-1), R = R2 R1. Returns dict(T, B, rank) with
    T = R^-T, so that B = T H^T and the implicit Q = G T^T.
    Numerically singular gram: eigendecomposition gram = W diag(lam) W^T,
    keep lam > l eps lam_max, T = diag(lam_r)^-1/2 W_r^T.
    """
    l = gram.shape[0]
    gram = 0.5 * (gram + gram.T)
    lam_max = max(float(np.max(np.abs(np.diag(gram)))), 0.0)
    tol = l * EPS64 * lam_max
    try:
        L1 = np.linalg.cholesky(gram)
        if np.min(np.diag(L1)) ** 2 <= tol:
            raise np.linalg.LinAlgError("pivot below tolerance")
        R = L1.T
        if refine:
            Rinv = sla.solve_triangular(R, np.eye(l), lower=False)
            X = Rinv.T @ gram @ Rinv
            R2 = np.linalg.cholesky(0.5 * (X + X.T)).T
            R = R2 @ R
        T = sla.solve_triangular(R, np.eye(l), trans="T", lower=False)   # R^-T
        return {"T": T, "B": T @ H.T, "rank": l, "route": "cholesky"}
    except np.linalg.LinAlgError:
        lam, W = np.linalg.eigh(gram)
        order = np.argsort(lam)[::-1]
        lam, W = lam[order], W[:, order]
        keep = lam > l * EPS64 * max(lam[0], 0.0)
        T = (W[:, keep] / np.sqrt(lam[keep])[None, :]).T
        return {"T": T, "B": T @ H.T, "rank": int(keep.sum()), "route": "eigen"}


# --------------------------------------------------------------------------
# Alg. 1 (two passes) and a brute-force SVD for pins.
# --------------------------------------------------------------------------

def randqb_two_pass(A, Omega):
    """Alg. 1 steps 3-4: Q = orth(A Omega), B = Q^T A (second pass over A)."""
    A = np.asarray(A, dtype=np.float64)
    Q, _ = qr(A @ Omega)
    return Q, Q.T @ A


def jacobi_svd(A, sweeps=60, tol=1e-15):
    """One-sided (Hestenes) Jacobi SVD of an m x n matrix, m >= n; brute force.

    Plane rotations orthogonalise the columns of A; the column norms are then the
    singular values, the normalised columns the left vectors and the accumulated
    rotations the right vectors. Returns (U, sigma, V), sigma descending.
    """
    X = np.array(A, dtype=np.float64, copy=True)
    m, n = X.shape
    if m < n:
        U, s, V = jacobi_svd(X.T, sweeps, tol)
        return V, s, U
    V = np.eye(n)
    for _ in range(sweeps):
        off = 0.0
        for p in range(n - 1):
            for q in range(p + 1, n):
                alpha = X[:, p] @ X[:, p]
                beta = X[:, q] @ X[:, q]
                gamma = X[:, p] @ X[:, q]
                if gamma == 0.0:
                    continue
                off = max(off, abs(gamma) / np.sqrt(alpha * beta))
                zeta = (beta - alpha) / (2.0 * gamma)
                t = np.sign(zeta) / (abs(zeta) + np.sqrt(1.0 + zeta * zeta)) if zeta != 0 else 1.0
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = c * t
                xp, xq = X[:, p].copy(), X[:, q].copy()
                X[:, p], X[:, q] = c * xp - s * xq, s * xp + c * xq
                vp, vq = V[:, p].copy(), V[:, q].copy()
                V[:, p], V[:, q] = c * vp - s * vq, s * vp + c * vq
        if off < tol:
            break
    sig = np.sqrt(np.sum(X * X, axis=0))
    order = np.argsort(sig)[::-1]
    sig, X, V = sig[order], X[:, order], V[:, order]
    U = np.where(sig[None, :] > 0, X / np.where(sig > 0, sig, 1.0)[None, :], 0.0)
    return U, sig, V


# --------------------------------------------------------------------------
# The whole method.
# --------------------------------------------------------------------------

def power_omega(H, omega_form="f64"):
    """The power scheme with P = 1 for Alg. 4 (Sec. 3.2, Sec. 4): the test matrix of the
    extra pass is H after ``orth`` - the Q factor of H's QR - defined, like the random
    Omega, as its value in the operand format."""
    Q, _ = qr(H)
    if omega_form == "f64":
        return Q
    return {"f32": round_f32, "bf16": round_bf16, "f16": round_f16}[omega_form](Q)


def single_pass_pca(A, k, p, seed, block_rows, *, center_columns=True, b=10,
                    finalize="blocked", omega_form="f64", keep_U=False, power=0):
    """Single-pass PCA (Alg. 4) of the rows of A, in FP64.

    A           m x n data (float64 view of the stored values), rows = observations
    k, p        rank and oversampling, l = k + p
    seed        Philox key for Omega
    block_rows  rows per streamed block (Alg. 4 step 5); the result does not
                depend on it in exact arithmetic
    finalize    'blocked' = Alg. 4 steps 9-16 on the stored G (the paper);
                'gram'    = R from the Gram matrix (G not stored)
    power       P of the power scheme (0 or more): each extra pass reruns the while
                loop with Omega replaced by orth(H) (Sec. 4)
    Returns dict(sigma (k), V (n x k), U (m x k) or None, Omega, G, H).
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    l = k + p
    Om = omega(n, l, seed, omega_form)
    A_bar = center(A) if center_columns else A
    G, H = sketch_pass(row_blocks(A_bar, block_rows), Om)
    for _ in range(power):   # the while loop once more, Omega replaced by orth(H)
        Om = power_omega(H, omega_form)
        G, H = sketch_pass(row_blocks(A_bar, block_rows), Om)
    if finalize == "blocked":
        Q, B = blocked_qb(G, H, Om, b)
    elif finalize == "gram":
        res = gram_qb(G.T @ G, H)
        B = res["B"]
        Q = G @ res["T"].T
    else:
        raise ValueError(finalize)
    U, sigma, V = svd_truncate(Q if keep_U else None, B, k)
    if sigma.shape[0] < k:
        pad = k - sigma.shape[0]
        sigma = np.concatenate([sigma, np.zeros(pad)])
        V = np.hstack([V, np.zeros((n, pad))])
        if U is not None:
            U = np.hstack([U, np.zeros((m, pad))])
    V, U = sign_fix(V, U)
    return {"sigma": sigma, "V": V, "U": U, "Omega": Om, "G": G, "H": H}


# --------------------------------------------------------------------------
# Error measures used by the tests and the benchmark.
# --------------------------------------------------------------------------

def rel_fro(x, ref):
    """||x - ref||_F / ||ref||_F."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / (den if den > 0 else 1.0))


def max_principal_sine(V1, V2):
    """sin of the largest principal angle between range(V1) and range(V2).

    Computed as ||(I - Q1 Q1^T) Q2||_2 (no cancellation for tiny angles).
    """
    Q1, _ = np.linalg.qr(np.asarray(V1, dtype=np.float64))
    Q2, _ = np.linalg.qr(np.asarray(V2, dtype=np.float64))
    resid = Q2 - Q1 @ (Q1.T @ Q2)
    return float(np.linalg.norm(resid, 2))
