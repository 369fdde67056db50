"""Seeded synthetic inputs: low-rank-plus-noise data matrices shaped like the paper's workloads.

This module only builds input matrices. It holds none of the PCA method's
arithmetic, and both the CUDA library's tests and the FP64 oracle's tests draw
their inputs from it.

A test matrix is A = U diag(sigma) V^T + noise + 1 mu^T, with U and V
Haar-distributed orthonormal factors (QR of a Gaussian matrix, columns scaled by
the sign of R's diagonal), as in the accuracy experiments of Sec. 4.1, which
multiply a prescribed spectrum by random orthogonal matrices. The spectra of
Sec. 4.1 (Types 1-5) and those of the benchmark workloads are provided.
"""
import math

import numpy as np
import torch


def _gen(seed, device="cpu"):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    return g


def haar(rows, cols, seed):
    """rows x cols matrix with orthonormal columns, Haar-distributed (float64, CPU)."""
    g = _gen(seed)
    X = torch.randn(rows, cols, generator=g, dtype=torch.float64)
    Q, R = torch.linalg.qr(X, mode="reduced")
    d = torch.sign(torch.diagonal(R))
    d[d == 0] = 1.0
    return Q * d[None, :]


def spectrum(kind, r):
    """Singular values sigma_1..sigma_r (float64 numpy).

    'type1'..'type5' are the five laws of Sec. 4.1; 'inv' is 1/i,
    'dec20' is 10^(-i/20), 'pow1.5' is i^-1.5.
    """
    i = np.arange(1, r + 1, dtype=np.float64)
    if kind == "type1":
        s = np.where(i <= 20, 10.0 ** (-4.0 * (i - 1.0) / 19.0),
                     1e-4 / np.maximum(i - 20.0, 1.0) ** 0.1)
        return s
    if kind == "type2":
        return i ** -2.0
    if kind == "type3":
        return i ** -3.0
    if kind == "type4":
        return np.exp(-i / 7.0)
    if kind == "type5":
        return 10.0 ** (-i / 10.0)
    if kind == "inv":
        return 1.0 / i
    if kind == "dec20":
        return 10.0 ** (-i / 20.0)
    if kind == "pow1.5":
        return i ** -1.5
    raise ValueError(kind)


def low_rank_plus_noise(m, n, sigma, *, noise_std=0.0, mean_std=0.0, seed=0,
                        device="cpu", dtype=torch.float64):
    """A = U diag(sigma) V^T + noise_std * N(0,1) + 1 mu^T with mu_j ~ N(0, mean_std^2).

    The factors are drawn in float64 on the CPU from ``seed``; the product, the
    noise and the means are formed on ``device`` in ``dtype``. Returns a torch
    tensor of shape (m, n), row-major.
    """
    sigma = np.asarray(sigma, dtype=np.float64)
    r = sigma.shape[0]
    U = haar(m, r, seed * 4 + 1)
    V = haar(n, r, seed * 4 + 2)
    work = torch.float64 if dtype == torch.float64 else torch.float32
    Us = (U * torch.from_numpy(sigma)[None, :]).to(device=device, dtype=work)
    A = Us @ V.to(device=device, dtype=work).T
    if noise_std:
        g = _gen(seed * 4 + 3, device)
        A.add_(torch.randn(m, n, generator=g, device=device, dtype=work), alpha=noise_std)
    if mean_std:
        mu = torch.randn(n, generator=_gen(seed * 4 + 4), dtype=torch.float64) * mean_std
        A.add_(mu.to(device=device, dtype=work)[None, :])
    return A.to(dtype)


def exact_rank(m, n, r, seed, sigma_kind="inv"):
    """Noise-free rank-r matrix (float64, CPU) with its exact factors.

    Returns (A, U, sigma, V) with A = U diag(sigma) V^T.
    """
    sigma = spectrum(sigma_kind, r)
    U = haar(m, r, seed * 4 + 1).numpy()
    V = haar(n, r, seed * 4 + 2).numpy()
    return (U * sigma[None, :]) @ V.T, U, sigma, V


# --------------------------------------------------------------------------
# Workloads of the benchmark and the parity tests.
# --------------------------------------------------------------------------

SEED_BASE = 17040769


def noise_std_for(level, sigma1, m, n):
    """Per-entry noise std whose m x n Gaussian matrix has spectral norm ~ level * sigma1."""
    return level * sigma1 / (math.sqrt(m) + math.sqrt(n))


def workload_small(seed=SEED_BASE):
    """2000 x 1000, sigma_i = 1/i, per-entry noise 1e-3, k = 10, p = 10, 100-row blocks."""
    m, n = 2000, 1000
    A = low_rank_plus_noise(m, n, spectrum("inv", 1000), noise_std=1e-3, seed=seed)
    return {"name": "2000x1000 f64, sigma_i=1/i + 1e-3 N(0,1), k=10 p=10, 100-row blocks",
            "A": A, "k": 10, "p": 10, "block_rows": 100, "center": True, "seed": seed}


def workload_c2(m=100_000, n=10_000, *, device="cpu", seed=SEED_BASE + 1, dtype=torch.float32):
    """Low-rank-plus-noise FP32 matrix: sigma_i = 10^(-i/20), i <= 200, noise 1e-4 sigma_1,
    column means N(0, 1); k = 50, p = 10 (l = 60), 4096-row blocks."""
    r = min(200, m, n)
    A = low_rank_plus_noise(m, n, spectrum("dec20", r),
                            noise_std=noise_std_for(1e-4, 1.0, m, n), mean_std=1.0,
                            seed=seed, device=device, dtype=dtype)
    return {"name": f"{m}x{n} f32, sigma_i=10^(-i/20) (r={r}) + noise 1e-4 sigma_1, "
                    f"column means N(0,1), k=50 p=10, 4096-row blocks",
            "A": A, "k": 50, "p": 10, "block_rows": 4096, "center": True, "seed": seed}


def workload_c3(m=400_000, n=40_000, *, device="cuda", seed=SEED_BASE + 2, block_rows=8192, r=1000):
    """The 400000 x 40000 precision-sweep matrix, generated one row block at a time on ``device``.

    A = U diag(sigma) V^T + noise with sigma_i = i^-1.5 (i <= r = 1000), per-entry
    noise std 1e-3 sigma_1 / (sqrt(m) + sqrt(n)) (noise spectral norm ~ 1e-3 sigma_1)
    and no column means; k = 100, p = 20 (l = 120), 8192-row blocks. U (m x r) and
    V (n x r) have orthonormal columns: QR of a Gaussian matrix in FP32 on the device
    (a 64 GB FP32 matrix, or even its FP64 factors, is never held whole). Block i's
    noise is drawn from its own seed, so a block can be regenerated alone.

    ``blocks()`` yields (row0, FP32 block) pairs as device tensors.
    """
    r = min(r, m, n)
    sigma = torch.from_numpy(spectrum("pow1.5", r)).to(device=device, dtype=torch.float32)
    noise = noise_std_for(1e-3, 1.0, m, n)

    def orth(rows, s):
        X = torch.randn(rows, r, generator=_gen(s, device), device=device, dtype=torch.float32)
        Q, R = torch.linalg.qr(X, mode="reduced")
        d = torch.sign(torch.diagonal(R))
        d[d == 0] = 1.0
        return Q * d[None, :]

    Us = orth(m, seed * 4 + 1) * sigma[None, :]
    Vt = orth(n, seed * 4 + 2).T.contiguous()

    def blocks():
        for r0 in range(0, m, block_rows):
            r1 = min(m, r0 + block_rows)
            a = Us[r0:r1] @ Vt
            g = _gen(seed * 4 + 3 + 1000 * (r0 // block_rows + 1), device)
            a.add_(torch.randn(r1 - r0, n, generator=g, device=device, dtype=torch.float32), alpha=noise)
            yield r0, a

    return {"name": f"{m}x{n}, sigma_i=i^-1.5 (r={r}) + noise 1e-3 sigma_1, no column means, "
                    f"k=100 p=20, {block_rows}-row blocks",
            "m": m, "n": n, "k": 100, "p": 20, "block_rows": block_rows, "seed": seed, "blocks": blocks}


def store_rows(a, kind):
    """Storage form of a row block: (stored tensor, per-block FP32 scale or None).

    'f32' keeps FP32, 'bf16' rounds to bfloat16 (RNE), 'f8e4m3' stores
    round(a / s) in FP8 e4m3 with the block's scale s = max|a| / 448.
    """
    if kind == "f32":
        return a, None
    if kind == "bf16":
        return a.to(torch.bfloat16), None
    if kind == "f8e4m3":
        amax = float(a.abs().max())
        s = float(np.float32(amax / 448.0)) if amax > 0 else 1.0
        return (a / s).clamp_(-448.0, 448.0).to(torch.float8_e4m3fn), s
    raise ValueError(kind)


def workload_c4(m=937_500, n=40_000, *, device="cuda", seed=SEED_BASE + 3, block_rows=16384, pool=4, r=60):
    """The 937500 x 40000 FP32 stream (150 GB), larger than the device: rows held on the host.

    Row a = sum_{j<r} w_j z_j v_j + eps xi with w_j = 10^(-j/20), z and xi N(0, 1)
    drawn per block from the block's seed, v_1..v_r orthonormal (QR of a Gaussian
    matrix in FP32 on the device), and eps chosen so that the noise spectral norm is
    about 1e-4 sigma_1 (sigma_1 ~ sqrt(m) w_0): eps = 1e-4 sqrt(m) / (sqrt(m) + sqrt(n)).
    k = 50, p = 10 (l = 60), 16384-row blocks.

    The 150 GB are not all materialised: ``pool`` distinct blocks are generated on
    ``device`` and kept in pinned host memory, and the stream cycles through them
    (block i is pool block i mod ``pool``; the ragged last block of m mod 16384 rows
    is the head of its pool block). ``schedule`` lists (pool index, rows) per block.
    """
    r = min(r, n)
    w = torch.tensor(10.0 ** (-np.arange(r) / 20.0), device=device, dtype=torch.float32)
    eps = 1e-4 * math.sqrt(m) / (math.sqrt(m) + math.sqrt(n))
    X = torch.randn(n, r, generator=_gen(seed * 4 + 2, device), device=device, dtype=torch.float32)
    Q, R = torch.linalg.qr(X, mode="reduced")
    d = torch.sign(torch.diagonal(R))
    d[d == 0] = 1.0
    Vt = (Q * d[None, :]).T.contiguous()
    blocks = []
    for b in range(min(pool, (m + block_rows - 1) // block_rows)):
        g = _gen(seed * 4 + 3 + 1000 * (b + 1), device)
        z = torch.randn(block_rows, r, generator=g, device=device, dtype=torch.float32)
        a = (z * w[None, :]) @ Vt
        a.add_(torch.randn(block_rows, n, generator=g, device=device, dtype=torch.float32), alpha=eps)
        host = torch.empty((block_rows, n), dtype=torch.float32, pin_memory=True)
        host.copy_(a)
        blocks.append(host)
        del a
    schedule = [((r0 // block_rows) % len(blocks), min(block_rows, m - r0)) for r0 in range(0, m, block_rows)]
    return {"name": f"{m}x{n} f32 stream from pinned host memory, rank-{r} factors (w_j=10^(-j/20)) + noise "
                    f"1e-4 sigma_1, k=50 p=10, {block_rows}-row blocks, {len(blocks)} distinct blocks cycled",
            "m": m, "n": n, "k": 50, "p": 10, "block_rows": block_rows, "seed": seed,
            "pool": blocks, "schedule": schedule}
