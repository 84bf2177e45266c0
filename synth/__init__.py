"""Seeded synthetic inputs for primed-PCA workloads.

This module is shared by the tests, ``bench.py`` and ``__graft_entry__.smoke()``
and feeds both the CUDA path and the FP64 oracle.  It holds none of the pPCA
arithmetic: it only draws data matrices with a prescribed population spectrum
and initial bases.

Generators:

* ``gaussian_data``: X = G diag(sqrt(lambda)) Q^T with G i.i.d. N(0, 1), Q Haar
  orthogonal, columns centred -- the known-lambda recipe of the workloads.
* ``exact_spectrum_data``: X = U diag(sigma) Q^T with U's orthonormal columns
  orthogonal to the all-ones vector, so X is centred and X^T X = Q diag(sigma^2)
  Q^T holds up to rounding: eigenpairs known in closed form.
* ``initial_basis``: Gaussian d x m starting basis for the primers.
* ``hadamard_rotated_data_torch``: the known-lambda recipe for very wide X
  (d = 2^18), with a structured orthogonal Q = H D1 P H D2 applied by fast
  Walsh-Hadamard transforms instead of a stored Haar matrix.

Small problems are drawn with numpy on the host (float64, then rounded to the
storage type).  Large problems (``*_torch``) are drawn on a torch device in
row chunks so that nothing larger than one chunk of G is ever materialised.
"""
from __future__ import annotations

import math

import numpy as np

from .configs import CONFIGS, Config, spectrum  # noqa: F401


def haar_orthogonal(d: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed d x d orthogonal matrix: QR of a Gaussian, R's diagonal made positive."""
    G = rng.standard_normal((d, d))
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))[None, :]


def gaussian_data(n: int, d: int, lam, seed: int, center: bool = True):
    """(X, Q): X = G diag(sqrt(lam)) Q^T in float64, columns centred."""
    lam = np.asarray(lam, dtype=np.float64)
    assert lam.shape == (d,)
    rng = np.random.default_rng(seed)
    Q = haar_orthogonal(d, rng)
    G = rng.standard_normal((n, d))
    X = (G * np.sqrt(lam)[None, :]) @ Q.T
    if center:
        X -= X.mean(axis=0, keepdims=True)
    return X, Q


def exact_spectrum_data(n: int, d: int, sigma, seed: int):
    """(X, Q): X = U diag(sigma) Q^T, U^T U = I, U^T 1 = 0, so X^T X = Q diag(sigma^2) Q^T.

    Requires n > d.  U is the QR factor of a column-centred Gaussian n x d.
    """
    sigma = np.asarray(sigma, dtype=np.float64)
    assert sigma.shape == (d,) and n > d
    rng = np.random.default_rng(seed)
    Q = haar_orthogonal(d, rng)
    A = rng.standard_normal((n, d))
    A -= A.mean(axis=0, keepdims=True)
    U, R = np.linalg.qr(A)
    U = U * np.sign(np.diag(R))[None, :]
    X = (U * sigma[None, :]) @ Q.T
    return X, Q


def paper_synthetic_spectrum(kind: str, d: int = 50, top: float = 1000.0, bottom: float = 1.0) -> np.ndarray:
    """The covariance spectra of the paper's synthetic small-scale data (Section 5):
    d = 50 eigenvalues decaying exponentially ("exponential") or linearly
    ("linear") over three orders of magnitude, from 1000 to 1."""
    t = np.arange(d) / (d - 1)
    if kind == "exponential":
        return top * (bottom / top) ** t
    if kind == "linear":
        return top + (bottom - top) * t
    raise ValueError(kind)


def initial_basis(d: int, m: int, seed: int) -> np.ndarray:
    """Gaussian d x m starting basis (float64)."""
    rng = np.random.default_rng(seed + 7919)
    return rng.standard_normal((d, m))


def affine_to_unit_and_recentre(X: np.ndarray) -> np.ndarray:
    """Global affine map of all entries to [0, 1], then columns re-centred (image-like data)."""
    lo, hi = float(X.min()), float(X.max())
    Y = (X - lo) / (hi - lo)
    return Y - Y.mean(axis=0, keepdims=True)


# ---------------------------------------------------------------------------
# Large problems on a torch device
# ---------------------------------------------------------------------------

def gaussian_data_torch(n: int, d: int, lam, seed: int, device, out_dtype, chunk_rows: int = 65536,
                        image_like: bool = False):
    """X = G diag(sqrt(lam)) Q^T drawn on ``device`` in row chunks, stored as ``out_dtype``.

    Returns (X, Q_host).  Q is Haar (drawn on the host in float64); G comes from
    a seeded torch generator on the device.  Columns are centred with column
    means accumulated in float64.  With ``image_like`` the values are mapped by
    one global affine map to [0, 1] and re-centred.
    """
    import torch

    lam = np.asarray(lam, dtype=np.float64)
    rng = np.random.default_rng(seed)
    Q = haar_orthogonal(d, rng)
    B = torch.from_numpy((np.sqrt(lam)[:, None] * Q.T).astype(np.float32)).to(device)   # d x d
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    X = torch.empty((n, d), dtype=torch.float32, device=device)
    for r0 in range(0, n, chunk_rows):
        r1 = min(n, r0 + chunk_rows)
        G = torch.randn((r1 - r0, d), generator=gen, device=device, dtype=torch.float32)
        X[r0:r1] = G @ B
        del G
    mean = torch.zeros(d, dtype=torch.float64, device=device)
    for r0 in range(0, n, chunk_rows):
        mean += X[r0:r0 + chunk_rows].double().sum(0)
    mean /= n
    X -= mean.float()[None, :]
    if image_like:
        lo, hi = float(X.min()), float(X.max())
        X -= lo
        X /= (hi - lo)
        mean.zero_()
        for r0 in range(0, n, chunk_rows):
            mean += X[r0:r0 + chunk_rows].double().sum(0)
        mean /= n
        X -= mean.float()[None, :]
    if out_dtype != torch.float32:
        Xo = torch.empty((n, d), dtype=out_dtype, device=device)
        for r0 in range(0, n, chunk_rows):
            Xo[r0:r0 + chunk_rows] = X[r0:r0 + chunk_rows].to(out_dtype)
        del X
        X = Xo
    return X, Q


def batch_instances(count: int, seed: int):
    """Shapes of a ragged batch: n ~ U[2000, 200000], d in {64, ..., 2048}, k ~ U[4, 32],
    l = k, lambda_i = rho^i with rho ~ U[0.8, 0.98] per instance (m = 2k <= min(d, 128))."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        d = int(rng.choice([64, 128, 256, 512, 1024, 2048]))
        k = int(rng.integers(4, 33))
        k = min(k, d // 2)
        out.append({"n": int(rng.integers(2000, 200001)), "d": d, "k": k, "m": 2 * k,
                    "rho": float(rng.uniform(0.8, 0.98)), "seed": int(seed * 100003 + i)})
    return out


def haar_orthogonal_torch(d: int, gen, device):
    """Haar orthogonal d x d on a torch device: QR of a Gaussian, R's diagonal made positive."""
    import torch
    G = torch.randn((d, d), generator=gen, device=device, dtype=torch.float64)
    Q, R = torch.linalg.qr(G)
    return Q * torch.sign(torch.diagonal(R))[None, :]


def instance_data_torch(n: int, d: int, lam, seed: int, device, out_dtype):
    """X = G diag(sqrt(lam)) Q^T, columns centred, drawn entirely on the device (for batches)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    Q = haar_orthogonal_torch(d, gen, device)
    B = (torch.sqrt(torch.as_tensor(np.asarray(lam), dtype=torch.float64, device=device))[:, None] * Q.T).float()
    X = torch.randn((n, d), generator=gen, device=device, dtype=torch.float32) @ B
    X -= X.double().mean(0).float()[None, :]
    return X.to(out_dtype) if out_dtype != torch.float32 else X


def _fwht_rows_(Y):
    """In-place normalised Walsh-Hadamard transform of each row of Y (last dim a power of two)."""
    import torch
    n, d = Y.shape
    h = 1
    while h < d:
        v = Y.view(n, d // (2 * h), 2, h)
        a = v[:, :, 0, :].clone()
        v[:, :, 0, :] += v[:, :, 1, :]
        v[:, :, 1, :] *= -1.0
        v[:, :, 1, :] += a
        h *= 2
    Y *= 1.0 / math.sqrt(d)
    return Y


def hadamard_rotated_data_torch(n: int, d: int, lam, seed: int, device, out_dtype, chunk_rows: int = 1024):
    """X = G diag(sqrt(lam)) Q^T for d a power of two, Q = H D1 P H D2 (H the normalised
    Walsh-Hadamard matrix, D1, D2 random sign diagonals, P a random permutation), columns
    centred, stored as ``out_dtype``.  Q is orthogonal and never formed: each row is
    rotated with two fast transforms, so d = 2^18 fits.  Drawn on ``device`` in row chunks
    from per-chunk torch generators (two passes: column means, then the centred rows).
    Returns (X, (D1, perm, D2)) with the signs and permutation as host arrays.
    """
    import torch

    assert d & (d - 1) == 0, "d must be a power of two"
    lam = np.asarray(lam, dtype=np.float64)
    rng = np.random.default_rng(seed)
    D1 = rng.choice([-1.0, 1.0], size=d)
    D2 = rng.choice([-1.0, 1.0], size=d)
    perm = rng.permutation(d)
    sq = torch.from_numpy(np.sqrt(lam)).to(device=device, dtype=torch.float32)
    d1 = torch.from_numpy(D1).to(device=device, dtype=torch.float32)
    d2 = torch.from_numpy(D2).to(device=device, dtype=torch.float32)
    pinv = torch.from_numpy(np.argsort(perm)).to(device=device)

    def rows(c):
        r0 = c * chunk_rows
        r1 = min(n, r0 + chunk_rows)
        gen = torch.Generator(device=device)
        gen.manual_seed(int(seed) * 1000003 + c)
        Y = torch.randn((r1 - r0, d), generator=gen, device=device, dtype=torch.float32)
        Y *= sq[None, :]                  # G diag(sqrt(lam))
        Y *= d2[None, :]                  # ... Q^T = D2 H P^T D1 H, applied on the right
        _fwht_rows_(Y)
        Y = Y[:, pinv]
        Y *= d1[None, :]
        _fwht_rows_(Y)
        return r0, r1, Y

    nchunks = (n + chunk_rows - 1) // chunk_rows
    mean = torch.zeros(d, dtype=torch.float64, device=device)
    for c in range(nchunks):
        _, _, Y = rows(c)
        mean += Y.double().sum(0)
    mean /= n
    meanf = mean.float()
    X = torch.empty((n, d), dtype=out_dtype, device=device)
    for c in range(nchunks):
        r0, r1, Y = rows(c)
        Y -= meanf[None, :]
        X[r0:r1] = Y.to(out_dtype)
    return X, (D1, perm, D2)


def counterexample_points():
    """The 6-point, 3-dimensional data set of the counterexample (Section 4.1)."""
    return np.array([[3, 0, 0], [-3, 0, 0], [0, 2, 0], [0, -2, 0], [0, 0, 1], [0, 0, -1]], dtype=np.float64)


def minibatch_schedule_rows(n: int, b: int, steps: int, t0: int = 0):
    """Row ranges a primer visits (for bookkeeping of bytes streamed)."""
    per_epoch = -(-n // b)
    out = []
    for t in range(t0, t0 + steps):
        j = t % per_epoch
        out.append((j * b, min(n, j * b + b)))
    return out


def bytes_of(n: int, d: int, dtype: str) -> int:
    return n * d * {"f32": 4, "bf16": 2, "fp8": 1}[dtype] + (4 * n if dtype == "fp8" else 0)


def ceil_div(a: int, b: int) -> int:
    return -(-a // b)


def log2_int(x: int) -> int:
    return int(math.log2(x))
