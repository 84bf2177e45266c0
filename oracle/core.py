"""FP64 oracle for primed PCA -- test infrastructure (see the package docstring).

Notation follows the paper: X is the centred n x d data matrix (Section 1),
V the d x m primed basis with m = k + l (Algorithm 1; Section 3.3), e_i the
principal directions (eigenvectors of X^T X), pPCA_l the method with l extra
components.

Readings taken where the paper is silent (they are the same readings the CUDA
path implements, restated here independently):

* eigenvalues are reported as eig(X^T X) / n (Section 1 uses X^T X, Section 4.1
  divides by the number of points); eigenvectors in descending eigenvalue
  order, each signed so that its largest-magnitude entry (lowest index among
  ties) is positive;
* the block power method is the simultaneous iteration the paper cites
  (Section 2.1): V <- orth(X^T X V), T times, orth = thin QR with a positive
  diagonal;
* the initial basis of every primer is orth(V0) for a caller-supplied V0;
* minibatch t (0-based) covers rows [j b, min((j+1) b, n)) with
  j = t mod ceil(n / b): contiguous, epoch-aligned, the last batch of each
  epoch partial and averaged over its true size;
* Oja/Sanger (Section 2.2) averaged over the minibatch, no renormalisation;
* EigenGame (Section 2.3): every player ascends its own utility with the
  others held fixed, the gradient projected on the sphere's tangent space,
  SGD with Nesterov momentum (Section 5), then renormalised; all players are
  updated in parallel from the same minibatch, M_b = X_b^T X_b / |b|.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

__all__ = [
    "build_native", "jacobi_eigh", "eigh_desc", "sign_fix", "orth", "qr_pos",
    "covariance", "ground_truth", "ppca_finalize",
    "power_step", "power_prime", "power_seq_prime", "minibatch_rows", "oja_step", "oja_prime",
    "eigengame_gradients", "eigengame_step", "eigengame_prime",
    "angle", "angles", "lces", "principal_angles", "variance_captured",
    "splitmix64", "sampled_tiles", "ppca_finalize_rows",
    "bf16_bits_to_f64", "bf16_round_rne", "e4m3_decode", "e4m3_encode_rne", "fp8_row_quantize",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIBPATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = [os.path.join(_HERE, "jacobi.c")]
_lib = None
_lock = threading.Lock()


def build_native(force: bool = False) -> str:
    """Compile the oracle's C sources with gcc into ``oracle/_build``.

    Plain ISO C, -O2, no fused multiply-add contraction, so the x86 build
    machine and the aarch64 GPU host give the same bits.
    """
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SOURCES)
    if not force and os.path.exists(_LIBPATH) and os.path.getmtime(_LIBPATH) >= newest:
        return _LIBPATH
    tmp = _LIBPATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, *_SOURCES, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIBPATH)
    return _LIBPATH


def _native():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_native())
            lib.oracle_jacobi_cyclic.restype = ctypes.c_int
            lib.oracle_jacobi_cyclic.argtypes = [
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int]
            assert lib.oracle_jacobi_abi_version() == 1
            _lib = lib
    return _lib


# ---------------------------------------------------------------------------
# Symmetric eigensolver (the "full-PCA" of Algorithm 1, step 4)
# ---------------------------------------------------------------------------

def jacobi_eigh(A, tol: float = 1e-14, max_sweeps: int = 60):
    """Eigenpairs of a real symmetric matrix by cyclic-by-row Jacobi (jacobi.c).

    Returns (w, U), unsorted: A = U diag(w) U^T.
    """
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("jacobi_eigh: square matrix required")
    if not np.allclose(A, A.T, rtol=0.0, atol=1e-12 * max(1.0, float(np.abs(A).max(initial=0.0)))):
        raise ValueError("jacobi_eigh: matrix is not symmetric")
    A = 0.5 * (A + A.T)
    n = A.shape[0]
    U = np.empty_like(A)
    if n == 0:
        return np.zeros(0), U
    sweeps = _native().oracle_jacobi_cyclic(A.ctypes.data, U.ctypes.data, n, tol, max_sweeps)
    if sweeps < 0:
        raise RuntimeError("jacobi_eigh: no convergence")
    return np.diag(A).copy(), U


def sign_fix(U):
    """Sign convention: each column's largest-|entry| (lowest index among ties) is positive."""
    U = np.array(U, dtype=np.float64, copy=True)
    for j in range(U.shape[1]):
        i = int(np.argmax(np.abs(U[:, j])))
        if U[i, j] < 0:
            U[:, j] = -U[:, j]
    return U


def eigh_desc(A):
    """Eigenpairs in descending eigenvalue order (stable for ties), sign-fixed."""
    w, U = jacobi_eigh(A)
    order = np.argsort(-w, kind="stable")
    return w[order], sign_fix(U[:, order])


# ---------------------------------------------------------------------------
# Orthonormalisation: thin QR with positive diagonal, by modified Gram-Schmidt
# applied twice.  The CUDA path uses CholeskyQR2; with a positive diagonal the
# thin QR factor is unique, so both must give the same Q up to rounding.
# ---------------------------------------------------------------------------

def orth(V):
    """Q with orthonormal columns, span(Q[:, :j]) = span(V[:, :j]) for every j."""
    Q = np.array(V, dtype=np.float64, copy=True)
    if Q.ndim != 2:
        raise ValueError("orth: matrix required")
    m = Q.shape[1]
    for _ in range(2):
        for j in range(m):
            for i in range(j):
                Q[:, j] -= (Q[:, i] @ Q[:, j]) * Q[:, i]
            nrm = math.sqrt(float(Q[:, j] @ Q[:, j]))
            if nrm == 0.0:
                raise np.linalg.LinAlgError("orth: rank-deficient basis")
            Q[:, j] /= nrm
    return Q


def qr_pos(V):
    """(Q, R) with V = Q R, R upper triangular with positive diagonal."""
    V = np.asarray(V, dtype=np.float64)
    Q = orth(V)
    R = np.triu(Q.T @ V)
    return Q, R


# ---------------------------------------------------------------------------
# O1: ground truth and O2: the pPCA step (Algorithm 1)
# ---------------------------------------------------------------------------

def covariance(X):
    """X^T X in FP64 from the stored values (Section 1)."""
    X = np.asarray(X, dtype=np.float64)
    return X.T @ X


def ground_truth(X, k: int | None = None):
    """Top-k principal directions and eig(X^T X)/n (Section 1), by Jacobi."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    w, U = eigh_desc(covariance(X))
    if k is None:
        k = U.shape[1]
    return U[:, :k], w[:k] / n


def ppca_finalize(X, V, k: int):
    """Algorithm 1, steps 2-5: span -> project -> full-PCA -> top k.

    Q = orth(V) spans V (step 2); the projected points x~_i = Q Q^T x_i (step 3)
    have covariance Q (Q^T X^T X Q) Q^T, whose nonzero eigenpairs are those of
    the m x m matrix G = (X Q)^T (X Q) rotated by Q (step 4; Section 4.2 shows
    the variance of X~ is that of X restricted to S).  Returns E (d x k) and
    eig/n, descending.
    """
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    Q = orth(V)
    Y = X @ Q
    G = Y.T @ Y
    w, U = eigh_desc(G)
    E = sign_fix(Q @ U[:, :k])
    return E, w[:k] / n


# ---------------------------------------------------------------------------
# O2s: the pPCA step on a seeded sample of the rows
# ---------------------------------------------------------------------------
#
# For its large-scale runs the paper projects only 10 % of the data in the
# full-PCA step (Section 5, ResNet activations) without saying which 10 %.
# Reading: the rows are taken in blocks of 128 consecutive rows; block t is
# kept when the t-th output of the SplitMix64 stream seeded with `seed`, as a
# 53-bit fraction, is below `fraction`; if no block is kept, the block with the
# smallest output (lowest index among ties) is.  The eigenvalues are those of
# the sampled Gram matrix divided by the number of sampled rows.

_MASK64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(state: int) -> int:
    """SplitMix64 output for the stream state after its increment (Steele,
    Lea and Flood, "Fast splittable pseudorandom number generators", 2014):
    z = state; z = (z ^ z >> 30) * 0xBF58476D1CE4E5B9; z = (z ^ z >> 27) *
    0x94D049BB133111EB; z ^ z >> 31, all modulo 2^64."""
    z = state & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def sampled_tiles(n: int, fraction: float, seed: int, tile: int = 128):
    """Indices of the kept 128-row blocks (ascending) and the kept row count."""
    nt = (n + tile - 1) // tile
    us = [splitmix64((seed + (t + 1) * _GOLDEN) & _MASK64) for t in range(nt)]
    keep = [t for t in range(nt) if (us[t] >> 11) * 2.0 ** -53 < fraction]
    if not keep:
        keep = [min(range(nt), key=lambda t: (us[t], t))]
    rows = sum(min(tile, n - t * tile) for t in keep)
    return keep, rows


def ppca_finalize_rows(X, V, k: int, tiles, tile: int = 128):
    """ppca_finalize restricted to the rows of the given 128-row blocks:
    G = (X_S Q)^T (X_S Q), eigenvalues / |S|."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    idx = np.concatenate([np.arange(t * tile, min((t + 1) * tile, n)) for t in tiles])
    Q = orth(V)
    Y = X[idx] @ Q
    G = Y.T @ Y
    w, U = eigh_desc(G)
    E = sign_fix(Q @ U[:, :k])
    return E, w[:k] / len(idx)


# ---------------------------------------------------------------------------
# O3: primers
# ---------------------------------------------------------------------------

def power_step(X, Q):
    """One simultaneous-iteration step (Section 2.1): orth(X^T X Q)."""
    X = np.asarray(X, dtype=np.float64)
    return orth(X.T @ (X @ Q))


def power_prime(X, V0, T: int):
    """Block power priming: Q0 = orth(V0), then T steps of power_step."""
    Q = orth(V0)
    for _ in range(T):
        Q = power_step(X, Q)
    return Q


def power_seq_prime(X, V0, T: int, eps: float):
    """The power method as Section 2.1 describes it: one direction at a time,
    x <- M x / |M x| with M = X^T X, each step orthogonalised against the
    directions already found (the complement of their span), until
    |x_t - x_{t+1}| < eps or T steps.  Direction j starts from column j of
    orth(V0); the orthogonalisation is classical Gram-Schmidt applied twice.
    Returns V (d x m) and the steps taken per direction."""
    X = np.asarray(X, dtype=np.float64)
    Q0 = orth(V0)
    d, m = Q0.shape
    V = np.zeros((d, m))
    steps = []
    for j in range(m):
        x = Q0[:, j].copy()
        Vp = V[:, :j]
        t = 0
        while t < T:
            y = X.T @ (X @ x)
            for _ in range(2):
                y = y - Vp @ (Vp.T @ y)
            x_new = y / np.linalg.norm(y)
            t += 1
            done = np.linalg.norm(x_new - x) < eps
            x = x_new
            if done:
                break
        V[:, j] = x
        steps.append(t)
    return V, steps


def minibatch_rows(t: int, n: int, b: int):
    """Rows [r0, r1) of minibatch t: epoch-aligned contiguous batches."""
    if b <= 0 or n <= 0:
        raise ValueError("minibatch_rows: n, b must be positive")
    per_epoch = -(-n // b)
    j = t % per_epoch
    r0 = j * b
    return r0, min(r0 + b, n)


def oja_step(X, W, t: int, b: int, lr: float):
    """Generalised Oja (Sanger) rule, Section 2.2, averaged over minibatch t.

    For one point: dw_j = lr * y_j * (x - sum_{l <= j} y_l w_l), y = W^T x.
    Summed over the batch and divided by its size this is
    dW = lr / |b| * (X_b^T Y - W triu(Y^T Y)).
    """
    X = np.asarray(X, dtype=np.float64)
    r0, r1 = minibatch_rows(t, X.shape[0], b)
    Xb = X[r0:r1]
    Y = Xb @ W
    S = Y.T @ Y
    m = W.shape[1]
    dW = Xb.T @ Y
    for j in range(m):
        for l in range(j + 1):
            dW[:, j] -= S[l, j] * W[:, l]
    return W + (lr / (r1 - r0)) * dW


def oja_prime(X, V0, b: int, steps: int, lr_fn, t0: int = 0):
    W = orth(V0)
    for t in range(t0, t0 + steps):
        W = oja_step(X, W, t, b, lr_fn(t))
    return W


def eigengame_gradients(Xb, V):
    """Utility gradients of all players (Section 2.3, Eq. 3), M = Xb^T Xb / |b|.

    dU_j/dv_j = 2 M v_j - 2 sum_{i<j} (v_j^T M v_i) / (v_i^T M v_i) M v_i.
    Returns (grad, MV, C) with C = V^T M V.
    """
    Xb = np.asarray(Xb, dtype=np.float64)
    MV = Xb.T @ (Xb @ V) / Xb.shape[0]
    C = V.T @ MV
    grad = 2.0 * MV.copy()
    for j in range(V.shape[1]):
        for i in range(j):
            grad[:, j] -= 2.0 * (C[i, j] / C[i, i]) * MV[:, i]
    return grad, MV, C


def eigengame_step(X, V, buf, t: int, b: int, lr: float, momentum: float = 0.9):
    """One parallel EigenGame step on minibatch t.

    Riemannian gradient g_j = grad_j - (v_j^T grad_j) v_j; Nesterov momentum
    (Section 5): buf <- mu buf + g, v <- v + lr (g + mu buf); then v_j <- v_j/|v_j|.
    """
    X = np.asarray(X, dtype=np.float64)
    r0, r1 = minibatch_rows(t, X.shape[0], b)
    grad, _, _ = eigengame_gradients(X[r0:r1], V)
    g = grad - V * np.sum(V * grad, axis=0, keepdims=True)
    buf = momentum * buf + g
    Vn = V + lr * (g + momentum * buf)
    Vn = Vn / np.linalg.norm(Vn, axis=0, keepdims=True)
    return Vn, buf


def eigengame_prime(X, V0, b: int, steps: int, lr: float, momentum: float = 0.9, t0: int = 0):
    V = orth(V0)
    buf = np.zeros_like(V)
    for t in range(t0, t0 + steps):
        V, buf = eigengame_step(X, V, buf, t, b, lr, momentum)
    return V


# ---------------------------------------------------------------------------
# O4: metrics (Section 5.3)
# ---------------------------------------------------------------------------

def angle(v, e):
    """Sign-invariant angle between directions v and e, in radians.

    arccos(|<v,e>| / (|v||e|)) written as atan2(|v_perp|, |<v,e>|) on unit
    vectors, which is the same angle but well conditioned near zero.
    """
    v = np.asarray(v, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    v = v / np.linalg.norm(v)
    e = e / np.linalg.norm(e)
    c = float(v @ e)
    perp = np.linalg.norm(v - c * e)
    return math.atan2(perp, abs(c))


def angles(Vhat, E):
    return np.array([angle(Vhat[:, i], E[:, i]) for i in range(min(Vhat.shape[1], E.shape[1]))])


def lces(angle_list, tol: float) -> int:
    """Longest correct eigenvector streak: leading count with angle < tol."""
    s = 0
    for a in angle_list:
        if a < tol:
            s += 1
        else:
            break
    return s


def principal_angles(Q, E):
    """Principal angles between span(Q) (orthonormal) and span(E), ascending.

    sin(theta_i) are the singular values of (I - Q Q^T) E_o, E_o = orth(E);
    squared singular values come from this package's Jacobi.
    """
    Q = orth(Q)
    Eo = orth(E)
    W = Eo - Q @ (Q.T @ Eo)
    s2, _ = jacobi_eigh(W.T @ W)
    s = np.sqrt(np.clip(s2, 0.0, 1.0))
    return np.sort(np.arcsin(s))


def variance_captured(X, v):
    """v^T (X^T X) v for a unit direction v (Section 5.3 footnote)."""
    X = np.asarray(X, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    v = v / np.linalg.norm(v)
    y = X @ v
    return float(y @ y)


# ---------------------------------------------------------------------------
# Storage formats: exact decoding of the stored low-precision values.
# ---------------------------------------------------------------------------

def bf16_bits_to_f64(bits):
    """bfloat16 bit patterns (uint16) -> exact float64 values."""
    b = np.asarray(bits, dtype=np.uint16).astype(np.uint32) << np.uint32(16)
    return b.view(np.float32).astype(np.float64)


def bf16_round_rne(x):
    """Values -> the nearest bfloat16 value (ties to even mantissa), as float64.

    The input is first taken to FP32 (the precision the data-format step and
    the tensor-core epilogues round from); the FP32 bit pattern is then rounded
    at bit 16 to nearest, ties to the even BF16 mantissa.  Finite inputs only
    (FP32 overflow to infinity is the caller's concern).
    """
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    keep = bits >> np.uint64(16)
    rest = bits & np.uint64(0xFFFF)
    up = (rest > np.uint64(0x8000)) | ((rest == np.uint64(0x8000)) & ((keep & np.uint64(1)) == np.uint64(1)))
    keep = keep + up.astype(np.uint64)
    return bf16_bits_to_f64(keep.astype(np.uint16))


def _e4m3_table():
    vals = np.empty(256, dtype=np.float64)
    for code in range(256):
        sign = -1.0 if code & 0x80 else 1.0
        exp = (code >> 3) & 0xF
        man = code & 0x7
        if exp == 0xF and man == 0x7:
            vals[code] = np.nan            # E4M3 has NaN but no infinities
        elif exp == 0:
            vals[code] = sign * (man / 8.0) * 2.0 ** (1 - 7)   # subnormal
        else:
            vals[code] = sign * (1.0 + man / 8.0) * 2.0 ** (exp - 7)
    return vals


_E4M3 = _e4m3_table()


def e4m3_decode(codes):
    """FP8 E4M3 (bias 7, max 448, NaN = S.1111.111, no inf) -> float64."""
    return _E4M3[np.asarray(codes, dtype=np.uint8)]


def e4m3_encode_rne(x):
    """float values -> nearest E4M3 code, ties to the even code, |x| > 448 saturates.

    Nearest-value search over the table of the 127 non-negative finite codes
    (the codes are monotone in value, so "even code" is "even mantissa").
    """
    x = np.asarray(x, dtype=np.float64)
    pos_codes = np.arange(0x7F, dtype=np.int64)            # 0x00 .. 0x7E
    pos_vals = _E4M3[pos_codes]
    a = np.minimum(np.abs(x), 448.0)
    j = np.searchsorted(pos_vals, a, side="left")
    jc = np.clip(j, 0, len(pos_vals) - 1)
    exact = pos_vals[jc] == a
    lo = np.clip(j - 1, 0, len(pos_vals) - 1)
    hi = jc
    dlo = a - pos_vals[lo]
    dhi = pos_vals[hi] - a
    pick_lo = (dlo < dhi) | ((dlo == dhi) & (pos_codes[lo] % 2 == 0))
    code = np.where(exact, pos_codes[jc], np.where(pick_lo, pos_codes[lo], pos_codes[hi]))
    neg = np.signbit(x)
    code = np.where(neg, code | 0x80, code)
    code = np.where(np.isnan(x), 0x7F, code)
    return code.astype(np.uint8)


def fp8_row_quantize(X32):
    """Per-row E4M3 quantisation of FP32 rows (data-format step, reading).

    s_r = max_j |x_rj| / 448 and q_rj = E4M3(x_rj / s_r), both divisions in
    IEEE FP32 (correctly rounded); an all-zero row gets s_r = 1.
    Returns (codes uint8 n x d, scales float32 n).
    """
    X32 = np.asarray(X32, dtype=np.float32)
    amax = np.max(np.abs(X32), axis=1)
    s = np.where(amax > 0, amax / np.float32(448.0), np.float32(1.0)).astype(np.float32)
    q = (X32 / s[:, None]).astype(np.float32)
    return e4m3_encode_rne(q), s
