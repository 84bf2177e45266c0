"""GPU parity of the projected Gram matrix G = (X Q)^T (X Q) of the pPCA step.

The reference is the same matrix formed in FP64 on the host from the stored
values of X (exact in FP64) and the FP32 Q.  Errors are measured entrywise on
the scale of the diagonal, |dG_ij| / sqrt(G_ii G_jj), the scale at which an
error moves eigenvalues and eigenvectors of G.  Bounds (u = 2^-24):
* ACCURATE: the operands are split into BF16 pieces whose dropped products are
  below u.  The leading piece product's FP32 tensor-core accumulator takes at
  most 48 MMAs (12 K-stages of 4) before it is folded into an FP32 running
  sum, which bounds its drift to about 1e-6; the other piece products, at most
  2^-8 of Y, accumulate over the whole tile in an accumulator of their own,
  whose drift is relative to that smaller sum.  Y's relative error is then
  ~1.5e-6 and G's about twice that: bound 4e-6.
* FAST, FP32 X (two pieces per operand, products to ~2^-16, no flushing):
  bound 1e-4.
* FAST, BF16 X (Q rounded to BF16, 2^-9 relative): bound 1e-2.
"""
import numpy as np
import pytest

import synth
from gpu_util import dev_basis, dev_matrix, stored_f64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P(cuda_device):
    import paper_2109_03709_gb300 as P
    P.load_library()
    return P


CASES = [
    # n, d, m, r0, r1, dtype, ld
    (1000, 64, 16, 0, 1000, "bf16", None),
    (4099, 200, 64, 3, 4099, "bf16", None),      # ragged d and rows
    (777, 256, 128, 100, 612, "f32", None),
    (50, 16, 1, 0, 1, "f32", None),              # one row, m = 1
    (300, 37, 5, 0, 300, "f32", 40),             # padded leading dimension, ragged d
    (300, 37, 5, 0, 300, "bf16", 40),
    (2050, 1024, 33, 1, 2050, "bf16", None),     # ragged m
    (20000, 2048, 128, 0, 20000, "bf16", None),  # long K: many flush groups
    (20000, 2048, 128, 0, 20000, "f32", None),
]


def scaled_err(G, Gref):
    s = np.sqrt(np.outer(np.diag(Gref), np.diag(Gref)))
    return float(np.max(np.abs(G - Gref) / s))


def run_gram(P, X, dtype, ld, Q, m, r0, r1, prec, flush=0):
    import torch
    Xd = dev_matrix(X, dtype, ld)
    h = P.ppca_create(Xd)
    if flush:
        P.ppca_set_schedule(h, flush=flush)
    G = torch.empty((m, m), dtype=torch.float64, device="cuda")
    P.ppca_projected_gram(h, dev_basis(Q), m, r0, r1, G, prec)
    P.ppca_sync(h)
    Xs = stored_f64(Xd)[r0:r1]
    Y = Xs @ Q.astype(np.float32).astype(np.float64)
    return G.cpu().numpy(), Y.T @ Y


def orthonormal(d, m, seed):
    q, _ = np.linalg.qr(synth.initial_basis(d, m, seed))
    return q


@pytest.mark.parametrize("n,d,m,r0,r1,dtype,ld", CASES)
@pytest.mark.parametrize("prec", ["ACCURATE", "FAST"])
def test_projected_gram(P, n, d, m, r0, r1, dtype, ld, prec):
    lam = 0.95 ** np.arange(1, d + 1)
    X, _ = synth.gaussian_data(n, d, lam, seed=n + d + m)
    Q = orthonormal(d, m, seed=d + m)
    G, Gref = run_gram(P, X, dtype, ld, Q, m, r0, r1, getattr(P, "PPCA_PREC_" + prec))
    assert np.array_equal(G, G.T)
    tol = 4e-6 if prec == "ACCURATE" else (1e-4 if dtype == "f32" else 1e-2)
    assert scaled_err(G, Gref) <= tol


def test_projected_gram_on_top_subspace(P):
    """Q spanning the leading eigenvectors: G is close to diag(lambda), with a
    spread of about 25x; the small diagonal entries keep their relative accuracy."""
    n, d, m = 30000, 512, 64
    lam = np.exp(-np.arange(1, d + 1) / 20.0)
    X, Qt = synth.exact_spectrum_data(n, d, np.sqrt(lam), seed=5)
    Q = Qt[:, :m]
    for dtype in ("f32", "bf16"):
        G, Gref = run_gram(P, X, dtype, None, Q, m, 0, n, P.PPCA_PREC_ACCURATE)
        assert scaled_err(G, Gref) <= 4e-6
        np.testing.assert_allclose(np.diag(G), np.diag(Gref), rtol=4e-6)


@pytest.mark.parametrize("flush", [1, 3, 8, 24])
def test_projected_gram_flush_schedule(P, flush):
    """Any flush interval gives a correct result within the drift it allows
    (about 2e-8 per accumulated MMA; the folded accumulator takes 4 MMAs per
    64-wide K-stage, bounded here as loosely as 24)."""
    n, d, m = 8192, 1024, 64
    lam = 0.97 ** np.arange(1, d + 1)
    X, _ = synth.gaussian_data(n, d, lam, seed=17)
    Q = orthonormal(d, m, seed=3)
    for dtype in ("bf16", "f32"):
        G, Gref = run_gram(P, X, dtype, None, Q, m, 0, n, P.PPCA_PREC_ACCURATE, flush=flush)
        assert scaled_err(G, Gref) <= 4e-6 + 2 * 24 * flush * 2e-8
