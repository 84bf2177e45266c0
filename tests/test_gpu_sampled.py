"""GPU parity of the sampled pPCA step and of the variance-captured metric.

* ppca_finalize_sampled vs the oracle's pPCA step restricted to the same
  128-row blocks (the oracle selects them with its own SplitMix64 from the
  generator's definition), fed the GPU's own primed basis: the sampled row
  count is equal; eigenvalue relative error <= 1e-5 and angles <= 1e-4 rad
  (the finalize tolerances, split-precision products);
* fraction 1 keeps every block: the result is bit for bit ppca_finalize's;
* a fraction that keeps no block keeps the one block the rule names;
* ppca_variance_captured vs the oracle's e^T X^T X e for each column:
  relative 4e-6 with ACCURATE products (the projected Gram bound), 1e-2 FAST
  on BF16 data.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev_basis, dev_matrix, host_basis, stored_f64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P(cuda_device):
    import paper_2109_03709_gb300 as P
    P.load_library()
    return P


def _primed(P, dtype, n, d, m, T, seed):
    lam = 0.97 ** np.arange(1, d + 1)
    X, _ = synth.gaussian_data(n, d, lam, seed=seed)
    Xd = dev_matrix(X, dtype)
    h = P.ppca_create(Xd)
    P.ppca_prime(h, P.PPCA_POWER, m, T, V0=dev_basis(synth.initial_basis(d, m, seed)))
    return h, Xd


def _outputs(P, k, d):
    import torch
    return (torch.empty((k, d), dtype=torch.float32, device="cuda"),
            torch.empty(k, dtype=torch.float64, device="cuda"))


def _basis(P, h, d, m):
    import torch
    V = torch.empty((m, d), dtype=torch.float32, device="cuda")
    P.ppca_get_basis(h, V)
    P.ppca_sync(h)
    return host_basis(V)


@pytest.mark.parametrize("dtype,n,fraction,seed", [
    ("bf16", 128 * 150 + 37, 0.1, 7),       # ragged last block
    ("f32", 128 * 150 + 37, 0.3, 11),
    ("bf16", 128 * 40, 0.5, 3),
])
def test_sampled_finalize_matches_oracle(P, dtype, n, fraction, seed):
    d, m, k = 256, 32, 16
    h, Xd = _primed(P, dtype, n, d, m, 5, seed=d + n % 97)
    E, lam = _outputs(P, k, d)
    rows = P.ppca_finalize_sampled(h, k, E, lam, P.PPCA_PREC_ACCURATE, fraction=fraction, seed=seed)
    P.ppca_sync(h)
    tiles, rows_o = oracle.sampled_tiles(n, fraction, seed)
    assert rows == rows_o
    Eo, lo = oracle.ppca_finalize_rows(stored_f64(Xd), _basis(P, h, d, m), k, tiles)
    np.testing.assert_allclose(lam.cpu().numpy(), lo, rtol=1e-5)
    assert oracle.angles(host_basis(E), Eo).max() <= 1e-4


def test_sampled_finalize_with_every_block_is_finalize(P):
    n, d, m, k = 128 * 60 + 5, 200, 24, 8
    h, _ = _primed(P, "bf16", n, d, m, 4, seed=2)
    E1, l1 = _outputs(P, k, d)
    E0, l0 = _outputs(P, k, d)
    rows = P.ppca_finalize_sampled(h, k, E1, l1, P.PPCA_PREC_ACCURATE, fraction=1.0, seed=5)
    P.ppca_finalize(h, k, E0, l0, P.PPCA_PREC_ACCURATE)
    P.ppca_sync(h)
    assert rows == n
    assert np.array_equal(E1.cpu().numpy(), E0.cpu().numpy())
    assert np.array_equal(l1.cpu().numpy(), l0.cpu().numpy())


def test_sampled_finalize_keeps_one_block_when_none_passes(P):
    n, d, m, k = 128 * 30 + 64, 128, 16, 4
    h, Xd = _primed(P, "f32", n, d, m, 3, seed=4)
    E, lam = _outputs(P, k, d)
    rows = P.ppca_finalize_sampled(h, k, E, lam, P.PPCA_PREC_ACCURATE, fraction=1e-300, seed=8)
    P.ppca_sync(h)
    tiles, rows_o = oracle.sampled_tiles(n, 1e-300, 8)
    assert len(tiles) == 1 and rows == rows_o
    Eo, lo = oracle.ppca_finalize_rows(stored_f64(Xd), _basis(P, h, d, m), k, tiles)
    np.testing.assert_allclose(lam.cpu().numpy(), lo, rtol=1e-5)
    assert oracle.angles(host_basis(E), Eo).max() <= 1e-4


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
def test_variance_captured_matches_oracle(P, dtype):
    import torch
    n, d, m, k = 5000, 304, 20, 12
    h, Xd = _primed(P, dtype, n, d, m, 6, seed=17)
    E, lam = _outputs(P, k, d)
    P.ppca_finalize(h, k, E, lam, P.PPCA_PREC_ACCURATE)
    var = torch.empty(k, dtype=torch.float64, device="cuda")
    P.ppca_variance_captured(h, E, k, var, P.PPCA_PREC_ACCURATE)
    P.ppca_sync(h)
    Xs, Eh = stored_f64(Xd), host_basis(E)
    ref = np.array([oracle.variance_captured(Xs, Eh[:, j]) * float(Eh[:, j] @ Eh[:, j]) for j in range(k)])
    np.testing.assert_allclose(var.cpu().numpy(), ref, rtol=4e-6)
    # on the pPCA output the variance captured is n * lambda (Rayleigh quotient of unit vectors)
    np.testing.assert_allclose(var.cpu().numpy(), n * lam.cpu().numpy(), rtol=1e-5)
    if dtype == "bf16":
        P.ppca_variance_captured(h, E, k, var, P.PPCA_PREC_FAST)
        P.ppca_sync(h)
        np.testing.assert_allclose(var.cpu().numpy(), ref, rtol=1e-2)


def test_variance_captured_rejects_k_above_primed_width(P):
    import torch
    h, _ = _primed(P, "bf16", 2000, 128, 8, 2, seed=1)
    E = torch.zeros((16, 128), dtype=torch.float32, device="cuda")
    var = torch.empty(16, dtype=torch.float64, device="cuda")
    with pytest.raises(P.PPCAError, match="INVALID"):
        P.ppca_variance_captured(h, E, 16, var)
