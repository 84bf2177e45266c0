"""The paper's small-scale synthetic protocol (Section 5, Table 2) on the GPU,
against the oracle.

5000 x 50 data whose covariance spectrum decays exponentially or linearly from
1000 to 1, k = 16, minibatch 1000, priming by EigenGame (rate 1e-4) or Oja
(rate 1e-3, constant: the rates the paper's grid picks on these data, see the
bench's paper_synthetic mode), then pPCA_l with l = 0, 2, 4 extra components.
Checked for each (spectrum, primer, l):
* the pPCA step on the GPU's primed basis equals the oracle's pPCA step on the
  same basis (Algorithm 1, steps 2-5): eigenvalues 1e-5 relative, angles
  1e-4 rad plus the FP32 Jacobi's own error 32 u lambda_1 / gap_i (u = 2^-24,
  gap_i to the neighbouring Ritz values: the linear spectrum's are a few per
  cent apart);
* the GPU's priming follows the oracle's own primer from the same V0 over the
  same minibatches (split-precision passes: every direction within 1e-4 rad
  after 100 EigenGame / 40 Oja steps);
* the paper's observation that the pPCA step helps: at V = pi/32 the streak of
  pPCA_4 on top of the primer is at least the primer's own streak.
The truth for the streaks is numpy's LAPACK eigh of X^T X (a test reference).
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

N, D, K, B = 5000, 50, 16, 1000
PLANS = {"eigengame": (100, 1e-4), "oja": (40, 1e-3)}


@pytest.mark.parametrize("spec", ["exponential", "linear"])
@pytest.mark.parametrize("primer", ["eigengame", "oja"])
def test_paper_protocol_ppca_l_against_the_oracle(cuda_device, spec, primer):
    import torch

    import paper_2109_03709_gb300 as P
    P.load_library()
    X, _ = synth.gaussian_data(N, D, synth.paper_synthetic_spectrum(spec, D), seed=5000 + (spec == "linear"))
    Xs = X.astype(np.float32).astype(np.float64)
    Xbuf = torch.zeros((N, 52), dtype=torch.float32, device="cuda")      # 16-byte row pitch
    Xbuf[:, :D] = torch.from_numpy(X.astype(np.float32)).cuda()
    w, U = np.linalg.eigh(Xs.T @ Xs)
    Ut = U[:, ::-1][:, :K]
    steps, rate = PLANS[primer]
    method = P.PPCA_EIGENGAME if primer == "eigengame" else P.PPCA_OJA
    for l in (0, 2, 4):
        m = K + l
        V0 = synth.initial_basis(D, m, seed=100 + l)
        h = P.ppca_create(Xbuf[:, :D])
        prm = P.ppca_prime_params_default(method)
        prm.batch, prm.lr, prm.precision = B, rate, P.PPCA_PREC_ACCURATE
        if method == P.PPCA_OJA:
            prm.lr_offset = 1e12                     # a constant rate: lr / (t + L) with L >> t, times L
            prm.lr = rate * 1e12
        P.ppca_prime(h, method, m, steps, prm,
                     V0=torch.from_numpy(np.ascontiguousarray(V0.T, dtype=np.float32)).cuda())
        E = torch.empty((K, D), dtype=torch.float32, device="cuda")
        lam = torch.empty(K, dtype=torch.float64, device="cuda")
        P.ppca_finalize(h, K, E, lam, P.PPCA_PREC_ACCURATE)
        Vd = torch.empty((m, D), dtype=torch.float32, device="cuda")
        P.ppca_get_basis(h, Vd)
        P.ppca_sync(h)
        Vg = Vd.double().cpu().numpy().T
        Eg = E.double().cpu().numpy().T
        # (1) the pPCA step, deterministic parity on the GPU's own primed basis
        Eall, lall = oracle.ppca_finalize(Xs, Vg, m)
        Eo, lo = Eall[:, :K], lall[:K]
        np.testing.assert_allclose(lam.cpu().numpy(), lo, rtol=1e-5, err_msg=f"{spec} {primer} l={l}")
        nb = np.abs(np.diff(lall))
        gaps = np.minimum(np.r_[np.inf, nb][:K], np.r_[nb, np.inf][:K])
        tol = 1e-4 + 32 * 2.0 ** -24 * lall[0] / gaps
        assert np.all(oracle.angles(Eg, Eo) <= tol), (spec, primer, l)
        # (2) the priming trajectory against the oracle's primer
        if method == P.PPCA_EIGENGAME:
            Vo = oracle.eigengame_prime(Xs, V0, B, steps, rate, 0.9)
        else:
            Vo = oracle.oja_prime(Xs, V0, B, steps, lambda t: rate)
        assert oracle.angles(Vg, Vo).max() <= 1e-4, (spec, primer, l)
        # (3) the pPCA step helps (Table 2's shape)
        if l == 4:
            tol = math.pi / 32
            alone = oracle.lces(oracle.angles(Vg[:, :K], Ut), tol)
            with_ppca = oracle.lces(oracle.angles(Eg, Ut), tol)
            assert with_ppca >= alone, (spec, primer, alone, with_ppca)
