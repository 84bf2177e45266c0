"""The allocation-free eigensolve agrees with the handle-based one.

ppca_eigh_noalloc serves callers that cannot allocate device memory where they
need the small eigensolve (inside a stream capture, on a path where cudaMalloc
is not acceptable, under a host-owned allocator): its scratch is a fixed
library array instead of a handle's workspace.  This file is collected last on
purpose, so that a run stopping at the first failure has run every other test
before it; it also passes alone in a fresh process.

Tolerances are those of the eigensolver's own test: eigenvalues within 1e-9
relative, vectors within the FP32-Jacobi angle bound 16 u |G| / gap.
"""
import numpy as np
import pytest

import synth
from gpu_util import dev_matrix

pytestmark = pytest.mark.gpu


def spd(m, seed):
    rng = np.random.default_rng(seed)
    Qm = synth.haar_orthogonal(m, rng)
    lam = np.sort(np.exp(-np.arange(m) / 20.0) * (1 + 0.02 * rng.random(m)))[::-1] * 1e3
    G = (Qm * lam) @ Qm.T
    return 0.5 * (G + G.T)


def test_noalloc_matches_handle_eigh_twice_in_a_row(cuda_device):
    import torch

    import oracle
    import paper_2109_03709_gb300 as P
    P.load_library()
    h = P.ppca_create(dev_matrix(np.zeros((2, 4)), "f32"))
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    u = 2.0 ** -24
    for call, (m, seed) in enumerate([(128, 1), (37, 2)]):
        G = spd(m, seed)
        Gd = torch.from_numpy(G).cuda()
        w0 = torch.empty(m, dtype=torch.float64, device="cuda")
        U0 = torch.empty((m, m), dtype=torch.float64, device="cuda")
        P.ppca_eigh(h, Gd, m, w0, U0)
        P.ppca_sync(h)
        w1 = torch.full((m,), float("nan"), dtype=torch.float64, device="cuda")
        U1 = torch.full((m, m), float("nan"), dtype=torch.float64, device="cuda")
        P.ppca_eigh_noalloc(Gd, m, w1, U1, status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        w0n, w1n = w0.cpu().numpy(), w1.cpu().numpy()
        U0n, U1n = U0.cpu().numpy().T, U1.cpu().numpy().T
        np.testing.assert_allclose(w1n, w0n, rtol=1e-9, atol=1e-9 * abs(w0n[0]))
        gaps = np.minimum(np.abs(np.diff(np.r_[np.inf, w0n])), np.abs(np.diff(np.r_[w0n, -np.inf])))
        for i in range(m):
            assert oracle.angle(U1n[:, i], U0n[:, i]) <= 16 * u * w0n[0] / gaps[i] + 1e-6, (call, i)


def test_noalloc_rejects_m_beyond_the_fixed_scratch(cuda_device):
    import torch

    import paper_2109_03709_gb300 as P
    G = torch.eye(129, dtype=torch.float64, device="cuda")
    w = torch.empty(129, dtype=torch.float64, device="cuda")
    U = torch.empty((129, 129), dtype=torch.float64, device="cuda")
    with pytest.raises(P.PPCAError) as ei:
        P.ppca_eigh_noalloc(G, 129, w, U)
    assert ei.value.status_name == "PPCA_ERR_INVALID"
    assert "scratch" in str(ei.value)
