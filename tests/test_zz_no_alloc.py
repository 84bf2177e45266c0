"""The allocation-free eigensolve agrees with the handle-based one and with the oracle.

ppca_eigh_noalloc serves callers that cannot allocate device memory where they
need the small eigensolve (a host program whose device memory comes from its
own allocator, or a latency-critical path where cudaMalloc is not acceptable):
its scratch is a fixed library array instead of a handle's workspace.  This
file is collected last on purpose, so that a run stopping at the first failure
has run every other test before it; it also passes alone in a fresh process.

Checks, on two calls in a row (the second reuses the array the first left
behind, with a smaller m):
* the outputs equal ppca_eigh's bit for bit (the same kernels run on the same
  input; only the scratch differs);
* against the oracle's FP64 cyclic Jacobi (oracle.eigh_desc): eigenvalues
  within 1e-9 relative (FP64 Rayleigh quotients of FP32 vectors), vectors
  within the FP32-Jacobi angle bound 16 u |G| / gap (u = 2^-24);
* the status word stays 0 on these well-conditioned inputs.
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


def test_noalloc_matches_handle_eigh_and_oracle_twice_in_a_row(cuda_device):
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
        assert int(status.item()) == 0, call
        assert torch.equal(w1, w0) and torch.equal(U1, U0), call
        w1n, U1n = w1.cpu().numpy(), U1.cpu().numpy().T
        wref, Uref = oracle.eigh_desc(G)
        np.testing.assert_allclose(w1n, wref, rtol=1e-9, atol=1e-9 * abs(wref[0]))
        gaps = np.minimum(np.abs(np.diff(np.r_[np.inf, wref])), np.abs(np.diff(np.r_[wref, -np.inf])))
        for i in range(m):
            assert oracle.angle(U1n[:, i], Uref[:, i]) <= 16 * u * wref[0] / gaps[i] + 1e-6, (call, i)


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
