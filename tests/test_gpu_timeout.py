"""A bounded device wait that runs out is reported, and the handle recovers.

Every wait inside the library's tensor-core kernels (an mbarrier phase, a
flag another CTA releases) gives up after a limit (2 s by default), records a
timeout in the handle's device status word, drains the copies and MMAs it has
in flight, frees its tensor memory and returns.  Here the limit is cut to 1 ns
with ppca_set_wait_limit, so the first wait that does not complete at once
runs out; no flag is left unset and nothing faults.  The test checks that
ppca_sync returns PPCA_ERR_TIMEOUT, then, with the default limit restored, that
the same handle runs the same pass cleanly and correctly (element by element,
tests/xpass_parity.py).
"""
import numpy as np
import pytest

import synth
from gpu_util import dev_basis, dev_matrix, empty_basis, host_basis, stored_f64
from xpass_parity import TAU_FAST_R, exact_reference, fast_reference, ratio

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P(cuda_device):
    import paper_2109_03709_gb300 as P
    P.load_library()
    return P


CASES = [
    # dtype, fused, what
    ("bf16", 1, "xpass"),        # fused single-read pass: producer / consumer flags and mbarriers
    ("bf16", 0, "xpass"),        # two-kernel pass
    ("f32", -1, "xpass"),        # 3xTF32 pass with transform warps
    ("bf16", -1, "gram"),        # projected Gram (split-precision Y = X Q)
]


@pytest.mark.parametrize("dtype,fused,what", CASES)
def test_wait_that_runs_out_is_reported_and_the_handle_recovers(P, dtype, fused, what):
    import torch
    n, d, m = 20000, 1024, 64
    X = np.random.default_rng(3).standard_normal((n, d)) * (0.99 ** np.arange(1, d + 1))[None, :]
    Xd = dev_matrix(X, dtype)
    Vd = dev_basis(synth.initial_basis(d, m, seed=4))
    h = P.ppca_create(Xd)
    if fused >= 0:
        P.ppca_set_schedule(h, fused=fused)
    Z = empty_basis(d, m)
    G = torch.empty((m, m), dtype=torch.float64, device="cuda")

    def run():
        if what == "xpass":
            P.ppca_xpass(h, Vd, m, 0, n, Z, P.PPCA_PREC_FAST)
        else:
            P.ppca_projected_gram(h, Vd, m, 0, n, G, P.PPCA_PREC_ACCURATE)

    P.ppca_set_wait_limit(1)
    try:
        run()
        with pytest.raises(P.PPCAError) as ei:
            P.ppca_sync(h)
        assert ei.value.status_name == "PPCA_ERR_TIMEOUT"
    finally:
        P.ppca_set_wait_limit(0)
    P.ppca_sync(h)                                   # the status word was cleared
    run()
    P.ppca_sync(h)
    Xs = stored_f64(Xd)
    V = host_basis(Vd)
    if what == "gram":
        Y = Xs @ V
        Gref = Y.T @ Y
        s = np.sqrt(np.outer(np.diag(Gref), np.diag(Gref)))
        assert np.max(np.abs(G.cpu().numpy() - Gref) / s) <= 4e-6
    elif dtype == "bf16":
        Zq, R = fast_reference(Xs, V)
        assert ratio(host_basis(Z), Zq, R, TAU_FAST_R, 5e-4) <= 1.0
    else:
        Ze, R = exact_reference(Xs, V)
        assert ratio(host_basis(Z), Ze, R, 2.0 ** -16, 5e-5) <= 1.0
