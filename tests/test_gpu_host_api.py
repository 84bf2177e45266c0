"""Host-buffer entry points: ppca_upload (X from host memory into the handle's
device buffer) and ppca_finalize_host (pPCA step, E and lambda into host memory).

The result of upload + prime + finalize_host must equal, bit for bit, the
result of the same calls on a handle created over a device copy of the same
values (the copies move bytes; the arithmetic is the same kernels on the same
values).  Also checked: padded host rows, pageable and page-locked host
buffers, FP8 data with row scales, and the argument errors.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P(cuda_device):
    import paper_2109_03709_gb300 as P
    P.load_library()
    return P


def _solve_device(P, Xd, k, m, T, scales=None):
    import torch
    h = P.ppca_create(Xd, row_scales=scales)
    prm = P.ppca_prime_params_default(P.PPCA_POWER)
    P.ppca_prime(h, P.PPCA_POWER, m, T, prm)
    E = torch.empty((k, Xd.shape[1]), dtype=torch.float32, device="cuda")
    lam = torch.empty(k, dtype=torch.float64, device="cuda")
    P.ppca_finalize(h, k, E, lam, P.PPCA_PREC_ACCURATE)
    P.ppca_sync(h)
    return E.cpu().numpy(), lam.cpu().numpy()


@pytest.mark.parametrize("dtype,pinned,pad", [("bf16", True, 0), ("bf16", False, 0), ("f32", True, 8),
                                              ("f32", False, 0), ("bf16", True, 24)])
def test_upload_and_finalize_host_match_device_path(P, dtype, pinned, pad):
    import torch
    n, d, k, m, T = 3000, 200, 6, 12, 4
    X, _ = synth.gaussian_data(n, d, 0.9 ** np.arange(1, d + 1), seed=d + pad)
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    Xd = torch.from_numpy(X.astype(np.float32)).to(tdt).cuda()
    E0, lam0 = _solve_device(P, Xd, k, m, T)

    host = torch.zeros((n, d + pad), dtype=tdt, pin_memory=pinned)
    host[:, :d] = Xd.cpu()
    Xbuf = torch.full_like(Xd, 7.0)                      # overwritten by the upload
    h = P.ppca_create(Xbuf)
    P.ppca_upload(h, host[:, :d] if pad else host, ld_host=d + pad)
    prm = P.ppca_prime_params_default(P.PPCA_POWER)
    P.ppca_prime(h, P.PPCA_POWER, m, T, prm)
    E_h = torch.empty((k, d), dtype=torch.float32, pin_memory=pinned)
    lam_h = torch.empty(k, dtype=torch.float64, pin_memory=pinned)
    P.ppca_finalize_host(h, k, E_h, lam_h, P.PPCA_PREC_ACCURATE)
    P.ppca_sync(h)
    assert torch.equal(Xbuf, Xd)
    assert np.array_equal(E_h.numpy(), E0)
    assert np.array_equal(lam_h.numpy(), lam0)


def test_upload_fp8_with_row_scales(P):
    import torch
    n, d, k, m, T = 2000, 128, 4, 8, 3
    X, _ = synth.gaussian_data(n, d, 0.9 ** np.arange(1, d + 1), seed=5)
    Xf = torch.from_numpy(X.astype(np.float32)).cuda()
    X8 = torch.empty((n, d), dtype=torch.uint8, device="cuda")
    s = torch.empty(n, dtype=torch.float32, device="cuda")
    P.ppca_quantize_fp8(Xf, X8, s)
    torch.cuda.synchronize()
    E0, lam0 = _solve_device(P, X8, k, m, T, scales=s)

    X8h, sh = X8.cpu().pin_memory(), s.cpu().pin_memory()
    buf8, bufs = torch.zeros_like(X8), torch.zeros_like(s)
    h = P.ppca_create(buf8, row_scales=bufs)
    P.ppca_upload(h, X8h, row_scales_host=sh)
    P.ppca_prime(h, P.PPCA_POWER, m, T, P.ppca_prime_params_default(P.PPCA_POWER))
    E_h = torch.empty((k, d), dtype=torch.float32)
    lam_h = torch.empty(k, dtype=torch.float64)
    P.ppca_finalize_host(h, k, E_h, lam_h, P.PPCA_PREC_ACCURATE)
    P.ppca_sync(h)
    assert np.array_equal(E_h.numpy(), E0)
    assert np.array_equal(lam_h.numpy(), lam0)


def test_host_api_argument_errors(P):
    import torch
    n, d = 500, 64
    Xd = torch.zeros((n, d), dtype=torch.bfloat16, device="cuda")
    h = P.ppca_create(Xd)
    host = torch.zeros((n, d), dtype=torch.bfloat16)
    with pytest.raises(P.PPCAError, match="INVALID"):
        P.ppca_upload(h, host, ld_host=d - 1)
    with pytest.raises(P.PPCAError, match="INVALID"):
        P.ppca_upload(h, host, row_scales_host=torch.ones(n))       # scales only for FP8 data
    with pytest.raises(P.PPCAError, match="STATE"):                  # finalize before prime
        P.ppca_finalize_host(h, 2, torch.empty((2, d)), torch.empty(2, dtype=torch.float64))
