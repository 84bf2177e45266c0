"""Graph-replayed minibatch steps give the same bits as step-by-step ones.

Oja (Section 2.2) and EigenGame (Section 2.3) take one minibatch per step.  By
default a handle runs blocks of 16 full-minibatch steps from a CUDA graph
captured once, the batch's first row and Oja's step size read from device
memory; steps that hold an epoch's partial batch run one by one.  Here the
same priming runs both ways from the same V0, across epoch boundaries and
partial batches, on FP32 and BF16 data: the primed bases must be equal bit for
bit, and the graph form must launch far fewer kernels from the host.
"""
import numpy as np
import pytest

import synth
from gpu_util import dev_basis, dev_matrix, empty_basis

pytestmark = pytest.mark.gpu


def prime(P, Xd, method, m, T, kw, V0, graphs, counter):
    import torch
    h = P.ppca_create(Xd)
    P.ppca_set_step_graphs(h, graphs)
    prm = P.ppca_prime_params_default(method)
    for k, v in kw.items():
        setattr(prm, k, v)
    prm.precision = P.PPCA_PREC_FAST
    P.ppca_set_timing(counter, True)                  # resets the library-wide launch count
    P.ppca_prime(h, method, m, T, prm, V0=V0)
    P.ppca_prime_continue(h, T)                       # a second call reuses the captured graph
    P.ppca_sync(h)
    launches = P.ppca_get_timing(counter).launches
    V = torch.empty((m, Xd.shape[1]), dtype=torch.float32, device="cuda")
    P.ppca_get_basis(h, V)
    P.ppca_sync(h)
    return V, launches


CASES = [
    # n, d, m, dtype, method, kw, T, bound on the launch ratio (graphs / step by step): an
    # epoch of E batches holds floor((E - 1) / 16) graph blocks; the rest and the capture
    # (16 steps, once) launch one by one
    (20000, 512, 32, "f32", "oja", {"batch": 256, "lr": 1.0, "lr_offset": 100.0}, 100, 0.5),
    (20000, 512, 32, "f32", "eigengame", {"batch": 1024, "lr": 0.1, "momentum": 0.9}, 45, 0.8),
    (12800, 256, 16, "f32", "oja", {"batch": 128, "lr": 0.5, "lr_offset": 50.0}, 120, 0.5),   # n % b == 0
    (20000, 384, 24, "bf16", "oja", {"batch": 256, "lr": 1.0, "lr_offset": 100.0}, 80, 0.6),
    (20000, 384, 24, "bf16", "eigengame", {"batch": 384, "lr": 0.1, "momentum": 0.9}, 70, 0.8),
]


@pytest.mark.parametrize("n,d,m,dtype,method,kw,T,ratio", CASES)
def test_step_graphs_equal_step_by_step(cuda_device, n, d, m, dtype, method, kw, T, ratio):
    import torch

    import paper_2109_03709_gb300 as P
    P.load_library()
    X, _ = synth.gaussian_data(n, d, 0.95 ** np.arange(1, d + 1), seed=31)
    Xd = dev_matrix(X, dtype)
    V0 = dev_basis(synth.initial_basis(d, m, seed=5))
    meth = P.PPCA_OJA if method == "oja" else P.PPCA_EIGENGAME
    counter = P.ppca_create(Xd)
    Vg, lg = prime(P, Xd, meth, m, T, kw, V0, True, counter)
    Vs, ls = prime(P, Xd, meth, m, T, kw, V0, False, counter)
    assert torch.equal(Vg, Vs), float((Vg - Vs).abs().max())
    assert torch.isfinite(Vg).all()
    print(method, dtype, "host launches: graphs", lg, "step by step", ls)
    assert lg < ratio * ls


def test_step_graphs_skip_ragged_batches(cuda_device):
    """A minibatch that is not whole 128-row tiles runs step by step (same launches)."""
    import torch

    import paper_2109_03709_gb300 as P
    P.load_library()
    n, d, m = 6000, 256, 16
    X, _ = synth.gaussian_data(n, d, 0.9 ** np.arange(1, d + 1), seed=2)
    Xd = dev_matrix(X, "f32")
    V0 = dev_basis(synth.initial_basis(d, m, seed=1))
    counter = P.ppca_create(Xd)
    kw = {"batch": 200, "lr": 1.0, "lr_offset": 100.0}
    Vg, lg = prime(P, Xd, P.PPCA_OJA, m, 40, kw, V0, True, counter)
    Vs, ls = prime(P, Xd, P.PPCA_OJA, m, 40, kw, V0, False, counter)
    assert torch.equal(Vg, Vs)
    assert lg == ls


def test_steps_inside_a_caller_capture(cuda_device):
    """A caller capturing the handle's stream gets plain steps it can capture:
    40 Oja steps captured with torch.cuda.graph and replayed once give the same
    bits as the same steps run directly (graph-replayed inside the library)."""
    import torch

    import paper_2109_03709_gb300 as P
    P.load_library()
    n, d, m = 20000, 512, 32
    X, _ = synth.gaussian_data(n, d, 0.95 ** np.arange(1, d + 1), seed=8)
    Xd = dev_matrix(X, "f32")
    V0 = dev_basis(synth.initial_basis(d, m, seed=9))
    kw = {"batch": 256, "lr": 1.0, "lr_offset": 100.0}
    out = []
    for captured in (False, True):
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            h = P.ppca_create(Xd, stream=st)
            prm = P.ppca_prime_params_default(P.PPCA_OJA)
            for k, v in kw.items():
                setattr(prm, k, v)
            prm.precision = P.PPCA_PREC_FAST
            P.ppca_prime(h, P.PPCA_OJA, m, 0, prm, V0=V0)
            P.ppca_sync(h)
            if captured:
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=st):
                    P.ppca_prime_continue(h, 40)
                g.replay()
            else:
                P.ppca_prime_continue(h, 40)
            V = torch.empty((m, d), dtype=torch.float32, device="cuda")
            P.ppca_get_basis(h, V)
            P.ppca_sync(h)
        torch.cuda.synchronize()
        out.append(V)
    assert torch.equal(out[0], out[1])
