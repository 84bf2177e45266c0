"""GPU parity of primed PCA end to end (Algorithm 1) against the FP64 oracle.

* finalize vs the oracle's pPCA step fed the GPU's own primed basis
  (deterministic parity): eigenvalue relative error <= 1e-5, angles <= 1e-4
  rad (the FP32-path tolerances);
* power priming vs the oracle's block power from the same V0: the primed
  subspaces agree (largest principal angle <= 1e-4);
* the whole pipeline vs the ground truth on the 4096 x 256 workload: the same
  LCES as the oracle's own pipeline, eigenvalues within 1e-5;
* Oja and EigenGame trajectories vs the oracle's, step by step, for a few
  steps (FP32 vs FP64: <= 1e-4 entrywise after 5 steps); EigenGame also on a
  32768 x 16 basis (1e-4 of the largest entry; unit columns to 1e-6);
* FP8 priming with the pPCA step on the BF16 copy (ppca_set_refine);
* priming state: finalize does not change it; checkpoint/resume is bit-exact;
* host-side errors: finalize before prime, workspace cap, bad k.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev_basis, dev_matrix, empty_basis, host_basis, stored_f64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P(cuda_device):
    import paper_2109_03709_gb300 as P
    P.load_library()
    return P


def finalize(P, h, d, k, precision=None):
    import torch
    E = torch.empty((k, d), dtype=torch.float32, device="cuda")
    lam = torch.empty(k, dtype=torch.float64, device="cuda")
    P.ppca_finalize(h, k, E, lam, P.PPCA_PREC_AUTO if precision is None else precision)
    P.ppca_sync(h)
    return host_basis(E), lam.cpu().numpy()


def get_basis(P, h, d, m):
    V = empty_basis(d, m)
    P.ppca_get_basis(h, V)
    P.ppca_sync(h)
    return host_basis(V)


def check_against(E, lam, Eref, lref, eig_rtol, angle_tol):
    np.testing.assert_allclose(lam, lref, rtol=eig_rtol)
    ang = oracle.angles(E, Eref)
    assert ang.max() <= angle_tol, ang


@pytest.fixture(scope="module")
def c1(P):
    cfg = synth.CONFIGS["power_fp32_4096x256"]
    X, _ = synth.gaussian_data(cfg.n, cfg.d, cfg.lam(), cfg.seed)
    Xd = dev_matrix(X, "f32")
    Xs = stored_f64(Xd)
    V0 = synth.initial_basis(cfg.d, cfg.m, cfg.seed)
    return cfg, Xd, Xs, V0


def test_power_pipeline_4096x256(P, c1):
    cfg, Xd, Xs, V0 = c1
    h = P.ppca_create(Xd)
    V0d = dev_basis(V0)
    P.ppca_prime(h, P.PPCA_POWER, cfg.m, cfg.primers["power"]["T"], V0=V0d)
    E, lam = finalize(P, h, cfg.d, cfg.k)
    Vg = get_basis(P, h, cfg.d, cfg.m)
    # (1) finalize parity on the GPU's own basis
    Eo, lo = oracle.ppca_finalize(Xs, Vg, cfg.k)
    check_against(E, lam, Eo, lo, 1e-5, 1e-4)
    # (2) primed subspace vs the oracle's block power from the same V0
    Vo = oracle.power_prime(Xs, host_basis(V0d), cfg.primers["power"]["T"])
    assert oracle.principal_angles(Vg, Vo).max() <= 1e-4
    # (3) against the ground truth: same streak as the oracle's pipeline
    Et, lt = oracle.ground_truth(Xs, cfg.k)
    Eop, lop = oracle.ppca_finalize(Xs, Vo, cfg.k)
    np.testing.assert_allclose(lam, lt, rtol=1e-5)
    assert oracle.lces(oracle.angles(E, Et), cfg.angle_tol) == oracle.lces(oracle.angles(Eop, Et), cfg.angle_tol)
    # the output is orthonormal and lies in span(V)
    assert np.abs(E.T @ E - np.eye(cfg.k)).max() <= 1e-5
    Qg = oracle.orth(Vg)
    assert np.abs(E - Qg @ (Qg.T @ E)).max() <= 1e-5


def test_power_more_iterations_reaches_full_streak(P, c1):
    cfg, Xd, Xs, V0 = c1
    h = P.ppca_create(Xd)
    P.ppca_prime(h, P.PPCA_POWER, cfg.m, 20, V0=dev_basis(V0))
    E, lam = finalize(P, h, cfg.d, cfg.k)
    Et, lt = oracle.ground_truth(Xs, cfg.k)
    check_against(E, lam, Et, lt, 1e-5, 1e-4)


def test_fp8_priming_then_refine_copy_finalize(P):
    """FP8 data (E4M3 + row scales) primes; the pPCA step reads the BF16 copy
    set with ppca_set_refine: parity with the oracle's pPCA step on the BF16
    values from the GPU's own primed basis (eigenvalues 1e-5, angles 1e-4 rad)."""
    import torch
    n, d, k, m, T = 3000, 256, 8, 16, 6
    X, _ = synth.gaussian_data(n, d, 0.9 ** np.arange(1, d + 1), seed=21)
    Xf = torch.from_numpy(X.astype(np.float32)).cuda()
    X16 = torch.empty((n, d), dtype=torch.bfloat16, device="cuda")
    X8 = torch.empty((n, d), dtype=torch.uint8, device="cuda")
    s = torch.empty(n, dtype=torch.float32, device="cuda")
    P.ppca_quantize_bf16(Xf, X16)
    P.ppca_quantize_fp8(Xf, X8, s)
    torch.cuda.synchronize()
    h = P.ppca_create(X8, row_scales=s)
    P.ppca_set_refine(h, X16)
    P.ppca_prime(h, P.PPCA_POWER, m, T, P.ppca_prime_params_default(P.PPCA_POWER),
                 V0=dev_basis(synth.initial_basis(d, m, 21)))
    E, lam = finalize(P, h, d, k, P.PPCA_PREC_ACCURATE)
    Vg = get_basis(P, h, d, m)
    Eo, lo = oracle.ppca_finalize(stored_f64(X16), Vg, k)
    check_against(E, lam, Eo, lo, 1e-5, 1e-4)


def test_finalize_does_not_change_priming_state(P, c1):
    cfg, Xd, Xs, V0 = c1
    h = P.ppca_create(Xd)
    P.ppca_prime(h, P.PPCA_POWER, cfg.m, 3, V0=dev_basis(V0))
    Va = get_basis(P, h, cfg.d, cfg.m)
    E1, l1 = finalize(P, h, cfg.d, cfg.k)
    E2, l2 = finalize(P, h, cfg.d, cfg.k)
    Vb = get_basis(P, h, cfg.d, cfg.m)
    np.testing.assert_array_equal(Va, Vb)
    np.testing.assert_array_equal(E1, E2)
    np.testing.assert_array_equal(l1, l2)


@pytest.mark.parametrize("method", ["OJA", "EIGENGAME"])
def test_checkpoint_resume_bit_exact(P, method):
    n, d, m = 3000, 128, 8
    X, _ = synth.gaussian_data(n, d, 0.9 ** np.arange(1, d + 1), seed=4)
    Xd = dev_matrix(X, "f32")
    V0 = dev_basis(synth.initial_basis(d, m, 1))
    meth = getattr(P, "PPCA_" + method)
    prm = P.ppca_prime_params_default(meth)
    prm.batch = 500
    prm.lr = 0.05 if method == "EIGENGAME" else 1.0
    h = P.ppca_create(Xd)
    P.ppca_prime(h, meth, m, 4, prm, V0=V0)
    state = P.ppca_get_state(h)
    P.ppca_prime_continue(h, 5)
    Va = get_basis(P, h, d, m)
    h2 = P.ppca_create(Xd)
    P.ppca_set_state(h2, state)
    P.ppca_prime_continue(h2, 5)
    Vb = get_basis(P, h2, d, m)
    np.testing.assert_array_equal(Va, Vb)


def _trajectory_problem():
    n, d, m = 2000, 96, 8
    X, _ = synth.gaussian_data(n, d, 2.0 * 0.85 ** np.arange(1, d + 1), seed=6)
    return X, n, d, m


def test_oja_trajectory_parity(P):
    X, n, d, m = _trajectory_problem()
    Xd = dev_matrix(X, "f32")
    Xs = stored_f64(Xd)
    V0d = dev_basis(synth.initial_basis(d, m, 5))
    prm = P.ppca_prime_params_default(P.PPCA_OJA)
    prm.batch = 256
    prm.precision = P.PPCA_PREC_ACCURATE
    h = P.ppca_create(Xd)
    for steps in [1, 5]:
        P.ppca_prime(h, P.PPCA_OJA, m, steps, prm, V0=V0d)
        Vg = get_basis(P, h, d, m)
        Vo = oracle.oja_prime(Xs, host_basis(V0d), 256, steps, lambda t: 1.0 / (t + 100.0))
        assert np.abs(Vg - Vo).max() <= 1e-4 * max(1.0, np.abs(Vo).max())


def test_eigengame_trajectory_parity(P):
    X, n, d, m = _trajectory_problem()
    Xd = dev_matrix(X, "f32")
    Xs = stored_f64(Xd)
    V0d = dev_basis(synth.initial_basis(d, m, 5))
    prm = P.ppca_prime_params_default(P.PPCA_EIGENGAME)
    prm.batch = 500
    prm.lr = 0.02
    prm.precision = P.PPCA_PREC_ACCURATE
    h = P.ppca_create(Xd)
    for steps in [1, 5]:
        P.ppca_prime(h, P.PPCA_EIGENGAME, m, steps, prm, V0=V0d)
        Vg = get_basis(P, h, d, m)
        Vo = oracle.eigengame_prime(Xs, host_basis(V0d), 500, steps, 0.02, 0.9)
        assert np.abs(Vg - Vo).max() <= 1e-4


def test_eigengame_trajectory_parity_long_narrow_basis(P):
    """A 32768 x 16 basis: the Gram C = V^T Z is summed over 256 row slices
    (32 lanes per output in the reduction) and the column norms over 512
    blocks, the many-slice forms of both reductions.  Entries are ~1/sqrt(d),
    so the bound is relative to the largest; the renormalised columns have
    unit norm to FP32 rounding."""
    import torch
    n, d, m, b = 600, 32768, 16, 300
    X = synth.hadamard_rotated_data_torch(n, d, 2.0 * 0.9995 ** np.arange(1, d + 1), 9, "cpu",
                                          torch.float32)[0].numpy()
    Xd = dev_matrix(X, "f32")
    Xs = stored_f64(Xd)
    V0d = dev_basis(synth.initial_basis(d, m, 11))
    prm = P.ppca_prime_params_default(P.PPCA_EIGENGAME)
    prm.batch = b
    prm.lr = 0.02
    prm.precision = P.PPCA_PREC_ACCURATE
    h = P.ppca_create(Xd)
    for steps in [1, 3]:
        P.ppca_prime(h, P.PPCA_EIGENGAME, m, steps, prm, V0=V0d)
        Vg = get_basis(P, h, d, m)
        Vo = oracle.eigengame_prime(Xs, host_basis(V0d), b, steps, 0.02, 0.9)
        assert np.abs(Vg - Vo).max() <= 1e-4 * np.abs(Vo).max()
        assert np.abs(np.linalg.norm(Vg, axis=0) - 1.0).max() <= 1e-6


def test_host_side_errors(P, c1):
    import torch
    cfg, Xd, Xs, V0 = c1
    h = P.ppca_create(Xd)
    E = torch.empty((4, cfg.d), dtype=torch.float32, device="cuda")
    lam = torch.empty(4, dtype=torch.float64, device="cuda")
    with pytest.raises(P.PPCAError) as ei:
        P.ppca_finalize(h, 4, E, lam)
    assert ei.value.status_name == "PPCA_ERR_STATE"
    with pytest.raises(P.PPCAError) as ei:
        P.ppca_prime(h, P.PPCA_POWER, 129, 1)
    assert ei.value.status_name == "PPCA_ERR_INVALID"
    h2 = P.ppca_create(Xd)
    P.ppca_set_workspace_limit(h2, 1024)
    with pytest.raises(P.PPCAError) as ei:
        P.ppca_prime(h2, P.PPCA_POWER, 8, 1)
    assert ei.value.status_name == "PPCA_ERR_OOM"
    P.ppca_prime(h, P.PPCA_POWER, 8, 1)
    with pytest.raises(P.PPCAError) as ei:
        P.ppca_finalize(h, 9, E, lam)
    assert ei.value.status_name == "PPCA_ERR_INVALID"


def test_default_initial_basis_is_seeded(P, c1):
    cfg, Xd, Xs, V0 = c1
    prm = P.ppca_prime_params_default(P.PPCA_POWER)
    prm.seed = 77
    h = P.ppca_create(Xd)
    P.ppca_prime(h, P.PPCA_POWER, cfg.m, 0, prm)
    Va = get_basis(P, h, cfg.d, cfg.m)
    P.ppca_prime(h, P.PPCA_POWER, cfg.m, 0, prm)
    Vb = get_basis(P, h, cfg.d, cfg.m)
    np.testing.assert_array_equal(Va, Vb)
    assert np.abs(Va.T @ Va - np.eye(cfg.m)).max() <= 1e-5
    prm.seed = 78
    P.ppca_prime(h, P.PPCA_POWER, cfg.m, 0, prm)
    Vc = get_basis(P, h, cfg.d, cfg.m)
    assert oracle.principal_angles(Va, Vc).max() > 0.1
