"""GPU parity of the ragged batch (many independent primed-PCA problems in one graph).

Each instance is block power priming (T iterations, fast 3xTF32 passes for
FP32 data) followed by the pPCA step (exact-FP32 pass), from a caller-supplied
V0.  Checks:
* deterministic parity of the pPCA step: each instance's E and lambda against
  the oracle's pPCA step fed the instance's own primed basis (V_out):
  eigenvalue relative error <= 1e-5, angles <= 1e-4 rad (FP32-path tolerances);
* the primed subspace against the oracle's FP64 block power from the same V0:
  principal angles <= 1e-2 rad.  The fast passes carry about 2e-5 relative
  error each (measured for 3xTF32 with long tensor-core accumulations); over
  T = 10 unconverged iterations this moves the subspace by well under 1e-2;
* a second launch of the captured graph reproduces the outputs bit for bit,
  and a problem gives the same bits in a batch as through a single handle.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import host_basis

pytestmark = pytest.mark.gpu


def make_batch(count, seed, T, nmax=20000, dtypes=None):
    import torch
    shapes = synth.batch_instances(count, seed)
    inst = []
    for i, s in enumerate(shapes):
        n = min(s["n"], nmax)
        d, k, m = s["d"], s["k"], s["m"]
        lam = s["rho"] ** np.arange(1, d + 1)
        dt = dtypes[i % len(dtypes)] if dtypes else torch.float32
        X = synth.instance_data_torch(n, d, lam, s["seed"], "cuda", dt)
        V0 = torch.from_numpy(np.ascontiguousarray(synth.initial_basis(d, m, s["seed"]).T,
                                                   dtype=np.float32)).cuda()
        inst.append({"X": X, "k": k, "m": m, "T": T, "V0": V0,
                     "E": torch.empty((k, d), dtype=torch.float32, device="cuda"),
                     "lam": torch.empty(k, dtype=torch.float64, device="cuda"),
                     "V_out": torch.empty((m, d), dtype=torch.float32, device="cuda")})
    return inst


def test_batch_matches_oracle(cuda_device):
    import torch

    import paper_2109_03709_gb300 as P
    inst = make_batch(12, seed=404, T=10)
    b = P.ppca_batch_create(inst, slots=4)
    assert P.ppca_batch_kernel_count(b) == 0          # the graph is captured by the first run
    P.ppca_batch_run(b)
    P.ppca_batch_sync(b)
    kernels = P.ppca_batch_kernel_count(b)
    assert kernels >= len(inst) * 10                  # at least one launch per power iteration
    for i, ins in enumerate(inst):
        Xs = ins["X"].double().cpu().numpy()
        Vg = host_basis(ins["V_out"])
        Eo, lo = oracle.ppca_finalize(Xs, Vg, ins["k"])
        E = host_basis(ins["E"])
        lam = ins["lam"].cpu().numpy()
        np.testing.assert_allclose(lam, lo, rtol=1e-5, err_msg=f"instance {i}")
        assert oracle.angles(E, Eo).max() <= 1e-4, i
        Vo = oracle.power_prime(Xs, host_basis(ins["V0"]), ins["T"])
        assert oracle.principal_angles(Vg, Vo).max() <= 1e-2, i
    before = [ins["E"].clone() for ins in inst]
    P.ppca_batch_run(b)
    P.ppca_batch_sync(b)
    for ins, e0 in zip(inst, before):
        assert torch.equal(ins["E"], e0)
    assert P.ppca_batch_kernel_count(b) == kernels    # replayed, not captured again


def test_batch_equals_single_handle(cuda_device):
    import torch

    import paper_2109_03709_gb300 as P
    inst = make_batch(5, seed=7, T=6, nmax=6000)
    b = P.ppca_batch_create(inst, slots=2)
    P.ppca_batch_run(b)
    P.ppca_batch_sync(b)
    for ins in inst:
        h = P.ppca_create(ins["X"])
        P.ppca_set_schedule(h, fused=0)
        prm = P.ppca_prime_params_default(P.PPCA_POWER)
        prm.precision = P.PPCA_PREC_FAST
        P.ppca_prime(h, P.PPCA_POWER, ins["m"], ins["T"], prm, V0=ins["V0"])
        E = torch.empty_like(ins["E"])
        lam = torch.empty_like(ins["lam"])
        P.ppca_finalize(h, ins["k"], E, lam, P.PPCA_PREC_ACCURATE)
        P.ppca_sync(h)
        assert torch.equal(E, ins["E"])
        assert torch.equal(lam, ins["lam"])


def test_batch_rejects_bad_descriptors(cuda_device):
    import torch

    import paper_2109_03709_gb300 as P
    X = torch.zeros((100, 32), device="cuda")
    bad = [{"X": X, "k": 5, "m": 4, "T": 1, "E": torch.empty((5, 32), device="cuda"),
            "lam": torch.empty(5, dtype=torch.float64, device="cuda")}]
    with pytest.raises(P.PPCAError) as ei:
        P.ppca_batch_create(bad)
    assert ei.value.status_name == "PPCA_ERR_INVALID"


def test_batch_autotuned_matches_oracle(cuda_device):
    """After ppca_batch_autotune (each (dtype, d, m, n-bucket) group runs the fastest
    measured engine), the pPCA step still equals the oracle's on the primed basis."""
    import paper_2109_03709_gb300 as P
    inst = make_batch(8, seed=23, T=8, nmax=12000)
    b = P.ppca_batch_create(inst, slots=3)
    groups = P.ppca_batch_autotune(b)
    assert 1 <= groups <= len(inst)
    P.ppca_batch_run(b)
    P.ppca_batch_sync(b)
    for i, ins in enumerate(inst):
        Xs = ins["X"].double().cpu().numpy()
        Vg = host_basis(ins["V_out"])
        Eo, lo = oracle.ppca_finalize(Xs, Vg, ins["k"])
        np.testing.assert_allclose(ins["lam"].cpu().numpy(), lo, rtol=1e-5, err_msg=f"instance {i}")
        assert oracle.angles(host_basis(ins["E"]), Eo).max() <= 1e-4, i
        Vo = oracle.power_prime(Xs, host_basis(ins["V0"]), ins["T"])
        assert oracle.principal_angles(Vg, Vo).max() <= 1e-2, i
    with pytest.raises(P.PPCAError) as ei:
        P.ppca_batch_autotune(b)                      # already captured
    assert ei.value.status_name == "PPCA_ERR_STATE"


def test_batch_bf16_priming_matches_oracle(cuda_device):
    """ppca_batch_set_priming(PPCA_BF16): each run rounds every FP32 instance to
    BF16 (bit-exact round to nearest even), primes on that rounding with the
    BF16 fast passes, and runs the pPCA step on the FP32 data.  The pPCA step
    still equals the oracle's on the primed basis (FP32 tolerances), and the
    primed subspace follows the oracle's FP64 block power on the BF16-rounded
    data: each fast pass rounds V and Y to BF16 (2^-8 relative), which over
    T = 10 unconverged iterations moves the subspace by a few 1e-3 rad (bound 3e-2)."""
    import paper_2109_03709_gb300 as P
    inst = make_batch(10, seed=505, T=10)
    b = P.ppca_batch_create(inst, slots=3)
    P.ppca_batch_set_priming(b, P.PPCA_BF16)
    P.ppca_batch_run(b)
    P.ppca_batch_sync(b)
    assert P.ppca_batch_lockstep(b)                   # all FP32, d % 8 == 0, one T: primed in lockstep
    worst = 0.0
    for i, ins in enumerate(inst):
        Xs = ins["X"].double().cpu().numpy()
        Vg = host_basis(ins["V_out"])
        Eo, lo = oracle.ppca_finalize(Xs, Vg, ins["k"])
        np.testing.assert_allclose(ins["lam"].cpu().numpy(), lo, rtol=1e-5, err_msg=f"instance {i}")
        assert oracle.angles(host_basis(ins["E"]), Eo).max() <= 1e-4, i
        Vo = oracle.power_prime(oracle.bf16_round_rne(Xs), host_basis(ins["V0"]), ins["T"])
        worst = max(worst, oracle.principal_angles(Vg, Vo).max())
    print("bf16-primed batch: largest principal angle to the oracle's power iterate", worst)
    assert worst <= 3e-2
    with pytest.raises(P.PPCAError) as ei:
        P.ppca_batch_set_priming(b, P.PPCA_F32)       # already captured
    assert ei.value.status_name == "PPCA_ERR_STATE"


def test_lockstep_priming_against_slots_and_oracle(cuda_device):
    """Lockstep batch (every instance's power iterations and pPCA step in
    grouped launches: one launch per kernel kind and iteration) on a mixed batch: FP32 instances primed on their BF16 rounding, BF16
    instances primed as stored, ragged n (not multiples of 128) and m (not
    multiples of 32), one instance drawing its V0 from its seed.  Against the
    same batch primed on its slots (the per-instance path): the same pPCA-step
    parity with the oracle on each primed basis, primed subspaces within
    3e-2 rad of the oracle's FP64 block power on the stored (BF16 or
    BF16-rounded) values, and far fewer kernel launches."""
    import torch

    import paper_2109_03709_gb300 as P
    T = 6
    runs = {}
    for lockstep in (True, False):
        inst = make_batch(9, seed=611, T=T, nmax=9000, dtypes=[torch.float32, torch.bfloat16, torch.float32])
        inst[4]["V0"] = None
        inst[4]["seed"] = 99
        b = P.ppca_batch_create(inst, slots=3)
        P.ppca_batch_set_priming(b, P.PPCA_BF16)
        P.ppca_batch_set_lockstep(b, lockstep)
        P.ppca_batch_run(b)
        P.ppca_batch_sync(b)
        assert P.ppca_batch_lockstep(b) == lockstep
        runs[lockstep] = (inst, P.ppca_batch_kernel_count(b))
    (inst_l, k_l), (inst_s, k_s) = runs[True], runs[False]
    print("kernels per run: lockstep", k_l, "slots", k_s)
    assert k_l <= 40 + 13 * T < k_s                   # independent of the instance count
    for i, (a, c) in enumerate(zip(inst_l, inst_s)):
        Xs = a["X"].double().cpu().numpy()            # stored values (BF16 instances exactly)
        Xp = oracle.bf16_round_rne(Xs)                # the priming data of both paths
        Va, Vc = host_basis(a["V_out"]), host_basis(c["V_out"])
        Eo, lo = oracle.ppca_finalize(Xs, Va, a["k"])
        np.testing.assert_allclose(a["lam"].cpu().numpy(), lo, rtol=1e-5, err_msg=f"instance {i}")
        assert oracle.angles(host_basis(a["E"]), Eo).max() <= 1e-4, i
        if a["V0"] is not None:
            Vo = oracle.power_prime(Xp, host_basis(a["V0"]), T)
            assert oracle.principal_angles(Va, Vo).max() <= 3e-2, i
        # the slot path from the same start (the seeded instance: the same Philox draw)
        assert oracle.principal_angles(Va, Vc).max() <= 3e-2, i


def test_lockstep_full_size_subset_matches_oracle(cuda_device):
    """16 instances of the 512-instance workload at full size (the first 16 that
    its generator draws: n up to 185952, d from 64 to 2048), FP32 data primed in
    lockstep on the BF16 rounding with the workload's T = 10: each instance's E
    and lambda against the oracle's pPCA step (Algorithm 1, steps 2-5, FP64) on
    the instance's own primed basis V_out (eigenvalues 1e-5 relative, angles
    1e-4 rad); for four of them also the primed subspace against the oracle's
    FP64 block power on the BF16-rounded data (3e-2 rad, as above); and the run
    takes the same 40 + 13T launches whatever the instance count."""
    import torch

    import paper_2109_03709_gb300 as P
    cfg = synth.CONFIGS["batch512_fp32"]
    T = cfg.primers["power"]["T"]
    shapes = synth.batch_instances(512, cfg.seed)[:16]
    inst = []
    for s in shapes:
        n, d, k, m = s["n"], s["d"], s["k"], s["m"]
        X = synth.instance_data_torch(n, d, s["rho"] ** np.arange(1, d + 1), s["seed"], "cuda", torch.float32)
        V0 = torch.from_numpy(np.ascontiguousarray(synth.initial_basis(d, m, s["seed"]).T, dtype=np.float32)).cuda()
        inst.append({"X": X, "k": k, "m": m, "T": T, "V0": V0,
                     "E": torch.empty((k, d), dtype=torch.float32, device="cuda"),
                     "lam": torch.empty(k, dtype=torch.float64, device="cuda"),
                     "V_out": torch.empty((m, d), dtype=torch.float32, device="cuda")})
    b = P.ppca_batch_create(inst, slots=4)
    P.ppca_batch_set_priming(b, P.PPCA_BF16)
    P.ppca_batch_run(b)
    P.ppca_batch_sync(b)
    assert P.ppca_batch_lockstep(b)
    assert P.ppca_batch_kernel_count(b) <= 40 + 13 * T
    for i, ins in enumerate(inst):
        Xs = ins["X"].double().cpu().numpy()
        Vg = host_basis(ins["V_out"])
        Eo, lo = oracle.ppca_finalize(Xs, Vg, ins["k"])
        np.testing.assert_allclose(ins["lam"].cpu().numpy(), lo, rtol=1e-5, err_msg=f"instance {i}")
        assert oracle.angles(host_basis(ins["E"]), Eo).max() <= 1e-4, i
        if i < 4:
            Vo = oracle.power_prime(oracle.bf16_round_rne(Xs), host_basis(ins["V0"]), T)
            assert oracle.principal_angles(Vg, Vo).max() <= 3e-2, i
        del Xs


def test_lockstep_ill_conditioned_start(cuda_device):
    """A starting basis with condition number 1e3 (kappa of its Gram matrix 1e6,
    past the FP32 factor's acceptance bound 2^16) makes CholeskyQR's FP32 factor
    fail its conditioning test, so the grouped factor kernel redoes it in
    double-float in the same block.  With T = 0 the lockstep output is orth(V0):
    orthonormal to 1e-5 and spanning the oracle's orthonormalisation of V0 to
    5e-4 rad (Q = V R^-1 applied in FP32 perturbs the span by about
    kappa(V) u = 6e-5 per column); the pPCA step on it matches the oracle's."""
    import torch

    import paper_2109_03709_gb300 as P
    for T, bound in ((0, 5e-4),):
        inst = make_batch(3, seed=733, T=T, nmax=8000, dtypes=[torch.bfloat16])
        V0 = host_basis(inst[1]["V0"])
        U, _, Wt = np.linalg.svd(V0, full_matrices=False)
        sv = np.logspace(0, -3, V0.shape[1])                 # kappa(V0) = 1e3
        inst[1]["V0"] = torch.from_numpy(np.ascontiguousarray(((U * sv) @ Wt).T, dtype=np.float32)).cuda()
        b = P.ppca_batch_create(inst, slots=2)
        P.ppca_batch_run(b)
        P.ppca_batch_sync(b)
        assert P.ppca_batch_lockstep(b)
        for i, a in enumerate(inst):
            Xs = a["X"].double().cpu().numpy()
            Va = host_basis(a["V_out"])
            Vo = oracle.power_prime(Xs, host_basis(a["V0"]), T) if T else oracle.orth(host_basis(a["V0"]))
            assert oracle.principal_angles(Va, Vo).max() <= bound, (T, i)
            if T == 0:
                assert np.abs(Va.T @ Va - np.eye(Va.shape[1])).max() <= 1e-5, i
            # the pPCA step's eigenvalues: relative 1e-5, or for the small ones of an
            # unprimed (T = 0) basis the projected Gram's bound, 4e-6 of its largest
            Eo, lo = oracle.ppca_finalize(Xs, Va, a["k"])
            np.testing.assert_allclose(a["lam"].cpu().numpy(), lo, rtol=1e-5, atol=4e-6 * lo.max(),
                                       err_msg=f"instance {i}")
