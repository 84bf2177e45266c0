"""Three primers compared on the 1e5 x 1024 FP32 workload, against the oracle.

lambda_i = 1/i, k = l = 32, the same seeded data and V0 on both sides:
block power (T = 20), Oja/Sanger (minibatch 256, lr 1/(t+100), one epoch =
391 steps) and EigenGame (200 parallel steps, minibatch 1024, lr 0.1,
Nesterov 0.9), each followed by the pPCA step (Algorithm 1).  The GPU runs the
priming passes at their fast precision (3xTF32 for FP32 data) and the pPCA
step at split precision; the oracle runs each primer and the pPCA step in FP64
(oracle.power_prime / oja_prime / eigengame_prime, oracle.ppca_finalize).

Checked per primer, against the eigenvectors of X^T X (numpy's LAPACK eigh in
FP64 on the stored values, a library routine as test reference; the oracle's
Jacobi at d = 1024 takes minutes):
* the GPU's pPCA output has the oracle's streak at the workload's 1e-4 rad and
  at each V = pi/8 ... pi/1024 of the paper's grid (within one direction where
  the streak ends on a direction whose angle sits near V);
* its largest angle over the k directions is within 10 % of the oracle's (or
  both within the 1e-4 rad tolerance), and its eigenvalues agree with the
  oracle's pPCA eigenvalues to 1e-4 relative;
* block power meets the workload's tolerance outright: streak 32 at 1e-4 rad,
  eigenvalue relative error <= 1e-5.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

GRID = [math.pi / 2 ** j for j in range(3, 11)]


def test_three_primers_match_the_oracle(cuda_device):
    import torch

    import paper_2109_03709_gb300 as P
    P.load_library()
    cfg = synth.CONFIGS["primers_fp32_100000x1024"]
    n, d, k, m = cfg.n, cfg.d, cfg.k, cfg.m
    X, _ = synth.gaussian_data_torch(n, d, cfg.lam(), cfg.seed, "cuda", torch.float32)
    Xs = X.double().cpu().numpy()
    w, U = np.linalg.eigh(Xs.T @ Xs)
    w, U = w[::-1] / n, U[:, ::-1][:, :k].copy()
    V0 = synth.initial_basis(d, m, cfg.seed)
    V0d = torch.from_numpy(np.ascontiguousarray(V0.T, dtype=np.float32)).cuda()
    pw, oj, eg = cfg.primers["power"], cfg.primers["oja"], cfg.primers["eigengame"]
    oja_steps = oj["epochs"] * -(-n // oj["batch"])
    runs = {
        "power": (P.PPCA_POWER, pw["T"], {},
                  lambda: oracle.power_prime(Xs, V0, pw["T"])),
        "oja": (P.PPCA_OJA, oja_steps, {"batch": oj["batch"], "lr": oj["lr0"], "lr_offset": oj["lr_offset"]},
                lambda: oracle.oja_prime(Xs, V0, oj["batch"], oja_steps,
                                         lambda t: oj["lr0"] / (t + oj["lr_offset"]))),
        "eigengame": (P.PPCA_EIGENGAME, eg["steps"], {"batch": eg["batch"], "lr": eg["lr"], "momentum": eg["momentum"]},
                      lambda: oracle.eigengame_prime(Xs, V0, eg["batch"], eg["steps"], eg["lr"], eg["momentum"])),
    }
    report = {}
    for name, (method, T, kw, oracle_prime) in runs.items():
        h = P.ppca_create(X)
        prm = P.ppca_prime_params_default(method)
        for key, v in kw.items():
            setattr(prm, key, v)
        prm.precision = P.PPCA_PREC_FAST
        P.ppca_prime(h, method, m, T, prm, V0=V0d)
        E = torch.empty((k, d), dtype=torch.float32, device="cuda")
        lam = torch.empty(k, dtype=torch.float64, device="cuda")
        P.ppca_finalize(h, k, E, lam, P.PPCA_PREC_ACCURATE)
        P.ppca_sync(h)
        Eg, lg = E.double().cpu().numpy().T, lam.cpu().numpy()
        Eo, lo = oracle.ppca_finalize(Xs, oracle_prime(), k)
        ag, ao = oracle.angles(Eg, U), oracle.angles(Eo, U)
        report[name] = (oracle.lces(ag, cfg.angle_tol), oracle.lces(ao, cfg.angle_tol), ag.max(), ao.max())
        print(name, "gpu/oracle streak", report[name][:2], "max angle", report[name][2:],
              "grid", [(oracle.lces(ag, v), oracle.lces(ao, v)) for v in GRID])
        for tol in [cfg.angle_tol] + GRID:
            sg, so = oracle.lces(ag, tol), oracle.lces(ao, tol)
            near = so < k and abs(ao[so] - tol) <= 0.1 * tol
            assert sg == so or (near and abs(sg - so) <= 1), (name, tol, sg, so)
        assert abs(ag.max() - ao.max()) <= 0.1 * ao.max() or max(ag.max(), ao.max()) <= cfg.angle_tol, name
        np.testing.assert_allclose(lg, lo, rtol=1e-4, err_msg=name)
        if name == "power":
            assert oracle.lces(ag, cfg.angle_tol) == k
            assert np.max(np.abs(lg - w[:k]) / w[:k]) <= cfg.eig_rtol
