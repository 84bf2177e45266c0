"""The element-wise X-pass criterion (tests/xpass_parity.py) on the CPU.

The GPU parity tests accept a pass when max_jc |dZ_jc| / (tau_r R_jc +
tau_z |Z_jc|) <= 1.  Here an emulation of the FAST BF16 pass -- Y accumulated
in FP32 over 64-column K-stages (a summation order unlike the FP64
reference's), rounded to BF16, Z accumulated in FP32 one 128-row tile at a
time -- must pass with a margin, and the same emulation with one planted
mistake must fail: a dropped row tile, a missing last row, a skipped K-stage
of Y, Y rounded toward zero instead of to nearest, a column pair of V swapped.
The ACCURATE criterion gets the same treatment with an FP32 emulation of the
split-precision pass.
"""
import numpy as np
import pytest

import oracle
import synth
from xpass_parity import TAU_FAST_R, exact_reference, fast_reference, ratio, split_ratio

TAU_Z_FAST = 5e-4


def _bf16_trunc(x):
    """BF16 by truncation toward zero (a planted rounding mistake)."""
    f = np.asarray(x, dtype=np.float32)
    bits = f.view(np.uint32) & np.uint32(0xFFFF0000)
    return bits.view(np.float32).astype(np.float64)


def emulate_fast(Xs, V32, *, drop_tile=None, drop_last_row=False, skip_stage=None, trunc=False, swap=None):
    X32 = Xs.astype(np.float32)
    Vh = oracle.bf16_round_rne(V32).astype(np.float32)
    if swap is not None:
        a, b = swap
        Vh[:, [a, b]] = Vh[:, [b, a]]
    n, d = X32.shape
    Y = np.zeros((n, Vh.shape[1]), dtype=np.float32)
    for k0 in range(0, d, 64):
        if skip_stage is not None and k0 // 64 == skip_stage:
            continue
        Y = Y + X32[:, k0:k0 + 64] @ Vh[k0:k0 + 64]
    Yh = _bf16_trunc(Y) if trunc else oracle.bf16_round_rne(Y)
    Z = np.zeros((d, Vh.shape[1]), dtype=np.float32)
    last = n - 1 if drop_last_row else n
    for t, r0 in enumerate(range(0, n, 128)):
        if drop_tile is not None and t == drop_tile:
            continue
        r1 = min(r0 + 128, last)
        if r1 > r0:
            Z = Z + (Xs[r0:r1].T @ Yh[r0:r1]).astype(np.float32)
    return Z.astype(np.float64)


def problem(n, d, m, seed):
    X, _ = synth.gaussian_data(n, d, 0.97 ** np.arange(1, d + 1), seed=seed)
    Xs = oracle.bf16_round_rne(X)                        # stored BF16 values
    V32 = synth.initial_basis(d, m, seed=seed + 1).astype(np.float32)
    return Xs, V32


SHAPES = [(5000, 512, 64, 1), (3001, 200, 33, 2), (20000, 256, 16, 3)]


@pytest.mark.parametrize("n,d,m,seed", SHAPES)
def test_fast_emulation_passes_with_margin(n, d, m, seed):
    Xs, V32 = problem(n, d, m, seed)
    Zref, R = fast_reference(Xs, V32)
    assert ratio(emulate_fast(Xs, V32), Zref, R, TAU_FAST_R, TAU_Z_FAST) <= 0.5


PLANTED = {
    "dropped row tile": dict(drop_tile=3),
    "missing last row": dict(drop_last_row=True),
    "skipped K-stage of Y": dict(skip_stage=1),
    "Y truncated, not rounded": dict(trunc=True),
    "columns of V swapped": dict(swap=(0, 1)),
}


@pytest.mark.parametrize("n,d,m,seed", SHAPES)
@pytest.mark.parametrize("name", sorted(PLANTED))
def test_fast_planted_mistakes_fail(n, d, m, seed, name):
    Xs, V32 = problem(n, d, m, seed)
    Zref, R = fast_reference(Xs, V32)
    assert ratio(emulate_fast(Xs, V32, **PLANTED[name]), Zref, R, TAU_FAST_R, TAU_Z_FAST) > 1.0


TAU_ACC = (2.0 ** -18, 2e-5)


def emulate_accurate(Xs, V32, *, drop_tile=None):
    """Split-precision pass: exact pieces, Y in FP32 per 64-wide K-stage, Z in FP32 per tile."""
    V = V32.astype(np.float64)
    n, d = Xs.shape
    Y = np.zeros((n, V.shape[1]), dtype=np.float32)
    for k0 in range(0, d, 64):
        Y = (Y + Xs[:, k0:k0 + 64] @ V[k0:k0 + 64]).astype(np.float32)
    Z = np.zeros((d, V.shape[1]), dtype=np.float64)
    for t, r0 in enumerate(range(0, n, 128)):
        if t != drop_tile:
            Z = Z + (Xs[r0:r0 + 128].T @ Y[r0:r0 + 128].astype(np.float64)).astype(np.float32)
    return Z


@pytest.mark.parametrize("n,d,m,seed", SHAPES)
def test_accurate_emulation_passes_and_dropped_tile_fails(n, d, m, seed):
    Xs, V32 = problem(n, d, m, seed)
    Zref, R = exact_reference(Xs, V32)
    assert ratio(emulate_accurate(Xs, V32), Zref, R, *TAU_ACC) <= 0.5
    assert ratio(emulate_accurate(Xs, V32, drop_tile=2), Zref, R, *TAU_ACC) > 1.0


@pytest.mark.parametrize("n,d,m,seed", SHAPES)
def test_split_criterion_accepts_emulation_and_rejects_dropped_tile(n, d, m, seed):
    Xs, V32 = problem(n, d, m, seed)
    tau = (2 * 2e-8 * 3 * -(-d // 16) + 2.0 ** -22, 2 * 2e-8 * 384 + 2.0 ** -22)
    assert split_ratio(emulate_accurate(Xs, V32), Xs, V32, *tau) <= 0.5
    assert split_ratio(emulate_accurate(Xs, V32, drop_tile=2), Xs, V32, *tau) > 1.0
