"""GPU parity of the individual steps, through the C ABI, against the FP64 oracle.

Tolerances (derived from the arithmetic; u = 2^-24):
* X-passes are checked element by element with the criterion of
  tests/xpass_parity.py: |dZ_jc| <= tau_r R_jc + tau_z |Z_jc|, R_jc the
  root-sum-square scale of the terms of Z_jc.  FAST passes of BF16 / FP8 data
  are compared with the same pass formed exactly in FP64 from BF16-rounded V
  and Y (tau_r = 2^-7 for one-unit flips of Y's rounding, tau_z for
  the FP32 accumulation drift); split-precision and FP32 passes with
  X^T X V itself (split precision: the drift of Y's and Z's accumulators
  relative to their running sums, split_ratio).  The normwise errors of the
  earlier bounds are kept as a second check.
* X-pass, FP32 data, ACCURATE (exact FP32 on CUDA cores): FP32 products,
  FP32 chunks of <= 256 terms folded into double-float sums: normwise
  ||dZ|| / ||Z|| <= 2e-5 (about u * (sqrt(d) + 16) with a safety factor ~3).
* X-pass, BF16 data, FAST: V and Y rounded to BF16 (2^-8 relative), so 1e-2
  normwise.
* CholeskyQR2 vs the oracle's MGS2 (both the unique thin-QR factor with a
  positive diagonal): entrywise <= 1e-5 for kappa(V) ~ 10 (about kappa * u * m).
* eigensolver: eigenvalues are FP64 Rayleigh quotients of FP32 Jacobi vectors,
  relative error <= 1e-9; vectors <= 2e-5 rad for relative gaps >= 1%.
* quantisers: bit-exact.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev_basis, dev_matrix, empty_basis, host_basis, normwise, stored_f64
from xpass_parity import TAU_FAST_R, exact_reference, fast_e4m3_reference, fast_reference, ratio, split_ratio

pytestmark = pytest.mark.gpu

# element-wise tolerances (tau_r, tau_z) per pass kind, see tests/xpass_parity.py:
# FAST BF16 / FP8 against the BF16-rounded exact pass: one-unit flips of Y
# (2^-7 R) and up to 16384 accumulating MMAs between folds (fused pass,
# ~2e-8 each: 3.3e-4 -> 5e-4); split precision (three BF16 pieces; Y's
# accumulator takes 3 d / 16 MMAs unfolded and the two-kernel pass folds its Z
# accumulator every 32 K-stages = 384 MMAs, drift ~2e-8 per MMA, x2 margin ->
# tau_z(d); Y's FP32 rounding 2^-24 of the terms, summed over d -> 2^-18 R);
# 3xTF32 (dropped lo*lo products ~2^-22 of each term, accumulation over d and
# n unfolded: 2^-16 R, 5e-5 |Z|); exact FP32 on CUDA cores (FP32 products,
# 256-term chunks folded: 2^-19 R, 1e-6 |Z|).
TAU_FAST = (TAU_FAST_R, 5e-4)


def tau_split(d):
    """(tau_y, tau_z) of split_ratio for the two-kernel split-precision pass: Y's
    accumulator takes 3 ceil(d / 16) MMAs (three pieces, K = 16) unfolded, Z's is
    folded every 32 K-stages of 64 rows (384 MMAs); ~2e-8 drift per MMA, x2, plus
    the FP32 roundings (2^-22)."""
    return (2 * 2e-8 * 3 * -(-d // 16) + 2.0 ** -22, 2 * 2e-8 * 384 + 2.0 ** -22)



TAU_3XTF32 = (2.0 ** -16, 5e-5)
TAU_F32_EXACT = (2.0 ** -19, 1e-6)


@pytest.fixture(scope="module")
def P(cuda_device):
    import paper_2109_03709_gb300 as P
    P.load_library()
    return P


XPASS_CASES = [
    # n, d, m, r0, r1, ld
    (1000, 64, 16, 0, 1000, None),
    (4099, 200, 64, 3, 4099, None),
    (777, 256, 128, 100, 612, None),
    (50, 16, 1, 0, 1, None),
    (300, 37, 5, 0, 300, 40),           # padded leading dimension, ragged d
    (2050, 1024, 33, 1, 2050, None),    # ragged m
]


@pytest.mark.parametrize("n,d,m,r0,r1,ld", XPASS_CASES)
def test_xpass_fp32(P, n, d, m, r0, r1, ld):
    lam = 0.95 ** np.arange(1, d + 1)
    X, _ = synth.gaussian_data(n, d, lam, seed=n + d)
    Xd = dev_matrix(X, "f32", ld)
    V = synth.initial_basis(d, m, seed=m)
    Vd = dev_basis(V)
    Zd = empty_basis(d, m)
    h = P.ppca_create(Xd)
    P.ppca_xpass(h, Vd, m, r0, r1, Zd, P.PPCA_PREC_ACCURATE)
    P.ppca_sync(h)
    Xs = stored_f64(Xd)[r0:r1]
    Vs = host_basis(Vd)
    Zref = Xs.T @ (Xs @ Vs)
    assert normwise(host_basis(Zd), Zref) <= 2e-5
    Ze, R = exact_reference(Xs, Vs)
    assert ratio(host_basis(Zd), Ze, R, *TAU_F32_EXACT) <= 1.0


@pytest.mark.parametrize("n,d,m,r0,r1,ld", XPASS_CASES)
def test_xpass_fp32_tensor_core_3xtf32(P, n, d, m, r0, r1, ld):
    """FAST pass for FP32 data: 3xTF32 on tensor cores.  Each operand is split
    into a TF32 head and an FP32 residual (products exact to ~2^-21); the
    tensor-core FP32 accumulation over long K adds up to ~2e-5 relative
    (measured at K = 2048), hence 5e-5 normwise."""
    lam = 0.95 ** np.arange(1, d + 1)
    X, _ = synth.gaussian_data(n, d, lam, seed=n + d)
    Xd = dev_matrix(X, "f32", ld)
    Vd = dev_basis(synth.initial_basis(d, m, seed=m))
    Zd = empty_basis(d, m)
    h = P.ppca_create(Xd)
    P.ppca_xpass(h, Vd, m, r0, r1, Zd, P.PPCA_PREC_FAST)
    P.ppca_sync(h)
    Xs = stored_f64(Xd)[r0:r1]
    Zref = Xs.T @ (Xs @ host_basis(Vd))
    assert normwise(host_basis(Zd), Zref) <= 5e-5
    Ze, R = exact_reference(Xs, host_basis(Vd))
    assert ratio(host_basis(Zd), Ze, R, *TAU_3XTF32) <= 1.0


def test_cuda_core_engine_on_bf16_data(P):
    """engine = 2 runs the exact-FP32 CUDA-core pass even for BF16 data: FP32
    products of the stored values, so the FP32 tolerance (2e-5) holds at FAST."""
    n, d, m = 3000, 384, 40
    X, _ = synth.gaussian_data(n, d, 0.97 ** np.arange(1, d + 1), seed=12)
    Xd = dev_matrix(X, "bf16")
    Vd = dev_basis(synth.initial_basis(d, m, seed=5))
    Zd = empty_basis(d, m)
    h = P.ppca_create(Xd)
    P.ppca_set_schedule(h, engine=2)
    P.ppca_xpass(h, Vd, m, 0, n, Zd, P.PPCA_PREC_FAST)
    P.ppca_sync(h)
    Xs = stored_f64(Xd)
    assert normwise(host_basis(Zd), Xs.T @ (Xs @ host_basis(Vd))) <= 2e-5
    Ze, R = exact_reference(Xs, host_basis(Vd))
    assert ratio(host_basis(Zd), Ze, R, *TAU_F32_EXACT) <= 1.0


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
def test_autotune_picks_a_valid_schedule(P, dtype):
    n, d, m = 20000, 1024, 64
    X, _ = synth.gaussian_data(n, d, 0.97 ** np.arange(1, d + 1), seed=13)
    Xd = dev_matrix(X, dtype)
    h = P.ppca_create(Xd)
    best = P.ppca_autotune(h, m, reps=2)
    assert best.engine in (1, 2)
    assert best.fused in (-1, 0, 1)
    if dtype == "f32":
        assert best.fused != 1
    Vd = dev_basis(synth.initial_basis(d, m, seed=6))
    Zd = empty_basis(d, m)
    P.ppca_xpass(h, Vd, m, 0, n, Zd, P.PPCA_PREC_FAST)
    P.ppca_sync(h)
    Xs = stored_f64(Xd)
    assert normwise(host_basis(Zd), Xs.T @ (Xs @ host_basis(Vd))) <= 1e-2


BF16_CASES = [
    # n, d, m, r0, r1
    (3001, 512, 64, 0, 3001),
    (1000, 200, 33, 17, 931),        # ragged d (not a multiple of 64), ragged m and rows
    (257, 64, 1, 0, 257),
    (5000, 1024, 128, 0, 5000),
    (600000, 64, 16, 0, 600000),     # many tiles per CTA, several flush blocks per row group
    (4096, 4096, 128, 0, 4096),
    (1000, 8192, 64, 0, 512),        # few row tiles, long K: split-K Y = X V
    (700, 20000, 32, 3, 300),        # split-K with ragged rows and a ragged last K-stage
]


@pytest.mark.parametrize("n,d,m,r0,r1", BF16_CASES)
@pytest.mark.parametrize("prec,tol", [("FAST", 1e-2), ("ACCURATE", 2e-5)])
def test_xpass_bf16(P, n, d, m, r0, r1, prec, tol):
    # a Haar rotation costs O(d^3) on the host: wide or very tall cases use axis-aligned data
    X, _ = synth.gaussian_data(n, d, 0.97 ** np.arange(1, d + 1), seed=9) if n * d <= 5e7 and d <= 4096 else \
        (np.random.default_rng(9).standard_normal((n, d)) * (0.9995 ** np.arange(1, d + 1))[None, :], None)
    Xd = dev_matrix(X, "bf16")
    V = synth.initial_basis(d, m, seed=3)
    Vd = dev_basis(V)
    Zd = empty_basis(d, m)
    h = P.ppca_create(Xd)
    P.ppca_xpass(h, Vd, m, r0, r1, Zd, getattr(P, "PPCA_PREC_" + prec))
    P.ppca_sync(h)
    Xs = stored_f64(Xd)[r0:r1]
    Zref = Xs.T @ (Xs @ host_basis(Vd))
    assert normwise(host_basis(Zd), Zref) <= tol
    # element by element: FAST against the BF16-rounded exact pass, ACCURATE against X^T X V
    Zg = host_basis(Zd)
    if prec == "FAST":
        Zq, R = fast_reference(Xs, host_basis(Vd))
        assert ratio(Zg, Zq, R, *TAU_FAST) <= 1.0
    else:
        assert split_ratio(Zg, Xs, host_basis(Vd), *tau_split(d)) <= 1.0


FUSED_CASES = [
    # n, d, m, r0, r1, producers, window
    (3001, 512, 64, 0, 3001, 0, 0),
    (5000, 1024, 128, 0, 5000, 0, 0),
    (600000, 64, 16, 0, 600000, 0, 0),      # d = 64: one slice, 152 row groups
    (4096, 4096, 128, 0, 4096, 0, 0),       # 32 slices x 4 row groups, one tile each
    (70000, 2048, 96, 5, 69000, 13, 5),     # few producers, short window: throttling
    (9000, 200, 33, 100, 8999, 3, 1),
]


@pytest.mark.parametrize("kparts", [1, 2])
@pytest.mark.parametrize("n,d,m,r0,r1,producers,window", FUSED_CASES)
def test_xpass_bf16_fused_single_read(P, n, d, m, r0, r1, producers, window, kparts):
    X = np.random.default_rng(n + d).standard_normal((n, d)) * (0.97 ** np.arange(1, d + 1))[None, :] ** 0.5
    Xd = dev_matrix(X, "bf16")
    V = synth.initial_basis(d, m, seed=4)
    Vd = dev_basis(V)
    Zf, Zu = empty_basis(d, m), empty_basis(d, m)
    h = P.ppca_create(Xd)
    P.ppca_set_schedule(h, fused=1, producers=producers, window=window, kparts=kparts)
    P.ppca_xpass(h, Vd, m, r0, r1, Zf, P.PPCA_PREC_FAST)
    P.ppca_sync(h)
    Zf2 = empty_basis(d, m)
    P.ppca_xpass(h, Vd, m, r0, r1, Zf2, P.PPCA_PREC_FAST)
    P.ppca_sync(h)
    assert np.array_equal(host_basis(Zf), host_basis(Zf2))   # run to run: bitwise
    P.ppca_set_schedule(h, fused=0)
    P.ppca_xpass(h, Vd, m, r0, r1, Zu, P.PPCA_PREC_FAST)
    P.ppca_sync(h)
    Xs = stored_f64(Xd)[r0:r1]
    Zref = Xs.T @ (Xs @ host_basis(Vd))
    Zg = host_basis(Zf)
    assert normwise(Zg, Zref) <= 1e-2
    Zq, R = fast_reference(Xs, host_basis(Vd))
    assert ratio(Zg, Zq, R, *TAU_FAST) <= 1.0
    # the two-kernel pass rounds the same Y to BF16, except where it splits K over
    # CTAs (few row tiles), or the fused pass sums two K halves (kparts = 2): there a
    # summation-order difference can move a Y element to the neighbouring BF16 value
    # (2^-8 relative); such elements move Z by ~1e-5 (split K) to ~5e-5 (two halves)
    assert normwise(Zg, host_basis(Zu)) <= (1e-4 if kparts == 1 else 2e-4)


@pytest.mark.parametrize("flush", [8, 64])
def test_xpass_bf16_fused_several_folds_at_d4096(P, flush):
    """The fused pass at d = 4096 with its consumers' TMEM sums folded into
    the double-float partials every flush / 2 row tiles (4 and 32 tiles: 16
    slice pairs x 9 row groups over 157 tiles, so each consumer folds several
    times, or once), element by element against the BF16-rounded exact pass."""
    n, d, m = 20000, 4096, 128
    X = np.random.default_rng(17).standard_normal((n, d)) * (0.999 ** np.arange(1, d + 1))[None, :]
    Xd = dev_matrix(X, "bf16")
    Vd = dev_basis(synth.initial_basis(d, m, seed=5))
    Zd = empty_basis(d, m)
    h = P.ppca_create(Xd)
    P.ppca_set_schedule(h, fused=1, flush=flush)
    P.ppca_xpass(h, Vd, m, 0, n, Zd, P.PPCA_PREC_FAST)
    P.ppca_sync(h)
    Xs = stored_f64(Xd)
    Zq, R = fast_reference(Xs, host_basis(Vd))
    assert ratio(host_basis(Zd), Zq, R, *TAU_FAST) <= 1.0


@pytest.mark.parametrize("d,m", [(64, 1), (256, 16), (1000, 64), (300, 33), (2000, 100), (4096, 128)])
def test_cholesky_qr2_matches_thin_qr(P, d, m):
    V = synth.initial_basis(d, m, seed=d)
    Vd = dev_basis(V)
    Qd = empty_basis(d, m)
    Xd = dev_matrix(np.zeros((2, d)), "f32", ld=(d + 3) // 4 * 4)
    h = P.ppca_create(Xd)
    P.ppca_orthonormalize(h, Vd, Qd, m)
    P.ppca_sync(h)
    Q = host_basis(Qd)
    Qref = oracle.orth(host_basis(Vd))
    assert np.abs(Q - Qref).max() <= 1e-5
    assert np.abs(Q.T @ Q - np.eye(m)).max() <= 1e-5


@pytest.mark.parametrize("kappa", [10.0, 1e3, 1e5])
def test_cholesky_qr2_tall_basis_tensor_core_gram(P, kappa):
    """d >= 16384: the Gram matrices come from the tensor cores (three BF16
    pieces); at kappa = 1e5 the FP32 factorisation is rejected and the
    double-float fallback recomputes its Gram in double-float."""
    d, m = 20000, 48
    rng = np.random.default_rng(int(kappa))
    U, _ = np.linalg.qr(rng.standard_normal((d, m)))
    W, _ = np.linalg.qr(rng.standard_normal((m, m)))
    V = (U * np.logspace(0, -np.log10(kappa), m)[None, :]) @ W.T
    Vd = dev_basis(V)
    Qd = empty_basis(d, m)
    h = P.ppca_create(dev_matrix(np.zeros((2, d)), "f32"))
    P.ppca_orthonormalize(h, Vd, Qd, m)
    P.ppca_sync(h)
    Q = host_basis(Qd)
    assert np.abs(Q.T @ Q - np.eye(m)).max() <= 1e-5
    assert oracle.principal_angles(Q, host_basis(Vd)).max() <= kappa * 1e-7 + 1e-5
    if kappa <= 1e3:
        assert np.abs(Q - oracle.orth(host_basis(Vd))).max() <= kappa * 1e-6


def test_cholesky_qr2_ill_conditioned(P):
    d, m = 512, 32
    rng = np.random.default_rng(1)
    U, _ = np.linalg.qr(rng.standard_normal((d, m)))
    W, _ = np.linalg.qr(rng.standard_normal((m, m)))
    V = (U * np.logspace(0, -5, m)[None, :]) @ W.T          # kappa = 1e5
    Vd = dev_basis(V)
    Qd = empty_basis(d, m)
    h = P.ppca_create(dev_matrix(np.zeros((2, d)), "f32"))
    P.ppca_orthonormalize(h, Vd, Qd, m)
    P.ppca_sync(h)
    Q = host_basis(Qd)
    assert np.abs(Q.T @ Q - np.eye(m)).max() <= 1e-5
    # span preserved: principal angles between span(Q) and span(V) small
    assert oracle.principal_angles(Q, host_basis(Vd)).max() < 1e-2


@pytest.mark.parametrize("kappa", [1.0, 30.0, 300.0, 3e3, 3e4, 1e6])
def test_cholesky_qr2_conditioning_sweep(P, kappa):
    """Across the switch between the FP32 first pass (accepted while the bound
    on kappa(V D)^2 stays below 2^16) and its double-float fallback: Q is
    orthonormal to 1e-5 and spans span(V) to kappa * 1e-7; for kappa <= 3e4 it equals the
    unique thin-QR factor of the oracle to kappa * 1e-7 (FP32 input V carries
    relative rounding 6e-8, amplified by kappa in R)."""
    d, m = 2048, 128
    rng = np.random.default_rng(int(kappa))
    U, _ = np.linalg.qr(rng.standard_normal((d, m)))
    W, _ = np.linalg.qr(rng.standard_normal((m, m)))
    s = np.logspace(0, -np.log10(kappa), m)
    V = (U * s[None, :]) @ W.T
    V = V * rng.uniform(0.1, 10.0, m)[None, :]               # column scales the diagonal scaling removes
    Vd = dev_basis(V)
    Qd = empty_basis(d, m)
    h = P.ppca_create(dev_matrix(np.zeros((2, d)), "f32"))
    P.ppca_orthonormalize(h, Vd, Qd, m)
    P.ppca_sync(h)
    Q = host_basis(Qd)
    assert np.abs(Q.T @ Q - np.eye(m)).max() <= 1e-5
    # span(V) itself is only defined to ~kappa u by the FP32 input and arithmetic
    assert oracle.principal_angles(Q, host_basis(Vd)).max() < 1e-5 + kappa * 1e-7
    if kappa <= 3e4:
        assert np.abs(Q - oracle.orth(host_basis(Vd))).max() <= max(1e-5, kappa * 1e-7)


def test_cholesky_breakdown_is_reported(P):
    """A zero column makes a pivot exactly zero in every precision.  (An exactly
    repeated column leaves a pivot at the rounding level of the double-float
    factorisation, ~1e-14 of the diagonal, which may land on either side of the
    1e-15 * trace(G) floor, so it is not a deterministic case.)"""
    d, m = 128, 8
    V = synth.initial_basis(d, m, seed=2)
    V[:, 5] = 0.0                                           # rank-deficient
    h = P.ppca_create(dev_matrix(np.zeros((2, d)), "f32"))
    Qd = empty_basis(d, m)
    P.ppca_orthonormalize(h, dev_basis(V), Qd, m)
    with pytest.raises(P.PPCAError) as ei:
        P.ppca_sync(h)
    assert ei.value.status_name == "PPCA_ERR_NUMERICAL"
    P.ppca_sync(h)                                          # status cleared


@pytest.mark.parametrize("m", [1, 2, 3, 16, 64, 127, 128])
def test_eigh_small(P, m):
    import torch
    rng = np.random.default_rng(m)
    Qm = synth.haar_orthogonal(m, rng)
    lam = np.sort(np.exp(-np.arange(m) / 20.0) * (1 + 0.02 * rng.random(m)))[::-1] * 1e3
    G = (Qm * lam) @ Qm.T
    G = 0.5 * (G + G.T)
    Gd = torch.from_numpy(G).cuda()
    wd = torch.empty(m, dtype=torch.float64, device="cuda")
    Ud = torch.empty((m, m), dtype=torch.float64, device="cuda")
    h = P.ppca_create(dev_matrix(np.zeros((2, 4)), "f32"))
    P.ppca_eigh(h, Gd, m, wd, Ud)
    P.ppca_sync(h)
    w = wd.cpu().numpy()
    U = Ud.cpu().numpy().T            # column-major m x m -> columns are eigenvectors
    wref, Uref = oracle.eigh_desc(G)
    # eigenvalues: FP64 Rayleigh quotients of vectors accurate to ~u*|G|/gap
    np.testing.assert_allclose(w, wref, rtol=1e-9, atol=1e-9 * wref[0])
    # vectors: FP32 Jacobi on a dense matrix; its backward error is c(m) u |G| with
    # c growing slowly with m and the sweep count, so the angle is <~ 16 u |G| / gap_i
    gaps = np.minimum(np.abs(np.diff(np.r_[np.inf, wref])), np.abs(np.diff(np.r_[wref, -np.inf])))
    u = 2.0 ** -24
    for i in range(m):
        assert oracle.angle(U[:, i], Uref[:, i]) <= 16 * u * wref[0] / gaps[i] + 1e-6


@pytest.mark.parametrize("n,d,ldo", [(257, 300, 304), (1000, 512, 512), (33, 1024, 1032)])
def test_quantize_bf16_bit_exact(P, n, d, ldo):
    """Round to nearest even, bit for bit: the oracle's codec and torch's conversion.
    d % 8 == 0 with 16-byte pitches takes the eight-wide kernel, 300 the scalar one."""
    import torch
    rng = np.random.default_rng(0)
    X = (rng.standard_normal((n, d)) * 10.0 ** rng.uniform(-3, 3, (n, d))).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    out = torch.empty((n, ldo), dtype=torch.int16, device="cuda")[:, :d]
    P.ppca_quantize_bf16(Xd, out)
    torch.cuda.synchronize()
    lib = torch.from_numpy(X).to(torch.bfloat16).view(torch.int16).numpy()
    np.testing.assert_array_equal(out.cpu().numpy(), lib)
    got = oracle.bf16_bits_to_f64(out.cpu().numpy().view(np.uint16))
    np.testing.assert_array_equal(got, oracle.bf16_round_rne(X))


FP8_CASES = [
    # n, d, m, r0, r1
    (3001, 512, 64, 0, 3001),
    (1000, 200, 33, 17, 931),        # ragged d and rows
    (257, 64, 1, 0, 257),
    (5000, 1024, 128, 0, 5000),
    (1000, 8192, 64, 0, 512),        # split-K Y = X V
    # enough row tiles for every SM: the FAST pass runs on the FP8 tensor cores
    (20000, 1024, 128, 0, 20000),
    (30001, 200, 33, 5, 29000),      # ragged d, rows and m
    (12000, 4096, 128, 0, 12000),
    (40000, 64, 1, 0, 40000),
]


@pytest.mark.parametrize("n,d,m,r0,r1", FP8_CASES)
@pytest.mark.parametrize("prec,tol", [("FAST", 1e-2), ("ACCURATE", 2e-5)])
def test_xpass_fp8_tensor_cores(P, n, d, m, r0, r1, prec, tol):
    """FP8 E4M3 data with per-row scales on tensor cores.  With row tiles for
    every SM the FAST pass runs on kind::f8f6f4 (V and Y' = diag(s^2) X8 V as
    two E4M3 pieces at a power-of-two scale); otherwise, and for ACCURATE, the
    E4M3 tiles are widened to BF16 in shared memory (exact) and s_r^2 scales Y.
    Normwise against X^T X V of the dequantised stored values in FP64 (FAST
    1e-2, ACCURATE with three BF16 pieces 2e-5), and element by element
    against the same pass formed exactly from the rounded pieces."""
    import torch
    X, _ = synth.gaussian_data(n, d, 0.97 ** np.arange(1, d + 1), seed=31) if d <= 4096 else \
        (np.random.default_rng(31).standard_normal((n, d)) * (0.9995 ** np.arange(1, d + 1))[None, :], None)
    codes, scales = oracle.fp8_row_quantize(X)
    ldp = (d + 15) // 16 * 16                          # 16-byte row pitch
    Xd = torch.zeros((n, ldp), dtype=torch.uint8, device="cuda")[:, :d]
    Xd.copy_(torch.from_numpy(codes))
    sd = torch.from_numpy(scales).cuda()
    Vd = dev_basis(synth.initial_basis(d, m, seed=8))
    Zd = empty_basis(d, m)
    h = P.ppca_create(Xd, row_scales=sd)
    P.ppca_xpass(h, Vd, m, r0, r1, Zd, getattr(P, "PPCA_PREC_" + prec))
    P.ppca_sync(h)
    Xs = (oracle.e4m3_decode(codes) * scales.astype(np.float64)[:, None])[r0:r1]
    Zref = Xs.T @ (Xs @ host_basis(Vd))
    assert normwise(host_basis(Zd), Zref) <= tol
    # element by element on the unscaled codes with the s_r^2 row factor of the pass
    X8 = oracle.e4m3_decode(codes)[r0:r1]
    s2 = scales.astype(np.float64)[r0:r1] ** 2
    if prec == "FAST" and (r1 - r0 + 127) // 128 * 2 > torch.cuda.get_device_properties(0).multi_processor_count:
        # kind::f8f6f4: V and Y as two E4M3 pieces at a power-of-two scale
        Zq, R = fast_e4m3_reference(X8, scales[r0:r1], host_basis(Vd))
        assert ratio(host_basis(Zd), Zq, R, *TAU_FAST) <= 1.0
    elif prec == "FAST":
        Zq, R = fast_reference(X8, host_basis(Vd), row_factor=s2)
        assert ratio(host_basis(Zd), Zq, R, *TAU_FAST) <= 1.0
    else:
        assert split_ratio(host_basis(Zd), X8, host_basis(Vd), *tau_split(d), row_factor=s2) <= 1.0


@pytest.mark.parametrize("d,ldo", [(520, 528), (4096, 4096), (7, 16), (2050, 2064)])
def test_quantize_fp8_bit_exact(P, d, ldo):
    """Per-row scale and E4M3 codes bit for bit against the oracle's codec; d % 4 == 0
    with aligned pitches takes the register-held row kernel, 7 the general one."""
    import torch
    rng = np.random.default_rng(1)
    X = (rng.standard_normal((129, d)) * 10.0 ** rng.uniform(-2, 2, (129, 1))).astype(np.float32)
    X[7] = 0.0
    X[8, 3] = 1e-30
    Xd = torch.from_numpy(X).cuda()
    out = torch.empty((129, ldo), dtype=torch.uint8, device="cuda")[:, :d]
    sc = torch.empty(129, dtype=torch.float32, device="cuda")
    P.ppca_quantize_fp8(Xd, out, sc)
    torch.cuda.synchronize()
    qref, sref = oracle.fp8_row_quantize(X)
    np.testing.assert_array_equal(sc.cpu().numpy(), sref)
    np.testing.assert_array_equal(out.cpu().numpy(), qref)


def test_fused_l2_keep_changes_only_cache_hints(P):
    """The L2 share kept for the consumers' re-read steers eviction hints only:
    every setting gives the same Z, bit for bit."""
    n, d, m = 20000, 1024, 64
    X = np.random.default_rng(9).standard_normal((n, d)) * (0.97 ** np.arange(1, d + 1))[None, :] ** 0.5
    Xd = dev_matrix(X, "bf16")
    Vd = dev_basis(synth.initial_basis(d, m, seed=2))
    h = P.ppca_create(Xd)
    out = []
    for keep in (0, 1, 40, 100):
        P.ppca_set_schedule(h, fused=1, l2_keep=keep)
        Z = empty_basis(d, m)
        P.ppca_xpass(h, Vd, m, 0, n, Z, P.PPCA_PREC_FAST)
        P.ppca_sync(h)
        out.append(host_basis(Z))
    for z in out[1:]:
        assert np.array_equal(z, out[0])
