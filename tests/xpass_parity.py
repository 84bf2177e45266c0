"""Element-wise parity criterion for the X-pass Z = X^T (X V) (test infrastructure).

The references are formed in FP64 on the host from the stored values of X
(exact in FP64) and the FP32 basis V; the only arithmetic they borrow is the
oracle's BF16 codec.

* ``fast_reference``: the FAST pass of BF16 and FP8 data as the method defines
  it -- V rounded to BF16, Y = X V_hat formed exactly, multiplied by an
  optional per-row factor (s_r^2 for FP8 rows), rounded to BF16, then
  Z = X^T Y_hat.  What the GPU may still do differently is (a) its FP32
  accumulation of Y moves Y across a BF16 rounding boundary now and then, a
  "flip" of one BF16 unit (<= 2^-7 |Y_rc|), and (b) its FP32 tensor-core
  accumulation of Z drifts by a relative amount of order 2e-8 per accumulating
  MMA (measured on sm_103a; at most 16384 MMAs between folds in the fused pass,
  i.e. ~3.3e-4).  Each flip enters Z_jc as one term of size <= 2^-7 |X_rj Y_rc|
  with an independent sign; flips hit a small fraction f of the elements (the
  FP32 error of Y is ~2^-24 sqrt(d) of its terms, a BF16 unit is 2^-7), so
  their sum is ~2^-7 sqrt(f) R_jc with R_jc = sqrt(sum_r X_rj^2 Y_rc^2).
  The share f grows with d (at d = 8192 about one element in eight flips), so
  the bound allows a full unit on every term: |dZ_jc| <= 2^-7 R_jc +
  tau_z |Z_jc|, which holds for any share of flips with independent signs.
* ``exact_reference``: Z = X^T X V in FP64, for the split-precision passes
  (ACCURATE; FP32 data).  Their Y carries accumulation error proportional to
  the sum of its terms' magnitudes, W_rc = (|X| |V|)_rc, so
  R_jc = sqrt(sum_r X_rj^2 W_rc^2), and the drift of the folded tensor-core
  accumulators is relative to Z itself.

* ``split_ratio``: the split-precision passes in full.  An FP32 tensor-core
  accumulator drifts by ~2e-8 per accumulating MMA relative to its running
  sum, which can exceed the final value when terms cancel.  Y_rc's running sum
  is bounded by W_rc, so Y's drift enters Z_jc as tau_y R_W,jc; Z_jc's running
  sum over rows is bounded by |Z_jc| plus the root-sum-square of its terms
  R_Z,jc = sqrt(sum_r X_rj^2 Y_rc^2), so Z's drift enters as
  tau_z (|Z_jc| + R_Z,jc).

``ratio`` returns max_jc |dZ_jc| / (tau_r R_jc + tau_z |Z_jc|): <= 1 passes.
A mistake confined to one 128-row tile, one row or one 64-wide K-stage moves
Z_jc by a sizeable share of R_jc (e.g. a dropped tile of n = 5000 rows by
about sqrt(128 / 5000) R = 0.16 R, twenty times 2^-7 R);
tests/test_xpass_parity_criterion.py plants such mistakes in an emulated pass
on the CPU and checks that the criterion rejects every one of them while it
accepts the correctly rounded emulation.
"""
import numpy as np

import oracle

TAU_FAST_R = 2.0 ** -7


def fast_reference(Xs, V32, row_factor=None):
    """(Z_ref, R) of the FAST pass: BF16-rounded V and Y, exact products."""
    Vh = oracle.bf16_round_rne(V32)
    Y = Xs @ Vh
    if row_factor is not None:
        Y = Y * np.asarray(row_factor, dtype=np.float64)[:, None]
    Yh = oracle.bf16_round_rne(Y)
    Z = Xs.T @ Yh
    R = np.sqrt((Xs * Xs).T @ (Yh * Yh))
    return Z, R


def _pow2_below(cap, v):
    """Largest power of two p with p * v <= cap (1 for v == 0)."""
    if not v > 0:
        return 1.0
    m, e = np.frexp(np.float32(cap) / np.float32(v))        # cap / v = m 2^e, m in [0.5, 1)
    return float(2.0 ** min(max(int(e) - 1, -126), 126))


def _e4m3_pieces(y):
    """hi = E4M3(y), lo = E4M3(y - hi) (round to nearest even, saturating): the value hi + lo."""
    hi = oracle.e4m3_decode(oracle.e4m3_encode_rne(y))
    lo = oracle.e4m3_decode(oracle.e4m3_encode_rne((np.asarray(y, dtype=np.float32) - hi).astype(np.float32)))
    return hi + lo


def fast_e4m3_reference(X8, scales, V32):
    """(Z_ref, R) of the FAST pass of E4M3 data on the FP8 tensor cores: V and
    Y' = diag(s^2) X8 V each carried as two E4M3 pieces at one power-of-two
    scale (2^a with max|V| 2^a <= 448; 2^b with sqrt(d) max s^2 max_c |v_c|
    2^b <= 1), products exact, Z = X8^T Y'."""
    V32 = np.asarray(V32, dtype=np.float32)
    s2 = np.asarray(scales, dtype=np.float32).astype(np.float64) ** 2
    d = V32.shape[0]
    sa = _pow2_below(448.0, float(np.max(np.abs(V32))))
    Vh = _e4m3_pieces((V32 * np.float32(sa)).astype(np.float32)) / sa
    vnorm = float(np.sqrt(np.max(np.sum(V32.astype(np.float64) ** 2, axis=0))))
    bound = np.float32(np.sqrt(np.float32(d))) * np.float32(np.max(s2)) * np.float32(vnorm)
    sb = _pow2_below(1.0, float(bound))
    Y = (X8 @ Vh) * s2[:, None] * sb
    Yh = _e4m3_pieces(Y.astype(np.float32)) / sb
    Z = X8.T @ Yh
    R = np.sqrt((X8 * X8).T @ (Yh * Yh))
    return Z, R


def exact_reference(Xs, V32, row_factor=None):
    """(Z_ref, R) of X^T diag(row_factor) X V in FP64 with the |X||V| term scale."""
    V = np.asarray(V32, dtype=np.float64)
    Y = Xs @ V
    W = np.abs(Xs) @ np.abs(V)
    if row_factor is not None:
        f = np.asarray(row_factor, dtype=np.float64)[:, None]
        Y, W = Y * f, W * np.abs(f)
    Z = Xs.T @ Y
    R = np.sqrt((Xs * Xs).T @ (W * W))
    return Z, R


def ratio(Z, Zref, R, tau_r, tau_z):
    """max over entries of |Z - Zref| / (tau_r R + tau_z |Zref|)."""
    den = tau_r * R + tau_z * np.abs(Zref)
    den = np.where(den > 0, den, np.finfo(np.float64).tiny)
    return float(np.max(np.abs(np.asarray(Z, dtype=np.float64) - Zref) / den))


def split_ratio(Z, Xs, V32, tau_y, tau_z, row_factor=None):
    """max_jc |Z - X^T D X V|_jc / (tau_y R_W,jc + tau_z (|Z_ref,jc| + R_Z,jc)), D = diag(row_factor)."""
    V = np.asarray(V32, dtype=np.float64)
    Y = Xs @ V
    W = np.abs(Xs) @ np.abs(V)
    if row_factor is not None:
        f = np.asarray(row_factor, dtype=np.float64)[:, None]
        Y, W = Y * f, W * np.abs(f)
    Zref = Xs.T @ Y
    X2 = Xs * Xs
    den = tau_y * np.sqrt(X2.T @ (W * W)) + tau_z * (np.abs(Zref) + np.sqrt(X2.T @ (Y * Y)))
    den = np.where(den > 0, den, np.finfo(np.float64).tiny)
    return float(np.max(np.abs(np.asarray(Z, dtype=np.float64) - Zref) / den))
