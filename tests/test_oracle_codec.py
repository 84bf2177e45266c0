"""Pins for the oracle's storage codecs (exact reading of BF16 / FP8 E4M3 data).

E4M3 values follow the OCP 8-bit floating point format (bias 7, 3 mantissa
bits, subnormals, maximum 448, S.1111.111 = NaN, no infinities); the table is
checked at the format's landmark values and against torch's float8_e4m3fn
conversion (a library routine) on every finite code.
"""
import math

import numpy as np
import pytest

import oracle


def test_e4m3_landmarks():
    v = oracle.e4m3_decode(np.array([0x00, 0x01, 0x07, 0x08, 0x38, 0x7E, 0x80, 0xFE, 0x3C]))
    np.testing.assert_array_equal(v[:8], [0.0, 2.0 ** -9, 7 * 2.0 ** -9, 2.0 ** -6, 1.0, 448.0, -0.0, -448.0])
    assert v[8] == 1.5
    assert math.isnan(oracle.e4m3_decode(np.array([0x7F]))[0])
    assert math.isnan(oracle.e4m3_decode(np.array([0xFF]))[0])


def test_e4m3_round_trip_all_finite_codes():
    codes = np.array([c for c in range(256) if (c & 0x7F) != 0x7F], dtype=np.uint8)
    back = oracle.e4m3_encode_rne(oracle.e4m3_decode(codes))
    np.testing.assert_array_equal(back, codes)


def test_e4m3_ties_to_even_and_saturation():
    vals = oracle.e4m3_decode(np.arange(0, 0x7F, dtype=np.uint8))
    mids = 0.5 * (vals[:-1] + vals[1:])
    codes = oracle.e4m3_encode_rne(mids)
    lo = np.arange(0, 0x7E)
    expect = np.where(lo % 2 == 0, lo, lo + 1)
    np.testing.assert_array_equal(codes, expect)
    np.testing.assert_array_equal(oracle.e4m3_encode_rne(np.array([1e6, -1e6, 460.0])), [0x7E, 0xFE, 0x7E])


def test_e4m3_matches_torch_library_conversion():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8")
    codes = np.array([c for c in range(256) if (c & 0x7F) != 0x7F], dtype=np.uint8)
    tv = torch.from_numpy(codes).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(oracle.e4m3_decode(codes), tv)
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(20000) * 10.0 ** rng.uniform(-4, 2.5, 20000)).astype(np.float32)
    x = x[np.abs(x) < 448.0]
    mine = oracle.e4m3_encode_rne(x)
    lib = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    np.testing.assert_array_equal(mine, lib)


def test_fp8_row_quantize_scale_and_error_bound():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((40, 33)).astype(np.float32)
    X[5] = 0.0
    q, s = oracle.fp8_row_quantize(X)
    assert s[5] == 1.0 and np.all(q[5] == 0)
    deq = oracle.e4m3_decode(q) * s[:, None]
    amax = np.abs(X).max(axis=1)
    # max-magnitude element maps to 448 (up to the FP32 division's rounding)
    assert np.all(np.abs(oracle.e4m3_decode(q)).max(axis=1)[amax > 0] == 448.0)
    # relative error of E4M3 normals <= 2^-4; subnormals <= half a step 2^-10 (times s)
    err = np.abs(deq - X)
    bound = np.maximum(np.abs(X) * 2.0 ** -4, s[:, None] * 2.0 ** -10) * (1 + 1e-6)
    assert np.all(err <= bound)


def test_bf16_bits():
    bits = np.array([0x3F80, 0xC000, 0x4049, 0x0001, 0x7F7F], dtype=np.uint16)
    v = oracle.bf16_bits_to_f64(bits)
    assert v[0] == 1.0 and v[1] == -2.0 and v[2] == 3.140625
    assert v[3] == 2.0 ** -133
    assert v[4] == (2 - 2.0 ** -7) * 2.0 ** 127


def test_bf16_round_landmarks_and_ties():
    """1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties go to the even
    mantissa (1); 1 + 3 * 2^-8 lies halfway between 1 + 2^-7 (odd) and
    1 + 2^-6 (even); just above a tie rounds up; signs and zero pass through;
    a carry out of the mantissa bumps the exponent."""
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -20, -2.5, 0.0,
                  2.0 - 2.0 ** -9, 3.0e38])
    r = oracle.bf16_round_rne(x)
    np.testing.assert_array_equal(r[:7], [1.0, 1.0, 1.0 + 2.0 ** -6, 1.0 + 2.0 ** -7, -2.5, 0.0, 2.0])
    assert abs(r[7] - 3.0e38) <= 2.0 ** -8 * 3.0e38


def test_bf16_round_matches_torch_library_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(50000) * 10.0 ** rng.uniform(-30, 30, 50000)).astype(np.float32)
    mine = oracle.bf16_round_rne(x)
    lib = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mine, lib)
    # and the relative error bound of round to nearest with 8 significant bits, u = 2^-8
    # (normal range: below 2^-126 BF16, like FP32, keeps fewer significant bits)
    xn = x.astype(np.float64)
    normal = np.isfinite(xn) & (np.abs(xn) >= 2.0 ** -126) & (np.abs(xn) < 3.0e38)
    assert np.all(np.abs(mine - xn)[normal] <= 2.0 ** -8 * np.abs(xn[normal]))
