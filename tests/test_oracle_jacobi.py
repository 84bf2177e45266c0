"""Pins for the oracle's cyclic Jacobi eigensolver (the full-PCA of Algorithm 1, step 4).

The solver is checked against closed forms (2x2; the trigonometric 3x3 formula
of O.K. Smith, CACM 1961), a generator whose eigenpairs are known by
construction, and a library routine (numpy.linalg.eigh) on random matrices.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def closed_form_2x2(a, b, c):
    mid = 0.5 * (a + c)
    rad = math.hypot(0.5 * (a - c), b)
    return np.array([mid + rad, mid - rad])


def smith_3x3(A):
    """Eigenvalues of a symmetric 3x3 matrix, descending (Smith 1961)."""
    p1 = A[0, 1] ** 2 + A[0, 2] ** 2 + A[1, 2] ** 2
    q = np.trace(A) / 3.0
    p2 = (A[0, 0] - q) ** 2 + (A[1, 1] - q) ** 2 + (A[2, 2] - q) ** 2 + 2.0 * p1
    p = math.sqrt(p2 / 6.0)
    B = (A - q * np.eye(3)) / p
    r = np.clip(np.linalg.det(B) / 2.0, -1.0, 1.0)
    phi = math.acos(r) / 3.0
    e1 = q + 2.0 * p * math.cos(phi)
    e3 = q + 2.0 * p * math.cos(phi + 2.0 * math.pi / 3.0)
    return np.array([e1, 3.0 * q - e1 - e3, e3])


@pytest.mark.parametrize("seed", range(8))
def test_2x2_closed_form(seed):
    rng = np.random.default_rng(seed)
    a, b, c = rng.standard_normal(3) * 10.0 ** rng.integers(-3, 4, size=3)
    A = np.array([[a, b], [b, c]])
    w, U = oracle.eigh_desc(A)
    np.testing.assert_allclose(w, closed_form_2x2(a, b, c), rtol=1e-13, atol=1e-13 * abs(A).max())
    np.testing.assert_allclose(A @ U, U * w, atol=1e-12 * abs(A).max())


@pytest.mark.parametrize("seed", range(8))
def test_3x3_trigonometric_closed_form(seed):
    rng = np.random.default_rng(100 + seed)
    M = rng.standard_normal((3, 3))
    A = M + M.T
    w, U = oracle.eigh_desc(A)
    np.testing.assert_allclose(w, smith_3x3(A), rtol=0, atol=1e-12 * abs(A).max())
    np.testing.assert_allclose(U.T @ U, np.eye(3), atol=1e-14)


def test_diagonal_and_permuted():
    A = np.diag([3.0, -1.0, 7.0, 0.0])
    w, U = oracle.eigh_desc(A)
    np.testing.assert_array_equal(w, [7.0, 3.0, 0.0, -1.0])
    np.testing.assert_array_equal(np.abs(U), np.eye(4)[:, [2, 0, 3, 1]])


def test_known_spectrum_generator():
    """X = U diag(sigma) Q^T with orthonormal U: X^T X = Q diag(sigma^2) Q^T."""
    n, d = 400, 40
    sigma = np.linspace(10.0, 1.0, d) ** 1.5
    X, Q = synth.exact_spectrum_data(n, d, sigma, seed=5)
    np.testing.assert_allclose(X.mean(axis=0), 0.0, atol=1e-12)
    E, lam = oracle.ground_truth(X)
    np.testing.assert_allclose(lam * n, sigma ** 2, rtol=1e-12)
    for i in range(d):
        assert oracle.angle(E[:, i], Q[:, i]) < 1e-10


@pytest.mark.parametrize("n", [5, 17, 64])
def test_against_library_eigh(n):
    rng = np.random.default_rng(n)
    M = rng.standard_normal((n, n))
    A = M @ M.T
    w, U = oracle.eigh_desc(A)
    wl = np.linalg.eigh(A)[0][::-1]
    np.testing.assert_allclose(w, wl, rtol=1e-11, atol=1e-12 * wl[0])
    np.testing.assert_allclose(U.T @ U, np.eye(n), atol=1e-12)
    np.testing.assert_allclose(A @ U, U * w, atol=1e-11 * wl[0])


def test_repeated_eigenvalues():
    rng = np.random.default_rng(7)
    Q = synth.haar_orthogonal(6, rng)
    lam = np.array([5.0, 5.0, 5.0, 2.0, 2.0, 1.0])
    A = (Q * lam) @ Q.T
    w, U = oracle.eigh_desc(A)
    np.testing.assert_allclose(w, lam, atol=1e-13)
    np.testing.assert_allclose(U.T @ U, np.eye(6), atol=1e-13)
    np.testing.assert_allclose(A @ U, U * w, atol=1e-12)


def test_sign_convention():
    U = np.array([[0.1, -0.9], [-0.8, 0.1], [0.2, 0.3]])
    F = oracle.sign_fix(U)
    assert F[1, 0] > 0 and F[0, 1] > 0
    # ties: the lowest index wins
    T = oracle.sign_fix(np.array([[-0.5], [0.5]]))
    assert T[0, 0] > 0


def test_rejects_nonsymmetric():
    with pytest.raises(ValueError):
        oracle.jacobi_eigh(np.array([[1.0, 2.0], [0.0, 1.0]]))
