"""Pins for the oracle's pPCA step (Algorithm 1), orthonormalisation and metrics.

* the counterexample of Section 4.1, with the paper's numbers (golden fixture);
* the variance identity of Section 4.2 (Var of X~ is Var of X restricted to S);
* the pPCA output lies in span(V), is orthonormal, depends only on span(V), and
  equals the top-k eigenpairs of P_V X^T X P_V (computed separately in d dims);
* exact recovery when span(V) is a dominant eigenspace (Theorem 4.4's limit);
* four planted mistakes in the step (no orthonormalisation, transposed
  rotation, eigenvalues not divided by n, ascending order) fail the
  projected-problem pin;
* the row-sampled step: SplitMix64's published outputs, the selection rules,
  and the support pin (data only inside the sample: eigenvalues scaled by
  n/|S|; only outside: zero), which two planted mistakes fail;
* Cauchy interlacing of the Ritz values;
* the LCES worked example of Section 5.3.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# --------------------------------------------------------------------------- orth

@pytest.mark.parametrize("shape", [(10, 1), (50, 7), (200, 32)])
def test_orth_is_thin_qr_with_positive_diagonal(shape):
    rng = np.random.default_rng(shape[0])
    V = rng.standard_normal(shape)
    Q, R = oracle.qr_pos(V)
    np.testing.assert_allclose(Q.T @ Q, np.eye(shape[1]), atol=1e-14)
    np.testing.assert_allclose(Q @ R, V, atol=1e-12)
    assert np.all(np.diag(R) > 0)
    assert np.allclose(np.tril(Q.T @ V, -1), 0.0, atol=1e-12)
    # unique thin QR: agrees with LAPACK's after fixing signs
    Ql, Rl = np.linalg.qr(V)
    Ql = Ql * np.sign(np.diag(Rl))[None, :]
    np.testing.assert_allclose(Q, Ql, atol=1e-12)


def test_orth_ill_conditioned():
    rng = np.random.default_rng(3)
    U, _ = np.linalg.qr(rng.standard_normal((300, 20)))
    V = U * (10.0 ** -np.arange(20) * 0.5)[None, :]   # kappa ~ 1e19 by column scaling
    Q = oracle.orth(V @ np.triu(np.ones((20, 20))))
    np.testing.assert_allclose(Q.T @ Q, np.eye(20), atol=1e-13)


# --------------------------------------------------------------- counterexample

def test_counterexample_covariance_matches_paper():
    g = load("counterexample.json")
    X = np.array(g["points"], dtype=float)
    np.testing.assert_array_equal(X, synth.counterexample_points())
    C = oracle.covariance(X) / X.shape[0]
    np.testing.assert_allclose(3.0 * C, np.array(g["covariance_over_n_times_3"], dtype=float), atol=1e-15)
    E, lam = oracle.ground_truth(X, 2)
    np.testing.assert_allclose(np.abs(E.T), np.array(g["top2_principal_directions"], dtype=float), atol=1e-15)
    np.testing.assert_allclose(lam, [3.0, 4.0 / 3.0], rtol=1e-15)


@pytest.mark.parametrize("eps", load("counterexample.json")["eps_cases"])
def test_counterexample_ppca(eps):
    X = synth.counterexample_points()
    V = np.array([[eps, 0.0], [0.0, 1.0], [math.sqrt(1 - eps * eps), 0.0]])
    E, lam = oracle.ppca_finalize(X, V, 2)
    # projected covariance diag((1 + 8 eps^2)/3, 4/3) (corrected (1,1) entry)
    expected = sorted([(1 + 8 * eps * eps) / 3.0, 4.0 / 3.0], reverse=True)
    np.testing.assert_allclose(lam, expected, rtol=1e-13)
    e1 = np.array([1.0, 0.0, 0.0])
    if eps * eps < 3.0 / 8.0:
        # pPCA swaps: its first direction is the second priming vector (0,1,0)
        assert oracle.angle(E[:, 0], [0.0, 1.0, 0.0]) < 1e-12
        assert abs(E[:, 0] @ e1) ** 2 < eps * eps + 1e-15 or eps == 0.0
        assert abs(E[:, 0] @ e1) < 1e-12
    else:
        assert oracle.angle(E[:, 0], V[:, 0]) < 1e-12
        assert oracle.angle(E[:, 1], [0.0, 1.0, 0.0]) < 1e-12


# ------------------------------------------------------------ pPCA invariants

def _problem(seed=11, n=500, d=30, m=6):
    rng = np.random.default_rng(seed)
    lam = 0.8 ** np.arange(1, d + 1)
    X, _ = synth.gaussian_data(n, d, lam, seed)
    V = rng.standard_normal((d, m))
    return X, V


def test_variance_restricted_to_S():
    """Section 4.2: v^T (X~^T X~) v = v^T (X^T X) v for v in S."""
    X, V = _problem()
    Q = oracle.orth(V)
    Xt = X @ Q @ Q.T                      # projected points x~_i = P_S x_i
    rng = np.random.default_rng(1)
    for _ in range(5):
        v = Q @ rng.standard_normal(Q.shape[1])
        v /= np.linalg.norm(v)
        assert math.isclose(oracle.variance_captured(Xt, v), oracle.variance_captured(X, v), rel_tol=1e-12)


def test_variance_captured_closed_forms():
    """An axis direction captures its column's sum of squares; an exact
    eigenvector of X^T X captures its eigenvalue; the direction's length and
    sign do not matter."""
    rng = np.random.default_rng(4)
    X = rng.standard_normal((40, 5))
    for j in range(5):
        e = np.zeros(5)
        e[j] = 1.0
        assert math.isclose(oracle.variance_captured(X, e), float((X[:, j] ** 2).sum()), rel_tol=1e-14)
    sigma = np.array([3.0, 2.0, 0.5])
    Xe, Q = synth.exact_spectrum_data(30, 3, sigma, seed=2)
    for j in range(3):
        assert math.isclose(oracle.variance_captured(Xe, -7.0 * Q[:, j]), sigma[j] ** 2, rel_tol=1e-12)


def test_ppca_output_in_span_orthonormal_and_top_eigs_of_projected_cov():
    X, V = _problem()
    n, d = X.shape
    k = 4
    E, lam = oracle.ppca_finalize(X, V, k)
    Q = oracle.orth(V)
    np.testing.assert_allclose(E.T @ E, np.eye(k), atol=1e-13)
    np.testing.assert_allclose(E - Q @ (Q.T @ E), 0.0, atol=1e-13)
    # full d x d eigenproblem of P C P, solved separately
    P = Q @ Q.T
    C = oracle.covariance(X)
    w_full, U_full = oracle.eigh_desc(P @ C @ P)
    np.testing.assert_allclose(lam * n, w_full[:k], rtol=1e-11)
    for i in range(k):
        assert oracle.angle(E[:, i], U_full[:, i]) < 1e-9
    # residual of the projected problem
    R = P @ C @ P @ E - E * (lam * n)[None, :]
    assert np.abs(R).max() < 1e-10 * lam[0] * n


def _projected_problem_pin(finalize) -> bool:
    """The pin above as a predicate on a pPCA-step implementation: output in
    span(V), orthonormal, and the top-k eigenpairs of P_V X^T X P_V / n."""
    X, V = _problem()
    n, k = X.shape[0], 4
    E, lam = finalize(X, V, k)
    Q = oracle.orth(V)
    P = Q @ Q.T
    w_full, U_full = oracle.eigh_desc(P @ oracle.covariance(X) @ P)
    return bool(np.allclose(E.T @ E, np.eye(k), atol=1e-12) and np.allclose(E - Q @ (Q.T @ E), 0.0, atol=1e-12)
                and np.allclose(lam * n, w_full[:k], rtol=1e-10)
                and all(oracle.angle(E[:, i], U_full[:, i]) < 1e-8 for i in range(k)))


def _step_parts(X, V):
    Q = oracle.orth(V)
    Y = X @ Q
    w, U = oracle.eigh_desc(Y.T @ Y)
    return Q, w, U


def test_planted_mistakes_in_the_ppca_step_fail_the_projected_problem_pin():
    assert _projected_problem_pin(oracle.ppca_finalize)

    def no_orthonormalisation(X, V, k):            # G from X V, rotation of V itself
        Y = X @ V
        w, U = oracle.eigh_desc(Y.T @ Y)
        return oracle.sign_fix(V @ U[:, :k]), w[:k] / X.shape[0]

    def transposed_rotation(X, V, k):              # E = Q U^T
        Q, w, U = _step_parts(X, V)
        return oracle.sign_fix(Q @ U.T[:, :k]), w[:k] / X.shape[0]

    def eigenvalues_not_divided_by_n(X, V, k):
        Q, w, U = _step_parts(X, V)
        return oracle.sign_fix(Q @ U[:, :k]), w[:k]

    def ascending_order(X, V, k):
        Q, w, U = _step_parts(X, V)
        return oracle.sign_fix(Q @ U[:, ::-1][:, :k]), w[::-1][:k] / X.shape[0]

    for bad in (no_orthonormalisation, transposed_rotation, eigenvalues_not_divided_by_n, ascending_order):
        assert not _projected_problem_pin(bad), bad.__name__


def test_ppca_depends_only_on_span():
    X, V = _problem(seed=4)
    rng = np.random.default_rng(9)
    M = rng.standard_normal((V.shape[1], V.shape[1])) + 3 * np.eye(V.shape[1])
    E1, l1 = oracle.ppca_finalize(X, V, 5)
    E2, l2 = oracle.ppca_finalize(X, V @ M, 5)
    np.testing.assert_allclose(l1, l2, rtol=1e-11)
    np.testing.assert_allclose(E1, E2, atol=1e-9)


def test_ppca_exact_when_span_is_dominant_eigenspace():
    X, _ = _problem(seed=8, n=600, d=25)
    Etrue, ltrue = oracle.ground_truth(X)
    rng = np.random.default_rng(2)
    m, k = 7, 5
    V = Etrue[:, :m] @ (rng.standard_normal((m, m)) + 2 * np.eye(m))
    E, lam = oracle.ppca_finalize(X, V, k)
    np.testing.assert_allclose(lam, ltrue[:k], rtol=1e-11)
    for i in range(k):
        assert oracle.angle(E[:, i], Etrue[:, i]) < 1e-9


def test_interlacing():
    X, V = _problem(seed=21, m=8)
    n = X.shape[0]
    _, lfull = oracle.ground_truth(X)
    _, lproj = oracle.ppca_finalize(X, V, 8)
    assert np.all(lproj <= lfull[:8] * (1 + 1e-12))


# --------------------------------------------------------------------- metrics

def test_lces_worked_example():
    g = load("lces_example.json")
    V = math.pi / 8
    angles = [a * V for a in g["angles_in_units_of_V"]]
    assert oracle.lces(angles, V) == g["expected_lces"]
    # strict inequality, and a full streak
    assert oracle.lces([V, 0.0], V) == 0
    assert oracle.lces([0.0, 0.1 * V], V) == 2


def test_angle_sign_invariant_and_small_angles():
    e = np.array([1.0, 0.0, 0.0])
    for t in [1e-9, 1e-6, 1e-3, 0.5, math.pi / 2]:
        v = np.array([math.cos(t), math.sin(t), 0.0])
        assert math.isclose(oracle.angle(v, e), t, rel_tol=1e-9, abs_tol=1e-15)
        assert math.isclose(oracle.angle(-3.0 * v, e), t, rel_tol=1e-9, abs_tol=1e-15)


def test_principal_angles_known():
    d = 6
    t = [0.3, 1e-5]
    Q = np.eye(d)[:, :2]
    E = np.zeros((d, 2))
    E[:, 0] = [math.cos(t[0]), 0, math.sin(t[0]), 0, 0, 0]
    E[:, 1] = [0, math.cos(t[1]), 0, math.sin(t[1]), 0, 0]
    pa = oracle.principal_angles(Q, E)
    np.testing.assert_allclose(pa, sorted(t), rtol=1e-9)


# --- pPCA step on a seeded sample of the rows (Section 5: 10 % projected) ---

def test_splitmix64_published_outputs():
    """The SplitMix64 stream seeded with 0: its first three outputs as published
    with the generator's reference implementation."""
    golden = 0x9E3779B97F4A7C15
    outs = [oracle.splitmix64((j * golden) & ((1 << 64) - 1)) for j in (1, 2, 3)]
    assert outs == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_sampled_tiles_selection_rules():
    n = 128 * 5000 + 77                              # ragged last block
    all_t, rows = oracle.sampled_tiles(n, 1.0, 3)
    assert all_t == list(range(5001)) and rows == n
    keep, rows = oracle.sampled_tiles(n, 0.1, 3)
    assert keep == sorted(keep) and keep == oracle.sampled_tiles(n, 0.1, 3)[0]
    # binomial(5001, 0.1): mean 500, sd 21
    assert abs(len(keep) - 500.1) < 5 * 21.2
    assert rows == 128 * len(keep) - (51 if 5000 in keep else 0)
    assert keep != oracle.sampled_tiles(n, 0.1, 4)[0]
    one, rows1 = oracle.sampled_tiles(1000, 1e-30, 9)    # nothing passes: one block is kept
    assert len(one) == 1 and rows1 == (128 if one[0] < 7 else 1000 - 7 * 128)


def test_ppca_finalize_rows_all_blocks_is_the_full_step():
    rng = np.random.default_rng(5)
    n, d, m, k = 700, 12, 6, 4
    X = rng.standard_normal((n, d)) * np.linspace(3, 0.5, d)
    V = rng.standard_normal((d, m))
    tiles, _ = oracle.sampled_tiles(n, 1.0, 1)
    E1, l1 = oracle.ppca_finalize_rows(X, V, k, tiles)
    E0, l0 = oracle.ppca_finalize(X, V, k)
    np.testing.assert_allclose(l1, l0, rtol=1e-12)
    np.testing.assert_allclose(E1, E0, atol=1e-10)


def _sample_support_pin(finalize_rows) -> bool:
    """Data nonzero only inside the sampled blocks: the sampled step equals the
    full step with eigenvalues scaled by n / |S| (same Gram matrix, other row
    count); data nonzero only outside them: every sampled eigenvalue is 0."""
    rng = np.random.default_rng(12)
    n, d, m, k = 128 * 12 + 50, 9, 5, 3                   # ragged last block
    tiles, rows = oracle.sampled_tiles(n, 0.3, 7)
    inside = np.zeros(n, dtype=bool)
    for t in tiles:
        inside[t * 128:min((t + 1) * 128, n)] = True
    X = rng.standard_normal((n, d)) * np.linspace(2.0, 0.4, d)
    V = rng.standard_normal((d, m))
    X_in, X_out = X * inside[:, None], X * (~inside)[:, None]
    E_full, l_full = oracle.ppca_finalize(X_in, V, k)
    E_s, l_s = finalize_rows(X_in, V, k, tiles)
    _, l_zero = finalize_rows(X_out, V, k, tiles)
    return bool(rows == inside.sum() and np.allclose(l_s, l_full * n / rows, rtol=1e-12)
                and max(oracle.angle(E_s[:, i], E_full[:, i]) for i in range(k)) < 1e-9
                and np.abs(l_zero).max() == 0.0)


def test_ppca_finalize_rows_sees_exactly_the_sampled_blocks():
    assert _sample_support_pin(oracle.ppca_finalize_rows)

    def divides_by_n(X, V, k, tiles, tile=128):
        E, lam = oracle.ppca_finalize_rows(X, V, k, tiles, tile)
        rows = sum(min((t + 1) * tile, X.shape[0]) - t * tile for t in tiles)
        return E, lam * rows / X.shape[0]

    def ignores_the_sample(X, V, k, tiles, tile=128):
        E, lam = oracle.ppca_finalize(X, V, k)
        rows = sum(min((t + 1) * tile, X.shape[0]) - t * tile for t in tiles)
        return E, lam * X.shape[0] / rows

    for bad in (divides_by_n, ignores_the_sample):
        assert not _sample_support_pin(bad), bad.__name__


def test_ppca_finalize_rows_on_repeated_block_matches_full():
    """Data made of one 128-row block repeated: every block-aligned sample has
    the same per-row covariance, so the sampled step returns the full result."""
    rng = np.random.default_rng(6)
    d, m, k = 10, 5, 3
    B = rng.standard_normal((128, d)) * np.linspace(2, 0.3, d)
    X = np.tile(B, (40, 1))
    V = rng.standard_normal((d, m))
    E0, l0 = oracle.ppca_finalize(X, V, k)
    for seed in (1, 2, 3):
        tiles, rows = oracle.sampled_tiles(X.shape[0], 0.25, seed)
        E1, l1 = oracle.ppca_finalize_rows(X, V, k, tiles)
        np.testing.assert_allclose(l1, l0, rtol=1e-12)
        np.testing.assert_allclose(E1, E0, atol=1e-10)
