"""Pins for the oracle's primers (block power, Oja/Sanger, EigenGame) and schedule.

* fixed points: the exact eigenvectors are fixed by a power step, give a zero
  Oja/Sanger update with the full batch (Section 2.2) and a zero Riemannian
  EigenGame gradient (the Nash equilibrium, Section 2.3);
* special cases: Oja with one point and one neuron is the paper's single-neuron
  rule (Section 2.2); EigenGame with one player is gradient ascent on
  v^T M v (Eq. 1);
* convergence rate of simultaneous iteration (Rutishauser's bound);
* EigenGame's step (Section 5: SGD with Nesterov momentum, on the tangent
  space) against torch autograd of Eq. 3 and torch.optim.SGD(nesterov=True),
  with heavy-ball momentum and a missing tangent projection planted as
  mistakes that fail it;
* ordered convergence: Sanger and EigenGame find the individual eigenvectors,
  not just the subspace -- and two planted mistakes (Oja's symmetric subspace
  rule, EigenGame without the penalty) are shown to fail that pin;
* the sequential power method (Section 2.1): closed-form iterates on a 2 x 2
  diagonal problem, the axes of a diagonal spectrum found in order, the stop
  at the first step below eps -- with two planted mistakes (no deflation, the
  stop test inverted) shown to fail the axes pin.
"""
import math

import numpy as np
import pytest

import oracle
import oracle.core as core
import synth


def small_problem(n=3000, d=12, seed=3):
    sigma = np.sqrt(n * np.linspace(3.0, 0.5, d) ** 2)
    X, Q = synth.exact_spectrum_data(n, d, sigma, seed)
    lam = sigma ** 2 / n                      # eig(X^T X)/n exactly
    return X, Q, lam


# ------------------------------------------------------------------ schedule

def test_minibatch_schedule_epoch_aligned():
    n, b = 1000, 256
    seen = np.zeros(n, dtype=int)
    for t in range(4):
        r0, r1 = oracle.minibatch_rows(t, n, b)
        seen[r0:r1] += 1
    assert np.all(seen == 1)
    assert oracle.minibatch_rows(3, n, b) == (768, 1000)
    assert oracle.minibatch_rows(4, n, b) == (0, 256)
    assert oracle.minibatch_rows(0, 100, 256) == (0, 100)


# ------------------------------------------------------------------ power

def test_power_fixed_point():
    X, Q, lam = small_problem()
    E = Q[:, :5]
    E = E * np.sign(E[np.argmax(np.abs(E), axis=0), np.arange(5)])
    S = oracle.power_step(X, E)
    # orth keeps a positive diagonal, E's columns are already orthonormal
    np.testing.assert_allclose(np.abs(S.T @ E), np.eye(5), atol=1e-12)


@pytest.mark.parametrize("T", [1, 3, 6])
def test_power_rutishauser_bound(T):
    X, Q, lam = small_problem(seed=7)
    m = 4
    rng = np.random.default_rng(T)
    V0 = rng.standard_normal((X.shape[1], m))
    Q0 = oracle.orth(V0)
    theta0 = oracle.principal_angles(Q0, Q[:, :m]).max()
    QT = oracle.power_prime(X, V0, T)
    for i in range(m):
        e = Q[:, i]
        s = np.linalg.norm(e - QT @ (QT.T @ e))
        tan_i = math.tan(math.asin(min(1.0, s)))
        bound = (lam[m] / lam[i]) ** T * math.tan(theta0)
        assert tan_i <= bound * (1 + 1e-9) + 1e-13


def test_power_then_ppca_converges_to_ground_truth():
    X, Q, lam = small_problem(seed=9)
    V = oracle.power_prime(X, np.random.default_rng(0).standard_normal((12, 6)), 60)
    E, l = oracle.ppca_finalize(X, V, 4)
    np.testing.assert_allclose(l, lam[:4], rtol=1e-10)
    for i in range(4):
        assert oracle.angle(E[:, i], Q[:, i]) < 1e-6


# ------------------------------------------------------------------ Oja / Sanger

def test_oja_full_batch_fixed_point():
    X, Q, lam = small_problem()
    W = Q[:, :5].copy()
    W2 = oracle.oja_step(X, W, 0, X.shape[0], lr=0.3)
    np.testing.assert_allclose(W2, W, atol=1e-12)


def test_oja_single_point_single_neuron_is_the_papers_rule():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((5, 7))
    w = rng.standard_normal((7, 1))
    alpha = 0.01
    for t in range(5):
        x = X[t:t + 1].T
        y = float((x.T @ w)[0, 0])
        paper = w + alpha * (x * y - y * y * w)          # dw = alpha (x y - y^2 w)
        np.testing.assert_allclose(oracle.oja_step(X, w, t, 1, alpha), paper, atol=1e-14)


def _ordered_convergence_oja(step_fn, X, Q, m, epochs=60, b=100):  # lr 0.02/(1+t/200)
    rng = np.random.default_rng(4)
    W = oracle.orth(rng.standard_normal((X.shape[1], m)))
    steps = epochs * (-(-X.shape[0] // b))
    for t in range(steps):
        W = step_fn(X, W, t, b, 0.02 / (1.0 + t / 200.0))
    return max(oracle.angle(W[:, i], Q[:, i]) for i in range(m))


def test_oja_sanger_finds_individual_eigenvectors():
    X, Q, lam = small_problem(n=2000, d=8, seed=12)
    assert _ordered_convergence_oja(oracle.oja_step, X, Q, 3) < 0.02


def _symmetric_subspace_rule(X, W, t, b, lr):
    """Planted mistake: full Y^T Y instead of its upper triangle (Oja's subspace rule)."""
    r0, r1 = oracle.minibatch_rows(t, X.shape[0], b)
    Xb = X[r0:r1]
    Y = Xb @ W
    return W + lr / (r1 - r0) * (Xb.T @ Y - W @ (Y.T @ Y))


def test_planted_mistake_in_oja_fails_the_ordering_pin():
    X, Q, lam = small_problem(n=2000, d=8, seed=12)
    assert _ordered_convergence_oja(_symmetric_subspace_rule, X, Q, 3) > 0.1


# ------------------------------------------------------------------ EigenGame

def test_eigengame_nash_equilibrium():
    X, Q, lam = small_problem()
    V = Q[:, :5].copy()
    grad, MV, C = oracle.eigengame_gradients(X, V)
    riem = grad - V * np.sum(V * grad, axis=0, keepdims=True)
    assert np.abs(riem).max() < 1e-12 * lam[0]
    V2, buf = oracle.eigengame_step(X, V, np.zeros_like(V), 0, X.shape[0], lr=0.1)
    np.testing.assert_allclose(V2, V, atol=1e-13)


def test_eigengame_single_player_is_rayleigh_ascent():
    X, Q, lam = small_problem()
    rng = np.random.default_rng(5)
    v = oracle.orth(rng.standard_normal((X.shape[1], 1)))
    grad, MV, C = oracle.eigengame_gradients(X, v)
    M = X.T @ X / X.shape[0]
    np.testing.assert_allclose(grad, 2.0 * M @ v, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(C, v.T @ M @ v, rtol=1e-13)


def test_eigengame_utilities_gradient_by_finite_differences():
    """Eq. 3: the oracle's gradient is the derivative of U_j in v_j."""
    rng = np.random.default_rng(6)
    Xb = rng.standard_normal((50, 6))
    V = rng.standard_normal((6, 3))
    M = Xb.T @ Xb / Xb.shape[0]

    def U(j, Vm):
        u = Vm[:, j] @ M @ Vm[:, j]
        for i in range(j):
            u -= (Vm[:, j] @ M @ Vm[:, i]) ** 2 / (Vm[:, i] @ M @ Vm[:, i])
        return u

    grad, _, _ = oracle.eigengame_gradients(Xb, V)
    h = 1e-6
    for j in range(3):
        for a in range(6):
            Vp, Vm_ = V.copy(), V.copy()
            Vp[a, j] += h
            Vm_[a, j] -= h
            fd = (U(j, Vp) - U(j, Vm_)) / (2 * h)
            assert abs(fd - grad[a, j]) < 1e-6 * max(1.0, abs(fd))


def _ordered_convergence_eg(grad_fn, X, Q, m, steps=3000, b=500, lr=0.005):
    saved = core.eigengame_gradients
    core.eigengame_gradients = grad_fn
    try:
        V = oracle.eigengame_prime(X, np.random.default_rng(8).standard_normal((X.shape[1], m)),
                                   b, steps, lr, 0.9)
    finally:
        core.eigengame_gradients = saved
    return max(oracle.angle(V[:, i], Q[:, i]) for i in range(m))


def test_eigengame_finds_individual_eigenvectors():
    X, Q, lam = small_problem(n=2000, d=8, seed=12)
    assert _ordered_convergence_eg(core.eigengame_gradients, X, Q, 3) < 0.02


def _no_penalty(Xb, V):
    """Planted mistake: each player ignores the others (drops Eq. 3's penalty)."""
    MV = Xb.T @ (Xb @ V) / Xb.shape[0]
    return 2.0 * MV, MV, V.T @ MV


def test_planted_mistake_in_eigengame_fails_the_ordering_pin():
    X, Q, lam = small_problem(n=2000, d=8, seed=12)
    assert _ordered_convergence_eg(_no_penalty, X, Q, 3) > 0.1


def _library_eigengame_steps(X, V0, b, steps, lr, momentum):
    """The same parallel EigenGame steps, built from library parts only: the
    Euclidean gradient of each player's utility (Eq. 3, the other players held
    fixed) from torch autograd, its projection on the tangent space of the
    player's sphere, torch.optim.SGD with Nesterov momentum (ascent: the
    optimiser descends -U), then each column renormalised."""
    import torch
    Vt = torch.tensor(oracle.orth(V0), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.SGD([Vt], lr=lr, momentum=momentum, nesterov=True)
    Xt = torch.tensor(X, dtype=torch.float64)
    m = V0.shape[1]
    for t in range(steps):
        r0, r1 = oracle.minibatch_rows(t, X.shape[0], b)
        Xb = Xt[r0:r1]
        M = Xb.T @ Xb / (r1 - r0)
        fixed = Vt.detach()
        total = 0.0
        for j in range(m):
            vj = Vt[:, j]
            u = vj @ M @ vj
            for i in range(j):
                vi = fixed[:, i]
                u = u - (vj @ M @ vi) ** 2 / (vi @ M @ vi)
            total = total + u
        opt.zero_grad()
        (-total).backward()
        with torch.no_grad():
            g = Vt.grad
            g -= Vt * (Vt * g).sum(dim=0, keepdim=True)        # tangent projection of the gradient
        opt.step()
        with torch.no_grad():
            Vt /= Vt.norm(dim=0, keepdim=True)
    return Vt.detach().numpy()


def test_eigengame_nesterov_step_matches_library_sgd():
    """Section 5 trains with SGD and Nesterov momentum 0.9.  Away from the
    fixed point (g != 0) three steps of the oracle equal three steps assembled
    from torch autograd and torch.optim.SGD(nesterov=True) to 1e-12."""
    pytest.importorskip("torch")
    rng = np.random.default_rng(21)
    X = rng.standard_normal((300, 7)) * np.linspace(2.0, 0.3, 7)[None, :]
    V0 = rng.standard_normal((7, 4))
    Vo = oracle.eigengame_prime(X, V0, b=100, steps=3, lr=0.05, momentum=0.9)
    Vl = _library_eigengame_steps(X, V0, b=100, steps=3, lr=0.05, momentum=0.9)
    assert np.abs(Vo - oracle.orth(V0)).max() > 1e-2          # the steps really move the basis
    np.testing.assert_allclose(Vo, Vl, rtol=0, atol=1e-12)


def _heavy_ball_step(X, V, buf, t, b, lr, momentum=0.9):
    """Planted mistake: heavy-ball momentum (v <- v + lr buf) instead of Nesterov."""
    r0, r1 = oracle.minibatch_rows(t, X.shape[0], b)
    grad, _, _ = oracle.eigengame_gradients(X[r0:r1], V)
    g = grad - V * np.sum(V * grad, axis=0, keepdims=True)
    buf = momentum * buf + g
    Vn = V + lr * buf
    return Vn / np.linalg.norm(Vn, axis=0, keepdims=True), buf


def _unprojected_step(X, V, buf, t, b, lr, momentum=0.9):
    """Planted mistake: the Euclidean gradient, no tangent projection."""
    r0, r1 = oracle.minibatch_rows(t, X.shape[0], b)
    g, _, _ = oracle.eigengame_gradients(X[r0:r1], V)
    buf = momentum * buf + g
    Vn = V + lr * (g + momentum * buf)
    return Vn / np.linalg.norm(Vn, axis=0, keepdims=True), buf


@pytest.mark.parametrize("planted", [_heavy_ball_step, _unprojected_step])
def test_planted_mistake_in_eigengame_step_fails_the_library_pin(planted):
    pytest.importorskip("torch")
    rng = np.random.default_rng(21)
    X = rng.standard_normal((300, 7)) * np.linspace(2.0, 0.3, 7)[None, :]
    V0 = rng.standard_normal((7, 4))
    saved = core.eigengame_step
    core.eigengame_step = planted
    try:
        Vo = oracle.eigengame_prime(X, V0, b=100, steps=3, lr=0.05, momentum=0.9)
    finally:
        core.eigengame_step = saved
    Vl = _library_eigengame_steps(X, V0, b=100, steps=3, lr=0.05, momentum=0.9)
    assert np.abs(Vo - Vl).max() > 1e-6


# --- sequential power method with epsilon termination (Section 2.1) ---

def test_power_seq_iterates_follow_the_closed_form():
    """M = diag(l1, l2): from x0 = (cos a, sin a) the power iterate after t steps
    is proportional to (l1^t cos a, l2^t sin a)."""
    l1, l2, a = 4.0, 1.0, 0.7
    X = np.diag(np.sqrt([l1, l2]))
    V0 = np.array([[math.cos(a)], [math.sin(a)]])
    for T in (1, 2, 5):
        V, steps = oracle.power_seq_prime(X, V0, T, 0.0)
        ref = np.array([l1 ** T * math.cos(a), l2 ** T * math.sin(a)])
        ref /= np.linalg.norm(ref)
        np.testing.assert_allclose(V[:, 0], ref, rtol=1e-12)
        assert steps == [T]


def test_power_seq_finds_the_axes_of_a_diagonal_spectrum():
    rng = np.random.default_rng(2)
    d, m = 8, 4
    lam = 2.0 ** -np.arange(d)
    X = np.diag(np.sqrt(lam))                     # X^T X = diag(lam): eigenvectors are the axes
    V, steps = oracle.power_seq_prime(X, rng.standard_normal((d, m)), 2000, 1e-12)
    for j in range(m):
        assert abs(abs(V[j, j]) - 1.0) < 1e-10
    assert np.abs(V.T @ V - np.eye(m)).max() < 1e-12
    # rate lam_{j+1}/lam_j = 1/2: about log2(1/eps) steps each
    assert all(30 <= s <= 60 for s in steps), steps


def _power_seq_axes_pin(power_seq) -> bool:
    """The pin above as a predicate on an implementation of the sequential power method."""
    rng = np.random.default_rng(2)
    d, m = 8, 4
    X = np.diag(np.sqrt(2.0 ** -np.arange(d)))
    V, steps = power_seq(X, rng.standard_normal((d, m)), 2000, 1e-12)
    return bool(all(abs(abs(V[j, j]) - 1.0) < 1e-10 for j in range(m))
                and np.abs(V.T @ V - np.eye(m)).max() < 1e-12 and all(30 <= s <= 60 for s in steps))


def _power_seq_variant(X, V0, T, eps, deflate=True, stop_below=True):
    """The sequential power method with switches that plant a mistake."""
    Q0 = oracle.orth(V0)
    d, m = Q0.shape
    V, steps = np.zeros((d, m)), []
    for j in range(m):
        x, Vp, t = Q0[:, j].copy(), V[:, :j], 0
        while t < T:
            y = X.T @ (X @ x)
            if deflate:
                for _ in range(2):
                    y = y - Vp @ (Vp.T @ y)
            xn = y / np.linalg.norm(y)
            t += 1
            diff = np.linalg.norm(xn - x)
            x = xn
            if (diff < eps) if stop_below else (diff >= eps):
                break
        V[:, j] = x
        steps.append(t)
    return V, steps


def test_planted_mistakes_in_power_seq_fail_the_axes_pin():
    assert _power_seq_axes_pin(oracle.power_seq_prime)
    assert _power_seq_axes_pin(_power_seq_variant)                       # switches off: the method
    assert not _power_seq_axes_pin(lambda *a: _power_seq_variant(*a, deflate=False))
    assert not _power_seq_axes_pin(lambda *a: _power_seq_variant(*a, stop_below=False))


def test_power_seq_stops_at_the_first_step_below_eps():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((200, 6)) * np.array([3.0, 2.0, 1.5, 1.0, 0.5, 0.2])
    V0 = rng.standard_normal((6, 2))
    V, steps = oracle.power_seq_prime(X, V0, 500, 1e-4)
    # rerun the first direction step by step: the recorded count is the first t with |x_t - x_{t-1}| < eps
    M = X.T @ X
    x = oracle.orth(V0)[:, 0]
    for t in range(1, steps[0] + 1):
        y = M @ x
        xn = y / np.linalg.norm(y)
        diff = np.linalg.norm(xn - x)
        x = xn
        assert (diff < 1e-4) == (t == steps[0])
