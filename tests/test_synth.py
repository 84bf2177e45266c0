"""The seeded input generators (`synth/`), which feed both the CUDA path and the
oracle, pinned to what holds by construction: orthogonality of the rotations,
the closed-form spectrum of `exact_spectrum_data`, the population spectrum of
the known-lambda recipes (sample eigenvalues within a few standard errors),
centring, the affine map of the image-like data, the shape ranges of the ragged
batch, and determinism in the seed."""
import numpy as np
import pytest

import synth


def test_haar_orthogonal_is_orthogonal():
    Q = synth.haar_orthogonal(40, np.random.default_rng(3))
    assert np.abs(Q.T @ Q - np.eye(40)).max() <= 1e-13
    assert abs(abs(np.linalg.det(Q)) - 1.0) <= 1e-12


def test_gaussian_data_seeded_centred_with_population_spectrum():
    n, d = 40000, 12
    lam = 0.7 ** np.arange(1, d + 1)
    X, Q = synth.gaussian_data(n, d, lam, seed=5)
    X2, _ = synth.gaussian_data(n, d, lam, seed=5)
    X3, _ = synth.gaussian_data(n, d, lam, seed=6)
    assert np.array_equal(X, X2) and not np.array_equal(X, X3)
    assert np.abs(X.mean(axis=0)).max() <= 1e-14
    # in the rotated frame the columns are independent with variances lambda:
    # relative standard error of each sample variance sqrt(2 / n) = 0.7 %
    var = ((X @ Q) ** 2).mean(axis=0)
    assert np.abs(var / lam - 1.0).max() <= 5 * np.sqrt(2.0 / n)


def test_exact_spectrum_data_has_the_closed_form_gram_matrix():
    n, d = 300, 20
    sigma = np.linspace(3.0, 0.1, d)
    X, Q = synth.exact_spectrum_data(n, d, sigma, seed=8)
    G = X.T @ X
    ref = (Q * sigma ** 2) @ Q.T
    assert np.abs(G - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(X.sum(axis=0)).max() <= 1e-12


def test_fast_walsh_hadamard_is_normalised_and_an_involution():
    torch = pytest.importorskip("torch")
    d = 64
    Y = torch.randn((5, d), dtype=torch.float64, generator=torch.Generator().manual_seed(1))
    Z = synth._fwht_rows_(Y.clone())
    assert torch.allclose(Z.norm(dim=1), Y.norm(dim=1), rtol=1e-13)   # orthogonal
    assert torch.allclose(synth._fwht_rows_(Z.clone()), Y, atol=1e-13)  # H = H^T = H^-1
    e0 = torch.zeros((1, d), dtype=torch.float64)
    e0[0, 0] = 1.0
    assert torch.allclose(synth._fwht_rows_(e0), torch.full((1, d), d ** -0.5, dtype=torch.float64))


def test_hadamard_rotated_data_spectrum_and_centring():
    torch = pytest.importorskip("torch")
    n, d = 30000, 32
    lam = 0.8 ** np.arange(1, d + 1)
    X, (D1, perm, D2) = synth.hadamard_rotated_data_torch(n, d, lam, 4, "cpu", torch.float32)
    X2, _ = synth.hadamard_rotated_data_torch(n, d, lam, 4, "cpu", torch.float32)
    assert torch.equal(X, X2)
    assert sorted(perm.tolist()) == list(range(d)) and set(np.abs(D1)) == {1.0} and set(np.abs(D2)) == {1.0}
    Xd = X.double().numpy()
    assert np.abs(Xd.mean(axis=0)).max() <= 1e-6
    # Q orthogonal: the sample covariance has the population eigenvalues lambda
    # (top ones, relative standard error about sqrt(2 / n) = 0.8 %)
    w = np.linalg.eigvalsh(Xd.T @ Xd / n)[::-1]
    assert np.abs(w[:6] / lam[:6] - 1.0).max() <= 0.05
    assert abs(w.sum() / lam.sum() - 1.0) <= 0.02


def test_gaussian_data_torch_image_like_is_unit_range_and_centred():
    torch = pytest.importorskip("torch")
    n, d = 5000, 24
    lam = np.exp(-np.arange(1, d + 1) / 5.0)
    X, Q = synth.gaussian_data_torch(n, d, lam, 7, "cpu", torch.float32, chunk_rows=1024, image_like=True)
    Xd = X.double().numpy()
    assert np.abs(Xd.mean(axis=0)).max() <= 1e-6
    span = Xd.max(axis=0) - Xd.min(axis=0)
    assert span.max() <= 1.0 + 1e-6          # one global map to [0, 1], then per-column shifts
    assert np.abs(Q.T @ Q - np.eye(d)).max() <= 1e-13


def test_affine_to_unit_and_recentre_closed_form():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((50, 7)) * 3.0 + 1.0
    Y = synth.affine_to_unit_and_recentre(X)
    ref = (X - X.mean(axis=0, keepdims=True)) / (X.max() - X.min())
    assert np.abs(Y - ref).max() <= 1e-15
    assert np.abs(Y.mean(axis=0)).max() <= 1e-15


def test_batch_instances_ranges_and_determinism():
    a = synth.batch_instances(300, seed=11)
    assert a == synth.batch_instances(300, seed=11) and a != synth.batch_instances(300, seed=12)
    for s in a:
        assert 2000 <= s["n"] <= 200000
        assert s["d"] in (64, 128, 256, 512, 1024, 2048)
        assert 4 <= s["k"] <= 32 and s["m"] == 2 * s["k"] <= min(s["d"], 128)
        assert 0.8 <= s["rho"] <= 0.98
    assert len({s["seed"] for s in a}) == len(a)


def test_paper_synthetic_spectra():
    e = synth.paper_synthetic_spectrum("exponential")
    li = synth.paper_synthetic_spectrum("linear")
    assert e.shape == li.shape == (50,)
    assert e[0] == pytest.approx(1000.0) and e[-1] == pytest.approx(1.0)
    assert li[0] == pytest.approx(1000.0) and li[-1] == pytest.approx(1.0)
    assert np.allclose(e[1:] / e[:-1], (1.0 / 1000.0) ** (1.0 / 49))
    assert np.allclose(np.diff(li), -999.0 / 49)
    with pytest.raises(ValueError):
        synth.paper_synthetic_spectrum("cubic")


def test_initial_basis_is_seeded():
    a = synth.initial_basis(30, 4, 9)
    assert a.shape == (30, 4)
    assert np.array_equal(a, synth.initial_basis(30, 4, 9))
    assert not np.array_equal(a, synth.initial_basis(30, 4, 10))


def test_workload_configs_are_the_documented_ones():
    """Shapes, spectra, primer settings and tolerances of the five workloads."""
    C = synth.CONFIGS
    c1, c2, c3, c4, c5 = (C[k] for k in ("power_fp32_4096x256", "primers_fp32_100000x1024",
                                         "precision_bf16_1000000x4096", "batch512_fp32",
                                         "largeD_bf16_50000x262144"))
    i = np.arange(1, 4097, dtype=np.float64)
    assert (c1.n, c1.d, c1.k, c1.l, c1.dtype, c1.primers["power"]["T"]) == (4096, 256, 8, 8, "f32", 10)
    assert np.array_equal(c1.lam(), 0.9 ** i[:256])
    assert (c2.n, c2.d, c2.k, c2.l, c2.dtype, c2.primers["power"]["T"]) == (100000, 1024, 32, 32, "f32", 20)
    assert np.array_equal(c2.lam(), 1.0 / i[:1024])
    oja, eg = c2.primers["oja"], c2.primers["eigengame"]
    assert (oja["batch"], oja["epochs"], oja["lr0"], oja["lr_offset"]) == (256, 1, 1.0, 100.0)
    assert (eg["steps"], eg["batch"], eg["momentum"]) == (200, 1024, 0.9)
    assert (c3.n, c3.d, c3.k, c3.l, c3.dtype, c3.primers["power"]["T"]) == (1000000, 4096, 64, 64, "bf16", 15)
    assert np.array_equal(c3.lam(), np.exp(-i / 50.0)) and (c3.eig_rtol, c3.angle_tol) == (1e-4, 1e-3)
    assert c4.primers["power"]["T"] == 10
    assert (c5.n, c5.d, c5.k, c5.l, c5.dtype) == (50000, 262144, 32, 32, "bf16")
    eg5 = c5.primers["eigengame"]
    assert (eg5["steps"], eg5["batch"], eg5["momentum"]) == (500, 4096, 0.9)
    assert np.allclose(c5.lam()[:4], np.arange(1, 5) ** -1.5 + 1e-4, rtol=1e-15)
    assert (c5.eig_rtol, c5.angle_tol) == (1e-3, 1e-2)
    assert all(c.m == c.k + c.l for c in C.values())
