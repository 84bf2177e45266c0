"""The Python binding refuses tensor arguments the library could not use, before
the call reaches the library: a host (CPU) tensor where a kernel reads or writes
device memory.  Host-buffer arguments take CPU tensors, and integer addresses
pass through unchecked.  Runs without a GPU: a handle with a NULL pointer stands
in for a real one, which the library itself rejects with PPCA_ERR_INVALID."""
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    from paper_2109_03709_gb300 import build as b
    b.build()
    import paper_2109_03709_gb300 as P
    P.load_library()
    return P


def test_host_tensors_are_refused_for_device_arguments(P):
    h = P.Handle(0, [])
    E = torch.empty((4, 8))
    lam = torch.empty(4, dtype=torch.float64)
    calls = {
        "ppca_create": lambda: P.ppca_create(E),
        "ppca_set_refine": lambda: P.ppca_set_refine(h, E),
        "ppca_prime": lambda: P.ppca_prime(h, P.PPCA_POWER, 4, 1, V0=E),
        "ppca_finalize": lambda: P.ppca_finalize(h, 4, E, lam),
        "ppca_finalize_sampled": lambda: P.ppca_finalize_sampled(h, 4, E, lam),
        "ppca_variance_captured": lambda: P.ppca_variance_captured(h, E, 4, lam),
        "ppca_get_basis": lambda: P.ppca_get_basis(h, E),
        "ppca_xpass": lambda: P.ppca_xpass(h, E, 4, 0, 8, E),
        "ppca_projected_gram": lambda: P.ppca_projected_gram(h, E, 4, 0, 8, lam),
        "ppca_orthonormalize": lambda: P.ppca_orthonormalize(h, E, E, 4),
        "ppca_eigh": lambda: P.ppca_eigh(h, lam, 2, lam, lam),
        "ppca_eigh_noalloc": lambda: P.ppca_eigh_noalloc(lam, 2, lam, lam),
        "ppca_quantize_bf16": lambda: P.ppca_quantize_bf16(E, E),
        "ppca_quantize_fp8": lambda: P.ppca_quantize_fp8(E, E, lam),
        "ppca_batch_create": lambda: P.ppca_batch_create([{"X": E, "k": 2, "m": 4, "T": 1, "E": E, "lam": lam}]),
    }
    for name, call in calls.items():
        try:
            call()
        except ValueError as e:
            assert "device memory" in str(e), name
        else:
            pytest.fail(f"{name} accepted a host tensor for a device argument")


def test_host_buffers_reach_the_library(P):
    h = P.Handle(0, [])
    E = torch.empty((4, 8))
    lam = torch.empty(4, dtype=torch.float64)
    for call in (lambda: P.ppca_finalize_host(h, 4, E, lam), lambda: P.ppca_upload(h, E)):
        with pytest.raises(P.PPCAError) as ei:
            call()
        assert ei.value.status_name == "PPCA_ERR_INVALID"       # the NULL handle, seen by the library


def test_addresses_and_none_pass_through(P):
    assert P._dev(4096, "x", 4) == 4096
    assert P._host(None, "x") is None
    t = torch.empty(3)
    assert P._host(t, "t", 4) == t.data_ptr()
    with pytest.raises(TypeError, match="8-byte"):
        P._host(t, "t", 8)
    with pytest.raises(ValueError, match="contiguous"):
        P._host(torch.empty((4, 4)).t(), "t", 4)
    assert P._host(torch.empty((4, 4))[:, :2], "t", 4, contiguous=False) is not None


def test_undersized_tensors_are_refused_for_the_eigensolves(P):
    """G and U must hold m*m values, w m and status one: a kernel given a smaller
    tensor would read or write past its end.  The sizes are checked before
    anything else, so host tensors show it here without a GPU."""
    h = P.Handle(0, [])
    f64 = dict(dtype=torch.float64)
    m = 4
    ok = dict(G=torch.empty(m * m, **f64), w=torch.empty(m, **f64), U=torch.empty(m * m, **f64))
    for bad, small in (("G", torch.empty(m * m - 1, **f64)), ("U", torch.empty(m * m - 1, **f64)),
                       ("w", torch.empty(m - 1, **f64))):
        args = dict(ok, **{bad: small})
        with pytest.raises(ValueError, match=f"{bad} holds"):
            P.ppca_eigh_noalloc(args["G"], m, args["w"], args["U"])
        with pytest.raises(ValueError, match=f"{bad} holds"):
            P.ppca_eigh(h, args["G"], m, args["w"], args["U"])
    with pytest.raises(ValueError, match="status holds"):
        P.ppca_eigh_noalloc(ok["G"], m, ok["w"], ok["U"], status=torch.empty(0, dtype=torch.int32))
