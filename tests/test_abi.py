"""The C-ABI library loads and exports every entry point include/ppca.h declares.

Runs without a GPU: only calls that the library answers from argument checks
alone (before any CUDA call) are made here.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ppca.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2109_03709_gb300 import build as b
    b.build()
    import paper_2109_03709_gb300 as P
    return P.load_library()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^PPCA_API\s+[\w\s\*]*?\b(ppca_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_expected_entry_points():
    import paper_2109_03709_gb300 as P
    assert declared_functions() == sorted(P.EXPORTED_SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_version_and_defaults(lib):
    import paper_2109_03709_gb300 as P
    assert P.ppca_version() >> 16 == 1
    oja = P.ppca_prime_params_default(P.PPCA_OJA)
    assert oja.batch == 256 and oja.lr == 1.0 and oja.lr_offset == 100.0
    eg = P.ppca_prime_params_default(P.PPCA_EIGENGAME)
    assert eg.batch == 1024 and eg.momentum == 0.9
    assert P.ppca_prime_params_default(P.PPCA_POWER_SEQ).eps == 1e-6
    with pytest.raises(P.PPCAError) as ei:
        P.ppca_prime_params_default(7)
    assert ei.value.status_name == "PPCA_ERR_INVALID"


def test_argument_checks_need_no_device(lib):
    import paper_2109_03709_gb300 as P
    out = ctypes.c_void_p(123)
    # NULL X
    assert lib.ppca_create(ctypes.byref(out), None, 10, 4, 4, P.PPCA_F32, None, None) == 1
    assert out.value is None
    assert "NULL" in P.ppca_last_error()
    fake = 1 << 20   # any 16-byte aligned address: rejected before it is touched
    assert lib.ppca_create(ctypes.byref(out), fake, 1, 4, 4, P.PPCA_F32, None, None) == 1       # n < 2
    assert lib.ppca_create(ctypes.byref(out), fake, 10, 4, 3, P.PPCA_F32, None, None) == 1      # ld < d
    assert lib.ppca_create(ctypes.byref(out), fake, 10, 3, 3, P.PPCA_F32, None, None) == 1      # 12-byte pitch
    assert lib.ppca_create(ctypes.byref(out), fake + 4, 10, 4, 4, P.PPCA_F32, None, None) == 1  # misaligned
    assert lib.ppca_create(ctypes.byref(out), fake, 10, 16, 16, P.PPCA_FP8_E4M3, None, None) == 1  # no scales
    assert lib.ppca_create(ctypes.byref(out), fake, 10, 16, 16, P.PPCA_F32, fake, None) == 1    # stray scales
    assert lib.ppca_create(ctypes.byref(out), fake, 10, 16, 16, 9, None, None) == 1             # dtype
    # NULL handle everywhere
    params = P.ppca_prime_params()
    assert lib.ppca_prime(None, 0, 4, 1, ctypes.byref(params)) == 1
    assert lib.ppca_finalize(None, 1, fake, fake, 0) == 1
    assert lib.ppca_upload(None, fake, 4, None) == 1
    assert lib.ppca_finalize_host(None, 1, fake, fake, 0) == 1
    assert lib.ppca_finalize_sampled(None, 1, fake, fake, 0, 0.1, 1, None) == 1
    assert lib.ppca_variance_captured(None, fake, 1, fake, 0) == 1
    assert lib.ppca_sync(None) == 1
    assert lib.ppca_destroy(None) == 0
    assert lib.ppca_quantize_bf16(None, 4, 4, 4, fake, 4, None) == 1
    assert lib.ppca_quantize_fp8(fake, 4, 8, 4, fake, 8, fake, None) == 1   # ld_in < d


def test_every_handle_or_batch_call_rejects_null(lib):
    """Each entry point that takes a handle or a batch answers a NULL one with
    PPCA_ERR_INVALID before any CUDA call (so no device is needed here)."""
    import paper_2109_03709_gb300 as P
    fake = 1 << 20
    i64, i32 = ctypes.c_int64(0), ctypes.c_int32(0)
    sched, timing = P.ppca_schedule(), P.ppca_timing()
    out = ctypes.c_void_p(123)
    statuses = {
        "ppca_set_refine": lib.ppca_set_refine(None, fake, 4, P.PPCA_F32),
        "ppca_set_workspace_limit": lib.ppca_set_workspace_limit(None, 0),
        "ppca_prime_continue": lib.ppca_prime_continue(None, 1),
        "ppca_get_basis": lib.ppca_get_basis(None, fake),
        "ppca_set_schedule": lib.ppca_set_schedule(None, ctypes.byref(sched)),
        "ppca_autotune": lib.ppca_autotune(None, 4, 0, 1, ctypes.byref(sched)),
        "ppca_set_timing": lib.ppca_set_timing(None, 1),
        "ppca_get_timing": lib.ppca_get_timing(None, ctypes.byref(timing)),
        "ppca_get_state": lib.ppca_get_state(None, None, ctypes.byref(i64)),
        "ppca_set_state": lib.ppca_set_state(None, fake, 64),
        "ppca_xpass": lib.ppca_xpass(None, fake, 4, 0, 1, fake, 0),
        "ppca_projected_gram": lib.ppca_projected_gram(None, fake, 4, 0, 1, fake, 0),
        "ppca_orthonormalize": lib.ppca_orthonormalize(None, fake, fake, 4),
        "ppca_eigh": lib.ppca_eigh(None, fake, 4, fake, fake),
        "ppca_eigh_noalloc": lib.ppca_eigh_noalloc(None, 4, fake, fake, None, None),
        "ppca_batch_create": lib.ppca_batch_create(ctypes.byref(out), None, 0, 0, None),
        "ppca_batch_run": lib.ppca_batch_run(None),
        "ppca_batch_autotune": lib.ppca_batch_autotune(None, 1, ctypes.byref(i32)),
        "ppca_batch_kernel_count": lib.ppca_batch_kernel_count(None, ctypes.byref(i64)),
        "ppca_batch_sync": lib.ppca_batch_sync(None),
    }
    for name, st in statuses.items():
        assert st == P.PPCA_ERR_INVALID, name
    assert out.value is None                      # ppca_batch_create cleared *out
    assert lib.ppca_batch_destroy(None) == P.PPCA_OK


def test_binding_constants_match_the_header_enums():
    import paper_2109_03709_gb300 as P
    text = open(HEADER).read()
    values = {name: int(v) for name, v in re.findall(r"^\s+(PPCA_[A-Z0-9_]+)\s*=\s*(\d+)", text, flags=re.M)}
    assert len(values) == 18               # status 8, dtype 3, method 4, precision 3
    for name, v in values.items():
        assert getattr(P, name) == v, name


def test_every_declaration_cites_its_passage_or_says_it_has_none():
    """Each entry point's comment either cites the passage of the paper that
    defines what it computes (Section, Algorithm or Eq.) or states that it has
    no counterpart in the paper (library infrastructure)."""
    lines = open(HEADER).read().split("\n")
    missing, text = [], ""
    for i, line in enumerate(lines):
        m = re.match(r"PPCA_API\s+[\w\s\*]*?\b(ppca_\w+)\s*\(", line)
        if not m:
            continue
        j, block = i - 1, []
        while j >= 0 and not lines[j].startswith(("PPCA_API", "typedef", "}")):
            block.append(lines[j])
            j -= 1
        if any(b.strip().startswith(("/*", "*")) for b in block):   # else: shares the previous comment
            text = " ".join(block)
        if not re.search(r"Section|Algorithm|Eq\.|no counterpart", text):
            missing.append(m.group(1))
    assert missing == [], missing


def test_wait_limit_above_a_minute_is_refused(lib):
    """ppca_set_wait_limit validates its argument before any CUDA call."""
    import paper_2109_03709_gb300 as P
    assert lib.ppca_set_wait_limit(61 * 10 ** 9) == P.PPCA_ERR_INVALID
