"""Host-side checks of the C ABI: the library builds, loads, exports every symbol that
include/lbmrv.h declares, and rejects invalid arguments before touching the GPU."""
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "lbmrv.h")


def declared_symbols():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^LBMRV_API\s+[\w\s\*]+?\b(lbmrv_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_entry_points():
    names = declared_symbols()
    for expected in ("lbmrv_create", "lbmrv_step", "lbmrv_moments", "lbmrv_destroy",
                     "lbmrv_conserved", "lbmrv_init_equilibrium"):
        assert expected in names


def test_library_exports_every_declared_symbol():
    from paper_1312_3297_gb300 import binding as B

    lib = B.load()
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1312_3297_gb300 import binding as B

    bound = {name for name, _, _ in B.SIGNATURES}
    assert set(declared_symbols()) <= bound
    for name in declared_symbols():
        assert callable(getattr(B, name)), name


def test_version_and_state_bytes():
    from paper_1312_3297_gb300 import binding as B

    assert B.lbmrv_version() == 1
    assert B.lbmrv_state_bytes(B.LBMRV_D2Q9, (64, 32, 1), B.LBMRV_FP32) == 9 * 64 * 32 * 4
    assert B.lbmrv_state_bytes(B.LBMRV_D2Q9, (7, 5, 1), B.LBMRV_FP16) == 9 * 35 * 2
    assert B.lbmrv_state_bytes(B.LBMRV_D2Q9, (7, 5, 1), B.LBMRV_BF16) == 9 * 35 * 2
    assert B.lbmrv_state_bytes(B.LBMRV_D2Q9, (0, 5, 1), B.LBMRV_FP32) == -1
    assert B.lbmrv_state_bytes(B.LBMRV_D2Q9, (4, 5, 1), 7) == -1
    assert B.lbmrv_state_bytes(5, (4, 5, 1), 0) == -1
    assert B.lbmrv_state_bytes(B.LBMRV_D3Q19, (4, 5, 6), B.LBMRV_FP32) == 19 * 120 * 4
    assert B.lbmrv_state_bytes(B.LBMRV_D3Q19, (4, 5, 0), B.LBMRV_FP32) == -1


S_OK = [0, 0, 0, 1.4, 1.9, 1.9, 1.2, 1.2, 1.4]


@pytest.mark.parametrize("kwargs,status,fragment", [
    (dict(s=[0.5] + S_OK[1:]), -1, "s[0]"),
    (dict(s=S_OK[:2] + [0.1] + S_OK[3:]), -1, "s[2]"),
    (dict(s=S_OK[:5] + [float("nan")] + S_OK[6:]), -1, "s[5]"),
    (dict(dims=(0, 4, 1)), -1, "dims"),
    (dict(dims=(4, 4, 2)), -1, "dims"),
    (dict(dims=(1 << 16, 1 << 15, 1)), -1, "2^31"),
    (dict(lam=0.0), -1, "lambda"),
    (dict(lam=float("inf")), -1, "lambda"),
    (dict(umode=3), -1, "mode"),
    (dict(storage=9), -1, "storage"),
    (dict(lattice=1), -1, "s[3]"),
    (dict(lattice=4), -1, "lattice"),
    (dict(rho_ref=float("nan")), -1, "rho_ref"),
])
def test_create_rejects_invalid_arguments(kwargs, status, fragment):
    from paper_1312_3297_gb300 import binding as B

    args = dict(lattice=0, dims=(8, 8, 1), lam=1.0, s=S_OK, umode=1, storage=0, rho_ref=0.0)
    args.update(kwargs)
    with pytest.raises(B.LbmrvError) as ei:
        B.lbmrv_create(args["lattice"], args["dims"], args["lam"], args["s"], args["umode"],
                       args["storage"], args["rho_ref"])
    assert ei.value.status == status
    assert fragment in str(ei.value)


def test_create_rejects_mismatched_buffers():
    from paper_1312_3297_gb300 import binding as B

    with pytest.raises(B.LbmrvError) as ei:
        B.lbmrv_create(0, (8, 8, 1), 1.0, S_OK, 1, 0, 0.0, None, 4096, None)
    assert ei.value.status == B.LBMRV_E_INVAL
    with pytest.raises(B.LbmrvError):
        B.lbmrv_create(0, (8, 8, 1), 1.0, S_OK, 1, 0, 0.0, None, 4096, 4096)
    with pytest.raises(B.LbmrvError) as ei:
        B.lbmrv_create(0, (8, 8, 1), 1.0, S_OK, 1, 0, 0.0, None, 4100, 8192)
    assert "aligned" in str(ei.value)


def test_null_handle_calls_fail_cleanly():
    from paper_1312_3297_gb300 import binding as B

    for fn, args in [(B.lbmrv_step, (None, 1)), (B.lbmrv_set_stream, (None, None)),
                     (B.lbmrv_set_utilde, (None, None, 0.0, 0.0)),
                     (B.lbmrv_init_equilibrium, (None, None, None)),
                     (B.lbmrv_moments, (None, None, None)),
                     (B.lbmrv_set_kernel_width, (None, 1)),
                     (B.lbmrv_step_conserved, (None, 1)), (B.lbmrv_conserved3, (None,))]:
        with pytest.raises(B.LbmrvError) as ei:
            fn(*args)
        assert ei.value.status == B.LBMRV_E_INVAL
    assert B.lbmrv_time(None) == -1
    # a NULL output array is rejected before the handle is used
    assert B.load().lbmrv_step_conserved(None, 1, None) == B.LBMRV_E_INVAL
    B.lbmrv_destroy(None)


def test_null_handle_reference_calls_fail_cleanly():
    from paper_1312_3297_gb300 import binding as B

    for fn, args in [(B.lbmrv_set_reference, (None, 1.0, (0.0, 0.0))),
                     (B.lbmrv_set_reference_auto, (None, 1.0)),
                     (B.lbmrv_get_reference, (None,))]:
        with pytest.raises(B.LbmrvError) as ei:
            fn(*args)
        assert ei.value.status == B.LBMRV_E_INVAL


@pytest.mark.gpu
@pytest.mark.parametrize("bad", [0.0, 2.0, 2.5, -0.3])
def test_rates_outside_0_2_are_accepted_with_a_warning(bad):
    """A non-conserved rate outside (0, 2) leaves its moment undamped or amplified; the
    handle is created (or the rates replaced) and the last-error message holds a warning
    naming the rate. Rates inside (0, 2) leave no warning."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_3297_gb300 import binding as B

    s = list(S_OK)
    s[7] = bad
    h = B.lbmrv_create(0, (8, 8, 1), 1.0, s, 1, 0, 1.0)
    try:
        msg = B.lbmrv_last_error(h)
        assert "warning" in msg and "s[7]" in msg, msg
        assert "warning" in B.lbmrv_last_error(None)
        B.lbmrv_set_rates(h, S_OK)
        h2 = B.lbmrv_create(0, (8, 8, 1), 1.0, S_OK, 1, 0, 1.0)
        assert "warning" not in B.lbmrv_last_error(h2)
        s2 = list(S_OK)
        s2[4] = bad
        B.lbmrv_set_rates(h2, s2)
        assert "s[4]" in B.lbmrv_last_error(h2)
        B.lbmrv_destroy(h2)
    finally:
        B.lbmrv_destroy(h)


def test_product_has_no_cpu_fallback():
    """The product package never imports the oracle and has no CPU compute path."""
    pkg = os.path.join(ROOT, "paper_1312_3297_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith(".py"):
                src = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in src and "from oracle" not in src, fn
                assert "lbm_inputs" not in src, fn
