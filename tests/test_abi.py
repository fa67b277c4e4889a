"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point declared in include/fofse.h; host-side argument validation."""
import ctypes

import pytest

from paper_2207_01205_gb300 import binding as B


@pytest.fixture(scope="module")
def lib():
    return B.load()


def test_every_declared_symbol_is_exported(lib):
    names = B.header_functions()
    assert {"fofse_plan_create", "fofse_extrapolate_batch", "fofse_backward"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_the_probes_live_in_their_own_library(lib):
    """The measurement probes (include/fofse_probes.h) are exported by
    libfofse_probes.so, and the product library exports none of them."""
    names = B.header_functions(B.PROBES_HEADER)
    assert names == ["fofse_probe_dfma", "fofse_probe_fma", "fofse_probe_smem"]
    probes = B.load_probes()
    for n in names:
        assert hasattr(probes, n), n
        with pytest.raises(AttributeError):
            getattr(lib, n)
    assert not set(names) & set(B.header_functions())


def test_the_binding_has_a_function_of_each_name(lib):
    """The Python binding mirrors the C ABI name for name."""
    names = B.header_functions() + B.header_functions(B.PROBES_HEADER)
    assert {"fofse_volume_plan_create", "fofse_extrapolate_volume_batch", "fofse_probe_dfma"} <= set(names)
    for n in names:
        assert callable(getattr(B, n, None)), n


def test_status_strings_and_version(lib):
    for s in range(7):
        assert B.fofse_status_string(s) != "unknown status"
    assert B.fofse_status_string(99) == "unknown status"
    assert B.fofse_version() >= 100


@pytest.mark.parametrize("args", [
    (0, 16, 64, 0.8, 0.5, 200),        # block < 1
    (16, -1, 64, 0.8, 0.5, 200),       # border < 0
    (16, 16, 48, 0.8, 0.5, 200),       # T not a power of two
    (16, 25, 64, 0.8, 0.5, 200),       # T < block + 2 border
    (16, 16, 64, 0.0, 0.5, 200),       # rho out of (0, 1]
    (16, 16, 64, 1.5, 0.5, 200),
    (16, 16, 64, 0.8, 0.0, 200),       # gamma out of (0, 1]
    (16, 16, 64, 0.8, 1.01, 200),
    (16, 16, 64, 0.8, 0.5, 0),         # iters < 1
    (16, 16, 64, float("nan"), 0.5, 10),
])
def test_plan_create_rejects_invalid_arguments(lib, args):
    h = ctypes.c_void_p()
    assert lib.fofse_plan_create(*args, ctypes.byref(h)) == B.E_ARG
    assert h.value is None


def test_plan_create_unsupported_fft_size(lib):
    h = ctypes.c_void_p()
    assert lib.fofse_plan_create(16, 16, 512, 0.8, 0.5, 10, ctypes.byref(h)) == B.E_UNSUPPORTED
    assert lib.fofse_plan_create(16, 16, 64, 0.8, 0.5, 10, None) == B.E_ARG


def test_batch_calls_reject_null_arguments(lib):
    null = ctypes.c_void_p()
    assert lib.fofse_extrapolate_batch(None, 1, null, 1, null, null, 8, 8, 8, null, null, null,
                                       null, null, null, null, null) == B.E_ARG
    assert lib.fofse_backward(None, 1, null, 1, null, null, 8, 8, 8, null, null, null, null, null,
                              null, null, null) == B.E_ARG
    assert lib.fofse_plan_set_support(None, 0) == B.E_ARG
    assert lib.fofse_plan_set_precision(None, 0) == B.E_ARG
    assert lib.fofse_workspace_bytes(None, 1, 10) == 0
    lib.fofse_plan_destroy(None)


def test_newer_entry_points_reject_null_arguments(lib):
    """Setters, the factor-returning batch call, the error curve and the
    probes validate their arguments on the host (no GPU needed)."""
    assert lib.fofse_plan_set_precision(None, 2) == B.E_ARG
    null = ctypes.c_void_p()
    assert lib.fofse_plan_set_compensation(None, 1) == B.E_ARG
    assert lib.fofse_plan_set_basis(None, 1) == B.E_ARG
    assert lib.fofse_plan_set_variant(None, 0) == B.E_ARG
    assert lib.fofse_plan_variant_count(None) == 0
    assert lib.fofse_extrapolate_batch_gamma(None, 1, null, 1, null, null, 8, 8, 8, null, null, null,
                                             null, null, null, null, null, null) == B.E_ARG
    assert lib.fofse_extrapolate_batch_noalloc(None, 1, null, 1, null, null, 8, 8, 8, null, null,
                                               null, null, null, null) == B.E_ARG
    assert lib.fofse_error_curve(None, 1, null, 1, null, null, 8, 8, 8, null, null) == B.E_ARG
    out = ctypes.c_double()
    probes = B.load_probes()
    assert probes.fofse_probe_smem(0, 1, null, ctypes.byref(out), null) == B.E_ARG
    assert probes.fofse_probe_fma(1, 0, null, ctypes.byref(out), null) == B.E_ARG
    assert probes.fofse_probe_smem(1, 1, None, ctypes.byref(out), null) == B.E_ARG
    assert probes.fofse_probe_dfma(1, 1, null, None, null) == B.E_ARG


def _foreign_plan():
    """A stand-in plan whose creating device (the first member of the plan
    struct) is 63, a device that is never current: the 2-D calls must refuse
    it before looking at anything else in it or launching."""
    buf = (ctypes.c_int32 * 2048)()
    buf[0] = 63
    return buf


def test_2d_calls_refuse_a_plan_of_another_device(lib):
    fake = _foreign_plan()
    plans = (ctypes.c_void_p * 1)(ctypes.addressof(fake))
    d = ctypes.c_void_p(256)  # never dereferenced: the call returns first
    null = ctypes.c_void_p()
    assert lib.fofse_extrapolate_batch(plans, 1, d, 1, d, d, 8, 8, 8, null, null, d, null, null,
                                       null, d, null) == B.E_ARG
    assert lib.fofse_extrapolate_batch_gamma(plans, 1, d, 1, d, d, 8, 8, 8, null, null, d, null,
                                             null, null, null, d, null) == B.E_ARG
    assert lib.fofse_extrapolate_batch_noalloc(plans, 1, d, 1, d, d, 8, 8, 8, null, d, null, null,
                                               null, null) == B.E_ARG
    assert lib.fofse_backward(plans, 1, d, 1, d, d, 8, 8, 8, null, d, d, d, d, null, d,
                              null) == B.E_ARG
    assert lib.fofse_error_curve(plans, 1, d, 1, d, d, 8, 8, 8, d, null) == B.E_ARG


def test_plan_shape_query_rejects_null(lib):
    v = ctypes.c_int()
    assert lib.fofse_plan_get_shape(None, ctypes.byref(v), None, None, None) == B.E_ARG


class _Called(Exception):
    pass


@pytest.fixture
def no_c_calls(monkeypatch):
    """Fails the test if a batch call reaches the C library."""
    def boom(*a, **k):
        raise _Called()
    L = B.load()
    for name in ("fofse_extrapolate_batch", "fofse_extrapolate_batch_gamma",
                 "fofse_extrapolate_batch_noalloc", "fofse_backward", "fofse_plan_get_shape",
                 "fofse_workspace_bytes"):
        monkeypatch.setattr(L, name, boom)


def _host_inputs():
    import torch
    blocks = torch.zeros((2, 3), dtype=torch.int32)
    frame = torch.zeros((32, 32), dtype=torch.float32)
    avail = torch.ones((32, 32), dtype=torch.uint8)
    return blocks, frame, avail


@pytest.mark.parametrize("call", ["batch", "gamma", "noalloc", "backward"])
def test_binding_rejects_host_tensors_and_wrong_dtypes_before_the_c_call(no_c_calls, call):
    import torch
    blocks, frame, avail = _host_inputs()

    def run(bl, fr, av):
        if call == "batch":
            B.fofse_extrapolate_batch([1], bl, fr, av)
        elif call == "gamma":
            B.fofse_extrapolate_batch_gamma([1], bl, fr, av)
        elif call == "noalloc":
            B.fofse_extrapolate_batch_noalloc([1], bl, fr, av)
        else:
            tr = torch.zeros((2, 4, 3), dtype=torch.int32)
            B.fofse_backward([1], bl, fr, av, tr, torch.zeros(2), torch.zeros((2, 4, 4)))

    with pytest.raises(ValueError, match="int32"):
        run(blocks.long(), frame, avail)
    with pytest.raises(ValueError, match="float32"):
        run(blocks, frame.double(), avail)
    with pytest.raises(ValueError, match="uint8"):
        run(blocks, frame, avail.bool())
    with pytest.raises(ValueError, match="CUDA"):
        run(blocks, frame, avail)
    with pytest.raises(ValueError, match=r"\(n, 3\)|shape"):
        run(blocks[:, :2].contiguous(), frame, avail)
