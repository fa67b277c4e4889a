"""Host-side logic of the Python layer (no GPU): plans released during a
CUDA-graph capture are destroyed after it, and the autotuner's cache keys
tell apart every plan setting that selects another kernel."""
import types

import pytest

from paper_2207_01205_gb300 import api, autotune


def test_plans_released_during_a_capture_are_destroyed_after_it(monkeypatch):
    destroyed = []
    monkeypatch.setattr(api.B, "fofse_plan_destroy", lambda h: destroyed.append(h))
    monkeypatch.setattr(api, "_deferred", [])
    monkeypatch.setattr(api, "_capturing", lambda: True)
    api._release(11)
    api._release(12)
    assert destroyed == [] and [h for _, h in api._deferred] == [11, 12]
    monkeypatch.setattr(api, "_capturing", lambda: False)
    api._release(13)
    assert sorted(destroyed) == [11, 12, 13] and api._deferred == []


def test_volume_plans_are_released_with_their_own_destroy(monkeypatch):
    destroyed = []
    monkeypatch.setattr(api.B, "fofse_plan_destroy", lambda h: destroyed.append(("2d", h)))
    monkeypatch.setattr(api.B, "fofse_volume_plan_destroy", lambda h: destroyed.append(("3d", h)))
    monkeypatch.setattr(api, "_deferred", [])
    monkeypatch.setattr(api, "_capturing", lambda: True)
    api._release(21)
    api._release(22, api.B.fofse_volume_plan_destroy)
    assert destroyed == []
    monkeypatch.setattr(api, "_capturing", lambda: False)
    api._destroy_deferred()
    assert sorted(destroyed) == [("2d", 21), ("3d", 22)]


def test_autotune_keys_separate_the_kernel_selecting_settings(monkeypatch):
    monkeypatch.setattr(autotune.torch.cuda, "get_device_name", lambda d=None: "GPU")
    base = dict(fft_size=64, block=16, border=16, iters=200, precision="fp32", support=0,
                compensation=0, basis=0)
    keys = set()
    for change in [{}, {"compensation": 1}, {"basis": 1}, {"precision": "fp64"}, {"support": 1},
                   {"iters": 100}, {"fft_size": 32}]:
        p = types.SimpleNamespace(**{**base, **change})
        keys.add(autotune._key(p, 804, 0))
    assert len(keys) == 7
    p = types.SimpleNamespace(**base)
    assert autotune._key(p, 700, 0) == autotune._key(p, 1000, 0)      # same power-of-two bucket
    assert autotune._key(p, 700, 0) != autotune._key(p, 1100, 0)


def test_volume_plan_arguments_are_checked_before_any_cuda_call():
    """fofse_volume_plan_create rejects invalid values (FOFSE_E_ARG) and grids
    without a kernel (FOFSE_E_UNSUPPORTED) before touching the device, and the
    batch call rejects a NULL plan; the library loads without a GPU."""
    from paper_2207_01205_gb300 import binding as B
    bad = [(0, 4, 1, 16, 4), (8, -1, 1, 16, 4), (8, 4, -1, 16, 4), (8, 5, 1, 16, 4),
           (8, 4, 2, 16, 4)]
    for args in bad:
        with pytest.raises(B.FofseError) as ei:
            B.fofse_volume_plan_create(*args, 0.8, 0.5, 10)
        assert ei.value.status == B.E_ARG, args
    for rho, gamma, iters in [(0.0, 0.5, 10), (1.5, 0.5, 10), (0.8, 0.0, 10), (0.8, 0.5, 0),
                              (0.8, 0.5, 5000), (float("nan"), 0.5, 10)]:
        with pytest.raises(B.FofseError) as ei:
            B.fofse_volume_plan_create(8, 4, 1, 16, 4, rho, gamma, iters)
        assert ei.value.status == B.E_ARG
    for args in [(8, 4, 1, 64, 8), (8, 4, 0, 128, 1), (8, 4, 1, 16, 16), (8, 4, 1, 16, 3),
                 (8, 4, 1, 48, 4)]:
        with pytest.raises(B.FofseError) as ei:
            B.fofse_volume_plan_create(*args, 0.8, 0.5, 10)
        assert ei.value.status == B.E_UNSUPPORTED, args
    L = B.load()
    st = L.fofse_extrapolate_volume_batch(None, None, 1, None, None, 1, 1, 1, 1, None, None,
                                          None, None, None, None, None)
    assert st == B.E_ARG
    assert L.fofse_volume_plan_set_precision(None, 0) == B.E_ARG
    assert L.fofse_volume_workspace_bytes(None, 10) == 0
    assert L.fofse_volume_plan_variant_count(None) == 0
    assert L.fofse_volume_plan_set_variant(None, 0) == B.E_ARG
    assert L.fofse_volume_backward(None, None, 1, None, None, 1, 1, 1, 1, None, None, None, None,
                                   None, None, None, None, None) == B.E_ARG
    assert L.fofse_volume_backward_workspace_bytes(None, 10) == 0


def test_volume_batch_rejects_host_tensors_and_wrong_dtypes():
    """The binding checks every tensor it hands to the C ABI as a device
    pointer (no GPU needed: the checks run before the call)."""
    import torch
    from paper_2207_01205_gb300 import binding as B
    n = 2
    blocks = torch.zeros((n, 3), dtype=torch.int32)
    video = torch.zeros((3, 8, 8), dtype=torch.float32)
    avail = torch.ones((3, 8, 8), dtype=torch.uint8)
    out = torch.zeros((n, 4, 4), dtype=torch.float32)
    with pytest.raises(ValueError, match="CUDA"):
        B.fofse_extrapolate_volume_batch(1, blocks, video, avail, out_blocks=out)

    class OnDevice:  # a host tensor that reports itself as a CUDA tensor
        is_cuda = True

        def __init__(self, t):
            self.t, self.dtype, self.shape = t, t.dtype, t.shape

        def __getattr__(self, k):
            return getattr(self.t, k)

    with pytest.raises(ValueError, match="int32"):
        B._require(OnDevice(blocks.long()), "blocks", torch.int32, (n, 3))
    with pytest.raises(ValueError, match="shape"):
        B._require(OnDevice(torch.zeros((3, 3), dtype=torch.int32)), "blocks", torch.int32, (2, 3))
    with pytest.raises(ValueError, match="contiguous"):
        B._require(OnDevice(torch.zeros((2, 6), dtype=torch.int32)[:, ::2]), "blocks", torch.int32)
    B._require(OnDevice(blocks), "blocks", torch.int32, (n, 3))
    with pytest.raises(ValueError, match="required"):
        B._require(None, "out_blocks", torch.float32)
    B._require(None, "path", torch.int32, optional=True)


def test_volume_backward_rejects_host_tensors_and_wrong_dtypes():
    """The backward's binding checks its tensors before the C call too."""
    import torch
    from paper_2207_01205_gb300 import binding as B
    n, it = 2, 5
    blocks = torch.zeros((n, 3), dtype=torch.int32)
    video = torch.zeros((3, 8, 8), dtype=torch.float32)
    avail = torch.ones((3, 8, 8), dtype=torch.uint8)
    path = torch.zeros((n, it, 3), dtype=torch.int32)
    coef = torch.zeros((n, it, 2), dtype=torch.float64)
    w0 = torch.ones((n,), dtype=torch.float64)
    gb = torch.zeros((n, 4, 4), dtype=torch.float32)
    with pytest.raises(ValueError, match="CUDA"):
        B.fofse_volume_backward(1, blocks, video, avail, path, coef, w0, gb)
    with pytest.raises(ValueError, match="float64"):
        B.fofse_volume_backward(1, blocks, video, avail, path, coef.float(), w0, gb)
