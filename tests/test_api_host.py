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
    assert destroyed == [] and api._deferred == [11, 12]
    monkeypatch.setattr(api, "_capturing", lambda: False)
    api._release(13)
    assert sorted(destroyed) == [11, 12, 13] and api._deferred == []


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
