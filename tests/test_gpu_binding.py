"""The Python binding checks every tensor it hands to the C ABI as a device
pointer (dtype, CUDA, device, size against the plans' shapes) and raises
before the call, so an undersized or misplaced buffer never reaches a kernel."""
import pytest
import torch

from paper_2207_01205_gb300 import api, binding

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(gpu_lib):
    return gpu_lib


def _case():
    plans = [api.Plan(16, 16, 64, 0.8, 0.5, 10), api.Plan(8, 8, 32, 0.8, 0.5, 12)]
    frame = torch.zeros((96, 96), device="cuda")
    avail = torch.ones((96, 96), dtype=torch.uint8, device="cuda")
    blocks = torch.tensor([[16, 16, 0], [64, 64, 1]], dtype=torch.int32, device="cuda")
    return plans, [p.handle for p in plans], frame, avail, blocks


def test_plan_shape_query():
    plans, handles, *_ = _case()
    assert binding.fofse_plan_get_shape(handles[0]) == (16, 16, 64, 10)
    assert binding.fofse_plan_get_shape(handles[1]) == (8, 8, 32, 12)


@pytest.mark.parametrize("what", ["out_blocks", "trace", "w0", "status", "workspace", "rho_gamma"])
def test_batch_call_rejects_undersized_outputs(what):
    plans, handles, frame, avail, blocks = _case()
    n = 2
    ob, tr, w0, st = api.alloc_outputs(plans, n, "cuda")   # bmax 16, imax 12
    ws = api.workspace(plans, n, "cuda")
    kw = dict(out_blocks=ob, trace=tr, w0=w0, status=st, workspace=ws)
    small = {"out_blocks": torch.empty((n, 8, 8), device="cuda"),
             "trace": torch.empty((n, 10, 3), dtype=torch.int32, device="cuda"),
             "w0": torch.empty((1,), device="cuda"),
             "status": torch.empty((1,), dtype=torch.int32, device="cuda"),
             "workspace": ws[:16],
             "rho_gamma": torch.empty((1, 2), device="cuda")}
    kw[what] = small[what]
    with pytest.raises(ValueError, match=what):
        binding.fofse_extrapolate_batch(handles, blocks, frame, avail, **kw)
    # the full-size buffers pass
    binding.fofse_extrapolate_batch(handles, blocks, frame, avail, out_blocks=ob, trace=tr, w0=w0,
                                    status=st, workspace=ws)
    torch.cuda.synchronize()


def test_calls_reject_host_tensors_wrong_dtypes_and_mismatched_frames():
    plans, handles, frame, avail, blocks = _case()
    ob, tr, w0, st = api.alloc_outputs(plans, 2, "cuda")
    with pytest.raises(ValueError, match="CUDA"):
        binding.fofse_extrapolate_batch(handles, blocks, frame.cpu(), avail.cpu())
    with pytest.raises(ValueError, match="status"):
        binding.fofse_extrapolate_batch(handles, blocks, frame, avail, status=w0)
    with pytest.raises(ValueError, match="out_frame"):
        binding.fofse_extrapolate_batch(handles, blocks, frame, avail, out_frame=frame[:, :64])
    with pytest.raises(ValueError, match="avail"):
        binding.fofse_extrapolate_batch(handles, blocks, frame, avail[:, :64])
    gb = torch.zeros_like(ob)
    with pytest.raises(ValueError, match="grad_frame"):
        binding.fofse_backward(handles, blocks, frame, avail, tr, w0, gb,
                               grad_frame=torch.zeros((8, 8), device="cuda"))
    with pytest.raises(ValueError, match="grad_blocks"):
        binding.fofse_backward(handles, blocks, frame, avail, tr, w0, gb[:, :8, :8].contiguous())
    with pytest.raises(ValueError, match="trace"):
        binding.fofse_backward(handles, blocks, frame, avail, tr[:, :5].contiguous(), w0, gb)


def test_a_plan_whose_settings_fail_is_destroyed_once():
    """A plan whose creation succeeds but whose settings are refused is
    destroyed by the constructor and never again by the finaliser (a second
    destroy would free its device tables twice)."""
    import gc
    with pytest.raises(binding.FofseError):
        api.Plan(8, 4, 32, 0.8, 0.5, 10, basis=7)
    with pytest.raises(binding.FofseError):
        api.VolumePlan(32, 16, 0, 64, 1, 0.8, 0.5, 10, precision="fp64")
    gc.collect()
    p, v = api.Plan(8, 4, 32, 0.8, 0.5, 10), api.VolumePlan(8, 4, 1, 16, 4, 0.8, 0.5, 10)
    assert p.handle and v.handle
