"""lx_eri_batch_static: the batch evaluation for callers that cannot allocate device memory
(their device memory is owned by a pool they cannot reach, or cudaMalloc is not permitted
where they run).  It uses the library's fixed device scratch array instead of a workspace.

Checked through the C ABI against lx_eri_batch on two different batches in a row (the
array keeps the first call's contents when the second one runs); one batch needs several
chunks of the array.  Collected last on purpose: a failure here leaves every other test run.
"""
import numpy as np
import pytest

from paper_2307_03452_gb300 import inputs, lx

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_ERI = 1e-11  # same bound as the parity tests: 1e-11 of the largest |integral|


def _reference(batch):
    ref = torch.empty(batch.out_size, dtype=torch.float64, device="cuda")
    batch.run(ref, lx.alloc_workspace(batch.workspace_size()))
    lx.sync_status()
    return ref


def test_static_scratch_matches_workspace_path_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    torch.cuda.set_device(0)
    # call 1: 48 (ii|ii) quartets, solid -- about 90 MB of workspace, so several chunks
    b1 = lx.Batch(*inputs.uniform_class((6, 6, 6, 6), 48, 77, cube=3.0, exps=(0.05, 20.0)), solid=True)
    assert b1.workspace_size() > lx.STATIC_SCRATCH_BYTES
    # call 2: mixed classes, contracted, Cartesian
    b2 = lx.Batch(*inputs.mixed_classes(10, seed=78, kmin=1, kmax=2, cube=3.0), solid=False)
    for b in (b1, b2):
        ref = _reference(b)
        out = torch.full_like(ref, float("nan"))
        lx.run_static(b, out)
        lx.sync_status()
        err = float((out - ref).abs().max())
        scale = float(ref.abs().max())
        assert err <= TOL_ERI * scale, f"static-scratch result differs: {err:.3e} vs scale {scale:.3e}"


def test_static_scratch_rejects_oversized_batch():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    # (ii|ii) with K = 5 on every shell, Cartesian: one quartet alone needs > 64 MiB
    basis, quartets = inputs.uniform_class((6, 6, 6, 6), 1, 79, kmin=5, kmax=5)
    b = lx.Batch(basis, quartets, solid=False)
    assert b.workspace_min() > lx.STATIC_SCRATCH_BYTES
    out = torch.empty(b.out_size, dtype=torch.float64, device="cuda")
    with pytest.raises(lx.LxError) as e:
        lx.run_static(b, out)
    assert e.value.code == -11


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")
def test_static_scratch_refuses_capture_and_stage_timing():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    torch.cuda.set_device(0)
    basis, quartets = inputs.uniform_class((2, 1, 2, 0), 3, 132, cube=3.0, exps=(0.2, 5.0))
    b = lx.Batch(basis, quartets, solid=True)
    out = torch.empty(b.out_size, dtype=torch.float64, device="cuda")
    lx.run_static(b, out)  # device set-up and the symbol lookup happen outside any capture
    lx.sync_status()
    ref = out.clone()
    # the descriptors are uploaded from host memory released on return: a capturing stream
    # is refused before anything is enqueued, and the capture ends cleanly (empty graph)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    code = None
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            lx.run_static(b, out, stream=s)
        except lx.LxError as exc:
            code = exc.code
        finally:
            g.capture_end()
    torch.cuda.synchronize()
    assert code == -7
    # stage timing would create CUDA events: refused with LX_ERR_FLAGS
    with pytest.raises(lx.LxError) as e:
        lx.run_static(b, out, time_stages=True)
    assert e.value.code == -5
    torch.cuda.synchronize()
    assert torch.equal(out, ref)  # neither refused call wrote anything
