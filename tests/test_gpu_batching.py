"""Mixed-class batches: FP64 GEMM tile shapes, the autotuner, and whole-batch CUDA graphs.

Every tile shape accumulates each output element in the same order, so all shapes give
bit-identical results; a graph replay must equal a direct call bit for bit as well."""
import numpy as np
import pytest

import oracle
from paper_2307_03452_gb300 import inputs, lx

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    torch.cuda.set_device(0)
    lx.tune_clear()
    yield
    lx.tune_clear()


def _mixed(n=30, seed=40, kmax=3):
    return inputs.mixed_classes(n, seed=seed, kmin=1, kmax=kmax, cube=4.0)


def _run(batch, ws_bytes=None):
    out = torch.full((batch.out_size,), float("nan"), dtype=torch.float64, device="cuda")
    batch.run(out, lx.alloc_workspace(ws_bytes or batch.workspace_size()))
    lx.sync_status()
    return out


def _keys(basis, quartets, solid):
    l, K = basis["l"], basis["nprim"]
    return sorted({(int(l[a]), int(l[b]), int(l[c]), int(l[d]), int(K[a] * K[b]), int(K[c] * K[d]), int(solid))
                   for a, b, c, d in quartets})


@pytest.mark.parametrize("solid", [True, False])
def test_every_tile_shape_gives_identical_results(solid):
    basis, quartets = _mixed()
    b = lx.Batch(basis, quartets, solid)
    lx.tune_clear()
    ref = _run(b)
    for v1 in range(4):
        v2 = 3 - v1
        lx.tune_import([k + (v1, v2) for k in _keys(basis, quartets, solid)])
        got = _run(b)
        assert torch.equal(got, ref), f"shapes {v1}, {v2}"
    lx.tune_clear()


def test_graph_replay_equals_direct_call_chunked():
    basis, quartets = _mixed(n=24, seed=41)
    b = lx.Batch(basis, quartets, True)
    ref = _run(b)
    ws = lx.alloc_workspace(max(b.workspace_min(), b.workspace_size() // 3))  # several chunks
    out = torch.full_like(ref, float("nan"))
    g = lx.Graph(b, out, ws)
    for _ in range(3):
        out.fill_(float("nan"))
        g.launch()
        lx.sync_status()
        assert torch.equal(out, ref)
    g.close()


def test_graph_of_split_path():
    basis, quartets = _mixed(n=12, seed=42, kmax=2)
    b = lx.Batch(basis, quartets, True, path="split")
    ref = _run(b)
    out = torch.zeros_like(ref)
    g = lx.Graph(b, out, lx.alloc_workspace(b.workspace_size()))
    g.launch()
    lx.sync_status()
    assert torch.equal(out, ref)
    g.close()


def test_autotune_records_valid_choices_and_keeps_results():
    basis, quartets = _mixed(n=40, seed=43)
    b = lx.Batch(basis, quartets, True)
    lx.tune_clear()
    ref = _run(b)
    rows = lx.autotune(b, max_keys=4, samples=4)
    assert 1 <= len(rows) <= 4
    keys = set(_keys(basis, quartets, True))
    for r in rows:
        assert tuple(int(x) for x in r[:7]) in keys
        assert 0 <= r[7] < 4 and 0 <= r[8] < 4
    assert torch.equal(_run(b), ref)
    lx.tune_clear()


def test_mixed_contracted_batch_against_oracle():
    # quartets of the batched workload (five classes, K = 1..5 per shell); the oracle judges
    # those whose primitive count keeps it fast, every output is finite
    basis, quartets = inputs.mixed_fp64(nquartet=300, seed=2309)
    b = lx.Batch(basis, quartets, True)
    out = torch.empty(b.out_size, dtype=torch.float64, device="cuda")
    ws = lx.alloc_workspace(min(b.workspace_size(), 8 << 30))
    g = lx.Graph(b, out, ws)
    g.launch()
    lx.sync_status()
    assert bool(torch.isfinite(out).all())
    K = basis["nprim"]
    cheap = [i for i, (a, bb, c, d) in enumerate(quartets) if K[a] * K[bb] * K[c] * K[d] <= 4][:12]
    assert len(cheap) >= 4
    sb, sq = inputs.subset(basis, quartets, cheap)
    ref, roff = oracle.eri(sb, sq, solid=True)
    off = b.quartets["out_offset"]
    got = np.concatenate([out[off[i]:off[i] + b.sizes[i]].cpu().numpy() for i in cheap])
    # class-relative bound against the largest integral of each class over the whole batch
    l = basis["l"]
    scale = {}
    for i, q in enumerate(quartets):
        cls = tuple(int(l[s]) for s in q)
        scale[cls] = max(scale.get(cls, 0.0), float(out[off[i]:off[i] + b.sizes[i]].abs().max()))
    pos = 0
    for j, i in enumerate(cheap):
        n = int(b.sizes[i])
        cls = tuple(int(l[s]) for s in quartets[i])
        assert np.abs(got[pos:pos + n] - ref[pos:pos + n]).max() <= 1e-11 * scale[cls]
        pos += n
    g.close()


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")
def test_batch_call_refuses_a_capturing_stream():
    # lx_eri_batch stages its uploads in reused pinned buffers, so it must not be captured;
    # it says so before touching the stream, and the capture ends cleanly (empty graph)
    basis, quartets = inputs.uniform_class((2, 1, 2, 0), 3, 131, cube=3.0, exps=(0.2, 5.0))
    b = lx.Batch(basis, quartets, solid=True)
    out = torch.empty(max(b.out_size, 1), dtype=torch.float64, device="cuda")
    ws = lx.alloc_workspace(b.workspace_size())
    b.run(out, ws)  # device set up outside the capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    s.wait_stream(torch.cuda.current_stream())
    code = None
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            b.run(out, ws, stream=s)
        except lx.LxError as exc:
            code = exc.code
        finally:
            g.capture_end()
    torch.cuda.synchronize()
    assert code == -7
