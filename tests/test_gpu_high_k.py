"""Parity at the largest contraction degrees of the batched and routed workloads.

The primitive sums sit inside the reduction index of the two transforms (paper, Section 2:
the cost of [p|q] and of the first transform grows with K_bra K_ket, that of the second with
K_ket), so quartets with K = 5 on every shell are the longest reductions the mixed-class and
routed workloads contain.  Each class of the mixed workload gets one such quartet, compared
element by element with the CPU oracle on every path:

* FP64 path, run as a captured graph (the batched form): within 1e-11 of the class's largest
  |integral|;
* split path and routed path: within 1e-10 absolute.

The routed workload (l = 4..6, K = 1..5 per shell, bra-ket separations up to 30 bohr) gets a
sample of far-separated quartets with K = 5 shells, and the full-size (ii|ii) batch gets a
sample of its Cartesian output (28^4 per quartet) in the launch configuration the benchmark
times.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2307_03452_gb300 import inputs, lx
from paper_2307_03452_gb300 import router as rt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-11  # of the class's largest |integral|
TOL_SPLIT = 1e-10  # absolute


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def k5_batch():
    """One quartet per mixed class, K = 5 on all four shells, exponents log-uniform in
    [0.05, 50] and raw coefficients uniform in (0, 1] as in the mixed workload, centers in a
    3-bohr cube so that every class has integrals of realistic size; the oracle's solid
    result (its (ii|ii) quartet takes about a minute of one CPU core)."""
    parts = [inputs.uniform_class(cls, 1, 900 + i, cube=3.0, exps=(0.05, 50.0), kmin=5, kmax=5)
             for i, cls in enumerate(inputs.MIXED_CLASSES)]
    basis, quartets = inputs.concat(parts)
    assert np.all(basis["nprim"] == 5)
    ref, off = oracle.eri(basis, quartets, solid=True)
    return basis, quartets, ref, off


def _blocks(basis, quartets, off):
    l = basis["l"]
    for i, q in enumerate(quartets):
        n = int(np.prod([2 * l[s] + 1 for s in q]))
        yield i, tuple(int(l[s]) for s in q), slice(int(off[i]), int(off[i]) + n)


def test_k5_every_class_fp64_graph(k5_batch):
    basis, quartets, ref, off = k5_batch
    b = lx.Batch(basis, quartets, True)
    out = torch.full((b.out_size,), float("nan"), dtype=torch.float64, device="cuda")
    g = lx.Graph(b, out, lx.alloc_workspace(b.workspace_size()))
    g.launch()
    lx.sync_status()
    got = out.cpu().numpy()
    g.close()
    assert np.array_equal(b.quartets["out_offset"], off)
    for i, cls, sl in _blocks(basis, quartets, off):
        scale = np.abs(ref[sl]).max()
        err = np.abs(got[sl] - ref[sl]).max()
        assert scale > 1e-6, f"class {cls}: integrals too small to judge ({scale:.2e})"
        assert err <= TOL_FP64 * scale, f"class {cls}: FP64 err {err:.3e} > 1e-11 * {scale:.3e}"


def test_k5_every_class_split(k5_batch):
    basis, quartets, ref, off = k5_batch
    out, goff = lx.eri(basis, quartets, solid=True, path="split")
    assert np.array_equal(goff, off)
    got = out.cpu().numpy()
    for i, cls, sl in _blocks(basis, quartets, off):
        err = np.abs(got[sl] - ref[sl]).max()
        assert err <= TOL_SPLIT, f"class {cls}: split err {err:.3e}"


@pytest.mark.skipif(not os.path.exists(rt.WEIGHTS), reason="no trained router weights")
def test_k5_every_class_routed(k5_batch):
    basis, quartets, ref, off = k5_batch
    r = rt.Router.load()
    out, goff, _ = rt.routed_eri(basis, quartets, r)
    assert np.array_equal(goff, off)
    assert np.abs(out.cpu().numpy() - ref).max() <= TOL_SPLIT


def _oracle_seconds(basis, q):
    """Rough single-core oracle cost of one quartet (proportional to its primitive quartets
    times the Cartesian first-transform size; about 0.2 s for one (ii|ii) primitive quartet)."""
    l, K = basis["l"], basis["nprim"]
    la, lb, lc, ld = (int(l[s]) for s in q)
    pyr = lambda n: (n + 1) * (n + 2) * (n + 3) // 6  # noqa: E731
    nc = lambda x: (x + 1) * (x + 2) // 2  # noqa: E731
    work = pyr(la + lb) * pyr(lc + ld) * nc(la) * nc(lb) * float(np.prod([K[s] for s in q]))
    return 0.2 * work / (455 * 455 * 784)


@pytest.mark.skipif(not os.path.exists(rt.WEIGHTS), reason="no trained router weights")
def test_routed_workload_sample_with_k5_shells():
    # quartets of the routed workload's distribution (its generator, another seed): the first
    # 16 with a K = 5 shell whose oracle cost stays under ~40 s of one core, plus the first 8
    # with K = 5 on a whole pair; every path against the oracle
    basis, quartets = inputs.routed(nquartet=3000, seed=2411)
    K = basis["nprim"]
    pick, pair5 = [], []
    for i, q in enumerate(quartets):
        if _oracle_seconds(basis, q) > 40.0:
            continue
        if (K[q[0]] == 5 and K[q[1]] == 5) or (K[q[2]] == 5 and K[q[3]] == 5):
            if len(pair5) < 8:
                pair5.append(i)
        elif K[q].max() == 5 and len(pick) < 16:
            pick.append(i)
        if len(pick) == 16 and len(pair5) == 8:
            break
    idx = pick + pair5
    assert len(idx) == 24
    sb, sq = inputs.subset(basis, quartets, idx)
    ref, off = oracle.eri(sb, sq, solid=True)
    r = rt.Router.load()
    routed, roff, _ = rt.routed_eri(sb, sq, r)
    assert np.array_equal(roff, off)
    assert np.abs(routed.cpu().numpy() - ref).max() <= TOL_SPLIT
    split, _ = lx.eri(sb, sq, solid=True, path="split")
    assert np.abs(split.cpu().numpy() - ref).max() <= TOL_SPLIT
    # FP64 path: far-separated quartets are sums with heavy cancellation, so per quartet the
    # bound is 1e-11 of the quartet's largest integral plus 20 times the oracle's own rounding
    # noise (its change under a rigid translation of the quartet)
    fp64, _ = lx.eri(sb, sq, solid=True, path="fp64")
    got = fp64.cpu().numpy()
    moved = dict(sb)
    moved["center"] = sb["center"] + np.array([0.37, -1.1, 0.53])
    ref2, _ = oracle.eri(moved, sq, solid=True)
    for i, cls, sl in _blocks(sb, sq, off):
        noise = np.abs(ref[sl] - ref2[sl]).max()
        assert np.abs(got[sl] - ref[sl]).max() <= TOL_FP64 * np.abs(ref[sl]).max() + 20 * noise + 1e-300


def test_full_size_iiii_cartesian_sampled():
    # (ii|ii), 4096 quartets, Cartesian output (28^4 per quartet, 20 GB), one launch sequence
    # with the workspace the benchmark gives it; sampled quartets against the oracle, every
    # output finite
    basis, quartets = inputs.iiii_fp64()
    b = lx.Batch(basis, quartets, False)
    out = torch.empty(b.out_size, dtype=torch.float64, device="cuda")
    b.run(out, lx.alloc_workspace(b.workspace_size()))
    lx.sync_status()
    assert bool(torch.isfinite(out).all())
    sample = [0, 2, 1999, 3001, 4095]
    sb, sq = inputs.subset(basis, quartets, sample)
    ref, _ = oracle.eri(sb, sq, solid=False)
    n = 28 ** 4
    got = np.concatenate([out[i * n:(i + 1) * n].cpu().numpy() for i in sample])
    scale = float(out.abs().max())  # the class scale of the whole batch
    del out
    torch.cuda.empty_cache()
    assert np.abs(got - ref).max() <= TOL_FP64 * scale
