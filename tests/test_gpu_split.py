"""The split path: Ozaki-style BF16 slice products on the tcgen05 tensor cores.

lx_split_gemm (C = A B^T) is checked first on integer-valued matrices whose split is exact,
so the tensor-core result must equal the FP64 product bit for bit (this pins the operand
layout, the descriptors and the recombination), then on random matrices against the
error bound of 48-bit operands, and on long positive rows, where the FP32 tensor-core
accumulators would round unless they are drained to 64-bit integers often enough.  The ERI
split path is checked against the oracle at max abs error 1e-10 on split-path classes."""
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


SHAPES = [(1, 1, 1), (128, 96, 32), (129, 97, 33), (300, 200, 455), (455, 169, 455), (64, 16, 1000), (7, 250, 70)]


@pytest.mark.parametrize("digits", [4, 5, 6])
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_split_gemm_exact_on_integer_rows(M, N, K, digits):
    # rows: integers |x| < 2^12 times a per-row power of two -> only the top two digits of each
    # value are nonzero, so even 4 digits (products s + t <= 3) represent every product exactly,
    # every partial sum stays exact, and C must equal the FP64 product exactly
    rng = np.random.default_rng(M * 1000 + N + K)
    A = rng.integers(-4095, 4096, (M, K)).astype(np.float64) * np.exp2(rng.integers(-20, 20, (M, 1)))
    B = rng.integers(-4095, 4096, (N, K)).astype(np.float64) * np.exp2(rng.integers(-20, 20, (N, 1)))
    ref = A @ B.T
    C = lx.split_gemm(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"), digits=digits).cpu().numpy()
    assert np.array_equal(C, ref)


@pytest.mark.parametrize("digits", [4, 5, 6])
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_split_gemm_random_within_bound(M, N, K, digits):
    # operands of 8 d bits (x = q 2^(e-48) truncated to d digits, |x| < 2^e <= 2|x|max) and the
    # dropped digit products (s + t >= d) cost at most a few units of 2^(eA+eB-8d) per k:
    # |C - AB^T| <= K * 2^(5-8d) * max_k|A_ik| * max_k|B_jk| (2^-43 for d = 6) with room to spare;
    # and one digit fewer must cost more than 2^6 of the error at the typical element
    rng = np.random.default_rng(7 + M + N + K)
    A = rng.normal(size=(M, K)) * np.exp(rng.uniform(-5, 5, (M, 1)))
    B = rng.normal(size=(N, K)) * np.exp(rng.uniform(-5, 5, (N, 1)))
    ref = A @ B.T
    At, Bt = torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")
    C = lx.split_gemm(At, Bt, digits=digits).cpu().numpy()
    scale = np.outer(np.abs(A).max(1), np.abs(B).max(1))
    bound = K * 2.0 ** (5 - 8 * digits) * scale
    assert np.all(np.abs(C - ref) <= bound)
    if digits > 4 and K >= 32:
        Cf = lx.split_gemm(At, Bt, digits=digits - 1).cpu().numpy()
        assert np.median(np.abs(Cf - ref) / scale) > 2.0 ** 6 * np.median(np.abs(C - ref) / scale)


@pytest.mark.parametrize("K", [300, 4096, 20000])
def test_split_gemm_long_positive_rows_stay_exact(K):
    # entries in [1, 2): every leading digit is 128..256, so one diagonal grows by ~2^15 per k
    # and passes 2^24 after a few hundred k.  Rounding there would cost ~1e-6 relative; the
    # periodic int64 drains keep the error at the 48-bit bound (K = 20000 also takes the
    # extra shift that keeps the 64-bit sum clear of overflow).
    rng = np.random.default_rng(K)
    A = rng.uniform(1.0, 2.0, (40, K))
    B = rng.uniform(1.0, 2.0, (24, K))
    ref = A @ B.T
    C = lx.split_gemm(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")).cpu().numpy()
    bound = K * 2.0 ** -43 * np.outer(np.abs(A).max(1), np.abs(B).max(1))
    assert np.all(np.abs(C - ref) <= bound), f"max rel err {np.abs(C / ref - 1).max():.3e}"


def _split_vs_oracle(basis, quartets, solid):
    out, off = lx.eri(basis, quartets, solid=solid, path="split")
    ref, roff = oracle.eri(basis, quartets, solid=solid)
    got = out.cpu().numpy()
    return got, ref, off


@pytest.mark.parametrize("solid", [True, False])
def test_eri_split_path_hhhh_iiii(solid):
    # (hh|hh) and (ii|ii), K = 1..3 per shell, compact and far quartets: max abs error <= 1e-10
    b1 = inputs.uniform_class((5, 5, 5, 5), 4, 91, cube=3.0, exps=(0.05, 20.0), kmin=1, kmax=2)
    b2 = inputs.uniform_class((6, 6, 6, 6), 3, 92, cube=3.0, exps=(0.05, 20.0), kmin=1, kmax=2)
    b3 = inputs.uniform_class((5, 5, 5, 5), 2, 93, cube=20.0, exps=(0.05, 20.0), kmin=1, kmax=3)
    basis, quartets = inputs.concat([b1, b2, b3])
    got, ref, _ = _split_vs_oracle(basis, quartets, solid)
    assert np.all(np.isfinite(got))
    assert np.abs(got - ref).max() <= 1e-10, f"max abs err {np.abs(got - ref).max():.3e}"


def test_eri_split_path_mixed_and_low_l():
    # every class the library accepts goes through the split path too
    mixed = inputs.mixed_classes(8, seed=94, kmin=1, kmax=2, cube=4.0)
    low = inputs.uniform_class((1, 0, 2, 3), 5, 95, cube=3.0, exps=(0.1, 10.0), kmin=1, kmax=3)
    basis, quartets = inputs.concat([mixed, low])
    got, ref, _ = _split_vs_oracle(basis, quartets, True)
    assert np.abs(got - ref).max() <= 1e-10


def test_split_and_fp64_paths_agree_on_full_size_iiii():
    # the 4096-quartet (ii|ii) workload: split path vs the FP64 path, max abs difference
    basis, quartets = inputs.iiii_fp64()
    a, _ = lx.eri(basis, quartets, solid=True, path="fp64")
    b, _ = lx.eri(basis, quartets, solid=True, path="split")
    assert float((a - b).abs().max()) <= 1e-10


def test_both_paths_at_maximum_contraction():
    # K = 16 on every shell, the library's limit.  The bra reduction of (ff|ss) and the ket
    # reduction of (ss|ff) are 256 x 84 = 21504 > 2^14 long, so the split path's 64-bit sums
    # take the extra shift in GEMM1 and in GEMM2; (dd|dd) with K = 8 rides along.
    b1 = inputs.uniform_class((3, 3, 0, 0), 2, 97, cube=3.0, exps=(0.1, 10.0), kmin=16, kmax=16)
    b2 = inputs.uniform_class((0, 0, 3, 3), 2, 99, cube=3.0, exps=(0.1, 10.0), kmin=16, kmax=16)
    b3 = inputs.uniform_class((2, 2, 2, 2), 1, 98, cube=3.0, exps=(0.1, 10.0), kmin=8, kmax=8)
    basis, quartets = inputs.concat([b1, b2, b3])
    ref, roff = oracle.eri(basis, quartets, solid=True)
    for path in ("split", "fp64"):
        out, off = lx.eri(basis, quartets, solid=True, path=path)
        assert np.array_equal(off, roff)
        err = np.abs(out.cpu().numpy() - ref).max()
        assert err <= 1e-10, f"{path}: max abs err {err:.3e}"


def test_split_and_routed_on_degenerate_geometry():
    # all four shells on one center (T = 0, P = A) with exponents from 0.05 to 50, plus a pair
    # of coincident centers far from the other pair: split and routed paths against the oracle
    ls = [6, 6, 5, 4]
    basis = {"l": np.asarray(ls, np.int32), "nprim": np.array([1, 2, 1, 1], np.int32),
             "prim_off": np.array([0, 1, 3, 4], np.int32), "center": np.zeros((4, 3)),
             "exps": np.array([50.0, 0.05, 3.0, 0.05, 20.0]), "coefs": np.array([1.0, 0.3, 0.7, 1.0, 1.0])}
    far = {k: v.copy() for k, v in basis.items()}
    far["center"] = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [9.0, 0.0, 0.0], [9.0, 0.0, 0.0]])
    b, q = inputs.concat([(basis, np.array([[0, 1, 2, 3], [3, 2, 1, 0]], np.int32)),
                          (far, np.array([[0, 1, 2, 3]], np.int32))])
    ref, roff = oracle.eri(b, q, solid=True)
    from paper_2307_03452_gb300 import router as rt
    import os
    paths = ["split"] + (["routed"] if os.path.exists(rt.WEIGHTS) else [])
    for path in paths:
        if path == "routed":
            r = rt.Router.load()
            lx.router_set(r.p16, r.tau)
        out, off = lx.eri(b, q, solid=True, path=path)
        assert np.array_equal(off, roff)
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= 1e-10, f"{path}: {np.abs(got - ref).max():.3e}"
