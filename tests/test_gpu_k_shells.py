"""k shells (l = 7), the library's largest angular momentum, on both paths.

At l = 7 every table grows past its l = 6 size: L reaches 28 (4495 Hermite indices per
quartet, 36 Boys orders), a shell has 36 Cartesian and 15 solid components, and the
factorised solid fold of (k k) pairs needs 5688 Q rows and 13542 W rows of shared memory.
Each stage is compared with the oracle: the [r]^(0) vectors at L = 28, H of pairs with a k
shell, and whole (kk|kk) and mixed-k batches on the FP64 path (1e-11 of each class's
largest integral) and the split path (max abs error 1e-10)."""
import numpy as np
import pytest

import oracle
from paper_2307_03452_gb300 import inputs, lx

from test_gpu_parity import R_SENS_FACTOR, oracle_H, run_and_check, tuv_list

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K_CLASSES = [(7, 6, 7, 5), (7, 0, 3, 7), (2, 7, 7, 1), (7, 7, 4, 4)]


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    torch.cuda.set_device(0)


def test_hermite_R_stage_at_L28():
    rng = np.random.default_rng(28)
    n = 37
    rho = np.exp(rng.uniform(np.log(0.02), np.log(40), n))
    PQ = rng.uniform(-4, 4, (n, 3))
    PQ[0] = 0.0
    PQ[1] = [9.0, -7.0, 5.0]  # T > 36: the upward recursion from F_0
    pref = np.exp(rng.uniform(-2, 2, n))
    R = lx.hermite_R(28, torch.tensor(np.column_stack([rho, PQ, pref]), device="cuda")).cpu().numpy()
    idx = tuv_list(28)
    for i in range(n):
        box = oracle.hermite_R(28, rho[i], PQ[i], pref[i])
        ref = np.array([box[t, u, v] for t, u, v in idx])
        # as at L <= 26: 2e-12 of the largest entry plus R_SENS_FACTOR times the oracle's own
        # change under a 16-ulp move of rho or PQ (Eq. md1 is ill-conditioned at high L)
        dlt = 16 * 2.2e-16
        s1 = oracle.hermite_R(28, rho[i] * (1 + dlt), PQ[i], pref[i])
        s2 = oracle.hermite_R(28, rho[i], PQ[i] * (1 + dlt), pref[i])
        sens = max(np.abs(s1 - box).max(), np.abs(s2 - box).max())
        assert np.abs(R[i] - ref).max() <= 2e-12 * np.abs(ref).max() + R_SENS_FACTOR * sens, f"item {i}"


@pytest.mark.parametrize("solid", [False, True])
def test_hermite_H_of_k_pairs(solid):
    pairs_l = [(7, 7), (7, 0), (0, 7), (7, 6), (3, 7)]
    ls = [x for pr in pairs_l for x in pr]
    rng = np.random.default_rng(7)
    K = rng.integers(1, 3, len(ls)).astype(np.int32)
    off = np.concatenate([[0], np.cumsum(K)[:-1]]).astype(np.int32)
    basis = {"l": np.asarray(ls, np.int32), "nprim": K, "prim_off": off, "center": rng.uniform(0, 3, (len(ls), 3)),
             "exps": np.exp(rng.uniform(np.log(0.05), np.log(50), K.sum())), "coefs": 1 - rng.uniform(0, 1, K.sum())}
    pairs = [(2 * i, 2 * i + 1) for i in range(len(pairs_l))]
    for ket_sign in (False, True):
        H, _ = lx.hermite_H(basis, pairs, solid, ket_sign)
        H = H.cpu().numpy()
        for k, (sa, sb) in enumerate(pairs):
            ref = oracle_H(basis, sa, sb, solid, ket_sign)
            got = H[k, :ref.size].reshape(ref.shape)
            assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), f"pair {pairs_l[k]} ket_sign {ket_sign}"


def test_kkkk_fp64_both_outputs():
    basis, quartets = inputs.uniform_class((7, 7, 7, 7), 2, 77, cube=3.0, exps=(0.05, 20.0))
    for solid in (True, False):
        run_and_check(basis, quartets, solid)


def _mixed_k():
    parts = [inputs.uniform_class(c, 2, 78 + i, cube=3.0, exps=(0.05, 20.0), kmin=1, kmax=2)
             for i, c in enumerate(K_CLASSES)]
    parts.append(inputs.uniform_class((6, 6, 6, 6), 2, 90, cube=3.0, exps=(0.05, 20.0)))
    # one compact quartet per class sets the class scale, as in any realistic batch (the
    # FP64 tolerance is relative to each class's largest integral)
    parts += [inputs.uniform_class(c, 1, 60 + i, cube=1.0, exps=(0.1, 5.0), kmin=1, kmax=2)
              for i, c in enumerate(K_CLASSES + [(6, 6, 6, 6)])]
    return inputs.concat(parts)


def test_mixed_k_classes_contracted_fp64():
    basis, quartets = _mixed_k()
    run_and_check(basis, quartets, True)


def test_k_classes_on_the_split_path():
    b1 = inputs.uniform_class((7, 7, 7, 7), 2, 77, cube=3.0, exps=(0.05, 20.0))
    basis, quartets = inputs.concat([b1, _mixed_k()])
    ref, roff = oracle.eri(basis, quartets, solid=True)
    out, off = lx.eri(basis, quartets, solid=True, path="split")
    assert np.array_equal(off, roff)
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    assert np.abs(got - ref).max() <= 1e-10, f"max abs err {np.abs(got - ref).max():.3e}"
