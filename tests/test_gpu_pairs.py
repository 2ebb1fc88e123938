"""The bra-list x ket-list form (lx_eri_pairs; the paper's engine interface, Section 3).

Each pair's H matrix, and on the split path its column scales and digit planes, is built
once per chunk and shared by every quartet of the chunk that contains it.  The shared
operands are the ones a quartet evaluated alone would build, so the pair form must equal
one-quartet-at-a-time evaluation bit for bit, chunked or not; and it must match the
oracle (FP64 path: 1e-11 of the largest integral; split path: max abs error 1e-10)."""
import numpy as np
import pytest

import oracle
from paper_2307_03452_gb300 import lx

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    torch.cuda.set_device(0)


def pair_basis(lbra=(5, 5), lket=(6, 6), nshell=3, seed=21, kmax=2):
    """nshell shells of each of the (at most two) distinct angular momenta, K in 1..kmax,
    centers in a 3-bohr cube: bra pairs from the first group, ket pairs from the second."""
    rng = np.random.default_rng(seed)
    ls = [lbra[0]] * nshell + [lbra[1]] * nshell + [lket[0]] * nshell + [lket[1]] * nshell
    K = rng.integers(1, kmax + 1, len(ls)).astype(np.int32)
    off = np.concatenate([[0], np.cumsum(K)[:-1]]).astype(np.int32)
    basis = {"l": np.asarray(ls, np.int32), "nprim": K, "prim_off": off, "center": rng.uniform(0, 3, (len(ls), 3)),
             "exps": np.exp(rng.uniform(np.log(0.1), np.log(10.0), K.sum())), "coefs": 1 - rng.uniform(0, 1, K.sum())}
    g = [list(range(k * nshell, (k + 1) * nshell)) for k in range(4)]
    bra = [(a, b) for a in g[0] for b in g[1]][: nshell + 1]
    ket = [(c, d) for c in g[2] for d in g[3]][: nshell + 2]
    return basis, bra, ket


def quartets_of(bra, ket):
    return [(a, b, c, d) for (a, b) in bra for (c, d) in ket]


@pytest.mark.parametrize("path", ["fp64", "split"])
def test_pair_form_matches_oracle(path):
    basis, bra, ket = pair_basis()
    got = lx.eri_pairs(basis, bra, ket, solid=True, path=path).cpu().numpy()
    ref, off = oracle.eri(basis, quartets_of(bra, ket), solid=True)
    ref = ref.reshape(got.shape)
    err = np.abs(got - ref).max()
    if path == "fp64":
        assert err <= 1e-11 * np.abs(ref).max(), f"max err {err:.3e}"
    else:
        assert err <= 1e-10, f"max abs err {err:.3e}"


@pytest.mark.parametrize("path", ["fp64", "split"])
@pytest.mark.parametrize("solid", [True, False])
def test_shared_pairs_equal_one_quartet_at_a_time(path, solid):
    basis, bra, ket = pair_basis(lbra=(4, 6), lket=(5, 4), seed=22)
    got = lx.eri_pairs(basis, bra, ket, solid=solid, path=path).cpu().numpy()
    for i, (a, b) in enumerate(bra):
        for j, (c, d) in enumerate(ket):
            one, _ = lx.eri(basis, [(a, b, c, d)], solid=solid, path=path)
            assert np.array_equal(got[i, j].ravel(), one.cpu().numpy()), f"quartet ({i}, {j})"


@pytest.mark.parametrize("path", ["fp64", "split"])
def test_pair_form_chunked_is_bitwise_identical(path):
    basis, bra, ket = pair_basis(nshell=4, seed=23)
    whole = lx.eri_pairs(basis, bra, ket, solid=True, path=path)
    pb = lx.PairBatch(basis, bra, ket, True, path=path)
    small = lx.eri_pairs(basis, bra, ket, solid=True, path=path, workspace_limit=pb.workspace_min())
    assert torch.equal(whole, small)
