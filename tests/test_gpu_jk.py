"""Coulomb/exchange digestion (lx_eri_jk) against the oracle's J and K.

Bounds follow from the integrals' own errors: every J or K entry is a sum of integrals times
density elements, so its error is at most (largest integral error) x W, with W the sum of
the |D| entries that multiply it:
    W_J[mu, nu]  = sum over listed quartets containing (mu nu) of sum_{lam, sig} |D[lam, sig]|
    W_K[mu, lam] = sum over listed quartets containing (mu .. lam .) of sum_{nu, sig} |D[nu, sig]|
The largest integral error is measured on the same quartets through lx_eri_batch (on the
FP64 path it must itself be within 1e-11 of the largest integral).  The split path's error
grows with the size of a quartet's intermediates: this compact basis has integrals up to
0.6, where it reaches about 1e-10."""
import os

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


def jk_basis(ls=(4, 5, 6, 2, 0, 6, 7), seed=41):
    rng = np.random.default_rng(seed)
    K = rng.integers(1, 3, len(ls)).astype(np.int32)
    off = np.concatenate([[0], np.cumsum(K)[:-1]]).astype(np.int32)
    return {"l": np.asarray(ls, np.int32), "nprim": K, "prim_off": off, "center": rng.uniform(0, 2.5, (len(ls), 3)),
            "exps": np.exp(rng.uniform(np.log(0.1), np.log(8.0), K.sum())), "coefs": 1 - rng.uniform(0, 1, K.sum())}


def jk_quartets(nshell, n, seed):
    rng = np.random.default_rng(seed)
    q = rng.integers(0, nshell, (n, 4))
    # repeated shells and bra = ket among them
    q[0] = [0, 0, 0, 0]
    q[1] = [2, 5, 2, 5]
    q[2] = [6, 6, 1, 1]
    return q.astype(np.int32)


def weights(basis, quartets, D, solid):
    bf, nbf = oracle.function_offsets(basis, solid)
    nf = [2 * int(l) + 1 if solid else (int(l) + 1) * (int(l) + 2) // 2 for l in basis["l"]]
    A = np.abs(D)
    WJ, WK = np.zeros((nbf, nbf)), np.zeros((nbf, nbf))
    for a, b, c, d in quartets:
        WJ[bf[a]:bf[a] + nf[a], bf[b]:bf[b] + nf[b]] += A[bf[c]:bf[c] + nf[c], bf[d]:bf[d] + nf[d]].sum()
        WK[bf[a]:bf[a] + nf[a], bf[c]:bf[c] + nf[c]] += A[bf[b]:bf[b] + nf[b], bf[d]:bf[d] + nf[d]].sum()
    return WJ, WK


def density(nbf, seed, sym=True):
    D = np.random.default_rng(seed).standard_normal((nbf, nbf))
    return D + D.T if sym else D


@pytest.mark.parametrize("solid", [True, False])
@pytest.mark.parametrize("path", ["fp64", "split"])
def test_jk_matches_oracle(solid, path):
    basis = jk_basis()
    q = jk_quartets(len(basis["l"]), 14, 42)
    _, nbf = oracle.function_offsets(basis, solid)
    D = density(nbf, 43, sym=not solid)  # a non-symmetric D on one of the outputs
    Jr, Kr = oracle.jk(basis, q, D, solid)
    J, K = lx.eri_jk(basis, q, D, solid=solid, path=path)
    J, K = J.cpu().numpy(), K.cpu().numpy()
    WJ, WK = weights(basis, q, D, solid)
    ref, _ = oracle.eri(basis, q, solid=solid)
    ints, _ = lx.eri(basis, q, solid=solid, path=path)
    per_int = np.abs(ints.cpu().numpy() - ref).max()  # this path's own integral error here
    if path == "fp64":
        assert per_int <= 1e-11 * np.abs(ref).max()
    # the digestion adds the rounding of its sums (a few ulps of the largest term)
    tol_j = (per_int + 1e-14 * np.abs(ref).max()) * WJ
    tol_k = (per_int + 1e-14 * np.abs(ref).max()) * WK
    assert np.all(np.abs(J - Jr) <= tol_j)
    assert np.all(np.abs(K - Kr) <= tol_k)
    assert np.abs(Jr).max() > 0 and np.abs(Kr).max() > 0


def test_j_only_k_only_and_chunked():
    basis = jk_basis(seed=44)
    q = jk_quartets(len(basis["l"]), 20, 45)
    _, nbf = oracle.function_offsets(basis, True)
    D = density(nbf, 46)
    J, K = lx.eri_jk(basis, q, D, solid=True)
    Jo, none = lx.eri_jk(basis, q, D, solid=True, want="J")
    assert none is None
    none, Ko = lx.eri_jk(basis, q, D, solid=True, want="K")
    assert none is None
    jb = lx.JKBatch(basis, q, True)
    Jc, Kc = lx.eri_jk(basis, q, D, solid=True, workspace_limit=jb.workspace_min())
    # the same integrals each time; only the order of the atomic additions differs
    for a, b in ((J, Jo), (K, Ko), (J, Jc), (K, Kc)):
        assert torch.allclose(a, b, rtol=0, atol=1e-14 * float(a.abs().max()))


def test_jk_equals_digesting_the_stored_blocks_at_full_size():
    # 64 x 64 (ii|ii) pair lists (4096 quartets, 256 shells, nbf 3328): J and K from the
    # digestion kernel equal the same contractions of the stored integral blocks (torch on
    # the GPU), on both paths
    basis, bra, ket = inputs.iiii_pairs()
    q = np.array([(a, b, c, d) for (a, b) in bra for (c, d) in ket], np.int32)
    nbf = 13 * len(basis["l"])
    D = torch.tensor(density(nbf, 47), device="cuda")
    for path in ("fp64", "split"):
        J, K = lx.eri_jk(basis, q, D, solid=True, path=path)
        blocks = lx.eri_pairs(basis, bra, ket, solid=True, path=path)  # [64][64][169][169]
        I = blocks.view(len(bra), len(ket), 13, 13, 13, 13)
        Dv = D.view(len(basis["l"]), 13, len(basis["l"]), 13)
        ba, bb = torch.tensor(bra[:, 0], device="cuda"), torch.tensor(bra[:, 1], device="cuda")
        kc, kd = torch.tensor(ket[:, 0], device="cuda"), torch.tensor(ket[:, 1], device="cuda")
        Dcd = Dv[kc, :, kd, :]                       # [ket][lam][sig]
        Jref = torch.zeros_like(D).view(len(basis["l"]), 13, len(basis["l"]), 13)
        jb = torch.einsum("ijmnls,jls->imn", I, Dcd)  # [bra][mu][nu]
        Jref[ba, :, bb, :] += jb
        Kref = torch.zeros_like(Jref)
        for i in range(len(bra)):
            # an int index keeps its place: Dv[b, :, kd, :] is [nu][ket][sig]
            Dbd = Dv[int(bra[i, 1]), :, kd, :].permute(1, 0, 2)  # [ket][nu][sig]
            kb = torch.einsum("jmnls,jns->jml", I[i], Dbd)        # [ket][mu][lam]
            Kref[int(bra[i, 0]), :, kc, :] += kb.permute(1, 0, 2)  # [mu][ket][lam]
        Jref, Kref = Jref.view(nbf, nbf), Kref.view(nbf, nbf)
        for got, ref in ((J, Jref), (K, Kref)):
            assert float((got - ref).abs().max()) <= 1e-13 * float(ref.abs().max()), path


def test_routed_jk_within_the_split_bound():
    from paper_2307_03452_gb300 import router as rt
    if not os.path.exists(rt.WEIGHTS):
        pytest.skip("no trained router")
    r = rt.Router.load()
    lx.router_set(r.p16, r.tau)
    basis = jk_basis(seed=48)
    q = jk_quartets(len(basis["l"]), 16, 49)
    _, nbf = oracle.function_offsets(basis, True)
    D = density(nbf, 50)
    Jr, Kr = oracle.jk(basis, q, D, True)
    J, K = lx.eri_jk(basis, q, D, solid=True, path="routed")
    WJ, WK = weights(basis, q, D, True)
    ref, _ = oracle.eri(basis, q, solid=True)
    ints, _ = lx.eri(basis, q, solid=True, path="routed")
    per_int = np.abs(ints.cpu().numpy() - ref).max() + 1e-14 * np.abs(ref).max()
    assert np.all(np.abs(J.cpu().numpy() - Jr) <= per_int * WJ)
    assert np.all(np.abs(K.cpu().numpy() - Kr) <= per_int * WK)


@pytest.mark.parametrize("path", ["fp64", "split"])
def test_jk_largest_blocks(path):
    # (kk|kk) Cartesian: 36^4 blocks; on the FP64 path the direct kernel stages one column of
    # X and H_cd at a time (its widest chunk that leaves room for two CTAs per SM)
    basis = jk_basis(ls=(7, 7, 7, 7), seed=51)
    q = np.array([[0, 1, 2, 3], [2, 3, 0, 1]], np.int32)
    _, nbf = oracle.function_offsets(basis, False)
    D = density(nbf, 52)
    Jr, Kr = oracle.jk(basis, q, D, False)
    J, K = lx.eri_jk(basis, q, D, solid=False, path=path)
    WJ, WK = weights(basis, q, D, False)
    ref, _ = oracle.eri(basis, q, solid=False)
    ints, _ = lx.eri(basis, q, solid=False, path=path)
    per_int = np.abs(ints.cpu().numpy() - ref).max() + 1e-14 * np.abs(ref).max()
    assert np.all(np.abs(J.cpu().numpy() - Jr) <= per_int * WJ)
    assert np.all(np.abs(K.cpu().numpy() - Kr) <= per_int * WK)
