"""Pins of the oracle's contracted integrals (ab|cd) against things other than itself:
brute-force quadrature of the defining 6-D integral, the (ss|ss) closed form,
permutational symmetry, translation / axis-permutation / rotation invariance,
Schwarz positivity, the centre-derivative identity, and an independent
Obara-Saika evaluator."""
import math

import numpy as np
import pytest
from numpy.polynomial import hermite as H
from scipy.integrate import quad_vec

import oracle


def cart(l):
    return [(l - i, i - j, j) for i in range(l + 1) for j in range(i + 1)]


def make_basis(ls, centers, exps, coefs=None):
    """One shell per entry; exps[k] is the list of exponents of shell k."""
    ks = [len(e) for e in exps]
    off = np.concatenate([[0], np.cumsum(ks)[:-1]]).astype(np.int32)
    ex = np.concatenate([np.asarray(e, float) for e in exps])
    co = np.ones_like(ex) if coefs is None else np.concatenate([np.asarray(c, float) for c in coefs])
    return {"l": np.asarray(ls, np.int32), "nprim": np.asarray(ks, np.int32), "prim_off": off,
            "center": np.asarray(centers, float).reshape(-1, 3), "exps": ex, "coefs": co}


def eri4(ls, centers, exps, coefs=None, solid=False, normalize=True, method="md"):
    b = make_basis(ls, centers, exps, coefs)
    out, _ = oracle.eri(b, [[0, 1, 2, 3]], solid=solid, normalize=normalize, method=method)
    dims = [2 * l + 1 if solid else (l + 1) * (l + 2) // 2 for l in ls]
    return out.reshape(dims)


# ------------------------------------------------------------ brute force

def brute_force_raw(ls, centers, z):
    """[ab|cd] over unnormalised primitives from the definition: 1/r12 written as
    (2/sqrt(pi)) int_0^inf exp(-t^2 r12^2) dt, each Cartesian direction a 2-D
    Gaussian-polynomial integral done exactly by Gauss-Hermite quadrature after a
    Cholesky change of variables, and the t integral by adaptive quadrature.
    No Boys function, Hermite expansion or recursion is involved."""
    la, lb, lc, ld = ls
    A, B, C, D = [np.asarray(c, float) for c in centers]
    za, zb, zc, zd = z
    zp, zq = za + zb, zc + zd
    P, Q = (za * A + zb * B) / zp, (zc * C + zd * D) / zq
    pre = math.exp(-za * zb / zp * np.sum((A - B) ** 2) - zc * zd / zq * np.sum((C - D) ** 2))
    y, w = H.hermgauss(12)
    Y1, Y2 = np.meshgrid(y, y, indexing="ij")
    W = np.outer(w, w)

    def direction_table(k, t):
        # exponent  -(zp u^2 + zq v^2 + s (u - v + d)^2), s = t^2, u = x1 - P, v = x2 - Q:
        # quadratic form M = [[zp+s, -s], [-s, zq+s]], linear term 2 b.z with b = s d (1, -1);
        # completing the square leaves exp(-s d^2 zp zq / det M), det M = zp zq + s (zp + zq)
        s = t * t
        d = P[k] - Q[k]
        det = zp * zq + s * (zp + zq)
        M = np.array([[zp + s, -s], [-s, zq + s]])
        z0 = -s * d * np.array([zq, -zp]) / det
        Lc = np.linalg.cholesky(M)
        LinvT = np.linalg.inv(Lc.T)
        fac = math.exp(-s * d * d * zp * zq / det) / math.sqrt(det)
        u = z0[0] + LinvT[0, 0] * Y1 + LinvT[0, 1] * Y2
        v = z0[1] + LinvT[1, 0] * Y1 + LinvT[1, 1] * Y2
        x1, x2 = P[k] + u, Q[k] + v
        T = np.zeros((la + 1, lb + 1, lc + 1, ld + 1))
        for i in range(la + 1):
            for j in range(lb + 1):
                f1 = (x1 - A[k]) ** i * (x1 - B[k]) ** j
                for m in range(lc + 1):
                    for n in range(ld + 1):
                        T[i, j, m, n] = fac * np.sum(W * f1 * (x2 - C[k]) ** m * (x2 - D[k]) ** n)
        return T

    ca, cb, cc, cd = cart(la), cart(lb), cart(lc), cart(ld)

    def integrand(t):
        Tx, Ty, Tz = (direction_table(k, t) for k in range(3))
        out = np.empty((len(ca), len(cb), len(cc), len(cd)))
        for ia, a in enumerate(ca):
            for ib, b in enumerate(cb):
                for ic, c in enumerate(cc):
                    for id_, dd in enumerate(cd):
                        out[ia, ib, ic, id_] = (Tx[a[0], b[0], c[0], dd[0]] * Ty[a[1], b[1], c[1], dd[1]] *
                                                Tz[a[2], b[2], c[2], dd[2]])
        return out.reshape(-1)

    val, _ = quad_vec(integrand, 0.0, np.inf, epsabs=0.0, epsrel=1e-12, limit=400)
    return (2.0 / math.sqrt(math.pi) * pre * val).reshape(len(ca), len(cb), len(cc), len(cd))


@pytest.mark.parametrize("ls", [(0, 0, 0, 0), (1, 0, 0, 0), (0, 1, 1, 0), (1, 1, 1, 1), (2, 0, 1, 0),
                                (2, 1, 0, 2), (0, 2, 2, 1), (2, 2, 1, 1)])
def test_brute_force_quadrature(ls):
    rng = np.random.default_rng(sum(ls) * 7 + ls[0])
    centers = rng.uniform(-1.0, 1.0, (4, 3))
    z = np.exp(rng.uniform(np.log(0.3), np.log(3.0), 4))
    ref = brute_force_raw(ls, centers, z)
    got = eri4(ls, centers, [[x] for x in z], normalize=False)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


# ------------------------------------------------------------ closed form

def test_ssss_closed_form_contracted():
    rng = np.random.default_rng(5)
    centers = rng.uniform(0, 3, (4, 3))
    exps = [np.exp(rng.uniform(np.log(0.05), np.log(50), 3)) for _ in range(4)]
    coefs = [1.0 - rng.uniform(0, 1, 3) for _ in range(4)]
    got = eri4((0, 0, 0, 0), centers, exps, coefs)[0, 0, 0, 0]

    def norm_coefs(z, c):
        # s-type normaliser (2 zeta / pi)^(3/4); contracted self-overlap sum c'c' (pi/(zi+zj))^(3/2) = 1
        cn = c * (2 * z / math.pi) ** 0.75
        s = sum(cn[i] * cn[j] * (math.pi / (z[i] + z[j])) ** 1.5 for i in range(3) for j in range(3))
        return cn / math.sqrt(s)

    cs = [norm_coefs(e, c) for e, c in zip(exps, coefs)]
    A, B, C, D = centers
    ref = 0.0
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    a, b, c, d = exps[0][i], exps[1][j], exps[2][k], exps[3][l]
                    p, q = a + b, c + d
                    P, Q = (a * A + b * B) / p, (c * C + d * D) / q
                    rho = p * q / (p + q)
                    T = rho * np.sum((P - Q) ** 2)
                    F0 = 1.0 if T == 0 else math.sqrt(math.pi / (4 * T)) * math.erf(math.sqrt(T))
                    ref += (cs[0][i] * cs[1][j] * cs[2][k] * cs[3][l] * 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) *
                            math.exp(-a * b / p * np.sum((A - B) ** 2) - c * d / q * np.sum((C - D) ** 2)) * F0)
    assert got == pytest.approx(ref, rel=1e-13)


def test_ssss_self_repulsion():
    # a normalised s Gaussian with itself: (ss|ss) = 2 sqrt(zeta / pi)... for one center
    # (s s|s s) with all four on one center and equal exponents z: 2 pi^(5/2)/(p q sqrt(p+q)) N^4, p = q = 2z
    z = 1.7
    got = eri4((0, 0, 0, 0), np.zeros((4, 3)), [[z]] * 4)[0, 0, 0, 0]
    N = (2 * z / math.pi) ** 0.75
    ref = 2 * math.pi ** 2.5 / ((2 * z) ** 2 * math.sqrt(4 * z)) * N ** 4
    assert got == pytest.approx(ref, rel=1e-14)
    assert ref == pytest.approx(2 * math.sqrt(z / math.pi), rel=1e-14)


# ------------------------------------------------------------ symmetry / invariance

def random_quartet(ls, seed, K=2, spread=2.5):
    rng = np.random.default_rng(seed)
    centers = rng.uniform(0, spread, (4, 3))
    exps = [np.exp(rng.uniform(np.log(0.1), np.log(20), K)) for _ in range(4)]
    coefs = [1.0 - rng.uniform(0, 1, K) for _ in range(4)]
    return centers, exps, coefs


@pytest.mark.parametrize("ls", [(2, 1, 3, 0), (4, 5, 6, 4), (3, 3, 2, 2), (7, 3, 7, 1)])
def test_eightfold_symmetry(ls):
    centers, exps, coefs = random_quartet(ls, 11, K=2 if sum(ls) < 16 else 1)
    ref = eri4(ls, centers, exps, coefs)
    scale = np.abs(ref).max()
    perms = [((1, 0, 2, 3), (1, 0, 2, 3)), ((0, 1, 3, 2), (0, 1, 3, 2)), ((2, 3, 0, 1), (2, 3, 0, 1)),
             ((3, 2, 1, 0), (3, 2, 1, 0))]
    for order, axes in perms:
        got = eri4([ls[i] for i in order], centers[list(order)], [exps[i] for i in order], [coefs[i] for i in order])
        # got[x_order0, x_order1, ...] = ref[...]: bring back to ref's index order
        back = np.transpose(got, np.argsort(axes))
        assert np.abs(back - ref).max() <= 1e-12 * scale


@pytest.mark.parametrize("ls", [(2, 2, 1, 3), (5, 4, 4, 6)])
def test_translation_invariance(ls):
    centers, exps, coefs = random_quartet(ls, 12, K=2 if sum(ls) < 16 else 1)
    a = eri4(ls, centers, exps, coefs)
    b = eri4(ls, centers + np.array([1.3, -0.7, 2.1]), exps, coefs)
    assert np.abs(a - b).max() <= 1e-11 * np.abs(a).max()


@pytest.mark.parametrize("ls", [(2, 1, 1, 3), (4, 4, 5, 5)])
def test_axis_permutation(ls):
    # relabelling x <-> y on every center permutes the Cartesian components exactly
    centers, exps, coefs = random_quartet(ls, 13, K=2 if sum(ls) < 16 else 1)
    a = eri4(ls, centers, exps, coefs)
    b = eri4(ls, centers[:, [1, 0, 2]], exps, coefs)
    perm = []
    for l in ls:
        comps = cart(l)
        perm.append([comps.index((c[1], c[0], c[2])) for c in comps])
    a_sw = a[np.ix_(*perm)]
    assert np.abs(a_sw - b).max() <= 1e-12 * np.abs(a).max()


@pytest.mark.parametrize("ls", [(1, 2, 2, 1), (4, 6, 5, 4)])
def test_rotation_invariance_solid(ls):
    # each shell's 2l+1 solid functions form an orthogonal representation of rotations,
    # so the Frobenius norm of the solid block is rotation invariant
    centers, exps, coefs = random_quartet(ls, 14, K=2 if sum(ls) < 16 else 1)
    rng = np.random.default_rng(3)
    Qm, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(Qm) < 0:
        Qm[:, 0] *= -1
    a = eri4(ls, centers, exps, coefs, solid=True)
    b = eri4(ls, (centers - 1.0) @ Qm.T + 0.5, exps, coefs, solid=True)
    assert np.linalg.norm(b) == pytest.approx(np.linalg.norm(a), rel=1e-11)
    assert not np.allclose(a, b)


def test_schwarz_positivity():
    # the matrix (ab|a'b') over all components of two shell pairs is positive semidefinite,
    # hence |(ab|cd)| <= sqrt((ab|ab)(cd|cd))
    rng = np.random.default_rng(21)
    ls = [2, 3, 1, 2]
    centers = rng.uniform(0, 2, (4, 3))
    exps = [np.exp(rng.uniform(np.log(0.2), np.log(5), 2)) for _ in range(4)]
    coefs = [1.0 - rng.uniform(0, 1, 2) for _ in range(4)]
    b = make_basis(ls, centers, exps, coefs)
    pairs = [(0, 1), (2, 3)]
    quartets = [[p[0], p[1], q[0], q[1]] for p in pairs for q in pairs]
    out, off = oracle.eri(b, quartets)
    n = [(ls[p[0]] + 1) * (ls[p[0]] + 2) // 2 * (ls[p[1]] + 1) * (ls[p[1]] + 2) // 2 for p in pairs]
    M = np.zeros((sum(n), sum(n)))
    starts = [0, n[0]]
    k = 0
    for i in range(2):
        for j in range(2):
            M[starts[i]:starts[i] + n[i], starts[j]:starts[j] + n[j]] = out[off[k]:off[k] + n[i] * n[j]].reshape(n[i], n[j])
            k += 1
    assert np.allclose(M, M.T, atol=1e-13 * np.abs(M).max())
    ev = np.linalg.eigvalsh(M)
    assert ev.min() >= -1e-12 * ev.max()
    d = np.diag(M)
    assert np.all(np.abs(M) <= np.sqrt(np.outer(d, d)) * (1 + 1e-12) + 1e-15)


@pytest.mark.parametrize("ls", [(2, 1, 1, 2), (3, 0, 2, 1), (4, 2, 3, 3)])
def test_center_derivative_identity(ls):
    # d/dA_x [ab|cd] = 2 za [a+1_x b|cd] - a_x [a-1_x b|cd]  (unnormalised primitives)
    rng = np.random.default_rng(sum(ls))
    centers = rng.uniform(-1, 1, (4, 3))
    z = np.exp(rng.uniform(np.log(0.3), np.log(4), 4))
    la = ls[0]

    def ev(l0, cen):
        return eri4((l0,) + tuple(ls[1:]), cen, [[x] for x in z], normalize=False)

    def fd(h):
        cp, cm = centers.copy(), centers.copy()
        cp[0, 0] += h
        cm[0, 0] -= h
        return (ev(la, cp) - ev(la, cm)) / (2 * h)

    deriv = (4 * fd(5e-4) - fd(1e-3)) / 3  # Richardson
    up = ev(la + 1, centers)
    dn = ev(la - 1, centers) if la > 0 else None
    ref = np.zeros_like(deriv)
    cu, cd = cart(la + 1), cart(la - 1) if la > 0 else []
    for ia, (ax, ay, az) in enumerate(cart(la)):
        ref[ia] = 2 * z[0] * up[cu.index((ax + 1, ay, az))]
        if ax > 0:
            ref[ia] -= ax * dn[cd.index((ax - 1, ay, az))]
    assert np.abs(deriv - ref).max() <= 1e-7 * np.abs(ref).max()


@pytest.mark.parametrize("ls,K", [((1, 2, 0, 3), 3), ((3, 3, 3, 3), 2), ((4, 4, 4, 4), 2), ((5, 5, 5, 5), 1),
                                  ((4, 5, 6, 6), 1), ((4, 6, 5, 5), 1), ((6, 6, 6, 6), 1),
                                  ((7, 2, 5, 6), 1), ((7, 7, 7, 7), 1)])
@pytest.mark.parametrize("seed", [0, 1])
def test_md_matches_obara_saika(ls, K, seed):
    # The horizontal recursion of the Obara-Saika route cancels badly for separated centers
    # at high l (its own result moves by up to 1e-5 under a rigid translation), so the
    # comparison uses compact quartets and allows for the OS route's own rounding noise,
    # measured by translating the quartet; that noise must itself stay small.
    centers, exps, coefs = random_quartet(ls, 31 + sum(ls) + 100 * seed, K=K, spread=0.5)
    md = eri4(ls, centers, exps, coefs, method="md")
    os_ = eri4(ls, centers, exps, coefs, method="os")
    os_shift = eri4(ls, centers - centers.mean(0), exps, coefs, method="os")
    scale = np.abs(md).max()
    noise = np.abs(os_ - os_shift).max()
    assert noise <= 1e-11 * scale
    assert np.abs(md - os_).max() <= 1e-12 * scale + 4 * noise
