"""Seeded synthetic shell-quartet workloads.

This module only draws random inputs (centers, exponents, raw contraction
coefficients, angular momenta); it holds none of the integral arithmetic, so
both the CUDA library's tests and the CPU oracle can be fed from it.

A workload is a pair (basis, quartets):

* ``basis`` -- dict of per-shell arrays ``l`` (int32), ``nprim`` (int32),
  ``prim_off`` (int32, offset into the primitive arrays), ``center`` (nshell x 3,
  bohr) and per-primitive ``exps`` and raw ``coefs`` (float64).
* ``quartets`` -- (nq x 4) int32 shell indices (a, b, c, d).

Every quartet owns four fresh shells, as in the paper's microbenchmarks of one
integral class over synthetic shells (Section 4).
"""
from __future__ import annotations

import numpy as np

L_OF = {"s": 0, "p": 1, "d": 2, "f": 3, "g": 4, "h": 5, "i": 6, "k": 7}

#: the mixed classes of the batched workload: (gg|gg), (hh|hh), (ii|ii), (gh|ii), (gi|hh)
MIXED_CLASSES = [(4, 4, 4, 4), (5, 5, 5, 5), (6, 6, 6, 6), (4, 5, 6, 6), (4, 6, 5, 5)]


def class_of(name: str) -> tuple[int, int, int, int]:
    """'(gh|ii)' or 'ghii' -> (4, 5, 6, 6)."""
    letters = [c for c in name if c in L_OF]
    if len(letters) != 4:
        raise ValueError(f"not a quartet class: {name!r}")
    return tuple(L_OF[c] for c in letters)


def _loguniform(rng, lo, hi, n):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n))


def _assemble(ls, ks, centers, exps_lo, exps_hi, rng, coef_uniform):
    """Build the basis dict for shells with angular momenta ls and degrees ks."""
    ls = np.asarray(ls, dtype=np.int32)
    ks = np.asarray(ks, dtype=np.int32)
    off = np.zeros(len(ls), dtype=np.int32)
    if len(ls):
        off[1:] = np.cumsum(ks)[:-1]
    nprim = int(ks.sum())
    exps = _loguniform(rng, exps_lo, exps_hi, nprim)
    if coef_uniform:
        coefs = 1.0 - rng.uniform(0.0, 1.0, nprim)  # uniform in (0, 1]
    else:
        coefs = np.ones(nprim)
    return {"l": ls, "nprim": ks, "prim_off": off, "center": np.asarray(centers, dtype=np.float64).reshape(-1, 3),
            "exps": exps, "coefs": coefs}


def uniform_class(cls, nquartet, seed, cube=10.0, exps=(0.1, 10.0), kmin=1, kmax=1):
    """nquartet quartets of one class; centers uniform in a cube of side `cube` bohr,
    exponents log-uniform in `exps`, contraction degree per shell uniform in kmin..kmax,
    raw coefficients 1 (K = 1) or uniform in (0, 1] (K > 1)."""
    rng = np.random.default_rng(seed)
    nsh = 4 * nquartet
    ls = np.tile(np.asarray(cls, dtype=np.int32), nquartet)
    ks = rng.integers(kmin, kmax + 1, nsh).astype(np.int32)
    centers = rng.uniform(0.0, cube, (nsh, 3))
    basis = _assemble(ls, ks, centers, exps[0], exps[1], rng, coef_uniform=kmax > 1)
    quartets = np.arange(nsh, dtype=np.int32).reshape(nquartet, 4)
    return basis, quartets


def class_sweep(cls, nquartet, k_per_shell, seed, cube=20.0, exps=(0.05, 20.0)):
    """nquartet quartets of one class with fixed contraction degrees (K_a, K_b, K_c, K_d):
    centers uniform in a cube of side `cube` bohr; per shell one exponent log-uniform in
    `exps`, its K primitives spaced by factors of 3 around it; raw coefficients uniform in
    (0, 1] (1 for K = 1).  The paper's class x contraction table uses such batches."""
    rng = np.random.default_rng(seed)
    nsh = 4 * nquartet
    ls = np.tile(np.asarray(cls, dtype=np.int32), nquartet)
    ks = np.tile(np.asarray(k_per_shell, dtype=np.int32), nquartet)
    centers = rng.uniform(0.0, cube, (nsh, 3))
    mid = _loguniform(rng, exps[0], exps[1], nsh)
    off = np.zeros(nsh, dtype=np.int32)
    off[1:] = np.cumsum(ks)[:-1]
    spread = [3.0 ** (np.arange(k) - (k - 1) / 2.0) for k in range(max(k_per_shell) + 1)]
    e = np.concatenate([mid[i] * spread[ks[i]] for i in range(nsh)])
    c = np.where(np.repeat(ks, ks) > 1, 1.0 - rng.uniform(0.0, 1.0, int(ks.sum())), 1.0)
    basis = {"l": ls, "nprim": ks, "prim_off": off, "center": centers, "exps": e, "coefs": c}
    return basis, np.arange(nsh, dtype=np.int32).reshape(nquartet, 4)


def mixed_classes(nquartet, seed, classes=MIXED_CLASSES, cube=20.0, exps=(0.05, 50.0), kmin=1, kmax=5):
    """Quartets drawn uniformly over `classes`, K per shell uniform in kmin..kmax,
    exponents log-uniform, raw coefficients uniform in (0, 1]."""
    rng = np.random.default_rng(seed)
    pick = rng.integers(0, len(classes), nquartet)
    ls = np.asarray([classes[i] for i in pick], dtype=np.int32).reshape(-1)
    nsh = 4 * nquartet
    ks = rng.integers(kmin, kmax + 1, nsh).astype(np.int32)
    centers = rng.uniform(0.0, cube, (nsh, 3))
    basis = _assemble(ls, ks, centers, exps[0], exps[1], rng, coef_uniform=True)
    quartets = np.arange(nsh, dtype=np.int32).reshape(nquartet, 4)
    return basis, quartets


def spread_distances(nquartet, seed, lvals=(4, 5, 6), exps=(0.05, 50.0), kmin=1, kmax=5, pair_radius=3.0,
                     max_sep=30.0):
    """Quartets whose magnitudes span many decades: l per shell from `lvals`, the two
    centers of a pair within `pair_radius` bohr of each other, bra-ket separation uniform
    in [0, max_sep] bohr along a random direction."""
    rng = np.random.default_rng(seed)
    nsh = 4 * nquartet
    ls = rng.choice(np.asarray(lvals, dtype=np.int32), nsh).astype(np.int32)
    ks = rng.integers(kmin, kmax + 1, nsh).astype(np.int32)
    centers = np.zeros((nquartet, 4, 3))
    base = rng.uniform(0.0, 20.0, (nquartet, 3))
    d = rng.normal(size=(nquartet, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    sep = rng.uniform(0.0, max_sep, (nquartet, 1))
    for k, origin in enumerate([base, base, base + sep * d, base + sep * d]):
        u = rng.normal(size=(nquartet, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        centers[:, k] = origin + u * rng.uniform(0.0, pair_radius, (nquartet, 1))
    basis = _assemble(ls, ks, centers.reshape(-1, 3), exps[0], exps[1], rng, coef_uniform=True)
    quartets = np.arange(nsh, dtype=np.int32).reshape(nquartet, 4)
    return basis, quartets


def subset(basis, quartets, idx):
    """The shells and quartets of quartet indices `idx`, renumbered from 0."""
    idx = np.asarray(idx)
    qs = np.asarray(quartets)[idx]
    shells = qs.reshape(-1)
    ls = basis["l"][shells]
    ks = basis["nprim"][shells]
    off = np.zeros(len(shells), dtype=np.int32)
    if len(shells):
        off[1:] = np.cumsum(ks)[:-1]
    exps = np.concatenate([basis["exps"][o:o + k] for o, k in zip(basis["prim_off"][shells], ks)]) if len(shells) else np.zeros(0)
    coefs = np.concatenate([basis["coefs"][o:o + k] for o, k in zip(basis["prim_off"][shells], ks)]) if len(shells) else np.zeros(0)
    sub = {"l": ls.astype(np.int32), "nprim": ks.astype(np.int32), "prim_off": off, "center": basis["center"][shells],
           "exps": exps, "coefs": coefs}
    return sub, np.arange(len(shells), dtype=np.int32).reshape(-1, 4)


# Named workloads (sizes of the paper-shaped microbenchmarks).
def gggg_fp64(seed=2307):
    """(gg|gg): 64 quartets, l = 4, K = 1, 10-bohr cube, exponents in [0.1, 10]."""
    return uniform_class((4, 4, 4, 4), 64, seed, cube=10.0, exps=(0.1, 10.0))


def iiii_fp64(nquartet=4096, seed=2308):
    """(ii|ii): 4096 quartets, l = 6, K = 1, 20-bohr cube, exponents in [0.05, 20]."""
    return uniform_class((6, 6, 6, 6), nquartet, seed, cube=20.0, exps=(0.05, 20.0))


def mixed_fp64(nquartet=200_000, seed=2309):
    """Mixed classes (gg|gg),(hh|hh),(ii|ii),(gh|ii),(gi|hh), K = 1..5, exponents in [0.05, 50]."""
    return mixed_classes(nquartet, seed)


def split_hhhh_iiii(nquartet_each=16384, seed=2310):
    """(hh|hh) and (ii|ii), K = 1..3 per shell, exponents in [0.05, 20]."""
    b1, q1 = uniform_class((5, 5, 5, 5), nquartet_each, seed, cube=20.0, exps=(0.05, 20.0), kmin=1, kmax=3)
    b2, q2 = uniform_class((6, 6, 6, 6), nquartet_each, seed + 1000, cube=20.0, exps=(0.05, 20.0), kmin=1, kmax=3)
    return concat([(b1, q1), (b2, q2)])


def pair_lists(cls, nbra, nket, seed, cube=20.0, exps=(0.05, 20.0), kmin=1, kmax=1):
    """Bra-list x ket-list workload (the engine form): nbra pairs of shells with angular
    momenta (cls[0], cls[1]) and nket pairs with (cls[2], cls[3]), every shell its own,
    centers uniform in a cube of side `cube` bohr, exponents log-uniform in `exps`, degree per
    shell uniform in kmin..kmax.  Returns (basis, bra_pairs, ket_pairs)."""
    rng = np.random.default_rng(seed)
    ls = [cls[0], cls[1]] * nbra + [cls[2], cls[3]] * nket
    ks = rng.integers(kmin, kmax + 1, len(ls))
    centers = rng.uniform(0.0, cube, (len(ls), 3))
    basis = _assemble(ls, ks, centers, exps[0], exps[1], rng, kmax > 1)
    bra = np.arange(2 * nbra, dtype=np.int32).reshape(-1, 2)
    ket = (2 * nbra + np.arange(2 * nket, dtype=np.int32)).reshape(-1, 2)
    return basis, bra, ket


def iiii_pairs(nbra=64, nket=64, seed=2312):
    """(ii|ii) in the engine form: 64 bra pairs x 64 ket pairs = 4096 quartets, K = 1,
    20-bohr cube, exponents in [0.05, 20] (the headline class and size)."""
    return pair_lists((6, 6, 6, 6), nbra, nket, seed)


def routed(nquartet=1_000_000, seed=2311):
    """l = 4..6, K = 1..5, bra-ket separations 0-30 bohr (magnitudes over many decades)."""
    return spread_distances(nquartet, seed)


def concat(parts):
    """Concatenate several (basis, quartets) workloads."""
    ls, ks, cen, ex, co, qs = [], [], [], [], [], []
    nsh = 0
    for b, q in parts:
        ls.append(b["l"]); ks.append(b["nprim"]); cen.append(b["center"]); ex.append(b["exps"]); co.append(b["coefs"])
        qs.append(np.asarray(q) + nsh)
        nsh += len(b["l"])
    ks_all = np.concatenate(ks).astype(np.int32)
    off = np.zeros(len(ks_all), dtype=np.int32)
    if len(ks_all):
        off[1:] = np.cumsum(ks_all)[:-1]
    basis = {"l": np.concatenate(ls).astype(np.int32), "nprim": ks_all, "prim_off": off,
             "center": np.concatenate(cen), "exps": np.concatenate(ex), "coefs": np.concatenate(co)}
    return basis, np.concatenate(qs).astype(np.int32)
