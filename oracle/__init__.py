"""CPU oracle for 4-center electron-repulsion integrals (ab|cd).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library and never calls it; the CUDA
product path never calls the oracle.

The C sources follow the paper's Section 2 (Formalism) step by step:

* ``eri_md_oracle.c`` -- plain McMurchie-Davidson: Boys function (Eq. boys), the
  auxiliary recursion (Eq. md1), the 2-index Hermite integrals (Eq. pq), the Hermite
  expansion coefficients (recursions after Eq. cart2herm-2) and the two Hermite-to-
  Cartesian transforms (Eq. ab_to_hermite, Eq. cd_to_hermite), then contraction and
  the Cartesian-to-solid transform (Section 2, definition of H).
* ``eri_os_oracle.c`` -- an independent Obara-Saika / Head-Gordon-Pople evaluator of
  the same Cartesian integrals, used only to pin the MD oracle.

``jk`` contracts the integral blocks with a density matrix into Coulomb and exchange
matrices, straight from the definition (numpy).

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(closed forms, brute-force quadrature, invariances, the paper's printed sizes).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liberi_oracle.so")
_SRCS = [os.path.join(_HERE, "eri_md_oracle.c"), os.path.join(_HERE, "eri_os_oracle.c")]
_lock = threading.Lock()
_lib = None

LMAX = 8  # largest shell angular momentum the oracle handles
KMAX = 64  # largest contraction degree of one shell


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (OpenMP) and return its path."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SRCS)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, *_SRCS, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            lp = ctypes.POINTER(ctypes.c_int64)
            lib.oracle_boys.argtypes = [ctypes.c_int, ctypes.c_double, dp]
            lib.oracle_boys.restype = None
            lib.oracle_prim_norm.argtypes = [ctypes.c_int, ctypes.c_double]
            lib.oracle_prim_norm.restype = ctypes.c_double
            lib.oracle_contract_norm.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
            lib.oracle_contract_norm.restype = None
            lib.oracle_solid_coefs.argtypes = [ctypes.c_int, dp]
            lib.oracle_solid_coefs.restype = None
            lib.oracle_hermite_E.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, dp]
            lib.oracle_hermite_E.restype = None
            lib.oracle_hermite_R.argtypes = [ctypes.c_int, ctypes.c_double, dp, ctypes.c_double, dp, dp]
            lib.oracle_hermite_R.restype = None
            lib.oracle_eri.argtypes = [ctypes.c_int, ip, ip, ip, dp, dp, dp, ctypes.c_int64, ip, lp,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
            lib.oracle_eri.restype = ctypes.c_int
            lib.oracle_max_threads.argtypes = []
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _lp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def ncart(l: int) -> int:
    return (l + 1) * (l + 2) // 2


def nsolid(l: int) -> int:
    return 2 * l + 1


def boys(mmax: int, T: float) -> np.ndarray:
    """F_m(T) for m = 0..mmax (Eq. boys)."""
    out = np.zeros(mmax + 1)
    _load().oracle_boys(int(mmax), float(T), _dp(out))
    return out


def prim_norm(l: int, zeta: float) -> float:
    """Normaliser of x^l exp(-zeta r^2)."""
    return _load().oracle_prim_norm(int(l), float(zeta))


def contract_norm(l: int, zeta, coef) -> np.ndarray:
    """Normalised contraction coefficients (primitive normaliser and contraction scale folded in)."""
    z = np.ascontiguousarray(zeta, dtype=np.float64)
    c = np.ascontiguousarray(coef, dtype=np.float64)
    out = np.zeros_like(z)
    _load().oracle_contract_norm(int(l), len(z), _dp(z), _dp(c), _dp(out))
    return out


def solid_coefs(l: int) -> np.ndarray:
    """(2l+1) x ncart(l) matrix of C^a_{lm} (rows m = -l..l) on x^l-normalised Cartesians."""
    out = np.zeros((2 * l + 1) * ncart(l))
    _load().oracle_solid_coefs(int(l), _dp(out))
    return out.reshape(2 * l + 1, ncart(l))


def hermite_E(la: int, lb: int, za: float, zb: float, Ax: float, Bx: float) -> np.ndarray:
    """1-D Hermite expansion coefficients E[i, j, t] (recursions after Eq. cart2herm-2)."""
    out = np.zeros((la + 1) * (lb + 1) * (la + lb + 1))
    _load().oracle_hermite_E(la, lb, za, zb, Ax, Bx, _dp(out))
    return out.reshape(la + 1, lb + 1, la + lb + 1)


def hermite_R(L: int, rho: float, PQ, pref: float) -> np.ndarray:
    """[r]^(0) on the (L+1)^3 box (entries with t+u+v <= L are set), Eq. md1."""
    pq = np.ascontiguousarray(PQ, dtype=np.float64)
    out = np.zeros((L + 1) ** 3)
    work = np.zeros((L + 1) ** 4)
    _load().oracle_hermite_R(L, rho, _dp(pq), pref, _dp(out), _dp(work))
    return out.reshape(L + 1, L + 1, L + 1)


def block_size(ls, solid: bool) -> int:
    n = 1
    for l in ls:
        n *= nsolid(l) if solid else ncart(l)
    return n


def eri(basis: dict, quartets, solid: bool = False, normalize: bool = True, method: str = "md",
        nthreads: int = 0, out_off=None) -> tuple[np.ndarray, np.ndarray]:
    """Contracted (ab|cd) for each quartet of shell indices.

    ``basis`` holds ``l``, ``nprim``, ``prim_off`` (int arrays per shell), ``center``
    (nshell x 3), ``exps`` and ``coefs`` (per primitive).  Returns (out, out_off):
    the flat output and the offset of each quartet's row-major (a,b,c,d) block.
    ``method`` is "md" (the paper's scheme) or "os" (independent Obara-Saika check).
    """
    lib = _load()
    l = np.ascontiguousarray(basis["l"], dtype=np.int32)
    K = np.ascontiguousarray(basis["nprim"], dtype=np.int32)
    off = np.ascontiguousarray(basis["prim_off"], dtype=np.int32)
    cen = np.ascontiguousarray(basis["center"], dtype=np.float64).reshape(-1, 3)
    ex = np.ascontiguousarray(basis["exps"], dtype=np.float64)
    co = np.ascontiguousarray(basis["coefs"], dtype=np.float64)
    qs = np.ascontiguousarray(quartets, dtype=np.int32).reshape(-1, 4)
    nq = qs.shape[0]
    sizes = np.array([block_size([l[s] for s in q], solid) for q in qs], dtype=np.int64)
    if out_off is None:
        out_off = np.zeros(nq, dtype=np.int64)
        if nq:
            out_off[1:] = np.cumsum(sizes)[:-1]
    out_off = np.ascontiguousarray(out_off, dtype=np.int64)
    total = int((out_off + sizes).max()) if nq else 0
    out = np.zeros(total)
    rc = lib.oracle_eri(len(l), _ip(l), _ip(K), _ip(off), _dp(cen), _dp(ex), _dp(co), nq, _ip(qs), _lp(out_off),
                        int(bool(solid)), int(bool(normalize)), 0 if method == "md" else 1, int(nthreads), _dp(out))
    if rc != 0:
        raise ValueError("oracle_eri rejected its arguments")
    return out, out_off


def function_offsets(basis: dict, solid: bool) -> tuple[np.ndarray, int]:
    """First basis function of each shell (shells in the given order, n(l) functions each)
    and the total number of functions."""
    n = np.array([nsolid(int(x)) if solid else ncart(int(x)) for x in basis["l"]], dtype=np.int64)
    off = np.zeros(len(n), dtype=np.int64)
    if len(n):
        off[1:] = np.cumsum(n)[:-1]
    return off, int(n.sum())


def jk(basis: dict, quartets, D, solid: bool = False) -> tuple[np.ndarray, np.ndarray]:
    """Coulomb and exchange contributions of a quartet list to a density matrix D
    (nbf x nbf; Section 3 names this digestion of the integrals into Fock matrix elements):
    for each listed quartet (ab|cd), with functions mu of a, nu of b, lam of c, sig of d,
        J[mu, nu]  += sum_{lam, sig} (mu nu | lam sig) D[lam, sig]
        K[mu, lam] += sum_{nu, sig}  (mu nu | lam sig) D[nu, sig]
    Each quartet counts once as listed: no permutational images are added."""
    l = np.asarray(basis["l"])
    qs = np.asarray(quartets, dtype=np.int64).reshape(-1, 4)
    bf, nbf = function_offsets(basis, solid)
    D = np.asarray(D, dtype=np.float64)
    assert D.shape == (nbf, nbf)
    J = np.zeros((nbf, nbf))
    K = np.zeros((nbf, nbf))
    out, off = eri(basis, qs, solid=solid)
    nf = [nsolid(int(x)) if solid else ncart(int(x)) for x in l]
    for i, (a, b, c, d) in enumerate(qs):
        na, nb, nc, nd = nf[a], nf[b], nf[c], nf[d]
        blk = out[off[i]:off[i] + na * nb * nc * nd].reshape(na, nb, nc, nd)
        ra, rb = slice(bf[a], bf[a] + na), slice(bf[b], bf[b] + nb)
        rc, rd = slice(bf[c], bf[c] + nc), slice(bf[d], bf[d] + nd)
        J[ra, rb] += np.einsum("abcd,cd->ab", blk, D[rc, rd])
        K[ra, rc] += np.einsum("abcd,bd->ac", blk, D[rb, rd])
    return J, K


def max_threads() -> int:
    return _load().oracle_max_threads()
