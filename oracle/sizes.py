"""Footprint and FLOP/byte model of the matrix form of MD4, as the paper states it.

TEST INFRASTRUCTURE ONLY (part of the oracle).

* Hermite counts: N_p = (l_bra+1)(l_bra+2)(l_bra+3)/6, N_r = (L+1)(L+2)(L+3)/6
  (Section 2, footprint paragraph, pyramidal-number formula).
* Transform FLOPs: 2 N_ab N_p N_q (Eq. make-abq) and 2 N_ab N_q N_cd (Eq. make-abcd),
  with [p|q] and the first transform scaling as K = K_bra K_ket and the second as K_ket.
* Bytes: 8 N_p N_q written for [p|q]; 8 (N_ab N_p + N_p N_q + N_ab N_q) and
  8 (N_ab N_q + N_cd N_q + N_ab N_cd) moved by the two transforms (Section 2 item 3).
* Arithmetic intensity, Eq. AI.
"""


def pyr(n: int) -> int:
    return (n + 1) * (n + 2) * (n + 3) // 6


def nfun(l: int, solid: bool) -> int:
    return 2 * l + 1 if solid else (l + 1) * (l + 2) // 2


def transform_flops(la, lb, lc, ld, solid=True, kbra=1, kket=1):
    """(first, second) transform FLOPs of one shell quartet (Eq. make-abq, Eq. make-abcd)."""
    nab = nfun(la, solid) * nfun(lb, solid)
    ncd = nfun(lc, solid) * nfun(ld, solid)
    np_, nq = pyr(la + lb), pyr(lc + ld)
    return 2 * nab * np_ * nq * kbra * kket, 2 * nab * nq * ncd * kket


def arithmetic_intensity(la, lb, lc, ld, solid=True):
    """Eq. AI: FLOP per byte of the two transforms for primitive FP64 integrals."""
    nab = nfun(la, solid) * nfun(lb, solid)
    ncd = nfun(lc, solid) * nfun(ld, solid)
    np_, nq = pyr(la + lb), pyr(lc + ld)
    num = nab * nq * (np_ + ncd)
    den = 2 * np_ * nq + nab * (np_ + 2 * nq + ncd) + ncd * nq
    return 0.25 * num / den
