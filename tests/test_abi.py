"""The C-ABI library loads, exports every symbol include/lx_eri.h declares, and its host
side rejects invalid input with the documented error codes (no GPU needed: validation
precedes any device work)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2307_03452_gb300 import inputs, lx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lx_eri.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lx_[a-zA-Z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = lx.load()
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), f"missing export {name}"
    assert sorted(lx.EXPORTS) == names


def test_error_strings():
    lib = lx.load()
    for code in [0, -1, -2, -3, -4, -5, -6, -7, -8, -9, -10, -11, -12, -13]:
        s = lib.lx_strerror(code).decode()
        assert s and s != "unknown error code"
    assert lib.lx_strerror(12345).decode() == "unknown error code"


def _batch(nq=2, l=(4, 4, 4, 4)):
    b, q = inputs.uniform_class(l, nq, 3)
    return b, q


def _call_batch(b, q, flags=lx.LX_SOLID, shells=None, exps=None, coefs=None, quartets=None, out=1, ws=256,
                nprim=None):
    lib = lx.load()
    sh = lx.pack_shells(b) if shells is None else shells
    ex = np.ascontiguousarray(b["exps"]) if exps is None else exps
    co = np.ascontiguousarray(b["coefs"]) if coefs is None else coefs
    qs = lx.pack_quartets(b, q, True)[0] if quartets is None else quartets
    npr = len(ex) if nprim is None else nprim
    # fake non-null device pointers: validation rejects the input before they are touched
    return lib.lx_eri_batch(sh.ctypes.data_as(ctypes.c_void_p), len(sh), ex.ctypes.data_as(ctypes.c_void_p),
                            co.ctypes.data_as(ctypes.c_void_p), npr, qs.ctypes.data_as(ctypes.c_void_p), len(qs),
                            flags, ctypes.c_void_p(out), ctypes.c_void_p(ws), 1 << 20, None)


def test_rejects_bad_angular_momentum():
    b, q = _batch()
    sh = lx.pack_shells(b)
    sh["l"][1] = 8
    assert _call_batch(b, q, shells=sh) == -2
    sh["l"][1] = -1
    assert _call_batch(b, q, shells=sh) == -2


def test_rejects_bad_contraction_degree_and_reserved():
    b, q = _batch()
    sh = lx.pack_shells(b)
    sh["nprim"][0] = 0
    assert _call_batch(b, q, shells=sh) == -2
    sh = lx.pack_shells(b)
    sh["nprim"][0] = 17
    assert _call_batch(b, q, shells=sh) == -2
    sh = lx.pack_shells(b)
    sh["reserved"][2] = 1
    assert _call_batch(b, q, shells=sh) == -2


def test_rejects_nonfinite_center_and_primitive_range():
    b, q = _batch()
    sh = lx.pack_shells(b)
    sh["center"][3, 1] = np.nan
    assert _call_batch(b, q, shells=sh) == -2
    sh = lx.pack_shells(b)
    sh["prim_offset"][0] = len(b["exps"])
    assert _call_batch(b, q, shells=sh) == -2


@pytest.mark.parametrize("bad", [0.0, -1.0, np.inf, np.nan])
def test_rejects_bad_exponent(bad):
    b, q = _batch()
    ex = np.ascontiguousarray(b["exps"]).copy()
    ex[2] = bad
    assert _call_batch(b, q, exps=ex) == -3


def test_rejects_bad_coefficient():
    b, q = _batch()
    co = np.ascontiguousarray(b["coefs"]).copy()
    co[0] = np.inf
    assert _call_batch(b, q, coefs=co) == -3


def test_rejects_bad_quartets_and_flags():
    b, q = _batch()
    qs = lx.pack_quartets(b, q, True)[0]
    qs["s"][1, 2] = 999
    assert _call_batch(b, q, quartets=qs) == -4
    qs = lx.pack_quartets(b, q, True)[0]
    qs["out_offset"][0] = -5
    assert _call_batch(b, q, quartets=qs) == -4
    assert _call_batch(b, q, flags=0x40) == -5


def test_rejects_null_and_workspace():
    b, q = _batch()
    assert _call_batch(b, q, out=0) == -1
    assert _call_batch(b, q, ws=0) == -6
    assert _call_batch(b, q, ws=8) == -6  # not 256-byte aligned


def test_empty_batch_is_a_noop():
    b, q = _batch()
    lib = lx.load()
    sh = lx.pack_shells(b)
    rc = lib.lx_eri_batch(sh.ctypes.data_as(ctypes.c_void_p), len(sh), b["exps"].ctypes.data_as(ctypes.c_void_p),
                          b["coefs"].ctypes.data_as(ctypes.c_void_p), len(b["exps"]), None, 0, 1, None, None, 0,
                          None)
    assert rc == 0


def test_sizes():
    b, q = inputs.iiii_fp64(8)
    bs = lx.Batch(b, q, True)
    assert bs.out_size == 8 * 13 ** 4
    bc = lx.Batch(b, q, False)
    assert bc.out_size == 8 * 28 ** 4
    # workspace: at least H (both sides), [r]^(0) and [ab|q] of every quartet
    per_q = 8 * (2 * 169 * 455 + 2925 + 169 * 455)
    assert bs.workspace_size() >= 8 * per_q
    assert bs.workspace_min() < bs.workspace_size()
    # custom offsets: out size follows the largest block end
    qs = np.asarray(q)
    off = np.arange(8, dtype=np.int64) * 13 ** 4 * 2
    b2 = lx.Batch(b, qs, True, out_off=off)
    assert b2.out_size == off[-1] + 13 ** 4


def test_tuning_table_round_trip(tmp_path):
    lx.tune_clear()
    rows = np.array([[4, 4, 4, 4, 1, 1, 1, 0, 3], [6, 6, 6, 6, 4, 9, 0, 2, 1]], dtype=np.int32)
    lx.tune_import(rows)
    got = lx.tune_export()
    assert sorted(map(tuple, got.tolist())) == sorted(map(tuple, rows.tolist()))
    path = tmp_path / "tune.json"
    lx.save_tuning(str(path))
    lx.tune_clear()
    assert len(lx.tune_export()) == 0
    lx.load_tuning(str(path))
    assert sorted(map(tuple, lx.tune_export().tolist())) == sorted(map(tuple, rows.tolist()))
    with pytest.raises(lx.LxError):
        lx.tune_import(np.array([[4, 4, 4, 4, 1, 1, 1, 9, 0]], dtype=np.int32))  # bad shape id
    lx.tune_clear()


def test_routed_flag_combinations():
    # routing picks the path itself: it cannot be combined with the split flag
    basis, quartets = inputs.uniform_class((1, 1, 1, 1), 2, 5)
    b = lx.Batch(basis, quartets, True)
    lib = lx.load()
    bad = lx.LX_SOLID | lx.LX_PATH_SPLIT | lx.LX_PATH_ROUTED
    assert lib.lx_eri_workspace_size(lx._ptr(b.shells), len(b.shells), lx._ptr(b.quartets), len(b.quartets), bad) == -5
    ok = lx.LX_SOLID | lx.LX_PATH_ROUTED
    need = lib.lx_eri_workspace_size(lx._ptr(b.shells), len(b.shells), lx._ptr(b.quartets), len(b.quartets), ok)
    split = lib.lx_eri_workspace_size(lx._ptr(b.shells), len(b.shells), lx._ptr(b.quartets), len(b.quartets),
                                      lx.LX_SOLID | lx.LX_PATH_SPLIT)
    assert need >= split > 0


def _pairs_basis():
    # shells 0-3: h, h, i, i;  4: g
    rng = np.random.default_rng(5)
    ls = np.array([5, 5, 6, 6, 4], np.int32)
    K = np.array([1, 2, 1, 3, 2], np.int32)
    off = np.concatenate([[0], np.cumsum(K)[:-1]]).astype(np.int32)
    return {"l": ls, "nprim": K, "prim_off": off, "center": rng.uniform(0, 3, (5, 3)),
            "exps": np.exp(rng.uniform(-2, 2, K.sum())), "coefs": np.ones(K.sum())}


def test_pair_lists_sizes_and_errors():
    b = _pairs_basis()
    lib = lx.load()
    pb = lx.PairBatch(b, [[0, 1], [1, 0], [1, 1]], [[2, 3], [3, 2]], True)
    assert pb.shape == (3, 2, 121, 169)
    assert pb.out_size == 3 * 2 * 121 * 169
    # the pair form is the flat form of the same quartets in bra-major order
    flat = lx.Batch(b, [[0, 1, 2, 3], [0, 1, 3, 2], [1, 0, 2, 3], [1, 0, 3, 2], [1, 1, 2, 3], [1, 1, 3, 2]], True)
    assert pb.workspace_size() == flat.workspace_size()
    assert 0 < pb.workspace_min() <= pb.workspace_size()
    sh = lx.pack_shells(b)

    def size(bra, ket, flags=lx.LX_SOLID):
        bra = np.ascontiguousarray(np.asarray(bra, np.int32).reshape(-1, 2))
        ket = np.ascontiguousarray(np.asarray(ket, np.int32).reshape(-1, 2))
        return lib.lx_eri_pairs_out_size(sh.ctypes.data_as(ctypes.c_void_p), len(sh),
                                         bra.ctypes.data_as(ctypes.c_void_p), len(bra),
                                         ket.ctypes.data_as(ctypes.c_void_p), len(ket), flags)
    assert size([[0, 1]], [[2, 3]], lx.LX_CART) == 21 * 21 * 28 * 28
    assert size([[0, 1], [0, 4]], [[2, 3]]) == -13        # bra pairs (h h) and (h g)
    assert size([[0, 1]], [[2, 3], [4, 2]]) == -13        # ket pairs (i i) and (g i)
    assert size([[0, 5]], [[2, 3]]) == -4                  # shell index out of range
    assert size([[0, -1]], [[2, 3]]) == -4
    assert size(np.zeros((0, 2)), [[2, 3]]) == 0           # no bra pairs: nothing to do
    assert size([[0, 1]], [[2, 3]], 0x1000) == -5          # unknown flag
    neg = lib.lx_eri_pairs_out_size(sh.ctypes.data_as(ctypes.c_void_p), len(sh), None, -1, None, 0, 1)
    assert neg == -10
    # an empty product enqueues nothing (no device needed)
    rc = lib.lx_eri_pairs(sh.ctypes.data_as(ctypes.c_void_p), len(sh), b["exps"].ctypes.data_as(ctypes.c_void_p),
                          b["coefs"].ctypes.data_as(ctypes.c_void_p), len(b["exps"]), None, 0, None, 0, 1, None,
                          None, 0, None)
    assert rc == 0


def test_jk_entry_points_validate_on_the_host():
    b = _pairs_basis()
    lib = lx.load()
    sh = lx.pack_shells(b)
    c = ctypes.c_void_p
    assert lib.lx_nbf(sh.ctypes.data_as(c), len(sh), lx.LX_SOLID) == 11 + 11 + 13 + 13 + 9
    assert lib.lx_nbf(sh.ctypes.data_as(c), len(sh), lx.LX_CART) == 21 + 21 + 28 + 28 + 15
    assert lib.lx_nbf(sh.ctypes.data_as(c), len(sh), 0x1000) == -5
    jb = lx.JKBatch(b, [[0, 1, 2, 3], [4, 4, 0, 2]], True)
    assert jb.nbf == 57
    # FP64 path: J and K straight from [ab|q], so no block is stored; split path: each
    # quartet's block is kept in the workspace for the digestion kernel
    plain = lx.Batch(b, [[0, 1, 2, 3], [4, 4, 0, 2]], True)
    assert jb.workspace_size() <= plain.workspace_size()
    assert 0 < jb.workspace_min() <= jb.workspace_size()
    js = lx.JKBatch(b, [[0, 1, 2, 3], [4, 4, 0, 2]], True, path="split")
    ps = lx.Batch(b, [[0, 1, 2, 3], [4, 4, 0, 2]], True, path="split")
    assert js.workspace_size() >= ps.workspace_size() + 8 * (121 * 169 + 81 * 143)
    assert ps.workspace_min() < js.workspace_min() <= js.workspace_size()
    q = jb.quartets
    ex, co = np.ascontiguousarray(b["exps"]), np.ascontiguousarray(b["coefs"])

    def call(D, J, K, flags=lx.LX_SOLID, nq=len(q)):
        return lib.lx_eri_jk(sh.ctypes.data_as(c), len(sh), ex.ctypes.data_as(c), co.ctypes.data_as(c), len(ex),
                             q.ctypes.data_as(c), nq, flags, c(D), c(J), c(K), c(1 << 20), 1 << 20, None)
    assert call(None, 8, 8) == -1            # no density
    assert call(8, None, None) == -1         # neither output
    assert call(8, 8, 8, flags=0x40000000) == -5   # the planner's internal bit is not a caller flag
    assert call(8, 8, 8, nq=0) == 0          # empty list: nothing to do
    # lx_eri_batch refuses the internal bit as well
    assert _call_batch(b, [[0, 1, 2, 3]], flags=lx.LX_SOLID | 0x40000000) == -5


def test_jk_workspace_for_routed_covers_both_paths():
    # a routed J/K call may send every quartet to either path, and needs the predictions'
    # room besides
    b = _pairs_basis()
    q = [[0, 1, 2, 3], [4, 4, 0, 2], [1, 1, 3, 3]]
    sizes = {p: lx.JKBatch(b, q, True, path=p).workspace_size() for p in ("fp64", "split", "routed")}
    mins = {p: lx.JKBatch(b, q, True, path=p).workspace_min() for p in ("fp64", "split", "routed")}
    assert sizes["routed"] >= max(sizes["fp64"], sizes["split"])
    assert mins["routed"] >= max(mins["fp64"], mins["split"])
    assert sizes["split"] > sizes["fp64"]  # the split path keeps each block for the digestion


def test_selftest_timeout_bounds_its_tries():
    # more tries than the library's own wait limit is refused on the host
    assert lx.load().lx_selftest_timeout((1 << 24) + 1, None) == -10
