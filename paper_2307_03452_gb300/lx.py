"""Python binding of the C ABI in ``include/lx_eri.h`` (argument marshalling only).

Every arithmetic step runs in the CUDA library ``liblx_eri.so``; this module packs the
host descriptors, passes device pointers taken from torch tensors, and raises if the
library cannot be loaded.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

SHELL_DTYPE = np.dtype([("l", "<i4"), ("nprim", "<i4"), ("prim_offset", "<i4"), ("reserved", "<i4"),
                        ("center", "<f8", (3,))])
QUARTET_DTYPE = np.dtype([("s", "<i4", (4,)), ("out_offset", "<i8")])
assert SHELL_DTYPE.itemsize == 40 and QUARTET_DTYPE.itemsize == 24

LX_CART = 0x0
LX_SOLID = 0x1
LX_KET_SIGN = 0x100  # lx_hermite_H: multiply column p by (-1)^|p|
LMAX = 7
KMAX = 16

_lock = threading.Lock()
_lib = None

#: every symbol the header declares
EXPORTS = sorted(["lx_eri_out_size", "lx_eri_workspace_size", "lx_eri_workspace_min", "lx_eri_batch",
                  "lx_eri_batch_static",
                  "lx_eri_sync_status", "lx_eri_stage_times", "lx_strerror", "lx_last_cuda_error", "lx_boys",
                  "lx_hermite_R", "lx_hermite_H", "lx_split_gemm", "lx_route_features", "lx_mlp_forward",
                  "lx_mlp_grad", "lx_mlp_adam", "lx_eri_graph_create", "lx_eri_graph_launch",
                  "lx_eri_graph_destroy", "lx_eri_autotune", "lx_tune_export", "lx_tune_import", "lx_tune_clear",
                  "lx_router_set", "lx_eri_pairs_out_size", "lx_eri_pairs_workspace_size",
                  "lx_eri_pairs_workspace_min", "lx_eri_pairs", "lx_nbf", "lx_eri_jk_workspace_size",
                  "lx_eri_jk_workspace_min", "lx_eri_jk", "lx_selftest_timeout"])
TILE_SHAPES = ["32x64", "64x32", "32x32", "64x64"]
MLP_NIN = 20
MLP_WIDTH = 64
MLP_NOUT = 2  # log10 max |integral|, log10 of the split path's error (6 digits)
MLP_NPARAM = MLP_WIDTH * MLP_NIN + MLP_WIDTH + MLP_WIDTH * MLP_WIDTH + MLP_WIDTH + MLP_NOUT * MLP_WIDTH + MLP_NOUT
ROUTE_TIERS = (4, 5, 6)  # digits of the split tiers of path "routed"
SPLIT_DIGITS_MASK = 0x70
LX_PATH_SPLIT = 0x2
LX_PATH_ROUTED = 0x4
LX_TIME_STAGES = 0x200
# "split4" / "split5": the split path keeping 4 / 5 digits per value ("split": 6)
PATH_FLAGS = {"fp64": 0, "split": LX_PATH_SPLIT, "split4": LX_PATH_SPLIT | (4 << 4), "split5": LX_PATH_SPLIT | (5 << 4),
              "split6": LX_PATH_SPLIT | (6 << 4), "routed": LX_PATH_ROUTED}
STAGES = ["norm", "pair_h", "boys_r", "gemm1", "gemm2", "split", "digest"]


class LxError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load()
        msg = lib.lx_strerror(code).decode()
        if code == -7:
            msg += f" ({lib.lx_last_cuda_error().decode()})"
        super().__init__(f"{where}: error {code}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load liblx_eri.so (building it first if it is missing and nvcc is present)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
            _build.build()
        lib = ctypes.CDLL(path)
        c_i32, c_i64, c_vp, c_sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t
        lib.lx_eri_out_size.argtypes = [c_vp, c_i32, c_vp, c_i64, c_i32]
        lib.lx_eri_out_size.restype = c_i64
        lib.lx_eri_workspace_size.argtypes = [c_vp, c_i32, c_vp, c_i64, c_i32]
        lib.lx_eri_workspace_size.restype = c_i64
        lib.lx_eri_workspace_min.argtypes = [c_vp, c_i32, c_vp, c_i64, c_i32]
        lib.lx_eri_workspace_min.restype = c_i64
        lib.lx_eri_batch.argtypes = [c_vp, c_i32, c_vp, c_vp, c_i32, c_vp, c_i64, c_i32, c_vp, c_vp, c_sz, c_vp]
        lib.lx_eri_batch.restype = ctypes.c_int
        for name in ("lx_eri_pairs_out_size", "lx_eri_pairs_workspace_size", "lx_eri_pairs_workspace_min"):
            getattr(lib, name).argtypes = [c_vp, c_i32, c_vp, c_i64, c_vp, c_i64, c_i32]
            getattr(lib, name).restype = c_i64
        lib.lx_eri_pairs.argtypes = [c_vp, c_i32, c_vp, c_vp, c_i32, c_vp, c_i64, c_vp, c_i64, c_i32, c_vp, c_vp, c_sz,
                                     c_vp]
        lib.lx_eri_pairs.restype = ctypes.c_int
        lib.lx_selftest_timeout.argtypes = [ctypes.c_uint64, c_vp]
        lib.lx_selftest_timeout.restype = ctypes.c_int
        lib.lx_nbf.argtypes = [c_vp, c_i32, c_i32]
        lib.lx_nbf.restype = c_i64
        for name in ("lx_eri_jk_workspace_size", "lx_eri_jk_workspace_min"):
            getattr(lib, name).argtypes = [c_vp, c_i32, c_vp, c_i64, c_i32]
            getattr(lib, name).restype = c_i64
        lib.lx_eri_jk.argtypes = [c_vp, c_i32, c_vp, c_vp, c_i32, c_vp, c_i64, c_i32, c_vp, c_vp, c_vp, c_vp, c_sz,
                                  c_vp]
        lib.lx_eri_jk.restype = ctypes.c_int
        lib.lx_eri_batch_static.argtypes = [c_vp, c_i32, c_vp, c_vp, c_i32, c_vp, c_i64, c_i32, c_vp, c_vp]
        lib.lx_eri_batch_static.restype = ctypes.c_int
        lib.lx_eri_sync_status.argtypes = [c_vp]
        lib.lx_eri_sync_status.restype = ctypes.c_int
        lib.lx_eri_stage_times.argtypes = [c_vp, c_vp, c_i32, c_vp]
        lib.lx_eri_stage_times.restype = ctypes.c_int
        lib.lx_strerror.argtypes = [ctypes.c_int]
        lib.lx_strerror.restype = ctypes.c_char_p
        lib.lx_last_cuda_error.argtypes = []
        lib.lx_last_cuda_error.restype = ctypes.c_char_p
        lib.lx_boys.argtypes = [c_i32, c_vp, c_i64, c_vp, c_vp]
        lib.lx_boys.restype = ctypes.c_int
        lib.lx_hermite_R.argtypes = [c_i32, c_vp, c_i64, c_vp, c_vp]
        lib.lx_hermite_R.restype = ctypes.c_int
        lib.lx_hermite_H.argtypes = [c_vp, c_i32, c_vp, c_vp, c_i32, c_vp, c_i32, c_i32, c_vp, c_i64, c_vp]
        lib.lx_hermite_H.restype = ctypes.c_int
        lib.lx_split_gemm.argtypes = [c_i32, c_i32, c_i32, c_vp, c_i32, c_vp, c_i32, c_vp, c_i32, c_i32, c_vp]
        lib.lx_split_gemm.restype = ctypes.c_int
        lib.lx_eri_graph_create.argtypes = [c_vp, c_i32, c_vp, c_vp, c_i32, c_vp, c_i64, c_i32, c_vp, c_vp, c_sz,
                                            ctypes.POINTER(c_vp)]
        lib.lx_eri_graph_create.restype = ctypes.c_int
        lib.lx_eri_graph_launch.argtypes = [c_vp, c_vp]
        lib.lx_eri_graph_launch.restype = ctypes.c_int
        lib.lx_eri_graph_destroy.argtypes = [c_vp]
        lib.lx_eri_graph_destroy.restype = ctypes.c_int
        lib.lx_eri_autotune.argtypes = [c_vp, c_i32, c_vp, c_vp, c_i32, c_vp, c_i64, c_i32, c_vp, c_i64, c_vp, c_sz,
                                        c_i32, c_i32, c_vp]
        lib.lx_eri_autotune.restype = ctypes.c_int
        lib.lx_tune_export.argtypes = [c_vp, c_i64]
        lib.lx_tune_export.restype = c_i64
        lib.lx_tune_import.argtypes = [c_vp, c_i64]
        lib.lx_tune_import.restype = ctypes.c_int
        lib.lx_tune_clear.argtypes = []
        lib.lx_tune_clear.restype = ctypes.c_int
        lib.lx_route_features.argtypes = [c_vp, c_i32, c_vp, c_i32, c_vp, c_i64, c_vp, c_vp]
        lib.lx_route_features.restype = ctypes.c_int
        lib.lx_router_set.argtypes = [c_vp, c_vp]
        lib.lx_router_set.restype = ctypes.c_int
        lib.lx_mlp_forward.argtypes = [c_vp, c_vp, c_i64, c_vp, c_vp]
        lib.lx_mlp_forward.restype = ctypes.c_int
        lib.lx_mlp_grad.argtypes = [c_vp, c_vp, c_vp, c_i64, c_vp, c_vp, c_vp]
        lib.lx_mlp_grad.restype = ctypes.c_int
        c_f32 = ctypes.c_float
        lib.lx_mlp_adam.argtypes = [c_vp, c_vp, c_vp, c_vp, c_vp, c_i32, c_f32, c_f32, c_f32, c_f32, c_vp]
        lib.lx_mlp_adam.restype = ctypes.c_int
        _lib = lib
        return lib


def _check(code: int, where: str):
    if code != 0:
        raise LxError(code, where)


def nfun(l: int, solid: bool) -> int:
    return 2 * l + 1 if solid else (l + 1) * (l + 2) // 2


def pack_shells(basis: dict) -> np.ndarray:
    n = len(basis["l"])
    sh = np.zeros(n, dtype=SHELL_DTYPE)
    sh["l"] = basis["l"]
    sh["nprim"] = basis["nprim"]
    sh["prim_offset"] = basis["prim_off"]
    sh["center"] = np.asarray(basis["center"], dtype=np.float64).reshape(n, 3)
    return sh


def pack_quartets(basis: dict, quartets, solid: bool, out_off=None) -> tuple[np.ndarray, np.ndarray]:
    qs = np.asarray(quartets, dtype=np.int32).reshape(-1, 4)
    l = np.asarray(basis["l"])
    nf = (2 * l + 1) if solid else (l + 1) * (l + 2) // 2
    sizes = nf[qs[:, 0]].astype(np.int64) * nf[qs[:, 1]] * nf[qs[:, 2]] * nf[qs[:, 3]]
    if out_off is None:
        out_off = np.zeros(len(qs), dtype=np.int64)
        if len(qs):
            out_off[1:] = np.cumsum(sizes)[:-1]
    q = np.zeros(len(qs), dtype=QUARTET_DTYPE)
    q["s"] = qs
    q["out_offset"] = out_off
    return q, sizes


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Batch:
    """Host descriptors of one batch, packed once (the planner's input)."""

    def __init__(self, basis: dict, quartets, solid: bool, out_off=None, path: str = "fp64"):
        if path not in PATH_FLAGS:
            raise ValueError(f"unknown path {path!r}")
        self.solid = bool(solid)
        self.path = path
        self.flags = (LX_SOLID if solid else LX_CART) | PATH_FLAGS[path]
        self.shells = pack_shells(basis)
        self.exps = np.ascontiguousarray(basis["exps"], dtype=np.float64)
        self.coefs = np.ascontiguousarray(basis["coefs"], dtype=np.float64)
        self.quartets, self.sizes = pack_quartets(basis, quartets, solid, out_off)
        lib = load()
        n = lib.lx_eri_out_size(_ptr(self.shells), len(self.shells), _ptr(self.quartets), len(self.quartets), self.flags)
        if n < 0:
            raise LxError(int(n), "lx_eri_out_size")
        self.out_size = int(n)

    def pin(self):
        """Keep the input arrays in pinned (page-locked) memory.  The library stages its own
        uploads in pinned memory, so calls are asynchronous without this; it only keeps the
        caller's arrays out of pageable memory."""
        import torch
        self._pinned = []

        def to_pinned(a):
            t = torch.empty(max(a.nbytes, 1), dtype=torch.uint8, pin_memory=True)
            v = t.numpy()[: a.nbytes].view(a.dtype).reshape(a.shape)
            v[...] = a
            self._pinned.append(t)
            return v

        self.shells = to_pinned(self.shells)
        self.exps = to_pinned(self.exps)
        self.coefs = to_pinned(self.coefs)
        self.quartets = to_pinned(self.quartets)
        return self

    def host_bytes(self) -> int:
        """Bytes of host descriptors passed per call (shells, exponents, coefficients, quartets)."""
        return int(self.shells.nbytes + self.exps.nbytes + self.coefs.nbytes + self.quartets.nbytes)

    @property
    def nquartet(self) -> int:
        return len(self.quartets)

    def workspace_size(self) -> int:
        n = load().lx_eri_workspace_size(_ptr(self.shells), len(self.shells), _ptr(self.quartets),
                                         len(self.quartets), self.flags)
        if n < 0:
            raise LxError(int(n), "lx_eri_workspace_size")
        return int(n)

    def workspace_min(self) -> int:
        n = load().lx_eri_workspace_min(_ptr(self.shells), len(self.shells), _ptr(self.quartets),
                                        len(self.quartets), self.flags)
        if n < 0:
            raise LxError(int(n), "lx_eri_workspace_min")
        return int(n)

    def run(self, out, workspace, stream=None, time_stages: bool = False):
        """Enqueue lx_eri_batch; out and workspace are CUDA tensors (float64 / uint8)."""
        flags = self.flags | (LX_TIME_STAGES if time_stages else 0)
        rc = load().lx_eri_batch(_ptr(self.shells), len(self.shells), _ptr(self.exps), _ptr(self.coefs),
                                 len(self.exps), _ptr(self.quartets), len(self.quartets), flags,
                                 ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(workspace.data_ptr()),
                                 workspace.numel() * workspace.element_size(), ctypes.c_void_p(_stream_ptr(stream)))
        _check(rc, "lx_eri_batch")


class PairBatch:
    """The bra-list x ket-list form: (ab|cd) for every bra pair and every ket pair, into a
    dense [nbra][nket][n_ab][n_cd] output (lx_eri_pairs)."""

    def __init__(self, basis: dict, bra_pairs, ket_pairs, solid: bool, path: str = "fp64"):
        if path not in PATH_FLAGS:
            raise ValueError(f"unknown path {path!r}")
        self.solid = bool(solid)
        self.path = path
        self.flags = (LX_SOLID if solid else LX_CART) | PATH_FLAGS[path]
        self.shells = pack_shells(basis)
        self.exps = np.ascontiguousarray(basis["exps"], dtype=np.float64)
        self.coefs = np.ascontiguousarray(basis["coefs"], dtype=np.float64)
        self.bra = np.ascontiguousarray(np.asarray(bra_pairs, dtype=np.int32).reshape(-1, 2))
        self.ket = np.ascontiguousarray(np.asarray(ket_pairs, dtype=np.int32).reshape(-1, 2))
        l = np.asarray(basis["l"])
        self.shape = (len(self.bra), len(self.ket),
                      nfun(int(l[self.bra[0, 0]]), solid) * nfun(int(l[self.bra[0, 1]]), solid) if len(self.bra) else 0,
                      nfun(int(l[self.ket[0, 0]]), solid) * nfun(int(l[self.ket[0, 1]]), solid) if len(self.ket) else 0)
        self.out_size = self._size(load().lx_eri_pairs_out_size, "lx_eri_pairs_out_size")

    def _args(self):
        return (_ptr(self.shells), len(self.shells), _ptr(self.bra), len(self.bra), _ptr(self.ket), len(self.ket),
                self.flags)

    def _size(self, fn, where):
        n = fn(*self._args())
        if n < 0:
            raise LxError(int(n), where)
        return int(n)

    def workspace_size(self) -> int:
        return self._size(load().lx_eri_pairs_workspace_size, "lx_eri_pairs_workspace_size")

    def workspace_min(self) -> int:
        return self._size(load().lx_eri_pairs_workspace_min, "lx_eri_pairs_workspace_min")

    def run(self, out, workspace, stream=None, time_stages: bool = False):
        """Enqueue lx_eri_pairs; out and workspace are CUDA tensors (float64 / uint8)."""
        flags = self.flags | (LX_TIME_STAGES if time_stages else 0)
        rc = load().lx_eri_pairs(_ptr(self.shells), len(self.shells), _ptr(self.exps), _ptr(self.coefs),
                                 len(self.exps), _ptr(self.bra), len(self.bra), _ptr(self.ket), len(self.ket), flags,
                                 ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(workspace.data_ptr()),
                                 workspace.numel() * workspace.element_size(), ctypes.c_void_p(_stream_ptr(stream)))
        _check(rc, "lx_eri_pairs")


def eri_pairs(basis: dict, bra_pairs, ket_pairs, solid: bool = True, device="cuda",
              workspace_limit: int | None = None, stream=None, path: str = "fp64"):
    """(ab|cd) for every bra pair and every ket pair on the GPU: a float64 CUDA tensor of shape
    (nbra, nket, n_ab, n_cd)."""
    import torch
    b = PairBatch(basis, bra_pairs, ket_pairs, solid, path=path)
    need = b.workspace_size()
    if workspace_limit is not None:
        need = max(min(need, int(workspace_limit)), b.workspace_min())
    out = torch.empty(max(b.out_size, 1), dtype=torch.float64, device=device)
    ws = alloc_workspace(need, device)
    b.run(out, ws, stream)
    sync_status(stream)
    return out[: b.out_size].view(b.shape)


class JKBatch(Batch):
    """A quartet list digested into Coulomb and exchange matrices (lx_eri_jk)."""

    def __init__(self, basis: dict, quartets, solid: bool, path: str = "fp64"):
        super().__init__(basis, quartets, solid, path=path)
        n = load().lx_nbf(_ptr(self.shells), len(self.shells), self.flags)
        if n < 0:
            raise LxError(int(n), "lx_nbf")
        self.nbf = int(n)

    def _need(self, fn, where):
        n = fn(_ptr(self.shells), len(self.shells), _ptr(self.quartets), len(self.quartets), self.flags)
        if n < 0:
            raise LxError(int(n), where)
        return int(n)

    def workspace_size(self) -> int:
        return self._need(load().lx_eri_jk_workspace_size, "lx_eri_jk_workspace_size")

    def workspace_min(self) -> int:
        return self._need(load().lx_eri_jk_workspace_min, "lx_eri_jk_workspace_min")

    def run_jk(self, D, J, K, workspace, stream=None, time_stages: bool = False):
        """Enqueue lx_eri_jk: D, J, K float64 CUDA tensors (nbf x nbf; J or K may be None)."""
        flags = self.flags | (LX_TIME_STAGES if time_stages else 0)
        ptr = lambda t: ctypes.c_void_p(t.data_ptr() if t is not None else None)  # noqa: E731
        rc = load().lx_eri_jk(_ptr(self.shells), len(self.shells), _ptr(self.exps), _ptr(self.coefs),
                              len(self.exps), _ptr(self.quartets), len(self.quartets), flags, ptr(D), ptr(J), ptr(K),
                              ctypes.c_void_p(workspace.data_ptr()), workspace.numel() * workspace.element_size(),
                              ctypes.c_void_p(_stream_ptr(stream)))
        _check(rc, "lx_eri_jk")


def eri_jk(basis: dict, quartets, D, solid: bool = True, want: str = "JK", device="cuda",
           workspace_limit: int | None = None, stream=None, path: str = "fp64"):
    """Coulomb and exchange contributions of the quartets to density D (nbf x nbf, any array
    or tensor): returns (J, K) as float64 CUDA tensors (None for the one not in `want`)."""
    import torch
    b = JKBatch(basis, quartets, solid, path=path)
    Dt = torch.as_tensor(np.asarray(D, dtype=np.float64) if not isinstance(D, torch.Tensor) else D,
                         dtype=torch.float64, device=device).contiguous()
    if Dt.shape != (b.nbf, b.nbf):
        raise ValueError(f"D must be {b.nbf} x {b.nbf}")
    J = torch.zeros_like(Dt) if "J" in want else None
    K = torch.zeros_like(Dt) if "K" in want else None
    need = b.workspace_size()
    if workspace_limit is not None:
        need = max(min(need, int(workspace_limit)), b.workspace_min())
    b.run_jk(Dt, J, K, alloc_workspace(need, device), stream)
    sync_status(stream)
    return J, K


def selftest_timeout(tries: int = 1000, stream=None):
    """Enqueue the library's bounded-wait timeout path on purpose (lx_selftest_timeout); the
    next sync_status raises LxError(LX_ERR_DEVICE_STATUS)."""
    _check(load().lx_selftest_timeout(int(tries), ctypes.c_void_p(_stream_ptr(stream))), "lx_selftest_timeout")


def stage_times(stream=None) -> tuple[dict, dict]:
    """Per-stage device milliseconds and launch counts of the LX_TIME_STAGES calls on `stream`
    since the last read (waits for the stream)."""
    ms = np.zeros(len(STAGES))
    n = np.zeros(len(STAGES), dtype=np.int64)
    _check(load().lx_eri_stage_times(_ptr(ms), _ptr(n), len(STAGES), ctypes.c_void_p(_stream_ptr(stream))),
           "lx_eri_stage_times")
    return dict(zip(STAGES, ms.tolist())), dict(zip(STAGES, n.tolist()))


STATIC_SCRATCH_BYTES = 64 << 20


def run_static(batch: "Batch", out, stream=None, time_stages: bool = False):
    """lx_eri_batch_static: the same evaluation with the library's fixed device scratch
    array instead of a caller workspace (for callers that cannot allocate device memory).
    time_stages passes LX_TIME_STAGES, which this entry refuses."""
    b = batch
    flags = b.flags | (LX_TIME_STAGES if time_stages else 0)
    rc = load().lx_eri_batch_static(_ptr(b.shells), len(b.shells), _ptr(b.exps), _ptr(b.coefs), len(b.exps),
                                    _ptr(b.quartets), len(b.quartets), flags, ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(_stream_ptr(stream)))
    _check(rc, "lx_eri_batch_static")


class Graph:
    """A batch captured into a CUDA graph (lx_eri_graph_create); replay with launch()."""

    def __init__(self, batch: "Batch", out, workspace):
        self._keep = (out, workspace)
        h = ctypes.c_void_p()
        b = batch
        rc = load().lx_eri_graph_create(_ptr(b.shells), len(b.shells), _ptr(b.exps), _ptr(b.coefs), len(b.exps),
                                        _ptr(b.quartets), len(b.quartets), b.flags, ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(workspace.data_ptr()),
                                        workspace.numel() * workspace.element_size(), ctypes.byref(h))
        _check(rc, "lx_eri_graph_create")
        self.handle = h

    def launch(self, stream=None):
        _check(load().lx_eri_graph_launch(self.handle, ctypes.c_void_p(_stream_ptr(stream))), "lx_eri_graph_launch")

    def close(self):
        if self.handle:
            load().lx_eri_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(batch: "Batch", max_keys=16, samples=8, workspace_bytes=None, stream=None):
    """Time the FP64 GEMM tile shapes on the batch's costliest classes; returns the table rows."""
    import torch
    b = batch
    ws_bytes = workspace_bytes or min(b.workspace_size(), 4 << 30)
    ws = alloc_workspace(max(ws_bytes, b.workspace_min()))
    nout = int(min(b.out_size, max(b.sizes[: max(samples, 1) * 64].sum(), int(b.sizes.max()) * samples)))
    out = torch.empty(max(nout, 1), dtype=torch.float64, device=ws.device)
    _check(load().lx_eri_autotune(_ptr(b.shells), len(b.shells), _ptr(b.exps), _ptr(b.coefs), len(b.exps),
                                  _ptr(b.quartets), len(b.quartets), b.flags, ctypes.c_void_p(out.data_ptr()),
                                  out.numel(), ctypes.c_void_p(ws.data_ptr()), ws.numel(), int(max_keys),
                                  int(samples), ctypes.c_void_p(_stream_ptr(stream))), "lx_eri_autotune")
    return tune_export()


def tune_export() -> np.ndarray:
    lib = load()
    n = int(lib.lx_tune_export(None, 0))
    rows = np.zeros((max(n, 1), 9), dtype=np.int32)
    lib.lx_tune_export(_ptr(rows), n)
    return rows[:n]


def tune_import(rows):
    rows = np.ascontiguousarray(rows, dtype=np.int32).reshape(-1, 9)
    _check(load().lx_tune_import(_ptr(rows), len(rows)), "lx_tune_import")


def tune_clear():
    load().lx_tune_clear()


TUNE_FORMAT = 1


def save_tuning(path):
    """Persist the tuning table as versioned JSON."""
    import json
    rows = tune_export()
    with open(path, "w") as f:
        json.dump({"format": TUNE_FORMAT, "columns": ["la", "lb", "lc", "ld", "kbra", "kket", "solid", "gemm1",
                                                      "gemm2"], "shapes": TILE_SHAPES, "rows": rows.tolist()}, f)


def load_tuning(path):
    import json
    with open(path) as f:
        d = json.load(f)
    if d.get("format") != TUNE_FORMAT or d.get("shapes") != TILE_SHAPES:
        raise ValueError(f"incompatible tuning file {path}")
    tune_import(np.asarray(d["rows"], dtype=np.int32).reshape(-1, 9))


def sync_status(stream=None):
    _check(load().lx_eri_sync_status(ctypes.c_void_p(_stream_ptr(stream))), "lx_eri_sync_status")


def alloc_workspace(nbytes: int, device="cuda"):
    import torch
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def eri(basis: dict, quartets, solid: bool = True, device="cuda", workspace_limit: int | None = None,
        stream=None, path: str = "fp64"):
    """Evaluate (ab|cd) for every quartet on the GPU; returns (out, out_offsets) with out a
    float64 CUDA tensor holding each quartet's row-major (a,b,c,d) block.  path "fp64" runs
    every step in FP64; "split" runs the two transforms as BF16 slice products on the
    tensor cores; "routed" sends each quartet to one of the two by the network installed
    with router_set."""
    import torch
    b = Batch(basis, quartets, solid, path=path)
    need = b.workspace_size()
    if workspace_limit is not None:
        need = max(min(need, int(workspace_limit)), b.workspace_min())
    out = torch.empty(max(b.out_size, 1), dtype=torch.float64, device=device)
    ws = alloc_workspace(need, device)
    b.run(out, ws, stream)
    sync_status(stream)
    return out[: b.out_size], b.quartets["out_offset"].copy()


def router_set(params_f16, tau):
    """Install the routing network of path "routed" on the current device: params_f16 holds
    the MLP_NPARAM FP16 parameters (any array or tensor; copied); tau the thresholds of the
    split tiers of 4, 5 and 6 digits on the network's output 1 (predicted log10 split error):
    a quartet takes the first tier whose threshold lies above its prediction, else the FP64
    path (a tier is disabled by -1e30)."""
    try:
        import torch
        if isinstance(params_f16, torch.Tensor):
            params_f16 = params_f16.detach().to("cpu").numpy()
    except ImportError:
        pass
    p = np.ascontiguousarray(np.asarray(params_f16, dtype=np.float16))
    if p.size != MLP_NPARAM:
        raise ValueError(f"expected {MLP_NPARAM} parameters, got {p.size}")
    t = np.ascontiguousarray(np.asarray(tau, dtype=np.float32).reshape(-1))
    if t.size != len(ROUTE_TIERS):
        raise ValueError(f"expected {len(ROUTE_TIERS)} thresholds, got {t.size}")
    _check(load().lx_router_set(_ptr(p), _ptr(t)), "lx_router_set")


def split_gemm(A, B, stream=None, digits: int = 6):
    """C = A @ B.T for float64 CUDA matrices through the split path's tensor-core kernels,
    keeping `digits` (4..6) BF16 digits per value."""
    import torch
    A = A.contiguous()
    B = B.contiguous()
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty((M, N), dtype=torch.float64, device=A.device)
    _check(load().lx_split_gemm(M, N, K, ctypes.c_void_p(A.data_ptr()), K, ctypes.c_void_p(B.data_ptr()), K,
                                ctypes.c_void_p(C.data_ptr()), N, int(digits), ctypes.c_void_p(_stream_ptr(stream))),
           "lx_split_gemm")
    return C


def route_features(basis: dict, quartets, device="cuda", stream=None):
    """Router features (nq, MLP_NIN) float32 CUDA tensor (lx_route_features)."""
    import torch
    sh = pack_shells(basis)
    ex = np.ascontiguousarray(basis["exps"], dtype=np.float64)
    q, _ = pack_quartets(basis, quartets, True)
    feat = torch.empty((len(q), MLP_NIN), dtype=torch.float32, device=device)
    _check(load().lx_route_features(_ptr(sh), len(sh), _ptr(ex), len(ex), _ptr(q), len(q),
                                    ctypes.c_void_p(feat.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))),
           "lx_route_features")
    return feat


def mlp_forward(params_f16, feat, stream=None):
    """(n, MLP_NOUT) outputs of the network for features (n, MLP_NIN)."""
    import torch
    out = torch.empty((feat.shape[0], MLP_NOUT), dtype=torch.float32, device=feat.device)
    _check(load().lx_mlp_forward(ctypes.c_void_p(params_f16.data_ptr()), ctypes.c_void_p(feat.data_ptr()),
                                 feat.shape[0], ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))),
           "lx_mlp_forward")
    return out


def mlp_grad(params, feat, target, stream=None):
    """(loss, grad) of the mean over samples of the summed squared errors of the outputs
    (target: (n, MLP_NOUT)), forward with FP16-rounded params."""
    import torch
    grad = torch.empty(MLP_NPARAM, dtype=torch.float32, device=params.device)
    loss = torch.empty(1, dtype=torch.float32, device=params.device)
    _check(load().lx_mlp_grad(ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(feat.data_ptr()),
                              ctypes.c_void_p(target.data_ptr()), feat.shape[0], ctypes.c_void_p(grad.data_ptr()),
                              ctypes.c_void_p(loss.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))), "lx_mlp_grad")
    return loss, grad


def mlp_adam(params, m, v, grad, params_f16, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(load().lx_mlp_adam(ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(m.data_ptr()),
                              ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(grad.data_ptr()),
                              ctypes.c_void_p(params_f16.data_ptr()), int(step), float(lr), float(beta1), float(beta2),
                              float(eps), ctypes.c_void_p(_stream_ptr(stream))), "lx_mlp_adam")


def boys(mmax: int, T, stream=None):
    """F_m(T) (Eq. boys) for a float64 CUDA tensor T: returns (len(T), mmax+1)."""
    import torch
    T = T.contiguous()
    F = torch.empty((T.numel(), mmax + 1), dtype=torch.float64, device=T.device)
    _check(load().lx_boys(mmax, ctypes.c_void_p(T.data_ptr()), T.numel(), ctypes.c_void_p(F.data_ptr()),
                          ctypes.c_void_p(_stream_ptr(stream))), "lx_boys")
    return F


def hermite_R(L: int, params, stream=None):
    """[r]^(0) (Eq. md1) for params (n, 5) = (rho, PQx, PQy, PQz, pref): returns (n, pyr(L))."""
    import torch
    params = params.contiguous()
    n = params.shape[0]
    npyr = (L + 1) * (L + 2) * (L + 3) // 6
    R = torch.empty((n, npyr), dtype=torch.float64, device=params.device)
    _check(load().lx_hermite_R(L, ctypes.c_void_p(params.data_ptr()), n, ctypes.c_void_p(R.data_ptr()),
                               ctypes.c_void_p(_stream_ptr(stream))), "lx_hermite_R")
    return R


def hermite_H(basis: dict, pairs, solid: bool, ket_sign: bool = False, device="cuda", stream=None):
    """H matrices of shell pairs: returns (npair, stride) float64 CUDA tensor and the stride."""
    import torch
    sh = pack_shells(basis)
    ex = np.ascontiguousarray(basis["exps"], dtype=np.float64)
    co = np.ascontiguousarray(basis["coefs"], dtype=np.float64)
    pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    l, K = np.asarray(basis["l"]), np.asarray(basis["nprim"])
    pyr = lambda n: (n + 1) * (n + 2) * (n + 3) // 6
    stride = max(nfun(l[a], solid) * nfun(l[b], solid) * K[a] * K[b] * pyr(l[a] + l[b]) for a, b in pr)
    H = torch.empty((len(pr), stride), dtype=torch.float64, device=device)
    flags = (LX_SOLID if solid else LX_CART) | (LX_KET_SIGN if ket_sign else 0)
    _check(load().lx_hermite_H(_ptr(sh), len(sh), _ptr(ex), _ptr(co), len(ex), _ptr(pr), len(pr), flags,
                               ctypes.c_void_p(H.data_ptr()), stride, ctypes.c_void_p(_stream_ptr(stream))),
           "lx_hermite_H")
    return H, stride
