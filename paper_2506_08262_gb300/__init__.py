"""Python binding of the GB300 RRS depth library (``include/rrs.h``).

Every function named ``rrs_*`` here forwards to the C ABI function of the
same name through ctypes: it only marshals arguments (torch tensors or numpy
arrays to pointers, CUDA streams to handles) and raises ``RRSError`` on a
non-zero status.  All computation runs in the sm_103a kernels of
``_build/librrs.so``; if that library is missing or fails to load, importing
the binding succeeds but every call raises, so nothing can silently fall back
to another implementation.

``Context`` is a small convenience wrapper that owns an ``rrs_ctx`` and takes
torch tensors.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librrs.so")

RRS_OK = 0
RRS_ERR_INVALID_ARG = -1
RRS_ERR_NOT_FOUND = -2
RRS_ERR_BUDGET = -3
RRS_ERR_CUDA = -4
RRS_ERR_TIMEOUT = -5
RRS_ERR_INTERNAL = -6
RRS_ERR_UNSUPPORTED = -7

RRS_F32, RRS_F64 = 0, 1
RRS_HALFSPACE, RRS_PROJECTION, RRS_ASYM_PROJECTION = 0, 1, 2
RRS_PREC_FP32_SIMT, RRS_PREC_SPLIT_BF16X3 = 0, 1
RRS_SELECT_WARP = 64
RRS_SELECT_STREAM = 32


class RRSError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: status {status}")
        self.status = status


class rrs_request(ctypes.Structure):
    _fields_ = [
        ("dataset_id", ctypes.c_int64),
        ("Z", ctypes.c_void_p),
        ("n_queries", ctypes.c_int64),
        ("dtype", ctypes.c_int32),
        ("kind", ctypes.c_int32),
        ("n_dirs", ctypes.c_int32),
        ("n_refinements", ctypes.c_int32),
        ("cap_shrink", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("depth_out", ctypes.c_void_p),
        ("count_out", ctypes.c_void_p),
        ("best_out", ctypes.c_void_p),
        ("round_choice_out", ctypes.c_void_p),
        ("precision", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


_lock = threading.Lock()
_lib = None

_SIGS = {
    "rrs_create": ([ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64], ctypes.c_int32),
    "rrs_destroy": ([ctypes.c_void_p], ctypes.c_int32),
    "rrs_register_dataset": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                              ctypes.c_int32, ctypes.c_void_p], ctypes.c_int32),
    "rrs_free": ([ctypes.c_void_p, ctypes.c_int64], ctypes.c_int32),
    "rrs_depth": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                   ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, ctypes.c_int32,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                   ctypes.c_void_p], ctypes.c_int32),
    "rrs_depth_batched": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p],
                          ctypes.c_int32),
    "rrs_status_string": ([ctypes.c_int32], ctypes.c_char_p),
    "rrs_last_error": ([], ctypes.c_char_p),
    "rrs_debug_directions": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                              ctypes.c_int32, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int32),
    "rrs_debug_round_depths": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int32),
    "rrs_check": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int32),
    "rrs_autotune": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                      ctypes.c_void_p], ctypes.c_int32),
    "rrs_select_kernel": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32],
                          ctypes.c_int32),
    "rrs_select_tc_tile": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32], ctypes.c_int32),
    "rrs_debug_wait_timeout": ([ctypes.c_void_p, ctypes.c_int64], ctypes.c_int32),
    "rrs_launch_count": ([ctypes.c_void_p], ctypes.c_uint64),
    "rrs_profile_enable": ([ctypes.c_void_p, ctypes.c_int32], ctypes.c_int32),
    "rrs_profile_read": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int32),
    "rrs_server_create": ([ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                           ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int32),
    "rrs_server_submit": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                           ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64,
                           ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int32),
    "rrs_server_step": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int32),
    "rrs_server_poll": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p], ctypes.c_int32),
    "rrs_server_set_work_limit": ([ctypes.c_void_p, ctypes.c_double], ctypes.c_int32),
    "rrs_server_destroy": ([ctypes.c_void_p], ctypes.c_int32),
    "rrs_depth_noalloc": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                           ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                           ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int32),
}

RRS_STAGES = ("prep", "gen", "hd_simt", "hd_tc", "pdap", "argmin", "keys")


def exported_symbols():
    """Names of the C ABI entry points this binding expects in librrs.so."""
    return sorted(_SIGS)


def load(path: Optional[str] = None):
    """Load librrs.so (idempotent).  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"librrs.so not built ({p}); run __graft_entry__.build() or "
                               "python paper_2506_08262_gb300/build.py")
        lib = ctypes.CDLL(p)
        for name, (args, res) in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(status: int, what: str):
    if status != RRS_OK:
        lib = load()
        detail = lib.rrs_last_error().decode(errors="replace")
        name = lib.rrs_status_string(status).decode()
        raise RRSError(status, f"{what} failed ({name}): {detail}")


def _ptr(x) -> Optional[int]:
    """Raw address of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s) -> Optional[int]:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ---- C ABI, same names ---------------------------------------------------------

def rrs_create(device: int = 0, hbm_budget_bytes: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load().rrs_create(ctypes.byref(h), device, hbm_budget_bytes), "rrs_create")
    return h.value


def rrs_destroy(ctx: int) -> None:
    _check(load().rrs_destroy(ctx), "rrs_destroy")


def rrs_register_dataset(ctx: int, X, n: int, d: int, dtype: int, x_on_device: bool) -> int:
    out = ctypes.c_int64()
    _check(load().rrs_register_dataset(ctx, _ptr(X), n, d, dtype, int(x_on_device), ctypes.byref(out)),
           "rrs_register_dataset")
    return out.value


def rrs_free(ctx: int, dataset_id: int) -> None:
    _check(load().rrs_free(ctx, dataset_id), "rrs_free")


def rrs_depth(ctx: int, dataset_id: int, Z, n_queries: int, dtype: int, z_on_device: bool, kind: int, n_dirs: int,
              n_refinements: int, cap_shrink: float, seed: int, precision: int, depth_out, count_out=None,
              best_out=None, round_choice_out=None, out_on_device: bool = True, stream=None) -> None:
    _check(load().rrs_depth(ctx, dataset_id, _ptr(Z), n_queries, dtype, int(z_on_device), kind, n_dirs,
                            n_refinements, float(cap_shrink), seed, precision, _ptr(depth_out), _ptr(count_out),
                            _ptr(best_out), _ptr(round_choice_out), int(out_on_device), _stream(stream)),
           "rrs_depth")


def rrs_depth_batched(ctx: int, reqs, use_graph: bool = False, stream=None) -> None:
    arr = (rrs_request * len(reqs))(*reqs)
    _check(load().rrs_depth_batched(ctx, arr, len(reqs), int(use_graph), _stream(stream)), "rrs_depth_batched")


def rrs_debug_directions(ctx: int, seed: int, q: int, round: int, m: int, d: int, cap_shrink: float, pole,
                         U) -> None:
    _check(load().rrs_debug_directions(ctx, seed, q, round, m, d, float(cap_shrink), _ptr(pole), _ptr(U)),
           "rrs_debug_directions")


def rrs_debug_round_depths(ctx: int, dataset_id: int, Z, n_queries: int, dtype: int, kind: int, m: int, U,
                           precision: int, depth_out, count_out=None, band_out=None) -> None:
    _check(load().rrs_debug_round_depths(ctx, dataset_id, _ptr(Z), n_queries, dtype, kind, m, _ptr(U), precision,
                                         _ptr(depth_out), _ptr(count_out), _ptr(band_out)),
           "rrs_debug_round_depths")


def rrs_depth_noalloc(X, n: int, d: int, dtype: int, Z, n_queries: int, kind: int, n_dirs: int,
                      n_refinements: int, cap_shrink: float, seed: int, depth_out, count_out=None,
                      stream=None) -> None:
    """For callers that cannot allocate device memory: all working memory comes from the
    library's fixed device array (RRS_NOALLOC_SCRATCH_BYTES); X, Z and the outputs are
    device pointers; calls must not overlap on the GPU.

    The C entry point takes raw device addresses and cannot tell a host buffer, a short
    buffer or a buffer of the wrong element type from a good one, so this wrapper checks
    every tensor it forwards (CUDA, on the current device, contiguous, dtype and length)
    and raises RRSError(RRS_ERR_INVALID_ARG) before anything reaches the GPU."""
    import torch

    def bad(why):
        raise RRSError(RRS_ERR_INVALID_ARG, f"rrs_depth_noalloc: {why}")

    if dtype not in (RRS_F32, RRS_F64):
        bad(f"unknown dtype code {dtype}")
    want = torch.float32 if dtype == RRS_F32 else torch.float64
    cur = torch.cuda.current_device()
    for name, t, tdt, need in (("X", X, want, n * d), ("Z", Z, want, n_queries * d),
                               ("depth_out", depth_out, torch.float64, n_queries),
                               ("count_out", count_out, torch.int64, n_queries)):
        if t is None:
            if name == "count_out":
                continue
            bad(f"{name} is missing")
        if not isinstance(t, torch.Tensor):
            bad(f"{name} must be a CUDA tensor, got {type(t).__name__}")
        if not t.is_cuda or t.device.index != cur:
            bad(f"{name} must live on the current CUDA device {cur}, got {t.device}")
        if not t.is_contiguous():
            bad(f"{name} must be contiguous")
        if t.dtype != tdt:
            bad(f"{name} must be {tdt}, got {t.dtype}")
        if t.numel() < need:
            bad(f"{name} holds {t.numel()} elements, needs {need}")
    _check(load().rrs_depth_noalloc(_ptr(X), n, d, dtype, _ptr(Z), n_queries, kind, n_dirs, n_refinements,
                                    float(cap_shrink), seed, _ptr(depth_out), _ptr(count_out), _stream(stream)),
           "rrs_depth_noalloc")


def rrs_server_create(ctx: int, max_slots: int, max_dirs_per_round: int, max_d: int, stream=None,
                      precision: int = RRS_PREC_FP32_SIMT) -> int:
    h = ctypes.c_void_p()
    _check(load().rrs_server_create(ctx, max_slots, max_dirs_per_round, max_d, precision, _stream(stream),
                                    ctypes.byref(h)), "rrs_server_create")
    return h.value


def rrs_server_submit(server: int, dataset_id: int, Z, n_queries: int, dtype: int, kind: int, n_dirs: int,
                      n_refinements: int, cap_shrink: float, seed: int, depth_out) -> int:
    rid = ctypes.c_int64()
    _check(load().rrs_server_submit(server, dataset_id, _ptr(Z), n_queries, dtype, kind, n_dirs, n_refinements,
                                    float(cap_shrink), seed, _ptr(depth_out), ctypes.byref(rid)),
           "rrs_server_submit")
    return rid.value


def rrs_server_step(server: int):
    """Returns (active queries, pending requests)."""
    a, p = ctypes.c_int32(), ctypes.c_int32()
    _check(load().rrs_server_step(server, ctypes.byref(a), ctypes.byref(p)), "rrs_server_step")
    return a.value, p.value


def rrs_server_set_work_limit(server: int, max_pairs_per_step: float) -> None:
    _check(load().rrs_server_set_work_limit(server, float(max_pairs_per_step)), "rrs_server_set_work_limit")


def rrs_server_poll(server: int, request_id: int) -> bool:
    done = ctypes.c_int32()
    _check(load().rrs_server_poll(server, request_id, ctypes.byref(done)), "rrs_server_poll")
    return bool(done.value)


def rrs_server_destroy(server: int) -> None:
    _check(load().rrs_server_destroy(server), "rrs_server_destroy")


def rrs_debug_wait_timeout(ctx: int, limit_cycles: int) -> None:
    _check(load().rrs_debug_wait_timeout(ctx, limit_cycles), "rrs_debug_wait_timeout")


def rrs_autotune(ctx: int, dataset_id: int, kind: int, n_dirs: int, n_refinements: int) -> int:
    """Time the selection kernels (projection depths) or the tensor-core tile widths (halfspace) for this
    dataset and cache the fastest; returns the choice."""
    choice = ctypes.c_int32()
    _check(load().rrs_autotune(ctx, dataset_id, kind, n_dirs, n_refinements, ctypes.byref(choice)), "rrs_autotune")
    return choice.value


def rrs_select_kernel(ctx: int, dataset_id: int, n_dirs: int, n_refinements: int, choice: int) -> None:
    """Fix the selection kernel (1, 2, 4 directions per CTA, RRS_SELECT_WARP, RRS_SELECT_STREAM, or 0 for
    the default)."""
    _check(load().rrs_select_kernel(ctx, dataset_id, n_dirs, n_refinements, choice), "rrs_select_kernel")


def rrs_select_tc_tile(ctx: int, dataset_id: int, tile_points: int) -> None:
    """Fix the tensor-core halfspace tile width (128 or 256 points, or 0 for the default)."""
    _check(load().rrs_select_tc_tile(ctx, dataset_id, tile_points), "rrs_select_tc_tile")


def rrs_check(ctx: int, stream=None) -> None:
    _check(load().rrs_check(ctx, _stream(stream)), "rrs_check")


def rrs_launch_count(ctx: int) -> int:
    return int(load().rrs_launch_count(ctx))


def rrs_profile_enable(ctx: int, on: bool = True) -> None:
    _check(load().rrs_profile_enable(ctx, int(on)), "rrs_profile_enable")


def rrs_profile_read(ctx: int):
    """{stage name: (milliseconds, launches)} accumulated since rrs_profile_enable."""
    ms = np.zeros(len(RRS_STAGES), np.float64)
    n = np.zeros(len(RRS_STAGES), np.int64)
    _check(load().rrs_profile_read(ctx, _ptr(ms), _ptr(n)), "rrs_profile_read")
    return {name: (float(ms[i]), int(n[i])) for i, name in enumerate(RRS_STAGES)}


def rrs_status_string(status: int) -> str:
    return load().rrs_status_string(status).decode()


def rrs_last_error() -> str:
    return load().rrs_last_error().decode(errors="replace")


# ---- convenience wrapper over torch tensors -------------------------------------

class Context:
    """Owns an ``rrs_ctx``; datasets and queries are torch tensors (CPU or CUDA)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.device = device
        self.handle = rrs_create(device, hbm_budget_bytes)
        self._dims = {}

    def close(self):
        if self.handle:
            rrs_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _dtype_code(t) -> int:
        import torch
        if t.dtype == torch.float32:
            return RRS_F32
        if t.dtype == torch.float64:
            return RRS_F64
        raise TypeError("X and Z must be float32 or float64")

    def register(self, X) -> int:
        X = X.contiguous()
        n, d = X.shape
        did = rrs_register_dataset(self.handle, X, n, d, self._dtype_code(X), X.is_cuda)
        self._dims[did] = d
        return did

    def free(self, dataset_id: int):
        rrs_free(self.handle, dataset_id)
        self._dims.pop(dataset_id, None)

    def depth(self, dataset_id: int, Z, kind: int, k: int, r: int, alpha: float, seed: int = 0,
              precision: int = RRS_PREC_FP32_SIMT, stream=None, rounds: bool = False):
        """RRS depth of every row of Z; returns CUDA tensors (depth, count, best[, choice])."""
        import torch
        Z = Z.contiguous()
        nq = Z.shape[0]
        dev = torch.device("cuda", self.device)
        depth = torch.empty(nq, dtype=torch.float64, device=dev)
        count = torch.empty(nq, dtype=torch.int64, device=dev)
        best = torch.empty(nq, dtype=torch.int32, device=dev)
        choice = torch.empty((nq, r), dtype=torch.int32, device=dev) if rounds else None
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        rrs_depth(self.handle, dataset_id, Z, nq, self._dtype_code(Z), Z.is_cuda, kind, k, r, alpha, seed,
                  precision, depth, count, best, choice, True, stream)
        rrs_check(self.handle, stream)
        return (depth, count, best, choice) if rounds else (depth, count, best)
