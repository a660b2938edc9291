"""Python binding of the C ABI in ``include/bblock.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does nothing
but check dtypes/shapes, turn tensors into pointers and raise on error codes:
all arithmetic of the path runs in the CUDA library ``_build/libbblock.so``.
PyTorch supplies device memory and streams. If the library has not been built,
:func:`load` raises; there is no fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbblock.so")

BBLOCK_OK = 0
ERRORS = {
    -1: "BBLOCK_ERR_INVALID_ARG",
    -2: "BBLOCK_ERR_UNSUPPORTED",
    -3: "BBLOCK_ERR_OOM",
    -4: "BBLOCK_ERR_CUDA",
    -5: "BBLOCK_ERR_TIMEOUT",
    -6: "BBLOCK_ERR_DEVICE_FLAG",
    -7: "BBLOCK_ERR_TOO_LARGE",
}
PRECISIONS = {"fp64": 0, "tf32x3": 1, "bf16": 2, "df64": 3, "fp16x3": 4, "ozaki": 5}

# Every symbol include/bblock.h declares.
EXPORTED = (
    "bblock_create", "bblock_destroy", "bblock_last_error", "bblock_status", "bblock_compute",
    "bblock_compute_host", "bblock_compute_batch", "bblock_workspace_bytes",
    "bblock_last_launch_count", "bblock_last_wave_count", "bblock_last_path",
    "bblock_profile_enable", "bblock_profile_read",
    "bblock_contract_noalloc", "bblock_set_option", "bblock_get_option", "bblock_autotune",
    "bblock_costmodel_create", "bblock_costmodel_destroy", "bblock_costmodel_num_params",
    "bblock_costmodel_get_params", "bblock_costmodel_set_params", "bblock_costmodel_gradient",
    "bblock_costmodel_train", "bblock_costmodel_predict", "bblock_mode_triplet",
    "bblock_from_triplet", "bblock_probe_fp64",
)
TUNE_FEATURES = 12
OPTIONS = {"graphs": 1, "tc_nc": 2, "tc_chunk": 3, "slabs": 4, "checks": 5, "wave_mb": 6,
           "wait_limit_us": 7, "fail_next_alloc": 8, "corrupt_canary": 9, "tc_cluster": 10,
           "host_chunks": 11, "tc_projection": 12, "tc_rows": 13}


class BblockError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class bblock_config(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("n_ev", ctypes.c_int), ("max_ndil", ctypes.c_int),
                ("precision", ctypes.c_int), ("bf16_products", ctypes.c_int),
                ("device", ctypes.c_int)]


class bblock_job(ctypes.Structure):
    _fields_ = [("V", ctypes.c_void_p), ("phi1", ctypes.c_void_p), ("phi2", ctypes.c_void_p),
                ("phi3", ctypes.c_void_p), ("nd1", ctypes.c_int), ("nd2", ctypes.c_int),
                ("nd3", ctypes.c_int), ("B_out", ctypes.c_void_p)]


class bblock_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int),
                ("total_ms", ctypes.c_double)]


class bblock_tune_entry(ctypes.Structure):
    _fields_ = [("nc", ctypes.c_int), ("chunk", ctypes.c_int), ("slabs", ctypes.c_int),
                ("features", ctypes.c_float * TUNE_FEATURES), ("predicted", ctypes.c_float),
                ("ms", ctypes.c_double)]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Open the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is missing; run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    P, I = ctypes.c_void_p, ctypes.c_int
    lib.bblock_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(bblock_config)]
    lib.bblock_create.restype = I
    lib.bblock_destroy.argtypes = [P]
    lib.bblock_destroy.restype = None
    lib.bblock_last_error.argtypes = [P]
    lib.bblock_last_error.restype = ctypes.c_char_p
    lib.bblock_status.argtypes = [P]
    lib.bblock_status.restype = I
    compute_sig = [P, I, P, P, P, P, I, I, I, P, I, P, P, I, I, P, P]
    lib.bblock_compute.argtypes = compute_sig
    lib.bblock_compute.restype = I
    lib.bblock_compute_host.argtypes = compute_sig
    lib.bblock_compute_host.restype = I
    lib.bblock_compute_batch.argtypes = [P, ctypes.POINTER(bblock_job), I, P, I, P, P, I, I, P]
    lib.bblock_compute_batch.restype = I
    lib.bblock_mode_triplet.argtypes = [P, I, P, P, I, P, P]
    lib.bblock_mode_triplet.restype = I
    lib.bblock_from_triplet.argtypes = [P, I, P, P, P, P, I, I, I, I, P, P, I, I, P, P]
    lib.bblock_from_triplet.restype = I
    lib.bblock_workspace_bytes.argtypes = [P]
    lib.bblock_workspace_bytes.restype = ctypes.c_size_t
    lib.bblock_last_launch_count.argtypes = [P]
    lib.bblock_last_launch_count.restype = I
    lib.bblock_last_wave_count.argtypes = [P]
    lib.bblock_last_wave_count.restype = I
    lib.bblock_last_path.argtypes = [P]
    lib.bblock_last_path.restype = I
    lib.bblock_probe_fp64.argtypes = [I, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double), P]
    lib.bblock_probe_fp64.restype = I
    lib.bblock_profile_enable.argtypes = [P, I]
    lib.bblock_profile_enable.restype = I
    lib.bblock_profile_read.argtypes = [P, ctypes.POINTER(bblock_kernel_stat), I,
                                        ctypes.POINTER(I)]
    lib.bblock_profile_read.restype = I
    lib.bblock_contract_noalloc.argtypes = [I, P, P, P, I, I, I, P, I, P, P, I, P, P,
                                            ctypes.c_char_p, ctypes.c_size_t]
    lib.bblock_contract_noalloc.restype = I
    lib.bblock_set_option.argtypes = [P, I, I]
    lib.bblock_set_option.restype = I
    lib.bblock_get_option.argtypes = [P, I]
    lib.bblock_get_option.restype = I
    lib.bblock_autotune.argtypes = [P, I, P, P, P, P, I, I, I, P, I, P, P, I, P, P, P, I, I,
                                    ctypes.POINTER(bblock_tune_entry), I, ctypes.POINTER(I)]
    lib.bblock_autotune.restype = I
    F = ctypes.POINTER(ctypes.c_float)
    lib.bblock_costmodel_create.argtypes = [ctypes.POINTER(P), I, I, ctypes.c_uint64, I]
    lib.bblock_costmodel_create.restype = I
    lib.bblock_costmodel_destroy.argtypes = [P]
    lib.bblock_costmodel_destroy.restype = None
    lib.bblock_costmodel_num_params.argtypes = [P]
    lib.bblock_costmodel_num_params.restype = I
    lib.bblock_costmodel_get_params.argtypes = [P, F, I]
    lib.bblock_costmodel_get_params.restype = I
    lib.bblock_costmodel_set_params.argtypes = [P, F, I]
    lib.bblock_costmodel_set_params.restype = I
    lib.bblock_costmodel_gradient.argtypes = [P, F, F, I, F, F]
    lib.bblock_costmodel_gradient.restype = I
    lib.bblock_costmodel_train.argtypes = [P, F, F, I, I, ctypes.c_float, F]
    lib.bblock_costmodel_train.restype = I
    lib.bblock_costmodel_predict.argtypes = [P, F, I, F]
    lib.bblock_costmodel_predict.restype = I
    _lib = lib
    return lib


class Context:
    """Owner of a ``bblock_ctx*``; destroyed with :func:`bblock_destroy` or on GC."""

    def __init__(self, handle: int, config: bblock_config):
        self.handle = handle
        self.config = config

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bblock_destroy(self.handle)
            self.handle = None


def _check(ctx: Optional[Context], rc: int):
    if rc != BBLOCK_OK:
        msg = load().bblock_last_error(ctx.handle).decode() if ctx is not None and ctx.handle else ""
        raise BblockError(rc, msg)


def bblock_create(L: int, n_ev: int, max_ndil: int, precision: str = "fp64",
                  bf16_products: int = 6, device: int = 0) -> Context:
    lib = load()
    cfg = bblock_config(L, n_ev, max_ndil, PRECISIONS[precision], bf16_products, device)
    h = ctypes.c_void_p()
    rc = lib.bblock_create(ctypes.byref(h), ctypes.byref(cfg))
    if rc != BBLOCK_OK:
        raise BblockError(rc, f"bblock_create({L}, {n_ev}, {max_ndil}, {precision}) failed")
    return Context(h.value, cfg)


def bblock_destroy(ctx: Context) -> None:
    if ctx.handle:
        load().bblock_destroy(ctx.handle)
        ctx.handle = None


def bblock_status(ctx: Context) -> None:
    _check(ctx, load().bblock_status(ctx.handle))


def bblock_last_error(ctx: Context) -> str:
    return load().bblock_last_error(ctx.handle).decode()


def bblock_workspace_bytes(ctx: Context) -> int:
    return int(load().bblock_workspace_bytes(ctx.handle))


def bblock_last_launch_count(ctx: Context) -> int:
    return int(load().bblock_last_launch_count(ctx.handle))


def bblock_last_wave_count(ctx: Context) -> int:
    return int(load().bblock_last_wave_count(ctx.handle))


PATHS = {0: "fp64", 1: "tc", 2: "tc_cluster", 3: "tc_pairs", 4: "tc_rows", 5: "tc_rows_cluster",
         6: "ozaki"}


def bblock_last_path(ctx: Context) -> str:
    """Contraction path of the last compute call (see BBLOCK_PATH_* in the header)."""
    return PATHS.get(int(load().bblock_last_path(ctx.handle)), "none")


def bblock_probe_fp64(device: int = 0, stream=None) -> dict:
    """Measured FP64 rates of the device: {"dfma_tflops": .., "dmma_tflops": ..}."""
    a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
    rc = load().bblock_probe_fp64(device, ctypes.byref(a), ctypes.byref(b),
                                  _stream_handle(stream))
    _check(None, rc)
    return {"dfma_tflops": a.value, "dmma_tflops": b.value}


def bblock_set_option(ctx: Context, option: str, value: int) -> None:
    """Set a context option: "graphs", "tc_nc", "tc_chunk" or "slabs" (see include/bblock.h)."""
    _check(ctx, load().bblock_set_option(ctx.handle, OPTIONS[option], int(value)))


def bblock_get_option(ctx: Context, option: str) -> int:
    v = load().bblock_get_option(ctx.handle, OPTIONS[option])
    _check(ctx, min(v, 0))
    return int(v)


def bblock_profile_enable(ctx: Context, enable: bool = True) -> None:
    _check(ctx, load().bblock_profile_enable(ctx.handle, 1 if enable else 0))


def bblock_profile_read(ctx: Context) -> dict:
    """{kernel name: (launches, total ms)} since the last read (synchronises)."""
    out = (bblock_kernel_stat * 16)()
    n = ctypes.c_int(0)
    _check(ctx, load().bblock_profile_read(ctx.handle, out, 16, ctypes.byref(n)))
    return {out[i].name.decode(): (out[i].launches, out[i].total_ms) for i in range(n.value)}


# ------------------------------------------------------------------ marshalling helpers

def _spin_arrays(momenta, spin_idx, spin_coeffs):
    mom = np.ascontiguousarray(np.asarray(momenta, dtype=np.int32).reshape(-1, 3))
    spins = np.ascontiguousarray(np.asarray(spin_idx, dtype=np.int32).reshape(-1, 3))
    coeffs = np.ascontiguousarray(np.asarray(spin_coeffs, dtype=np.complex128))
    per_mom = 1 if coeffs.ndim == 2 else 0
    if per_mom and coeffs.shape != (mom.shape[0], spins.shape[0]):
        raise ValueError("per-momentum spin_coeffs must have shape (n_mom, n_spin)")
    if not per_mom and coeffs.shape != (spins.shape[0],):
        raise ValueError("spin_coeffs must have shape (n_spin,) or (n_mom, n_spin)")
    return mom, spins, coeffs, per_mom


def _dev_ptr(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA torch tensor")
    if t.dtype != torch.complex128 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous complex128 tensor")
    return t.data_ptr()


def _host_ptr(a, name):
    import torch
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != torch.complex128 or not a.is_contiguous():
            raise TypeError(f"{name} must be a contiguous complex128 host tensor")
        return a.data_ptr()
    if not isinstance(a, np.ndarray) or a.dtype != np.complex128 or not a.flags.c_contiguous:
        raise TypeError(f"{name} must be a C-contiguous complex128 array")
    return a.ctypes.data


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _shape_checks(ctx, V, phis, n_t):
    cfg = ctx.config
    X = cfg.L ** 3
    if tuple(V.shape) != (n_t, cfg.n_ev, X, 3):
        raise ValueError(f"V must have shape (n_t, n_ev, L^3, 3) = {(n_t, cfg.n_ev, X, 3)}")
    nds = []
    for i, p in enumerate(phis):
        if p.ndim != 3 or p.shape[0] != n_t or p.shape[1] != 4 * cfg.n_ev:
            raise ValueError(f"phi{i + 1} must have shape (n_t, 4*n_ev, nd)")
        nds.append(int(p.shape[2]))
    return nds


def bblock_compute(ctx: Context, V, phi1, phi2, phi3, momenta, spin_idx, spin_coeffs,
                   B_out=None, stream=None):
    """Blocks B[t][p][d1][d2][d3] of device tensors (see include/bblock.h). Returns B_out."""
    import torch
    n_t = int(V.shape[0])
    nds = _shape_checks(ctx, V, (phi1, phi2, phi3), n_t)
    mom, spins, coeffs, per_mom = _spin_arrays(momenta, spin_idx, spin_coeffs)
    if B_out is None:
        B_out = torch.empty((n_t, mom.shape[0], *nds), dtype=torch.complex128, device=V.device)
    rc = load().bblock_compute(
        ctx.handle, n_t, _dev_ptr(V, "V"), _dev_ptr(phi1, "phi1"), _dev_ptr(phi2, "phi2"),
        _dev_ptr(phi3, "phi3"), nds[0], nds[1], nds[2], mom.ctypes.data, mom.shape[0],
        spins.ctypes.data, coeffs.ctypes.data, spins.shape[0], per_mom, _dev_ptr(B_out, "B_out"),
        _stream_handle(stream))
    _check(ctx, rc)
    return B_out


def bblock_mode_triplet(ctx: Context, V, momenta, T_out=None, stream=None):
    """Eq. (4): T[t][p][l1][l2][l3] of device eigenvectors V (n_t, n_ev, L^3, 3)."""
    import torch
    cfg = ctx.config
    n_t = int(V.shape[0])
    if tuple(V.shape) != (n_t, cfg.n_ev, cfg.L ** 3, 3):
        raise ValueError("V must have shape (n_t, n_ev, L^3, 3)")
    mom = np.ascontiguousarray(np.asarray(momenta, dtype=np.int32).reshape(-1, 3))
    shape = (n_t, mom.shape[0], cfg.n_ev, cfg.n_ev, cfg.n_ev)
    if T_out is None:
        T_out = torch.empty(shape, dtype=torch.complex128, device=V.device)
    elif tuple(T_out.shape) != shape:
        raise ValueError(f"T_out must have shape {shape}")
    rc = load().bblock_mode_triplet(ctx.handle, n_t, _dev_ptr(V, "V"), mom.ctypes.data,
                                    mom.shape[0], _dev_ptr(T_out, "T_out"), _stream_handle(stream))
    _check(ctx, rc)
    return T_out


def bblock_from_triplet(ctx: Context, T, phi1, phi2, phi3, spin_idx, spin_coeffs, B_out=None,
                        stream=None):
    """Blocks from the mode triplet (Eq. 3 in mode-triplet order); T as returned by
    bblock_mode_triplet, phi_i (n_t, 4 n_ev, nd_i) device tensors."""
    import torch
    cfg = ctx.config
    n_t, n_mom = int(T.shape[0]), int(T.shape[1])
    if tuple(T.shape) != (n_t, n_mom, cfg.n_ev, cfg.n_ev, cfg.n_ev):
        raise ValueError("T must have shape (n_t, n_mom, n_ev, n_ev, n_ev)")
    nds = []
    for i, p in enumerate((phi1, phi2, phi3)):
        if p.ndim != 3 or p.shape[0] != n_t or p.shape[1] != 4 * cfg.n_ev:
            raise ValueError(f"phi{i + 1} must have shape (n_t, 4*n_ev, nd)")
        nds.append(int(p.shape[2]))
    _, spins, coeffs, per_mom = _spin_arrays(np.zeros((n_mom, 3), np.int32), spin_idx, spin_coeffs)
    if B_out is None:
        B_out = torch.empty((n_t, n_mom, *nds), dtype=torch.complex128, device=T.device)
    rc = load().bblock_from_triplet(
        ctx.handle, n_t, _dev_ptr(T, "T"), _dev_ptr(phi1, "phi1"), _dev_ptr(phi2, "phi2"),
        _dev_ptr(phi3, "phi3"), nds[0], nds[1], nds[2], n_mom, spins.ctypes.data,
        coeffs.ctypes.data, spins.shape[0], per_mom, _dev_ptr(B_out, "B_out"),
        _stream_handle(stream))
    _check(ctx, rc)
    return B_out


def bblock_compute_host(ctx: Context, V, phi1, phi2, phi3, momenta, spin_idx, spin_coeffs,
                        B_out, stream=None):
    """Same as bblock_compute from host buffers (numpy or CPU tensors); blocks until done."""
    n_t = int(V.shape[0])
    nds = _shape_checks(ctx, V, (phi1, phi2, phi3), n_t)
    mom, spins, coeffs, per_mom = _spin_arrays(momenta, spin_idx, spin_coeffs)
    if tuple(B_out.shape) != (n_t, mom.shape[0], *nds):
        raise ValueError("B_out has the wrong shape")
    rc = load().bblock_compute_host(
        ctx.handle, n_t, _host_ptr(V, "V"), _host_ptr(phi1, "phi1"), _host_ptr(phi2, "phi2"),
        _host_ptr(phi3, "phi3"), nds[0], nds[1], nds[2], mom.ctypes.data, mom.shape[0],
        spins.ctypes.data, coeffs.ctypes.data, spins.shape[0], per_mom, _host_ptr(B_out, "B_out"),
        _stream_handle(stream))
    _check(ctx, rc)
    return B_out


def bblock_compute_batch(ctx: Context, jobs: Sequence[tuple], momenta, spin_idx, spin_coeffs,
                         stream=None) -> None:
    """jobs: sequence of (V_t, phi1_t, phi2_t, phi3_t, B_out_t) single-slice device tensors."""
    cfg = ctx.config
    arr = (bblock_job * max(1, len(jobs)))()
    for k, (V, p1, p2, p3, B) in enumerate(jobs):
        if tuple(V.shape) != (cfg.n_ev, cfg.L ** 3, 3):
            raise ValueError("job V must have shape (n_ev, L^3, 3)")
        nds = [int(p.shape[1]) for p in (p1, p2, p3)]
        arr[k] = bblock_job(_dev_ptr(V, "V"), _dev_ptr(p1, "phi1"), _dev_ptr(p2, "phi2"),
                            _dev_ptr(p3, "phi3"), nds[0], nds[1], nds[2], _dev_ptr(B, "B_out"))
    mom, spins, coeffs, per_mom = _spin_arrays(momenta, spin_idx, spin_coeffs)
    rc = load().bblock_compute_batch(ctx.handle, arr, len(jobs), mom.ctypes.data, mom.shape[0],
                                     spins.ctypes.data, coeffs.ctypes.data, spins.shape[0],
                                     per_mom, _stream_handle(stream))
    _check(ctx, rc)


def bblock_contract_noalloc(L: int, q1, q2, q3, momenta, spin_idx, spin_coeffs, B_out,
                            stream=None):
    """Allocation-free contraction from reconstructed fields q_i[alpha][x][a][d]
    (device complex128 [4][L^3][3][nd_i]) into B_out [n_mom][nd1][nd2][nd3]; see
    include/bblock.h. For callers that must not allocate device memory."""
    X = L ** 3
    nds = []
    for i, q in enumerate((q1, q2, q3)):
        if q.ndim != 4 or tuple(q.shape[:3]) != (4, X, 3):
            raise ValueError(f"q{i + 1} must have shape (4, L^3, 3, nd)")
        nds.append(int(q.shape[3]))
    mom, spins, coeffs, per_mom = _spin_arrays(momenta, spin_idx, spin_coeffs)
    if per_mom:
        raise ValueError("bblock_contract_noalloc takes one coefficient per spin triple")
    if tuple(B_out.shape) != (mom.shape[0], *nds):
        raise ValueError("B_out must have shape (n_mom, nd1, nd2, nd3)")
    err = ctypes.create_string_buffer(256)
    rc = load().bblock_contract_noalloc(
        L, _dev_ptr(q1, "q1"), _dev_ptr(q2, "q2"), _dev_ptr(q3, "q3"), nds[0], nds[1], nds[2],
        mom.ctypes.data, mom.shape[0], spins.ctypes.data, coeffs.ctypes.data, spins.shape[0],
        _dev_ptr(B_out, "B_out"), _stream_handle(stream), err, len(err))
    if rc != BBLOCK_OK:
        raise BblockError(rc, err.value.decode())
    return B_out


# ------------------------------------------------------------------ autotuner and cost model

def _f32(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class CostModel:
    """Owner of a ``bblock_costmodel*`` (MLP trained on the GPU by the library's kernels)."""

    def __init__(self, n_features: int = TUNE_FEATURES, hidden: int = 32, seed: int = 1,
                 device: int = 0):
        lib = load()
        h = ctypes.c_void_p()
        rc = lib.bblock_costmodel_create(ctypes.byref(h), n_features, hidden, seed, device)
        if rc != BBLOCK_OK:
            raise BblockError(rc, "bblock_costmodel_create failed")
        self.handle, self.F, self.H = h.value, n_features, hidden

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bblock_costmodel_destroy(self.handle)
            self.handle = None

    def num_params(self) -> int:
        return int(load().bblock_costmodel_num_params(self.handle))

    def get_params(self) -> np.ndarray:
        out, ptr = _f32(np.zeros(self.num_params()))
        _check(None, load().bblock_costmodel_get_params(self.handle, ptr, out.size))
        return out

    def set_params(self, p) -> None:
        a, ptr = _f32(p)
        _check(None, load().bblock_costmodel_set_params(self.handle, ptr, a.size))

    def gradient(self, X, y):
        Xa, xp = _f32(X)
        ya, yp = _f32(y)
        loss, lp = _f32(np.zeros(1))
        grad, gp = _f32(np.zeros(self.num_params()))
        _check(None, load().bblock_costmodel_gradient(self.handle, xp, yp, ya.size, lp, gp))
        return float(loss[0]), grad

    def train(self, X, y, epochs: int = 500, lr: float = 1e-2) -> float:
        Xa, xp = _f32(X)
        ya, yp = _f32(y)
        loss, lp = _f32(np.zeros(1))
        _check(None, load().bblock_costmodel_train(self.handle, xp, yp, ya.size, epochs, lr, lp))
        return float(loss[0])

    def predict(self, X) -> np.ndarray:
        Xa, xp = _f32(X)
        n = Xa.shape[0]
        out, op = _f32(np.zeros(n))
        _check(None, load().bblock_costmodel_predict(self.handle, xp, n, op))
        return out


def bblock_autotune(ctx: Context, V, phi1, phi2, phi3, momenta, spin_idx, spin_coeffs, B_out,
                    stream=None, model: Optional[CostModel] = None, top_k: int = 3,
                    repeats: int = 3):
    """Time tile candidates, keep the fastest in the context; returns one dict per candidate."""
    n_t = int(V.shape[0])
    nds = _shape_checks(ctx, V, (phi1, phi2, phi3), n_t)
    mom, spins, coeffs, per_mom = _spin_arrays(momenta, spin_idx, spin_coeffs)
    if per_mom:
        raise ValueError("bblock_autotune takes one coefficient per spin triple")
    rep = (bblock_tune_entry * 64)()
    n = ctypes.c_int(0)
    rc = load().bblock_autotune(
        ctx.handle, n_t, _dev_ptr(V, "V"), _dev_ptr(phi1, "phi1"), _dev_ptr(phi2, "phi2"),
        _dev_ptr(phi3, "phi3"), nds[0], nds[1], nds[2], mom.ctypes.data, mom.shape[0],
        spins.ctypes.data, coeffs.ctypes.data, spins.shape[0], _dev_ptr(B_out, "B_out"),
        _stream_handle(stream), model.handle if model is not None else None, top_k, repeats,
        rep, 64, ctypes.byref(n))
    _check(ctx, rc)
    return [{"nc": rep[i].nc, "chunk": rep[i].chunk, "slabs": rep[i].slabs,
             "features": np.array(rep[i].features[:], np.float32),
             "predicted": float(rep[i].predicted), "ms": float(rep[i].ms)} for i in range(n.value)]
