"""ctypes binding of librankest.so (the C ABI in include/rankest.h).

Argument marshalling only: every numerical step runs in the library's CUDA
kernels.  Functions keep the C names; device buffers may be given as torch CUDA
tensors (their data pointer is passed) or as raw integer addresses.  Loading
fails loudly when the library has not been built; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librankest.so")

RE_OK = 0
RE_ERR_ARG = -1
RE_ERR_CUDA = -2
RE_ERR_NONFINITE = -3
RE_ERR_TIMEOUT = -4
RE_ERR_NOMEM = -5
RE_ERR_UNSUPPORTED = -6

RE_F32 = 0
RE_F64 = 1
RE_GAUSSIAN = 0
RE_SRHT = 1
RE_HRTT = 2
RE_SRCT = 3
RE_HRCT = 4
RE_PREC_FP32 = 0
RE_PREC_BF16X3 = 1
RE_PREC_EXACT = 2
RE_SIGMA_SVD = 0
RE_SIGMA_QRDIAG = 1

RE_MLP_IN = 18
RE_MLP_OUT = 12
RE_MLP_PARAMS = 20492

RE_CONVERGED = 1
RE_LOWER_BOUND_ONLY = 2
RE_TRANSPOSED = 4
RE_QB_DEFLATED = 8


class re_opts(ctypes.Structure):
    _fields_ = [("s0", ctypes.c_int), ("s_max", ctypes.c_int), ("precision", ctypes.c_int),
                ("y_kind", ctypes.c_int), ("norm_a", ctypes.c_double), ("learned", ctypes.c_int),
                ("test_drop_load", ctypes.c_int), ("sigma_est", ctypes.c_int),
                ("batch_first_width", ctypes.c_int), ("first_width", ctypes.c_int),
                ("reserved", ctypes.c_int * 3)]


class re_result(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int), ("gap_index", ctypes.c_int), ("gap_ratio", ctypes.c_double),
                ("tau", ctypes.c_double), ("n_sigma", ctypes.c_int), ("final_s", ctypes.c_int),
                ("passes", ctypes.c_int), ("flags", ctypes.c_uint32), ("status", ctypes.c_int),
                ("svd_sweeps", ctypes.c_int), ("reserved", ctypes.c_int * 2)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class re_block(ctypes.Structure):
    _fields_ = [("ptr", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("ld", ctypes.c_int64)]


class re_kblock(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int64)]


class re_qb_result(ctypes.Structure):
    _fields_ = [("r", ctypes.c_int), ("k", ctypes.c_int), ("final_s", ctypes.c_int), ("passes", ctypes.c_int),
                ("flags", ctypes.c_uint32), ("status", ctypes.c_int), ("bound", ctypes.c_double),
                ("norm_a", ctypes.c_double)]


class re_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("right_launches", ctypes.c_int64),
                ("right_ms", ctypes.c_double), ("right_bytes", ctypes.c_double),
                ("right_flops", ctypes.c_double), ("left_ms", ctypes.c_double),
                ("svd_ms", ctypes.c_double), ("other_ms", ctypes.c_double),
                ("passes", ctypes.c_int64), ("qb_precondition_ms", ctypes.c_double),
                ("qb_orthonormalise_ms", ctypes.c_double), ("qb_product_ms", ctypes.c_double),
                ("reserved", ctypes.c_int64 * 1)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class RankEstError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rankest error {code}: {msg}")
        self.code = code


_lib = None

_VP = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_D = ctypes.c_double

_SIGS = {
    "re_version": (_I, []),
    "re_last_error": (ctypes.c_char_p, []),
    "re_opts_default": (None, [ctypes.POINTER(re_opts)]),
    "re_create": (_I, [ctypes.POINTER(_VP), _I, ctypes.POINTER(re_opts)]),
    "re_destroy": (_I, [_VP]),
    "re_set_opts": (_I, [_VP, ctypes.POINTER(re_opts)]),
    "re_stats_enable": (_I, [_VP, _I]),
    "re_stats_reset": (_I, [_VP]),
    "re_stats_get": (_I, [_VP, ctypes.POINTER(re_stats)]),
    "re_rank_estimate": (_I, [_VP, _VP, _I, _I64, _I64, _I64, _D, _I, _U64, _VP, _I,
                              ctypes.POINTER(re_result), _VP]),
    "re_rank_estimate_host": (_I, [_VP, _VP, _I, _I64, _I64, _I64, _D, _I, _U64, _VP, _I,
                                   ctypes.POINTER(re_result), _VP]),
    "re_sketch_apply": (_I, [_VP, _VP, _I, _I64, _I64, _I64, _I, _I, _I, _U64, _VP, _I64, _VP,
                             _I64, _VP]),
    "re_sketch_apply_exact": (_I, [_VP, _VP, _I64, _I64, _I64, _I, _I, _U64, _VP, _I64, _VP, _I64, _VP]),
    "re_core_sigma": (_I, [_VP, _VP, _I, _I, _I64, _VP, _VP]),
    "re_core_sigma_exact": (_I, [_VP, _VP, _I, _I, _I64, _VP, _VP]),
    "re_embedding_x": (_I, [_VP, _I, _U64, _I64, _I, _I, _VP, _VP]),
    "re_embedding_y": (_I, [_VP, _I, _U64, _I64, _I, _I, _VP, _VP]),
    "re_rank_estimate_batched": (_I, [_VP, ctypes.POINTER(re_block), _I, _I, _D, _I, _U64, _VP,
                                      _I, ctypes.POINTER(re_result), _VP]),
    "re_rank_estimate_kernel_blocks": (_I, [_VP, ctypes.POINTER(re_kblock), _I, _D, _U64, _VP, _I,
                                            ctypes.POINTER(re_result), _VP]),
    "re_rank_estimate_qb": (_I, [_VP, _VP, _I64, _I64, _I64, _D, _I, _U64, _VP, _I64, _VP, _I64, _I,
                                 ctypes.POINTER(re_qb_result), _VP]),
    "re_sketch_apply_noalloc": (_I, [_VP, _I, _I64, _I64, _I64, _I, _I, _U64, _VP, _I64, _VP, _I64,
                                     _VP]),
    "re_mlp_init": (_I, [_VP, _U64]),
    "re_mlp_set_params": (_I, [_VP, _VP, _I]),
    "re_mlp_get_params": (_I, [_VP, _VP, _I]),
    "re_mlp_save": (_I, [_VP, ctypes.c_char_p]),
    "re_mlp_load": (_I, [_VP, ctypes.c_char_p]),
    "re_mlp_predict": (_I, [_VP, _VP, _I, _VP, _VP]),
    "re_mlp_grad": (_I, [_VP, _VP, _VP, _I, _VP, _VP]),
    "re_mlp_train": (_I, [_VP, _VP, _VP, _I, _I, _I, ctypes.c_float, ctypes.c_float, _U64, _VP]),
    "re_mlp_features": (_I, [_VP, _VP, _I, _I64, _I64, _I64, _D, _U64, _VP]),
}

# Symbols declared in include/rankest.h; tests check that the library exports all of them.
EXPORTED = tuple(_SIGS)


def lib():
    """Load librankest.so (raises when it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(code: int) -> None:
    if code != RE_OK:
        raise RankEstError(code, lib().re_last_error().decode())


def re_version() -> int:
    return lib().re_version()


def re_opts_default() -> re_opts:
    o = re_opts()
    lib().re_opts_default(ctypes.byref(o))
    return o


def make_opts(**kw) -> re_opts:
    o = re_opts_default()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def re_create(device: int = 0, opts: re_opts | None = None) -> int:
    h = _VP()
    _check(lib().re_create(ctypes.byref(h), device, ctypes.byref(opts) if opts else None))
    return h.value


def re_destroy(h: int) -> None:
    _check(lib().re_destroy(h))


def re_set_opts(h: int, opts: re_opts) -> None:
    _check(lib().re_set_opts(h, ctypes.byref(opts)))


def re_stats_enable(h: int, timing_on: bool = True) -> None:
    _check(lib().re_stats_enable(h, 1 if timing_on else 0))


def re_stats_reset(h: int) -> None:
    _check(lib().re_stats_reset(h))


def re_stats_get(h: int) -> re_stats:
    st = re_stats()
    _check(lib().re_stats_get(h, ctypes.byref(st)))
    return st


def _dtype_code(A) -> int:
    name = str(getattr(A, "dtype", ""))
    if name.endswith("float32"):
        return RE_F32
    if name.endswith("float64"):
        return RE_F64
    raise TypeError(f"A must be float32 or float64, got {name}")


def re_rank_estimate(h: int, A, eps: float, sketch_kind: int = RE_GAUSSIAN, seed: int = 0,
                     sigma_cap: int = 1024, stream=None, m=None, n=None, ld=None, dtype=None):
    """Algorithm 1 on a device matrix (torch CUDA tensor, 2-D row-major with unit column stride).

    Returns (re_result, sigma) where sigma holds the trusted sketched singular values.
    """
    if m is None:
        m, n = A.shape
        ld = A.stride(0)
        assert A.stride(1) == 1
        dtype = _dtype_code(A)
    sig = np.zeros(max(sigma_cap, 0), dtype=np.float64)
    res = re_result()
    _check(lib().re_rank_estimate(h, _ptr(A), dtype, m, n, ld, eps, sketch_kind, seed,
                                  sig.ctypes.data if sigma_cap else None, sigma_cap,
                                  ctypes.byref(res), _stream(stream)))
    return res, sig[:min(res.n_sigma, sigma_cap)].copy()


def re_rank_estimate_host(h: int, A: np.ndarray, eps: float, sketch_kind: int = RE_GAUSSIAN,
                          seed: int = 0, sigma_cap: int = 1024, stream=None):
    """Algorithm 1 on a host matrix (numpy, C-contiguous float32/float64, or a CPU tensor)."""
    if hasattr(A, "numpy"):
        A = A.numpy()
    A = np.asarray(A)
    assert A.ndim == 2 and A.flags["C_CONTIGUOUS"]
    m, n = A.shape
    sig = np.zeros(max(sigma_cap, 0), dtype=np.float64)
    res = re_result()
    _check(lib().re_rank_estimate_host(h, A.ctypes.data, _dtype_code(A), m, n, n, eps,
                                       sketch_kind, seed, sig.ctypes.data if sigma_cap else None,
                                       sigma_cap, ctypes.byref(res), _stream(stream)))
    return res, sig[:min(res.n_sigma, sigma_cap)].copy()


def re_sketch_apply(h: int, A, col0: int, s: int, sketch_kind: int, seed: int, AX, core=None,
                    stream=None) -> None:
    m, n = A.shape
    assert A.stride(1) == 1 and AX.stride(1) == 1
    # the library writes rows max(m, n) of AX (A^T is sketched when m < n) and the
    # leading 2 (col0 + s) x (col0 + s) block of core
    if AX.shape[0] < max(m, n) or AX.shape[1] < col0 + s:
        raise ValueError(f"AX must be at least {max(m, n)} x {col0 + s}, got {tuple(AX.shape)}")
    if core is not None and (core.shape[0] < 2 * (col0 + s) or core.shape[1] < col0 + s):
        raise ValueError(f"core must be at least {2 * (col0 + s)} x {col0 + s}, got {tuple(core.shape)}")
    ld_core = core.stride(0) if core is not None else 0
    _check(lib().re_sketch_apply(h, _ptr(A), _dtype_code(A), m, n, A.stride(0), col0, s,
                                 sketch_kind, seed, _ptr(AX), AX.stride(0), _ptr(core), ld_core,
                                 _stream(stream)))


def re_sketch_apply_exact(h: int, A, col0: int, s: int, seed: int, AX, core=None, stream=None) -> None:
    """Exact-product sketch step (precision mode): A FP32 CUDA tensor (m >= n), AX
    FP64 (rows x >= col0 + s) receives columns col0..col0+s-1, core FP64 optional."""
    import torch
    m, n = A.shape
    if A.dtype != torch.float32:
        raise ValueError("A must be float32")
    if AX.dtype != torch.float64 or (core is not None and core.dtype != torch.float64):
        raise ValueError("AX and core must be float64")
    if A.stride(1) != 1 or AX.stride(1) != 1 or (core is not None and core.stride(1) != 1):
        raise ValueError("A, AX and core must be row-major (unit column stride)")
    if AX.shape[0] < max(m, n) or AX.shape[1] < col0 + s:
        raise ValueError(f"AX must be at least {max(m, n)} x {col0 + s}")
    if core is not None and (core.shape[0] < 2 * (col0 + s) or core.shape[1] < col0 + s):
        raise ValueError(f"core must be at least {2 * (col0 + s)} x {col0 + s}")
    _check(lib().re_sketch_apply_exact(h, _ptr(A), m, n, A.stride(0), col0, s, seed, _ptr(AX), AX.stride(0),
                                       _ptr(core), core.stride(0) if core is not None else 0, _stream(stream)))


def re_core_sigma(h: int, core, sigma, stream=None, r2=None, s=None) -> None:
    r2 = core.shape[0] if r2 is None else r2
    s = core.shape[1] if s is None else s
    _check(lib().re_core_sigma(h, _ptr(core), r2, s, core.stride(0), _ptr(sigma), _stream(stream)))


def re_core_sigma_exact(h: int, core, sigma, stream=None, r2=None, s=None) -> None:
    r2 = core.shape[0] if r2 is None else r2
    s = core.shape[1] if s is None else s
    _check(lib().re_core_sigma_exact(h, _ptr(core), r2, s, core.stride(0), _ptr(sigma), _stream(stream)))


def re_embedding_x(h: int, kind: int, seed: int, n: int, col0: int, s: int, out, stream=None):
    _check(lib().re_embedding_x(h, kind, seed, n, col0, s, _ptr(out), _stream(stream)))


def re_embedding_y(h: int, kind: int, seed: int, m: int, row0: int, r2: int, out, stream=None):
    _check(lib().re_embedding_y(h, kind, seed, m, row0, r2, _ptr(out), _stream(stream)))


def re_rank_estimate_batched(h: int, blocks, eps: float, sketch_kind: int = RE_GAUSSIAN,
                             seed: int = 0, sigma_cap: int = 0, stream=None, dtype=None):
    """blocks: list of 2-D device tensors (same dtype).  Returns (results, sigma or None)."""
    count = len(blocks)
    arr = (re_block * max(count, 1))()
    for i, B in enumerate(blocks):
        arr[i].ptr = _ptr(B)
        arr[i].m, arr[i].n = B.shape
        arr[i].ld = B.stride(0)
    if dtype is None:
        dtype = _dtype_code(blocks[0]) if count else RE_F32
    res = (re_result * max(count, 1))()
    sig = np.zeros((count, sigma_cap), dtype=np.float64) if sigma_cap > 0 else None
    _check(lib().re_rank_estimate_batched(h, arr, count, dtype, eps, sketch_kind, seed,
                                          sig.ctypes.data if sig is not None else None,
                                          sigma_cap, res, _stream(stream)))
    return [res[i] for i in range(count)], sig


def re_rank_estimate_qb(h: int, A, eps: float, p: int = 10, seed: int = 0, Q=None, B=None, k_cap: int = 0,
                        stream=None):
    """Algorithm 3: returns (result, Q[:, :k], B[:k]) for FP32 device A.  Unless
    given, Q and B are allocated with k_cap = min(min(m, n), 512) columns / rows,
    enough for any width of the ladder; given buffers too small for the chosen k
    raise RankEstError with code RE_ERR_ARG."""
    import torch
    m, n = A.shape
    assert A.stride(1) == 1 and A.is_floating_point() and A.element_size() == 4
    rows, cols = max(m, n), min(m, n)
    if k_cap <= 0:
        k_cap = min(cols, 512)
    if Q is None:
        Q = torch.empty(rows, k_cap, dtype=torch.float32, device=A.device)
    if B is None:
        B = torch.empty(k_cap, cols, dtype=torch.float32, device=A.device)
    res = re_qb_result()
    _check(lib().re_rank_estimate_qb(h, _ptr(A), m, n, A.stride(0), eps, p, seed, _ptr(Q), Q.stride(0), _ptr(B),
                                     B.stride(0), k_cap, ctypes.byref(res), _stream(stream)))
    return res, Q[:, :res.k], B[:res.k]


def re_rank_estimate_kernel_blocks(h: int, points, eps: float, seed: int = 0, sigma_cap: int = 0,
                                   stream=None):
    """points: list of (x, y) device FP32 tensors of shapes (m, 3) and (n, 3), each
    the matrix-free block K = 1/|x_i - y_j|.  Returns (results, sigma or None)."""
    count = len(points)
    arr = (re_kblock * max(count, 1))()
    for i, (x, y) in enumerate(points):
        for t in (x, y):
            if not (t.is_floating_point() and t.element_size() == 4 and t.is_contiguous() and t.shape[1] == 3):
                raise ValueError("points must be contiguous FP32 tensors of shape (k, 3)")
        arr[i].x, arr[i].y = x.data_ptr(), y.data_ptr()
        arr[i].m, arr[i].n = x.shape[0], y.shape[0]
    res = (re_result * max(count, 1))()
    sig = np.zeros((count, sigma_cap), dtype=np.float64) if sigma_cap > 0 else None
    _check(lib().re_rank_estimate_kernel_blocks(h, arr, count, eps, seed,
                                                sig.ctypes.data if sig is not None else None,
                                                sigma_cap, res, _stream(stream)))
    return [res[i] for i in range(count)], sig


def re_sketch_apply_noalloc(A, col0: int, s: int, seed: int, AX, core=None, stream=None) -> None:
    """Gaussian sketch step without device allocation (static 16 MiB scratch, no handle).
    A (FP32 or FP64), AX (FP32) and core (FP64, optional) must be CUDA tensors of one device."""
    import torch
    m, n = A.shape
    if AX.dtype != torch.float32:
        raise ValueError("AX must be float32")
    if core is not None and core.dtype != torch.float64:
        raise ValueError("core must be float64")
    for name, t in (("A", A), ("AX", AX), ("core", core)):
        if t is not None and t.device.type != "cuda":
            raise ValueError(f"{name} must be a CUDA tensor")
    if AX.device != A.device or (core is not None and core.device != A.device):
        raise ValueError("A, AX and core must be on the same device")
    if A.stride(1) != 1 or AX.stride(1) != 1 or (core is not None and core.stride(1) != 1):
        raise ValueError("A, AX and core must be row-major (unit column stride)")
    if AX.shape[0] < max(m, n) or AX.shape[1] < col0 + s:
        raise ValueError(f"AX must be at least {max(m, n)} x {col0 + s}, got {tuple(AX.shape)}")
    if core is not None and (core.shape[0] < 2 * (col0 + s) or core.shape[1] < col0 + s):
        raise ValueError(f"core must be at least {2 * (col0 + s)} x {col0 + s}, got {tuple(core.shape)}")
    ld_core = core.stride(0) if core is not None else 0
    _check(lib().re_sketch_apply_noalloc(_ptr(A), _dtype_code(A), m, n, A.stride(0), col0, s, seed,
                                         _ptr(AX), AX.stride(0), _ptr(core), ld_core,
                                         _stream(stream)))


# ---- sketch-size proposal network ---------------------------------------------
def re_mlp_init(h: int, seed: int = 0) -> None:
    _check(lib().re_mlp_init(h, seed))


def re_mlp_set_params(h: int, params) -> None:
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(lib().re_mlp_set_params(h, p.ctypes.data, p.size))


def re_mlp_get_params(h: int) -> np.ndarray:
    p = np.zeros(RE_MLP_PARAMS, dtype=np.float32)
    _check(lib().re_mlp_get_params(h, p.ctypes.data, p.size))
    return p


def re_mlp_save(h: int, path: str) -> None:
    _check(lib().re_mlp_save(h, path.encode()))


def re_mlp_load(h: int, path: str) -> None:
    _check(lib().re_mlp_load(h, path.encode()))


def re_mlp_predict(h: int, X):
    X = np.ascontiguousarray(X, dtype=np.float32)
    n = X.shape[0]
    cls = np.zeros(n, dtype=np.int32)
    logits = np.zeros((n, RE_MLP_OUT), dtype=np.float32)
    _check(lib().re_mlp_predict(h, X.ctypes.data, n, cls.ctypes.data, logits.ctypes.data))
    return cls, logits


def re_mlp_grad(h: int, X, y):
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.int32)
    g = np.zeros(RE_MLP_PARAMS, dtype=np.float32)
    loss = np.zeros(1, dtype=np.float32)
    _check(lib().re_mlp_grad(h, X.ctypes.data, y.ctypes.data, X.shape[0], g.ctypes.data, loss.ctypes.data))
    return float(loss[0]), g


def re_mlp_train(h: int, X, y, epochs: int = 10, batch: int = 256, lr: float = 1e-3,
                 weight_decay: float = 0.0, seed: int = 0) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.int32)
    losses = np.zeros(epochs, dtype=np.float32)
    _check(lib().re_mlp_train(h, X.ctypes.data, y.ctypes.data, X.shape[0], epochs, batch, lr,
                              weight_decay, seed, losses.ctypes.data))
    return losses


def re_mlp_features(h: int, A, eps: float, seed: int) -> np.ndarray:
    m, n = A.shape
    f = np.zeros(RE_MLP_IN, dtype=np.float32)
    _check(lib().re_mlp_features(h, _ptr(A), _dtype_code(A), m, n, A.stride(0), eps, seed, f.ctypes.data))
    return f
