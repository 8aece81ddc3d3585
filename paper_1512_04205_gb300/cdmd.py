"""Python binding of libcdmd (ctypes): argument marshalling only.

Every function here forwards to the C ABI declared in include/cdmd.h under the
same name; all arithmetic runs in the library's CUDA kernels.  PyTorch only
provides device memory and the current CUDA stream.  The library must be
built (paper_1512_04205_gb300.build); importing without it fails loudly.

Tensor conventions (torch views of the C layouts):
  D      uint8 (n, m) frame-major, row stride ldd >= m (the paper's m x n video)
  DY     float64 (n, k): DY[t, i] = (C D)[i, t]  (C layout: k x n column-major)
  lambda complex128 (r,); G complex128 (r, n-1) (G[c, t] = G_tc);
  PhiY   complex128 (r, k); beta complex128 (r,); sel int32 (K,)
  Phi    complex64 (m, ncols) pixel-major
  mask   int32 (n, ceil(m/32)) holding the uint32 words (bit j%32 of word j//32)
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcdmd.so")

CDMD_OK = 0
STATUS_NAMES = {0: "CDMD_OK", 1: "CDMD_ERR_INVALID_ARG", 2: "CDMD_ERR_CUDA", 3: "CDMD_ERR_NOMEM",
                4: "CDMD_ERR_NOT_CONVERGED", 5: "CDMD_ERR_RANK_DEFICIENT", 6: "CDMD_ERR_NONFINITE",
                7: "CDMD_ERR_UNSUPPORTED", 8: "CDMD_ERR_TIMEOUT"}
CTYPES = {"gaussian": 0, "rademacher": 1, "sparse": 2, "rowsample": 3, "srft": 4}
PRECS = {"fp32": 0, "bf16x2": 1}
BGMODES = {"modulus": 0, "real": 1, "static": 2}
SELECTORS = {"omp": 0, "lstsq": 1, "mlp": 2}
MLP_FEATURES, MLP_HIDDEN, MLP_PARAMS, MLP_HEADER, MLP_BLOB = 4, 64, 385, 12, 397

EXPORTED = ["cdmd_create", "cdmd_destroy", "cdmd_last_error", "cdmd_status_string", "cdmd_status_sync",
            "cdmd_measure_sparse_nnz", "cdmd_measure_build", "cdmd_sketch", "cdmd_sketch_gather",
            "cdmd_decompose", "cdmd_lift", "cdmd_subtract", "cdmd_run", "cdmd_run_host",
            "cdmd_workspace_views", "cdmd_sketch_noalloc", "cdmd_set_sm_limit", "cdmd_selector_load",
            "cdmd_selector_features", "cdmd_selector_fallbacks", "cdmd_mlp_forward", "cdmd_mlp_grad",
            "cdmd_mlp_train_step", "cdmd_synth_clip", "cdmd_selector_relabel", "cdmd_batch_create",
            "cdmd_batch_run", "cdmd_batch_status_sync", "cdmd_batch_views", "cdmd_batch_tuning",
            "cdmd_batch_destroy", "cdmd_copy", "cdmd_sketch_shared", "cdmd_run_shared", "cdmd_run_host_shared",
            "cdmd_selftest_wait", "cdmd_median3x3", "cdmd_snapshot_gram", "cdmd_decompose_gram",
            "cdmd_run_exact", "cdmd_decompose_auto", "cdmd_selftest_recip"]
BATCH_GRAPH, BATCH_AUTOTUNE, BATCH_GROUPED = 1, 2, 4


class CdmdError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class cdmd_measure(ctypes.Structure):
    _fields_ = [("ctype", ctypes.c_int), ("k", ctypes.c_int32), ("m", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("density", ctypes.c_double),
                ("col_ptr", ctypes.c_void_p), ("row_idx", ctypes.c_void_p),
                ("nnz_capacity", ctypes.c_int64), ("rows", ctypes.c_void_p)]


class cdmd_clip(ctypes.Structure):
    _fields_ = [("D", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int32), ("ldd", ctypes.c_int64),
                ("k", ctypes.c_int32), ("r", ctypes.c_int32), ("K", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("mask", ctypes.c_void_p)]


class cdmd_batch_params(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("selector", ctypes.c_int), ("bgmode", ctypes.c_int), ("tau", ctypes.c_float),
                ("lanes", ctypes.c_int32), ("flags", ctypes.c_int32), ("selector_blob", ctypes.c_void_p)]


class cdmd_params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("r", ctypes.c_int32), ("K", ctypes.c_int32),
                ("ctype", ctypes.c_int), ("seed", ctypes.c_uint64), ("prec", ctypes.c_int),
                ("selector", ctypes.c_int), ("bgmode", ctypes.c_int), ("tau", ctypes.c_float)]


_lib = None


def load_library(path=LIB_PATH):
    """Load libcdmd.so (raises if it has not been built) and declare prototypes."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libcdmd is not built ({path} missing); run "
                          "python -m paper_1512_04205_gb300.build")
    lib = ctypes.CDLL(path)
    vp, i32, i64, u64, dbl, flt = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                   ctypes.c_double, ctypes.c_float)
    proto = {
        "cdmd_create": [ctypes.POINTER(vp), ctypes.c_int],
        "cdmd_destroy": [vp],
        "cdmd_last_error": [],
        "cdmd_status_string": [ctypes.c_int],
        "cdmd_status_sync": [vp, vp],
        "cdmd_set_sm_limit": [vp, ctypes.c_int],
        "cdmd_measure_sparse_nnz": [vp, i64, ctypes.c_int, u64, dbl, ctypes.POINTER(i64), vp],
        "cdmd_measure_build": [vp, ctypes.POINTER(cdmd_measure), vp],
        "cdmd_sketch": [vp, vp, i64, ctypes.c_int, i64, ctypes.c_int, ctypes.c_int, u64, ctypes.c_int, vp, vp],
        "cdmd_sketch_gather": [vp, vp, i64, ctypes.c_int, i64, ctypes.POINTER(cdmd_measure), vp, vp],
        "cdmd_decompose": [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                           vp, vp, vp, vp, vp, vp, vp, vp],
        "cdmd_lift": [vp, vp, i64, ctypes.c_int, i64, vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, vp, vp],
        "cdmd_subtract": [vp, vp, i64, ctypes.c_int, i64, vp, ctypes.c_int, vp, vp, vp, ctypes.c_int, flt,
                          ctypes.c_int, vp, vp, vp],
        "cdmd_run": [vp, vp, i64, ctypes.c_int, i64, ctypes.POINTER(cdmd_params), vp, vp],
        "cdmd_run_host": [vp, vp, i64, ctypes.c_int, ctypes.POINTER(cdmd_params), vp, vp],
        "cdmd_sketch_shared": [vp, ctypes.c_int, vp, i64, vp, vp, ctypes.c_int, ctypes.c_int, u64, ctypes.c_int, vp,
                               vp],
        "cdmd_run_shared": [vp, ctypes.c_int, vp, i64, vp, vp, ctypes.POINTER(cdmd_params), vp, vp],
        "cdmd_selftest_wait": [vp, ctypes.c_uint32, vp],
        "cdmd_selftest_recip": [vp, vp, i64, vp, vp, vp],
        "cdmd_median3x3": [vp, vp, i64, i64, ctypes.c_int, vp, vp],
        "cdmd_snapshot_gram": [vp, vp, i64, ctypes.c_int, i64, vp, vp],
        "cdmd_decompose_gram": [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int] + [vp] * 7,
        "cdmd_run_exact": [vp, vp, i64, ctypes.c_int, i64, ctypes.POINTER(cdmd_params), vp, vp],
        "cdmd_decompose_auto": [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
                               + [vp] * 7 + [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), vp],
        "cdmd_run_host_shared": [vp, ctypes.c_int, vp, i64, vp, ctypes.POINTER(cdmd_params), vp, vp],
        "cdmd_workspace_views": [vp] + [ctypes.POINTER(vp)] * 8,
        "cdmd_sketch_noalloc": [vp, i64, ctypes.c_int, i64, ctypes.c_int, ctypes.c_int, u64, vp, vp],
        "cdmd_selector_load": [vp, vp, vp],
        "cdmd_batch_create": [ctypes.POINTER(vp), ctypes.c_int, vp, ctypes.c_int, vp, vp],
        "cdmd_batch_run": [vp, vp],
        "cdmd_batch_status_sync": [vp, vp],
        "cdmd_batch_views": [vp, ctypes.c_int] + [ctypes.POINTER(vp)] * 5,
        "cdmd_batch_tuning": [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                              ctypes.POINTER(i32),
                              ctypes.POINTER(flt)],
        "cdmd_batch_destroy": [vp],
        "cdmd_copy": [vp, vp, ctypes.c_size_t, vp],
        "cdmd_selector_relabel": [vp, vp, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_int, vp, ctypes.c_int, vp, vp],
        "cdmd_synth_clip": [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, vp, ctypes.c_int,
                            ctypes.c_int, flt, flt, u64, vp, i64, vp],
        "cdmd_selector_features": [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp, vp, vp],
        "cdmd_selector_fallbacks": [vp, ctypes.POINTER(i64), ctypes.c_int, vp],
        "cdmd_mlp_forward": [vp, vp, vp, i64, ctypes.c_int, vp, vp, vp],
        "cdmd_mlp_grad": [vp, vp, vp, vp, i64, vp, vp, vp],
        "cdmd_mlp_train_step": [vp, vp, vp, vp, ctypes.c_int, flt, flt, flt, flt, vp, vp, i64, vp, vp],
    }
    for name, args in proto.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.cdmd_destroy.restype = None
    lib.cdmd_batch_destroy.restype = None
    lib.cdmd_last_error.restype = ctypes.c_char_p
    lib.cdmd_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status):
    if status != CDMD_OK:
        msg = load_library().cdmd_last_error().decode(errors="replace")
        raise CdmdError(status, msg)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _video(D):
    import torch
    if D.dtype != torch.uint8 or D.dim() != 2 or D.stride(1) != 1 or not D.is_cuda:
        raise ValueError("D must be a CUDA uint8 tensor (n, m) with unit pixel stride")
    n, m = D.shape
    return n, m, D.stride(0)


class Context:
    """Owns a cdmd_ctx (workspace + device status word) on one device."""

    def __init__(self, device=0):
        self.lib = load_library()
        self.handle = ctypes.c_void_p()
        _check(self.lib.cdmd_create(ctypes.byref(self.handle), int(device)))
        self.device = int(device)

    def close(self):
        if self.handle:
            self.lib.cdmd_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cdmd_set_sm_limit(ctx, max_sms):
    """Cap the full-data passes of this context at max_sms SMs (0 = all)."""
    _check(ctx.lib.cdmd_set_sm_limit(ctx.handle, int(max_sms)))


def cdmd_status_sync(ctx, stream=None):
    """Synchronise the stream and raise if the device recorded an error."""
    _check(ctx.lib.cdmd_status_sync(ctx.handle, _stream(stream)))


def cdmd_sketch(ctx, D, k, seed, ctype="gaussian", prec="fp32", DY=None, stream=None):
    """Pass (a): DY = C D with C generated in-kernel (returns (n, k) float64)."""
    import torch
    n, m, ldd = _video(D)
    if DY is None:
        DY = torch.empty((n, k), dtype=torch.float64, device=D.device)
    _check(ctx.lib.cdmd_sketch(ctx.handle, _ptr(D), m, n, ldd, CTYPES[ctype], int(k), int(seed) & (2**64 - 1),
                               PRECS[prec], _ptr(DY), _stream(stream)))
    return DY


def _arrays(tensors):
    """Host arrays of device pointers, frame counts and row strides of a
    list of videos (n, m) of one pixel count."""
    vids = [_video(D) for D in tensors]
    ms = {v[1] for v in vids}
    if len(ms) != 1:
        raise ValueError("every clip must have the same pixel count")
    cnt = len(tensors)
    ptrs = (ctypes.c_void_p * cnt)(*[t.data_ptr() for t in tensors])
    ns = (ctypes.c_int * cnt)(*[v[0] for v in vids])
    ldds = (ctypes.c_int64 * cnt)(*[v[2] for v in vids])
    return ptrs, ns, ldds, ms.pop()


def cdmd_sketch_shared(ctx, Ds, k, seed, ctype="gaussian", prec="fp32", DYs=None, stream=None):
    """Pass (a) for several clips of one pixel count with one C: returns
    [DY_i (n_i, k) float64]; with prec="bf16x2" consecutive clips share the
    generator two at a time."""
    import torch
    ptrs, ns, ldds, m = _arrays(Ds)
    if DYs is None:
        DYs = [torch.empty((D.shape[0], k), dtype=torch.float64, device=D.device) for D in Ds]
    out = (ctypes.c_void_p * len(Ds))(*[t.data_ptr() for t in DYs])
    _check(ctx.lib.cdmd_sketch_shared(ctx.handle, len(Ds), ptrs, m, ns, ldds, CTYPES[ctype], int(k),
                                      int(seed) & (2**64 - 1), PRECS[prec], out, _stream(stream)))
    return DYs


def cdmd_sketch_noalloc(D, k, seed, ctype="gaussian", DY=None, stream=None):
    """Pass (a) in FP32 without any device allocation by the library: the
    partial sums live in a fixed 16 MiB array inside libcdmd (for callers
    that cannot allocate once running).  Runs on the current device; the
    first call on a device must precede any stream capture; k * n is limited
    to 4,194,304.  Returns DY (n, k) float64 (allocated here by torch unless
    DY is given)."""
    import torch
    n, m, ldd = _video(D)
    if D.device.index != torch.cuda.current_device():
        raise ValueError("cdmd_sketch_noalloc runs on the current device (cuda:%d); D is on %s"
                         % (torch.cuda.current_device(), D.device))
    if DY is None:
        DY = torch.empty((n, k), dtype=torch.float64, device=D.device)
    elif (DY.dtype != torch.float64 or tuple(DY.shape) != (n, k) or not DY.is_contiguous()
          or DY.device != D.device):
        raise ValueError("DY must be a contiguous float64 tensor (n, k) = (%d, %d) on %s" % (n, k, D.device))
    _check(load_library().cdmd_sketch_noalloc(_ptr(D), m, n, ldd, CTYPES[ctype], int(k), int(seed) & (2**64 - 1),
                                              _ptr(DY), _stream(stream)))
    return DY


class Measure:
    """Device-resident SPARSE, ROWSAMPLE or SRFT measurement matrix."""

    def __init__(self, ctx, ctype, m, k, seed, density=0.0, stream=None):
        import torch
        self.struct = cdmd_measure()
        s = self.struct
        s.ctype, s.k, s.m, s.seed, s.density = CTYPES[ctype], int(k), int(m), int(seed) & (2**64 - 1), float(density)
        dev = torch.device("cuda", ctx.device)
        self.col_ptr = self.row_idx = self.rows = None
        if ctype == "sparse":
            nnz = ctypes.c_int64()
            _check(ctx.lib.cdmd_measure_sparse_nnz(ctx.handle, int(m), int(k), s.seed, float(density),
                                                   ctypes.byref(nnz), _stream(stream)))
            self.nnz = nnz.value
            self.col_ptr = torch.empty(int(m) + 1, dtype=torch.int64, device=dev)
            self.row_idx = torch.empty(max(1, self.nnz), dtype=torch.int32, device=dev)
            s.col_ptr, s.row_idx, s.nnz_capacity = self.col_ptr.data_ptr(), self.row_idx.data_ptr(), self.row_idx.numel()
        elif ctype == "rowsample":
            self.rows = torch.empty(int(k), dtype=torch.int64, device=dev)
            s.rows = self.rows.data_ptr()
        elif ctype == "srft":
            self.rows = torch.empty((int(k) + 1) // 2, dtype=torch.int64, device=dev)   # kept frequencies
            s.rows = self.rows.data_ptr()
        else:
            raise ValueError("Measure holds SPARSE, ROWSAMPLE or SRFT matrices")
        _check(ctx.lib.cdmd_measure_build(ctx.handle, ctypes.byref(s), _stream(stream)))


def cdmd_sketch_gather(ctx, D, meas, DY=None, stream=None):
    """Pass (a) with a sparse or single-pixel C (returns (n, k) float64)."""
    import torch
    n, m, ldd = _video(D)
    if DY is None:
        DY = torch.empty((n, meas.struct.k), dtype=torch.float64, device=D.device)
    _check(ctx.lib.cdmd_sketch_gather(ctx.handle, _ptr(D), m, n, ldd, ctypes.byref(meas.struct), _ptr(DY),
                                      _stream(stream)))
    return DY


def decompose_outputs(n, k, r, K, device, with_phiy=False):
    """Preallocated output tensors for cdmd_decompose."""
    import torch
    dev = device
    return dict(sigma=torch.empty(r, dtype=torch.float64, device=dev),
                lam=torch.empty((r, 2), dtype=torch.float64, device=dev),
                G=torch.empty((r, n - 1, 2), dtype=torch.float64, device=dev),
                PhiY=torch.empty((r, k, 2), dtype=torch.float64, device=dev) if with_phiy else None,
                beta=torch.empty((r, 2), dtype=torch.float64, device=dev),
                sel=torch.empty(K, dtype=torch.int32, device=dev),
                nsel=torch.empty(1, dtype=torch.int32, device=dev))


def cdmd_decompose(ctx, DY, r, K, selector="omp", with_phiy=False, stream=None, out=None):
    """Steps 4-7 and 9 on the device; returns a dict of device tensors."""
    import torch
    n, k = DY.shape
    dev = DY.device
    if out is not None:
        _check(ctx.lib.cdmd_decompose(ctx.handle, _ptr(DY), int(k), int(n), int(r), int(K), SELECTORS[selector],
                                      _ptr(out["sigma"]), _ptr(out["lam"]), _ptr(out["G"]), _ptr(out["PhiY"]),
                                      _ptr(out["beta"]), _ptr(out["sel"]), _ptr(out["nsel"]), _stream(stream)))
        return out
    out = dict(sigma=torch.empty(r, dtype=torch.float64, device=dev),
               lam=torch.empty((r, 2), dtype=torch.float64, device=dev),
               G=torch.empty((r, n - 1, 2), dtype=torch.float64, device=dev),
               PhiY=torch.empty((r, k, 2), dtype=torch.float64, device=dev) if with_phiy else None,
               beta=torch.empty((r, 2), dtype=torch.float64, device=dev),
               sel=torch.empty(K, dtype=torch.int32, device=dev),
               nsel=torch.empty(1, dtype=torch.int32, device=dev))
    _check(ctx.lib.cdmd_decompose(ctx.handle, _ptr(DY), int(k), int(n), int(r), int(K), SELECTORS[selector],
                                  _ptr(out["sigma"]), _ptr(out["lam"]), _ptr(out["G"]), _ptr(out["PhiY"]),
                                  _ptr(out["beta"]), _ptr(out["sel"]), _ptr(out["nsel"]), _stream(stream)))
    return out


def cdmd_decompose_auto(ctx, DY, r_max, K, selector="omp", with_phiy=False, stream=None, out=None):
    """cdmd_decompose with the rank from the optimal hard threshold (at most
    r_max); synchronises the stream once.  Returns (outputs, r, tau); the
    outputs are sized for r_max and their first r entries are valid."""
    n, k = DY.shape
    if out is None:
        out = decompose_outputs(n, k, r_max, K, DY.device, with_phiy=with_phiy)
    r = ctypes.c_int(0)
    tau = ctypes.c_double(0.0)
    _check(ctx.lib.cdmd_decompose_auto(ctx.handle, _ptr(DY), int(k), int(n), int(r_max), int(K), SELECTORS[selector],
                                       _ptr(out["sigma"]), _ptr(out["lam"]), _ptr(out["G"]), _ptr(out["PhiY"]),
                                       _ptr(out["beta"]), _ptr(out["sel"]), _ptr(out["nsel"]), ctypes.byref(r),
                                       ctypes.byref(tau), _stream(stream)))
    return out, r.value, tau.value


def cdmd_snapshot_gram(ctx, D, R=None, stream=None):
    """Exact DMD's full-data pass: R = D^T D (n, n) float64 of a device video."""
    import torch
    n, m, ldd = _video(D)
    if R is None:
        R = torch.empty((n, n), dtype=torch.float64, device=D.device)
    _check(ctx.lib.cdmd_snapshot_gram(ctx.handle, _ptr(D), m, n, ldd, _ptr(R), _stream(stream)))
    return R


def cdmd_decompose_gram(ctx, R, r, K, selector="omp", stream=None, out=None):
    """cdmd_decompose's outputs (no PhiY) from an (n, n) float64 Gram."""
    import torch
    n = R.shape[0]
    if out is None:
        dev = R.device
        out = dict(sigma=torch.empty(r, dtype=torch.float64, device=dev),
                   lam=torch.empty((r, 2), dtype=torch.float64, device=dev),
                   G=torch.empty((r, n - 1, 2), dtype=torch.float64, device=dev),
                   beta=torch.empty((r, 2), dtype=torch.float64, device=dev),
                   sel=torch.empty(K, dtype=torch.int32, device=dev),
                   nsel=torch.empty(1, dtype=torch.int32, device=dev))
    _check(ctx.lib.cdmd_decompose_gram(ctx.handle, _ptr(R), int(n), int(r), int(K), SELECTORS[selector],
                                       _ptr(out["sigma"]), _ptr(out["lam"]), _ptr(out["G"]), _ptr(out["beta"]),
                                       _ptr(out["sel"]), _ptr(out["nsel"]), _stream(stream)))
    return out


def cdmd_lift(ctx, D, G, cols=None, ncols=None, prec="fp32", Phi=None, stream=None):
    """Pass (b): Phi = X' G[:, cols] (returns (m, ncols, 2) float32)."""
    import torch
    n, m, ldd = _video(D)
    r = G.shape[0]
    if ncols is None:
        ncols = cols.numel() if cols is not None else r
    if Phi is None:
        Phi = torch.empty((m, ncols, 2), dtype=torch.float32, device=D.device)
    _check(ctx.lib.cdmd_lift(ctx.handle, _ptr(D), m, n, ldd, _ptr(G), int(r), _ptr(cols), int(ncols), PRECS[prec],
                             _ptr(Phi), _stream(stream)))
    return Phi


def cdmd_subtract(ctx, D, Phi, beta, lam, tau, cols=None, mode="modulus", want_bg=False, mask=None, stream=None,
                  bg=None):
    """Pass (c): bit-packed foreground mask (n, ceil(m/32)) int32, optional bg."""
    import torch
    n, m, ldd = _video(D)
    ncols = Phi.shape[1]
    r = beta.shape[0]
    if mask is None:
        mask = torch.empty((n, (m + 31) // 32), dtype=torch.int32, device=D.device)
    if want_bg and bg is None:
        bg = torch.empty((n, m), dtype=torch.float32, device=D.device)
    _check(ctx.lib.cdmd_subtract(ctx.handle, _ptr(D), m, n, ldd, _ptr(Phi), int(ncols), _ptr(cols), _ptr(beta),
                                 _ptr(lam), int(r), float(tau), BGMODES[mode], _ptr(mask), _ptr(bg),
                                 _stream(stream)))
    return (mask, bg) if want_bg else mask


def make_params(k, r, K, tau, seed=0, ctype="gaussian", prec="fp32", selector="omp", bgmode="modulus"):
    return cdmd_params(int(k), int(r), int(K), CTYPES[ctype], int(seed) & (2**64 - 1), PRECS[prec],
                       SELECTORS[selector], BGMODES[bgmode], float(tau))


def cdmd_run(ctx, D, params, mask=None, stream=None):
    """Whole pipeline on a device video; returns the mask (n, ceil(m/32)) int32."""
    import torch
    n, m, ldd = _video(D)
    if mask is None:
        mask = torch.empty((n, (m + 31) // 32), dtype=torch.int32, device=D.device)
    _check(ctx.lib.cdmd_run(ctx.handle, _ptr(D), m, n, ldd, ctypes.byref(params), _ptr(mask), _stream(stream)))
    return mask


def cdmd_run_exact(ctx, D, params, mask=None, stream=None):
    """Exact DMD end to end on a device video (snapshot Gram, decompose, lift,
    subtract); returns the mask (n, ceil(m/32)) int32."""
    import torch
    n, m, ldd = _video(D)
    if mask is None:
        mask = torch.empty((n, (m + 31) // 32), dtype=torch.int32, device=D.device)
    _check(ctx.lib.cdmd_run_exact(ctx.handle, _ptr(D), m, n, ldd, ctypes.byref(params), _ptr(mask),
                                  _stream(stream)))
    return mask


def cdmd_run_host(ctx, D_host, params, mask_host=None, stream=None):
    """Whole pipeline on a host video (n, m) uint8 (pinned torch tensor or
    numpy array); copies in, runs, copies the mask out and synchronises."""
    import torch
    if isinstance(D_host, np.ndarray):
        D_host = torch.from_numpy(np.ascontiguousarray(D_host))
    if D_host.dtype != torch.uint8 or D_host.dim() != 2 or not D_host.is_contiguous() or D_host.is_cuda:
        raise ValueError("D_host must be a contiguous host uint8 tensor (n, m)")
    n, m = D_host.shape
    if mask_host is None:
        mask_host = torch.empty((n, (m + 31) // 32), dtype=torch.int32, pin_memory=D_host.is_pinned())
    _check(ctx.lib.cdmd_run_host(ctx.handle, _ptr(D_host), m, n, ctypes.byref(params), _ptr(mask_host),
                                 _stream(stream)))
    return mask_host


def cdmd_run_shared(ctx, Ds, params, masks=None, stream=None):
    """Whole pipeline on 1..8 device videos of one pixel count with one C;
    returns their masks."""
    import torch
    ptrs, ns, ldds, m = _arrays(Ds)
    if masks is None:
        masks = [torch.empty((D.shape[0], (m + 31) // 32), dtype=torch.int32, device=D.device) for D in Ds]
    out = (ctypes.c_void_p * len(Ds))(*[t.data_ptr() for t in masks])
    _check(ctx.lib.cdmd_run_shared(ctx.handle, len(Ds), ptrs, m, ns, ldds, ctypes.byref(params), out,
                                   _stream(stream)))
    return masks


def cdmd_run_host_shared(ctx, D_hosts, params, mask_hosts=None, stream=None):
    """cdmd_run_shared on host videos (n_i, m) uint8 (pinned for full copy
    bandwidth): copies in, runs, copies the masks out and synchronises."""
    import torch
    hs = []
    for D in D_hosts:
        if isinstance(D, np.ndarray):
            D = torch.from_numpy(np.ascontiguousarray(D))
        if D.dtype != torch.uint8 or D.dim() != 2 or not D.is_contiguous() or D.is_cuda:
            raise ValueError("each host video must be a contiguous host uint8 tensor (n, m)")
        hs.append(D)
    m = hs[0].shape[1]
    if any(D.shape[1] != m for D in hs):
        raise ValueError("every clip must have the same pixel count")
    if mask_hosts is None:
        mask_hosts = [torch.empty((D.shape[0], (m + 31) // 32), dtype=torch.int32, pin_memory=D.is_pinned())
                      for D in hs]
    cnt = len(hs)
    ptrs = (ctypes.c_void_p * cnt)(*[D.data_ptr() for D in hs])
    ns = (ctypes.c_int * cnt)(*[D.shape[0] for D in hs])
    out = (ctypes.c_void_p * cnt)(*[t.data_ptr() for t in mask_hosts])
    _check(ctx.lib.cdmd_run_host_shared(ctx.handle, cnt, ptrs, m, ns, ctypes.byref(params), out, _stream(stream)))
    return mask_hosts


def cdmd_median3x3(ctx, mask, W, H, out=None, stream=None):
    """3 x 3 median filter of each frame of a bit-packed mask (n, ceil(W*H/32))
    int32 on the device; returns a new mask (or fills `out`)."""
    import torch
    if mask.dim() != 2 or not mask.is_contiguous() or mask.dtype != torch.int32:
        raise ValueError("mask must be a contiguous (n, words) int32 tensor")
    n = mask.shape[0]
    if mask.shape[1] != (int(W) * int(H) + 31) // 32:
        raise ValueError("mask has %d words per frame, W*H needs %d" % (mask.shape[1], (W * H + 31) // 32))
    if out is None:
        out = torch.empty_like(mask)
    _check(ctx.lib.cdmd_median3x3(ctx.handle, _ptr(mask), int(W), int(H), int(n), _ptr(out), _stream(stream)))
    return out


def cdmd_selftest_wait(ctx, limit_us, stream=None):
    """Enqueue a kernel whose bounded wait on a barrier nothing arrives at gives
    up after limit_us; the next cdmd_status_sync raises CDMD_ERR_TIMEOUT."""
    _check(ctx.lib.cdmd_selftest_wait(ctx.handle, int(limit_us), _stream(stream)))


def cdmd_selftest_recip(ctx, a, stream=None):
    """The small solves' FP64 reciprocal and reciprocal square root applied
    to a float64 device tensor; returns (1/a, 1/sqrt(a))."""
    import torch
    if a.dtype != torch.float64 or not a.is_cuda or not a.is_contiguous():
        raise ValueError("a must be a contiguous float64 CUDA tensor")
    r = torch.empty_like(a)
    q = torch.empty_like(a)
    _check(ctx.lib.cdmd_selftest_recip(ctx.handle, _ptr(a), int(a.numel()), _ptr(r), _ptr(q), _stream(stream)))
    return r, q


def cdmd_workspace_views(ctx):
    """Raw device pointers of the last cdmd_run's intermediates."""
    ptrs = [ctypes.c_void_p() for _ in range(8)]
    _check(ctx.lib.cdmd_workspace_views(ctx.handle, *[ctypes.byref(p) for p in ptrs]))
    keys = ["DY", "sigma", "lambda", "G", "beta", "sel", "nsel", "Phi"]
    return {k: p.value for k, p in zip(keys, ptrs)}


def workspace_tensors(ctx, m, n, k, r, K, stream=None):
    """Device copies of the last cdmd_run's intermediates on ctx (the last
    clip of a cdmd_run_shared): DY (n, k), sigma (r,), lam (r, 2), G
    (r, n-1, 2), beta (r, 2), sel (K,), nsel (1,), Phi (m, K, 2) float32."""
    import torch
    v = cdmd_workspace_views(ctx)
    dev = torch.device("cuda", torch.cuda.current_device())
    shapes = dict(DY=((n, k), torch.float64), sigma=((r,), torch.float64), lambda_=((r, 2), torch.float64),
                  G=((r, n - 1, 2), torch.float64), beta=((r, 2), torch.float64), sel=((K,), torch.int32),
                  nsel=((1,), torch.int32), Phi=((m, K, 2), torch.float32))
    out = {}
    for name, (shape, dtype) in shapes.items():
        key = "lambda" if name == "lambda_" else name
        t = torch.empty(shape, dtype=dtype, device=dev)
        _check(ctx.lib.cdmd_copy(_ptr(t), ctypes.c_void_p(v[key]), t.numel() * t.element_size(), _stream(stream)))
        out["lam" if key == "lambda" else key] = t
    return out


def unpack_mask(mask, m):
    """(n, words) int32 mask -> (m, n) bool array (host), pixel j = bit j%32."""
    words = np.asarray(mask.cpu().numpy() if hasattr(mask, "cpu") else mask).view(np.uint32)
    bits = np.unpackbits(words.view(np.uint8), axis=1, bitorder="little")
    return bits[:, :m].astype(bool).T


# ---------------------------------------------------------------------------
# learned mode selector
# ---------------------------------------------------------------------------


def cdmd_selector_load(ctx, blob, stream=None):
    """Load a model blob (float32 device tensor of MLP_BLOB values) for selector='mlp'."""
    assert blob.dtype.is_floating_point and blob.numel() == MLP_BLOB
    _check(ctx.lib.cdmd_selector_load(ctx.handle, _ptr(blob), _stream(stream)))


def cdmd_selector_features(ctx, lam, sel, r, K, labels=True, stream=None):
    """Features (r, 4) and OMP labels (r,) of the last decomposition on ctx."""
    import torch
    feats = torch.empty((r, MLP_FEATURES), dtype=torch.float32, device=lam.device)
    lab = torch.empty(r, dtype=torch.float32, device=lam.device) if labels else None
    _check(ctx.lib.cdmd_selector_features(ctx.handle, _ptr(lam), _ptr(sel), int(r), int(K), _ptr(feats),
                                          _ptr(lab), _stream(stream)))
    return feats, lab


def cdmd_selector_relabel(ctx, DY, dec, r, y_target, K, stream=None):
    """OMP picks (K,) on the last decomposition's modes against y_target (k,)."""
    import torch
    n, k = DY.shape
    sel = torch.empty(K, dtype=torch.int32, device=DY.device)
    _check(ctx.lib.cdmd_selector_relabel(ctx.handle, _ptr(DY), int(k), int(n), _ptr(dec["G"]), _ptr(dec["lam"]),
                                         int(r), _ptr(y_target), int(K), _ptr(sel), _stream(stream)))
    return sel


def cdmd_selector_fallbacks(ctx, reset=False, stream=None):
    """Fallbacks to OMP taken by selector='mlp' since the last load/reset."""
    c = ctypes.c_int64()
    _check(ctx.lib.cdmd_selector_fallbacks(ctx.handle, ctypes.byref(c), int(bool(reset)), _stream(stream)))
    return c.value


def cdmd_mlp_forward(ctx, blob, X, bf16=True, stream=None):
    """Logits and probabilities of N feature rows (device tensors)."""
    import torch
    N = X.shape[0]
    s = torch.empty(N, dtype=torch.float32, device=X.device)
    p = torch.empty(N, dtype=torch.float32, device=X.device)
    _check(ctx.lib.cdmd_mlp_forward(ctx.handle, _ptr(blob), _ptr(X), int(N), int(bool(bf16)), _ptr(s), _ptr(p),
                                    _stream(stream)))
    return s, p


def cdmd_mlp_grad(ctx, blob, X, Y, stream=None):
    """Mean BCE loss and gradient over the rows (device tensors)."""
    import torch
    grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device=X.device)
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    _check(ctx.lib.cdmd_mlp_grad(ctx.handle, _ptr(blob), _ptr(X), _ptr(Y), int(X.shape[0]), _ptr(grad), _ptr(loss),
                                 _stream(stream)))
    return loss, grad


def cdmd_mlp_train_step(ctx, blob, m, v, step, lr, X, Y, beta1=0.9, beta2=0.999, eps=1e-8, loss=None, stream=None):
    """One Adam step in place on blob's parameters and the moments m, v."""
    _check(ctx.lib.cdmd_mlp_train_step(ctx.handle, _ptr(blob), _ptr(m), _ptr(v), int(step), float(lr), float(beta1),
                                       float(beta2), float(eps), _ptr(X), _ptr(Y), int(X.shape[0]), _ptr(loss),
                                       _stream(stream)))


def cdmd_synth_clip(ctx, spec, seed, D=None, stream=None):
    """Render a clip described by a scene spec (videogen.clip_spec layout:
    width, height, n, waves, objects, shape, drift, noise_sigma) on the
    device; returns (n, width*height) uint8."""
    import torch
    W, H, n = spec["width"], spec["height"], spec["n"]
    dev = torch.device("cuda", ctx.device)
    if D is None:
        D = torch.empty((n, W * H), dtype=torch.uint8, device=dev)
    waves = torch.as_tensor(np.asarray(spec["waves"], dtype=np.float32)).to(dev)
    objs = torch.as_tensor(np.asarray(spec["objects"], dtype=np.float32)).to(dev)
    _check(ctx.lib.cdmd_synth_clip(ctx.handle, int(W), int(H), int(n), _ptr(waves), int(waves.shape[0]), _ptr(objs),
                                   int(objs.shape[1]) if objs.ndim == 3 else 0, int(spec["shape"] == "ellipse"),
                                   float(spec["drift"]), float(spec["noise_sigma"]), int(seed) & (2**64 - 1),
                                   _ptr(D), int(D.stride(0)), _stream(stream)))
    return D


# ---------------------------------------------------------------------------
# batches
# ---------------------------------------------------------------------------


class Batch:
    """A planned batch of clips (see cdmd_batch_create).

    clips: list of dicts with D (CUDA uint8 (n, m) tensor, unit pixel
    stride), k, r, K, seed.  Masks are allocated here (self.masks[i],
    (n, ceil(m/32)) int32).  The tensors must stay alive and unmoved while
    the batch exists; this object keeps references to them."""

    def __init__(self, clips, tau, prec="fp32", selector="omp", bgmode="modulus", lanes=0, graph=True,
                 autotune=False, grouped=True, selector_blob=None, device=0, stream=None):
        import torch
        self.lib = load_library()
        self.handle = ctypes.c_void_p()
        self.videos = [c["D"] for c in clips]
        self.masks = []
        arr = (cdmd_clip * len(clips))()
        for i, c in enumerate(clips):
            n, m, ldd = _video(c["D"])
            mask = torch.empty((n, (m + 31) // 32), dtype=torch.int32, device=c["D"].device)
            self.masks.append(mask)
            arr[i] = cdmd_clip(c["D"].data_ptr(), m, n, ldd, int(c["k"]), int(c["r"]), int(c["K"]),
                               int(c["seed"]) & (2**64 - 1), mask.data_ptr())
        self.meta = [dict(m=int(c["D"].shape[1]), n=int(c["D"].shape[0]), k=int(c["k"]), r=int(c["r"]),
                          K=int(c["K"])) for c in clips]
        self.selector = selector
        flags = (BATCH_GRAPH if graph else 0) | (BATCH_AUTOTUNE if autotune else 0) | (BATCH_GROUPED if grouped else 0)
        self.blob = selector_blob
        p = cdmd_batch_params(PRECS[prec], SELECTORS[selector], BGMODES[bgmode], float(tau), int(lanes), flags,
                              _ptr(selector_blob))
        _check(self.lib.cdmd_batch_create(ctypes.byref(self.handle), int(device), arr, len(clips), ctypes.byref(p),
                                          _stream(stream)))

    def run(self, stream=None):
        _check(self.lib.cdmd_batch_run(self.handle, _stream(stream)))

    def status_sync(self, stream=None):
        _check(self.lib.cdmd_batch_status_sync(self.handle, _stream(stream)))

    def tuning(self):
        v = [ctypes.c_int32() for _ in range(5)]
        ms = ctypes.c_float()
        _check(self.lib.cdmd_batch_tuning(self.handle, *[ctypes.byref(x) for x in v], ctypes.byref(ms)))
        return dict(lanes=v[0].value, sm_limit=v[1].value, waves=v[2].value, sketch_steps=v[3].value,
                    subtract_tiles=v[4].value, run_ms=ms.value)

    def views(self, i, stream=None):
        """Host copies of clip i's DY (n, k), lambda (r,), beta (r,), sel (K,)."""
        ptrs = [ctypes.c_void_p() for _ in range(5)]
        _check(self.lib.cdmd_batch_views(self.handle, int(i), *[ctypes.byref(q) for q in ptrs]))
        md = self.meta[i]

        def fetch(ptr, shape, dtype):
            out = np.empty(shape, dtype=dtype)
            _check(self.lib.cdmd_copy(out.ctypes.data_as(ctypes.c_void_p), ptr, out.nbytes, _stream(stream)))
            return out
        import torch
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        DY = fetch(ptrs[0], (md["n"], md["k"]), np.float64)
        lam = fetch(ptrs[1], (md["r"], 2), np.float64)
        beta = fetch(ptrs[2], (md["r"], 2), np.float64)
        sel = fetch(ptrs[3], (md["K"],), np.int32)
        torch.cuda.synchronize()
        return dict(DY=DY, lam=lam[:, 0] + 1j * lam[:, 1], beta=beta[:, 0] + 1j * beta[:, 1], sel=sel)

    def close(self):
        if self.handle:
            self.lib.cdmd_batch_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
