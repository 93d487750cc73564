"""Python binding of the C ABI in include/omp_gb300.h (argument marshalling only).

The functions carry the C names and take torch CUDA tensors; every computation runs in
``libomp_gb300.so``. There is no fallback: if the library is missing or the GPU is not an sm_103
device, the calls raise.

Tensor conventions (same as the C ABI):
  A            (M, N) float32 in column-major storage, i.e. ``A.stride() == (1, M)``
               (``At.t()`` for a contiguous (N, M) ``At``, or ``torch.from_numpy`` of a Fortran
               array)
  Y / R        (B, M) float32, contiguous
  X_out        (B, S) float32, support_out (B, S) int32
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

from .build import LIB

PRECISIONS = {"fp32": 0, "bf16": 1, "fp8": 2, "fp8_e4m3": 2}
STATUS = {0: "OMP_OK", 1: "OMP_ERR_INVALID_ARGUMENT", 2: "OMP_ERR_UNSUPPORTED_DEVICE",
          3: "OMP_ERR_OUT_OF_MEMORY", 4: "OMP_ERR_CUDA", 5: "OMP_ERR_DEVICE_TIMEOUT",
          6: "OMP_ERR_NUMERICAL"}
DEVERR_WAIT_TIMEOUT, DEVERR_NONFINITE, DEVERR_BAD_STATE = 0x1, 0x2, 0x4
STOP_ITERS, STOP_EPS, STOP_DEPENDENT, STOP_ZERO = 0, 1, 2, 3

# every symbol include/omp_gb300.h declares
EXPORTS = ["omp_desc_default", "omp_create", "omp_destroy", "omp_prepare_dictionary",
           "omp_solve_batch", "omp_solve_batch_ex", "omp_solve_batch_host", "omp_correlate_topk",
           "omp_get_error", "omp_status_string", "omp_profile_enable", "omp_profile_read",
           "omp_correlate_argmax_noalloc", "omp_solve_batch_trace", "omp_handle_info",
           "omp_proposal_desc_default", "omp_proposal_create", "omp_proposal_destroy",
           "omp_proposal_set_weights", "omp_proposal_get_weights", "omp_proposal_train_step",
           "omp_proposal_gradients", "omp_proposal_infer", "omp_proposal_set_thresholds",
           "omp_proposal_get_thresholds", "omp_proposal_calibrate", "omp_topk_rows",
           "omp_proposal_baseline_candidates", "omp_solve_batch_candidates",
           "omp_synthesize_signals", "omp_solve_batch_learned", "omp_autotune",
           "omp_loop_passes", "omp_read_bandwidth_probe", "omp_solve_batch_gram",
           "omp_score_error_bound", "omp_proposal_save", "omp_proposal_load", "omp_tuning"]
NOALLOC_MAX_SIGNALS = 65536


class omp_desc(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int64), ("N", ctypes.c_int64), ("max_batch", ctypes.c_int64),
                ("max_iters", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("rescore_topk", ctypes.c_int32), ("eps_relative", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("device", ctypes.c_int32),
                ("gather24", ctypes.c_int32)]


class omp_proposal_desc(ctypes.Structure):
    _fields_ = [("hidden", ctypes.c_int32), ("topk", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("train_batch", ctypes.c_int32), ("lr", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("weight_decay", ctypes.c_float),
                ("adam_eps", ctypes.c_float), ("pos_weight", ctypes.c_float)]


class OmpError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


_lib = None
_P = ctypes.c_void_p
_I64, _I32, _F32 = ctypes.c_int64, ctypes.c_int32, ctypes.c_float


def load(path: Optional[str] = None):
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(the CUDA library is required; there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    sig = {
        "omp_desc_default": (None, [ctypes.POINTER(omp_desc), _I64, _I64]),
        "omp_create": (_I32, [ctypes.POINTER(omp_desc), ctypes.POINTER(_P)]),
        "omp_destroy": (_I32, [_P]),
        "omp_prepare_dictionary": (_I32, [_P, _P, _P]),
        "omp_solve_batch": (_I32, [_P, _P, _P, _I64, _I32, _F32, _P, _P, _P]),
        "omp_solve_batch_ex": (_I32, [_P, _P, _P, _I64, _I32, _F32, _P, _P, _P, _P, _P, _P, _P]),
        "omp_solve_batch_host": (_I32, [_P, _P, _P, _I64, _I32, _F32, _P, _P, _P]),
        "omp_correlate_topk": (_I32, [_P, _P, _P, _I64, _I32, _P, _P, _P]),
        "omp_get_error": (_I32, [_P, ctypes.POINTER(_I32), _P]),
        "omp_status_string": (ctypes.c_char_p, [_I32]),
        "omp_profile_enable": (_I32, [_P, _I32]),
        "omp_profile_read": (_I32, [_P, _I32, _P, _P, _P, _P]),
        "omp_correlate_argmax_noalloc": (_I32, [_P, _P, _I64, _I64, _I64, _P, _P, _P]),
        "omp_solve_batch_trace": (_I32, [_P, _P, _P, _I64, _I32, _F32, _P, _P, _P, _P]),
        "omp_handle_info": (_I32, [_P, ctypes.POINTER(omp_desc), ctypes.POINTER(_I32)]),
        "omp_loop_passes": (_I32, [_P, ctypes.POINTER(_I32), _P]),
        "omp_solve_batch_gram": (_I32, [_P, _P, _P, _I64, _I32, _F32, _P, _P, _P, _P, _P, _P]),
        "omp_read_bandwidth_probe": (_I32, [_P, _I64, _I32, _P, _I32, _P]),
        "omp_score_error_bound": (_F32, [_I32, _I64]),
        "omp_proposal_desc_default": (None, [ctypes.POINTER(omp_proposal_desc)]),
        "omp_proposal_create": (_I32, [_P, ctypes.POINTER(omp_proposal_desc), ctypes.POINTER(_P)]),
        "omp_proposal_destroy": (_I32, [_P]),
        "omp_proposal_set_weights": (_I32, [_P, _P, _P, _P, _P, _P, _P]),
        "omp_proposal_get_weights": (_I32, [_P, _P, _P, _P, _P, _P, _P]),
        "omp_proposal_train_step": (_I32, [_P, _P, _P, _P, _I64, _I32, _P, _P]),
        "omp_proposal_gradients": (_I32, [_P, _P, _P, _P, _I64, _I32, _P, _P, _P, _P, _P, _P, _P]),
        "omp_proposal_infer": (_I32, [_P, _P, _P, _I64, _P, _P, _P]),
        "omp_proposal_set_thresholds": (_I32, [_P, _P, _I32]),
        "omp_proposal_get_thresholds": (_I32, [_P, _P, _I32]),
        "omp_proposal_calibrate": (_I32, [_P, _P, _I64, _I32, _F32, _P]),
        "omp_proposal_save": (_I32, [_P, ctypes.c_char_p]),
        "omp_proposal_load": (_I32, [_P, ctypes.c_char_p]),
        "omp_topk_rows": (_I32, [_P, _I64, _I64, _I32, _P, _P]),
        "omp_proposal_baseline_candidates": (_I32, [_P, _P, _P, _I64, _P, _P]),
        "omp_solve_batch_candidates": (_I32, [_P, _P, _P, _I64, _I32, _F32, _P, _I32, _P, _P, _P, _P,
                                              _P, _P, _P]),
        "omp_synthesize_signals": (_I32, [_P, _I64, _I64, _P, _P, _P, _I64, _I32, _P, _P]),
        "omp_solve_batch_learned": (_I32, [_P, _P, _P, _P, _I64, _I32, _F32, _P, _P, _P, _P, _P, _P]),
        "omp_autotune": (_I32, [_P, _P, _P, _I64, _I32, _F32, _I32, ctypes.POINTER(_I32), _P]),
        "omp_tuning": (_I32, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                              ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(st: int, where: str):
    if st != 0:
        raise OmpError(st, where)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _check_A(A, M, N):
    if A.dtype.is_floating_point is False or str(A.dtype) != "torch.float32":
        raise ValueError("A must be float32")
    if tuple(A.shape) != (M, N) or A.stride() != (1, M):
        raise ValueError(f"A must be an ({M}, {N}) column-major tensor (stride (1, {M}))")


def omp_desc_default(M: int, N: int) -> omp_desc:
    d = omp_desc()
    load().omp_desc_default(ctypes.byref(d), M, N)
    return d


class Handle:
    """An ``omp_handle`` plus the descriptor it was created with."""

    def __init__(self, ptr: ctypes.c_void_p, desc: omp_desc):
        self.ptr = ptr
        self.desc = desc

    @property
    def M(self):
        return self.desc.M

    @property
    def N(self):
        return self.desc.N

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.omp_destroy(self.ptr)
            self.ptr = None


def omp_create(M: int, N: int, max_batch: int = 4096, max_iters: int = 64,
               precision: str = "bf16", rescore_topk: int = 8, eps_relative: bool = True,
               use_graph: int = 1, device: int = 0, gather24: bool = False) -> Handle:
    lib = load()
    d = omp_desc()
    lib.omp_desc_default(ctypes.byref(d), M, N)
    d.max_batch, d.max_iters = max_batch, max_iters
    d.precision = PRECISIONS[precision]
    d.rescore_topk, d.eps_relative = rescore_topk, int(eps_relative)
    d.use_graph, d.device = int(use_graph), device
    d.gather24 = int(gather24)
    h = ctypes.c_void_p()
    _check(lib.omp_create(ctypes.byref(d), ctypes.byref(h)), "omp_create")
    return Handle(h, d)


def omp_destroy(h: Handle):
    if h.ptr:
        _check(load().omp_destroy(h.ptr), "omp_destroy")
        h.ptr = None


def omp_prepare_dictionary(h: Handle, A, stream=None):
    _check_A(A, h.M, h.N)
    _check(load().omp_prepare_dictionary(h.ptr, _ptr(A), _stream(stream)),
           "omp_prepare_dictionary")


def omp_solve_batch(h: Handle, A, Y, S: int, eps: float, X_out, support_out, stream=None):
    _check_A(A, h.M, h.N)
    B = Y.shape[0]
    _check(load().omp_solve_batch(h.ptr, _ptr(A), _ptr(Y), B, S, eps, _ptr(X_out),
                                  _ptr(support_out), _stream(stream)), "omp_solve_batch")


def omp_solve_batch_ex(h: Handle, A, Y, S: int, eps: float, X_out, support_out, n_iter_out=None,
                       resid_norm_out=None, stop_out=None, stream=None, margin_out=None):
    """Outputs as omp_solve_batch plus the optional diagnostics; margin_out (B, S) float32 asks
    for each step's top-two score margin (see include/omp_gb300.h)."""
    _check_A(A, h.M, h.N)
    B = Y.shape[0]
    _check(load().omp_solve_batch_ex(h.ptr, _ptr(A), _ptr(Y), B, S, eps, _ptr(X_out),
                                     _ptr(support_out), _ptr(n_iter_out), _ptr(resid_norm_out),
                                     _ptr(margin_out), _ptr(stop_out), _stream(stream)),
           "omp_solve_batch_ex")


def omp_solve_batch_gram(h: Handle, A, Y, S: int, eps: float, X_out, support_out, n_iter_out=None,
                         resid_norm_out=None, stop_out=None, stream=None):
    """Gram-space solve (no correlation GEMM per step); outputs as omp_solve_batch_ex."""
    _check_A(A, h.M, h.N)
    B = Y.shape[0]
    _check(load().omp_solve_batch_gram(h.ptr, _ptr(A), _ptr(Y), B, S, eps, _ptr(X_out),
                                       _ptr(support_out), _ptr(n_iter_out), _ptr(resid_norm_out),
                                       _ptr(stop_out), _stream(stream)), "omp_solve_batch_gram")


def omp_solve_batch_host(h: Handle, A, Y_host, S: int, eps: float, X_host, support_host,
                         stream=None):
    """Y_host, X_host, support_host: CPU tensors (pinned for asynchronous copies)."""
    _check_A(A, h.M, h.N)
    B = Y_host.shape[0]
    _check(load().omp_solve_batch_host(h.ptr, _ptr(A), _ptr(Y_host), B, S, eps, _ptr(X_host),
                                       _ptr(support_host), _stream(stream)),
           "omp_solve_batch_host")


def omp_correlate_topk(h: Handle, A, R, topk: int, idx_out, score_out, stream=None):
    _check_A(A, h.M, h.N)
    _check(load().omp_correlate_topk(h.ptr, _ptr(A), _ptr(R), R.shape[0], topk, _ptr(idx_out),
                                     _ptr(score_out), _stream(stream)), "omp_correlate_topk")


def omp_get_error(h: Handle, stream=None):
    """Returns (status, flags) and clears the device error word."""
    flags = _I32(0)
    st = load().omp_get_error(h.ptr, ctypes.byref(flags), _stream(stream))
    return st, flags.value


def omp_profile_enable(h: Handle, enable: bool = True):
    _check(load().omp_profile_enable(h.ptr, int(enable)), "omp_profile_enable")


def omp_profile_read(h: Handle, S: int, stream=None):
    """Per-iteration (correlation ms, update ms, live count) of the last profiled solve."""
    import numpy as np
    corr = np.zeros(S, dtype=np.float32)
    upd = np.zeros(S, dtype=np.float32)
    live = np.zeros(S, dtype=np.int32)
    _check(load().omp_profile_read(h.ptr, S, corr.ctypes.data_as(_P), upd.ctypes.data_as(_P),
                                   live.ctypes.data_as(_P), _stream(stream)), "omp_profile_read")
    return corr, upd, live


def omp_correlate_argmax_noalloc(A, R, idx_out, score_out, stream=None):
    """Allocation-free argmax of |<r_b, a_n>| / ||a_n|| for callers that cannot allocate device
    memory (see include/omp_gb300.h). A: (M, N) float32 column-major; R: (B, M) float32
    contiguous; idx_out: >= B int32; score_out: >= B float32, all on one CUDA device (checked
    here: ValueError before any call into C). Raises OmpError(OMP_ERR_INVALID_ARGUMENT) for
    B > NOALLOC_MAX_SIGNALS."""
    if A.dim() != 2 or R.dim() != 2:
        raise ValueError("A must be (M, N) and R (B, M)")
    M, N = A.shape
    _check_A(A, M, N)
    B = R.shape[0]
    if R.dtype.is_floating_point is False or str(R.dtype) != "torch.float32":
        raise ValueError("R must be float32")
    if R.shape[1] != M or not R.is_contiguous():
        raise ValueError(f"R must be a contiguous (B, {M}) tensor")
    for name, t, dt in (("idx_out", idx_out, "torch.int32"), ("score_out", score_out, "torch.float32")):
        if str(t.dtype) != dt or not t.is_contiguous() or t.numel() < B:
            raise ValueError(f"{name} must be a contiguous {dt[6:]} tensor with at least {B} elements")
    if len({str(t.device) for t in (A, R, idx_out, score_out)}) != 1 or not R.is_cuda:
        raise ValueError("A, R, idx_out and score_out must be on the same CUDA device")
    _check(load().omp_correlate_argmax_noalloc(_ptr(A), _ptr(R), M, N, R.shape[0], _ptr(idx_out),
                                               _ptr(score_out), _stream(stream)),
           "omp_correlate_argmax_noalloc")


def omp_status_string(status: int) -> str:
    return load().omp_status_string(status).decode()


def omp_score_error_bound(precision: int, Mp: int) -> float:
    """Bound per unit of ||a|| ||r|| on |quantised score - FP32 score| (host only, no GPU)."""
    return float(load().omp_score_error_bound(precision, Mp))


def omp_solve_batch_trace(h: Handle, A, Y, S: int, eps: float, X_out, support_out, drop_out,
                          stream=None):
    _check_A(A, h.M, h.N)
    _check(load().omp_solve_batch_trace(h.ptr, _ptr(A), _ptr(Y), Y.shape[0], S, eps, _ptr(X_out),
                                        _ptr(support_out), _ptr(drop_out), _stream(stream)),
           "omp_solve_batch_trace")


def omp_autotune(h: Handle, A, Y, S: int, eps: float = 0.0, repeats: int = 2, stream=None) -> int:
    """Pick the fastest append/update launch shape for this workload; returns warps per signal."""
    _check_A(A, h.M, h.N)
    c = _I32(0)
    _check(load().omp_autotune(h.ptr, _ptr(A), _ptr(Y), Y.shape[0], S, eps, repeats,
                               ctypes.byref(c), _stream(stream)), "omp_autotune")
    return c.value


def omp_tuning(h: Handle):
    """(update warps per signal, update persistent form, correlation stages, correlation CTAs,
    correlation CTAs per cluster)."""
    w, pe, st, g, cl = _I32(0), _I32(0), _I32(0), _I32(0), _I32(0)
    _check(load().omp_tuning(h.ptr, ctypes.byref(w), ctypes.byref(pe), ctypes.byref(st), ctypes.byref(g),
                             ctypes.byref(cl)), "omp_tuning")
    return w.value, pe.value, st.value, g.value, cl.value


def omp_handle_info(h: Handle):
    d = omp_desc()
    sms = _I32(0)
    _check(load().omp_handle_info(h.ptr, ctypes.byref(d), ctypes.byref(sms)), "omp_handle_info")
    return d, sms.value


def omp_loop_passes(h: Handle, stream=None) -> int:
    """Passes of the device-side iteration loop in the last graph solve (0 if it ran unrolled)."""
    v = _I32(0)
    _check(load().omp_loop_passes(h.ptr, ctypes.byref(v), _stream(stream)), "omp_loop_passes")
    return v.value


def read_bandwidth_gbs(mbytes: int = 64, reps: int = 50, blocks: int = 0, stream=None) -> float:
    """Streaming L2-only read bandwidth over a device buffer of `mbytes` MiB (best of three runs
    of `reps` passes, CUDA events); a measurement helper for the benchmark's L2 roofline."""
    import torch
    n = mbytes * 1024 * 1024 // 4
    buf = torch.randn(n, device="cuda")
    if blocks <= 0:
        blocks = 4 * torch.cuda.get_device_properties(buf.device).multi_processor_count
    out = torch.empty(blocks, device=buf.device)
    lib = load()
    st = _stream(stream)
    _check(lib.omp_read_bandwidth_probe(_ptr(buf), n * 4, 2, _ptr(out), blocks, st), "probe")
    best = float("inf")
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _check(lib.omp_read_bandwidth_probe(_ptr(buf), n * 4, reps, _ptr(out), blocks, st), "probe")
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return reps * n * 4 / (best / 1e3) / 1e9


def omp_synthesize_signals(A, sup, coef, noise, Y_out, stream=None):
    """Y_out = A[:, sup] coef + noise per row, on the device (A column-major (M, N))."""
    M, N = A.shape
    _check(load().omp_synthesize_signals(_ptr(A), M, N, _ptr(sup), _ptr(coef), _ptr(noise),
                                         sup.shape[0], sup.shape[1], _ptr(Y_out), _stream(stream)),
           "omp_synthesize_signals")


def omp_topk_rows(logits, K: int, idx_out, stream=None):
    _check(load().omp_topk_rows(_ptr(logits), logits.shape[0], logits.shape[1], K, _ptr(idx_out),
                                _stream(stream)), "omp_topk_rows")


class Proposal:
    """An ``omp_proposal`` (learned candidate proposal) bound to a handle."""

    def __init__(self, h: Handle, hidden=1024, topk=256, max_batch=None, train_batch=4096,
                 lr=1e-3, beta1=0.9, beta2=0.999, weight_decay=0.0, adam_eps=1e-8,
                 pos_weight=1.0):
        lib = load()
        d = omp_proposal_desc()
        lib.omp_proposal_desc_default(ctypes.byref(d))
        d.hidden, d.topk = hidden, topk
        d.max_batch = max_batch if max_batch is not None else int(h.desc.max_batch)
        d.train_batch = train_batch
        d.lr, d.beta1, d.beta2, d.weight_decay, d.adam_eps = lr, beta1, beta2, weight_decay, adam_eps
        d.pos_weight = pos_weight
        ptr = ctypes.c_void_p()
        _check(lib.omp_proposal_create(h.ptr, ctypes.byref(d), ctypes.byref(ptr)),
               "omp_proposal_create")
        self.ptr, self.desc, self.h = ptr, d, h

    def close(self):
        if self.ptr:
            load().omp_proposal_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.omp_proposal_destroy(self.ptr)
            self.ptr = None

    def set_weights(self, W1, b1, W2, b2, beta, stream=None):
        _check(load().omp_proposal_set_weights(self.ptr, _ptr(W1), _ptr(b1), _ptr(W2), _ptr(b2),
                                               _ptr(beta), _stream(stream)),
               "omp_proposal_set_weights")

    def get_weights(self, W1, b1, W2, b2, beta, stream=None):
        _check(load().omp_proposal_get_weights(self.ptr, _ptr(W1), _ptr(b1), _ptr(W2), _ptr(b2),
                                               _ptr(beta), _stream(stream)),
               "omp_proposal_get_weights")

    def train_step(self, A, Y, labels, loss_out=None, stream=None):
        _check(load().omp_proposal_train_step(self.ptr, _ptr(A), _ptr(Y), _ptr(labels), Y.shape[0],
                                              labels.shape[1], _ptr(loss_out), _stream(stream)),
               "omp_proposal_train_step")

    def gradients(self, A, Y, labels, dW1=None, db1=None, dW2=None, db2=None, dbeta=None,
                  loss_out=None, stream=None):
        _check(load().omp_proposal_gradients(self.ptr, _ptr(A), _ptr(Y), _ptr(labels), Y.shape[0],
                                             labels.shape[1], _ptr(dW1), _ptr(db1), _ptr(dW2),
                                             _ptr(db2), _ptr(dbeta), _ptr(loss_out),
                                             _stream(stream)), "omp_proposal_gradients")

    def infer(self, A, Y, cand_out, logits_out=None, stream=None):
        _check(load().omp_proposal_infer(self.ptr, _ptr(A), _ptr(Y), Y.shape[0], _ptr(cand_out),
                                         _ptr(logits_out), _stream(stream)), "omp_proposal_infer")

    def baseline_candidates(self, A, Y, cand_out, stream=None):
        _check(load().omp_proposal_baseline_candidates(self.ptr, _ptr(A), _ptr(Y), Y.shape[0],
                                                       _ptr(cand_out), _stream(stream)),
               "omp_proposal_baseline_candidates")

    def set_thresholds(self, tau):
        import numpy as np
        t = np.ascontiguousarray(tau, dtype=np.float32)
        _check(load().omp_proposal_set_thresholds(self.ptr, t.ctypes.data_as(_P), t.size),
               "omp_proposal_set_thresholds")

    def get_thresholds(self, S):
        import numpy as np
        t = np.zeros(S, dtype=np.float32)
        _check(load().omp_proposal_get_thresholds(self.ptr, t.ctypes.data_as(_P), S),
               "omp_proposal_get_thresholds")
        return t

    def save(self, path: str):
        """Write the weights and thresholds to `path` (omp_proposal_save)."""
        _check(load().omp_proposal_save(self.ptr, os.fsencode(path)), "omp_proposal_save")

    def load(self, path: str):
        """Read weights and thresholds saved by save() for the same N and hidden width."""
        _check(load().omp_proposal_load(self.ptr, os.fsencode(path)), "omp_proposal_load")

    def calibrate(self, drops, quantile=1e-3, stream=None):
        _check(load().omp_proposal_calibrate(self.ptr, _ptr(drops), drops.shape[0], drops.shape[1],
                                             quantile, _stream(stream)), "omp_proposal_calibrate")


def omp_solve_batch_candidates(h: Handle, A, Y, S, eps, cand, tau, X_out, support_out,
                               n_iter_out=None, resid_norm_out=None, fallback_out=None,
                               stream=None):
    _check_A(A, h.M, h.N)
    _check(load().omp_solve_batch_candidates(h.ptr, _ptr(A), _ptr(Y), Y.shape[0], S, eps,
                                             _ptr(cand), cand.shape[1], _ptr(tau), _ptr(X_out),
                                             _ptr(support_out), _ptr(n_iter_out),
                                             _ptr(resid_norm_out), _ptr(fallback_out),
                                             _stream(stream)), "omp_solve_batch_candidates")


def omp_solve_batch_learned(h: Handle, p: Proposal, A, Y, S, eps, X_out, support_out,
                            n_iter_out=None, resid_norm_out=None, fallback_out=None, stream=None):
    _check_A(A, h.M, h.N)
    _check(load().omp_solve_batch_learned(h.ptr, p.ptr, _ptr(A), _ptr(Y), Y.shape[0], S, eps,
                                          _ptr(X_out), _ptr(support_out), _ptr(n_iter_out),
                                          _ptr(resid_norm_out), _ptr(fallback_out),
                                          _stream(stream)), "omp_solve_batch_learned")


class OmpSolver:
    """Convenience wrapper: owns a handle and allocates the outputs of each solve."""

    def __init__(self, M, N, max_batch=4096, max_iters=64, precision="bf16", **kw):
        self.h = omp_create(M, N, max_batch, max_iters, precision, **kw)

    def solve_gram(self, A, Y, S, eps=0.0, stream=None, diagnostics=False):
        """The Gram-space solve of the same batch (see omp_solve_batch_gram)."""
        import torch
        B = Y.shape[0]
        X = torch.empty((B, S), dtype=torch.float32, device=Y.device)
        sup = torch.empty((B, S), dtype=torch.int32, device=Y.device)
        n_iter = torch.empty(B, dtype=torch.int32, device=Y.device)
        resid = torch.empty(B, dtype=torch.float32, device=Y.device)
        stop = torch.empty(B, dtype=torch.int32, device=Y.device)
        omp_solve_batch_gram(self.h, A, Y, S, eps, X, sup, n_iter, resid, stop, stream)
        return (X, sup, n_iter, resid, stop) if diagnostics else (X, sup)

    def solve(self, A, Y, S, eps=0.0, stream=None, diagnostics=False, margins=False):
        """(X, support), or with diagnostics (X, support, n_iter, resid_norm, stop), plus the
        (B, S) per-step margins last when margins=True."""
        import torch
        B = Y.shape[0]
        X = torch.empty((B, S), dtype=torch.float32, device=Y.device)
        sup = torch.empty((B, S), dtype=torch.int32, device=Y.device)
        if not diagnostics and not margins:
            omp_solve_batch(self.h, A, Y, S, eps, X, sup, stream)
            return X, sup
        n_iter = torch.empty(B, dtype=torch.int32, device=Y.device)
        resid = torch.empty(B, dtype=torch.float32, device=Y.device)
        stop = torch.empty(B, dtype=torch.int32, device=Y.device)
        margin = torch.empty((B, S), dtype=torch.float32, device=Y.device) if margins else None
        omp_solve_batch_ex(self.h, A, Y, S, eps, X, sup, n_iter, resid, stop, stream,
                           margin_out=margin)
        out = (X, sup, n_iter, resid, stop) if diagnostics else (X, sup)
        return out + (margin,) if margins else out

    def close(self):
        omp_destroy(self.h)
