"""ctypes binding of include/nk_tune.h (schedule search and the cost-model
kernels): argument marshalling only; the work runs in libnk's kernels."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import nk
from .nk import _I32, _I64, _P, _SZ, _check, _stream, nk_schedule

NK_OP_MATMUL, NK_OP_CONV2D = 0, 1
NK_TUNE_EXHAUSTIVE, NK_TUNE_MODEL_TOPK, NK_TUNE_EVOLUTION = 0, 1, 2
NK_TUNE_FEATURES = 16


class nk_problem(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("op", "precision", "M", "N", "K", "n", "h", "w", "c", "f", "kh", "kw", "stride", "pad")]


class nk_tune_report(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_int32), ("timed", ctypes.c_int32), ("best_ms", ctypes.c_float),
                ("default_ms", ctypes.c_float)]


_PP = ctypes.POINTER(nk_problem)
_PS = ctypes.POINTER(nk_schedule)

SIGNATURES = {
    "nk_enumerate_schedules": (_I32, [_PP, _PS, _I32, ctypes.POINTER(_I32)]),
    "nk_default_schedule": (_I32, [_PP, _PS]),
    "nk_conv_window_tile": (_I32, [_I32] * 9 + [ctypes.POINTER(_I32), _PS, ctypes.POINTER(_I32)]),
    "nk_workspace_size": (_I32, [_PP, _PS, ctypes.POINTER(_SZ)]),
    "nk_schedule_features": (_I32, [_PP, _PS, _I32, ctypes.POINTER(ctypes.c_float)]),
    "nk_time_schedule": (_I32, [_PP, _PS, _I32, ctypes.POINTER(ctypes.c_float), _P]),
    "nk_tune_release": (_I32, []),
    "nk_tune": (_I32, [_PP, _I32, _I32, _P, _I32, _PS, ctypes.POINTER(nk_tune_report), _P]),
    "nk_grouped_tune": (_I32, [_I32, _P, _I32, _I32, _PS, ctypes.POINTER(nk_tune_report), _P]),
    "nk_conv2d_grouped_tune": (_I32, [_I32, _P, _I32, _PS, ctypes.POINTER(nk_tune_report), _P]),
    "nk_mlp_param_count": (_SZ, []),
    "nk_mlp_forward": (_I32, [_P, _P, _I64, _P, _P]),
    "nk_mlp_workspace_size": (_SZ, [_I64]),
    "nk_mlp_grad": (_I32, [_P, _P, _P, _I64, _P, _P, _P, _SZ, _P]),
    "nk_mlp_adam": (_I32, [_P, _P, _P, _P, _I32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                           ctypes.c_float, _P]),
}

_done = False


def lib():
    global _done
    L = nk.lib()
    if not _done:
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _done = True
    return L


def timing_method() -> str:
    """How nk_time_schedule / nk_tune time a schedule (tune.cu)."""
    return ("device time of CUDA-graph replays of back-to-back calls behind a hold kernel, median of reps; "
            "the calls rotate over as many copies of operands, outputs and workspace as hold twice the L2 "
            "(at most 128), so each call starts with its operands out of L2")


def matmul_problem(M, N, K, precision="bf16") -> nk_problem:
    return nk_problem(NK_OP_MATMUL, nk.PREC[precision], M, N, K, 0, 0, 0, 0, 0, 0, 0, 0, 0)


def conv_problem(n, h, w, c, f, kh, kw, stride, pad, precision="bf16") -> nk_problem:
    return nk_problem(NK_OP_CONV2D, nk.PREC[precision], 0, 0, 0, n, h, w, c, f, kh, kw, stride, pad)


def nk_enumerate_schedules(p: nk_problem):
    cnt = ctypes.c_int32(0)
    _check(lib().nk_enumerate_schedules(ctypes.byref(p), None, 0, ctypes.byref(cnt)))
    arr = (nk_schedule * max(cnt.value, 1))()
    _check(lib().nk_enumerate_schedules(ctypes.byref(p), arr, cnt.value, ctypes.byref(cnt)))
    return [arr[i].as_tuple() for i in range(cnt.value)]


def nk_default_schedule(p: nk_problem):
    s = nk_schedule()
    _check(lib().nk_default_schedule(ctypes.byref(p), ctypes.byref(s)))
    return s.as_tuple()


WINDOW_TILE_FIELDS = ("P", "Q", "R", "NB", "WR", "rows", "slot_rows", "stk", "tiles", "chains")


def nk_conv_window_tile(n, h, w, c, f, kh, kw, dilation=(1, 1), pad=(0, 0, 0, 0), schedule=None) -> dict:
    """Host-side geometry of the tile a window schedule launches (no GPU)."""
    pd = (_I32 * 4)(*pad)
    out = (_I32 * 10)()
    _check(lib().nk_conv_window_tile(n, h, w, c, f, kh, kw, dilation[0], dilation[1], pd,
                                     ctypes.byref(nk_schedule(*schedule)), out))
    return dict(zip(WINDOW_TILE_FIELDS, list(out)))


def nk_workspace_size(p: nk_problem, schedule=None) -> int:
    n = ctypes.c_size_t(0)
    s = ctypes.byref(nk_schedule(*schedule)) if schedule is not None else None
    _check(lib().nk_workspace_size(ctypes.byref(p), s, ctypes.byref(n)))
    return n.value


def nk_schedule_features(p: nk_problem, schedules) -> np.ndarray:
    n = len(schedules)
    arr = (nk_schedule * max(n, 1))(*[nk_schedule(*s) for s in schedules])
    out = np.zeros((n, NK_TUNE_FEATURES), np.float32)
    _check(lib().nk_schedule_features(ctypes.byref(p), arr, n,
                                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return out


def nk_time_schedule(p: nk_problem, schedule, reps=5, stream=None) -> float:
    ms = ctypes.c_float(0)
    s = nk_schedule(*schedule)
    _check(lib().nk_time_schedule(ctypes.byref(p), ctypes.byref(s), int(reps), ctypes.byref(ms), _stream(stream)))
    return ms.value


def nk_tune_release():
    _check(lib().nk_tune_release())


def nk_tune(p: nk_problem, mode=NK_TUNE_EXHAUSTIVE, topk=5, params: torch.Tensor | None = None, reps=5,
            stream=None):
    best = nk_schedule()
    rep = nk_tune_report()
    _check(lib().nk_tune(ctypes.byref(p), mode, topk, params.data_ptr() if params is not None else None, reps,
                         ctypes.byref(best), ctypes.byref(rep), _stream(stream)))
    return best.as_tuple(), rep


def nk_grouped_tune(groups, G, precision="bf16", reps=3, stream=None):
    """Fastest grouped-plan schedule for these groups (from nk.make_groups);
    overwrites every group's C while timing."""
    best = nk_schedule()
    rep = nk_tune_report()
    _check(lib().nk_grouped_tune(G, ctypes.cast(groups, ctypes.c_void_p), nk.PREC[precision], reps,
                                 ctypes.byref(best), ctypes.byref(rep), _stream(stream)))
    return best.as_tuple(), rep


def nk_conv2d_grouped_tune(groups, G, reps=3, stream=None):
    """Fastest grouped-conv plan schedule for these groups (from
    nk.make_conv_groups); overwrites every group's O while timing."""
    best = nk_schedule()
    rep = nk_tune_report()
    _check(lib().nk_conv2d_grouped_tune(G, ctypes.cast(groups, ctypes.c_void_p), reps, ctypes.byref(best),
                                        ctypes.byref(rep), _stream(stream)))
    return best.as_tuple(), rep


def nk_mlp_param_count() -> int:
    return lib().nk_mlp_param_count()


def nk_mlp_forward(params: torch.Tensor, X: torch.Tensor, y: torch.Tensor | None = None, stream=None):
    B = X.shape[0]
    if y is None:
        y = torch.empty(B, device=X.device)
    _check(lib().nk_mlp_forward(params.data_ptr(), X.data_ptr(), B, y.data_ptr(), _stream(stream)))
    return y


def nk_mlp_workspace_size(B: int) -> int:
    return lib().nk_mlp_workspace_size(B)


def nk_mlp_grad(params, X, t, grad, loss=None, ws=None, stream=None):
    B = X.shape[0]
    if ws is None:
        ws = torch.empty(nk_mlp_workspace_size(B), dtype=torch.uint8, device=X.device)
    _check(lib().nk_mlp_grad(params.data_ptr(), X.data_ptr(), t.data_ptr(), B, grad.data_ptr(),
                             loss.data_ptr() if loss is not None else None, ws.data_ptr(), ws.numel(),
                             _stream(stream)))
    return grad


def nk_mlp_adam(params, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().nk_mlp_adam(params.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), int(step), lr,
                             beta1, beta2, eps, _stream(stream)))
