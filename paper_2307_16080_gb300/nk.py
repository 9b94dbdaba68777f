"""Thin Python binding of libnk (ctypes): argument marshalling only.

Every function here forwards to the C entry point of the same name declared
in include/nk.h; all arithmetic runs in the library's CUDA kernels.  PyTorch
tensors serve as device memory and torch's current stream as the stream.
Importing this module loads libnk.so and raises if it is missing: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnk.so")

NK_OK = 0
STATUS = {0: "NK_OK", -1: "NK_ERR_INVALID_ARG", -2: "NK_ERR_UNSUPPORTED", -3: "NK_ERR_MISALIGNED",
          -4: "NK_ERR_WORKSPACE", -5: "NK_ERR_CUDA", -6: "NK_ERR_TIMEOUT", -7: "NK_ERR_NO_SCHEDULE"}
NK_F32, NK_BF16, NK_F8E4M3, NK_F64 = 0, 1, 2, 3
PREC = {"f32": 0, "bf16": 1, "bf16x3": 2, "fp8": 3}


class NkError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class nk_tensor(ctypes.Structure):
    _fields_ = [("ptr", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("rank", ctypes.c_int32),
                ("shape", ctypes.c_int64 * 4), ("stride", ctypes.c_int64 * 4)]


NK_EW_MAX = 4
EW_OPS = {"mul": 1, "add": 2, "affine": 3, "relu": 4, "gelu": 5, "gelu_tanh": 6, "silu": 7, "sigmoid": 8,
          "tanh": 9, "clamp": 10}


class nk_ew_op(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("a", ctypes.c_float), ("b", ctypes.c_float), ("t", nk_tensor)]


class nk_ew_program(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("ops", nk_ew_op * NK_EW_MAX)]


class nk_epilogue(ctypes.Structure):
    _fields_ = [("bias", ctypes.c_void_p), ("relu", ctypes.c_int32), ("accumulate", ctypes.c_int32),
                ("scale_a", ctypes.c_float), ("scale_b", ctypes.c_float), ("ew", ctypes.c_void_p),
                ("pro_a", ctypes.c_void_p), ("pro_b", ctypes.c_void_p)]


class nk_schedule(ctypes.Structure):
    _fields_ = [("tile_m", ctypes.c_int32), ("tile_n", ctypes.c_int32), ("tile_k", ctypes.c_int32),
                ("cluster", ctypes.c_int32), ("stages", ctypes.c_int32), ("split_k", ctypes.c_int32)]

    def as_tuple(self):
        return (self.tile_m, self.tile_n, self.tile_k, self.cluster, self.stages, self.split_k)


class nk_gemm_group(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int32), ("N", ctypes.c_int32), ("K", ctypes.c_int32),
                ("accumulate", ctypes.c_int32), ("A", ctypes.c_void_p), ("Bt", ctypes.c_void_p),
                ("C", ctypes.c_void_p), ("lda", ctypes.c_int64), ("ldb", ctypes.c_int64),
                ("ldc", ctypes.c_int64)]


_P = ctypes.c_void_p
_I32, _I64, _SZ = ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
class nk_conv_group(ctypes.Structure):
    _fields_ = [("I", nk_tensor), ("W", nk_tensor), ("O", nk_tensor), ("stride", ctypes.c_int64 * 2),
                ("dilation", ctypes.c_int64 * 2), ("pad", ctypes.c_int64 * 4), ("bias", ctypes.c_void_p),
                ("relu", ctypes.c_int32), ("accumulate", ctypes.c_int32)]


_PT = ctypes.POINTER(nk_tensor)
_PE = ctypes.POINTER(nk_epilogue)
_PS = ctypes.POINTER(nk_schedule)

# name -> (restype, argtypes); mirrors include/nk.h
SIGNATURES = {
    "nk_matmul": (_I32, [_PT, _PT, _PT, _I32, _PE, _PS, _P, _SZ, _P]),
    "nk_matmul_workspace_size": (_I32, [_PT, _PT, _PT, _I32, _PS, ctypes.POINTER(_SZ)]),
    "nk_grouped_plan_create": (_I32, [_I32, ctypes.POINTER(nk_gemm_group), _I32, _PS, ctypes.POINTER(_P)]),
    "nk_conv2d_grouped_plan_create": (_I32, [_I32, ctypes.POINTER(nk_conv_group), _PS, ctypes.POINTER(_P)]),
    "nk_grouped_plan_run": (_I32, [_P, _P]),
    "nk_grouped_plan_destroy": (_I32, [_P]),
    "nk_batch_matmul_grouped": (_I32, [_I32, ctypes.POINTER(nk_gemm_group), _I32, _PS, _P, _SZ, _P]),
    "nk_grouped_workspace_size": (_I32, [_I32, ctypes.POINTER(nk_gemm_group), _I32, _PS, ctypes.POINTER(_SZ)]),
    "nk_conv2d_nhwc_hwcf": (_I32, [_PT, _PT, _PT, ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                   ctypes.POINTER(_I64), _I32, _PE, _PS, _P, _SZ, _P]),
    "nk_conv2d_workspace_size": (_I32, [_PT, _PT, _PT, ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                        ctypes.POINTER(_I64), _I32, _PS, ctypes.POINTER(_SZ)]),
    "nk_conv2d_pack_weights": (_I32, [_PT, _P, _I64, _P]),
    "nk_conv2d_pack_weights_fp8": (_I32, [_PT, _P, _I64, _P, _P, _SZ, _P]),
    "nk_conv2d_pack_weights_fp8_workspace_size": (_SZ, []),
    "nk_conv2d_nchw_fchw": (_I32, [_PT, _PT, _PT, ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                   ctypes.POINTER(_I64), _PE, _P]),
    "nk_amax": (_I32, [_P, _I64, _P, _P, _SZ, _P]),
    "nk_prep_workspace_size": (_SZ, [_I64]),
    "nk_cast_bf16": (_I32, [_P, _I64, _I64, _I64, _P, _I64, _I32, _P]),
    "nk_cast_fp8": (_I32, [_P, _I64, _I64, _I64, _P, _P, _I64, _I32, _P, _P]),
    "nk_split_bf16x3": (_I32, [_P, _I64, _I64, _I64, _P, _P, _I64, _I32, _P]),
    "nk_rel_frobenius": (_I32, [_P, _I64, _P, _I64, _I64, _I64, _P, _P, _SZ, _P]),
    "nk_norm_workspace_size": (_SZ, [_I64, _I64]),
    "nk_matmul_f32_splitk_noalloc": (_I32, [_P, _I64, _P, _I64, _P, _I64, _I32, _I32, _I32, _I32, _P]),
    "nk_last_error": (ctypes.c_char_p, []),
    "nk_sync_status": (_I32, [_P]),
    "nk_set_wait_budget": (_I32, [_I64]),
    "nk_set_pdl": (_I32, [_I32]),
    "nk_get_pdl": (_I32, []),
    "nk_device_info": (_I32, [ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "nk_elementwise": (_I32, [_PT, _PT, ctypes.POINTER(nk_ew_program), _P]),
}

_lib = None


def lib():
    """Load libnk.so (built by __graft_entry__.build()); raise if it is absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libnk.so not built at {LIB_PATH}: run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            if hasattr(L, name):
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    return lib().nk_last_error().decode()


def _check(status: int):
    if status != NK_OK:
        raise NkError(status, last_error())


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


_DT = {torch.float32: NK_F32, torch.bfloat16: NK_BF16, torch.float8_e4m3fn: NK_F8E4M3,
       torch.uint8: NK_F8E4M3, torch.float64: NK_F64}


def as_nk_tensor(t: torch.Tensor) -> nk_tensor:
    if t.dim() > 4:
        raise ValueError("rank > 4")
    d = nk_tensor()
    d.ptr = t.data_ptr() if t.numel() else None
    d.dtype = _DT[t.dtype]
    d.rank = t.dim()
    for i in range(t.dim()):
        d.shape[i] = t.shape[i]
        d.stride[i] = t.stride(i)
    return d


def _sched(schedule):
    if schedule is None:
        return None
    if isinstance(schedule, nk_schedule):
        return ctypes.byref(schedule)
    return ctypes.byref(nk_schedule(*schedule))


def make_ew_program(spec) -> nk_ew_program | None:
    """An nk_ew_program from a list of steps, each a tuple: ("mul", T),
    ("add", T), ("affine", a, b), ("clamp", lo, hi) or (name,) for "relu",
    "gelu", "gelu_tanh", "silu", "sigmoid", "tanh".  T: an FP32 CUDA tensor
    with the shape and strides of the tensor the program runs over.  The
    caller keeps the T tensors alive until the call's kernels have run."""
    if spec is None:
        return None
    prog = nk_ew_program()
    spec = list(spec)
    prog.n = len(spec)   # above NK_EW_MAX the library rejects the count
    for i, step in enumerate(spec[:NK_EW_MAX]):
        name, *args = step
        op = prog.ops[i]
        op.op = EW_OPS.get(name, -1) if isinstance(name, str) else int(name)
        if name in ("mul", "add"):
            op.t = as_nk_tensor(args[0])
        elif name in ("affine", "clamp"):
            op.a, op.b = float(args[0]), float(args[1])
    return prog


def _epi(bias, relu, accumulate, scale_a, scale_b, ew=None, pro_a=None, pro_b=None):
    """The epilogue struct plus the program structs it points to (returned so
    that they outlive the call)."""
    e = nk_epilogue()
    e.bias = bias.data_ptr() if bias is not None else None
    e.relu = int(bool(relu))
    e.accumulate = int(bool(accumulate))
    e.scale_a = float(scale_a)
    e.scale_b = float(scale_b)
    keep = []
    for field, spec in (("ew", ew), ("pro_a", pro_a), ("pro_b", pro_b)):
        prog = make_ew_program(spec)
        if prog is not None:
            keep.append(prog)
            setattr(e, field, ctypes.addressof(prog))
    e._keep = keep
    return e


def nk_matmul_workspace_size(A, B, C, precision="f32", schedule=None) -> int:
    n = ctypes.c_size_t(0)
    ta, tb, tc = as_nk_tensor(A), as_nk_tensor(B), as_nk_tensor(C)
    _check(lib().nk_matmul_workspace_size(ctypes.byref(ta), ctypes.byref(tb), ctypes.byref(tc),
                                          PREC[precision], _sched(schedule), ctypes.byref(n)))
    return n.value


def workspace(nbytes: int, device=None) -> torch.Tensor | None:
    if nbytes == 0:
        return None
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


def nk_matmul(A, B, C, precision="f32", bias=None, relu=False, accumulate=False, scale_a=1.0,
              scale_b=1.0, schedule=None, ws=None, stream=None, ew=None, pro_a=None, pro_b=None):
    """C = ew(ReLU?(accumulate*C + alpha*(pro_a(A) @ pro_b(B)) + bias)) through
    nk_matmul; ew / pro_a / pro_b are program step lists (make_ew_program)."""
    ta, tb, tc = as_nk_tensor(A), as_nk_tensor(B), as_nk_tensor(C)
    if ws is None:
        ws = workspace(nk_matmul_workspace_size(A, B, C, precision, schedule), C.device)
    e = _epi(bias, relu, accumulate, scale_a, scale_b, ew, pro_a, pro_b)
    _check(lib().nk_matmul(ctypes.byref(ta), ctypes.byref(tb), ctypes.byref(tc), PREC[precision],
                           ctypes.byref(e), _sched(schedule), ws.data_ptr() if ws is not None else None,
                           ws.numel() if ws is not None else 0, _stream(stream)))
    return C


def _conv_args(stride, dilation, pad):
    st = (ctypes.c_int64 * 2)(*stride)
    dl = (ctypes.c_int64 * 2)(*dilation)
    pd = (ctypes.c_int64 * 4)(*pad)
    return st, dl, pd


def nk_conv2d_workspace_size(I, W, O, stride=(1, 1), dilation=(1, 1), pad=(0, 0, 0, 0),
                             precision="f32", schedule=None) -> int:
    n = ctypes.c_size_t(0)
    ti, tw, to = as_nk_tensor(I), as_nk_tensor(W), as_nk_tensor(O)
    st, dl, pd = _conv_args(stride, dilation, pad)
    _check(lib().nk_conv2d_workspace_size(ctypes.byref(ti), ctypes.byref(tw), ctypes.byref(to), st, dl, pd,
                                          PREC[precision], _sched(schedule), ctypes.byref(n)))
    return n.value


def nk_conv2d_nhwc_hwcf(I, W, O, stride=(1, 1), dilation=(1, 1), pad=(0, 0, 0, 0), precision="f32",
                        bias=None, relu=False, accumulate=False, schedule=None, ws=None, stream=None,
                        ew=None, pro_i=None, pro_w=None, scale_i=1.0, scale_w=1.0):
    """O = ew(ReLU?(accumulate*O + conv(pro_i(I), pro_w(W)) + bias)); the
    programs are step lists (make_ew_program), the zero padding stays 0.
    scale_i, scale_w: the quantisation scales of E4M3 operands the caller
    quantised (read only for those)."""
    ti, tw, to = as_nk_tensor(I), as_nk_tensor(W), as_nk_tensor(O)
    st, dl, pd = _conv_args(stride, dilation, pad)
    if ws is None:
        ws = workspace(nk_conv2d_workspace_size(I, W, O, stride, dilation, pad, precision, schedule), O.device)
    e = _epi(bias, relu, accumulate, scale_i, scale_w, ew, pro_i, pro_w)
    _check(lib().nk_conv2d_nhwc_hwcf(ctypes.byref(ti), ctypes.byref(tw), ctypes.byref(to), st, dl, pd,
                                     PREC[precision], ctypes.byref(e), _sched(schedule),
                                     ws.data_ptr() if ws is not None else None,
                                     ws.numel() if ws is not None else 0, _stream(stream)))
    return O


def nk_conv2d_pack_weights(W, ldw=None, stream=None) -> torch.Tensor:
    """FP32 HWCF W [KH,KW,C,F] -> the BF16 packed layout, returned as a
    [KH,KW,C,F] strided view (strides {KW*ldw, ldw, 1, KH*KW*ldw}) that
    nk_conv2d_nhwc_hwcf takes as W without a per-call cast."""
    KH, KW, C, F = W.shape
    ldw = (C + 7) // 8 * 8 if ldw is None else int(ldw)
    buf = torch.empty(F * KH * KW * ldw, dtype=torch.bfloat16, device=W.device)
    tw = as_nk_tensor(W)
    _check(lib().nk_conv2d_pack_weights(ctypes.byref(tw), buf.data_ptr(), ldw, _stream(stream)))
    return buf.as_strided((KH, KW, C, F), (KW * ldw, ldw, 1, KH * KW * ldw))


def nk_conv2d_pack_weights_fp8(W, ldw=None, stream=None):
    """FP32 HWCF W [KH,KW,C,F] -> (E4M3 packed weights as a [KH,KW,C,F]
    strided uint8 view, the device scale s_w as a 1-element FP32 tensor)."""
    KH, KW, C, F = W.shape
    ldw = (C + 15) // 16 * 16 if ldw is None else int(ldw)
    buf = torch.empty(F * KH * KW * ldw, dtype=torch.uint8, device=W.device)
    scale = torch.empty(1, device=W.device)
    ws = workspace(lib().nk_conv2d_pack_weights_fp8_workspace_size(), W.device)
    tw = as_nk_tensor(W)
    _check(lib().nk_conv2d_pack_weights_fp8(ctypes.byref(tw), buf.data_ptr(), ldw, scale.data_ptr(), ws.data_ptr(),
                                            ws.numel(), _stream(stream)))
    return buf.as_strided((KH, KW, C, F), (KW * ldw, ldw, 1, KH * KW * ldw)), scale


def quantize_nhwc_fp8(I, stream=None):
    """FP32 NHWC I [N,H,W,C] -> (E4M3 [N,H,W,C] uint8 view with channel
    rows padded to 16 bytes, the device scale s_i = 448/amax(|I|)): nk_amax,
    then nk_cast_fp8 of the [N*H*W, C] view."""
    N, H, Wd, C = I.shape
    cp = (C + 15) // 16 * 16
    buf = torch.zeros(N * H * Wd * cp, dtype=torch.uint8, device=I.device)
    amax = torch.empty(1, device=I.device)
    scale = torch.empty(1, device=I.device)
    flat = I.reshape(N * H * Wd, C)
    nk_amax(flat, amax, stream=stream)
    nk_cast_fp8(flat, amax, buf.view(N * H * Wd, cp), scale_out=scale, stream=stream)
    return buf.as_strided((N, H, Wd, C), (H * Wd * cp, Wd * cp, cp, 1)), scale


def nk_conv2d_nchw_fchw(I, K, O, stride=(1, 1), dilation=(1, 1), pad=(0, 0, 0, 0), bias=None, relu=False,
                        accumulate=False, stream=None, ew=None):
    """Direct NCHW / FCHW convolution (Listing "2dnchwconv" layout)."""
    ti, tk, to = as_nk_tensor(I), as_nk_tensor(K), as_nk_tensor(O)
    st, dl, pd = _conv_args(stride, dilation, pad)
    e = _epi(bias, relu, accumulate, 1.0, 1.0, ew)
    _check(lib().nk_conv2d_nchw_fchw(ctypes.byref(ti), ctypes.byref(tk), ctypes.byref(to), st, dl, pd,
                                     ctypes.byref(e), _stream(stream)))
    return O


def nk_elementwise(X, Y, prog, stream=None):
    """Y = prog(X) elementwise (the GPUModule kernel of Sec. 3.1 as one pass)."""
    tx, ty = as_nk_tensor(X), as_nk_tensor(Y)
    p = make_ew_program(prog)
    _check(lib().nk_elementwise(ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(p) if p is not None else None,
                                _stream(stream)))
    return Y


def nk_amax(x: torch.Tensor, out: torch.Tensor, ws=None, stream=None):
    n = x.numel()
    if ws is None:
        ws = workspace(lib().nk_prep_workspace_size(n), x.device)
    _check(lib().nk_amax(x.data_ptr(), n, out.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream)))
    return out


def nk_cast_bf16(x: torch.Tensor, out: torch.Tensor, transpose=False, stream=None):
    rows, cols = x.shape
    _check(lib().nk_cast_bf16(x.data_ptr(), rows, cols, x.stride(0), out.data_ptr(), out.stride(0),
                              int(transpose), _stream(stream)))
    return out


def nk_cast_fp8(x: torch.Tensor, amax: torch.Tensor, out: torch.Tensor, transpose=False, scale_out=None,
                stream=None):
    rows, cols = x.shape
    _check(lib().nk_cast_fp8(x.data_ptr(), rows, cols, x.stride(0), amax.data_ptr(), out.data_ptr(),
                             out.stride(0), int(transpose),
                             scale_out.data_ptr() if scale_out is not None else None, _stream(stream)))
    return out


def nk_split_bf16x3(x: torch.Tensor, hi: torch.Tensor, lo: torch.Tensor, transpose=False, stream=None):
    rows, cols = x.shape
    _check(lib().nk_split_bf16x3(x.data_ptr(), rows, cols, x.stride(0), hi.data_ptr(), lo.data_ptr(),
                                 hi.stride(0), int(transpose), _stream(stream)))
    return hi, lo


def nk_rel_frobenius(C: torch.Tensor, R: torch.Tensor, out: torch.Tensor | None = None, ws=None,
                     stream=None) -> torch.Tensor:
    """Device FP64 sums [sum (C-R)^2, sum R^2]; returns the 2-element tensor."""
    M, N = C.shape
    if out is None:
        out = torch.empty(2, dtype=torch.float64, device=C.device)
    if ws is None:
        ws = workspace(lib().nk_norm_workspace_size(M, N), C.device)
    _check(lib().nk_rel_frobenius(C.data_ptr(), C.stride(0), R.data_ptr(), R.stride(0), M, N,
                                  out.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream)))
    return out


def nk_sync_status(stream=None):
    _check(lib().nk_sync_status(_stream(stream)))


def nk_set_wait_budget(iterations: int):
    _check(lib().nk_set_wait_budget(int(iterations)))


def nk_set_pdl(enabled: bool):
    """Programmatic dependent launch of the library's kernels (on by default)."""
    _check(lib().nk_set_pdl(1 if enabled else 0))


def nk_get_pdl() -> bool:
    return bool(lib().nk_get_pdl())


def nk_device_info():
    a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().nk_device_info(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


# ------------------------------------------------------------------ grouped GEMM
def make_groups(As, Bts, Cs, accumulate=False):
    """nk_gemm_group array for BF16 A_g [M,K], Bt_g [N,K] (row-major) and FP32 C_g [M,N]."""
    G = len(As)
    arr = (nk_gemm_group * max(G, 1))()
    for g, (a, bt, c) in enumerate(zip(As, Bts, Cs)):
        q = arr[g]
        q.M, q.K = a.shape
        q.N = bt.shape[0]
        q.accumulate = int(bool(accumulate))
        q.A, q.Bt, q.C = a.data_ptr(), bt.data_ptr(), c.data_ptr()
        q.lda, q.ldb, q.ldc = a.stride(0), bt.stride(0), c.stride(0)
    return arr, G


def nk_grouped_workspace_size(G: int) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().nk_grouped_workspace_size(G, None, PREC["bf16"], None, ctypes.byref(n)))
    return n.value


def make_conv_groups(convs):
    """nk_conv_group array from dicts with I (BF16 NHWC), W (packed BF16, from
    nk_conv2d_pack_weights), O (FP32 NHWC) and optional stride, dilation,
    pad (top, bottom, left, right), bias, relu, accumulate."""
    G = len(convs)
    arr = (nk_conv_group * max(G, 1))()
    for g, d in enumerate(convs):
        q = arr[g]
        q.I, q.W, q.O = as_nk_tensor(d["I"]), as_nk_tensor(d["W"]), as_nk_tensor(d["O"])
        st, dl, pd = d.get("stride", (1, 1)), d.get("dilation", (1, 1)), d.get("pad", (0, 0, 0, 0))
        for i in range(2):
            q.stride[i], q.dilation[i] = int(st[i]), int(dl[i])
        for i in range(4):
            q.pad[i] = int(pd[i])
        b = d.get("bias")
        q.bias = b.data_ptr() if b is not None else None
        q.relu = int(bool(d.get("relu", False)))
        q.accumulate = int(bool(d.get("accumulate", False)))
    return arr, G


def nk_conv2d_grouped_plan_create(groups, G, schedule=None):
    h = ctypes.c_void_p()
    _check(lib().nk_conv2d_grouped_plan_create(G, groups, _sched(schedule), ctypes.byref(h)))
    return h


def nk_grouped_plan_create(groups, G, precision="bf16", schedule=None):
    h = ctypes.c_void_p()
    _check(lib().nk_grouped_plan_create(G, groups, PREC[precision], _sched(schedule), ctypes.byref(h)))
    return h


def nk_grouped_plan_run(plan, stream=None):
    _check(lib().nk_grouped_plan_run(plan, _stream(stream)))


def nk_grouped_plan_destroy(plan):
    _check(lib().nk_grouped_plan_destroy(plan))


def nk_batch_matmul_grouped(groups, G, precision="bf16", schedule=None, ws=None, stream=None):
    if ws is None:
        ws = workspace(nk_grouped_workspace_size(G))
    _check(lib().nk_batch_matmul_grouped(G, groups, PREC[precision], _sched(schedule),
                                         ws.data_ptr() if ws is not None else None,
                                         ws.numel() if ws is not None else 0, _stream(stream)))
    return ws


def nk_matmul_f32_splitk_noalloc(A, B, C, split_k, stream=None):
    """C = A @ B (FP32, row-major) with split-K partials in the library's static scratch."""
    M, K = A.shape
    N = B.shape[1]
    _check(lib().nk_matmul_f32_splitk_noalloc(A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0),
                                              C.data_ptr(), C.stride(0), M, N, K, int(split_k),
                                              _stream(stream)))
    return C
