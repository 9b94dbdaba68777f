"""FP64 CPU oracle for the dense contractions -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this module.  The product path (the CUDA library
and its binding) never calls it, and this module imports nothing from the
product: the two share no code.

What it computes, and where the paper defines it:

* ``matmul``: the contraction ``C[m,n] += sum_k A[m,k] * B[k,n]`` of the
  affine loop nest in Listing "for->affine" (Sec. 1) and of the
  ``linalg.generic`` body ``out + in * in_2`` with maps (d0,d2),(d2,d1)->(d0,d1)
  and iterators (parallel, parallel, reduction) of Listing "linalg-matmul"
  (Sec. 2.1.1).  The paper's index names (A:(M,N), B:(N,K), reduction over j)
  are read as the linalg convention A[M,K] B[K,N] with K reduced.
* ``epilogue``: zero-fill then accumulate, then the bias add, as in the
  lowered ``torch.nn.Linear(32,32)`` of Listing "listing1" (Sec. 2.1.2) and the
  ``aten.add`` of the torch-dialect listing (Sec. 2.1.1); ReLU is applied last.
* ``conv2d_nhwc_hwcf``: the output-parallel convolution of Listing
  "2dnchwconv" (Sec. 4.1) -- output += input[ho+ki, wo+kj] * kernel, no
  flip -- adapted to NHWC input / HWCF filter with stride, dilation and
  zero padding (out-of-range input reads as 0).
* ``batch_matmul`` / ``grouped_matmul``: the matmul with a leading batch
  (group) index, one independent contraction per group.
* ``ew_program`` / ``matmul_fused`` / ``conv2d_fused``: elementwise programs
  folded around the contraction -- the bias-add loop that follows the matmul
  of the lowered ``torch.nn.Linear`` (Listing "listing1", Sec. 2.1.2) and the
  elementwise product ``C[x,y] = A[x,y] * B[x,y]`` of the GPUModule kernel
  (Listing "gpumodules", Sec. 3.1) -- as epilogues on the output and
  prologues on the operands, with the usual activations written from their
  definitions.
* Number formats (BF16, FP8 E4M3, the BF16 hi/lo split) written from the
  format definitions, not from any conversion routine.
* The tile-cost MLP (forward, backward, Adam) that ranks schedules for the
  tile-size search of Sec. 4.3.

Floating point is FP64 throughout.  ``numpy.matmul`` on FP64 arrays serves as
the library primitive for the inner sums; everything around it follows the
definitions above step by step.
"""
from __future__ import annotations

import math

import numpy as np

# ------------------------------------------------------------------ formats
BF16_FRAC_BITS = 7            # 1 implicit + 7 stored significand bits
BF16_EMIN = -126              # same exponent range as FP32
BF16_MAX = (2.0 - 2.0 ** -7) * 2.0 ** 127
E4M3_FRAC_BITS = 3
E4M3_EMIN = -6                # bias 7: smallest normal exponent 1 - 7
E4M3_MAX = 448.0              # 1.110b * 2^8 (S.1111.111 is NaN, no infinities)


def _round_to_precision(x: np.ndarray, frac_bits: int, emin: int) -> np.ndarray:
    """Round finite x (FP64) to a binary format with ``frac_bits`` fraction
    bits and minimum normal exponent ``emin``; round-to-nearest, ties to even
    (np.rint rounds halves to even).  Zeros keep their sign; a nonzero value
    that rounds to zero keeps it too (np.rint(-0.3) is -0.0).  No overflow
    handling."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    nz = (x != 0) & np.isfinite(x)
    ax = np.abs(x[nz])
    e = np.floor(np.log2(ax))
    # log2 can be off by one ulp near powers of two: fix the binade exactly.
    e = np.where(np.ldexp(1.0, e.astype(np.int64)) > ax, e - 1, e)
    e = np.where(np.ldexp(1.0, (e + 1).astype(np.int64)) <= ax, e + 1, e)
    e = np.maximum(e, emin)                       # subnormal range: fixed quantum
    quantum_exp = (e - frac_bits).astype(np.int64)
    q = np.rint(np.ldexp(x[nz], -quantum_exp))
    out[nz] = np.ldexp(q, quantum_exp)
    out[~np.isfinite(x)] = x[~np.isfinite(x)]
    out[x == 0] = x[x == 0]                       # a zero keeps its sign (IEEE conversion)
    return out


def bf16_rn(x) -> np.ndarray:
    """Round FP32 values to bfloat16 (RNE), returned as exact FP64 values.

    bfloat16: 1 sign, 8 exponent (bias 127), 7 fraction bits.  Values that
    round beyond the largest finite bf16 become +-inf; NaN stays NaN.
    """
    x = np.asarray(x, dtype=np.float64)
    r = _round_to_precision(x, BF16_FRAC_BITS, BF16_EMIN)
    # rounding up past the largest finite value (at or above the midpoint
    # between BF16_MAX and 2^128, ties go to the even neighbour 2^128) overflows
    big = np.isfinite(x) & (np.abs(r) > BF16_MAX)
    r[big] = np.copysign(np.inf, x[big])
    return r


def e4m3_rn_sat(x) -> np.ndarray:
    """Round to OCP FP8 E4M3 with RNE and saturation to +-448, as FP64 values.

    E4M3: 1 sign, 4 exponent (bias 7), 3 fraction bits; normals from 2^-6,
    subnormals in steps of 2^-9, largest finite 448, no infinities.
    Saturating conversion clamps every finite result (and +-inf) to +-448;
    NaN stays NaN.
    """
    x = np.asarray(x, dtype=np.float64)
    r = _round_to_precision(x, E4M3_FRAC_BITS, E4M3_EMIN)
    r = np.where(np.isnan(x), np.nan, np.clip(r, -E4M3_MAX, E4M3_MAX))
    return r


def e4m3_decode(code: int) -> float:
    """Value of an 8-bit E4M3 code (sign|eeee|mmm), from the format definition."""
    s = -1.0 if code & 0x80 else 1.0
    e = (code >> 3) & 0xF
    m = code & 0x7
    if e == 0xF and m == 0x7:
        return math.nan
    if e == 0:
        return s * m * 2.0 ** (E4M3_EMIN - E4M3_FRAC_BITS)
    return s * (1.0 + m / 8.0) * 2.0 ** (e - 7)


def bf16x3_split(x32) -> tuple[np.ndarray, np.ndarray]:
    """hi = bf16(x), lo = bf16(x - hi).  x - hi is exact in FP32 and FP64."""
    x = np.asarray(x32, dtype=np.float64)
    hi = bf16_rn(x)
    lo = bf16_rn(x - hi)
    return hi, lo


def fp8_scale(x32) -> np.float32:
    """Per-tensor scale s = 448 / amax(|x|) computed in FP32 (s = 1 if amax = 0)."""
    amax = np.float32(np.max(np.abs(np.asarray(x32, dtype=np.float32)))) if np.size(x32) else np.float32(0)
    if amax == 0 or not np.isfinite(amax):
        return np.float32(1.0)
    return np.float32(np.float32(E4M3_MAX) / amax)


def fp8_quantize(x32, s: np.float32) -> np.ndarray:
    """q = e4m3_rn_sat(fl32(x * s)): the product is taken in FP32 so the
    rounding decision is made on the same value the GPU rounds."""
    y = (np.asarray(x32, dtype=np.float32) * np.float32(s)).astype(np.float32)
    return e4m3_rn_sat(y.astype(np.float64))


# ------------------------------------------------------------------ contractions
def matmul(A, B) -> np.ndarray:
    """sum_k A[m,k] * B[k,n] in FP64 (numpy.matmul as the inner-sum primitive)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    assert A.ndim == 2 and B.ndim == 2 and A.shape[1] == B.shape[0]
    return A @ B


def matmul_loops(A, B, C=None) -> np.ndarray:
    """The affine loop nest of Listing "for->affine" written out in Python:
    for each (i, n, k): C[i, n] = C[i, n] + A[i, k] * B[k, n].  Tiny inputs only."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    M, K = A.shape
    N = B.shape[1]
    C = np.zeros((M, N)) if C is None else np.array(C, dtype=np.float64)
    for i in range(M):
        for k in range(K):
            a = A[i, k]
            for n in range(N):
                C[i, n] = C[i, n] + a * B[k, n]
    return C


def epilogue(acc, c_in=None, bias=None, relu=False, alpha=1.0, beta=0.0) -> np.ndarray:
    """out = ReLU?(beta * C_in + alpha * acc + bias[n]).

    beta = 1 is linalg's accumulate-into-outs; beta = 0 is the zero-filled
    output of Listing "listing1"; the bias is added after the contraction as
    in that listing's last loop nest.  ReLU(NaN) stays NaN.
    """
    out = float(alpha) * np.asarray(acc, dtype=np.float64)
    if beta != 0.0 and c_in is not None:
        out = out + float(beta) * np.asarray(c_in, dtype=np.float64)
    if bias is not None:
        out = out + np.asarray(bias, dtype=np.float64)
    if relu:
        out = np.where(np.isnan(out), out, np.maximum(out, 0.0))
    return out


PRECISIONS = ("f32", "bf16", "bf16x3", "fp8")


def prepared_operands(A32, B32, precision: str):
    """The values each precision multiplies, and the dequantisation scales.

    f32: the FP32 inputs; bf16: bf16_rn of each; fp8: e4m3(x * s) with the
    per-tensor scales (s_a, s_b) -- the result is divided by s_a * s_b;
    bf16x3: the (hi, lo) pairs.  Non-FP8 precisions return scale 1.0.
    """
    if precision == "f32":
        return (np.asarray(A32, np.float64), np.asarray(B32, np.float64)), 1.0
    if precision == "bf16":
        return (bf16_rn(A32), bf16_rn(B32)), 1.0
    if precision == "fp8":
        sa, sb = fp8_scale(A32), fp8_scale(B32)
        return (fp8_quantize(A32, sa), fp8_quantize(B32, sb)), (float(sa), float(sb))
    if precision == "bf16x3":
        return (bf16x3_split(A32), bf16x3_split(B32)), 1.0
    raise ValueError(precision)


def matmul_precision(A32, B32, precision: str) -> np.ndarray:
    """Exact (FP64) value of what a precision's arithmetic targets.

    bf16x3 keeps hi*hi + hi*lo + lo*hi and drops lo*lo, the split-precision
    scheme named in the precision extension.
    """
    ops, scale = prepared_operands(A32, B32, precision)
    if precision == "bf16x3":
        (ah, al), (bh, bl) = ops
        return matmul(ah, bh) + matmul(ah, bl) + matmul(al, bh)
    if precision == "fp8":
        # s_a * s_b is exact in FP64 (24 + 24 bits); dividing rounds once
        return matmul(ops[0], ops[1]) / (scale[0] * scale[1])
    return matmul(ops[0], ops[1])


def batch_matmul(A, B) -> np.ndarray:
    """C[b] = A[b] @ B[b] for every batch index b (linalg.batch_matmul)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    assert A.ndim == 3 and B.ndim == 3 and A.shape[0] == B.shape[0]
    return np.stack([matmul(A[b], B[b]) for b in range(A.shape[0])])


def grouped_matmul(As, Bs) -> list:
    """One independent matmul per group (uneven shapes)."""
    return [matmul(a, b) for a, b in zip(As, Bs)]


def conv_out_size(H, KH, stride, dilation, pad_lo, pad_hi):
    return (H + pad_lo + pad_hi - dilation * (KH - 1) - 1) // stride + 1


def conv2d_nhwc_hwcf(I, W, stride=(1, 1), dilation=(1, 1), pad=(0, 0, 0, 0)) -> np.ndarray:
    """O[n,oh,ow,f] = sum_{kh,kw,c} I[n, oh*sh + kh*dh - ph, ow*sw + kw*dw - pw, c] * W[kh,kw,c,f].

    pad = (top, bottom, left, right); reads outside the input are 0.  The sum
    is taken one filter tap (kh, kw) at a time; within a tap the sum over c
    is a matmul of the shifted input window with W[kh, kw].
    """
    I = np.asarray(I, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    N, H, Wd, C = I.shape
    KH, KW, C2, F = W.shape
    assert C == C2
    sh, sw = stride
    dh, dw = dilation
    pt, pb, pl, pr = pad
    OH = conv_out_size(H, KH, sh, dh, pt, pb)
    OW = conv_out_size(Wd, KW, sw, dw, pl, pr)
    Ip = np.zeros((N, H + pt + pb, Wd + pl + pr, C))
    Ip[:, pt:pt + H, pl:pl + Wd, :] = I
    O = np.zeros((N, OH, OW, F))
    for kh in range(KH):
        for kw in range(KW):
            r0, c0 = kh * dh, kw * dw
            win = Ip[:, r0:r0 + sh * (OH - 1) + 1:sh, c0:c0 + sw * (OW - 1) + 1:sw, :]
            O += (win.reshape(-1, C) @ W[kh, kw]).reshape(N, OH, OW, F)
    return O


def conv2d_loops(I, W, stride=(1, 1), dilation=(1, 1), pad=(0, 0, 0, 0)) -> np.ndarray:
    """The 7-deep loop of the convolution definition, in pure Python (tiny only)."""
    I = np.asarray(I, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    N, H, Wd, C = I.shape
    KH, KW, _, F = W.shape
    sh, sw = stride
    dh, dw = dilation
    pt, pb, pl, pr = pad
    OH = conv_out_size(H, KH, sh, dh, pt, pb)
    OW = conv_out_size(Wd, KW, sw, dw, pl, pr)
    O = np.zeros((N, OH, OW, F))
    for n in range(N):
        for oh in range(OH):
            for ow in range(OW):
                for f in range(F):
                    s = 0.0
                    for kh in range(KH):
                        for kw in range(KW):
                            ih = oh * sh + kh * dh - pt
                            iw = ow * sw + kw * dw - pl
                            if 0 <= ih < H and 0 <= iw < Wd:
                                for c in range(C):
                                    s += I[n, ih, iw, c] * W[kh, kw, c, f]
                    O[n, oh, ow, f] = s
    return O


def im2col(I, KH, KW, stride=(1, 1), dilation=(1, 1), pad=(0, 0, 0, 0)) -> np.ndarray:
    """Patch matrix P[(n,oh,ow), (kh,kw,c)] = I[n, ih, iw, c] (0 outside the
    input), built element by element with explicit bounds checks -- a path
    separate from ``conv2d_nhwc_hwcf``; conv = P @ W.reshape(KH*KW*C, F)."""
    I = np.asarray(I, dtype=np.float64)
    N, H, Wd, C = I.shape
    sh, sw = stride
    dh, dw = dilation
    pt, pb, pl, pr = pad
    OH = conv_out_size(H, KH, sh, dh, pt, pb)
    OW = conv_out_size(Wd, KW, sw, dw, pl, pr)
    P = np.zeros((N, OH, OW, KH, KW, C))
    oh = np.arange(OH)
    ow = np.arange(OW)
    for kh in range(KH):
        ih = oh * sh + kh * dh - pt
        okh = (ih >= 0) & (ih < H)
        for kw in range(KW):
            iw = ow * sw + kw * dw - pl
            okw = (iw >= 0) & (iw < Wd)
            for a in np.nonzero(okh)[0]:
                for b in np.nonzero(okw)[0]:
                    P[:, a, b, kh, kw, :] = I[:, ih[a], iw[b], :]
    return P.reshape(N * OH * OW, KH * KW * C)


def conv2d_nchw_fchw_loops(inp, ker) -> np.ndarray:
    """Listing "2dnchwconv" as printed: NCHW input, FCHW kernel, stride 1, no
    padding; out[n,co,ho,wo] += inp[n,ci,ho+ki,wo+kj] * ker[co,ci,ki,kj]."""
    inp = np.asarray(inp, dtype=np.float64)
    ker = np.asarray(ker, dtype=np.float64)
    N, CI, HI, WI = inp.shape
    CO, _, K, _ = ker.shape
    HO, WO = HI - K + 1, WI - K + 1
    out = np.zeros((N, CO, HO, WO))
    for n in range(N):
        for co in range(CO):
            for ho in range(HO):
                for wo in range(WO):
                    for ci in range(CI):
                        for ki in range(K):
                            for kj in range(K):
                                out[n, co, ho, wo] += inp[n, ci, ho + ki, wo + kj] * ker[co, ci, ki, kj]
    return out


# ------------------------------------------------------------------ elementwise programs
def sigmoid(x) -> np.ndarray:
    """The logistic function 1 / (1 + e^-x), written per sign so that exp never
    overflows: for x < 0 it is e^x / (1 + e^x)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    pos = x >= 0
    out[pos] = 1.0 / (1.0 + np.exp(-x[pos]))
    ex = np.exp(x[~pos])
    out[~pos] = ex / (1.0 + ex)
    return out


def silu(x) -> np.ndarray:
    """x * sigmoid(x) (the sigmoid-weighted linear unit, also called swish)."""
    x = np.asarray(x, dtype=np.float64)
    return x * sigmoid(x)


def gelu_tanh(x) -> np.ndarray:
    """The tanh approximation of GELU from Hendrycks and Gimpel (2016):
    0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3)))."""
    x = np.asarray(x, dtype=np.float64)
    return 0.5 * x * (1.0 + np.tanh(math.sqrt(2.0 / math.pi) * (x + 0.044715 * x ** 3)))


EW_STEPS = ("mul", "add", "affine", "relu", "gelu", "gelu_tanh", "silu", "sigmoid", "tanh", "clamp")


def ew_program(x, prog) -> np.ndarray:
    """Run an elementwise program on x, step by step in the given order, in FP64.

    Steps: ("mul", T) -> x * T and ("add", T) -> x + T with T of x's shape (the
    GPUModule product and the Linear layer's bias-add loop, generalised to a
    full operand); ("affine", a, b) -> a x + b; ("relu",) -> max(x, 0) with NaN
    kept; ("gelu",) -> x Phi(x); ("gelu_tanh",); ("silu",); ("sigmoid",);
    ("tanh",); ("clamp", lo, hi) -> lo below lo, hi above hi, NaN kept.
    """
    out = np.array(x, dtype=np.float64)
    for step in prog or ():
        name, *args = step
        if name == "mul":
            out = out * np.asarray(args[0], dtype=np.float64)
        elif name == "add":
            out = out + np.asarray(args[0], dtype=np.float64)
        elif name == "affine":
            out = float(args[0]) * out + float(args[1])
        elif name == "relu":
            out = np.where(np.isnan(out), out, np.maximum(out, 0.0))
        elif name == "gelu":
            out = gelu(out)
        elif name == "gelu_tanh":
            out = gelu_tanh(out)
        elif name == "silu":
            out = silu(out)
        elif name == "sigmoid":
            out = sigmoid(out)
        elif name == "tanh":
            out = np.tanh(out)
        elif name == "clamp":
            lo, hi = float(args[0]), float(args[1])
            out = np.where(out < lo, lo, np.where(out > hi, hi, out))
        else:
            raise ValueError(f"unknown step {name!r}")
    return out


def prologue(x32, prog) -> np.ndarray:
    """An operand after its prologue, as the value the precision then rounds:
    the program in FP64, rounded once to FP32 (the precision in which the
    kernels hand the transformed operand to the BF16 / E4M3 conversion, so
    that both sides take the rounding decision on the same FP32 value)."""
    if not prog:
        return np.asarray(x32, dtype=np.float32)
    return ew_program(np.asarray(x32, dtype=np.float32), prog).astype(np.float32)


def matmul_fused(A32, B32, precision="f32", pro_a=None, pro_b=None, c_in=None, bias=None,
                 relu=False, beta=0.0, ew=None) -> np.ndarray:
    """ew(ReLU?(beta*C_in + op(pro_a(A)) @ op(pro_b(B)) + bias)): the prologues
    on the FP32 operands, the precision's arithmetic (matmul_precision), the
    epilogue, then the epilogue program on each output element."""
    A = prologue(A32, pro_a)
    B = prologue(B32, pro_b)
    acc = matmul_precision(A, B, precision)
    return ew_program(epilogue(acc, c_in, bias, relu, beta=beta), ew)


def conv2d_precision(I32, W32, precision="f32", stride=(1, 1), dilation=(1, 1), pad=(0, 0, 0, 0)) -> np.ndarray:
    """The convolution on the values a precision multiplies: FP32 as given,
    bf16_rn of I and W, or E4M3 codes with per-tensor scales (result divided
    by s_i * s_w)."""
    if precision == "f32":
        return conv2d_nhwc_hwcf(I32, W32, stride, dilation, pad)
    if precision == "bf16":
        return conv2d_nhwc_hwcf(bf16_rn(I32), bf16_rn(W32), stride, dilation, pad)
    if precision == "fp8":
        si, sw = fp8_scale(I32), fp8_scale(W32)
        O = conv2d_nhwc_hwcf(fp8_quantize(I32, si), fp8_quantize(W32, sw), stride, dilation, pad)
        return O / (float(si) * float(sw))
    raise ValueError(precision)


def conv2d_fused(I32, W32, precision="f32", stride=(1, 1), dilation=(1, 1), pad=(0, 0, 0, 0), pro_i=None,
                 pro_w=None, o_in=None, bias=None, relu=False, beta=0.0, ew=None) -> np.ndarray:
    """ew(ReLU?(beta*O_in + conv(pro_i(I), pro_w(W)) + bias)).  The prologue
    runs on the input tensor itself, so the zero padding the convolution
    reads outside it stays zero."""
    I = prologue(I32, pro_i)
    W = prologue(W32, pro_w)
    acc = conv2d_precision(I, W, precision, stride, dilation, pad)
    return ew_program(epilogue(acc, o_in, bias, relu, beta=beta), ew)


def rel_frobenius(C, R) -> float:
    """||C - R||_F / ||R||_F in FP64 (0/0 is 0)."""
    C = np.asarray(C, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    num = math.sqrt(float(np.sum((C - R) ** 2)))
    den = math.sqrt(float(np.sum(R ** 2)))
    if den == 0.0:
        return 0.0 if num == 0.0 else math.inf
    return num / den


# ------------------------------------------------------------------ MLP cost model
MLP_DIMS = (16, 128, 128, 1)
MLP_PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def mlp_param_shapes(dims=MLP_DIMS):
    d0, d1, d2, d3 = dims
    return {"W1": (d1, d0), "b1": (d1,), "W2": (d2, d1), "b2": (d2,), "W3": (d3, d2), "b3": (d3,)}


def gelu(x) -> np.ndarray:
    """Exact GELU: x * Phi(x) = 0.5 x (1 + erf(x / sqrt 2))."""
    x = np.asarray(x, dtype=np.float64)
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x) -> np.ndarray:
    """d/dx [x Phi(x)] = Phi(x) + x phi(x)."""
    x = np.asarray(x, dtype=np.float64)
    Phi = 0.5 * (1.0 + _erf(x / math.sqrt(2.0)))
    phi = np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    return Phi + x * phi


def _erf(x: np.ndarray) -> np.ndarray:
    try:
        from scipy.special import erf
        return erf(x)
    except ImportError:  # pragma: no cover - scipy is present on both hosts
        return np.vectorize(math.erf, otypes=[np.float64])(x)


def mlp_forward(params: dict, X):
    """y = W3 GELU(W2 GELU(W1 x + b1) + b2) + b3 for each row x of X [B, 16]."""
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ params["W1"].T + params["b1"]
    h1 = gelu(z1)
    z2 = h1 @ params["W2"].T + params["b2"]
    h2 = gelu(z2)
    y = h2 @ params["W3"].T + params["b3"]
    cache = dict(X=X, z1=z1, h1=h1, z2=z2, h2=h2)
    return y[:, 0], cache


def mse_loss(y, t) -> float:
    """L = mean_i (y_i - t_i)^2."""
    d = np.asarray(y, np.float64) - np.asarray(t, np.float64)
    return float(np.mean(d * d))


def mlp_backward(params: dict, cache: dict, y, t) -> dict:
    """Gradients of the MSE loss with respect to every parameter (chain rule)."""
    B = cache["X"].shape[0]
    dy = (2.0 / B) * (np.asarray(y, np.float64) - np.asarray(t, np.float64))[:, None]
    g = {}
    g["W3"] = dy.T @ cache["h2"]
    g["b3"] = dy.sum(axis=0)
    dh2 = dy @ params["W3"]
    dz2 = dh2 * gelu_grad(cache["z2"])
    g["W2"] = dz2.T @ cache["h1"]
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ params["W2"]
    dz1 = dh1 * gelu_grad(cache["z1"])
    g["W1"] = dz1.T @ cache["X"]
    g["b1"] = dz1.sum(axis=0)
    return g


def adam_step(params: dict, grads: dict, m: dict, v: dict, t: int, lr=1e-3,
              beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1), step t >= 1:
    m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; m^ = m/(1-b1^t); v^ = v/(1-b2^t);
    theta -= lr m^ / (sqrt(v^) + eps).  Returns new (params, m, v)."""
    P, Mo, Vo = {}, {}, {}
    for k in params:
        g = np.asarray(grads[k], np.float64)
        Mo[k] = beta1 * m[k] + (1.0 - beta1) * g
        Vo[k] = beta2 * v[k] + (1.0 - beta2) * g * g
        mh = Mo[k] / (1.0 - beta1 ** t)
        vh = Vo[k] / (1.0 - beta2 ** t)
        P[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return P, Mo, Vo
