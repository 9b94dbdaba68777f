"""Pins for the FP64 oracle against facts fixed outside it (CPU only).

Each test ties an oracle function to something other than itself: a value
read off the paper's listings, a hand-derived format boundary, a closed form,
an algebraic identity, brute force on tiny inputs, or an independent library
routine (torch's CPU conversions, conv2d, autograd and Adam in FP64).
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle.nk_oracle as O
from paper_2307_16080_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([p.strip() for p in line.split("|")])
    return rows


def _parse(v):
    v = v.strip()
    if v in ("inf", "-inf"):
        return float(v)
    return float.fromhex(v) if "0x" in v else float(v)


# ------------------------------------------------------------------ formats
def test_format_golden_cases():
    rows = _read_golden("format_cases.txt")
    assert len(rows) >= 20
    for fmt, x, want in rows:
        x, want = _parse(x), _parse(want)
        got = (O.bf16_rn if fmt == "bf16" else O.e4m3_rn_sat)(np.array([x]))[0]
        assert got == want or (math.isnan(got) and math.isnan(want)), (fmt, x, got, want)


def _fp32_bit_patterns(n, seed=7):
    bits = synth.raw_u64(seed, 0, n).astype(np.uint32)  # low 32 bits
    x = bits.view(np.float32)
    return x[np.isfinite(x)]


def test_bf16_matches_torch_cpu_conversion():
    x = _fp32_bit_patterns(200_000)
    # add ties and values near every binade edge
    k = np.arange(-140, 128, dtype=np.float64)
    extra = np.concatenate([np.ldexp(1.0 + 2.0 ** -8, k.astype(int)),
                            np.ldexp(1.0 + 3 * 2.0 ** -8, k.astype(int)),
                            np.ldexp(2.0 - 2.0 ** -9, k.astype(int))]).astype(np.float32)
    x = np.concatenate([x, extra[np.isfinite(extra)]])
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    got = O.bf16_rn(x)
    np.testing.assert_array_equal(got, want)
    assert np.isnan(O.bf16_rn(np.array([np.nan]))[0])
    assert O.bf16_rn(np.array([np.inf]))[0] == np.inf


def test_e4m3_code_table_is_fixed_point_and_complete():
    vals = np.array([O.e4m3_decode(c) for c in range(256)])
    finite = vals[~np.isnan(vals)]
    assert np.sum(np.isnan(vals)) == 2           # S.1111.111 only
    assert finite.max() == 448.0 and finite.min() == -448.0
    assert np.min(np.abs(finite[finite != 0])) == 2.0 ** -9
    np.testing.assert_array_equal(O.e4m3_rn_sat(finite), finite)
    # every rounding result lands in the code table
    x = synth.normal(3, 0, (50_000,), sigma=60.0).astype(np.float64)
    r = O.e4m3_rn_sat(x)
    assert np.isin(r, finite).all()
    # midpoints between neighbours go to the code with an even last bit
    pos = np.array(sorted(set(finite[finite >= 0].tolist())))
    codes = {O.e4m3_decode(c): c for c in range(0x7F)}
    for lo, hi in zip(pos[:-1], pos[1:]):
        mid = 0.5 * (lo + hi)
        even = lo if codes[lo] % 2 == 0 else hi
        assert O.e4m3_rn_sat(np.array([mid]))[0] == even


def test_e4m3_matches_torch_cpu_conversion_in_range():
    x = synth.normal(4, 0, (200_000,), sigma=100.0)
    x = x[np.abs(x) < 464.0]   # torch's e4m3fn cast is non-saturating above this
    want = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(O.e4m3_rn_sat(x), want)
    big = np.array([464.0, 500.0, 1e6, -465.0, np.inf, -np.inf])
    np.testing.assert_array_equal(O.e4m3_rn_sat(big), [448, 448, 448, -448, 448, -448])


def test_conversions_keep_the_sign_of_zero():
    """IEEE round-to-nearest keeps the sign of a zero, and of a value that
    rounds to zero; assert_array_equal cannot see it, so compare sign bits
    against torch's conversions."""
    x = np.array([-0.0, 0.0, -1e-30, 1e-30, -1e-45, 1e-45, 2.0 ** -10, -2.0 ** -10, -2.0 ** -11, -3e-3, 3e-3],
                 np.float32)
    x = np.concatenate([x, _fp32_bit_patterns(20_000)])
    b = O.bf16_rn(x)
    tb = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(b, tb)
    np.testing.assert_array_equal(np.signbit(b), np.signbit(tb))
    xe = x[np.abs(x) < 464.0]
    e = O.e4m3_rn_sat(xe)
    te = torch.from_numpy(xe).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(e, te)
    np.testing.assert_array_equal(np.signbit(e), np.signbit(te))
    assert np.signbit(O.fp8_quantize(np.array([-0.0], np.float32), np.float32(2.0))[0])


def test_bf16x3_split_properties():
    x = synth.outlier_normal(5, 0, (100_000,)).astype(np.float64)
    hi, lo = O.bf16x3_split(x)
    np.testing.assert_array_equal(O.bf16_rn(hi), hi)
    np.testing.assert_array_equal(O.bf16_rn(lo), lo)
    # hi + lo carries at least 16 significant bits of x
    rel = np.abs(x - hi - lo) / np.maximum(np.abs(x), 1e-300)
    assert rel.max() <= 2.0 ** -16
    # |lo| is at most half a bf16 ulp of hi
    assert np.all(np.abs(lo) <= np.abs(hi) * 2.0 ** -8 + 1e-300)


def test_fp8_scale_closed_forms():
    assert O.fp8_scale(np.zeros(4, np.float32)) == 1.0
    assert O.fp8_scale(np.array([448.0, -3.0], np.float32)) == 1.0
    assert O.fp8_scale(np.array([3.5, 1.0], np.float32)) == 128.0
    x = synth.outlier_normal(6, 0, (10_000,))
    s = O.fp8_scale(x)
    q = O.fp8_quantize(x, s)
    assert np.max(np.abs(q)) == 448.0        # the amax entry maps to the format max
    # relative quantisation error of normal-range values is at most 2^-4
    big = np.abs(x * float(s)) >= 2.0 ** -6
    rel = np.abs(q[big] - x[big] * float(s)) / np.abs(x[big] * float(s))
    assert rel.max() <= 2.0 ** -4 * (1 + 1e-6)


# ------------------------------------------------------------------ matmul
def test_paper_matmul_ones_and_linear_literals():
    rows = {r[0]: r for r in _read_golden("paper_cases.txt")}
    # Listing "for->affine": 4x16x8 with ones
    C = O.matmul_loops(np.ones((4, 16)), np.ones((16, 8)))
    assert np.all(C == float(rows["matmul_ones"][2]))
    # torch-dialect Linear(32,32): y = x W^T + b, W = b = 1
    W = np.ones((32, 32))
    b = np.ones(32)
    y = O.epilogue(O.matmul(np.ones((32, 32)), W.T), bias=b)
    assert np.all(y == float(rows["linear_ones"][2]))
    x = np.tile(np.arange(32.0), (32, 1))
    y = O.epilogue(O.matmul(x, W.T), bias=b)
    assert np.all(y == float(rows["linear_ramp"][2]))


@pytest.mark.parametrize("prec", O.PRECISIONS)
def test_all_ones_closed_form(prec):
    for M, N, K in [(3, 5, 7), (16, 32, 64), (33, 17, 129)]:
        C = O.matmul_precision(np.ones((M, K), np.float32), np.ones((K, N), np.float32), prec)
        assert np.all(C == K)


def test_identity_and_transpose():
    A = synth.uniform(9, 0, (37, 53))
    B = synth.uniform(9, 1, (53, 29))
    np.testing.assert_array_equal(O.matmul(A, np.eye(53)), A.astype(np.float64))
    np.testing.assert_array_equal(O.matmul(np.eye(37), A), A.astype(np.float64))
    lhs = O.matmul(A, B).T
    rhs = O.matmul(B.T, A.T)
    assert O.rel_frobenius(lhs, rhs) < 1e-15
    # a swapped or transposed operand is caught by this identity
    assert O.rel_frobenius(O.matmul(A[:29, :29], B[:29, :29]),
                           O.matmul(B[:29, :29], A[:29, :29])) > 1e-2


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (3, 8, 5), (4, 8, 16), (15, 17, 16), (8, 31, 33)])
def test_brute_force_small_ints_exact(M, N, K):
    A = synth.small_ints(11, M * 100 + K, (M, K))
    B = synth.small_ints(11, N * 100 + K + 1, (K, N))
    np.testing.assert_array_equal(O.matmul(A, B), O.matmul_loops(A, B))
    for prec in ("f32", "bf16", "bf16x3"):
        np.testing.assert_array_equal(O.matmul_precision(A, B, prec), O.matmul_loops(A, B))
    # FP8: half-integers up to 3.5 with amax 3.5 give s = 128 and exact codes
    A8, B8 = A.copy() / 2 + 0.0, B.copy() / 2 + 0.0
    A8.flat[0], B8.flat[0] = 3.5, -3.5
    np.testing.assert_array_equal(O.matmul_precision(A8, B8, "fp8"), O.matmul_loops(A8, B8))


def test_precision_errors_have_expected_size():
    A, B = synth.matmul_outlier(128, 128, 512, seed=17)
    R = O.matmul(A, B)
    e_bf16 = O.rel_frobenius(O.matmul_precision(A, B, "bf16"), R)
    e_x3 = O.rel_frobenius(O.matmul_precision(A, B, "bf16x3"), R)
    e_fp8 = O.rel_frobenius(O.matmul_precision(A, B, "fp8"), R)
    assert 5e-4 < e_bf16 < 8e-3
    assert e_x3 < 2e-5 and e_x3 < e_bf16 / 100
    assert 5e-3 < e_fp8 < 6e-2


def test_epilogue_closed_form():
    acc = np.array([[1.0, -2.0], [3.0, np.nan]])
    cin = np.array([[10.0, 10.0], [-10.0, 0.0]])
    out = O.epilogue(acc, c_in=cin, bias=np.array([0.5, -0.5]), relu=True, alpha=2.0, beta=1.0)
    # ReLU(1*C_in + 2*acc + bias)
    assert out[0, 0] == 12.5 and out[0, 1] == 5.5 and out[1, 0] == 0.0 and np.isnan(out[1, 1])
    out = O.epilogue(acc, c_in=cin, beta=0.0)
    np.testing.assert_array_equal(out[:, 0], [1.0, 3.0])


def test_batch_and_grouped():
    A = synth.uniform(12, 0, (3, 7, 9))
    B = synth.uniform(12, 1, (3, 9, 5))
    want = np.einsum("bmk,bkn->bmn", A.astype(np.float64), B.astype(np.float64))
    assert O.rel_frobenius(O.batch_matmul(A, B), want) < 1e-15
    g = O.grouped_matmul([A[0]], [B[0]])
    np.testing.assert_array_equal(g[0], O.matmul(A[0], B[0]))
    shapes = synth.grouped_problems(512)
    assert shapes.min() >= 32 and shapes.max() <= 2048 and np.all(shapes % 16 == 0)


def test_rel_frobenius_closed_forms():
    R = synth.uniform(13, 0, (20, 30)).astype(np.float64)
    assert abs(O.rel_frobenius(R * (1 + 1e-3), R) - 1e-3) < 1e-12
    assert O.rel_frobenius(np.zeros(3), np.zeros(3)) == 0.0
    assert O.rel_frobenius(np.zeros(3), R[0, :3]) == pytest.approx(1.0)


# ------------------------------------------------------------------ conv
CONV_CASES = [
    # N, H, W, C, F, KH, KW, stride, dilation, pad
    (1, 5, 6, 2, 3, 3, 3, (1, 1), (1, 1), (0, 0, 0, 0)),
    (2, 7, 5, 3, 4, 3, 3, (1, 1), (1, 1), (1, 1, 1, 1)),
    (1, 9, 8, 2, 2, 3, 2, (2, 1), (1, 2), (1, 0, 2, 1)),
    (2, 6, 6, 4, 3, 1, 1, (2, 2), (1, 1), (0, 0, 0, 0)),
]


@pytest.mark.parametrize("case", CONV_CASES)
def test_conv_equals_loops_im2col_and_torch(case):
    N, H, W, C, F, KH, KW, st, dl, pad = case
    I = synth.normal(14, 0, (N, H, W, C))
    Wt = synth.normal(14, 1, (KH, KW, C, F))
    O1 = O.conv2d_nhwc_hwcf(I, Wt, st, dl, pad)
    O2 = O.conv2d_loops(I, Wt, st, dl, pad)
    P = O.im2col(I, KH, KW, st, dl, pad)
    O3 = (P @ Wt.astype(np.float64).reshape(KH * KW * C, F)).reshape(O1.shape)
    assert O.rel_frobenius(O1, O2) < 1e-14
    assert O.rel_frobenius(O1, O3) < 1e-14
    # independent library routine: torch conv2d in FP64 (NCHW / FCHW, explicit pad)
    t = torch.from_numpy(I.astype(np.float64)).permute(0, 3, 1, 2)
    t = torch.nn.functional.pad(t, (pad[2], pad[3], pad[0], pad[1]))
    w = torch.from_numpy(Wt.astype(np.float64)).permute(3, 2, 0, 1)
    ref = torch.nn.functional.conv2d(t, w, stride=st, dilation=dl).permute(0, 2, 3, 1).numpy()
    assert O.rel_frobenius(O1, ref) < 1e-14


def test_conv_1x1_is_matmul():
    I = synth.normal(15, 0, (2, 5, 7, 6))
    Wt = synth.normal(15, 1, (1, 1, 6, 4))
    out = O.conv2d_nhwc_hwcf(I, Wt)
    mm = O.matmul(I.reshape(-1, 6), Wt.reshape(6, 4)).reshape(2, 5, 7, 4)
    np.testing.assert_array_equal(out, mm)


def test_conv_matches_paper_nchw_listing():
    # Listing "2dnchwconv" layout (NCHW / FCHW, stride 1, no pad), Ci=1, Co=3, K=3
    # as in the tuning experiment, on a reduced spatial size.
    rows = {r[0]: r for r in _read_golden("paper_cases.txt")}
    inp = synth.normal(16, 0, (1, 1, 12, 11))
    ker = synth.normal(16, 1, (3, 1, 3, 3))
    want = O.conv2d_nchw_fchw_loops(inp, ker)
    got = O.conv2d_nhwc_hwcf(inp.transpose(0, 2, 3, 1), ker.transpose(2, 3, 1, 0)).transpose(0, 3, 1, 2)
    assert O.rel_frobenius(got, want) < 1e-14
    # the experiment's full size with unit input/kernel: every output is 9
    exp = rows["conv_nchw_ones"]
    out = O.conv2d_nhwc_hwcf(np.ones((1, 1280, 1280, 1)), np.ones((3, 3, 1, 3)))
    assert out.shape == (1, 1278, 1278, 3) and "HO=1278" in exp[2]
    assert np.all(out == 9.0)


# ------------------------------------------------------------------ MLP
def _mlp_params(seed=21):
    shapes = O.mlp_param_shapes()
    p = {}
    for i, name in enumerate(O.MLP_PARAM_NAMES):
        fan_in = shapes[name][-1] if name.startswith("W") else 16
        p[name] = synth.normal(seed, i, shapes[name], sigma=1.0 / math.sqrt(fan_in)).astype(np.float64)
    return p


def test_mlp_param_count():
    shapes = O.mlp_param_shapes()
    assert sum(int(np.prod(s)) for s in shapes.values()) == 18817


def test_gelu_closed_forms_and_torch():
    x = np.linspace(-6, 6, 1001)
    np.testing.assert_allclose(O.gelu(-x), O.gelu(x) - x, atol=1e-15)
    assert O.gelu(np.array([0.0]))[0] == 0.0
    assert abs(O.gelu(np.array([10.0]))[0] - 10.0) < 1e-15
    ref = torch.nn.functional.gelu(torch.from_numpy(x)).numpy()
    np.testing.assert_allclose(O.gelu(x), ref, rtol=1e-14, atol=1e-15)
    h = 1e-6
    fd = (O.gelu(x + h) - O.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(O.gelu_grad(x), fd, atol=1e-8)


def test_mlp_forward_backward_vs_finite_differences_and_autograd():
    p = _mlp_params()
    X = synth.normal(22, 0, (24, 16)).astype(np.float64)
    t = synth.normal(22, 1, (24,)).astype(np.float64)
    y, cache = O.mlp_forward(p, X)
    g = O.mlp_backward(p, cache, y, t)
    # central finite differences on a sample of coordinates of every tensor
    h = 1e-6
    for name in O.MLP_PARAM_NAMES:
        flat = p[name].reshape(-1)
        idx = np.unique(synth.raw_u64(23, len(name), 6) % np.uint64(flat.size)).astype(int)
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp = O.mse_loss(O.mlp_forward(p, X)[0], t)
            flat[i] = old - h
            lm = O.mse_loss(O.mlp_forward(p, X)[0], t)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, i, fd, an)
    # independent library routine: torch autograd in FP64
    tp = {k: torch.tensor(v, requires_grad=True) for k, v in p.items()}
    tx = torch.from_numpy(X)
    h1 = torch.nn.functional.gelu(tx @ tp["W1"].T + tp["b1"])
    h2 = torch.nn.functional.gelu(h1 @ tp["W2"].T + tp["b2"])
    ty = (h2 @ tp["W3"].T + tp["b3"])[:, 0]
    loss = torch.mean((ty - torch.from_numpy(t)) ** 2)
    loss.backward()
    np.testing.assert_allclose(y, ty.detach().numpy(), rtol=1e-13, atol=1e-14)
    assert abs(O.mse_loss(y, t) - loss.item()) < 1e-13
    for k in p:
        np.testing.assert_allclose(g[k], tp[k].grad.numpy(), rtol=1e-11, atol=1e-14)


def test_adam_first_step_closed_form_and_torch():
    p = _mlp_params(31)
    g = {k: synth.normal(32, i, v.shape).astype(np.float64) for i, (k, v) in enumerate(p.items())}
    z = {k: np.zeros_like(v) for k, v in p.items()}
    lr, eps = 1e-2, 1e-8
    p1, m1, v1 = O.adam_step(p, g, z, z, 1, lr=lr, eps=eps)
    for k in p:   # at t = 1: theta -= lr * g / (|g| + eps)
        np.testing.assert_allclose(p1[k], p[k] - lr * g[k] / (np.abs(g[k]) + eps), rtol=1e-14, atol=1e-15)
    # three steps against torch.optim.Adam in FP64
    tp = [torch.tensor(p[k], requires_grad=True) for k in O.MLP_PARAM_NAMES]
    opt = torch.optim.Adam(tp, lr=lr, betas=(0.9, 0.999), eps=eps)
    cur, m, v = p, z, z
    for step in range(1, 4):
        gs = {k: g[k] * (1.0 + 0.5 * step) for k in p}
        for t_, k in zip(tp, O.MLP_PARAM_NAMES):
            t_.grad = torch.from_numpy(gs[k].copy())
        opt.step()
        cur, m, v = O.adam_step(cur, gs, m, v, step, lr=lr, eps=eps)
    for t_, k in zip(tp, O.MLP_PARAM_NAMES):
        np.testing.assert_allclose(cur[k], t_.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_mlp_learns_linear_target():
    p = _mlp_params(41)
    X = synth.normal(42, 0, (256, 16)).astype(np.float64)
    w = synth.normal(42, 1, (16,)).astype(np.float64)
    t = X @ w * 0.3 + 1.0
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(x) for k, x in p.items()}
    first = None
    for step in range(1, 301):
        y, cache = O.mlp_forward(p, X)
        loss = O.mse_loss(y, t)
        first = loss if first is None else first
        g = O.mlp_backward(p, cache, y, t)
        p, m, v = O.adam_step(p, g, m, v, step, lr=3e-3)
    assert loss < 0.02 * first
