"""CPU checks of the fused elementwise programs at the C ABI: the ctypes
structs match the header's layout, and every malformed program is refused
before anything touches a device (arguments are host-side views only)."""
import ctypes
import os
import shutil
import subprocess

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nk():
    from paper_2307_16080_gb300 import _build
    _build.build()
    import paper_2307_16080_gb300.nk as nk
    return nk


def test_struct_layout_matches_header(nk, tmp_path):
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    src = tmp_path / "probe.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "nk.h"\n'
        "int main(void) {\n"
        '  printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(nk_epilogue), sizeof(nk_ew_program),\n'
        "         sizeof(nk_ew_op), offsetof(nk_epilogue, ew), offsetof(nk_epilogue, pro_a),\n"
        "         offsetof(nk_epilogue, pro_b), offsetof(nk_ew_op, t), offsetof(nk_ew_program, ops));\n"
        "  return 0;\n}\n")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(nk.nk_epilogue), ctypes.sizeof(nk.nk_ew_program), ctypes.sizeof(nk.nk_ew_op),
            nk.nk_epilogue.ew.offset, nk.nk_epilogue.pro_a.offset, nk.nk_epilogue.pro_b.offset,
            nk.nk_ew_op.t.offset, nk.nk_ew_program.ops.offset]
    assert got == want


def _status(fn, *a, **k):
    from paper_2307_16080_gb300.nk import NkError
    k.setdefault("stream", 0)   # no torch CUDA stream on a CPU-only host
    try:
        fn(*a, **k)
    except NkError as e:
        return e.status, str(e)
    return 0, ""


BAD_PROGRAMS = [
    ([("relu",)] * 5, "operations"),
    ([(99,)], "unknown opcode"),
    ([("clamp", 1.0, -1.0)], "CLAMP"),
    ([("clamp", float("nan"), 1.0)], "CLAMP"),
    ([("affine", float("nan"), 0.0)], "NaN"),
]


@pytest.mark.parametrize("prog,msg", BAD_PROGRAMS)
def test_elementwise_rejects_malformed_programs(nk, prog, msg):
    x = torch.zeros(4, 8)
    st, text = _status(nk.nk_elementwise, x, x, prog)
    assert st == -1 and msg in text, text


def test_tensor_operand_must_match_output_layout(nk):
    y = torch.zeros(4, 8)
    cases = [
        (torch.zeros(4, 9), "dim 1"),                     # shape
        (torch.zeros(8, 4).t(), "stride"),                 # same shape, other strides
        (torch.zeros(4, 8, dtype=torch.float64), "FP32"),  # dtype
        (torch.zeros(32), "rank"),                         # rank
    ]
    for t, msg in cases:
        st, text = _status(nk.nk_elementwise, y, y, [("mul", t)])
        assert st == -1 and msg in text, (msg, text)
    # a misaligned operand (4-byte rule): a float view shifted by 2 bytes
    raw = torch.zeros(4 * 8 * 4 + 8, dtype=torch.uint8)
    t = nk.as_nk_tensor(y)
    t.ptr = raw.data_ptr() + 2
    prog = nk.nk_ew_program()
    prog.n = 1
    prog.ops[0].op = nk.EW_OPS["add"]
    prog.ops[0].t = t
    ty = nk.as_nk_tensor(y)
    st = nk.lib().nk_elementwise(ctypes.byref(ty), ctypes.byref(ty), ctypes.byref(prog), None)
    assert st == -1 and "aligned" in nk.last_error()
    # NULL operand with elements present (ctypes copied t into the program)
    prog.ops[0].t.ptr = None
    st = nk.lib().nk_elementwise(ctypes.byref(ty), ctypes.byref(ty), ctypes.byref(prog), None)
    assert st == -1 and "NULL" in nk.last_error()


def test_elementwise_shape_checks(nk):
    st, text = _status(nk.nk_elementwise, torch.zeros(4, 8), torch.zeros(4, 9), [("relu",)])
    assert st == -1 and "shapes" in text
    st, text = _status(nk.nk_elementwise, torch.zeros(4, 8, dtype=torch.float64), torch.zeros(4, 8), [("relu",)])
    assert st == -2


def test_matmul_and_conv_validate_programs_before_the_device(nk):
    A, B, C = torch.zeros(16, 32), torch.zeros(32, 24), torch.zeros(16, 24)
    for prec in ("f32", "bf16"):
        st, text = _status(nk.nk_matmul, A, B, C, prec, ew=[("add", torch.zeros(16, 25))], ws=None)
        assert st == -1 and "ew op 0" in text, text
        st, text = _status(nk.nk_matmul, A, B, C, prec, pro_a=[("mul", torch.zeros(32, 24))])
        assert st == -1 and "pro_a" in text, text
        st, text = _status(nk.nk_matmul, A, B, C, prec, pro_b=[("clamp", 2, 1)])
        assert st == -1 and "pro_b" in text, text
    # operands already in BF16 take no prologue
    Ab = torch.zeros(16, 32, dtype=torch.bfloat16)
    Bb = torch.zeros(24, 32, dtype=torch.bfloat16).t()
    st, text = _status(nk.nk_matmul, Ab, Bb, C, "bf16", pro_a=[("relu",)], ws=torch.zeros(1 << 20, dtype=torch.uint8))
    assert st == -2 and "prologue" in text, text
    I, W, O_ = torch.zeros(1, 6, 6, 8), torch.zeros(3, 3, 8, 16), torch.zeros(1, 6, 6, 16)
    st, text = _status(nk.nk_conv2d_nhwc_hwcf, I, W, O_, pad=(1, 1, 1, 1), ew=[("mul", torch.zeros(1, 6, 6, 15))])
    assert st == -1 and "ew" in text, text
    st, text = _status(nk.nk_conv2d_nhwc_hwcf, I, W, O_, pad=(1, 1, 1, 1), pro_i=[("add", torch.zeros(1, 6, 6, 16))])
    assert st == -1 and "pro_a (I)" in text, text
    Ib = torch.zeros(1, 6, 6, 8, dtype=torch.bfloat16)
    st, text = _status(nk.nk_conv2d_nhwc_hwcf, Ib, W, O_, pad=(1, 1, 1, 1), precision="bf16", pro_i=[("relu",)],
                       ws=torch.zeros(1 << 20, dtype=torch.uint8))
    assert st == -2 and "prologue" in text, text
    Ic, Kc, Oc = torch.zeros(1, 1, 8, 8), torch.zeros(3, 1, 3, 3), torch.zeros(1, 3, 6, 6)
    st, text = _status(nk.nk_conv2d_nchw_fchw, Ic, Kc, Oc, ew=[("add", torch.zeros(1, 3, 6, 7))])
    assert st == -1 and "ew" in text, text
