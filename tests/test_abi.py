"""CPU checks of the C ABI: the library builds, loads, and exports every entry
point that include/*.h declares; the ctypes binding covers them all.  No
compute call is made (there is no GPU here)."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(nk_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2307_16080_gb300 import _build
    return _build.build()


def test_headers_declare_entry_points():
    names = _declared()
    for must in ("nk_matmul", "nk_batch_matmul_grouped", "nk_conv2d_nhwc_hwcf", "nk_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = sorted(_declared() - exported)
    assert not missing, missing


def test_ctypes_binding_loads_and_covers_header(libpath):
    import paper_2307_16080_gb300.nk as nk
    import paper_2307_16080_gb300.nk_tune as nt
    L = nt.lib()
    for name in _declared():
        assert hasattr(L, name), name
        assert name in nk.SIGNATURES or name in nt.SIGNATURES, name
    assert nk.last_error() == ""
    assert nt.nk_mlp_param_count() == 18817


def test_no_device_means_error_not_fallback(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2307_16080_gb300.nk as nk
    sms = nk.ctypes.c_int32()
    st = nk.lib().nk_device_info(nk.ctypes.byref(sms), None, None)
    assert st == -5 and "cuda" in nk.last_error().lower() or st == -5


def test_workspace_size_from_problem_matches_operand_form(libpath):
    """nk_workspace_size(problem, schedule) is the operand-based query on
    dense FP32 operands of that problem (planning only: no device needed)."""
    import torch
    import paper_2307_16080_gb300.nk as nk
    import paper_2307_16080_gb300.nk_tune as nt
    for (M, N, K, prec, sched) in [(1000, 900, 700, "bf16", None), (512, 512, 512, "fp8", (128, 128, 128, 1, 4, 4)),
                                   (300, 200, 96, "bf16x3", None), (64, 64, 64, "f32", (64, 64, 16, 1, 2, 3))]:
        a, b, c = torch.empty(M, K), torch.empty(K, N), torch.empty(M, N)
        want = nk.nk_matmul_workspace_size(a, b, c, prec, sched)
        assert nt.nk_workspace_size(nt.matmul_problem(M, N, K, prec), sched) == want
    for (n, h, c_, f, k, s, prec) in [(8, 56, 64, 64, 3, 1, "bf16"), (2, 15, 20, 40, 3, 2, "fp8"), (1, 7, 512, 512, 1, 1, "bf16")]:
        oh = (h + 2 * (k // 2) - k) // s + 1
        i, w, o = torch.empty(n, h, h, c_), torch.empty(k, k, c_, f), torch.empty(n, oh, oh, f)
        want = nk.nk_conv2d_workspace_size(i, w, o, (s, s), (1, 1), (k // 2,) * 4, prec)
        assert nt.nk_workspace_size(nt.conv_problem(n, h, h, c_, f, k, k, s, k // 2, prec)) == want
