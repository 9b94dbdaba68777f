"""Host-side schedule space (no GPU): which convolutions get the window
kernel with stacked kernel rows (tile_k = 64 * KH), and that its workspace
is only the operand casts, as for the plain window kernel.  The schedule
space is what the tuner and the cost model rank."""
import pytest

nt = pytest.importorskip("paper_2307_16080_gb300.nk_tune")


def _stacked(p):
    return [s for s in nt.nk_enumerate_schedules(p) if s[2] == 64 * p.kh and p.kw >= 2]


def test_stacked_schedules_for_stride1_3x3():
    p = nt.conv_problem(8, 56, 56, 64, 64, 3, 3, 1, 1)
    got = _stacked(p)
    assert got == [(128, 64, 192, 1, st, 1) for st in (1, 2, 3, 4)]
    plain = nt.nk_workspace_size(p, (128, 64, 576, 1, 1, 1))
    assert all(nt.nk_workspace_size(p, s) == plain for s in got)


@pytest.mark.parametrize("args", [
    (8, 56, 56, 64, 64, 3, 3, 2, 1),     # strided
    (8, 56, 56, 64, 64, 5, 5, 1, 2),     # KW = 5: N = 320 > 256
    (8, 56, 56, 64, 64, 1, 1, 1, 0),     # one tap
])
def test_no_stacked_schedules(args):
    p = nt.conv_problem(*args)
    assert not [s for s in nt.nk_enumerate_schedules(p) if s[2] == 64 * p.kh and p.kh >= 2 and p.kw >= 2]


def test_stacked_schedules_for_deep_layers():
    """C = 512: weights stream through a ring; still a legal schedule."""
    p = nt.conv_problem(8, 7, 7, 512, 512, 3, 3, 1, 1)
    assert _stacked(p)
