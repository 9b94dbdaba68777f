"""Host-side geometry of the window convolution tiles (no GPU).

The window kernels read every A-operand row from one shared-memory window
per tile; the stacked variant also adds, for output row m, accumulator rows
m + kw * dw with warp shuffles.  Neither has a bounds check in the hot loop,
so these invariants carry its memory safety, and here they are checked on
the tile the library actually chooses (nk_conv_window_tile) for every valid
output of a tile:

- GEMM row m = (b * WR + y) * P + x lies in the tile's chains * 128 rows;
- every A row a tap reads lies inside the loaded box (rows) and the
  reserved slot (slot_rows), and is window pixel (b, y + kh*dh, x + kw*dw);
- stacked: row m + kw*dw lies in the same warp (32 rows) and in the MMA's
  first 128 rows, so the shuffle reads a row the MMA computed;
- stacked whole-width tiles (one column tile, Q = OW > P - (KW-1)*dw, only
  for single-buffered schedules): a shift that leaves the window row
  (x + kw*dw >= P) is left out by the epilogue, and exactly then the input
  column it stands for is >= W, zero padding, so the result is exact.
"""
import itertools

import pytest

from paper_2307_16080_gb300 import synth

nt = pytest.importorskip("paper_2307_16080_gb300.nk_tune")


def _check(n, h, w, c, f, kh, kw, dl, pad, sched):
    try:
        t = nt.nk_conv_window_tile(n, h, w, c, f, kh, kw, dl, pad, sched)
    except Exception:
        return None   # not a legal window schedule for this geometry
    P, Q, R, NB, WR = t["P"], t["Q"], t["R"], t["NB"], t["WR"]
    stk, rows, slot = t["stk"], t["rows"], t["slot_rows"]
    ow = w + pad[2] + pad[3] - (kw - 1) * dl[1]
    assert rows == NB * WR * P and slot >= rows
    assert R + (kh - 1) * dl[0] == WR
    wrap = Q + (kw - 1) * dl[1] != P
    if wrap:   # whole-width stacked tile
        assert stk > 1 and sched[0] == 128, (t, sched)
        assert Q == ow <= P and P - pad[2] >= w and Q + (kw - 1) * dl[1] > P, t
    if stk > 1:
        assert stk == kw and P in (8, 16, 32) and t["chains"] == 1
    for b, y, x in itertools.product(range(NB), range(R), range(Q)):
        m = (b * WR + y) * P + x
        assert m < 128 * t["chains"], (t, m)
        for j in range(kw):
            if stk > 1 and x + j * dl[1] >= P:
                # left out by the epilogue: the input column is right padding
                assert wrap and x + j * dl[1] - pad[2] >= w, (t, x, j)
                continue
            mm = m + j * dl[1] if stk > 1 else m
            if stk > 1:
                assert mm < 128 and mm // 32 == m // 32, (t, m, j)
            for i in range(kh):
                a = mm + i * dl[0] * P + (0 if stk > 1 else j * dl[1])
                assert a < rows and a < slot, (t, m, i, j)
                off = a - b * WR * P
                assert (off // P, off % P) == (y + i * dl[0], x + j * dl[1]), (t, m, i, j)
    return t


GEOMETRIES = [
    # N, H, W, C, F, KH, KW, dilation, pad
    (8, 56, 56, 64, 64, 3, 3, (1, 1), (1, 1, 1, 1)),
    (32, 28, 28, 128, 128, 3, 3, (1, 1), (1, 1, 1, 1)),
    (8, 14, 14, 256, 256, 3, 3, (1, 1), (1, 1, 1, 1)),
    (8, 7, 7, 512, 512, 3, 3, (1, 1), (1, 1, 1, 1)),
    (2, 13, 11, 16, 24, 3, 3, (1, 2), (1, 0, 2, 1)),
    (1, 12, 12, 5, 7, 3, 3, (1, 1), (0, 0, 0, 0)),
    (1, 20, 18, 32, 130, 3, 2, (2, 1), (2, 2, 1, 1)),
    (3, 9, 11, 40, 96, 3, 3, (1, 1), (1, 1, 1, 1)),
    (5, 7, 7, 64, 64, 3, 3, (1, 1), (1, 1, 1, 1)),
    (1, 6, 140, 64, 64, 3, 3, (1, 1), (1, 1, 1, 1)),
    (2, 17, 19, 64, 48, 4, 4, (1, 1), (1, 2, 1, 2)),
    (2, 17, 19, 64, 48, 2, 2, (1, 1), (0, 1, 0, 1)),
    (2, 21, 23, 64, 64, 3, 3, (2, 2), (2, 2, 2, 2)),
    (1, 20, 18, 32, 300, 5, 3, (2, 1), (2, 2, 1, 1)),
    # whole-width stacked tiles: 7 and 15 wide, dilated, asymmetric pads
    (32, 7, 7, 512, 512, 3, 3, (1, 1), (1, 1, 1, 1)),
    (3, 7, 7, 96, 130, 3, 3, (1, 1), (1, 1, 0, 2)),
    (2, 15, 15, 64, 48, 3, 3, (1, 1), (1, 1, 1, 1)),
    (2, 13, 13, 64, 64, 3, 3, (2, 2), (2, 2, 2, 2)),
    (4, 6, 7, 64, 64, 2, 2, (1, 1), (0, 1, 0, 1)),
    (2, 30, 31, 64, 64, 3, 3, (1, 1), (1, 1, 1, 1)),
]


def test_whole_width_tiles_are_chosen_where_they_save_tiles():
    t = nt.nk_conv_window_tile(32, 7, 7, 512, 512, 3, 3, (1, 1), (1, 1, 1, 1), (128, 64, 192, 1, 2, 1))
    assert (t["P"], t["Q"], t["NB"], t["tiles"]) == (8, 7, 2, 16)
    db = nt.nk_conv_window_tile(32, 7, 7, 512, 512, 3, 3, (1, 1), (1, 1, 1, 1), (256, 64, 192, 1, 2, 1))
    assert db["Q"] + 2 == db["P"]   # the double-buffered kernel never wraps
    # no whole-width tile when the left pad would leave input columns out
    t2 = nt.nk_conv_window_tile(2, 7, 7, 64, 64, 3, 3, (1, 1), (1, 1, 2, 0), (128, 64, 192, 1, 2, 1))
    assert t2["Q"] + 2 == t2["P"]


def _schedules(kh, kw):
    out = [(128, 64, 64 * kh, 1, st, 1) for st in (1, 2, 3, 4)]                     # stacked rows
    out += [(256, 64, 64 * kh, 1, st, 1) for st in (2, 4)]                           # double-buffered
    out += [(tm, tn, 64 * kh * kw, 1, st, 1) for tm in (128, 256, 512) for tn in (64, 128, 256)
            for st in (1, 2, 4)]                                                      # plain window
    return out


@pytest.mark.parametrize("geom", GEOMETRIES)
def test_window_tiles_stay_in_bounds(geom):
    n, h, w, c, f, kh, kw, dl, pad = geom
    legal = [t for t in (_check(n, h, w, c, f, kh, kw, dl, pad, s) for s in _schedules(kh, kw)) if t]
    assert legal, "no legal window schedule"
    if 2 <= kw <= 4 and kh >= 2:
        assert any(t["stk"] == kw for t in legal), "no stacked schedule"


def test_window_tiles_random_geometries():
    """Seeded random stride-1 geometries (extents, kernel, dilation, pads)."""
    u = synth.uniform01(94, 0, 8 * 64)
    for g in range(64):
        r = u[8 * g: 8 * g + 8]
        kh, kw = 1 + int(r[0] * 5), 1 + int(r[1] * 5)
        if kh * kw == 1:
            continue
        dh, dw = 1 + int(r[2] * 2), 1 + int(r[3] * 2)
        h, w = kh * dh + int(r[4] * 40), kw * dw + int(r[5] * 70)
        n, c, f = 1 + int(r[6] * 6), 8 * (1 + int(r[7] * 24)), 16 + int(r[0] * 300)
        pad = (int(r[1] * kh), int(r[2] * kh), int(r[3] * kw), int(r[4] * kw))
        for s in _schedules(kh, kw):
            _check(n, h, w, c, f, kh, kw, (dh, dw), pad, s)


def test_window_tile_rejects_non_window_schedules():
    with pytest.raises(Exception):
        nt.nk_conv_window_tile(8, 56, 56, 64, 64, 3, 3, (1, 1), (1, 1, 1, 1), (128, 64, 64, 1, 2, 1))
    with pytest.raises(Exception):
        nt.nk_conv_window_tile(8, 56, 56, 64, 64, 5, 5, (1, 1), (2, 2, 2, 2), (128, 64, 320, 1, 2, 1))
