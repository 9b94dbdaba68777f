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
    # one accumulator buffer, 1-4 window slots; two buffers, 2-8 slots
    assert got == [(128, 64, 192, 1, st, 1) for st in (1, 2, 3, 4)] + [(256, 64, 192, 1, st, 1) for st in range(2, 9)]
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


@pytest.mark.parametrize("batch", [1, 8, 32])
def test_default_schedules_for_the_resnet_stack(batch):
    """Built-in choice per layer: stacked kernel rows for the stride-1 3x3
    layers (except batch-1 layers with C > 128, whose few tiles go to the
    per-tap kernel with split-K) -- two accumulator buffers on one CTA per
    SM once there are 4 tiles per SM, else one buffer on two CTAs -- and
    128 x 64 per-tap tiles everywhere else."""
    from paper_2307_16080_gb300 import synth
    for L in synth.resnet_stack(batch):
        p = nt.conv_problem(L["N"], L["H"], L["W"], L["C"], L["F"], L["KH"], L["KW"], L["stride"], L["pad"])
        s = nt.nk_default_schedule(p)
        assert s in nt.nk_enumerate_schedules(p), (L, s)
        stackable = L["stride"] == 1 and L["KH"] == 3
        if stackable and not (batch == 1 and L["C"] > 128):
            assert s[0] in (128, 256) and s[1:3] == (64, 192) and s[5] == 1, (L, s)
            tiles = nt.nk_conv_window_tile(L["N"], L["H"], L["W"], L["C"], L["F"], 3, 3, (1, 1), (1, 1, 1, 1),
                                           s)["tiles"] * ((L["F"] + 63) // 64)
            assert (s[0] == 256) == (tiles >= 4 * 152), (L, s, tiles)
        else:
            assert s[:3] == (128, 64, 64), (L, s)


def _default_regret(path):
    """Regret of the live built-in default rule on a stored corpus of GPU
    timings (every legal schedule of each problem was timed): mean per
    (op, precision), and per batch over the conv problems."""
    import numpy as np
    from paper_2307_16080_gb300 import costmodel
    c = costmodel.load_corpus(path)
    per, stack = {}, {}
    for i, pr in enumerate(c["problems"]):
        rows = np.nonzero(c["pid"] == i)[0]
        ms = {tuple(int(v) for v in c["sched"][j]): float(np.exp(c["y"][j])) for j in rows}
        d = tuple(nt.nk_default_schedule(nt.nk_problem(*[int(v) for v in pr])))
        assert d in ms, d
        best = min(ms.values())
        per.setdefault((int(pr[0]), int(pr[1])), []).append(ms[d] / best - 1)
        if int(pr[0]) == nt.NK_OP_CONV2D:
            b = stack.setdefault(int(pr[5]), [0.0, 0.0])   # problem field n: the batch
            b[0] += best
            b[1] += ms[d]
    return {k: float(np.mean(v)) for k, v in per.items()}, {k: v[1] / v[0] - 1 for k, v in stack.items()}


def test_default_regret_on_stored_corpora():
    """The default rules were fitted to these corpora; this pins their
    quality, so a change that loses more fails here first."""
    import os
    from paper_2307_16080_gb300 import costmodel
    tr = os.path.join(costmodel.MODEL_DIR, "corpus_train.npz")
    ho = os.path.join(costmodel.MODEL_DIR, "corpus_heldout.npz")
    if not (os.path.exists(tr) and os.path.exists(ho)):
        pytest.skip("no stored corpora")
    mean_tr, _ = _default_regret(tr)
    mean_ho, stack = _default_regret(ho)
    conv, mm = nt.NK_OP_CONV2D, nt.NK_OP_MATMUL
    bf16, bf16x3, fp8 = (nt.nk.PREC[k] for k in ("bf16", "bf16x3", "fp8"))
    assert mean_tr[(conv, bf16)] <= 0.08, mean_tr
    assert mean_tr[(mm, bf16)] <= 0.12 and mean_tr[(mm, fp8)] <= 0.08, mean_tr
    assert mean_tr[(mm, bf16x3)] <= 0.20, mean_tr
    assert mean_ho[(conv, bf16)] <= 0.03, mean_ho
    assert all(r <= 0.05 for r in stack.values()), stack


def test_defaults_are_legal_schedules_everywhere():
    """Every built-in default lies in the problem's legal schedule space:
    matmuls from one row to 8192 (ragged and tiny included) in every
    tensor-core precision, and seeded random convolutions."""
    from paper_2307_16080_gb300 import synth
    sizes = [1, 16, 100, 128, 300, 1000, 2048, 8192]
    for M, N, K in zip(sizes * 3, sizes[::-1] * 3, [16, 64, 700, 4096, 8192, 1, 33, 256] * 3):
        for prec in ("bf16", "fp8", "bf16x3"):
            p = nt.matmul_problem(M, N, K, prec)
            assert nt.nk_default_schedule(p) in nt.nk_enumerate_schedules(p), (M, N, K, prec)
    u = synth.uniform01(95, 0, 6 * 40)
    for g in range(40):
        r = u[6 * g: 6 * g + 6]
        k = (1, 3, 5)[int(r[0] * 3)]
        s = 1 + int(r[1] * 2)
        h = k + int(r[2] * 60)
        n, c, f = 1 + int(r[3] * 32), 8 * (1 + int(r[4] * 64)), 8 * (1 + int(r[5] * 64))
        for prec in ("bf16", "fp8"):
            p = nt.conv_problem(n, h, h, c, f, k, k, s, k // 2, prec)
            assert nt.nk_default_schedule(p) in nt.nk_enumerate_schedules(p), (n, h, c, f, k, s, prec)


def test_headline_gemms_keep_the_wide_pair_tile():
    for prec, tk in (("bf16", 64), ("fp8", 128)):
        for n in (4096, 8192):
            assert nt.nk_default_schedule(nt.matmul_problem(n, n, n, prec)) == (256, 512, tk, 2, 4, 1)


def test_no_tma_load_is_multicast():
    """Every TMA load of the library lands in the issuing CTA's own shared
    memory (a CTA pair's loads signal the even CTA's barrier, but each CTA
    copies its own operand halves): no cp.async.bulk instruction in the
    sources carries a .multicast qualifier."""
    import glob
    import os
    import re
    root = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "paper_2307_16080_gb300", "csrc")
    srcs = glob.glob(os.path.join(root, "*.cu")) + glob.glob(os.path.join(root, "*.cuh"))
    assert srcs
    for path in srcs:
        text = open(path).read()
        # an asm string may span several adjacent literals: join each asm block
        for block in re.findall(r"asm\s+volatile\s*\((.*?)\);", text, flags=re.S):
            if "cp.async.bulk" in block:
                assert "multicast" not in block, path


@pytest.mark.parametrize("prob", [
    ("mm", 8192, 8192, 8192, "bf16"), ("mm", 300, 520, 700, "bf16"), ("mm", 4096, 4096, 4096, "fp8"),
    ("mm", 1024, 1024, 4096, "bf16x3"), ("conv", 8, 56, 56, 64, 64, 3, 3, 1, 1), ("conv", 32, 14, 14, 256, 512, 3, 3, 2, 1),
])
def test_cluster_two_is_always_a_cta_pair(prob):
    """cluster 2 only with tile_m 256 (a CTA pair issuing 2-SM MMAs); E4M3
    convolutions use one CTA per tile."""
    precs = ["bf16", "fp8"] if prob[0] == "conv" else [prob[-1]]
    for prec in precs:
        if prob[0] == "mm":
            p = nt.matmul_problem(prob[1], prob[2], prob[3], prec)
        else:
            p = nt.conv_problem(*prob[1:], precision=prec)
        scheds = nt.nk_enumerate_schedules(p)
        assert scheds
        for s in scheds:
            if s[3] == 2:
                assert s[0] == 256, s
                assert not (prob[0] == "conv" and prec == "fp8"), s


@pytest.mark.parametrize("name", ["corpus_train.npz", "corpus_heldout.npz", "corpus_heldout2.npz"])
def test_stored_corpora_cover_todays_schedule_space(name):
    """Each stored corpus timed exactly the legal schedules the library
    enumerates today for each of its problems (a change of the schedule space
    makes the corpora stale and fails here)."""
    import os
    import numpy as np
    from paper_2307_16080_gb300 import costmodel
    path = os.path.join(costmodel.MODEL_DIR, name)
    if not os.path.exists(path):
        pytest.skip("no stored corpus")
    c = costmodel.load_corpus(path)
    for i, pr in enumerate(c["problems"]):
        rows = np.nonzero(c["pid"] == i)[0]
        stored = {tuple(int(v) for v in c["sched"][j]) for j in rows}
        live = set(nt.nk_enumerate_schedules(nt.nk_problem(*[int(v) for v in pr])))
        assert stored == live, (name, i, len(stored), len(live))


def test_heldout2_shares_no_problem_with_training():
    from paper_2307_16080_gb300 import costmodel
    train = {tuple(costmodel.problem_dict(p).values()) for p in costmodel.training_problems()}
    h2 = [tuple(costmodel.problem_dict(p).values()) for p in costmodel.heldout2_problems()]
    assert h2 and not (set(h2) & train)
