"""The learned tile-cost model: measurement corpus, GPU training, regret.

The paper tunes tile sizes and unroll factors of its kernel by black-box
search, timing every point it tries (Sec. 4.3).  This module replaces most of
that timing with a model:

  collect   time every legal schedule of a set of training problems on the GPU
            (nk_time_schedule) -> corpus of (features, ln ms)
  train     fit the 16 -> 128 -> 128 -> 1 GELU MLP to standardised ln ms with
            MSE + Adam, on the GPU, with the library's own kernels
            (nk_mlp_grad / nk_mlp_adam)
  evaluate  on held-out problems: the 20-layer ResNet-style conv stack at
            batch 1, 8, 32, and a second set that neither the model nor the
            built-in default rule was fitted with (a 20-layer conv stack of
            other widths, spatial sizes and strides, and 20 matmuls drawn
            like the grouped-GEMM workload): regret = t(best of the model's
            top-k) / t(exhaustive best) - 1, beside random-k, the built-in
            default and the (1+1) evolution strategy given k timings

Python here only orders the calls; every measurement and every training
step runs in libnk.  Usage:
  python -m paper_2307_16080_gb300.costmodel all --out DIR
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import nk_tune as nt
from . import synth

MODEL_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "model")
MODEL_PATH = os.path.join(MODEL_DIR, "cost_mlp.npz")


def _r64(x):
    return int(max(64, round(x / 64) * 64))


def training_problems(seed: int = synth.SEED_COSTMODEL):
    """~250 matmul and conv problems (none of them a held-out ResNet layer)."""
    probs = []
    u = synth.uniform01(seed, 500, 4096)
    k = 0

    def nxt():
        nonlocal k
        k += 1
        return u[k - 1]

    precs = ["bf16", "fp8", "bf16x3"]
    for i in range(150):
        prec = precs[i % 3]
        hi = 8192 if prec != "bf16x3" else 4096
        M, N, K = (_r64(math.exp(math.log(128) + (math.log(hi) - math.log(128)) * nxt())) for _ in range(3))
        probs.append(nt.matmul_problem(M, N, K, prec))
    resnet = {(L["H"], L["C"], L["F"], L["KH"], L["stride"]) for b in (1, 8, 32) for L in synth.resnet_stack(b)}
    chans = [16, 32, 48, 64, 96, 128, 192, 256, 384]
    sizes = [8, 12, 16, 20, 24, 32, 40, 48, 64]
    while len(probs) < 250:
        n = [1, 2, 4, 8, 16][int(nxt() * 5)]
        h = sizes[int(nxt() * len(sizes))]
        c = chans[int(nxt() * len(chans))]
        f = chans[int(nxt() * len(chans))]
        kk = [1, 3, 3, 5][int(nxt() * 4)]
        st = 1 if nxt() < 0.6 else 2
        if (h, c, f, kk, st) in resnet:
            continue
        probs.append(nt.conv_problem(n, h, h, c, f, kk, kk, st, kk // 2))
    return probs


def heldout_problems():
    out = []
    for b in (1, 8, 32):
        for L in synth.resnet_stack(b):
            out.append(nt.conv_problem(L["N"], L["H"], L["W"], L["C"], L["F"], L["KH"], L["KW"], L["stride"],
                                       L["pad"]))
    return out


def heldout2_problems(seed: int = synth.SEED_COSTMODEL + 100):
    """A second held-out set, fitted by nothing: 20 conv layers of a stack
    with other channel counts (48 -> 384), spatial sizes (60 -> 8) and a
    batch of 4 and 16, and 20 BF16 matmuls drawn like the grouped workload
    (M, N, K log-uniform in [32, 2048], multiples of 16).  Problems that
    coincide with a training problem are dropped."""
    train = {tuple(problem_dict(p).values()) for p in training_problems()}
    stack = []
    for n in (4, 16):
        cin, h = 48, 60
        for cout, st in ((48, 1), (96, 2), (96, 1), (192, 2), (192, 1), (384, 2), (384, 1)):
            if st == 2:
                stack.append(nt.conv_problem(n, h, h, cin, cout, 3, 3, 2, 1))
                h = (h + 2 - 3) // 2 + 1
            else:
                stack.append(nt.conv_problem(n, h, h, cin, cout, 3, 3, 1, 1))
            cin = cout
        stack.append(nt.conv_problem(n, h, h, cin, cin, 1, 1, 1, 0))
        stack.append(nt.conv_problem(n, h, h, cin, 2 * cin, 1, 1, 1, 0))
        stack.append(nt.conv_problem(n, 2 * h, 2 * h, cin // 2, cin, 1, 1, 2, 0))
    shapes = synth.grouped_problems(20, seed)
    mm = [nt.matmul_problem(int(M), int(N), int(K), "bf16") for M, N, K in shapes]
    out = []
    for p in stack + mm:
        if tuple(problem_dict(p).values()) not in train:
            out.append(p)
    return out


def problem_dict(p):
    return {f: int(getattr(p, f)) for f, _ in nt.nk_problem._fields_}


def collect(problems, reps: int = 3, log=None, evolution_k: int = 0):
    """Time every legal schedule of every problem.  Returns a corpus dict.
    evolution_k > 0 also runs the library's (1+1) evolution strategy with
    that many timings per problem and keeps its pick ("es_pick"), so that
    its regret is scored on the same exhaustive timings as the rest."""
    feats, y, pid, sched, es = [], [], [], [], []
    for i, p in enumerate(problems):
        cands = nt.nk_enumerate_schedules(p)
        F = nt.nk_schedule_features(p, cands)
        for s, f in zip(cands, F):
            ms = nt.nk_time_schedule(p, s, reps)
            feats.append(f)
            y.append(math.log(max(ms, 1e-6)))
            pid.append(i)
            sched.append(s)
        if evolution_k > 0:
            pick, _ = nt.nk_tune(p, nt.NK_TUNE_EVOLUTION, topk=evolution_k, reps=reps)
            es.append(pick)
        if log:
            log(f"problem {i + 1}/{len(problems)}: {len(cands)} schedules")
    nt.nk_tune_release()
    defaults = [nt.nk_default_schedule(p) for p in problems]
    c = {"X": np.asarray(feats, np.float32), "y": np.asarray(y, np.float64), "pid": np.asarray(pid),
         "sched": np.asarray(sched, np.int32), "problems": np.asarray([list(problem_dict(p).values())
                                                                       for p in problems], np.int32),
         "defaults": np.asarray(defaults, np.int32)}
    if evolution_k > 0:
        c["es_pick"] = np.asarray(es, np.int32)
    return c


def init_params(seed: int = 7) -> np.ndarray:
    """He-style initial weights from the seeded generator, zero biases."""
    n = nt.nk_mlp_param_count()
    p = np.zeros(n, np.float32)
    o = 0
    for i, (rows, cols) in enumerate(((128, 16), (128, 128), (1, 128))):
        w = synth.normal(seed, i, (rows * cols,), sigma=math.sqrt(2.0 / cols))
        p[o:o + rows * cols] = w
        o += rows * cols + rows
    return p


def train(X: np.ndarray, y: np.ndarray, epochs: int = 400, batch: int = 1024, lr: float = 2e-3,
          seed: int = 11, log=None):
    """Fit the MLP on the GPU.  Returns (params, y_mean, y_std, loss history)."""
    dev = torch.device("cuda")
    ym, ys = float(np.mean(y)), float(np.std(y) + 1e-12)
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).to(dev)
    td = torch.from_numpy(((y - ym) / ys).astype(np.float32)).to(dev)
    P = torch.from_numpy(init_params()).to(dev)
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    g = torch.zeros_like(P)
    loss = torch.zeros(1, device=dev)
    ws = torch.empty(nt.nk_mlp_workspace_size(batch), dtype=torch.uint8, device=dev)
    n = X.shape[0]
    hist = []
    step = 0
    for ep in range(epochs):
        perm = np.argsort(synth.uniform01(seed, ep, n))
        idx = torch.from_numpy(perm).to(dev)
        tot = 0.0
        for b0 in range(0, n - batch + 1 if n >= batch else 1, batch):
            sel = idx[b0:b0 + batch]
            xb, tb = Xd[sel].contiguous(), td[sel].contiguous()
            step += 1
            nt.nk_mlp_grad(P, xb, tb, g, loss, ws)
            rate = lr * (0.5 * (1 + math.cos(math.pi * ep / epochs)) * 0.95 + 0.05)
            nt.nk_mlp_adam(P, g, m, v, step, lr=rate)
            tot += float(loss.item()) if b0 == 0 else 0.0
        hist.append(tot)
        if log and (ep % 50 == 0 or ep == epochs - 1):
            log(f"epoch {ep}: loss {tot:.4f}")
    return P.cpu().numpy(), ym, ys, hist


def predict(params: np.ndarray, X: np.ndarray) -> np.ndarray:
    dev = torch.device("cuda")
    P = torch.from_numpy(params.astype(np.float32)).to(dev)
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).to(dev)
    return nt.nk_mlp_forward(P, Xd).cpu().numpy()


def predicted_ms(params: np.ndarray, y_mean: float, y_std: float, problems, schedules=None) -> np.ndarray:
    """The model's predicted time (ms) of each problem under its schedule
    (default: the built-in one), e.g. as LPT costs for spreading a grouped
    GEMM's groups over GPUs."""
    scheds = schedules or [nt.nk_default_schedule(p) for p in problems]
    X = np.concatenate([nt.nk_schedule_features(p, [s]) for p, s in zip(problems, scheds)]).astype(np.float32)
    return np.exp(predict(params, X) * y_std + y_mean)


def regrets(corpus, pred: np.ndarray, k: int = 5, seed: int = 13):
    """Per problem: model top-k, random-k and default regret vs the exhaustive best."""
    out = []
    pid = corpus["pid"]
    for i in range(int(pid.max()) + 1):
        rows = np.nonzero(pid == i)[0]
        ms = np.exp(corpus["y"][rows])
        best = ms.min()
        top = rows[np.argsort(pred[rows], kind="stable")[:k]]
        model = np.exp(corpus["y"][top]).min()
        r = synth.uniform01(seed, i, len(rows))
        rnd = np.exp(corpus["y"][rows[np.argsort(r)[:k]]]).min()
        d = tuple(corpus["defaults"][i])
        drow = [j for j in rows if tuple(corpus["sched"][j]) == d]
        dms = np.exp(corpus["y"][drow[0]]) if drow else float("nan")
        r = {"model": model / best - 1, "random": rnd / best - 1, "default": dms / best - 1,
             "best_ms": float(best), "candidates": int(len(rows))}
        if "es_pick" in corpus:
            e = tuple(corpus["es_pick"][i])
            erow = [j for j in rows if tuple(corpus["sched"][j]) == e]
            r["evolution"] = np.exp(corpus["y"][erow[0]]) / best - 1 if erow else float("nan")
        out.append(r)
    return out


def summarise(rs):
    keys = ("model", "random", "default") + (("evolution",) if rs and "evolution" in rs[0] else ())
    s = {f"mean_{k}_regret": float(np.nanmean([r[k] for r in rs])) for k in keys}
    s.update({f"max_{k}_regret": float(np.nanmax([r[k] for r in rs])) for k in keys})
    tot_best = sum(r["best_ms"] for r in rs)
    s.update({f"stack_{k}_regret": float(sum(r["best_ms"] * (1 + r[k]) for r in rs) / tot_best - 1) for k in keys})
    s["problems"] = len(rs)
    return s


def save_model(path, params, ym, ys):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez_compressed(path, params=params.astype(np.float32), y_mean=ym, y_std=ys, features=16)


def load_model(path=MODEL_PATH):
    z = np.load(path)
    return z["params"], float(z["y_mean"]), float(z["y_std"])


def save_corpus(path, c):
    np.savez_compressed(path, **c)


def load_corpus(path):
    z = np.load(path)
    return {k: z[k] for k in z.files}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["collect", "train", "eval", "all", "defaults"])
    ap.add_argument("--out", default=MODEL_DIR)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--k", type=int, default=5)
    a = ap.parse_args()
    os.makedirs(a.out, exist_ok=True)
    log = lambda m: print(m, flush=True)  # noqa: E731
    t0 = time.time()
    tr_path = os.path.join(a.out, "corpus_train.npz")
    ho_path = os.path.join(a.out, "corpus_heldout.npz")
    h2_path = os.path.join(a.out, "corpus_heldout2.npz")
    evals = (("train", tr_path), ("heldout_resnet_stack", ho_path), ("heldout2_unfitted", h2_path))
    if a.cmd in ("collect", "all"):
        save_corpus(tr_path, collect(training_problems(), a.reps, log))
        save_corpus(ho_path, collect(heldout_problems(), a.reps, log, evolution_k=a.k))
        save_corpus(h2_path, collect(heldout2_problems(), a.reps, log, evolution_k=a.k))
        log(f"collected in {time.time() - t0:.0f} s")
    if a.cmd == "defaults":
        # After a change of the built-in default rule: re-derive each stored
        # problem's default schedule (host logic, no GPU) so that the default
        # regret of `eval` scores the current rule on the stored timings.
        for path in (tr_path, ho_path, h2_path):
            if not os.path.exists(path):
                continue
            c = load_corpus(path)
            c["defaults"] = np.asarray([nt.nk_default_schedule(nt.nk_problem(*[int(v) for v in pr]))
                                        for pr in c["problems"]], np.int32)
            save_corpus(path, c)
            log(f"defaults re-derived for {len(c['problems'])} problems in {path}")
        # The default columns of regret.json need no model (no GPU): rescore
        # them on the stored timings and keep the model and random columns.
        rj = os.path.join(a.out, "regret.json")
        if os.path.exists(rj):
            with open(rj) as f:
                res = json.load(f)
            for name, path in evals:
                if name not in res or not os.path.exists(path):
                    continue
                c = load_corpus(path)
                fresh = summarise(regrets(c, np.zeros(len(c["y"])), a.k))
                res[name].update({k: v for k, v in fresh.items() if "default" in k})
            with open(rj, "w") as f:
                json.dump(res, f, indent=1)
            log(f"default regret rescored in {rj}")
    if a.cmd in ("train", "all"):
        c = load_corpus(tr_path)
        P, ym, ys, hist = train(c["X"], c["y"], a.epochs, log=log)
        save_model(os.path.join(a.out, "cost_mlp.npz"), P, ym, ys)
        log(f"trained: final loss {hist[-1]:.4f}")
    if a.cmd in ("eval", "all"):
        P, ym, ys = load_model(os.path.join(a.out, "cost_mlp.npz"))
        res = {}
        for name, path in evals:
            if not os.path.exists(path):
                continue
            c = load_corpus(path)
            res[name] = summarise(regrets(c, predict(P, c["X"]), a.k))
        res["k"] = a.k
        res["timing"] = nt.timing_method()
        print(json.dumps(res, indent=1), flush=True)
        with open(os.path.join(a.out, "regret.json"), "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
