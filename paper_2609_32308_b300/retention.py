"""Retention-count predictor: labels from the exact DP, training, evaluation.

The labels are what the exact fill itself retains: for every codon position k
of a protein and span band s (band = floor(log2 span) - 2 clamped to 0..7),
the number of multiloop candidates (Eq. candidates) whose right endpoint lies
in codon k and whose span is in band s.  The network sees only the protein,
its codon weights and lambda, and learns log1p of those counts.  A trained
predictor presizes the candidate lists of a plan (``Plan(..., predictor=)``);
the exact test B(c,b) < P_S(c,b) still decides every candidate, and a list
that outgrows its room makes the plan repeat that design with worst-case room.

Everything here drives the library's own kernels (fill, retention histogram,
BF16/FP32 forward, backward and Adam); nothing is computed on the host except
batching and log1p of integer counts.

Command line (trains on the GPU, writes the FP32 parameters as .npy):

    python -m paper_2609_32308_b300.retention --out weights.npy
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import Energy, Plan, Predictor, inputs

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "data", "retention_predictor.npy")
BANDS = 8


def corpus(count: int, seed: int, lo: int = 50, hi: int = 2000, mu: float = math.log(400.0),
           sigma: float = 0.8):
    """Seeded synthetic proteins: log-normal lengths clipped to [lo, hi],
    amino acids from the Swiss-Prot composition, per-protein codon weights,
    lambda drawn from {0, 4}."""
    lengths = inputs.lengths_log_normal(count, mu, sigma, lo, hi, seed)
    return inputs.protein_batch(lengths, seed, lambdas=(0.0, 4.0))


def _chunks(items, max_nt_sq: float):
    """Group items (sorted longest first) so that sum of n^2 stays bounded."""
    order = sorted(range(len(items)), key=lambda k: -len(items[k][0]))
    out, cur, acc = [], [], 0.0
    for k in order:
        n = 3.0 * len(items[k][0])
        if cur and acc + n * n > max_nt_sq:
            out.append(cur)
            cur, acc = [], 0.0
        cur.append(k)
        acc += n * n
    if cur:
        out.append(cur)
    return out


def retention_labels(energy: Energy, items, max_nt_sq: float = 1.5e8):
    """Run the exact DP on every item and return its retention counts
    (A x 8 int32 arrays, in item order)."""
    counts = [None] * len(items)
    for grp in _chunks(items, max_nt_sq):
        sub = [items[k] for k in grp]
        plan = Plan(energy, [p for p, _, _ in sub], np.stack([w for _, w, _ in sub]),
                    [lam for _, _, lam in sub])
        try:
            plan.run()
            res = plan.results()
            for j, k in enumerate(grp):
                if res[j]["status"] != 0:
                    raise RuntimeError(f"design {k} failed: status {res[j]['status']}")
                counts[k] = plan.retention(j)
        finally:
            plan.free()
    return counts


def batch_arrays(items, counts, idx):
    """Padded features / targets / lengths for the items `idx`."""
    L = max(len(items[k][0]) for k in idx)
    B = len(idx)
    f = np.zeros((B, L, 32), dtype=np.float32)
    t = np.zeros((B, L, BANDS), dtype=np.float32)
    ln = np.zeros(B, dtype=np.int32)
    for b, k in enumerate(idx):
        p, w, lam = items[k]
        A = len(p)
        f[b, :A] = Predictor.features(p, w, lam)
        if counts is not None:
            t[b, :A] = np.log1p(counts[k].astype(np.float64))
        ln[b] = A
    return f, t, ln


def train(pred: Predictor, items, counts, epochs: int = 40, batch: int = 16, lr: float = 2e-3,
          seed: int = 0, log=None):
    """Adam on the mean squared log1p error; batches of similar length."""
    rng = np.random.default_rng(seed)
    order = sorted(range(len(items)), key=lambda k: len(items[k][0]))
    groups = [order[i:i + batch] for i in range(0, len(order), batch)]
    cache = [batch_arrays(items, counts, g) for g in groups]
    history = []
    for ep in range(epochs):
        step_lr = lr * 0.5 * (1.0 + math.cos(math.pi * ep / max(1, epochs)))
        tot = 0.0
        for gi in rng.permutation(len(groups)):
            f, t, ln = cache[gi]
            tot += pred.train_step(f, t, ln, step_lr) * len(groups[gi])
        history.append(tot / len(items))
        if log:
            log(f"epoch {ep:3d} lr {step_lr:.2e} loss {history[-1]:.4f}")
    return history


def predict_totals(pred: Predictor, items, idx):
    """Predicted retained candidates per codon (summed over bands)."""
    f, _, ln = batch_arrays(items, None, idx)
    y = pred.forward(f, ln)
    return [np.expm1(np.maximum(y[b, :ln[b]], 0.0)).sum(axis=1) for b in range(len(idx))]


def load(path: str = DEFAULT_WEIGHTS) -> Predictor:
    """A predictor with trained parameters (the shipped ones by default)."""
    pred = Predictor()
    pred.set_params(np.load(path))
    return pred


def evaluate(energy: Energy, pred: Predictor, items, margin: float = 2.0,
             max_nt_sq: float = 1.5e8, streams: int = 1):
    """Run every item with the plain schedule (worst-case room, one launch
    sequence) and with the predicted one (predicted room, designs over
    `streams` concurrent streams longest predicted work first); return the
    reserved room, the retained candidates, the regrow count, the device
    bytes and wall times of both, and whether every design is identical."""
    room_worst = room_pred = regrows = retained = 0
    bytes_worst = bytes_pred = 0
    t_plain = t_pred = 0.0
    identical = True
    for grp in _chunks(items, max_nt_sq):
        sub = [items[k] for k in grp]
        args = ([p for p, _, _ in sub], np.stack([w for _, w, _ in sub]),
                [lam for _, _, lam in sub])
        t0 = time.perf_counter()
        plain = Plan(energy, *args)
        try:
            plain.run()
            r0 = plain.results()
            t_plain += time.perf_counter() - t0
            room_worst += plain.candidate_room
            bytes_worst += plain.device_bytes
        finally:
            plain.free()
        t0 = time.perf_counter()
        pres = Plan(energy, *args, predictor=pred, margin=margin)
        try:
            pres.streams = streams
            pres.run()
            r1 = pres.results()
            t_pred += time.perf_counter() - t0
            room_pred += pres.candidate_room
            bytes_pred += pres.device_bytes
        finally:
            pres.free()
        for a, b in zip(r0, r1):
            regrows += b["regrows"]
            retained += a["Z"]
            for key in ("status", "mrna", "structure", "energy", "objective_fx", "Z",
                        "retained_cells"):
                if a[key] != b[key]:
                    identical = False
    return {"room_worst": room_worst, "room_pred": room_pred, "retained": retained,
            "regrows": regrows, "designs": len(items), "identical": identical,
            "room_ratio": room_pred / max(1, room_worst),
            "device_bytes_worst": bytes_worst, "device_bytes_pred": bytes_pred,
            "wall_s_plain": t_plain, "wall_s_pred": t_pred}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--train", type=int, default=6000)
    ap.add_argument("--held-out", type=int, default=1600)
    ap.add_argument("--hi", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--margin", type=float, default=2.0)
    ap.add_argument("--energy-seed", type=int, default=1)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--report", default=None, help="write a JSON summary here")
    ap.add_argument("--eval-only", action="store_true",
                    help="evaluate the parameters in --out on the held-out designs again "
                         "(no labels, no training); keeps the training figures of --report")
    args = ap.parse_args()
    energy = Energy(None, args.energy_seed)  # the library's seeded synthetic set
    items = corpus(args.train + args.held_out, args.seed, hi=args.hi)
    tr, ho = items[:args.train], items[args.train:]
    if args.eval_only:
        prev = {}
        if args.report and os.path.exists(args.report):
            with open(args.report) as fh:
                prev = json.load(fh)
        t0 = time.time()
        prev.update(evaluate(energy, load(args.out), ho, margin=args.margin))
        prev.update({"eval_s": time.time() - t0, "margin": args.margin})
        print(json.dumps(prev))
        if args.report:
            with open(args.report, "w") as fh:
                json.dump(prev, fh, indent=1)
        return
    t0 = time.time()
    counts = retention_labels(energy, tr)
    t_label = time.time() - t0
    pred = Predictor(seed=args.seed)
    t0 = time.time()
    hist = train(pred, tr, counts, epochs=args.epochs, log=print)
    t_train = time.time() - t0
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.save(args.out, pred.params())
    t0 = time.time()
    ev = evaluate(energy, pred, ho, margin=args.margin)
    ev.update({"label_s": t_label, "train_s": t_train, "eval_s": time.time() - t0,
               "train_designs": len(tr), "final_loss": hist[-1], "first_loss": hist[0],
               "margin": args.margin})
    print(json.dumps(ev))
    if args.report:
        with open(args.report, "w") as fh:
            json.dump(ev, fh, indent=1)


if __name__ == "__main__":
    main()
