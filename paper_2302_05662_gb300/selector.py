"""The learned selector: training, evaluation and the weight blob.

The paper trains multi-class classifiers that map sparsity features to the
best configuration (Section 5.4) on an 80/20 split of its dataset (Section
6.4).  Here the classifier is a 2-layer MLP (20 -> H -> K, ReLU) whose
classes are the points of sweep.label_space() (format x threads per block x
threads per row).  Labels come from the exhaustive sweep: every class is
scored by its measured time, and the training target puts weight on every
configuration within a few percent of the fastest one, so near-ties
(configurations within timing noise) are not treated as errors.

Inference runs on the device (spmv_select / spmv_selector_infer, one fused
kernel); this module only trains offline with PyTorch on the CPU and writes
the float32 blob that spmv_selector_load reads.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from . import binding as B

PKG = os.path.dirname(os.path.abspath(__file__))
DEFAULT_BLOB = os.path.join(PKG, "selector_gb300.f32")
# the exhaustive-sweep records the committed selector was trained on
DEFAULT_DATA = os.path.join(PKG, "data", "sweep_gb300_f64.jsonl.gz")
MAGIC, VERSION = 2302.0, 1.0
CFG_FIELDS = ("format", "threads_per_block", "threads_per_row", "unroll", "regcap", "carveout",
              "bsr_block", "hyb_ell_width")
# features entering the network as log1p(value) (indices into the 20)
LOG_IDX = (0, 1, 3, 4, 5, 6, 7, 8, 9, 14, 15)


def full_config(d: dict) -> list:
    """The 8 spmv_config fields of a (partial) label dict; unset fields stay
    0 (the library's per-format default) except carveout -1 (driver default)."""
    base = {"format": 0, "threads_per_block": 256, "threads_per_row": 0, "unroll": 0, "regcap": 0,
            "carveout": -1, "bsr_block": 0, "hyb_ell_width": 0}
    base.update(d)
    return [int(base[k]) for k in CFG_FIELDS]


def make_blob(mu, sigma, W1, b1, W2, b2, labels) -> np.ndarray:
    W1 = np.asarray(W1, np.float32)
    W2 = np.asarray(W2, np.float32)
    H, F = W1.shape
    K = W2.shape[0]
    parts = [np.array([MAGIC, VERSION, F, H, K], np.float32), np.asarray(mu, np.float32),
             np.asarray(sigma, np.float32), W1.reshape(-1), np.asarray(b1, np.float32), W2.reshape(-1),
             np.asarray(b2, np.float32), np.array([full_config(l) for l in labels], np.float32).reshape(-1)]
    return np.concatenate(parts)


def parse_blob(blob) -> dict:
    b = np.asarray(blob, np.float32)
    assert b[0] == MAGIC and b[1] == VERSION
    F, H, K = int(b[2]), int(b[3]), int(b[4])
    o = 5
    def take(n):
        nonlocal o
        v = b[o:o + n]
        o += n
        return v
    mu, sigma = take(F), take(F)
    W1 = take(H * F).reshape(H, F)
    b1 = take(H)
    W2 = take(K * H).reshape(K, H)
    b2 = take(K)
    labels = take(K * 8).reshape(K, 8).astype(np.int64)
    assert o == b.size
    return dict(F=F, H=H, K=K, mu=mu, sigma=sigma, W1=W1, b1=b1, W2=W2, b2=b2, labels=labels)


def load_default_selector(path: str = DEFAULT_BLOB) -> dict:
    """Load the committed trained selector onto the current device."""
    blob = np.fromfile(path, dtype=np.float32)
    B.spmv_selector_load(blob)
    return parse_blob(blob)


# ---------------------------------------------------------------------------
# dataset from sweep records
# ---------------------------------------------------------------------------
def load_records(paths):
    """Sweep records (JSON lines, optionally gzip-compressed) keyed by matrix."""
    import gzip
    recs = {}
    for p in paths:
        with (gzip.open(p, "rt") if p.endswith(".gz") else open(p)) as fh:
            for line in fh:
                try:
                    r = json.loads(line)
                except Exception:
                    continue
                if "features" in r:
                    recs[r["matrix"]] = r
    return [recs[k] for k in sorted(recs)]


def dataset(records, label_keys):
    """X (N x 20 features), T (N x K times in us, inf where refused), the
    default-CSR time per matrix, matrix ids and families."""
    K = len(label_keys)
    X = np.array([r["features"] for r in records], np.float64)
    T = np.full((len(records), K), np.inf)
    for i, r in enumerate(records):
        tm = dict((k, t) for k, t in r["times"])
        for j, key in enumerate(label_keys):
            t = tm.get(key)
            if t is not None:
                T[i, j] = t
    D = np.array([r["default_us"] for r in records], np.float64)
    ids = np.array([r["matrix"] for r in records])
    fams = [r["family"] for r in records]
    return X, T, D, ids, fams


def transform(X, mu=None, sigma=None):
    Z = np.array(X, np.float64)
    Z[:, LOG_IDX] = np.log1p(Z[:, LOG_IDX])
    if mu is None:
        mu = Z.mean(axis=0)
        sigma = Z.std(axis=0)
        sigma = np.where(sigma > 1e-12, sigma, 1.0)
    return (Z - mu) / sigma, mu, sigma


def soft_targets(T, tau: float = 0.05):
    """Class weights exp(-(t/t_best - 1)/tau), normalised per matrix."""
    best = T.min(axis=1, keepdims=True)
    rel = T / best - 1.0
    w = np.where(np.isfinite(rel), np.exp(-rel / tau), 0.0)
    return w / w.sum(axis=1, keepdims=True)


def train(X, T, hidden: int = 64, epochs: int = 3000, lr: float = 3e-3, wd: float = 1e-3, seed: int = 0,
          tau: float = 0.05):
    """Full-batch Adam on the soft cross-entropy; returns float64 weights.
    tau = 0.05 and weight decay 1e-3 were chosen by 5-fold cross-validation
    on the training matrices only (fraction within 10% of the best)."""
    import torch
    torch.manual_seed(seed)
    Z, mu, sigma = transform(X)
    P = soft_targets(T, tau)
    Zt = torch.tensor(Z, dtype=torch.float32)
    Pt = torch.tensor(P, dtype=torch.float32)
    mask = torch.tensor(np.isfinite(T), dtype=torch.bool)
    K = T.shape[1]
    net = torch.nn.Sequential(torch.nn.Linear(Z.shape[1], hidden), torch.nn.ReLU(), torch.nn.Linear(hidden, K))
    opt = torch.optim.Adam(net.parameters(), lr=lr, weight_decay=wd)
    for _ in range(epochs):
        opt.zero_grad()
        logits = net(Zt).masked_fill(~mask, -1e4)
        loss = -(Pt * torch.log_softmax(logits, dim=1)).sum(dim=1).mean()
        loss.backward()
        opt.step()
    W1 = net[0].weight.detach().numpy().astype(np.float64)
    b1 = net[0].bias.detach().numpy().astype(np.float64)
    W2 = net[2].weight.detach().numpy().astype(np.float64)
    b2 = net[2].bias.detach().numpy().astype(np.float64)
    return dict(mu=mu, sigma=sigma, W1=W1, b1=b1, W2=W2, b2=b2)


def predict(w, X):
    Z, _, _ = transform(X, w["mu"], w["sigma"])
    H = np.maximum(Z @ np.asarray(w["W1"]).T + w["b1"], 0.0)
    return H @ np.asarray(w["W2"]).T + w["b2"]


def evaluate(choice, T, D):
    """Selector quality: slowdown t(choice)/t(best) per matrix, the fraction
    within 10% of the exhaustive best, and the geometric-mean speedup over
    default CSR."""
    best = T.min(axis=1)
    t_sel = T[np.arange(len(choice)), choice]
    slow = t_sel / best
    return {"n": int(len(choice)), "within_10pct": float(np.mean(slow <= 1.10)),
            "median_slowdown": float(np.median(slow)), "max_slowdown": float(np.max(slow)),
            "geomean_slowdown": float(np.exp(np.mean(np.log(slow)))),
            "geomean_speedup_vs_default_csr": float(np.exp(np.mean(np.log(D / t_sel)))),
            "geomean_best_vs_default_csr": float(np.exp(np.mean(np.log(D / best))))}


def main():
    """Train on the sweep records (matrices 0-1799), evaluate on 1800-1999,
    write the blob and a JSON report."""
    import argparse
    from . import sweep
    ap = argparse.ArgumentParser(description="train the selector MLP from sweep records")
    ap.add_argument("--data", nargs="+", required=True)
    ap.add_argument("--out", default=DEFAULT_BLOB)
    ap.add_argument("--report", default=None)
    ap.add_argument("--hidden", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=3000)
    ap.add_argument("--holdout-start", type=int, default=1800)
    args = ap.parse_args()
    recs = load_records(args.data)
    labels = sweep.label_space()
    keys = [sweep.config_key(c) for c in labels]
    X, T, D, ids, fams = dataset(recs, keys)
    ok = np.isfinite(T).any(axis=1) & np.isfinite(D)
    train_m = ok & (ids < args.holdout_start)
    test_m = ok & (ids >= args.holdout_start)
    w = train(X[train_m], T[train_m], hidden=args.hidden, epochs=args.epochs)
    report = {"train_matrices": int(train_m.sum()), "heldout_matrices": int(test_m.sum()),
              "classes": len(labels), "hidden": args.hidden}
    for name, msk in (("train", train_m), ("heldout", test_m)):
        if msk.any():
            logits = predict(w, X[msk])
            logits = np.where(np.isfinite(T[msk]), logits, -np.inf)
            choice = np.argmax(logits, axis=1)
            report[name] = evaluate(choice, T[msk], D[msk])
            fam_arr = np.array(fams)[msk]
            report[name + "_by_family"] = {
                f: evaluate(choice[fam_arr == f], T[msk][fam_arr == f], D[msk][fam_arr == f])
                for f in sorted(set(fam_arr))}
    blob = make_blob(w["mu"], w["sigma"], w["W1"], w["b1"], w["W2"], w["b2"], labels)
    blob.tofile(args.out)
    txt = json.dumps(report, indent=1)
    if args.report:
        with open(args.report, "w") as fh:
            fh.write(txt + "\n")
    print(txt)


if __name__ == "__main__":
    main()
