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
# trained on fp32-value sweeps; used for fp32 handles, and for bf16 handles
# when no bf16-trained blob is present
LOWP_BLOB = os.path.join(PKG, "selector_gb300_fp32_values.f32")
BF16_BLOB = os.path.join(PKG, "selector_gb300_bf16_values.f32")
# the exhaustive-sweep records the committed fp64 selector was trained on
# (every label point of the 2000 dataset matrices, L2 flushed by reading,
# trimmed means), the conversion-time calibration of its cost model, and the
# GPU-measured held-out evaluations (sweep --heldout-eval) of the fp64, fp32 and
# bf16 selectors
DEFAULT_DATA = os.path.join(PKG, "data", "sweep_gb300_f64_readflush.jsonl.gz")
DEFAULT_CALIB = os.path.join(PKG, "data", "convert_calib_gb300_f64.jsonl.gz")
RETIMED_F64 = os.path.join(PKG, "data", "heldout_retimed_gb300_f64.jsonl.gz")
RETIMED_F32 = os.path.join(PKG, "data", "heldout_retimed_gb300_f32.jsonl.gz")
RETIMED_BF16 = os.path.join(PKG, "data", "heldout_retimed_gb300_bf16.jsonl.gz")
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


NFMT = 6   # formats 0..5 in the conversion-cost model


def make_blob(mu, sigma, W1, b1, W2, b2, labels, W3=None, b3=None, pack=None) -> np.ndarray:
    """Float32 blob for spmv_selector_load: version 1 (classifier) or, with
    W3/b3 (time head, K+1 rows) and pack (NFMT x 3 cost model), version 2."""
    W1 = np.asarray(W1, np.float32)
    W2 = np.asarray(W2, np.float32)
    H, F = W1.shape
    K = W2.shape[0]
    version = 2.0 if W3 is not None else 1.0
    parts = [np.array([MAGIC, version, F, H, K], np.float32), np.asarray(mu, np.float32),
             np.asarray(sigma, np.float32), W1.reshape(-1), np.asarray(b1, np.float32), W2.reshape(-1),
             np.asarray(b2, np.float32), np.array([full_config(l) for l in labels], np.float32).reshape(-1)]
    if W3 is not None:
        W3 = np.asarray(W3, np.float32)
        assert W3.shape == (K + 1, H)
        parts += [W3.reshape(-1), np.asarray(b3, np.float32).reshape(K + 1),
                  np.asarray(pack, np.float32).reshape(NFMT * 3)]
    return np.concatenate(parts)


def parse_blob(blob) -> dict:
    b = np.asarray(blob, np.float32)
    assert b[0] == MAGIC and b[1] in (1.0, 2.0)
    version = int(b[1])
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
    out = dict(version=version, F=F, H=H, K=K, mu=mu, sigma=sigma, W1=W1, b1=b1, W2=W2, b2=b2, labels=labels)
    if version == 2:
        out["W3"] = take((K + 1) * H).reshape(K + 1, H)
        out["b3"] = take(K + 1)
        out["pack"] = take(NFMT * 3).reshape(NFMT, 3)
    assert o == b.size
    return out


def load_default_selector(path: str = DEFAULT_BLOB, lowp_path: str | None = LOWP_BLOB,
                          bf16_path: str | None = BF16_BLOB) -> dict:
    """Load the committed trained selector onto the current device (for every
    value type), then the ones trained on fp32 and on bf16 values, where
    present, for handles of those value types (bf16 handles fall back to the
    fp32-trained blob)."""
    blob = np.fromfile(path, dtype=np.float32)
    B.spmv_selector_load(blob)
    for vt in (B.SPMV_F32, B.SPMV_BF16):
        own = bf16_path if vt == B.SPMV_BF16 and bf16_path and os.path.exists(bf16_path) else lowp_path
        if own and os.path.exists(own):
            B.spmv_selector_load_vt(vt, np.fromfile(own, dtype=np.float32))
        else:
            B.spmv_selector_load_vt(vt, None)
    return parse_blob(blob)


def default_is_v2(path: str = DEFAULT_BLOB) -> bool:
    """Whether the committed blob carries the time head and conversion model."""
    import os
    return os.path.exists(path) and parse_blob(np.fromfile(path, dtype=np.float32))["version"] >= 2


# ---------------------------------------------------------------------------
# dataset from sweep records
# ---------------------------------------------------------------------------
def load_records(paths):
    """Sweep records (JSON lines, optionally gzip-compressed) keyed by matrix.

    Supplementary records (a later sweep of some formats only) are merged
    into the full record of the same matrix: their times are rescaled by the
    ratio of the two default-CSR times measured in each sweep, so that
    timings taken on another GPU or day land on the full record's scale."""
    import gzip
    recs, supp = {}, []
    for p in paths:
        with (gzip.open(p, "rt") if p.endswith(".gz") else open(p)) as fh:
            for line in fh:
                try:
                    r = json.loads(line)
                except Exception:
                    continue
                if "features" in r:
                    recs[r["matrix"]] = r
                elif "supplement" in r:
                    supp.append(r)
    for r in supp:
        base = recs.get(r["matrix"])
        if base is None or not base.get("default_us") or not r.get("default_us"):
            continue
        scale = base["default_us"] / r["default_us"]
        tm = dict((k, t) for k, t in base["times"])
        for k, t in r["times"]:
            tm[k] = None if t is None else t * scale
        base["times"] = [[k, t] for k, t in tm.items()]
    return [recs[k] for k in sorted(recs)]


def has_sell(records) -> bool:
    """Whether any record holds SELL timings (then SELL joins the labels)."""
    return any(k.startswith("format=5,") for r in records for k, _ in r["times"])


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


def hidden(w, X):
    Z, _, _ = transform(X, w["mu"], w["sigma"])
    return np.maximum(Z @ np.asarray(w["W1"], np.float64).T + np.asarray(w["b1"], np.float64), 0.0)


def train_time_head(w, X, T, D, lam: float = 1e-2):
    """Ridge regression of log(us per product) on the hidden layer, one row
    per label class (matrices where the class ran) plus one for default CSR:
    the regression alternative of Section 5.4 on top of the classifier."""
    Hh = hidden(w, X)
    A = np.hstack([Hh, np.ones((Hh.shape[0], 1))])
    K = T.shape[1]
    W3 = np.zeros((K + 1, Hh.shape[1]))
    b3 = np.zeros(K + 1)
    targets = [T[:, k] for k in range(K)] + [D]
    for k, t in enumerate(targets):
        ok = np.isfinite(t) & (t > 0)
        if ok.sum() < 5:
            b3[k] = np.log(np.nanmedian(np.where(np.isfinite(t), t, np.nan))) if np.isfinite(t).any() else 0.0
            continue
        Ak = A[ok]
        G = Ak.T @ Ak + lam * np.eye(Ak.shape[1])
        beta = np.linalg.solve(G, Ak.T @ np.log(t[ok]))
        W3[k] = beta[:-1]
        b3[k] = beta[-1]
    return W3, b3


def predict_logt(w, W3, b3, X):
    return hidden(w, X) @ np.asarray(W3, np.float64).T + np.asarray(b3, np.float64)


def fit_pack_model(calib):
    """Least squares of measured conversion time (us) on [1, nnz, m] per
    format: the conversion-overhead predictor (Section 5.3 step 3).  `calib`
    is a list of records {format, nnz, m, us}.  Coefficients are clipped at
    zero so the model never predicts a negative cost."""
    P = np.zeros((NFMT, 3))
    for f in range(NFMT):
        rs = [r for r in calib if r["format"] == f and r["us"] is not None]
        if len(rs) < 3:
            continue
        A = np.array([[1.0, r["nnz"], r["m"]] for r in rs])
        y = np.array([r["us"] for r in rs])
        coef, *_ = np.linalg.lstsq(A, y, rcond=None)
        P[f] = np.maximum(coef, 0.0)
    return P


def gate_decision(t_cur, t_sel, select_us, pack_us, runs):
    """Convert iff the gain over `runs` products exceeds the overhead."""
    return (t_cur - t_sel) * runs > select_us + pack_us


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


KNOBS = ("regcap", "unroll", "carveout")
DEFAULT_KNOBS = (0, 0, -1)   # the library defaults (resolved per format and value type)


def _parse_key(key: str) -> dict:
    return {kv.split("=")[0]: int(kv.split("=")[1]) for kv in key.split(",")}


def _class_key(d: dict) -> str:
    from . import sweep
    return sweep.config_key({k: v for k, v in d.items() if k not in KNOBS})


def load_refine(paths) -> dict:
    """Refine records by matrix: {matrix: (base class key, {knobs: us})},
    knobs = (regcap, unroll, carveout), DEFAULT_KNOBS for the base point."""
    import gzip
    out = {}
    for p in paths:
        with (gzip.open(p, "rt") if p.endswith(".gz") else open(p)) as fh:
            for line in fh:
                if not line.strip():
                    continue
                r = json.loads(line)
                t = {DEFAULT_KNOBS: r["best_us"]}
                for key, us in r["refine"]:
                    d = _parse_key(key)
                    t[tuple(d[k] for k in KNOBS)] = us
                out[r["matrix"]] = (_class_key(_parse_key(r["best"])), t)
    return out


def knob_table(refine: dict, train_ids) -> dict:
    """The paper's compile-time knobs (Section 4 items 1-3: register cap,
    memory configuration; plus unroll) chosen per label class from the
    training matrices whose best class it is: the knob setting with the
    smallest geometric-mean time relative to each matrix's refined best.
    The library defaults are a candidate, so a class keeps them unless a
    setting beats them on its matrices."""
    by_class = {}
    for mid in train_ids:
        if mid not in refine:
            continue
        base, t = refine[mid]
        ok = {k: v for k, v in t.items() if v is not None}
        if not ok:
            continue
        best = min(ok.values())
        by_class.setdefault(base, []).append({k: v / best for k, v in ok.items()})
    table = {}
    for base, mats in by_class.items():
        cands = set().union(*[set(m) for m in mats])
        score = {}
        for c in cands:
            rs = [m.get(c) for m in mats]
            if any(r is None for r in rs):
                continue
            score[c] = float(np.exp(np.mean(np.log(rs))))
        if score:
            table[base] = min(score, key=score.get)
    return table


def evaluate_refined(choice_keys, ids, refine: dict, T, labels_keys, table: dict):
    """Slowdown against the refined exhaustive best (the best label point
    with its knobs refined) of the selector's choice, with and without the
    knob table, on matrices that have refine records.  Times come from the
    refine session; a choice other than the refined class is rescaled from
    the main sweep by the ratio of the two sessions' times of that class."""
    slow_k, slow_0 = [], []
    kidx = {k: j for j, k in enumerate(labels_keys)}
    for i, mid in enumerate(ids):
        if mid not in refine:
            continue
        base, t = refine[mid]
        ok = {k: v for k, v in t.items() if v is not None}
        if not ok or base not in kidx or not np.isfinite(T[i, kidx[base]]):
            continue
        best = min(ok.values())
        ck = choice_keys[i]
        if ck == base:
            t0 = ok.get(DEFAULT_KNOBS)
            tk = ok.get(table.get(ck, DEFAULT_KNOBS), t0)
        else:
            scale = ok[DEFAULT_KNOBS] / T[i, kidx[base]]
            t0 = tk = T[i, kidx[ck]] * scale
        slow_0.append(t0 / best)
        slow_k.append(tk / best)
    def summ(v):
        v = np.array(v)
        return {"n": int(v.size), "within_10pct": float(np.mean(v <= 1.10)),
                "geomean_slowdown": float(np.exp(np.mean(np.log(v)))), "median_slowdown": float(np.median(v))}
    return {"with_knob_table": summ(slow_k), "class_only": summ(slow_0)}


def evaluate_retimed(paths) -> dict:
    """The held-out evaluation measured on the GPU (sweep --heldout-eval): per
    matrix, the device selector's pick and the refined exhaustive best
    (label space, then register cap x unroll x carveout around its winner)
    timed again in one session with interleaved repetitions.  Slowdown =
    t(pick) / t(refined best); also with the per-class knob table applied to
    the pick, and the pick's speedup over default CSR."""
    import gzip
    recs = []
    for path in paths:
        with (gzip.open(path, "rt") if path.endswith(".gz") else open(path)) as fh:
            recs += [json.loads(l) for l in fh if l.strip()]
    def summ(rs):
        slow = np.array([r["final"]["pick"] / r["final"]["winner"] for r in rs])
        slk = np.array([r["final"].get("pick_knob_table", r["final"]["pick"]) / r["final"]["winner"] for r in rs])
        spd = np.array([r["final"]["default_csr"] / r["final"]["pick"] for r in rs])
        best = np.array([r["final"]["default_csr"] / r["final"]["winner"] for r in rs])
        return {"n": len(rs), "within_10pct": float(np.mean(slow <= 1.10)),
                "median_slowdown": float(np.median(slow)), "max_slowdown": float(slow.max()),
                "geomean_slowdown": float(np.exp(np.mean(np.log(slow)))),
                "within_10pct_with_knob_table": float(np.mean(slk <= 1.10)),
                "geomean_slowdown_with_knob_table": float(np.exp(np.mean(np.log(slk)))),
                "geomean_speedup_vs_default_csr": float(np.exp(np.mean(np.log(spd)))),
                "geomean_best_vs_default_csr": float(np.exp(np.mean(np.log(best))))}
    out = {"all": summ(recs), "dtype": sorted({r["dtype"] for r in recs}),
           "flush": sorted({r["flush"] for r in recs})}
    out["by_family"] = {f: summ([r for r in recs if r["family"] == f]) for f in sorted({r["family"] for r in recs})}
    sizes = (("under_15us", 0, 15), ("15_to_40us", 15, 40), ("over_40us", 40, float("inf")))
    out["by_refined_best_time"] = {k: summ([r for r in recs if lo <= r["final"]["winner"] < hi])
                                   for k, lo, hi in sizes if any(lo <= r["final"]["winner"] < hi for r in recs)}
    return out


def main():
    """Train on the sweep records (matrices 0-1799), evaluate on 1800-1999,
    write the blob and a JSON report.  With --calib (conversion-time
    records) the blob is version 2: time head + conversion-cost model, and
    the report evaluates the run-time gate on the held-out matrices."""
    import argparse
    from . import sweep
    ap = argparse.ArgumentParser(description="train the selector MLP from sweep records")
    ap.add_argument("--data", nargs="+", required=True)
    ap.add_argument("--out", default=DEFAULT_BLOB)
    ap.add_argument("--report", default=None)
    ap.add_argument("--hidden", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=3000)
    ap.add_argument("--holdout-start", type=int, default=1800)
    ap.add_argument("--from-blob", default=None, help="reuse this blob's classifier, fit only the heads")
    ap.add_argument("--calib", nargs="*", default=None, help="conversion-time records (JSON lines)")
    ap.add_argument("--refine", nargs="*", default=None,
                    help="refine records (sweep --refine-from): evaluate a per-class register cap / unroll / "
                         "carveout table against the refined exhaustive best")
    ap.add_argument("--heldout-retimed", nargs="*", default=None,
                    help="records of sweep --heldout-eval: the GPU-measured evaluation of the blob, added to "
                         "the report")
    ap.add_argument("--apply-knobs", action="store_true",
                    help="write the per-class knob table into the blob's labels (default: report only)")
    args = ap.parse_args()
    recs = load_records(args.data)
    labels = sweep.label_space(include_sell=has_sell(recs))
    keys = [sweep.config_key(c) for c in labels]
    X, T, D, ids, fams = dataset(recs, keys)
    ok = np.isfinite(T).any(axis=1) & np.isfinite(D)
    train_m = ok & (ids < args.holdout_start)
    test_m = ok & (ids >= args.holdout_start)
    if args.from_blob:
        p = parse_blob(np.fromfile(args.from_blob, dtype=np.float32))
        w = {k: p[k].astype(np.float64) for k in ("mu", "sigma", "W1", "b1", "W2", "b2")}
    else:
        w = train(X[train_m], T[train_m], hidden=args.hidden, epochs=args.epochs)
    report = {"train_matrices": int(train_m.sum()), "heldout_matrices": int(test_m.sum()),
              "classes": len(labels), "hidden": int(np.asarray(w["W1"]).shape[0])}
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
    W3 = b3 = pack = None
    if args.calib is not None:
        import gzip
        calib = []
        for path in args.calib:
            with (gzip.open(path, "rt") if path.endswith(".gz") else open(path)) as fh:
                calib += [json.loads(l) for l in fh if l.strip()]
        W3, b3 = train_time_head(w, X[train_m], T[train_m], D[train_m])
        pack = fit_pack_model([c for c in calib if c["matrix"] < args.holdout_start])
        # time head on held-out matrices: error of the selected class and default CSR
        if not test_m.any():   # no held-out sweep records (evaluated by --heldout-retimed instead)
            test_m = train_m & False
        lt = predict_logt(w, W3, b3, X[test_m]) if test_m.any() else None
        if lt is not None:
            logits = np.where(np.isfinite(T[test_m]), predict(w, X[test_m]), -np.inf)
            choice = np.argmax(logits, axis=1)
            rows = np.arange(choice.size)
            e_sel = np.abs(lt[rows, choice] - np.log(T[test_m][rows, choice]))
            e_def = np.abs(lt[:, -1] - np.log(D[test_m]))
            report["time_head_heldout"] = {"median_abs_log_error_selected": float(np.median(e_sel)),
                                           "median_abs_log_error_default_csr": float(np.median(e_def)),
                                           "p90_abs_log_error_selected": float(np.quantile(e_sel, 0.9))}
        # conversion-cost model on held-out calibration records
        held = [c for c in calib if c["matrix"] >= args.holdout_start and c["us"] is not None]
        if held and lt is not None:
            pred = np.array([pack[c["format"]] @ [1.0, c["nnz"], c["m"]] for c in held])
            meas = np.array([c["us"] for c in held])
            ss_res = float(((pred - meas) ** 2).sum())
            ss_tot = float(((meas - meas.mean()) ** 2).sum())
            report["pack_model_heldout"] = {"n": len(held), "r2": 1.0 - ss_res / ss_tot,
                                            "median_abs_rel_error": float(np.median(np.abs(pred - meas) / meas))}
            # the gate on held-out matrices: predicted vs measured decision
            by = {}
            for c in held:
                by.setdefault(c["matrix"], {})[c["format"]] = c["us"]
            id_test = ids[test_m]
            agree = {}
            for runs in (1, 10, 100, 1000, 10000):
                hits = tot = 0
                for i, mid in enumerate(id_test):
                    if mid not in by:
                        continue
                    f = int(labels[choice[i]]["format"])
                    if f not in by[mid]:
                        continue
                    t_def, t_sel = D[test_m][i], T[test_m][i, choice[i]]
                    truth = gate_decision(t_def, t_sel, 0.0, by[mid][f], runs)
                    guess = gate_decision(np.exp(lt[i, -1]), np.exp(lt[i, choice[i]]), 0.0,
                                          pack[f] @ [1.0, by_nnz(recs, mid), by_m(recs, mid)], runs)
                    hits += int(truth == guess)
                    tot += 1
                agree[str(runs)] = hits / tot if tot else None
            report["gate_agreement_heldout"] = agree
        report["pack_model_us"] = {str(f): [float(v) for v in pack[f]] for f in range(NFMT)}
    if args.refine:
        refine = load_refine(args.refine)
        table = knob_table(refine, ids[train_m])
        if args.apply_knobs:
            labels = [dict(c, **dict(zip(KNOBS, table[keys[j]]))) if keys[j] in table else c
                      for j, c in enumerate(labels)]
        report["knob_table"] = {k: dict(zip(KNOBS, v)) for k, v in sorted(table.items())}
        report["knob_table_applied"] = bool(args.apply_knobs)
        for name, msk in (("train", train_m), ("heldout", test_m)):
            logits = np.where(np.isfinite(T[msk]), predict(w, X[msk]), -np.inf)
            choice = np.argmax(logits, axis=1)
            report[name + "_vs_refined_best"] = evaluate_refined([keys[c] for c in choice], ids[msk], refine,
                                                                 T[msk], keys, table)
    if args.heldout_retimed:
        report["heldout_retimed"] = evaluate_retimed(args.heldout_retimed)
    blob = make_blob(w["mu"], w["sigma"], w["W1"], w["b1"], w["W2"], w["b2"], labels, W3, b3, pack)
    blob.tofile(args.out)
    txt = json.dumps(report, indent=1)
    if args.report:
        with open(args.report, "w") as fh:
            fh.write(txt + "\n")
    print(txt)


def by_nnz(recs, mid):
    return next(r["nnz"] for r in recs if r["matrix"] == mid)


def by_m(recs, mid):
    return next(r["m"] for r in recs if r["matrix"] == mid)


if __name__ == "__main__":
    main()
