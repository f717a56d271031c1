"""Host-side selector logic: blob layout, soft targets, training on a
separable toy set, and the evaluation arithmetic."""
import numpy as np

from paper_2302_05662_gb300 import selector as S


def test_blob_roundtrip():
    rng = np.random.default_rng(0)
    H, K = 8, 5
    w = dict(mu=rng.normal(size=20), sigma=rng.uniform(1, 2, 20), W1=rng.normal(size=(H, 20)),
             b1=rng.normal(size=H), W2=rng.normal(size=(K, H)), b2=rng.normal(size=K))
    labels = [dict(format=k, threads_per_block=64) for k in range(K)]
    blob = S.make_blob(w["mu"], w["sigma"], w["W1"], w["b1"], w["W2"], w["b2"], labels)
    assert blob.size == 5 + 40 + H * 20 + H + K * H + K + 8 * K
    p = S.parse_blob(blob)
    assert (p["F"], p["H"], p["K"]) == (20, H, K)
    assert np.allclose(p["W2"], w["W2"].astype(np.float32))
    assert list(p["labels"][3]) == [3, 64, 0, 0, 0, -1, 0, 0]


def test_soft_targets_favour_near_ties():
    T = np.array([[10.0, 10.1, 20.0, np.inf]])
    P = S.soft_targets(T, tau=0.02)
    assert P[0, 3] == 0.0 and P[0, 0] > P[0, 1] > P[0, 2]
    assert abs(P.sum() - 1.0) < 1e-12


def test_training_learns_separable_toy():
    rng = np.random.default_rng(1)
    X = np.abs(rng.normal(size=(400, 20))) + 1.0
    cls = (X[:, 2] > np.median(X[:, 2])).astype(int)       # density feature decides
    T = np.where(np.arange(3)[None, :] == cls[:, None], 1.0, 2.0)
    w = S.train(X, T, hidden=16, epochs=400, lr=1e-2)
    pred = np.argmax(S.predict(w, X), axis=1)
    assert np.mean(pred == cls) > 0.95


def test_evaluate_arithmetic():
    T = np.array([[1.0, 2.0], [4.0, 3.0]])
    D = np.array([2.0, 6.0])
    e = S.evaluate(np.array([0, 0]), T, D)
    assert e["within_10pct"] == 0.5
    assert abs(e["geomean_slowdown"] - np.sqrt(1.0 * 4.0 / 3.0)) < 1e-12
    assert abs(e["geomean_speedup_vs_default_csr"] - np.sqrt(2.0 * 1.5)) < 1e-12


def test_committed_selector_matches_its_report():
    """The committed blob, evaluated on the committed held-out records,
    reproduces the committed report (fraction within 10% of the exhaustive
    best, geometric-mean slowdown and speedup over default CSR)."""
    import json
    import os
    from paper_2302_05662_gb300 import sweep
    if not os.path.exists(S.DEFAULT_BLOB):
        import pytest
        pytest.skip("no committed selector")
    p = S.parse_blob(np.fromfile(S.DEFAULT_BLOB, dtype=np.float32))
    recs = S.load_records([S.DEFAULT_DATA])
    labels = sweep.label_space(include_sell=S.has_sell(recs))
    keys = [sweep.config_key(c) for c in labels]
    assert len(labels) == p["K"] == 78
    for k, c in enumerate(labels):                   # the blob's classes are the label space, in order
        lab = dict(zip(S.CFG_FIELDS, p["labels"][k].tolist()))
        assert all(lab[f] == c.get(f, 0) for f in ("format", "threads_per_block", "threads_per_row"))
    X, T, D, ids, fams = S.dataset(recs, keys)
    msk = (ids >= 1800) & np.isfinite(T).any(axis=1) & np.isfinite(D)
    w = {k: p[k].astype(np.float64) for k in ("mu", "sigma", "W1", "b1", "W2", "b2")}
    lg = np.where(np.isfinite(T[msk]), S.predict(w, X[msk]), -np.inf)
    got = S.evaluate(np.argmax(lg, axis=1), T[msk], D[msk])
    rep = json.load(open(os.path.join(os.path.dirname(S.DEFAULT_BLOB), "selector_gb300_report.json")))
    assert got["n"] == rep["heldout"]["n"] == 200
    assert abs(got["within_10pct"] - rep["heldout"]["within_10pct"]) <= 0.01
    assert got["within_10pct"] >= 0.90
    assert got["geomean_speedup_vs_default_csr"] > 1.0
    assert p["version"] == 2 and rep["pack_model_heldout"]["r2"] > 0.9


def test_committed_gpu_evaluations_match_their_reports():
    """The held-out evaluations measured on the GPU (the device selector's pick
    against the refined exhaustive best, both re-timed in one session),
    recomputed from the committed records, equal the committed reports of
    the fp64, fp32 and bf16 selectors, and each pick is a class of the
    label space."""
    import json
    import os
    from paper_2302_05662_gb300 import sweep
    keys = {sweep.config_key(c) for c in sweep.label_space(include_sell=True)}
    pkg = os.path.dirname(S.DEFAULT_BLOB)
    for recs, report in ((S.RETIMED_F64, "selector_gb300_report.json"),
                         (S.RETIMED_F32, "selector_gb300_fp32_values_report.json"),
                         (S.RETIMED_BF16, "selector_gb300_bf16_values_report.json")):
        got = S.evaluate_retimed([recs])
        rep = json.load(open(os.path.join(pkg, report)))["heldout_retimed"]
        assert got["all"] == rep["all"]
        assert got["all"]["n"] == 200 and got["all"]["within_10pct"] >= 0.90
        import gzip
        with gzip.open(recs, "rt") as fh:
            rows = [json.loads(l) for l in fh]
        assert sorted(r["matrix"] for r in rows) == list(range(1800, 2000))
        assert all(r["pick"] in keys and r["flush"] == "read" for r in rows)


def test_blob_v2_roundtrip_and_heads():
    rng = np.random.default_rng(2)
    H, K = 8, 5
    w = dict(mu=rng.normal(size=20), sigma=rng.uniform(1, 2, 20), W1=rng.normal(size=(H, 20)),
             b1=rng.normal(size=H), W2=rng.normal(size=(K, H)), b2=rng.normal(size=K))
    W3, b3 = rng.normal(size=(K + 1, H)), rng.normal(size=K + 1)
    pack = rng.uniform(0, 1, (S.NFMT, 3))
    labels = [dict(format=k, threads_per_block=64) for k in range(K)]
    blob = S.make_blob(w["mu"], w["sigma"], w["W1"], w["b1"], w["W2"], w["b2"], labels, W3, b3, pack)
    p = S.parse_blob(blob)
    assert p["version"] == 2 and p["W3"].shape == (K + 1, H)
    assert np.allclose(p["pack"], pack.astype(np.float32))
    assert blob.size == 5 + 40 + H * 20 + H + K * H + K + 8 * K + (K + 1) * H + (K + 1) + S.NFMT * 3


def test_time_head_recovers_a_linear_law():
    rng = np.random.default_rng(3)
    X = np.abs(rng.normal(size=(300, 20))) + 1.0
    w = S.train(X, np.ones((300, 3)) + rng.uniform(0, 1, (300, 3)), hidden=16, epochs=50)
    Hh = S.hidden(w, X)
    true_w = rng.normal(size=Hh.shape[1])
    T = np.exp(np.stack([Hh @ true_w + 1.0, Hh @ (0.5 * true_w) - 1.0, Hh @ true_w * 0 + 2.0], axis=1))
    D = np.exp(Hh @ true_w + 0.3)
    W3, b3 = S.train_time_head(w, X, T, D, lam=1e-8)
    lt = S.predict_logt(w, W3, b3, X)
    assert np.max(np.abs(lt[:, :3] - np.log(T))) < 1e-5
    assert np.max(np.abs(lt[:, 3] - np.log(D))) < 1e-5


def test_pack_model_fit_and_gate():
    calib = [{"format": f, "nnz": n, "m": m, "us": 50.0 + 0.002 * n + 0.01 * m + 7 * f}
             for f in range(S.NFMT) for n, m in ((1e5, 1e4), (5e5, 2e4), (2e6, 3e5), (8e6, 5e5))]
    P = S.fit_pack_model(calib)
    assert np.allclose(P[2], [64.0, 0.002, 0.01], rtol=1e-6)
    # gain (100 - 60) x runs against overhead 1000 + 500: pays off from 38 runs
    assert not S.gate_decision(100.0, 60.0, 1000.0, 500.0, 37)
    assert S.gate_decision(100.0, 60.0, 1000.0, 500.0, 38)
    assert not S.gate_decision(50.0, 60.0, 0.0, 0.0, 10 ** 9)      # never when slower


def test_supplementary_records_merge_on_the_base_scale(tmp_path):
    import json
    base = {"matrix": 3, "family": "stencil", "features": [0.0] * 20, "default_us": 100.0,
            "times": [["format=0,threads_per_block=32,threads_per_row=1", 50.0],
                      ["format=1,threads_per_block=32", None]]}
    supp = {"matrix": 3, "family": "stencil", "default_us": 200.0, "supplement": "sell",
            "times": [["format=5,threads_per_block=32", 80.0], ["format=5,threads_per_block=64", None]]}
    orphan = dict(supp, matrix=4)
    p1, p2 = tmp_path / "a.jsonl", tmp_path / "b.jsonl"
    p1.write_text(json.dumps(base) + "\n")
    p2.write_text(json.dumps(supp) + "\n" + json.dumps(orphan) + "\n")
    recs = S.load_records([str(p1), str(p2)])
    assert [r["matrix"] for r in recs] == [3]
    tm = dict((k, t) for k, t in recs[0]["times"])
    assert tm["format=5,threads_per_block=32"] == 40.0          # 80 us x (100 / 200)
    assert tm["format=5,threads_per_block=64"] is None
    assert tm["format=0,threads_per_block=32,threads_per_row=1"] == 50.0
    assert S.has_sell(recs) and not S.has_sell(S.load_records([str(p1)]))


def _refine(base, times):
    """A refine record: base class key, {(regcap, unroll, carveout): us}."""
    return (base, dict(times))


def test_knob_table_picks_the_best_shared_setting():
    A = "format=2,threads_per_block=32"
    refine = {
        0: _refine(A, {S.DEFAULT_KNOBS: 10.0, (32, 4, 0): 8.0, (64, 2, -1): 9.0}),
        1: _refine(A, {S.DEFAULT_KNOBS: 20.0, (32, 4, 0): 17.0, (64, 2, -1): 15.0}),
        2: _refine("format=1,threads_per_block=64", {S.DEFAULT_KNOBS: 5.0, (32, 1, 100): 6.0}),
        3: _refine(A, {S.DEFAULT_KNOBS: 1.0, (32, 4, 0): 0.1}),            # held out: ignored
    }
    table = S.knob_table(refine, train_ids=[0, 1, 2])
    # (32,4,0): geomean(8/8, 17/15) = 1.0646; (64,2,-1): geomean(9/8, 15/15) = 1.0607
    assert table[A] == (64, 2, -1)
    assert table["format=1,threads_per_block=64"] == S.DEFAULT_KNOBS   # defaults win there


def test_evaluate_refined_uses_the_refine_session():
    A, Bk = "format=2,threads_per_block=32", "format=5,threads_per_block=32"
    keys = [A, Bk]
    refine = {7: _refine(A, {S.DEFAULT_KNOBS: 10.0, (32, 4, 0): 8.0}),
              8: _refine(A, {S.DEFAULT_KNOBS: 10.0, (32, 4, 0): 8.0})}
    T = np.array([[20.0, 30.0], [20.0, 30.0]])     # main sweep: another session, 2x slower
    table = {A: (32, 4, 0)}
    r = S.evaluate_refined([A, Bk], np.array([7, 8]), refine, T, keys, table)
    # matrix 7 chose its refined class: 8/8 with the table, 10/8 without;
    # matrix 8 chose B: 30 * (10/20) = 15, against the refined best 8
    assert r["with_knob_table"]["n"] == 2
    assert np.isclose(r["with_knob_table"]["geomean_slowdown"], np.sqrt(1.0 * 15 / 8))
    assert np.isclose(r["class_only"]["geomean_slowdown"], np.sqrt(10 / 8 * 15 / 8))
    assert r["with_knob_table"]["within_10pct"] == 0.5


def test_sweep_statistics_and_label_keys():
    """The sweep timer's trimmed mean drops the outer fifth on each side
    (median below five repetitions); a full configuration maps to the key
    of its label point (threads per row only for CSR and BSR, block size
    only for BSR), and every label point maps to itself."""
    from paper_2302_05662_gb300 import sweep
    assert sweep.summarize([5.0, 1.0, 3.0], "trimmed") == 3.0
    assert sweep.summarize([1.0, 2.0, 3.0, 4.0, 100.0], "median") == 3.0
    assert sweep.summarize([1.0, 2.0, 3.0, 4.0, 100.0], "trimmed") == 3.0      # drops 1 and 100
    assert abs(sweep.summarize([8.83, 10.88, 8.83, 10.88, 8.83, 10.88, 8.83, 10.88, 8.83, 10.88], "trimmed")
               - 9.855) < 1e-9
    full = dict(format=5, threads_per_block=64, threads_per_row=1, unroll=8, regcap=64, carveout=-1,
                bsr_block=1, hyb_ell_width=128)
    assert sweep.label_key(full) == "format=5,threads_per_block=64"
    full_bsr = dict(full, format=4, threads_per_row=4, bsr_block=4)
    assert sweep.label_key(full_bsr) == "bsr_block=4,format=4,threads_per_block=64,threads_per_row=4"
    for c in sweep.label_space(include_sell=True):
        d = dict(dict(threads_per_row=0, bsr_block=0), **c)
        assert sweep.label_key(d) == sweep.config_key(c)
