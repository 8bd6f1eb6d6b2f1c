"""Contraction-tree search ranked by predicted contraction time.

The paper searches contraction orders with the multiple-amplitude cost S_k
of main text Eq. (1) as the loss and refines the sliced set by lifetime
(SM Sec. IV.A-B).  On GB300 the steps are bound by their bytes and shapes
more than by their flops (a tree with 3x fewer Eq. (1) flops ran 2x slower),
so this search ranks candidate trees by the time the learned cost model
predicts for their steps:

1. candidates: the seeded random-greedy trees of ``rqc.tree.candidate_trees``
   and the neighbours of a start tree under *rotations* -- a node v = (x, y)
   with y = (y1, y2) becomes ((x, y1), y2) or ((x, y2), y1), the two other
   ways of pairing its three subtrees;
2. a cheap filter: the candidate is sliced under the rank cap
   (``rqc.tree.choose_slices``) and kept if its Eq. (1) flops stay within a
   factor of the best seen;
3. the ranking: the candidate is planned on the host (``tn.Plan``: instance
   DAG, step shapes, runs), every (step, configuration) pair is scored by the
   cost model (``Trainer.predict``: log2 ms per pass), each step takes its
   fastest allowed configuration, and the predicted time is the sum over
   steps of that time x the step's passes;
4. a hill climb over rotations accepts a neighbour whose predicted time is
   lower, from the best-ranked start;
5. the best few are measured (plan, bind, autotune, contract) against the
   start tree, so the choice rests on measured time.

``python -m paper_2212_04749_gb300.treesearch --workload diamond53_m12``
prints the ranking and the measurements as JSON.
"""

import json
import time
from typing import Dict, List, Optional, Tuple

import numpy as np

from . import costmodel, tn


def _children(ssa: np.ndarray, T: int) -> Dict[int, Tuple[int, int]]:
    return {T + i: (int(a), int(b)) for i, (a, b) in enumerate(np.asarray(ssa).reshape(-1, 2))}


def _to_ssa(ch: Dict[int, Tuple[int, int]], root: int, T: int) -> np.ndarray:
    """SSA pair list of a tree given as children per internal node: post
    order from the root, internal nodes renumbered T, T+1, ... as they close."""
    out: List[Tuple[int, int]] = []
    ids: Dict[int, int] = {}
    stack = [(root, False)]
    while stack:
        v, done = stack.pop()
        if v < T:
            continue
        if done:
            a, b = ch[v]
            out.append((ids.get(a, a), ids.get(b, b)))
            ids[v] = T + len(out) - 1
        else:
            stack.append((v, True))
            a, b = ch[v]
            stack.append((b, False))
            stack.append((a, False))
    return np.asarray(out, np.int64)


def rotations(ssa: np.ndarray, T: int) -> List[np.ndarray]:
    """Every tree one rotation away: for each internal v = (x, y) with y
    internal, the two re-pairings ((x, y1), y2) and ((x, y2), y1), with x and
    y taken in both orders."""
    ch = _children(ssa, T)
    root = 2 * T - 2
    out = []
    for v, (p, q) in ch.items():
        for x, y in ((p, q), (q, p)):
            if y < T:
                continue
            y1, y2 = ch[y]
            for keep, move in ((y2, y1), (y1, y2)):
                nch = dict(ch)
                nch[y] = (x, move)   # y now pairs x with one of its children
                nch[v] = (y, keep)   # v pairs that with the other
                out.append(_to_ssa(nch, root, T))
    return out


class Ranker:
    """Predicted contraction time of a tree for one workload."""

    def __init__(self, circuit, bits, struct, trainer: costmodel.Trainer, precision: str,
                 max_rank: Optional[int], workspace_limit: int):
        self.circuit, self.bits, self.struct = circuit, bits, struct
        self.k = bits.shape[0]
        self.trainer, self.precision = trainer, precision
        self.max_rank, self.limit = max_rank, workspace_limit
        # roofline rates (GB/s, algorithmic TFLOP/s): the measured copy rate,
        # BF16x3 = the measured BF16 rate / 3 products (TF32 about twice
        # that), the measured FP32 FMA rate
        self.hbm_gbs, self.fp32_tflops = 6780.0, 65.0
        self.tensor_tflops = 1700.0 / 3 if precision == "bf16x3" else 1050.0

    def slice(self, ssa):
        from rqc.tree import ContractionTree, choose_slices, estimate_cost
        c = estimate_cost(self.struct, ssa, self.k)
        sl = []
        if self.max_rank is not None and c.max_rank > self.max_rank:
            sl = choose_slices(self.struct, ContractionTree(ssa=ssa), self.k, None, self.max_rank)
            c = estimate_cost(self.struct, ssa, self.k, sl)
        return sl, c

    def predict(self, ssa, sl) -> Optional[dict]:
        try:
            p = tn.Plan(self.circuit, self.bits, ssa, sl, workspace_limit=self.limit, fuse=0)
        except tn.TnError:
            return None  # does not fit the workspace limit
        n = p.info["n_steps"]
        steps = p.tn_plan_steps()
        runs = np.array([s["runs"] for s in steps], np.float64)
        feats, ok = [], []
        for c in range(tn.TN_NCONFIG):
            f, e = p.tn_plan_features(self.precision, c)
            feats.append(f)
            ok.append(e)
        y = self.trainer.predict(np.concatenate(feats)).reshape(tn.TN_NCONFIG, n)
        # no configuration beats its roofline: the prediction is floored at
        # the step's bytes at the HBM rate and its flops at the rate of the
        # configuration's unit (tensor cores for a GEMM step they can take)
        by = np.array([s["bytes"] for s in steps], np.float64) / (self.hbm_gbs * 1e6)
        fl = np.array([s["flops"] for s in steps], np.float64)
        tc_ok = np.array([s["kb"] >= 3 and 6 <= s["mb"] <= 30 for s in steps])
        floor = np.empty((tn.TN_NCONFIG, n))
        for c in range(tn.TN_NCONFIG):
            rate = np.where((c >= 2) & tc_ok & (self.precision != "fp32"), self.tensor_tflops, self.fp32_tflops)
            floor[c] = np.maximum(by, fl / (rate * 1e9))
        ms = np.where(np.stack(ok), np.maximum(2.0 ** y, floor), np.inf).min(axis=0)
        info = p.info
        return {"predicted_ms": float(np.sum(ms * runs)), "flops_eq1": info["flops_ma"],
                "bytes": info["bytes_min"], "workspace_gib": info["workspace_bytes"] / 2 ** 30,
                "max_rank": info["max_rank"], "n_sliced": len(sl)}


def measure(circuit, bits, ssa, sl, precision, workspace_limit, reps=3) -> Optional[float]:
    """Contraction time (ms, CUDA events, median of reps) after the
    exhaustive autotuner configured the plan."""
    import torch
    try:
        p = tn.Plan(circuit, bits, ssa, sl, workspace_limit=workspace_limit, fuse=0)
    except tn.TnError:
        return None
    ws = torch.empty(p.info["workspace_bytes"], dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    p.tn_plan_bind(ws, stream=st)
    amps = torch.zeros(2 * bits.shape[0], dtype=torch.float64, device="cuda")
    p.tn_plan_autotune(precision, amps, reps=1, stream=st)
    ts = []
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        p.tn_contract(amps, precision, stream=st)
        e1.record(st)
        e1.synchronize()
        if r:
            ts.append(e0.elapsed_time(e1))
    p.tn_plan_check(stream=st)
    p._ws = None
    del ws, amps, p
    torch.cuda.empty_cache()
    return float(np.median(ts))


def search(ranker: Ranker, start: np.ndarray, seeds=(), trials=16, steps=40, flops_slack=1.5, per_step=150,
           log=None):
    """Rank the start tree and the random-greedy candidates, then hill-climb
    over rotations from the best (per step at most per_step seeded random
    neighbours, first improvement taken); returns every ranked tree, best
    first."""
    from rqc.tree import candidate_trees
    T = ranker.struct.n_tensors
    seen = {}

    def rank(ssa):
        key = np.asarray(ssa).tobytes()
        if key in seen:
            return seen[key]
        sl, c = ranker.slice(ssa)
        r = None
        if ranker.max_rank is None or c.max_rank <= ranker.max_rank:
            r = ranker.predict(ssa, sl)
            if r is not None:
                r.update({"ssa": np.asarray(ssa).tolist(), "sliced": [int(e) for e in sl]})
        seen[key] = r
        return r

    ranked = [rank(start)]
    for sd in seeds:
        for ssa in candidate_trees(ranker.struct, ranker.k, sd, trials):
            ranked.append(rank(ssa))
    ranked = [r for r in ranked if r is not None]
    best = min(ranked, key=lambda r: r["predicted_ms"])
    if log:
        log(f"start {ranked[0]['predicted_ms']:.1f} ms predicted; best of {len(ranked)} candidates "
            f"{best['predicted_ms']:.1f} ms")
    for it in range(steps):
        cur = np.asarray(best["ssa"])
        from rqc.tree import estimate_cost
        base_flops = estimate_cost(ranker.struct, cur, ranker.k).flops
        improved = False
        nbrs = rotations(cur, T)
        order = np.random.default_rng(it).permutation(len(nbrs))[:per_step]
        for j in order:
            ssa = nbrs[j]
            if estimate_cost(ranker.struct, ssa, ranker.k).flops > flops_slack * base_flops:
                continue
            r = rank(ssa)
            if r is not None and r["predicted_ms"] < best["predicted_ms"] * (1 - 1e-3):
                best = r
                improved = True
                break
        if log:
            log(f"climb {it}: {best['predicted_ms']:.1f} ms predicted, {len(seen)} trees ranked")
        if not improved:
            break
    out = [r for r in seen.values() if r is not None]
    out.sort(key=lambda r: r["predicted_ms"])
    return out


def measured_climb(ranker: Ranker, start: np.ndarray, measure_fn, steps=20, per_step=150, k_measure=4,
                   flops_slack=1.5, min_gain=0.01, explore=0, seed=0, log=None):
    """Hill climb that moves only on measured time: per step, up to
    per_step seeded random rotations of the current tree are ranked by the
    cost model, the k_measure best (distinct predictions) and `explore`
    more drawn at random from the rest are measured, and the best of them
    replaces the current tree if it is at least min_gain faster.  Returns
    the walk: every measured tree with its times."""
    from rqc.tree import estimate_cost
    T = ranker.struct.n_tensors
    sl, _ = ranker.slice(start)
    cur = {"ssa": np.asarray(start).tolist(), "sliced": [int(e) for e in sl]}
    cur["measured_ms"] = measure_fn(np.asarray(start), cur["sliced"])
    walk = [dict(cur, step=-1)]
    seen = {np.asarray(start).tobytes()}
    if cur["measured_ms"] is None:  # the start tree does not plan within the workspace limit
        if log:
            log("measured climb: the start tree cannot be planned within the workspace limit")
        return cur, walk
    if log:
        log(f"measured climb: start {cur['measured_ms']:.2f} ms")
    for it in range(steps):
        base = np.asarray(cur["ssa"])
        base_flops = estimate_cost(ranker.struct, base, ranker.k).flops
        nbrs = rotations(base, T)
        cands = []
        for j in np.random.default_rng([seed, 1000 + it]).permutation(len(nbrs))[:per_step]:
            ssa = nbrs[j]
            key = ssa.tobytes()
            if key in seen or estimate_cost(ranker.struct, ssa, ranker.k).flops > flops_slack * base_flops:
                continue
            seen.add(key)
            sl2, c = ranker.slice(ssa)
            if ranker.max_rank is not None and c.max_rank > ranker.max_rank:
                continue
            r = ranker.predict(ssa, sl2)
            if r is not None:
                r.update({"ssa": ssa.tolist(), "sliced": [int(e) for e in sl2]})
                cands.append(r)
        cands.sort(key=lambda r: r["predicted_ms"])
        picked, preds = [], set()
        rest = []
        for r in cands:
            key = round(r["predicted_ms"], 3)
            if key in preds:
                continue
            preds.add(key)
            if len(picked) < k_measure:
                picked.append(r)
            else:
                rest.append(r)
        # a few more at random: the ones the model ranks wrongly
        if explore > 0 and rest:
            for j in np.random.default_rng([seed, 2000 + it]).permutation(len(rest))[:explore]:
                picked.append(rest[j])
        best = None
        for r in picked:
            r["measured_ms"] = measure_fn(np.asarray(r["ssa"]), r["sliced"])
            walk.append(dict(r, step=it))
            if r["measured_ms"] is not None and (best is None or r["measured_ms"] < best["measured_ms"]):
                best = r
        moved = best is not None and best["measured_ms"] < cur["measured_ms"] * (1 - min_gain)
        if moved:
            cur = best
        if log:
            log(f"measured climb {it}: {len(picked)} measured, best {best['measured_ms'] if best else None} ms, "
                f"current {cur['measured_ms']:.2f} ms")
        if not moved:
            break
    return cur, walk


def kick(ranker: Ranker, start: np.ndarray, moves: int, seed: int, flops_slack=1.5) -> np.ndarray:
    """`moves` seeded random rotations in a row, each keeping the estimated
    flops within flops_slack of the start tree's and the rank cap."""
    from rqc.tree import estimate_cost
    T = ranker.struct.n_tensors
    rng = np.random.default_rng([seed, 7])
    base = estimate_cost(ranker.struct, start, ranker.k).flops
    cur = np.asarray(start)
    for _ in range(moves):
        nbrs = rotations(cur, T)
        for j in rng.permutation(len(nbrs)):
            c = estimate_cost(ranker.struct, nbrs[j], ranker.k)
            if c.flops <= flops_slack * base and (ranker.max_rank is None or c.max_rank <= ranker.max_rank):
                cur = nbrs[j]
                break
    return cur


def main():
    import argparse
    import torch
    from rqc import make_workload
    ap = argparse.ArgumentParser(description="contraction-tree search ranked by the cost model's predicted time")
    ap.add_argument("--workload", default="diamond53_m12")
    ap.add_argument("--precision", default="bf16x3")
    ap.add_argument("--cases", type=int, default=40, help="random plans for the cost model's corpus")
    ap.add_argument("--budget-s", type=float, default=90.0)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--seeds", default="3004,3104,3204")
    ap.add_argument("--climb", type=int, default=40)
    ap.add_argument("--measure", type=int, default=3, help="measure the best N predicted trees")
    ap.add_argument("--ws-gib", type=float, default=120.0)
    ap.add_argument("--per-step", type=int, default=150, help="rotations tried per climb step")
    ap.add_argument("--start", default=None, help="JSON with a start tree (its 'ssa' and 'sliced', e.g. "
                                                    "an earlier --out's 'best')")
    ap.add_argument("--out", default=None)
    ap.add_argument("--measured-climb", type=int, default=0,
                    help="instead of ranking by prediction alone: hill-climb from the start tree, measuring the "
                         "N best predicted rotations per step and moving only on a measured gain")
    ap.add_argument("--min-gain", type=float, default=0.01, help="measured climb: smallest relative gain to move")
    ap.add_argument("--climb-seed", type=int, default=0, help="measured climb: seed of the rotations it samples")
    ap.add_argument("--kick", type=int, default=0,
                    help="measured climb: start from this many seeded random rotations (within the flops slack) "
                         "of the start tree, to leave its local optimum")
    ap.add_argument("--explore", type=int, default=0,
                    help="measured climb: rotations measured per step beyond the best predicted, drawn at random")
    args = ap.parse_args()
    torch.cuda.init()
    log = lambda m: print(m, flush=True)  # noqa: E731
    w = make_workload(args.workload)
    limit = int(args.ws_gib * 2 ** 30)
    # corpus: the workload's own steps under its start tree, then random plans
    corpus = costmodel.Corpus()
    b = costmodel.bind(costmodel.workload_case(args.workload), ws_limit=limit)
    if b is not None:
        X, y, _ = costmodel.autotune_rows(b, args.precision)
        corpus.add(X, y, -1)
        del b
        torch.cuda.empty_cache()
    costmodel.collect([costmodel.random_case(s) for s in range(args.cases)], corpus, precisions=(args.precision,),
                      reps=1, log=None, budget_s=args.budget_s, flops_range=(1e8, 1e15))
    tr = costmodel.Trainer(seed=0)
    tr.fit(corpus.X, corpus.y, epochs=args.epochs)
    log(f"cost model: {len(corpus.y)} timings")
    ranker = Ranker(w.circuit, w.bits, w.struct, tr, args.precision, w.spec.max_rank, limit)
    t0 = time.time()
    start = np.asarray(w.tree.ssa)
    if args.start:
        with open(args.start) as f:
            st = json.load(f)
        start = np.asarray(st.get("best", st)["ssa"])
    if args.measured_climb > 0:
        mfn = lambda ssa, sl: measure(w.circuit, w.bits, ssa, sl, args.precision, limit)  # noqa: E731
        if args.kick > 0:
            start = kick(ranker, start, args.kick, args.climb_seed)
        best, walk = measured_climb(ranker, start, mfn, steps=args.climb, per_step=args.per_step,
                                    k_measure=args.measured_climb, min_gain=args.min_gain, explore=args.explore,
                                    seed=args.climb_seed, log=log)
        res = {"workload": args.workload, "precision": args.precision, "search_s": time.time() - t0,
               "corpus_rows": int(len(corpus.y)), "start_ms": walk[0]["measured_ms"],
               "best_ms": best["measured_ms"], "measured": [{k: v for k, v in r.items() if k != "ssa"} for r in walk],
               "best": best}
        if args.out:
            with open(args.out, "w") as f:
                json.dump(res, f)
        print(json.dumps({k: v for k, v in res.items() if k not in ("best", "measured")}))
        return
    ranked = search(ranker, start, seeds=[int(s) for s in args.seeds.split(",") if s],
                    steps=args.climb, per_step=args.per_step, log=log)
    search_s = time.time() - t0
    start_key = np.asarray(w.tree.ssa).tolist()  # the workload's own tree is always measured
    res = {"workload": args.workload, "precision": args.precision, "ranked": len(ranked), "search_s": search_s,
           "corpus_rows": int(len(corpus.y)), "measured": []}
    todo = ranked[:args.measure]
    if not any(r["ssa"] == start_key for r in todo):
        own = [r for r in ranked if r["ssa"] == start_key][:1]
        if not own:
            sl, _ = ranker.slice(np.asarray(w.tree.ssa))
            r = ranker.predict(np.asarray(w.tree.ssa), sl)
            if r is not None:
                r.update({"ssa": start_key, "sliced": [int(e) for e in sl]})
                own = [r]
        todo = todo + own
    for r in todo:
        ms = measure(w.circuit, w.bits, np.asarray(r["ssa"]), r["sliced"], args.precision, limit)
        rec = {k: v for k, v in r.items() if k != "ssa"}
        rec["measured_ms"] = ms
        rec["is_start_tree"] = r["ssa"] == start_key
        res["measured"].append(rec)
        log(json.dumps(rec))
    if args.out:
        best = min((m for m in zip(todo, res["measured"]) if m[1]["measured_ms"]), key=lambda m: m[1]["measured_ms"])
        res["best"] = {"ssa": best[0]["ssa"], "sliced": best[0]["sliced"], **best[1]}
        with open(args.out, "w") as f:
            json.dump(res, f)
    print(json.dumps({k: v for k, v in res.items() if k != "best"}))


if __name__ == "__main__":
    main()
