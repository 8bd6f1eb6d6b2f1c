"""Learned configuration selection for the contraction steps.

The exhaustive autotuner (``tn_plan_autotune``) measures every kernel
configuration of every step; the cost model learns those timings so that a
new plan can be configured without measuring it:

1. ``collect``: for seeded plans (the synthetic workloads' trees plus random
   trees on random 20-53-qubit Sycamore-style circuits), run the autotuner
   and keep one row per measured (step, configuration, precision): the
   step's ``tn_plan_features`` and log2 of its time per pass.
2. ``Trainer``: the MLP of ``tn_mlp_*`` (TN_MLP_IN -> 128 -> 128 -> 1),
   trained on the GPU by the library's own forward/backward and Adam
   kernels on mini-batches of the corpus (mean squared error in log2 time).
3. ``select``: FP16 copy of the network -> ``tn_plan_select`` picks each
   step's predicted fastest configuration; steps whose two best predictions
   are within a margin go to the autotuner (``tn_plan_autotune`` with a
   step mask) -- the fallback.
4. ``evaluate``: end-to-end contraction time under the plan's built-in
   rule, the cost model's choice and the exhaustive autotuner's choice; the
   regret is the model's time over the autotuner's.

Everything numeric on the device runs in the library's kernels; this module
only orders the calls and holds the buffers (torch tensors).
"""

import json
import time
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import tn

PRECS = ("fp32", "bf16x3")


@dataclass
class Case:
    name: str
    circuit: object
    bits: np.ndarray
    ssa: np.ndarray
    sliced: List[int]
    seed: int


def random_case(seed: int, max_rank_choices=(20, 22, 24)) -> Case:
    """A random Sycamore-style circuit on a 20-53-qubit layout with a seeded
    random-greedy tree, sliced under a rank cap (small enough to contract in
    well under a second)."""
    from rqc import diamond_layout, grid_layout, network_structure, random_circuit
    from rqc.bitstrings import uniform_bitstrings
    from rqc.tree import ContractionTree, candidate_trees, choose_slices
    rng = np.random.default_rng([7001, seed])
    if rng.random() < 0.15:
        lay, name = diamond_layout(), "diamond53"
    else:
        while True:
            r, c = int(rng.integers(4, 8)), int(rng.integers(5, 9))
            if 20 <= r * c <= 53:
                break
        lay, name = grid_layout(r, c), f"grid{r}x{c}"
    cycles = int(rng.integers(4, 9))
    circ = random_circuit(lay, cycles, seed=int(rng.integers(1 << 30)))
    n = circ.n_qubits
    k = int(2 ** rng.integers(4, 12))
    bits = uniform_bitstrings(n, k, seed=int(rng.integers(1 << 30)))
    st = network_structure(circ)
    ssa = candidate_trees(st, k, seed=int(rng.integers(1 << 30)), trials=1)[int(rng.integers(0, 2))]
    cap = int(rng.choice(max_rank_choices))
    sliced = choose_slices(st, ContractionTree(ssa=ssa), k, max_rank=cap)
    return Case(f"{name}_m{cycles}_k{k}_r{cap}", circ, bits, ssa, sliced, seed)


def workload_case(name: str) -> Case:
    from rqc import make_workload
    w = make_workload(name)
    return Case(name, w.circuit, w.bits, w.tree.ssa, list(w.tree.sliced), -1)


@dataclass
class Bound:
    """A plan bound to a device workspace, with an amplitude buffer."""
    case: Case
    plan: object
    ws: object
    amps: object
    stream: object


def bind(case: Case, ws_limit: int = 4 << 30) -> Optional[Bound]:
    """Plan and bind a case (None if it needs more than ws_limit bytes)."""
    import torch
    try:
        p = tn.Plan(case.circuit, case.bits, case.ssa, case.sliced, workspace_limit=ws_limit)
    except tn.TnError:
        return None
    info = p.info
    ws = torch.empty(info["workspace_bytes"], dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    p.tn_plan_bind(ws, stream=st)
    amps = torch.zeros(2 * max(p.k, 1), dtype=torch.float64, device="cuda")
    return Bound(case, p, ws, amps, st)


@dataclass
class Corpus:
    X: np.ndarray = field(default_factory=lambda: np.zeros((0, tn.TN_NFEAT), np.float32))
    y: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float32))
    group: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))  # case seed of each row

    def add(self, X, y, g):
        self.X = np.concatenate([self.X, X.astype(np.float32)])
        self.y = np.concatenate([self.y, y.astype(np.float32)])
        self.group = np.concatenate([self.group, np.full(len(y), g, np.int64)])

    def save(self, path):
        np.savez_compressed(path, X=self.X, y=self.y, group=self.group)

    @staticmethod
    def load(path):
        d = np.load(path)
        return Corpus(d["X"], d["y"], d["group"])


def autotune_rows(b: Bound, precision: str, reps: int = 2):
    """Run the exhaustive autotuner on a bound plan; return (X, log2 ms per
    pass) for every measured (step, configuration) and the times table."""
    times = b.plan.tn_plan_autotune(precision, b.amps, reps=reps, stream=b.stream)
    Xs, ys = [], []
    for c in range(tn.TN_NCONFIG):
        f, _ = b.plan.tn_plan_features(precision, c)
        ok = np.isfinite(times[:, c]) & (times[:, c] > 0)
        Xs.append(f[ok])
        ys.append(np.log2(times[ok, c]))
    return np.concatenate(Xs), np.concatenate(ys), times


def collect(cases, corpus: Corpus, precisions=PRECS, reps: int = 2, log=None, budget_s: float = 1e9,
            flops_range=(0.0, float("inf"))):
    """Autotune every case whose executed flops lie in flops_range (plans
    that do not fit the workspace limit are skipped) until budget_s."""
    t0 = time.time()
    for case in cases:
        if time.time() - t0 > budget_s:
            break
        b = bind(case)
        if b is None:
            continue
        if not flops_range[0] <= b.plan.info["flops_exec"] <= flops_range[1]:
            del b
            continue
        for prec in precisions:
            X, y, _ = autotune_rows(b, prec, reps)
            corpus.add(X, y, case.seed)
        if log:
            log(f"{case.name}: {len(corpus.y)} rows, {time.time() - t0:.1f} s")
        del b
    return corpus


class Trainer:
    """The cost-model network on the device, trained by tn_mlp_grad + tn_mlp_adam."""

    def __init__(self, seed: int = 0):
        import torch
        rng = np.random.default_rng(seed)
        D, H = tn.TN_MLP_IN, tn.TN_MLP_HIDDEN
        p = np.concatenate([
            rng.uniform(-1, 1, H * D) * np.sqrt(6.0 / D), np.zeros(H),
            rng.uniform(-1, 1, H * H) * np.sqrt(6.0 / H), np.zeros(H),
            rng.uniform(-1, 1, H) * np.sqrt(3.0 / H), np.zeros(1)]).astype(np.float32)
        dev = "cuda"
        self.params = torch.from_numpy(p).to(dev)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self.params16 = torch.zeros(tn.TN_MLP_NPARAMS, dtype=torch.int16, device=dev)
        self.step = 0

    def fit(self, X: np.ndarray, y: np.ndarray, epochs: int = 200, batch: int = 4096, lr: float = 2e-3,
            seed: int = 0, log=None):
        import torch
        rng = np.random.default_rng(seed)
        order = rng.permutation(len(y))
        Xd = torch.from_numpy(np.ascontiguousarray(X[order], np.float32)).cuda()
        yd = torch.from_numpy(np.ascontiguousarray(y[order], np.float32)).cuda()
        n = len(y)
        batch = min(batch, n)
        if self.step == 0:  # start the output bias at the target mean
            self.params[tn.TN_MLP_NPARAMS - 1] = float(np.mean(y))
        scratch = torch.empty(tn.tn_mlp_grad_scratch_bytes(batch), dtype=torch.uint8, device="cuda")
        st = torch.cuda.current_stream()
        D = tn.TN_MLP_IN
        hist = []
        for ep in range(epochs):
            lr_e = lr * (0.5 * (1 + np.cos(np.pi * ep / epochs)) * 0.9 + 0.1)
            for s0 in range(0, n - batch + 1, batch):
                Xb = Xd.data_ptr() + 4 * s0 * D
                tb = yd.data_ptr() + 4 * s0
                tn.tn_mlp_grad(self.params, Xb, tb, batch, self.grad, self.loss, scratch, stream=st)
                self.step += 1
                tn.tn_mlp_adam(self.params, self.grad, self.m, self.v, self.step, lr=lr_e, stream=st)
            if log and (ep % max(1, epochs // 10) == 0 or ep == epochs - 1):
                torch.cuda.synchronize()
                hist.append(float(self.loss.item()))
                log(f"epoch {ep}: batch loss {hist[-1]:.4f}")
        torch.cuda.synchronize()
        return hist

    def save(self, path):
        np.save(path, self.params.cpu().numpy())

    @classmethod
    def load(cls, path):
        import torch
        tr = cls()
        tr.params.copy_(torch.from_numpy(np.load(path).astype(np.float32)))
        tr.step = 1
        return tr

    def predict(self, X: np.ndarray, f16: bool = False) -> np.ndarray:
        import torch
        Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
        y = torch.empty(len(X), dtype=torch.float32, device="cuda")
        st = torch.cuda.current_stream()
        if f16:
            tn.tn_mlp_to_half(self.params, self.params16, stream=st)
            tn.tn_mlp_forward_f16(self.params16, Xd, len(X), y, stream=st)
        else:
            tn.tn_mlp_forward(self.params, Xd, len(X), y, stream=st)
        torch.cuda.synchronize()
        return y.cpu().numpy()

    def half(self):
        tn.tn_mlp_to_half(self.params, self.params16)
        return self.params16


def select(b: Bound, precision: str, trainer: Trainer, margin: float = 0.0, fallback: bool = False):
    """Configure every step of a bound plan with the cost model; with
    fallback, steps whose two best predictions are within `margin` are
    re-decided by the autotuner.  Returns (uncertain flags, seconds)."""
    import torch
    t0 = time.perf_counter()
    ns = b.plan.info["n_steps"]
    scratch = torch.empty(ns * tn.TN_NCONFIG * (tn.TN_NFEAT + 1) * 4, dtype=torch.uint8, device="cuda")
    unc = b.plan.tn_plan_select(precision, trainer.half(), scratch, margin=margin, stream=b.stream)
    if fallback and unc.any():
        b.plan.tn_plan_autotune(precision, b.amps, reps=1, step_mask=unc.astype(np.uint8), stream=b.stream)
    return unc, time.perf_counter() - t0


def contraction_ms(b: Bound, precision: str, reps: int = 3) -> float:
    import torch
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b.plan.tn_contract(b.amps, precision, stream=b.stream)  # warm-up
    ts = []
    for _ in range(reps):
        ev0.record(b.stream)
        b.plan.tn_contract(b.amps, precision, stream=b.stream)
        ev1.record(b.stream)
        ev1.synchronize()
        ts.append(ev0.elapsed_time(ev1))
    return float(np.median(ts))


def evaluate(b: Bound, precision: str, trainer: Trainer, reps: int = 3, margin: float = 0.0,
             hybrid_margin: float = 0.2) -> dict:
    """End-to-end times (ms) under the plan's rule, the cost model and the
    exhaustive autotuner, plus the time each selection took."""
    ns = b.plan.info["n_steps"]
    for s in range(ns):
        b.plan.tn_plan_set_config(s, -1)
    t_rule = contraction_ms(b, precision, reps)
    _, sel_s = select(b, precision, trainer, margin=margin)
    cfg_model = b.plan.tn_plan_get_configs().copy()
    t_model = contraction_ms(b, precision, reps)
    # the network with the autotuner as its fallback: steps whose two best
    # predictions lie within hybrid_margin (log2 ms) are timed instead
    for s in range(ns):
        b.plan.tn_plan_set_config(s, -1)
    unc, hyb_s = select(b, precision, trainer, margin=hybrid_margin, fallback=True)
    t_hybrid = contraction_ms(b, precision, reps)
    t0 = time.perf_counter()
    table = b.plan.tn_plan_autotune(precision, b.amps, reps=2, stream=b.stream)
    tune_s = time.perf_counter() - t0
    cfg_tuned = b.plan.tn_plan_get_configs().copy()
    t_tuned = contraction_ms(b, precision, reps)
    # regret on the measured table: the model's per-step choice against the best
    runs = np.array([s["runs"] for s in b.plan.tn_plan_steps()])
    best = np.nanmin(table, axis=1)
    chosen = table[np.arange(ns), cfg_model]
    ok = np.isfinite(chosen) & np.isfinite(best)
    table_regret = float(np.sum((chosen[ok] - best[ok]) * runs[ok]) / max(np.sum(best[ok] * runs[ok]), 1e-12))
    return {"case": b.case.name, "precision": precision, "steps": ns, "rule_ms": t_rule, "model_ms": t_model,
            "tuned_ms": t_tuned, "model_select_s": sel_s, "autotune_s": tune_s,
            "regret_vs_tuned": t_model / t_tuned - 1.0, "gain_vs_rule": t_rule / t_model - 1.0,
            "table_regret": table_regret, "agree_with_tuned": float(np.mean(cfg_model == cfg_tuned)),
            "hybrid_ms": t_hybrid, "hybrid_select_s": hyb_s, "uncertain_frac": float(np.mean(unc))}


def main():
    import argparse
    import torch
    ap = argparse.ArgumentParser(description="collect autotuner timings, train the cost model, report regret")
    ap.add_argument("--cases", type=int, default=60, help="random plans for the corpus")
    ap.add_argument("--eval-cases", type=int, default=6, help="held-out random plans")
    ap.add_argument("--workloads", default="grid3x4_m8,grid5x6_m14,grid6x7_m10",
                    help="named workloads added to the corpus")
    ap.add_argument("--workload-ws-gib", type=float, default=96.0)
    ap.add_argument("--budget-s", type=float, default=600.0, help="corpus collection time bound")
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--corpus", default=None, help="save the corpus (npz) here")
    ap.add_argument("--out", default=None, help="write the JSON report here")
    ap.add_argument("--save-model", default=None, help="save the trained parameters (npy) here")
    ap.add_argument("--precisions", default="fp32,bf16x3,tf32")
    args = ap.parse_args()
    torch.cuda.init()
    log = lambda m: print(m, flush=True)  # noqa: E731
    precs = tuple(args.precisions.split(","))
    corpus = Corpus()
    # the named workloads (bound with room for their full workspace; the
    # autotuner times one slice batch), then random plans
    for wi, w in enumerate([x for x in args.workloads.split(",") if x]):
        b = bind(workload_case(w), ws_limit=int(args.workload_ws_gib * 2 ** 30))
        if b is None:
            log(f"{w}: does not fit, skipped")
            continue
        for prec in precs:
            X, y, _ = autotune_rows(b, prec)
            corpus.add(X, y, -1 - wi)
        log(f"{w}: {len(corpus.y)} rows")
        del b
    cases = [random_case(s) for s in range(args.cases)]
    collect(cases, corpus, precisions=precs, log=log, budget_s=args.budget_s, flops_range=(1e8, 1e15))
    if args.corpus:
        corpus.save(args.corpus)
    # 80/20 split by case seed
    seeds = np.unique(corpus.group)
    val = set(seeds[(np.arange(len(seeds)) % 5) == 4].tolist())
    vm = np.array([g in val for g in corpus.group])
    tr = Trainer(seed=0)
    hist = tr.fit(corpus.X[~vm], corpus.y[~vm], epochs=args.epochs, log=log)
    if args.save_model:
        tr.save(args.save_model)
    pv = tr.predict(corpus.X[vm]) if vm.any() else np.zeros(0)
    val_mse = float(np.mean((pv - corpus.y[vm]) ** 2)) if vm.any() else None
    evals = []
    n_eval = 0
    for s in range(10000, 10400):
        if n_eval >= args.eval_cases:
            break
        b = bind(random_case(s))
        if b is None:
            continue
        if not 1e10 <= b.plan.info["flops_exec"] <= 2e12:  # plans where the configuration matters
            del b
            continue
        n_eval += 1
        for prec in precs:
            evals.append(evaluate(b, prec, tr))
            log(json.dumps(evals[-1]))
        del b
    rep = {"rows": int(len(corpus.y)), "train_rows": int((~vm).sum()), "val_rows": int(vm.sum()),
           "val_mse_log2": val_mse, "loss_history": hist, "eval": evals,
           "mean_regret_vs_tuned": float(np.mean([e["regret_vs_tuned"] for e in evals])) if evals else None,
           "mean_gain_vs_rule": float(np.mean([e["gain_vs_rule"] for e in evals])) if evals else None}
    if args.out:
        with open(args.out, "w") as f:
            json.dump(rep, f, indent=1)
    print(json.dumps({k: v for k, v in rep.items() if k not in ("eval", "loss_history")}))


if __name__ == "__main__":
    main()
