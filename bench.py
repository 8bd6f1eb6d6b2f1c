"""Throughput of the multiple-amplitude contraction on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload grid5x6_m14] [--precision fp32|tf32|bf16x3]

One step = one full tn_contract over every slice batch of the workload's
plan: the amplitudes of all its bitstrings (30 qubits, 14 cycles, 4096
bitstrings, 2^10 slices by default).  Prints one JSON line (rank 0).

value      amplitudes/s over all ranks: bitstrings x ranks / max-over-ranks
           device time (CUDA events around each tn_contract; inputs and
           plan resident in HBM; a 512 MiB write flushes L2 between steps).
e2e        the same metric through the public API from host data: tn_plan
           (host), tn_plan_bind (tables up), tn_contract, amplitudes down,
           timed on the host clock.
roofline   the kernel family with the largest share of device time,
           algorithmic bytes or flops / its measured launch time, against
           the measured peak.
cpu_baseline  the CPU oracle (state vector, complex128) on this host's
           cores, timed on a bounded sample of its gate passes.
--impl reference times that oracle as the reference arm.
Multi-GPU (torchrun): each rank contracts its own seeded bitstrings (weak
scaling, no collective on the data path).
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "amplitudes/sec & TFLOP/s (frac of peak), mixed vs FP32 at stated amp error"
UNIT = "amplitudes/s"
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None,
                "samples": len(rows), "reasons": reasons}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _bits_for_rank(w, rank):
    from rqc.bitstrings import uniform_bitstrings
    if rank == 0:
        return w.bits
    return uniform_bitstrings(w.circuit.n_qubits, w.bits.shape[0], seed=2000 + w.spec.index + 1000 * rank)


def _golden(name):
    path = os.path.join(ROOT, "tests", "golden", f"{name}_sv.txt")
    if not os.path.exists(path):
        return None
    vals = []
    for line in open(path):
        if not line.startswith("#"):
            re_, im_ = line.split()
            vals.append(complex(float(re_), float(im_)))
    return np.asarray(vals, np.complex128)


def cpu_oracle_sample(w, budget_s=20.0):
    """The complex128 state-vector oracle on a bounded sample: the state is
    evolved through the first g gates (g grown until ~budget_s of CPU work),
    and the full run's time is extrapolated per gate pass."""
    from oracle import sv as osv
    from rqc.circuit import Circuit
    total = len(w.circuit.gates)
    g = 8
    while True:
        c = Circuit(n_qubits=w.circuit.n_qubits, gates=w.circuit.gates[:g])
        t0 = time.perf_counter()
        osv.state(c)
        dt = time.perf_counter() - t0
        if dt > budget_s / 3 or g >= total:
            break
        g = min(total, max(g + 1, int(g * min(8.0, budget_s / 3 / max(dt, 1e-3)))))
    t_full = dt * (total + 1) / (g + 1)
    k = w.bits.shape[0]
    return {"value": k / t_full, "unit": UNIT, "cores": osv.threads(), "kind": "oracle",
            "sample": f"state-vector oracle (complex128, 2^{w.circuit.n_qubits} amplitudes) through the first "
                      f"{g} of {total} gates in {dt:.2f} s, extrapolated per gate pass to {t_full:.1f} s "
                      f"for the {k} bitstrings"}


def measure_correlated(w, precision, torch, tn, stream, ws, limit, rows=256, n_open=4, reps=3):
    """Correlated batches (SM Sec. II): `rows` of the workload's bitstrings
    with their last `n_open` qubits left open, so that one contraction
    yields rows x 2^n_open amplitudes (the same count as the headline
    batch when rows x 2^n_open = k), then one perfect sample per row
    (tn_sample_completions, uniform numbers drawn on the host, seed 5).
    CUDA-event time of the contraction (the plan's rule configuration)
    and of the sampling."""
    n = w.circuit.n_qubits
    oq = list(range(n - n_open, n))
    p = tn.Plan(w.circuit, w.bits[:rows], w.tree.ssa, w.tree.sliced, workspace_limit=min(limit, ws.numel()),
                open_qubits=oq)
    if p.info["workspace_bytes"] > ws.numel():
        return {"skipped": f"needs {p.info['workspace_bytes'] / 2**30:.1f} GiB"}
    p.tn_plan_bind(ws, stream=stream)
    m = rows << n_open
    amps = torch.zeros(2 * m, dtype=torch.float64, device="cuda")
    u = torch.from_numpy(np.random.default_rng(5).random(rows)).cuda()
    picks = torch.empty(rows, dtype=torch.int64, device="cuda")
    ts, tsamp = [], []
    for r in range(reps + 1):
        amps.zero_()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        p.tn_contract(amps, precision, stream=stream)
        e1.record(stream)
        tn.tn_sample_completions(amps, rows, n_open, u, picks, stream=stream)
        e2.record(stream)
        e2.synchronize()
        if r > 0:
            ts.append(e0.elapsed_time(e1))
            tsamp.append(e1.elapsed_time(e2))
    ms = statistics.mean(ts)
    return {"rows": rows, "open_qubits": oq, "amplitudes": m, "ms_per_contraction": ms,
            "amplitudes_per_s": m / (ms / 1000.0), "sampling_ms": statistics.mean(tsamp),
            "samples_per_s": rows / ((ms + statistics.mean(tsamp)) / 1000.0),
            "workspace_gib": p.info["workspace_bytes"] / 2 ** 30}


def measure_chain(name, precision, torch, tn, stream, fuse_bits, batches=4):
    """Fused chains (tn_options.fuse) against the unfused steps on a workload
    whose heaviest chain is worth fusing: per-step CUDA-event times over the
    first `batches` slice batches, the chain kernel's algorithmic bytes (A_1
    read, B_j reads, C_L write; its intermediates are never stored) and its
    HBM roofline."""
    from rqc import make_workload
    w = make_workload(name)
    peaks, _ = _peaks()
    plans = {f: tn.Plan(w.circuit, w.bits, w.tree.ssa, w.tree.sliced, workspace_limit=200 << 30, fuse=f,
                        fuse_max_bits=fuse_bits) for f in (0, 1)}
    need = max(p.info["workspace_bytes"] for p in plans.values())
    free, _ = torch.cuda.mem_get_info()
    if need > 0.9 * free:
        return {"workload": name, "skipped": f"needs {need / 2**30:.1f} GiB"}
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    amps = torch.zeros(2 * w.bits.shape[0], dtype=torch.float64, device="cuda")
    nb = min(batches, plans[1].info["n_batches"])
    res = {}
    for f, p in plans.items():
        p.tn_plan_bind(ws, stream=stream)
        p.tn_plan_profile(True)
        p.tn_contract(amps, precision, 0, nb, stream=stream)  # warm-up
        p.tn_contract(amps, precision, 0, nb, stream=stream)
        ms, fam = p.tn_plan_step_times()
        res[f] = (ms, fam, p.tn_plan_steps())
        p.tn_plan_profile(False)
    ms1, fam1, st1 = res[1]
    ms0, _, st0 = res[0]
    chains = {}
    for i, s in enumerate(st1):
        if s["chain"] >= 0:
            chains.setdefault(s["chain"], []).append(i)
    best = max(chains.values(), key=lambda ids: sum(ms0[i] for i in ids))
    t_unfused = float(sum(ms0[i] for i in best))
    t_fused = float(ms1[best[-1]])
    first, last = st1[best[0]], st1[best[-1]]
    # algorithmic bytes per pass: A_1 + every B_j + C_L
    a_bytes = 8.0 * first["n_inst_a"] * 2.0 ** first["rank_a"]
    b_bytes = sum(8.0 * st1[i]["n_inst_b"] * 2.0 ** st1[i]["rank_b"] for i in best)
    c_bytes = 8.0 * last["n_inst"] * 2.0 ** (last["mb"] + last["nb"])
    runs = sum(1 for b in range(nb) if b == 0 or st1[best[-1]]["level"] <= (b & -b).bit_length() - 1)
    alg = (a_bytes + b_bytes + c_bytes) * runs
    ach = alg / (t_fused / 1e3) / 1e9
    del ws
    torch.cuda.empty_cache()
    return {"workload": name, "precision": precision, "slice_batches": nb, "chains": len(chains), "d_t": fuse_bits,
            "heaviest_chain_steps": best, "unfused_ms": t_unfused, "fused_ms": t_fused,
            "speedup": t_unfused / t_fused if t_fused > 0 else None,
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": ach / peaks["hbm_gbs"], "algorithmic_bytes": alg, "kernel": "k_chain"}}


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    from rqc import make_workload
    w = make_workload(args.workload)
    vals = []
    for _ in range(args.warmup):
        cpu_oracle_sample(w, budget_s=3.0)
    for _ in range(args.steps):
        vals.append(cpu_oracle_sample(w, budget_s=args.ref_budget))
    v = statistics.median(x["value"] for x in vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * w.bits.shape[0] / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[-1]["cores"], "kind": "oracle",
                             "sample": vals[-1]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, world, rank, local):
    import torch
    from paper_2212_04749_gb300 import builder, tn
    from rqc import make_workload

    builder.build()
    tn.load()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w = make_workload(args.workload)
    bits = _bits_for_rank(w, rank)
    k = bits.shape[0]
    stream = torch.cuda.current_stream()
    free, _ = torch.cuda.mem_get_info()
    limit = min(int(args.ws_gib * 2 ** 30), int(free * 0.8))
    t0 = time.perf_counter()
    plan = tn.Plan(w.circuit, bits, w.tree.ssa, w.tree.sliced, workspace_limit=limit, fuse=args.fuse,
                   fuse_max_bits=args.fuse_bits, rescale=args.rescale)
    t_plan = time.perf_counter() - t0
    info = plan.info
    ws = torch.empty(info["workspace_bytes"], dtype=torch.uint8, device="cuda")
    plan.tn_plan_bind(ws, stream=stream)
    amps = torch.zeros(2 * k, dtype=torch.float64, device="cuda")
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device="cuda")

    def select(prec):
        """Configure every step for `prec`; returns the selection record."""
        for s_ in range(info["n_steps"]):
            plan.tn_plan_set_config(s_, -1)
        if args.select == "rule":
            return {"mode": "rule"}
        rule_ms = statistics.median(one_step(prec) for _ in range(2))
        t0 = time.perf_counter()
        if args.select == "autotune":
            plan.tn_plan_autotune(prec, amps, reps=2, stream=stream)
        else:
            from paper_2212_04749_gb300 import costmodel
            tr = costmodel.Trainer.load(args.model)
            costmodel.select(costmodel.Bound(None, plan, ws, amps, stream), prec, tr)
        sel_s = time.perf_counter() - t0
        cfg = plan.tn_plan_get_configs()
        return {"mode": args.select, "rule_ms": rule_ms, "selection_s": sel_s,
                "configs": np.bincount(cfg, minlength=tn.TN_NCONFIG).tolist()}

    def one_step(prec, profile=False):
        amps.zero_()
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        plan.tn_plan_profile(profile)
        e0.record(stream)
        plan.tn_contract(amps, prec, stream=stream)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    selection = select(args.precision)
    for _ in range(args.warmup):
        one_step(args.precision)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    times = []
    # NVTX range "bench_timed": a profiler can restrict itself to the timed
    # steps (ncu --nvtx --nvtx-include "bench_timed/")
    torch.cuda.nvtx.range_push("bench_timed")
    with Clocks(torch.cuda.current_device()) as clk:
        for _ in range(args.steps):
            times.append(one_step(args.precision))
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if dist is not None:
        dist.barrier()
    clocks = clk.summary()
    mean_ms = sum(times) / len(times)
    t_max = mean_ms
    if dist is not None:
        tt = torch.tensor([mean_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = tt.item()
    value = k * world / (t_max / 1000.0)
    # per-step device times: separate runs with CUDA events around every
    # launch (no graph replay), averaged
    prof_runs = 2
    step_ms = np.zeros(info["n_steps"])
    kernels = None
    for _ in range(prof_runs):
        one_step(args.precision, profile=True)
        ms, kernels = plan.tn_plan_step_times()
        step_ms += ms / prof_runs
    plan.tn_plan_profile(False)

    # linear XEB of this run's amplitudes (FP64 reduction on the device) and
    # the maximum-likelihood fidelity under Eq. (fxeb) with error bars (the
    # stand-in bitstrings are uniform: both near 0)
    xeb_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    tn.tn_xeb(amps, k, w.circuit.n_qubits, xeb_dev, stream=stream)
    torch.cuda.synchronize()
    xeb = float(xeb_dev.item())
    from paper_2212_04749_gb300.xeb import porter_thomas_fit
    xeb_fit = porter_thomas_fit(amps, k, w.circuit.n_qubits, stream=stream)

    # accuracy of this run against the stored oracle values
    got = amps.cpu().numpy().view(np.complex128)
    ref = _golden(args.workload) if rank == 0 else None
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref)) if ref is not None and len(ref) == k else None

    selection["tuned_ms"] = t_max

    # the other forms on the same workload (each with its own configuration)
    others = {}
    if args.mixed and rank == 0:
        for prec in ("fp32", "bf16x3", "tf32"):
            if prec == args.precision:
                continue
            sel2 = select(prec)
            one_step(prec)
            ts = [one_step(prec) for _ in range(max(2, args.steps // 2))]
            g2 = amps.cpu().numpy().view(np.complex128)
            e2 = float(np.linalg.norm(g2 - ref) / np.linalg.norm(ref)) if ref is not None else None
            others[prec] = {"amplitudes_per_s": k / (statistics.mean(ts) / 1000.0), "ms_per_step": statistics.mean(ts),
                            "rel_l2_vs_oracle": e2, "selection": sel2}
        select(args.precision)  # back to the headline form's configuration

    # roofline of the dominant kernel family
    peaks, peak_src = _peaks()
    steps = plan.tn_plan_steps()
    fam_names = {0: "k_step_row", 1: "k_step_gemm_simt", 2: "k_step_gemm_tc", 3: "k_chain"}
    fam_ms, fam_bytes, fam_flops, fam_launch = {}, {}, {}, {}
    for s, st in enumerate(steps):
        f = int(kernels[s]) if kernels is not None else 0
        fam_ms[f] = fam_ms.get(f, 0.0) + step_ms[s]
        fam_bytes[f] = fam_bytes.get(f, 0.0) + st["bytes"] * st["runs"]
        fam_flops[f] = fam_flops.get(f, 0.0) + st["flops"] * st["runs"]
        fam_launch[f] = fam_launch.get(f, 0) + int(st["runs"])
    if args.dump_steps and rank == 0:
        rows = []
        cfgs = plan.tn_plan_get_configs()
        for s_, st in enumerate(steps):
            r = dict(st)
            r["config"] = int(cfgs[s_])
            r["ms_per_call"] = float(step_ms[s_])
            r["family"] = int(kernels[s_]) if kernels is not None else -1
            rows.append(r)
        with open(args.dump_steps, "w") as f:
            json.dump({"precision": args.precision, "workload": args.workload, "steps": rows}, f)
    dom = max(fam_ms, key=fam_ms.get)
    sec = fam_ms[dom] / 1000.0
    if dom in (0, 3):
        ach = fam_bytes[dom] / sec / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s"}
    elif dom == 1:
        pk = SM_COUNT * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        ach = fam_flops[dom] / sec / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s"}
    else:
        # tensor-core steps: bound by the tensor pipe or by HBM, whichever
        # takes longer for the family's algorithmic flops and bytes
        base = peaks["bf16_tflops_sustained"]
        pk = base / 3.0 if args.precision == "bf16x3" else base * (1.1 / 2.25)
        ach = fam_flops[dom] / sec / 1e12
        t_tensor = fam_flops[dom] / (pk * 1e12)
        t_hbm = fam_bytes[dom] / (peaks["hbm_gbs"] * 1e9)
        if t_hbm >= t_tensor:
            roof = {"bound": "hbm", "achieved": fam_bytes[dom] / sec / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "tensor_tflops": ach, "tensor_frac": ach / pk}
        else:
            roof = {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # per-step bound: each of the family's steps takes at least the longer of
    # its flops at the compute peak and its bytes at the HBM peak
    t_bound = 0.0
    for s, st in enumerate(steps):
        if (int(kernels[s]) if kernels is not None else 0) != dom:
            continue
        tb = st["bytes"] * st["runs"] / (peaks["hbm_gbs"] * 1e9)
        if dom == 1:
            tb = max(tb, st["flops"] * st["runs"] / (SM_COUNT * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6))
        elif dom == 2:
            base = peaks["bf16_tflops_sustained"]
            pk2 = base / 3.0 if args.precision == "bf16x3" else base * (1.1 / 2.25)
            tb = max(tb, st["flops"] * st["runs"] / (pk2 * 1e12))
        t_bound += tb
    roof["step_bound_frac"] = t_bound / sec
    # the whole path: every step's bound (its bytes at the HBM peak, or its
    # flops at its kernel's compute peak when longer) over the step's time
    t_path = 0.0
    for s, st in enumerate(steps):
        fam = int(kernels[s]) if kernels is not None else 0
        tb = st["bytes"] * st["runs"] / (peaks["hbm_gbs"] * 1e9)
        if fam == 1:
            tb = max(tb, st["flops"] * st["runs"] / (SM_COUNT * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6))
        elif fam == 2:
            base = peaks["bf16_tflops_sustained"]
            pk2 = base / 3.0 if args.precision == "bf16x3" else base * (1.1 / 2.25)
            tb = max(tb, st["flops"] * st["runs"] / (pk2 * 1e12))
        t_path += tb
    path_bound_frac = t_path / (sum(fam_ms.values()) / 1000.0)
    # DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)
    # of the tensor-core launches of one timed step of this workload, from
    # one ncu capture of the current kernel build (815.0 GB over 52
    # launches: 1.107 x the algorithmic bytes); unknown for other cases
    measured_traffic = {("grid5x6_m14", "bf16x3", "k_step_gemm_tc"): (815.0e9 / 52, 1.107)}
    mt = measured_traffic.get((args.workload, args.precision, fam_names[dom]))
    roof["traffic"] = mt[0] if mt else None
    if mt:
        roof["traffic_over_algorithmic"] = mt[1]
    roof["kernel"] = fam_names[dom]
    roof["launches_per_step"] = fam_launch[dom]
    roof["share_of_step_time"] = fam_ms[dom] / max(sum(fam_ms.values()), 1e-12)
    roof["peak_source"] = peak_src
    roof["per_kernel_ms"] = {fam_names[f]: fam_ms[f] for f in fam_ms}

    # end to end through the public API from host buffers
    e2e = None
    if args.e2e_steps > 0:
        # successive batches through the public pipeline: each batch is
        # planned on the host (overlapped with the previous batch's device
        # work), its tables uploaded (host to device), contracted, and its
        # amplitudes read back to pinned host memory; steady-state time per
        # batch between the first and the last result
        from paper_2212_04749_gb300.pipeline import contract_batches
        cfg_now = plan.tn_plan_get_configs()
        marks = []
        ws_b = torch.empty_like(ws)  # second workspace: the next batch binds while this one runs
        for _i, _a in contract_batches(w.circuit, [bits] * (args.e2e_steps + 1), w.tree.ssa, w.tree.sliced,
                                       args.precision, (ws, ws_b), stream=stream, configs=cfg_now,
                                       workspace_limit=limit, fuse=args.fuse, fuse_max_bits=args.fuse_bits,
                                       rescale=args.rescale):
            marks.append(time.perf_counter())
        del ws_b
        torch.cuda.empty_cache()  # the later measurements size themselves by free device memory
        plan.tn_plan_bind(ws, stream=stream)
        e2e_s = (marks[-1] - marks[0]) / args.e2e_steps
        e2e = {"value": k * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(info["upload_bytes"]),
               "d2h_bytes_per_step": int(16 * k), "host_plan_s": t_plan,
               "planning": "overlapped", "table_upload": "overlapped (two workspaces)"}

    correlated = None
    if rank == 0 and args.correlated:
        correlated = measure_correlated(w, args.precision, torch, tn, stream, ws, limit)
        plan.tn_plan_bind(ws, stream=stream)

    chain = None
    if rank == 0 and args.chain_workload:
        chain = measure_chain(args.chain_workload, args.precision, torch, tn, stream, args.fuse_bits)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(w, budget_s=args.ref_budget)

    tflops = info["flops_ma"] / (t_max / 1000.0) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "fp32", "tf32": "tf32", "bf16x3": "bf16x3"}[args.precision],
        "data": "synthetic",
        "config": {"workload": args.workload, "qubits": w.circuit.n_qubits, "cycles": w.spec.cycles,
                   "bitstrings": k, "sliced_edges": len(w.tree.sliced), "slices": 2 ** len(w.tree.sliced),
                   "slice_batch": 2 ** info["slice_batch_log2"], "precision": args.precision,
                   "l2": "512 MiB write between steps; intermediates exceed L2",
                   "flops_eq1": info["flops_ma"], "flops_single_amplitude_x_k": info["flops_sa"],
                   "bytes_algorithmic": info["bytes_min"], "max_rank": info["max_rank"],
                   "workspace_gib": info["workspace_bytes"] / 2 ** 30, "rescale": bool(args.rescale)},
        "tflops_algorithmic": tflops,
        "path_bound_frac": path_bound_frac,
        "rel_l2_vs_oracle": err,
        "xeb": xeb,
        "xeb_fit": xeb_fit,
        "correlated_batches": correlated,
        "other_forms": others or None,
        "config_selection": selection,
        "roofline": roof,
        "cpu_baseline": cpu,
        "fused_chain": chain,
        "e2e": e2e,
        "gpu_launches": int(info["launches_per_call"]) * args.steps,
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="grid5x6_m14")
    ap.add_argument("--precision", choices=["fp32", "tf32", "bf16x3"], default="bf16x3",
                    help="headline form (default: the mixed BF16x3 split form); the others run beside it")
    ap.add_argument("--select", choices=["autotune", "model", "rule"], default="autotune",
                    help="per-step kernel configuration: exhaustive autotuner, cost model (--model), or the plan's rule")
    ap.add_argument("--model", default=None, help="cost-model parameters (npy) for --select model")
    ap.add_argument("--ws-gib", type=float, default=64.0)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-mixed", dest="mixed", action="store_false")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-budget", type=float, default=20.0)
    ap.add_argument("--dump-steps", default=None, help="write per-step features and times (JSON) here")
    ap.add_argument("--fuse", type=int, choices=[0, 1], default=1, help="fused chains of small-operand steps")
    ap.add_argument("--correlated", type=int, choices=[0, 1], default=1,
                    help="also time correlated batches (open qubits) and perfect-sample extraction")
    ap.add_argument("--rescale", type=int, choices=[0, 1], default=0,
                    help="per-instance power-of-two rescaling (a safety net of this library, not part of the "
                         "paper's method; off: the paper's plain arithmetic)")
    ap.add_argument("--fuse-bits", type=int, default=9, help="d^t: largest fused-chain tile, 2^d^t entries")
    ap.add_argument("--chain-workload", default="grid6x7_m10",
                    help="workload whose heaviest fused chain is timed against the unfused steps ('' to skip)")
    args = ap.parse_args()
    world, rank, local = _dist()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
