"""Throughput of the multiple-amplitude contraction on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload diamond53_m12] [--precision bf16x3|fp32|tf32]

One step = one full tn_contract of the workload's plan: every slice batch,
the amplitudes of all its bitstrings.  Default workload: the 53-qubit
diamond (54 sites, one dead), 12 cycles, 8192 bitstrings, contracted with
the largest per-instance intermediate at 2^26 entries, in the mixed BF16x3
form with the per-instance power-of-two rescale; FP32 and TF32 run beside
it on the same plan.  Prints one JSON line (rank 0).

value      amplitudes/s over all ranks: bitstrings / max-over-ranks device
           time (CUDA events around each step on the launching stream;
           plan and inputs resident in HBM; a 512 MiB write flushes L2
           between steps).
e2e        the same metric through the public pipeline from host data:
           host plan (overlapped), table upload, contraction, amplitudes
           back to pinned host memory.
roofline   the kernel family with the largest share of device time:
           algorithmic bytes or flops / its measured launch time, against
           the measured peak that binds it.
peaks      denominators measured in this run on this device: the FP32 FMA
           rate (tn_fma_probe), the TF32 and FP64 matrix-multiply rates
           (torch.matmul); HBM and BF16 from the driver's measurements.
cpu_baseline  the CPU oracle on this host's cores on a bounded sample: the
           tensor-network contractor on a few of the workload's bitstrings
           (53 qubits), or the state vector through a prefix of the gates.
--impl reference times that oracle as the reference arm.
Multi-GPU (torchrun): strong scaling.  All ranks contract the same
bitstrings with one plan whose slice batches are split into contiguous
ranges (the plan is sliced further until it has a batch per rank); the
k complex128 amplitudes are all-gathered and summed in rank order.
"""

import argparse
import hashlib
import json
import math
import os
import re
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
FAMILIES = {0: "k_step_row", 1: "k_step_gemm_simt", 2: "k_step_gemm_tc", 3: "k_chain"}
TOL = {"fp32": 1e-5, "bf16x3": 1e-3, "tf32": 1e-3}


def _driver_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def measure_peaks(torch, tn, stream):
    """Compute-rate denominators measured now on this device (best of a few
    runs, CUDA events): FP32 FMA (the library's probe kernel: 152 x 8 blocks
    of 256 threads, 16 flops per thread per round), TF32 tensor (torch.matmul
    of 8192^3 FP32 with TF32 allowed: 2 N^3 flops) and FP64 (torch.matmul of
    4096^3 float64)."""
    out = {}

    def best(fn, reps):
        fn()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return min(ts)

    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks, iters = sms * 8, 1 << 16
    sink = torch.zeros(blocks, dtype=torch.float32, device="cuda")
    t = best(lambda: tn.tn_fma_probe(blocks, iters, sink, stream=stream), 5)
    out["fp32_fma_tflops"] = blocks * 256 * 16 * iters / t / 1e12
    prev = torch.backends.cuda.matmul.allow_tf32
    with torch.cuda.stream(stream):
        n = 8192
        a = torch.randn(n, n, device="cuda", dtype=torch.float32)
        b = torch.randn(n, n, device="cuda", dtype=torch.float32)
        torch.backends.cuda.matmul.allow_tf32 = True
        t = best(lambda: torch.matmul(a, b), 5)
        out["tf32_tflops"] = 2 * n ** 3 / t / 1e12
        torch.backends.cuda.matmul.allow_tf32 = prev
        del a, b
        n = 4096
        a = torch.randn(n, n, device="cuda", dtype=torch.float64)
        b = torch.randn(n, n, device="cuda", dtype=torch.float64)
        t = best(lambda: torch.matmul(a, b), 3)
        out["fp64_tflops"] = 2 * n ** 3 / t / 1e12
        del a, b
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    out["how"] = ("fp32_fma: tn_fma_probe, %d blocks x 256 threads x 16 x %d flops, best of 5; tf32: torch.matmul "
                  "8192^3 fp32 with TF32 allowed, best of 5; fp64: torch.matmul 4096^3 float64, best of 3" %
                  (blocks, iters))
    return out


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


def _golden_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(ROOT, "tests", "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    return mg


def reference_values(name, w):
    """Stored CPU-oracle values of the workload: (rows, complex128 values),
    rows None for every bitstring (state vector), else the sampled rows
    (tensor-network oracle); None if nothing is stored or the stored values
    belong to other inputs."""
    mg = _golden_module()
    if os.path.exists(mg.path_for(name)):
        digest, amps = mg.read(name)
        rows = None
    elif os.path.exists(mg.sample_path(name)):
        rec = mg.read_json(mg.sample_path(name))
        digest, amps, rows = rec["inputs_sha256"], rec["amplitudes"], rec["rows"]
    else:
        return None
    if digest != mg.input_digest(w.circuit, w.bits):
        return None
    return rows, np.asarray(amps, np.complex128)


def rel_l2_against(got, ref):
    if ref is None:
        return None, 0
    rows, vals = ref
    g = got if rows is None else got[rows]
    if len(g) != len(vals):
        return None, 0
    return float(np.linalg.norm(g - vals) / np.linalg.norm(vals)), len(vals)


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def cpu_oracle_sample(w, budget_s=20.0, max_rows=None):
    """The CPU oracle as it stands on a bounded sample of the workload.

    Above 30 qubits: the complex128 tensor-network oracle (oracle/tn.py,
    memo cache over shared sub-networks) contracts the first n bitstrings of
    the workload, n grown until about budget_s of CPU work; value = n / time
    (measured, not extrapolated).  Up to 30 qubits: the complex128 state
    vector through the first g gates, extrapolated per gate pass to the full
    circuit (value = k / extrapolated time)."""
    n_q = w.circuit.n_qubits
    if n_q > 30:
        from oracle import tn as otn
        n = 1
        while True:
            t0 = time.perf_counter()
            otn.partial_amplitudes(w.circuit, w.tree.ssa, w.bits[:n], [tuple(int(x) for x in w.struct.edge_wire[e])
                                                                       for e in w.tree.sliced],
                                   list(range(1 << len(w.tree.sliced))))
            dt = time.perf_counter() - t0
            if dt > budget_s / 3 or n >= w.bits.shape[0] or (max_rows and n >= max_rows):
                break
            n = min(w.bits.shape[0], max(n + 1, int(n * min(8.0, budget_s / 2 / max(dt, 1e-3)))))
            if max_rows:
                n = min(n, max_rows)
        return {"value": n / dt, "unit": UNIT, "cores": _cores(), "kind": "oracle",
                "sample": f"tensor-network oracle (complex128, unfused network, memo cache) on the first {n} of the "
                          f"{w.bits.shape[0]} bitstrings, all {1 << len(w.tree.sliced)} slices, in {dt:.2f} s"}
    from oracle import sv as osv
    from rqc.circuit import Circuit
    total = len(w.circuit.gates)
    g = 8
    while True:
        c = Circuit(n_qubits=n_q, gates=w.circuit.gates[:g])
        t0 = time.perf_counter()
        osv.state(c)
        dt = time.perf_counter() - t0
        if dt > budget_s / 3 or g >= total:
            break
        g = min(total, max(g + 1, int(g * min(8.0, budget_s / 3 / max(dt, 1e-3)))))
    t_full = dt * (total + 1) / (g + 1)
    k = w.bits.shape[0]
    return {"value": k / t_full, "unit": UNIT, "cores": osv.threads(), "kind": "oracle",
            "sample": f"state-vector oracle (complex128, 2^{n_q} amplitudes) through the first {g} of {total} gates "
                      f"in {dt:.2f} s, extrapolated per gate pass to {t_full:.1f} s for the {k} bitstrings"}


def traffic_record(kernel):
    """DRAM traffic over algorithmic bytes of `kernel` from the committed ncu
    summary profiles/<kernel>_traffic_small_case.md, if that summary was
    taken on the current source of the kernel (its sha256 line matches);
    else None.  The summary's ratio comes from a small case of the same
    kernel (the bench workload is too large for a counter capture)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic_small_case.md")
    src = os.path.join(ROOT, "paper_2212_04749_gb300", "csrc", "gemm_tc.cu" if kernel == "k_step_gemm_tc" else
                       "kernels.cu")
    try:
        text = open(path).read()
        cur = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    m = re.search(r"traffic_over_algorithmic:\s*([0-9.]+)", text)
    h = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    if not m or not h or h.group(1) != cur:
        return None
    return float(m.group(1))


def family_breakdown(steps, step_ms, kernels):
    fam = {}
    for s, st in enumerate(steps):
        f = int(kernels[s]) if kernels is not None else 0
        r = fam.setdefault(f, {"ms": 0.0, "bytes": 0.0, "flops": 0.0, "launches": 0, "steps": []})
        r["ms"] += float(step_ms[s])
        r["bytes"] += st["bytes"] * st["runs"]
        r["flops"] += st["flops"] * st["runs"]
        r["launches"] += int(st["runs"])
        r["steps"].append(s)
    return fam


def compute_peak(family, precision, peaks):
    """Compute-rate peak (TFLOP/s, algorithmic) of a kernel family at a
    precision and its source: tensor-core BF16x3 = measured BF16 (sustained)
    / 3 products; TF32 = measured TF32; SIMT = measured FP32 FMA."""
    if family == 2:
        if precision == "bf16x3":
            return peaks["bf16_tflops_sustained"] / 3.0, "measured bf16 sustained / 3"
        return peaks.get("tf32_tflops"), "measured tf32"
    if family in (0, 1, 3):
        return peaks.get("fp32_fma_tflops"), "measured fp32 fma"
    return None, None


def roofline_of(steps, step_ms, kernels, precision, peaks):
    """Roofline of the dominant kernel family, the per-step bound fraction
    and the whole path's bound fraction.  A step's bound time is the longer
    of its algorithmic bytes at the HBM peak and its flops at its family's
    compute peak; a family is reported HBM-bound when its summed bytes at
    the HBM peak take longer than its summed flops at the compute peak."""
    fam = family_breakdown(steps, step_ms, kernels)
    hbm = peaks["hbm_gbs"]

    def bound_time(s, st, f):
        tb = st["bytes"] * st["runs"] / (hbm * 1e9)
        pk, _ = compute_peak(f, precision, peaks)
        if pk and f in (1, 2):
            tb = max(tb, st["flops"] * st["runs"] / (pk * 1e12))
        return tb

    total_ms = sum(r["ms"] for r in fam.values())
    dom = max(fam, key=lambda f: fam[f]["ms"])
    r = fam[dom]
    sec = r["ms"] / 1e3
    pk, pk_src = compute_peak(dom, precision, peaks)
    t_hbm = r["bytes"] / (hbm * 1e9)
    t_cmp = r["flops"] / (pk * 1e12) if pk and dom in (1, 2) else 0.0
    if t_hbm >= t_cmp:
        roof = {"bound": "hbm", "achieved": r["bytes"] / sec / 1e9, "peak": hbm, "unit": "GB/s"}
        if pk:
            roof["tensor_tflops" if dom == 2 else "alu_tflops"] = r["flops"] / sec / 1e12
            roof["tensor_frac" if dom == 2 else "alu_frac"] = r["flops"] / sec / 1e12 / pk
    else:
        roof = {"bound": "tensor" if dom == 2 else "alu", "achieved": r["flops"] / sec / 1e12, "peak": pk,
                "unit": "TFLOP/s", "peak_source": pk_src}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["step_bound_frac"] = sum(bound_time(s, steps[s], dom) for s in r["steps"]) / sec
    roof["kernel"] = FAMILIES[dom]
    roof["launches_per_step"] = r["launches"]
    roof["algorithmic_bytes_per_launch"] = r["bytes"] / max(r["launches"], 1)
    roof["share_of_step_time"] = r["ms"] / max(total_ms, 1e-12)
    roof["per_kernel_ms"] = {FAMILIES[f]: fam[f]["ms"] for f in fam}
    path_bound = sum(bound_time(s, steps[s], f) for f in fam for s in fam[f]["steps"])
    # HBM fraction of every other family (the row kernel: bandwidth steps)
    others = {}
    for f, rr in fam.items():
        if f == dom or rr["ms"] <= 0:
            continue
        others[FAMILIES[f]] = {"ms": rr["ms"], "hbm_frac": rr["bytes"] / (rr["ms"] / 1e3) / 1e9 / hbm,
                               "launches": rr["launches"]}
    roof["other_families"] = others
    return roof, path_bound / (total_ms / 1e3), dom


def measure_correlated(w, precision, torch, tn, stream, ws, limit, rescale, rows=256, n_open=4, reps=3):
    """Correlated batches (SM Sec. II): `rows` of the workload's bitstrings
    with their last `n_open` qubits left open, so that one contraction
    yields rows x 2^n_open amplitudes, then one perfect sample per row
    (tn_sample_completions, uniform numbers drawn on the host, seed 5).
    CUDA-event time of the contraction (the plan's rule configuration)
    and of the sampling."""
    n = w.circuit.n_qubits
    oq = list(range(n - n_open, n))
    p = tn.Plan(w.circuit, w.bits[:rows], w.tree.ssa, w.tree.sliced, workspace_limit=min(limit, ws.numel()),
                open_qubits=oq, rescale=rescale)
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


def measure_fusion(plan, precision, tn, one_step, peaks):
    """Fused chains (SM Sec. V.C) on the timed plan, after the autotuner
    chose per chain: every chain's time fused (its kernel, booked on its
    last step) and unfused (the sum of its steps, each with its tuned
    configuration), one profiled contraction each way, and the chain
    kernel's HBM roofline (algorithmic bytes: A_1 read, every B_j read, C_L
    written; the intermediates are never stored)."""
    n = plan.info["n_chains"]
    if n == 0:
        return {"chains": 0}
    keep = plan.tn_plan_get_chains().copy()
    steps = plan.tn_plan_steps()
    members = {}
    for i, st in enumerate(steps):
        if st["chain"] >= 0:
            members.setdefault(st["chain"], []).append(i)
    res = {}
    for on in (1, 0):
        for c in range(n):
            plan.tn_plan_set_chain(c, on)
        one_step(precision, profile=True)
        res[on] = plan.tn_plan_step_times()[0]
    for c in range(n):
        plan.tn_plan_set_chain(c, int(keep[c]))
    fused = {c: float(res[1][ids[-1]]) for c, ids in members.items()}
    unfused = {c: float(sum(res[0][i] for i in ids)) for c, ids in members.items()}
    kept = [c for c in range(n) if keep[c]]
    rej = [c for c in range(n) if not keep[c]]

    def alg_bytes(ids):
        first, last = steps[ids[0]], steps[ids[-1]]
        a = 8.0 * first["n_inst_a"] * 2.0 ** first["rank_a"]
        b = sum(8.0 * steps[i]["n_inst_b"] * 2.0 ** steps[i]["rank_b"] for i in ids)
        cc = 8.0 * last["n_inst"] * 2.0 ** (last["mb"] + last["nb"])
        return (a + b + cc) * last["runs"]
    tf = sum(fused[c] for c in kept)
    tu = sum(unfused[c] for c in kept)
    out = {"chains": n, "kept_fused": len(kept),
           "kept": {"fused_ms": tf, "unfused_ms": tu, "speedup": tu / tf if tf > 0 else None},
           "rejected": {"fused_ms": sum(fused[c] for c in rej), "unfused_ms": sum(unfused[c] for c in rej)}}
    if kept and tf > 0:
        ach = sum(alg_bytes(members[c]) for c in kept) / (tf / 1e3) / 1e9
        out["roofline"] = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                           "frac": ach / peaks["hbm_gbs"], "kernel": "k_chain"}
    heavy = max(members, key=lambda c: unfused[c])
    out["heaviest"] = {"steps": members[heavy], "fused_ms": fused[heavy], "unfused_ms": unfused[heavy],
                       "kept_fused": bool(keep[heavy])}
    return out


def run_reference(args, world, rank):
    """The reference arm: the CPU oracle as it stands on this host's cores,
    each step a bounded sample of the workload (rank 0 only)."""
    if rank != 0:
        return 0
    from rqc import make_workload
    w = make_workload(args.workload)
    for _ in range(args.warmup):
        cpu_oracle_sample(w, budget_s=min(3.0, args.ref_budget), max_rows=1)
    vals, times = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        vals.append(cpu_oracle_sample(w, budget_s=args.ref_budget))
        times.append(time.perf_counter() - t0)
    v = statistics.median(x["value"] for x in vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * statistics.mean(times),
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[-1]["cores"], "kind": "oracle",
                             "sample": "each step: " + vals[-1]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def sliced_for_world(w, world):
    """Sliced edges of the plan all ranks share: the workload's own, plus
    (for world > 1) further edges chosen by the greedy slicer until the
    slices can be split into at least one batch per rank."""
    sl = list(w.tree.sliced)
    need = max(0, math.ceil(math.log2(world))) if world > 1 else 0
    if len(sl) >= need:
        return sl
    from rqc.tree import choose_slices
    extra = choose_slices(w.struct, w.tree, w.bits.shape[0], n_sliced=need)
    for e in extra:
        if e not in sl and len(sl) < need:
            sl.append(e)
    return sorted(sl)


def run_ours(args, world, rank, local):
    import torch
    from paper_2212_04749_gb300 import builder, tn
    from paper_2212_04749_gb300.multi import batch_range
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

    if args.case is not None:
        from types import SimpleNamespace
        from paper_2212_04749_gb300 import costmodel
        from rqc.network import network_structure
        cs = costmodel.random_case(args.case)
        w = SimpleNamespace(circuit=cs.circuit, bits=cs.bits, struct=network_structure(cs.circuit),
                            tree=SimpleNamespace(ssa=cs.ssa, sliced=list(cs.sliced)),
                            spec=SimpleNamespace(cycles=None, index=None))
        args.workload = "case" + str(args.case) + "_" + cs.name
    else:
        w = make_workload(args.workload)
    bits = w.bits if not args.rows else w.bits[:args.rows]
    k = bits.shape[0]
    sliced = sliced_for_world(w, world)
    stream = torch.cuda.current_stream()
    dpeaks, dpeak_src = _driver_peaks()
    peaks = dict(dpeaks)
    live = measure_peaks(torch, tn, stream) if rank == 0 and args.peaks else {}
    peaks.update({kk: v for kk, v in live.items() if kk != "how"})
    free, _ = torch.cuda.mem_get_info()
    limit = min(int(args.ws_gib * 2 ** 30), int(free * 0.8))
    popts = dict(workspace_limit=limit, fuse=args.fuse, fuse_max_bits=args.fuse_bits, rescale=args.rescale)
    if world > 1:
        # one slice per batch so the batches split over the ranks
        popts["slice_batch_log2"] = max(0, len(sliced) - math.ceil(math.log2(world)))
    t0 = time.perf_counter()
    plan = tn.Plan(w.circuit, bits, w.tree.ssa, sliced, **popts)
    t_plan = time.perf_counter() - t0
    info = plan.info
    lo, hi = batch_range(info["n_batches"], rank, world)
    if args.batches:
        hi = min(hi, lo + args.batches)
    ws = torch.empty(info["workspace_bytes"], dtype=torch.uint8, device="cuda")
    plan.tn_plan_bind(ws, stream=stream)
    amps = torch.zeros(2 * k, dtype=torch.float64, device="cuda")
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device="cuda")
    gathered = [torch.empty_like(amps) for _ in range(world)] if world > 1 else None
    total = torch.empty_like(amps)

    def reduce_in_rank_order():
        # the one exchange of the path: every rank's k complex128 partial
        # sums, added in rank order (deterministic)
        if dist is None:
            return amps
        dist.all_gather(gathered, amps)
        total.copy_(gathered[0])
        for g in gathered[1:]:
            total.add_(g)
        return total

    def one_step(prec, profile=False):
        amps.zero_()
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        plan.tn_plan_profile(profile)
        e0.record(stream)
        if hi > lo:
            plan.tn_contract(amps, prec, lo, hi, stream=stream)
        reduce_in_rank_order()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    def select(prec):
        """Configure every step for `prec`; returns the selection record."""
        for s_ in range(info["n_steps"]):
            plan.tn_plan_set_config(s_, -1)
        for c_ in range(info["n_chains"]):
            plan.tn_plan_set_chain(c_, 1)
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
        ch = plan.tn_plan_get_chains()
        return {"mode": args.select, "rule_ms": rule_ms, "selection_s": sel_s,
                "configs": np.bincount(cfg, minlength=tn.TN_NCONFIG).tolist(),
                "chains_fused": int(np.sum(ch)), "chains": int(len(ch))}

    def profile_steps(prec, runs=2):
        step_ms = np.zeros(info["n_steps"])
        kernels = None
        for _ in range(runs):
            one_step(prec, profile=True)
            ms, kernels = plan.tn_plan_step_times()
            step_ms += ms / runs
        plan.tn_plan_profile(False)
        return step_ms, kernels

    ref = reference_values(args.workload, w) if rank == 0 and not args.rows and args.case is None else None
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
    value = k / (t_max / 1000.0)
    got = reduce_in_rank_order().cpu().numpy().view(np.complex128).copy()
    err, n_cmp = rel_l2_against(got, ref)

    step_ms, kernels = profile_steps(args.precision)
    steps = plan.tn_plan_steps()
    roof, path_bound_frac, dom = roofline_of(steps, step_ms, kernels, args.precision, peaks)
    ratio = traffic_record(roof["kernel"])
    roof["traffic"] = ratio * roof["algorithmic_bytes_per_launch"] if ratio else None
    roof["traffic_over_algorithmic"] = ratio
    roof["traffic_source"] = ("ncu dram__bytes_read+write of a small case of the same kernel source, scaled by "
                              "algorithmic bytes" if ratio else "no capture of the current kernel source")
    roof["peak_source"] = roof.get("peak_source", dpeak_src)
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

    # linear XEB of this run's amplitudes (FP64 reduction on the device) and
    # the maximum-likelihood fidelity under Eq. (fxeb) with error bars (the
    # stand-in bitstrings are uniform: both near 0)
    xeb = xeb_fit = None
    if rank == 0:
        dev = torch.from_numpy(got.view(np.float64).copy()).cuda()
        xeb_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
        tn.tn_xeb(dev, k, w.circuit.n_qubits, xeb_dev, stream=stream)
        torch.cuda.synchronize()
        xeb = float(xeb_dev.item())
        from paper_2212_04749_gb300.xeb import porter_thomas_fit
        xeb_fit = porter_thomas_fit(dev, k, w.circuit.n_qubits, stream=stream)

    selection["tuned_ms"] = t_max

    # the other forms on the same plan (each with its own configuration)
    others = {}
    if args.mixed:
        for prec in ("fp32", "tf32", "bf16x3"):
            if prec == args.precision:
                continue
            sel2 = select(prec)
            one_step(prec)
            ts = [one_step(prec) for _ in range(max(2, args.steps // 2))]
            tmx = statistics.mean(ts)
            if dist is not None:
                tt = torch.tensor([tmx], device="cuda")
                dist.all_reduce(tt, op=dist.ReduceOp.MAX)
                tmx = tt.item()
            g2 = reduce_in_rank_order().cpu().numpy().view(np.complex128).copy()
            e2, _ = rel_l2_against(g2, ref)
            sm2, kn2 = profile_steps(prec)
            roof2, pbf2, _ = roofline_of(steps, sm2, kn2, prec, peaks)
            others[prec] = {"amplitudes_per_s": k / (tmx / 1000.0), "ms_per_step": tmx,
                            "tflops_algorithmic": info["flops_ma"] / (tmx / 1000.0) / 1e12,
                            "rel_l2_vs_oracle": e2, "tolerance": TOL[prec],
                            "within_tolerance": (e2 <= TOL[prec]) if e2 is not None else None,
                            "path_bound_frac": pbf2, "roofline": roof2, "selection": sel2}
        select(args.precision)  # back to the headline form's configuration

    # end to end through the public API from host buffers
    e2e = None
    if args.e2e_steps > 0 and world == 1:
        # successive batches through the public pipeline: each batch is
        # planned on the host (overlapped with the previous batch's device
        # work), its tables uploaded (host to device), contracted, and its
        # amplitudes read back to pinned host memory; steady-state time per
        # batch between the first and the last result
        from paper_2212_04749_gb300.pipeline import contract_batches
        cfg_now = plan.tn_plan_get_configs()
        chains_now = plan.tn_plan_get_chains()
        marks = []
        # further workspaces: the next batches are planned (two host threads)
        # and bound while this one runs, as far as device memory allows
        free_b, _ = torch.cuda.mem_get_info()
        n_extra = max(1, min(2, int(free_b * 0.9) // max(ws.numel(), 1)))
        extra = [torch.empty_like(ws) for _ in range(n_extra)]
        for _i, _a in contract_batches(w.circuit, [bits] * (args.e2e_steps + 1), w.tree.ssa, sliced,
                                       args.precision, [ws] + extra, stream=stream, configs=cfg_now,
                                       chains=chains_now, **popts):
            marks.append(time.perf_counter())
        del extra
        torch.cuda.empty_cache()  # the later measurements size themselves by free device memory
        plan.tn_plan_bind(ws, stream=stream)
        e2e_s = (marks[-1] - marks[0]) / args.e2e_steps
        e2e = {"value": k / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(info["upload_bytes"]),
               "d2h_bytes_per_step": int(16 * k), "host_plan_s": t_plan,
               "planning": f"overlapped ({n_extra} host threads)",
               "table_upload": f"overlapped ({n_extra + 1} workspaces)"}

    correlated = None
    if rank == 0 and world == 1 and args.correlated:
        correlated = measure_correlated(w, args.precision, torch, tn, stream, ws, limit, args.rescale)
        plan.tn_plan_bind(ws, stream=stream)

    fusion = None
    if rank == 0 and args.fuse:
        fusion = measure_fusion(plan, args.precision, tn, one_step, peaks)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(w, budget_s=args.ref_budget)

    tflops = info["flops_ma"] / (t_max / 1000.0) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": args.workload, "qubits": w.circuit.n_qubits, "cycles": w.spec.cycles,
                   "bitstrings": k, "rows_of_workload": args.rows or None, "sliced_edges": len(sliced), "slices": 2 ** len(sliced),
                   "slice_batch": 2 ** info["slice_batch_log2"], "batches_per_rank": hi - lo, "partial": bool(args.batches) or None,
                   "precision": args.precision,
                   "l2": "512 MiB write between steps; intermediates exceed L2",
                   "flops_eq1": info["flops_ma"], "flops_single_amplitude_x_k": info["flops_sa"],
                   "bytes_algorithmic": info["bytes_min"], "max_rank": info["max_rank"],
                   "workspace_gib": info["workspace_bytes"] / 2 ** 30, "rescale": bool(args.rescale)},
        "tflops_algorithmic": tflops,
        "path_bound_frac": path_bound_frac,
        "rel_l2_vs_oracle": err,
        "oracle_amplitudes_compared": n_cmp,
        "tolerance": TOL[args.precision],
        "xeb": xeb,
        "xeb_fit": xeb_fit,
        "other_forms": others or None,
        "mixed_over_fp32": (value / others["fp32"]["amplitudes_per_s"]) if "fp32" in others else None,
        "config_selection": selection,
        "roofline": roof,
        "peaks": {"hbm_gbs": peaks["hbm_gbs"], "bf16_tflops_sustained": peaks["bf16_tflops_sustained"],
                  "bf16_source": dpeak_src, **live},
        "cpu_baseline": cpu,
        "correlated_batches": correlated,
        "fused_chains": fusion,
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
    ap.add_argument("--workload", default="diamond53_m12")
    ap.add_argument("--precision", choices=["fp32", "tf32", "bf16x3"], default="bf16x3",
                    help="headline form (default: the mixed BF16x3 split form); the others run beside it")
    ap.add_argument("--select", choices=["autotune", "model", "rule"], default="autotune",
                    help="per-step kernel configuration: exhaustive autotuner, cost model (--model), or the plan's rule")
    ap.add_argument("--model", default=None, help="cost-model parameters (npy) for --select model")
    ap.add_argument("--ws-gib", type=float, default=120.0)
    ap.add_argument("--rows", type=int, default=0,
                    help="contract only the first ROWS bitstrings of the workload with its own tree (a smaller "
                         "case of the same step shapes, e.g. for profiler captures); 0: all")
    ap.add_argument("--batches", type=int, default=0,
                    help="contract only the first BATCHES slice batches of each rank's range (a partial "
                         "contraction, e.g. for profiler captures of a heavily sliced --case); 0: all")
    ap.add_argument("--case", type=int, default=None,
                    help="instead of a named workload, the seeded random circuit and tree of "
                         "costmodel.random_case(CASE) (small plans of a few GB, e.g. for profiler captures)")
    ap.add_argument("--no-peaks", dest="peaks", action="store_false",
                    help="skip the live FP32/TF32/FP64 peak measurements")
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--no-mixed", dest="mixed", action="store_false")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-budget", type=float, default=20.0,
                    help="seconds of CPU work per oracle sample (cpu_baseline; per step of --impl reference)")
    ap.add_argument("--dump-steps", default=None, help="write per-step features and times (JSON) here")
    ap.add_argument("--fuse", type=int, choices=[0, 1], default=1, help="fused chains of small-operand steps")
    ap.add_argument("--correlated", type=int, choices=[0, 1], default=1,
                    help="also time correlated batches (open qubits) and perfect-sample extraction")
    ap.add_argument("--rescale", type=int, choices=[0, 1], default=1,
                    help="per-instance power-of-two rescaling (on by default; 0: the paper's plain arithmetic)")
    ap.add_argument("--fuse-bits", type=int, default=9, help="d^t: largest fused-chain tile, 2^d^t entries")
    args = ap.parse_args()
    world, rank, local = _dist()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
