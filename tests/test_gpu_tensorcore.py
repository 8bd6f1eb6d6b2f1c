"""Tensor-core forms (TF32 and BF16x3 on tcgen05) against the oracle.

Bound for the mixed form (BF16x3): relative L2 amplitude error <= 1e-3.
TF32 keeps 10 mantissa bits per product; over the 90-300 contraction steps
of these circuits its error sits near 1e-3 (measured 1.0e-3 on 20 qubits),
so it is held to 1e-2 and reported, and BF16x3 is the mixed form that
carries the 1e-3 claim.  A 20-qubit
circuit has every GEMM-shaped step forced onto the grouped GEMM kernel so
that the tensor-core path sees many shapes (ragged M and column tiles,
K below one chunk); the 30-qubit workload checks all 4096 amplitudes.
"""

import numpy as np
import pytest

from gpu_helpers import rel_l2, require_cuda, run_plan
from oracle import sv
from rqc import grid_layout, make_workload, network_structure, random_circuit
from rqc.bitstrings import uniform_bitstrings
from rqc.tree import candidate_trees, choose_slices

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-3
TF32_TOL = 1e-2


def _tol(prec):
    return {"fp32": 1e-5, "tf32": TF32_TOL, "bf16x3": MIXED_TOL}[prec]


def _gemm_everywhere(st):
    return 1


def _case20(tree):
    from rqc.tree import ContractionTree
    c = random_circuit(grid_layout(4, 5), 12, seed=21)
    s = network_structure(c)
    bits = uniform_bitstrings(20, 1500, seed=5)
    ssa = candidate_trees(s, 1500, seed=2, trials=2)[tree]
    sl = choose_slices(s, ContractionTree(ssa=ssa), 1500, n_sliced=2)
    return c, bits, ssa, sl, sv.amplitudes(c, bits)


@pytest.fixture(scope="module")
def case20():
    return _case20(0)


@pytest.fixture(scope="module")
def case20_shapes():
    # another candidate tree of the same circuit: its GEMM-shaped steps span
    # M = 2^6 .. 2^16 rows, so the tensor-core path meets its edge shapes
    return _case20(2)


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16x3"])
@pytest.mark.parametrize("case", ["case20", "case20_shapes"])
def test_forced_gemm_path_matches_state_vector(case, prec, request):
    c, bits, ssa, sl, ref = request.getfixturevalue(case)
    got, p = run_plan(c, bits, ssa, sl, precision=prec, force_kernel=_gemm_everywhere)
    if case == "case20_shapes" and prec != "fp32":
        # the tensor-core steps include K = 8 (half a chunk), M = 64 (half a
        # row tile), partial column tiles, and both N < 16 and N >= 64 per
        # instance
        tc = [s for s, k in zip(p.tn_plan_steps(), p.tn_plan_step_times()[1]) if k == 2]
        assert any(s["kb"] == 3 for s in tc) and any(s["mb"] == 6 for s in tc)
        assert any(s["nb"] < 4 for s in tc) and any(s["nb"] >= 6 for s in tc)
        assert any((s["n_inst"] // max(s["n_groups"], 1) << s["nb"]) % 64 for s in tc)
    err = rel_l2(got, ref)
    print(f"forced GEMM 20q {case} {prec}: rel-L2 {err:.3e}")
    assert err <= _tol(prec), err


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
@pytest.mark.parametrize("resident", [True, False])
@pytest.mark.parametrize("config", [2, 3])
def test_tensor_core_forms_match_state_vector(case20_shapes, prec, resident, config):
    # configuration 2 walks a group's tiles row tile by row tile, 3 column
    # tile by column tile; with resident B each CTA takes a contiguous range
    # of tiles and keeps B in shared memory (configuration 2: all of the
    # step's B instances when they fit one 64-column tile, else the group's;
    # 3: a column tile's), without it B is gathered chunk by chunk: all the
    # forms against the state vector
    torch, tn = require_cuda()
    c, bits, ssa, sl, ref = case20_shapes
    p = tn.Plan(c, bits, ssa, sl)
    for s, st in enumerate(p.tn_plan_steps()):
        p.tn_plan_set_config(s, config)
    p.tn_plan_set_tc_resident_b(resident)
    ws = torch.empty(max(p.info["workspace_bytes"], 256), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    p.tn_plan_bind(ws, stream=stream)
    amps = torch.zeros(2 * len(bits), dtype=torch.float64, device="cuda")
    p.tn_contract(amps, prec, stream=stream)
    p.tn_plan_check(stream=stream)
    torch.cuda.synchronize()
    kinds = p.tn_plan_step_times()[1]
    assert sum(1 for k in kinds if k == 2) >= 5
    if config == 2 and resident:
        # B dictionaries (every B instance of the step in one 64-column
        # tile) whose groups hold several instances: their columns are
        # gathered from the accumulator
        assert any((s["n_inst_b"] << s["nb"]) <= 64 and s["n_inst"] > s["n_groups"]
                   for s, k in zip(p.tn_plan_steps(), kinds) if k == 2)
    err = rel_l2(amps.cpu().numpy().view(np.complex128), ref)
    print(f"tensor-core 20q config {config} resident-B {resident} {prec}: rel-L2 {err:.3e}")
    assert err <= _tol(prec), err


def _row_where_it_fits(st):
    return 0 if (st["nb"] <= 4 and st["kb"] + st["nb"] <= 8) else 1


@pytest.mark.parametrize("sched", [0, 1])
@pytest.mark.parametrize("case", ["case20", "case16"])
def test_forced_row_kernel_matches_state_vector(case, sched, request):
    # every step the grouped row kernel can take runs on it (schedule 1:
    # small-M steps one instance row per lane group); on 16 qubits with 4096
    # bitstrings some groups hold more instances than one staging chunk
    # (their B blocks are staged in chunks)
    if case == "case20":
        c, bits, ssa, sl, ref = request.getfixturevalue("case20")
    else:
        c = random_circuit(grid_layout(4, 4), 10, seed=21)
        bits = uniform_bitstrings(16, 4096, seed=5)
        ssa = candidate_trees(network_structure(c), 4096, seed=2, trials=2)[1]
        sl, ref = [], sv.amplitudes(c, bits)
    got, p = run_plan(c, bits, ssa, sl, precision="fp32", force_kernel=_row_where_it_fits,
                      force_config=lambda st: sched if _row_where_it_fits(st) == 0 else None)
    steps = p.tn_plan_steps()
    # mean group size over the instances one staging chunk holds (at most 32
    # instances and 2048 complex B entries)
    big = max(s["n_inst"] / max(s["n_groups"], 1) / min(32, 2048 >> (s["kb"] + s["nb"]))
              for s in steps if _row_where_it_fits(s) == 0)
    err = rel_l2(got, ref)
    print(f"forced row kernel {case} schedule {sched} fp32: rel-L2 {err:.3e}, largest mean group {big:.1f} chunks")
    if case == "case16":
        assert big > 1  # chunked staging is exercised
    assert err <= _tol("fp32"), err


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_plan_choice_matches_state_vector(case20, prec):
    c, bits, ssa, sl, ref = case20
    got, p = run_plan(c, bits, ssa, sl, precision=prec)
    assert rel_l2(got, ref) <= _tol(prec)


def test_bf16x3_is_closer_than_tf32(case20):
    c, bits, ssa, sl, ref = case20
    e_tf, _ = run_plan(c, bits, ssa, sl, precision="tf32", force_kernel=_gemm_everywhere)
    e_bf, _ = run_plan(c, bits, ssa, sl, precision="bf16x3", force_kernel=_gemm_everywhere)
    assert rel_l2(e_bf, ref) < rel_l2(e_tf, ref)


@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
def test_grid5x6_mixed_matches_stored_state_vector(prec):
    import importlib.util, os
    spec = importlib.util.spec_from_file_location(
        "make_golden", os.path.join(os.path.dirname(__file__), "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    _, ref = mg.read("grid5x6_m14")
    w = make_workload("grid5x6_m14")
    got, p = run_plan(w.circuit, w.bits, w.tree.ssa, w.tree.sliced, precision=prec)
    err = rel_l2(got, ref)
    print(f"grid5x6_m14 {prec}: rel-L2 {err:.3e}")
    assert err <= _tol(prec), err
    if prec == "bf16x3":
        # configuration 3 on every GEMM-shaped step: schedule 1 with the
        # group's two column tiles walked by CTA pairs where every group has
        # two (M = 2^12 x 4 columns, 2^21 / 2^18 x 64 columns, ...)
        got3, p3 = run_plan(w.circuit, w.bits, w.tree.ssa, w.tree.sliced, precision=prec,
                            force_config=lambda st: 3 if st["kb"] >= 3 and st["mb"] >= 6 else None)
        err3 = rel_l2(got3, ref)
        print(f"grid5x6_m14 {prec}, configuration 3: rel-L2 {err3:.3e}")
        assert err3 <= _tol(prec), err3
