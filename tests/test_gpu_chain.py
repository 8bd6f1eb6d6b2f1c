"""Fused chains (tn_options.fuse) against the oracles.

A chain runs several small-operand steps in one kernel with its
intermediates in shared memory (SM Sec. V.C).  Its arithmetic is the same
sum per output element as the unfused steps (the contraction order inside
each element is k ascending), so FP32 stays within 1e-5 of the complex128
oracles; BF16x3 / TF32 only change the non-chain steps.  Checked on the
12-qubit workload (state vector), a 20-qubit circuit with 1500 bitstrings
and 2 sliced edges (state vector), the 30-qubit workload (stored state
vector, all 4096 amplitudes) and the 42-qubit workload's stored oracle
slices; every case holds several chains (asserted).
"""

import importlib.util
import os

import numpy as np
import pytest

from gpu_helpers import rel_l2, require_cuda, run_plan, run_slices
from oracle import sv
from rqc import grid_layout, make_workload, network_structure, random_circuit
from rqc.bitstrings import uniform_bitstrings
from rqc.tree import ContractionTree, candidate_trees, choose_slices

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "bf16x3": 1e-3, "tf32": 1e-2}


def _mg():
    spec = importlib.util.spec_from_file_location(
        "make_golden", os.path.join(os.path.dirname(__file__), "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    return mg


def _n_chains(p):
    return len({s["chain"] for s in p.tn_plan_steps() if s["chain"] >= 0})


@pytest.mark.parametrize("bits_max", [5, 7, 9])
def test_grid3x4_chains_match_state_vector(bits_max):
    w = make_workload("grid3x4_m8")
    ref = sv.amplitudes(w.circuit, w.bits)
    got, p = run_plan(w.circuit, w.bits, w.tree.ssa, [], fuse=1, fuse_max_bits=bits_max)
    assert _n_chains(p) >= 2
    err = rel_l2(got, ref)
    print(f"grid3x4_m8 fused (d^t = {bits_max}, {_n_chains(p)} chains): rel-L2 {err:.2e}")
    assert err <= 1e-5


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_sliced_20_qubit_chains_match_state_vector(prec):
    c = random_circuit(grid_layout(4, 5), 12, seed=21)
    s = network_structure(c)
    bits = uniform_bitstrings(20, 1500, seed=5)
    ssa = candidate_trees(s, 1500, seed=2, trials=2)[0]
    sl = choose_slices(s, ContractionTree(ssa=ssa), 1500, n_sliced=2)
    ref = sv.amplitudes(c, bits)
    got, p = run_plan(c, bits, ssa, sl, precision=prec, fuse=1, slice_batch_log2=1)
    assert _n_chains(p) >= 2
    err = rel_l2(got, ref)
    print(f"20q fused {prec} ({_n_chains(p)} chains): rel-L2 {err:.2e}")
    assert err <= TOL[prec]


def test_fused_equals_unfused_closely_and_rescale_neutral():
    w = make_workload("grid3x4_m8")
    a, _ = run_plan(w.circuit, w.bits, w.tree.ssa, [], fuse=0)
    b, _ = run_plan(w.circuit, w.bits, w.tree.ssa, [], fuse=1)
    c, _ = run_plan(w.circuit, w.bits, w.tree.ssa, [], fuse=1, rescale=0)
    assert rel_l2(b, a) <= 1e-6
    # power-of-two rescaling is exact: with and without it the fused FP32
    # results are the same bits
    assert np.array_equal(b, c)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_grid5x6_fused_matches_stored_state_vector(prec):
    mg = _mg()
    _, ref = mg.read("grid5x6_m14")
    w = make_workload("grid5x6_m14")
    got, p = run_plan(w.circuit, w.bits, w.tree.ssa, w.tree.sliced, precision=prec, fuse=1)
    assert _n_chains(p) >= 10
    err = rel_l2(got, ref)
    print(f"grid5x6_m14 fused {prec} ({_n_chains(p)} chains): rel-L2 {err:.2e}")
    assert err <= TOL[prec]


def test_grid6x7_fused_sampled_slices():
    mg = _mg()
    rec = mg.read_json(mg.slices_path("grid6x7_m10"))
    w = make_workload("grid6x7_m10")
    bits = w.bits[rec["rows"]]
    got = run_slices(w.circuit, bits, rec["tree_ssa"], rec["sliced_edges"], rec["slice_ids"], precision="fp32",
                     fuse=1)
    err = rel_l2(got, rec["partials"])
    print(f"grid6x7_m10 fused fp32: rel-L2 over {got.size} partials {err:.3e}")
    assert err <= 1e-5


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_chains_fused_or_unfused_per_chain_and_autotuned(prec):
    # every chain can run fused or as its separate steps (tn_plan_set_chain);
    # both match the state vector, mixed settings too, and the autotuner
    # keeps a chain fused only where its kernel beat the sum of its steps
    torch, tn = require_cuda()
    c = random_circuit(grid_layout(4, 5), 12, seed=21)
    s = network_structure(c)
    bits = uniform_bitstrings(20, 1500, seed=5)
    ssa = candidate_trees(s, 1500, seed=2, trials=2)[0]
    sl = choose_slices(s, ContractionTree(ssa=ssa), 1500, n_sliced=2)
    ref = sv.amplitudes(c, bits)
    stream = torch.cuda.current_stream()
    p = tn.Plan(c, bits, ssa, sl, fuse=1, fuse_max_bits=9, rescale=1)
    nch = p.info["n_chains"]
    assert nch >= 2 and nch == _n_chains(p)
    ws = torch.empty(p.info["workspace_bytes"], dtype=torch.uint8, device="cuda")
    p.tn_plan_bind(ws, stream=stream)
    amps = torch.zeros(2 * len(bits), dtype=torch.float64, device="cuda")
    launches_fused = p.info["launches_per_call"]
    for pattern in ("all_off", "alternate", "all_on"):
        for ch in range(nch):
            p.tn_plan_set_chain(ch, {"all_off": 0, "alternate": ch & 1, "all_on": 1}[pattern])
        amps.zero_()
        p.tn_contract(amps, prec, stream=stream)
        p.tn_plan_check(stream=stream)
        torch.cuda.synchronize()
        err = rel_l2(amps.cpu().numpy().view(np.complex128), ref)
        print(f"20q {prec} chains {pattern}: rel-L2 {err:.2e}, launches {p.info['launches_per_call']}")
        assert err <= TOL[prec], (pattern, err)
        if pattern == "all_off":
            assert p.info["launches_per_call"] > launches_fused
    times = p.tn_plan_autotune(prec, amps, reps=1, stream=stream)
    on = p.tn_plan_get_chains()
    print(f"20q {prec}: autotuner keeps {int(on.sum())} of {nch} chains fused")
    amps.zero_()
    p.tn_contract(amps, prec, stream=stream)
    p.tn_plan_check(stream=stream)
    torch.cuda.synchronize()
    assert rel_l2(amps.cpu().numpy().view(np.complex128), ref) <= TOL[prec]
