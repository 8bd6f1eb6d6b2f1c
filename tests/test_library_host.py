"""Host-side checks of the CUDA library: it loads, exports every entry point
declared in include/tn.h, builds the same network as the input generators,
and its reuse-instance DAG has the widths of Eq. (1) (brute-force counts,
the paper's bounds, and the uniform-bitstring law behind Table S2).  No
GPU is touched: tn_plan is host-only.
"""

import os
import re

import numpy as np
import pytest

from rqc import make_workload, network_structure, random_circuit, grid_layout
from rqc.bitstrings import uniform_bitstrings
from rqc.tree import candidate_trees, expected_width


@pytest.fixture(scope="module")
def tn():
    from paper_2212_04749_gb300 import builder
    builder.build()
    from paper_2212_04749_gb300 import tn as mod
    mod.load()
    return mod


def test_library_exports_every_declared_entry_point(tn, root):
    hdr = open(os.path.join(root, "include", "tn.h")).read()
    declared = set(re.findall(r"^\s*(?:int|void|size_t|const char \*)\s*(tn_\w+)\s*\(", hdr, re.M))
    assert declared, "no declarations parsed"
    lib = tn.load()
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared == set(tn.EXPORTS)


@pytest.mark.parametrize("name", ["grid3x4_m8", "grid5x6_m14", "diamond53_m12"])
def test_network_matches_generator_structure(tn, name):
    w = make_workload(name)
    nt, ne, ends, outs = tn.tn_network(w.circuit)
    assert nt == w.struct.n_tensors and ne == w.struct.n_edges
    assert np.array_equal(ends, w.struct.edge_ends)
    for q in range(w.circuit.n_qubits):
        assert q in w.struct.tensor_outputs[outs[q]]


def _subtree_outs(struct, ssa):
    T = struct.n_tensors
    outs = [set(struct.tensor_outputs[t]) for t in range(T)]
    for a, b in ssa:
        outs.append(outs[a] | outs[b])
    return outs


@pytest.mark.parametrize("name", ["grid3x4_m8", "grid5x6_m14"])
def test_widths_are_distinct_projection_counts(tn, name):
    w = make_workload(name)
    p = tn.Plan(w.circuit, w.bits, w.tree.ssa, w.tree.sliced)
    width, rank, nsl = p.tn_plan_widths()
    outs = _subtree_outs(w.struct, w.tree.ssa)
    ku = len({b.tobytes() for b in w.bits})
    for v, o in enumerate(outs):
        cols = sorted(o)
        brute = len({row.tobytes() for row in w.bits[:, cols]}) if cols else 1
        assert width[v] == brute, v
    # Eq. (1) bounds: the root carries every bitstring, widths never shrink
    # towards the root, a leaf carries at most its 2 output legs' 4 values
    assert width[-1] == ku
    T = w.struct.n_tensors
    for i, (a, b) in enumerate(w.tree.ssa):
        assert width[T + i] >= max(width[a], width[b])
        assert width[T + i] <= width[a] * width[b]
    assert width[:T].max() <= 4


def test_widths_follow_the_uniform_occupancy_law(tn):
    # the law the paper's Table S2 widths obey (2^j (1-(1-2^-j)^k)); for
    # k = 3e6 it gives 988,587 at j = 20 against the printed 981,285
    c = random_circuit(grid_layout(4, 5), 6, seed=12)
    s = network_structure(c)
    k = 3000
    bits = uniform_bitstrings(20, k, seed=99)
    ssa = candidate_trees(s, k, seed=1, trials=1)[0]
    p = tn.Plan(c, bits, ssa, [])
    width, _, _ = p.tn_plan_widths()
    outs = _subtree_outs(s, ssa)
    for v, o in enumerate(outs):
        j = len(o)
        mu = expected_width(j, k)
        # variance of the occupied-bin count is below its mean
        assert abs(width[v] - mu) <= 6 * np.sqrt(max(mu, 1.0)) + 1, (v, j, width[v], mu)
    assert abs(expected_width(20, 3 * 10 ** 6) - 988587) < 1
    assert abs(expected_width(16, 3 * 10 ** 6) - 65536) < 1


def test_all_amplitudes_give_doubling_widths(tn):
    # SM Sec. III.B: computing all 2^n amplitudes, every output leg met
    # doubles the width (w_l = 2^{l-1})
    w = make_workload("grid3x4_m8")
    allbits = ((np.arange(4096)[:, None] >> np.arange(11, -1, -1)[None, :]) & 1).astype(np.uint8)
    p = tn.Plan(w.circuit, allbits, w.tree.ssa, [])
    width, _, _ = p.tn_plan_widths()
    outs = _subtree_outs(w.struct, w.tree.ssa)
    for v, o in enumerate(outs):
        assert width[v] == 2 ** len(o)


def _eq1_flops(w, p):
    width, rank, nsl = p.tn_plan_widths()
    T = w.struct.n_tensors
    total = 0.0
    for i, (a, b) in enumerate(w.tree.ssa):
        v = T + i
        union = (rank[a] + rank[b] + rank[v]) // 2
        total += 8.0 * (2.0 ** union) * (2.0 ** nsl[v]) * width[v]
    return total


@pytest.mark.parametrize("name", ["grid3x4_m8", "grid5x6_m14"])
def test_plan_cost_is_eq1_and_executed_without_recomputation(tn, name):
    w = make_workload(name)
    p = tn.Plan(w.circuit, w.bits, w.tree.ssa, w.tree.sliced)
    info = p.info
    assert info["flops_ma"] == pytest.approx(_eq1_flops(w, p), rel=1e-12)
    # the slice loop recomputes a node only when one of its sliced values
    # changes; with the plan's slice order that is (nearly) never more often
    # than Eq. (1) counts
    assert info["flops_ma"] <= info["flops_exec"] <= info["flops_ma"] * (1 + 1e-4)
    assert info["flops_ma"] < info["flops_sa"]
    steps = p.tn_plan_steps()
    assert len(steps) == w.struct.n_tensors - 1
    assert sum(s["flops"] * s["runs"] for s in steps) == pytest.approx(info["flops_exec"], rel=1e-12)


def test_n64_steps_carry_padded_pair_tiles(tn):
    # steps with N = 64 (one 64-column tile per output instance) carry the
    # tile space of the tensor cores' column-tile pairs: each group's tiles
    # padded to an even count, so the pad tiles are the groups of odd size
    w = make_workload("diamond53_m12")
    p = tn.Plan(w.circuit, w.bits, w.tree.ssa, w.tree.sliced, workspace_limit=120 << 30)
    steps = p.tn_plan_steps()
    n64 = [s for s in steps if s["nb"] == 6]
    assert n64
    for s in steps:
        if s["nb"] != 6:
            assert s["n_pair_tiles"] == 0
            continue
        n, g, mg, npt = s["n_inst"], s["n_groups"], s["max_group"], s["n_pair_tiles"]
        odd = npt - n  # groups of odd size
        assert npt % 2 == 0 and 0 <= odd <= g
        assert odd % 2 == n % 2  # the sizes sum to n
        assert 1 <= mg <= n and mg * g >= n
        if mg == 1:
            assert odd == g
        if n == g * mg and mg % 2 == 0:
            assert odd == 0
    # groups of both parities in one step (the 2^10 x 2^9 x 2^6 step: 8113
    # instances in 256 groups)
    assert any(0 < s["n_pair_tiles"] - s["n_inst"] < s["n_groups"] for s in n64)


def test_slice_batch_trades_memory_for_passes(tn):
    w = make_workload("grid5x6_m14")
    infos = [tn.Plan(w.circuit, w.bits, w.tree.ssa, w.tree.sliced, slice_batch_log2=b).info for b in (2, 5)]
    assert infos[0]["n_batches"] == 2 ** 8 and infos[1]["n_batches"] == 2 ** 5
    assert infos[0]["workspace_bytes"] < infos[1]["workspace_bytes"]
    assert infos[0]["flops_exec"] == pytest.approx(infos[1]["flops_exec"], rel=1e-4)


def test_duplicate_bitstrings_are_planned_once(tn):
    w = make_workload("grid3x4_m8")
    bits = np.concatenate([w.bits, w.bits[:10]])
    p = tn.Plan(w.circuit, bits, w.tree.ssa, [])
    assert p.info["n_unique"] == 64


@pytest.mark.parametrize("case", ["tree_reuse", "tree_forward", "bits_value", "slice_range", "slice_dup"])
def test_invalid_inputs_are_rejected(tn, case):
    w = make_workload("grid3x4_m8")
    ssa, bits, sl = w.tree.ssa.copy(), w.bits.copy(), [0, 1]
    if case == "tree_reuse":
        ssa[5] = ssa[4]
    elif case == "tree_forward":
        ssa[0, 0] = 60
    elif case == "bits_value":
        bits[3, 4] = 2
    elif case == "slice_range":
        sl = [10 ** 6]
    else:
        sl = [3, 3]
    with pytest.raises(tn.TnError) as ei:
        tn.Plan(w.circuit, bits, ssa, sl)
    assert ei.value.code == tn.TN_EINVAL
    assert str(ei.value)


def test_qubit_without_two_qubit_gate_is_rejected(tn):
    from rqc.circuit import product_circuit
    with pytest.raises(tn.TnError):
        tn.tn_network(product_circuit(3, 2, seed=1))


def test_contract_before_bind_is_a_state_error(tn):
    w = make_workload("grid3x4_m8")
    p = tn.Plan(w.circuit, w.bits, w.tree.ssa, [])
    with pytest.raises(tn.TnError) as ei:
        p.tn_contract(12345, "fp32")
    assert ei.value.code == tn.TN_ESTATE


def _row_allowed(st):
    return st["nb"] <= 4 and st["kb"] + st["nb"] <= 8


@pytest.mark.parametrize("name", ["grid3x4_m8", "grid5x6_m14"])
def test_features_and_config_eligibility(tn, name):
    # one row of TN_NFEAT features per step; the per-row configurations are
    # allowed exactly where the per-row kernel's shape condition holds, the
    # GEMM ones everywhere; the one-hot blocks are one-hot
    w = make_workload(name)
    p = tn.Plan(w.circuit, w.bits, w.tree.ssa, w.tree.sliced)
    steps = p.tn_plan_steps()
    for prec in ("fp32", "tf32", "bf16x3"):
        for c in range(tn.TN_NCONFIG):
            f, ok = p.tn_plan_features(prec, c)
            assert f.shape == (len(steps), tn.TN_NFEAT)
            assert np.all(np.isfinite(f)) and np.all(np.abs(f) <= 2.0)
            want = np.array([c >= 2 or _row_allowed(st) for st in steps])
            assert np.array_equal(ok, want)
            assert np.all(f[:, 19] + f[:, 20] + f[:, 21] == 1.0)  # exactly one kernel family
            assert np.all(f[:, 22] == (c & 1))
            assert np.all(f[:, 17] == (prec == "tf32")) and np.all(f[:, 18] == (prec == "bf16x3"))
            if prec == "fp32":
                assert not np.any(f[:, 20])  # no tensor cores in FP32
            np.testing.assert_allclose(f[:, 0] * 32, [st["mb"] for st in steps])
            np.testing.assert_allclose(f[:, 1] * 32, [st["kb"] for st in steps])
            np.testing.assert_allclose(f[:, 2] * 32, [st["nb"] for st in steps])


def test_config_override_rules(tn):
    w = make_workload("grid5x6_m14")
    p = tn.Plan(w.circuit, w.bits, w.tree.ssa, w.tree.sliced)
    steps = p.tn_plan_steps()
    base = p.tn_plan_get_configs()
    assert np.array_equal(base, [0 if st["kernel"] == 0 else 2 for st in steps])
    big = next(i for i, st in enumerate(steps) if not _row_allowed(st))
    with pytest.raises(tn.TnError) as ei:
        p.tn_plan_set_config(big, 1)
    assert ei.value.code == tn.TN_EINVAL
    for bad in (-2, tn.TN_NCONFIG):
        with pytest.raises(tn.TnError):
            p.tn_plan_set_config(0, bad)
    p.tn_plan_set_config(big, 3)
    p.tn_plan_set_kernel(0, 1)
    got = p.tn_plan_get_configs()
    assert got[big] == 3 and got[0] == 2
    p.tn_plan_set_config(big, -1)
    assert p.tn_plan_get_configs()[big] == base[big]


def test_tensor_core_switches(tn):
    # the resident-B and column-tile-pair switches act at launch time: a
    # null plan is an argument error, and either setting leaves the plan's
    # configuration choices as they were
    lib = tn.load()
    for fn in ("tn_plan_set_tc_resident_b", "tn_plan_set_tc_pairs"):
        assert getattr(lib, fn)(None, 1) == tn.TN_EINVAL
    w = make_workload("grid5x6_m14")
    p = tn.Plan(w.circuit, w.bits, w.tree.ssa, w.tree.sliced)
    base = p.tn_plan_get_configs()
    for on in (False, True):
        p.tn_plan_set_tc_pairs(on)
        p.tn_plan_set_tc_resident_b(on)
        assert np.array_equal(p.tn_plan_get_configs(), base)


@pytest.mark.parametrize("name", ["grid3x4_m8", "grid5x6_m14"])
def test_fused_chains_are_well_formed(tn, name):
    # every chain: consecutive producer -> consumer steps on the A side,
    # small side operands, one slice level, equal instance counts; the plan
    # launches fewer kernels and counts fewer algorithmic bytes
    w = make_workload(name)
    p0 = tn.Plan(w.circuit, w.bits, w.tree.ssa, w.tree.sliced, fuse=0)
    p1 = tn.Plan(w.circuit, w.bits, w.tree.ssa, w.tree.sliced, fuse=1)
    st = p1.tn_plan_steps()
    chains = {}
    for i, s in enumerate(st):
        if s["chain"] >= 0:
            chains.setdefault(s["chain"], []).append(i)
    assert chains
    for ids in chains.values():
        assert 2 <= len(ids) <= 6 and ids == sorted(ids)
        assert [st[i]["chain_last"] for i in ids] == [0] * (len(ids) - 1) + [1]
        for i, j in zip(ids, ids[1:]):
            assert st[j]["a"] == st[i]["node"]
            assert st[j]["n_inst"] == st[i]["n_inst"] and st[j]["level"] == st[i]["level"]
        for i in ids:
            assert st[i]["kb"] + st[i]["nb"] <= 8
    assert p1.info["launches_per_call"] < p0.info["launches_per_call"]
    assert p1.info["bytes_min"] < p0.info["bytes_min"]
    assert p1.info["flops_exec"] == p0.info["flops_exec"]


def test_chains_follow_data_dependency_not_step_order(tn):
    # The TNCO rearrangement of paper SM Sec. V.B: a chain is a run of
    # producer -> consumer steps, and it runs at its last step, which moves
    # its earlier steps next to their consumers.  That is legal because every
    # side operand B_j is produced earlier in the tree's order.  Fusing only
    # steps that are adjacent in the tree's own order finds fewer fused steps.
    w = make_workload("grid5x6_m14")
    p = tn.Plan(w.circuit, w.bits, w.tree.ssa, w.tree.sliced, fuse=1)
    st = p.tn_plan_steps()
    step_of = {s["node"]: i for i, s in enumerate(st)}
    chains = {}
    for i, s in enumerate(st):
        if s["chain"] >= 0:
            chains.setdefault(s["chain"], []).append(i)
    rearranged = [ids for ids in chains.values() if ids[-1] - ids[0] != len(ids) - 1]
    assert rearranged
    for ids in rearranged:
        for i in ids:
            b = st[i]["b"]
            assert b not in step_of or step_of[b] < ids[-1]  # side operands exist by the chain's last step
    # steps fused when a chain may only continue into the next step in order
    adjacent = sum(len(ids) for ids in chains.values()
                   if all(j == i + 1 for i, j in zip(ids, ids[1:])))
    fused = sum(len(ids) for ids in chains.values())
    assert fused > adjacent


def test_open_qubits_plan_structure(tn):
    # correlated batches: open output qubits reach the root, whose instances
    # then hold 2^r amplitudes; rows equal up to their open bits share one
    # distinct bitstring; bad masks and sliced open legs are rejected
    w = make_workload("grid3x4_m8")
    bits = w.bits.copy()
    bits[1] = bits[0]
    bits[1, 5] ^= 1  # differs from row 0 only at an open qubit
    p = tn.Plan(w.circuit, bits, w.tree.ssa, w.tree.sliced, open_qubits=[2, 5, 11])
    assert p.info["n_open"] == 3 and p.info["amps_per_row"] == 8
    masked = bits.copy()
    masked[:, [2, 5, 11]] = 0
    assert p.info["n_unique"] == len({r.tobytes() for r in masked})
    assert p.info["n_unique"] < len({r.tobytes() for r in bits})
    width, rank, _ = p.tn_plan_widths()
    assert rank[-1] == 3 and width[-1] == p.info["n_unique"]
    with pytest.raises(Exception):
        tn.Plan(w.circuit, bits, w.tree.ssa, w.tree.sliced, open_mask=1 << 12)
    nt, ne, ends, outs = tn.tn_network(w.circuit)
    with pytest.raises(Exception):  # edge id ne would be an open leg: not a bond
        tn.Plan(w.circuit, bits, w.tree.ssa, [ne], open_qubits=[0])
