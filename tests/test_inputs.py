"""Input generators: gate set, ABCD patterns, circuits, network structure,
trees and slices (SM Sec. I-II)."""

import numpy as np
import pytest

from rqc import (SQRT_W, SQRT_X, SQRT_Y, diamond_layout, fsim, grid_layout,
                 make_workload, network_structure, pattern_sequence,
                 random_circuit, uniform_bitstrings)
from rqc.bitstrings import bitstring_indices, bitstrings_from_indices
from rqc.tree import candidate_trees, estimate_cost, expected_width


def test_single_qubit_gates_are_the_printed_square_roots():
    # SM Sec. I: sqrt(X), sqrt(Y), sqrt(W) with the printed global phase;
    # each squares to its Pauli up to that phase.
    X = np.array([[0, 1], [1, 0]], complex)
    Y = np.array([[0, -1j], [1j, 0]], complex)
    W = (X + Y) / np.sqrt(2)
    for g, p in ((SQRT_X, X), (SQRT_Y, Y), (SQRT_W, W)):
        assert np.allclose(g.conj().T @ g, np.eye(2), atol=1e-15)
        sq = g @ g
        phase = sq[np.nonzero(p)][0] / p[np.nonzero(p)][0]
        assert abs(abs(phase) - 1) < 1e-15
        assert np.allclose(sq, phase * p, atol=1e-15)
    assert np.allclose(SQRT_X, np.sqrt(0.5) * np.array([[1, -1j], [-1j, 1]]))


def test_single_qubit_gates_entry_by_entry():
    # The matrices exactly as printed (SM Sec. I), row = output state: a
    # transposed sqrt(Y) or sqrt(W) squares to Y or W up to a phase as well,
    # so each entry is pinned on its own.
    h = np.sqrt(2.0) / 2.0
    printed = {
        "sqrtX": [[h, -1j * h], [-1j * h, h]],
        "sqrtY": [[h, -h], [h, h]],
        "sqrtW": [[h, -h * h * (1 + 1j)], [h * h * (1 - 1j), h]],
    }
    for g, name in ((SQRT_X, "sqrtX"), (SQRT_Y, "sqrtY"), (SQRT_W, "sqrtW")):
        for r in range(2):
            for c in range(2):
                assert abs(g[r, c] - printed[name][r][c]) < 1e-15, (name, r, c)
    # applied to |0>: sqrt(Y)|0> = (|0> + |1>)/sqrt(2), sqrt(W)|0> has the
    # phase (1 - i)/sqrt(2) on |1>
    assert np.allclose(SQRT_Y @ [1, 0], [h, h], atol=1e-15)
    assert np.allclose(SQRT_W @ [1, 0], [h, 0.5 * (1 - 1j)], atol=1e-15)


def test_fsim_pi2_pi6_closed_form():
    m = fsim(np.pi / 2, np.pi / 6)
    ref = np.zeros((4, 4), complex)
    ref[0, 0] = 1
    ref[1, 2] = ref[2, 1] = -1j
    ref[3, 3] = np.exp(-1j * np.pi / 6)
    assert np.allclose(m, ref, atol=1e-15)
    assert np.allclose(m.conj().T @ m, np.eye(4), atol=1e-15)


def test_pattern_sequences_match_the_paper():
    assert pattern_sequence(8) == "ABCDCDAB"
    assert pattern_sequence(12) == "ABCDCDABABCD"


@pytest.mark.parametrize("layout,ncoup", [(grid_layout(3, 4), 17), (grid_layout(5, 6), 49),
                                          (grid_layout(6, 7), 71), (diamond_layout(), 86)])
def test_patterns_are_matchings_covering_each_coupler_once(layout, ncoup):
    seen = []
    for p in "ABCD":
        qs = [q for c in layout.patterns[p] for q in c]
        assert len(qs) == len(set(qs)), f"pattern {p} is not a matching"
        seen.extend(layout.patterns[p])
    assert len(seen) == len(set(seen)) == ncoup


def test_diamond_has_53_qubits_with_nearest_neighbour_couplers():
    lay = diamond_layout()
    assert lay.n_qubits == 53
    deg = np.zeros(53, int)
    for a, b in lay.couplers:
        deg[a] += 1
        deg[b] += 1
    assert deg.max() <= 4 and deg.min() >= 1


@pytest.mark.parametrize("name,n2q", [("grid3x4_m8", 34), ("grid5x6_m14", 171),
                                      ("grid6x7_m10", 178), ("diamond53_m12", 258)])
def test_workload_gate_counts(name, n2q):
    from rqc.configs import WORKLOADS, _layout
    spec = WORKLOADS[name]
    c = random_circuit(_layout(spec.layout), spec.cycles, seed=1000 + spec.index)
    assert len(c.two_qubit_gates) == n2q
    assert len(c.gates) - n2q == c.n_qubits * (spec.cycles + 1)


def test_single_qubit_gates_never_repeat_on_a_qubit():
    c = random_circuit(grid_layout(3, 4), 20, seed=7)
    last = {}
    for g in c.gates:
        if len(g.qubits) == 1:
            q = g.qubits[0]
            assert last.get(q) != g.kind
            last[q] = g.kind


def test_bitstring_index_round_trip():
    idx = np.array([0, 1, 5, 2 ** 11 + 3, 4095], np.uint64)
    b = bitstrings_from_indices(idx, 12)
    assert b[2].tolist() == [0] * 9 + [1, 0, 1]
    assert np.array_equal(bitstring_indices(b), idx)
    u = uniform_bitstrings(12, 1000, seed=3)
    assert u.shape == (1000, 12) and set(np.unique(u)) <= {0, 1}


def test_network_structure_invariants():
    c = random_circuit(grid_layout(3, 4), 8, seed=1001)
    s = network_structure(c)
    assert s.n_tensors == 34
    cnt = np.zeros(s.n_edges, int)
    for t in range(s.n_tensors):
        for e in s.tensor_edges[t]:
            cnt[e] += 1
        assert len(s.tensor_edges[t]) + len(s.tensor_outputs[t]) <= 4
    assert np.all(cnt == 2)
    assert sorted(q for o in s.tensor_outputs for q in o) == list(range(12))
    # edge count: per qubit (number of 2q gates on it) - 1
    per_q = np.zeros(12, int)
    for g in c.two_qubit_gates:
        for q in g.qubits:
            per_q[q] += 1
    assert s.n_edges == int((per_q - 1).sum())
    for e, (q, g) in enumerate(s.edge_wire):
        assert q in c.gates[g].qubits and len(c.gates[g].qubits) == 2


def test_expected_width_formula():
    assert expected_width(0, 100) == 1.0
    assert abs(expected_width(3, 10 ** 6) - 8) < 1e-9
    assert abs(expected_width(40, 1000) - 1000) < 1e-3


def _check_ssa(ssa, T):
    used = np.zeros(2 * T - 1, int)
    for i, (a, b) in enumerate(ssa):
        assert a < T + i and b < T + i and a != b
        used[a] += 1
        used[b] += 1
    assert np.all(used[:-1] == 1) and used[-1] == 0


def test_trees_are_valid_ssa_and_sliced_counts():
    w = make_workload("grid3x4_m8")
    _check_ssa(w.tree.ssa, w.struct.n_tensors)
    for ssa in candidate_trees(w.struct, 64, seed=1, trials=3):
        _check_ssa(ssa, w.struct.n_tensors)
    w2 = make_workload("grid5x6_m14")
    _check_ssa(w2.tree.ssa, w2.struct.n_tensors)
    assert len(w2.tree.sliced) == 10
    c = estimate_cost(w2.struct, w2.tree.ssa, 4096, w2.tree.sliced)
    assert c.max_rank <= 28


def test_refine_slices_keeps_size_and_rank_and_never_raises_cost():
    from rqc.tree import ContractionTree, choose_slices, refine_slices
    w = make_workload("grid3x4_m8")
    for seed in (1, 2):
        ssa = candidate_trees(w.struct, 64, seed=seed, trials=2)[0]
        tree = ContractionTree(ssa=ssa)
        sl = choose_slices(w.struct, tree, 64, n_sliced=2)
        c0 = estimate_cost(w.struct, ssa, 64, sl)
        ref = refine_slices(w.struct, tree, 64, sl, max_evals=300)
        c1 = estimate_cost(w.struct, ssa, 64, ref)
        assert len(ref) == len(set(ref)) == len(sl)
        assert all(0 <= e < w.struct.n_edges for e in ref)
        assert c1.flops <= c0.flops and c1.max_rank <= c0.max_rank
