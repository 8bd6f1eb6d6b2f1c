"""Host logic of the tree search: tree rotations stay valid contraction
trees of the same network, and contracting along one gives the same
amplitudes (the oracle's own contractor follows the tree)."""

import numpy as np

from oracle import sv
from oracle import tn as otn
from paper_2212_04749_gb300.treesearch import _children, _to_ssa, rotations
from rqc import make_workload
from rqc.tree import estimate_cost


def _valid(ssa, T):
    seen = set()
    for i, (a, b) in enumerate(np.asarray(ssa)):
        for x in (a, b):
            assert 0 <= x < T + i, "a child must exist before its parent"
            assert x not in seen, "every node is used once"
            seen.add(int(x))
    assert seen == set(range(2 * T - 2))


def test_round_trip_and_rotations_are_valid_trees():
    w = make_workload("grid3x4_m8")
    T = w.struct.n_tensors
    ssa = np.asarray(w.tree.ssa)
    back = _to_ssa(_children(ssa, T), 2 * T - 2, T)
    _valid(back, T)
    assert estimate_cost(w.struct, back, 64).flops == estimate_cost(w.struct, ssa, 64).flops
    nb = rotations(ssa, T)
    assert len(nb) >= T  # about four per internal node with an internal child
    costs = set()
    for r in nb:
        _valid(r, T)
        costs.add(round(estimate_cost(w.struct, r, 64).flops))
    assert len(costs) > 1  # rotations reach trees of other costs


def test_contracting_along_a_rotated_tree_gives_the_same_amplitudes():
    w = make_workload("grid3x4_m8")
    T = w.struct.n_tensors
    ref = sv.amplitudes(w.circuit, w.bits[:8])
    for r in rotations(np.asarray(w.tree.ssa), T)[::9]:
        got = otn.partial_amplitudes(w.circuit, r, w.bits[:8])[0]
        assert np.max(np.abs(got - ref)) < 1e-13


def test_stored_diamond53_tree_is_a_valid_tree_of_its_circuit():
    # the benchmark's tree comes from the time-ranked search; it must be a
    # tree of exactly this circuit's network and keep every intermediate
    # within the 2^32-entry cap of the workload
    w = make_workload("diamond53_m12")
    T = w.struct.n_tensors
    _valid(np.asarray(w.tree.ssa), T)
    c = estimate_cost(w.struct, w.tree.ssa, w.bits.shape[0], w.tree.sliced)
    assert c.max_rank <= 32
    seeded = make_workload("diamond53_m12", seeded_tree=True)
    assert c.flops < estimate_cost(seeded.struct, seeded.tree.ssa, w.bits.shape[0]).flops
