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
    # the benchmark's tree comes from the tree search; it must be a
    # tree of exactly this circuit's network and keep every intermediate
    # within the 2^32-entry cap of the workload
    w = make_workload("diamond53_m12")
    T = w.struct.n_tensors
    _valid(np.asarray(w.tree.ssa), T)
    c = estimate_cost(w.struct, w.tree.ssa, w.bits.shape[0], w.tree.sliced)
    assert c.max_rank <= 32
    seeded = make_workload("diamond53_m12", seeded_tree=True)
    assert c.flops < estimate_cost(seeded.struct, seeded.tree.ssa, w.bits.shape[0]).flops


class _FlopsRanker:
    """Stands in for the cost-model ranker: predicts a tree's time as its
    Eq. (1) flops (no GPU), unsliced."""

    def __init__(self, w):
        self.struct, self.k, self.max_rank = w.struct, w.bits.shape[0], None

    def slice(self, ssa):
        return [], estimate_cost(self.struct, ssa, self.k)

    def predict(self, ssa, sl):
        return {"predicted_ms": estimate_cost(self.struct, ssa, self.k).flops / 1e6}


def test_measured_climb_moves_only_on_measured_gains():
    # measured time and prediction both = the tree's flops: the walk must
    # end on a tree no worse than it started, move only on a measured gain
    # of at least min_gain, and measure only valid trees
    from paper_2212_04749_gb300.treesearch import measured_climb
    w = make_workload("grid3x4_m8")
    T = w.struct.n_tensors
    rk = _FlopsRanker(w)
    calls = []

    def fake_measure(ssa, sl):
        _valid(ssa, T)
        calls.append(1)
        return estimate_cost(w.struct, ssa, rk.k).flops / 1e6

    start = np.asarray(w.tree.ssa)
    best, walk = measured_climb(rk, start, fake_measure, steps=6, per_step=60, k_measure=3, min_gain=0.01)
    t0 = walk[0]["measured_ms"]
    assert best["measured_ms"] <= t0
    assert len(calls) == len(walk) and len(walk) <= 1 + 6 * 3
    cur = t0
    for step in sorted({r["step"] for r in walk if r["step"] >= 0}):
        got = min(r["measured_ms"] for r in walk if r["step"] == step)
        if got < cur * 0.99:
            cur = got
    assert best["measured_ms"] == cur
    _valid(np.asarray(best["ssa"]), T)

    # a measurement that never improves: the walk stops after one step
    flat = lambda ssa, sl: 1.0  # noqa: E731
    best2, walk2 = measured_climb(rk, start, flat, steps=6, per_step=60, k_measure=3)
    assert best2["measured_ms"] == 1.0 and max(r["step"] for r in walk2) == 0


def test_measured_climb_stops_on_an_unplannable_start():
    from paper_2212_04749_gb300.treesearch import measured_climb
    w = make_workload("grid3x4_m8")
    best, walk = measured_climb(_FlopsRanker(w), np.asarray(w.tree.ssa), lambda ssa, sl: None, steps=3)
    assert best["measured_ms"] is None and len(walk) == 1
