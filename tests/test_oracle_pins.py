"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the property it checks.  None of them re-derives the
oracle's own formula: brute force uses per-gate full matrices, the
projector pin inserts |s><s| into a state-vector run, the closed forms are
written independently, and the planted-mistake tests show that a plausible
slip in the oracle (a transposed gate, the wrong bit order, a wire sliced
on the wrong side of a gate) fails a pin.
"""

import numpy as np
import pytest

from oracle import brute, sv, tn, xeb
from rqc import grid_layout, make_workload, network_structure, random_circuit
from rqc.bitstrings import bitstrings_from_indices, uniform_bitstrings
from rqc.circuit import Circuit, Gate, inverse_circuit, product_circuit
from rqc.tree import ContractionTree, candidate_trees, choose_slices


def _all_bits(n):
    return bitstrings_from_indices(np.arange(1 << n, dtype=np.uint64), n)


SMALL = [(grid_layout(2, 3), 8, 5), (grid_layout(3, 3), 6, 11), (grid_layout(2, 5), 10, 2)]


# P1: brute force ------------------------------------------------------------
@pytest.mark.parametrize("layout,cycles,seed", SMALL)
def test_sv_matches_brute_force_unitary(layout, cycles, seed):
    c = random_circuit(layout, cycles, seed)
    a = brute.amplitudes(c)
    assert np.max(np.abs(sv.state(c) - a)) < 1e-13
    u = brute.unitary(c)
    assert np.allclose(u.conj().T @ u, np.eye(u.shape[0]), atol=1e-12)


@pytest.mark.parametrize("layout,cycles,seed", SMALL)
def test_tn_matches_brute_force(layout, cycles, seed):
    c = random_circuit(layout, cycles, seed)
    n = c.n_qubits
    s = network_structure(c)
    ssa = candidate_trees(s, 1 << n, seed=seed, trials=2)[0]
    amps = tn.partial_amplitudes(c, ssa, _all_bits(n))[0]
    assert np.max(np.abs(amps - brute.amplitudes(c))) < 1e-13
    # a second, unrelated order gives the same numbers (c10)
    ssa2 = candidate_trees(s, 1, seed=seed + 100, trials=3)[-1]
    amps2 = tn.partial_amplitudes(c, ssa2, _all_bits(n))[0]
    assert np.max(np.abs(amps2 - amps)) < 1e-13


def test_tn_open_network_is_the_state():
    c = random_circuit(grid_layout(2, 3), 6, 3)
    net = tn.UnfusedNetwork(c)
    assert np.max(np.abs(net.contract_all_open() - brute.amplitudes(c))) < 1e-13


# P2: norm -------------------------------------------------------------------
@pytest.mark.parametrize("rows,cols,cycles", [(3, 4, 8), (4, 5, 12)])
def test_norm_is_one(rows, cols, cycles):
    psi = sv.state(random_circuit(grid_layout(rows, cols), cycles, seed=rows * cols))
    assert abs(np.vdot(psi, psi).real - 1.0) < 1e-12


# P3: circuit followed by its inverse ---------------------------------------
def test_circuit_then_inverse_returns_to_zero_state():
    c = inverse_circuit(random_circuit(grid_layout(3, 4), 8, seed=1001))
    zero = np.zeros((1, 12), np.uint8)
    assert abs(sv.amplitudes(c, zero)[0] - 1.0) < 1e-12
    s = network_structure(c)
    ssa = candidate_trees(s, 1, seed=4, trials=2)[0]
    assert abs(tn.partial_amplitudes(c, ssa, zero)[0, 0] - 1.0) < 1e-12


# P4: product state closed form ---------------------------------------------
def test_product_circuit_closed_form():
    c = product_circuit(6, 4, seed=9)
    mats = {q: np.eye(2, dtype=complex) for q in range(6)}
    for g in c.gates:
        (q,) = g.qubits
        mats[q] = g.matrix @ mats[q]
    bits = uniform_bitstrings(6, 20, seed=1)
    expect = np.array([np.prod([mats[q][b[q], 0] for q in range(6)]) for b in bits])
    assert np.max(np.abs(sv.amplitudes(c, bits) - expect)) < 1e-14


# P5/P6: Porter-Thomas and XEB (Eq. fxeb) -----------------------------------
def _deep_state():
    return sv.state(random_circuit(grid_layout(4, 5), 20, seed=77))


def test_porter_thomas_at_zero_fidelity():
    psi = _deep_state()
    n = 20
    x = np.sort((2 ** n) * np.abs(psi) ** 2)
    emp = np.arange(1, x.size + 1) / x.size
    d = np.max(np.abs(emp - xeb.porter_thomas_cdf(x, 0.0)))
    assert d < 5e-3, d
    # a shallow circuit is far from the law: the test discriminates
    shallow = sv.state(random_circuit(grid_layout(4, 5), 2, seed=77))
    xs = np.sort((2 ** n) * np.abs(shallow) ** 2)
    ds = np.max(np.abs(emp - xeb.porter_thomas_cdf(xs, 0.0)))
    assert ds > 0.05


def test_xeb_of_exact_samples_and_of_uniform_bitstrings():
    psi = _deep_state()
    n, k = 20, 20000
    p = np.abs(psi) ** 2
    rng = np.random.default_rng(5)
    idx = rng.choice(p.size, size=k, p=p / p.sum())
    f_exact = xeb.linear_xeb(psi[idx], n)
    assert abs(f_exact - 1.0) < 4 * np.sqrt(2.0 / k), f_exact
    uni = rng.integers(0, p.size, size=k)
    f_uni = xeb.linear_xeb(psi[uni], n)
    assert abs(f_uni) < 4 * np.sqrt(1.0 / k), f_uni
    # samples at fidelity F follow Eq. (fxeb): their mean x is 1 + F
    mix = np.where(rng.random(k) < 0.3, idx, uni)
    assert abs(xeb.linear_xeb(psi[mix], n) - 0.3) < 4 * np.sqrt(2.0 / k)


def test_porter_thomas_pdf_normalised_and_mean():
    x = np.linspace(0, 60, 600001)
    for f in (0.0, 0.002, 0.5, 1.0):
        pdf = xeb.porter_thomas_pdf(x, f)
        assert abs(np.trapezoid(pdf, x) - 1) < 1e-6
        assert abs(np.trapezoid(x * pdf, x) - (1 + f)) < 1e-6


# Slicing: projector pin and slicing invariance (P7) -----------------------
def _with_projectors(circ, wires, values):
    """The circuit with |v><v| inserted on each sliced wire (q, g), right
    after two-qubit gate g."""
    out = Circuit(n_qubits=circ.n_qubits, name=circ.name + "_proj")
    for gi, g in enumerate(circ.gates):
        out.gates.append(g)
        for (q, gg), v in zip(wires, values):
            if gg == gi:
                P = np.zeros((2, 2), complex)
                P[v, v] = 1.0
                out.gates.append(Gate((q,), P, g.layer, "proj"))
    return out


def _sliced_case():
    w = make_workload("grid3x4_m8")
    sl = choose_slices(w.struct, w.tree, 64, n_sliced=3)
    wires = [tuple(int(x) for x in w.struct.edge_wire[e]) for e in sl]
    return w, wires


def test_sliced_partials_equal_projected_state_vector():
    w, wires = _sliced_case()
    parts = tn.partial_amplitudes(w.circuit, w.tree.ssa, w.bits, wires, range(8))
    for s in range(8):
        vals = [(s >> j) & 1 for j in range(3)]
        ref = sv.amplitudes(_with_projectors(w.circuit, wires, vals), w.bits)
        assert np.max(np.abs(parts[s] - ref)) < 1e-14
    assert np.max(np.abs(parts)) > 1e-3


def test_slicing_invariance_sum_over_slices():
    w, wires = _sliced_case()
    parts = tn.partial_amplitudes(w.circuit, w.tree.ssa, w.bits, wires, range(8))
    amps = sv.amplitudes(w.circuit, w.bits)
    assert np.max(np.abs(parts.sum(axis=0) - amps)) < 1e-14
    assert np.max(np.abs(tn.partial_amplitudes(w.circuit, w.tree.ssa, w.bits)[0] - amps)) < 1e-14


def test_tn_matches_sv_on_the_12_qubit_workload():
    w = make_workload("grid3x4_m8")
    amps = sv.amplitudes(w.circuit, w.bits)
    parts = tn.partial_amplitudes(w.circuit, w.tree.ssa, w.bits)
    rel = np.linalg.norm(parts[0] - amps) / np.linalg.norm(amps)
    assert rel < 1e-13
    # this 8-cycle circuit is shallow for 12 qubits: report, do not demand, PT
    f = xeb.linear_xeb(amps, 12)
    assert abs(f) < 1.0


# Planted mistakes: each one fails a pin ------------------------------------
def _mutate(circ, fn):
    out = Circuit(n_qubits=circ.n_qubits, name=circ.name + "_mut")
    out.gates = [Gate(g.qubits, fn(g), g.layer, g.kind) for g in circ.gates]
    return out


def test_planted_transposed_two_qubit_gate_fails_brute_force():
    c = random_circuit(grid_layout(2, 3), 8, 5)
    bad = _mutate(c, lambda g: g.matrix.T.copy() if len(g.qubits) == 2 and g.layer == 3 else g.matrix)
    # fSim at Delta = 0 is symmetric; make the slip visible with a 1q gate too
    bad = _mutate(bad, lambda g: g.matrix.T.copy() if len(g.qubits) == 1 else g.matrix)
    assert np.max(np.abs(sv.state(bad) - brute.amplitudes(c))) > 1e-3


def test_planted_reversed_bit_order_fails_brute_force():
    c = random_circuit(grid_layout(2, 3), 8, 5)
    n = c.n_qubits
    bits = _all_bits(n)
    good = sv.amplitudes(c, bits)
    bad = sv.amplitudes(c, bits[:, ::-1])
    assert np.max(np.abs(good - brute.amplitudes(c))) < 1e-13
    assert np.max(np.abs(bad - brute.amplitudes(c))) > 1e-3


def test_planted_wrong_slice_wire_fails_projector_pin():
    w, wires = _sliced_case()
    # the slip: slicing the wire *before* the gate instead of after it
    net = tn.UnfusedNetwork(w.circuit)
    q, g = wires[0]
    prev = [gi for gi in range(g) if len(w.circuit.gates[gi].qubits) == 2 and q in w.circuit.gates[gi].qubits]
    if not prev:
        pytest.skip("first sliced wire has no earlier two-qubit gate")
    bad_wires = [(q, prev[-1])] + wires[1:]
    parts_bad = tn.partial_amplitudes(w.circuit, w.tree.ssa, w.bits, bad_wires, range(8))
    vals = [0, 0, 0]
    ref = sv.amplitudes(_with_projectors(w.circuit, wires, vals), w.bits)
    assert np.max(np.abs(parts_bad[0] - ref)) > 1e-4
    # ... although slicing invariance alone would not notice it
    amps = sv.amplitudes(w.circuit, w.bits)
    assert np.max(np.abs(parts_bad.sum(axis=0) - amps)) < 1e-13
    assert net.n_groups == 34
