"""Seeded random quantum circuits of the Sycamore family (SM Sec. I).

A circuit of m cycles on a layout is: for t = 0..m-1, a layer of
single-qubit gates on every qubit followed by the two-qubit layer of
pattern ``pattern_sequence(m)[t]``; then one final single-qubit layer, so
there are m+1 single-qubit layers.  Single-qubit gates are drawn uniformly
from {sqrtX, sqrtY, sqrtW} in the first layer and, in later layers,
uniformly from the two gates that differ from the previous gate on the same
qubit.  Every two-qubit gate is fSim(theta, phi).  The input state is
|0...0>.

Gate list order is the time order of the circuit; within a layer gates are
listed by ascending qubit (single-qubit) or ascending coupler (two-qubit).
"""

from dataclasses import dataclass, field
from typing import List

import numpy as np

from .gates import SINGLE_QUBIT_GATES, fsim
from .layouts import Layout, pattern_sequence


@dataclass
class Gate:
    qubits: tuple          # (q,) or (a, b) with a < b
    matrix: np.ndarray     # 2x2 or 4x4 complex128, row = output index
    layer: int             # 2*t for single-qubit layer t, 2*t+1 for two-qubit layer t
    kind: str = ""         # gate name, informational


@dataclass
class Circuit:
    n_qubits: int
    gates: List[Gate] = field(default_factory=list)
    name: str = ""

    @property
    def two_qubit_gates(self) -> List[Gate]:
        return [g for g in self.gates if len(g.qubits) == 2]

    def to_arrays(self):
        """Flat arrays for a C interface: q0, q1 (-1 for 1q), layer, and the
        row-major complex128 matrix padded to 16 entries (re, im interleaved)."""
        g = len(self.gates)
        q0 = np.empty(g, np.int32)
        q1 = np.empty(g, np.int32)
        layer = np.empty(g, np.int32)
        m = np.zeros((g, 32), np.float64)
        for i, gate in enumerate(self.gates):
            q0[i] = gate.qubits[0]
            q1[i] = gate.qubits[1] if len(gate.qubits) == 2 else -1
            layer[i] = gate.layer
            flat = np.asarray(gate.matrix, np.complex128).reshape(-1)
            m[i, 0 : 2 * flat.size : 2] = flat.real
            m[i, 1 : 2 * flat.size : 2] = flat.imag
        return q0, q1, layer, m


def random_circuit(layout: Layout, cycles: int, seed: int,
                   theta: float = np.pi / 2, phi: float = np.pi / 6) -> Circuit:
    rng = np.random.default_rng(seed)
    n = layout.n_qubits
    two = fsim(theta, phi)
    seq = pattern_sequence(cycles)
    circ = Circuit(n_qubits=n, name=f"{layout.name}_m{cycles}_s{seed}")
    prev = np.full(n, -1, dtype=np.int64)

    def one_qubit_layer(layer_idx):
        for q in range(n):
            if prev[q] < 0:
                choice = int(rng.integers(0, 3))
            else:
                others = [c for c in range(3) if c != prev[q]]
                choice = others[int(rng.integers(0, 2))]
            prev[q] = choice
            circ.gates.append(Gate((q,), SINGLE_QUBIT_GATES[choice].copy(),
                                   2 * layer_idx, ("sqrtX", "sqrtY", "sqrtW")[choice]))

    for t in range(cycles):
        one_qubit_layer(t)
        for (a, b) in layout.patterns[seq[t]]:
            circ.gates.append(Gate((a, b), two.copy(), 2 * t + 1, "fsim"))
    one_qubit_layer(cycles)
    return circ


def product_circuit(n_qubits: int, layers: int, seed: int) -> Circuit:
    """Single-qubit gates only (no entanglement): used to pin amplitudes to
    the closed form prod_q (G_q ... G_1)[b_q, 0]."""
    rng = np.random.default_rng(seed)
    circ = Circuit(n_qubits=n_qubits, name=f"product{n_qubits}_l{layers}_s{seed}")
    for t in range(layers):
        for q in range(n_qubits):
            c = int(rng.integers(0, 3))
            circ.gates.append(Gate((q,), SINGLE_QUBIT_GATES[c].copy(), 2 * t))
    return circ


def inverse_circuit(circ: Circuit) -> Circuit:
    """The circuit followed by its inverse (conjugate-transposed gates in
    reverse order): it maps |0...0> back to |0...0>."""
    out = Circuit(n_qubits=circ.n_qubits, name=circ.name + "_inv")
    out.gates = list(circ.gates)
    last = max(g.layer for g in circ.gates) + 1
    for i, g in enumerate(reversed(circ.gates)):
        out.gates.append(Gate(g.qubits, np.conj(g.matrix.T).copy(), last + i, g.kind + "^dag"))
    return out
