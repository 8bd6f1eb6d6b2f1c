"""Brute-force circuit unitary (test only; n <= 10).

Each gate is expanded to its full 2^n x 2^n matrix element by element from
the definition: <y| G_full |x> = G[y restricted to the gate's qubits,
x restricted to the gate's qubits] when y and x agree on every other
qubit, else 0.  The circuit unitary is the product of those matrices in
time order.  Nothing here is shared with the state-vector code.
"""

import numpy as np


def _bit(x, q, n):
    return (x >> (n - 1 - q)) & 1


def gate_full(gate, n):
    dim = 1 << n
    full = np.zeros((dim, dim), np.complex128)
    qs = gate.qubits
    others = [q for q in range(n) if q not in qs]
    for x in range(dim):
        xin = 0
        for q in qs:
            xin = 2 * xin + _bit(x, q, n)
        for yin in range(1 << len(qs)):
            y = x
            for j, q in enumerate(qs):
                bitval = (yin >> (len(qs) - 1 - j)) & 1
                mask = 1 << (n - 1 - q)
                y = (y | mask) if bitval else (y & ~mask)
            # other qubits untouched by construction
            assert all(_bit(y, q, n) == _bit(x, q, n) for q in others)
            full[y, x] += gate.matrix[yin, xin]
    return full


def unitary(circ):
    n = circ.n_qubits
    if n > 10:
        raise ValueError("brute force is limited to n <= 10")
    u = np.eye(1 << n, dtype=np.complex128)
    for g in circ.gates:
        u = gate_full(g, n) @ u
    return u


def amplitudes(circ):
    """All 2^n amplitudes <x|U|0>, the first column of the unitary."""
    return unitary(circ)[:, 0].copy()
