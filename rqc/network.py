"""Connectivity of the fused tensor network of a circuit (SM Sec. II).

Only structure lives here (which tensor touches which wire); the tensor
entries are computed by each consumer on its own.

Definition used by every part of this project:

* One tensor per two-qubit gate, numbered 0..T-1 in gate-list order.  All
  single-qubit gates and the |0> inputs are absorbed into two-qubit gates
  (SM Sec. II): a single-qubit gate goes into the next two-qubit gate on its
  qubit; the final single-qubit layer goes into the last two-qubit gate on
  its qubit.
* A bond edge is the wire segment of qubit q between two consecutive
  two-qubit gates on q.  Bond edges are numbered 0..E-1 in creation order:
  walk the two-qubit gates in gate-list order and, for each gate (a, b), for
  q in (a, b): if q already saw a two-qubit gate, the segment from that gate
  to this one gets the next id.
* The output leg of qubit q sits on the last two-qubit gate acting on q.
* Every qubit must take part in at least one two-qubit gate.

``edge_wire[e] = (q, g)`` names bond edge e by circuit location: the wire
of qubit q right after the two-qubit gate whose index in the *full* gate
list is g.  Slicing that wire is the same operation on any network built
from the circuit, fused or not.
"""

from dataclasses import dataclass
from typing import List, Tuple

import numpy as np

from .circuit import Circuit


@dataclass
class NetworkStructure:
    n_qubits: int
    n_tensors: int
    n_edges: int
    tensor_gate: np.ndarray            # (T,) index into circuit.gates
    tensor_qubits: np.ndarray          # (T, 2)
    tensor_edges: List[List[int]]      # bond edges of each tensor
    tensor_outputs: List[List[int]]    # output qubits whose leg is on the tensor
    edge_ends: np.ndarray              # (E, 2) tensor ids, [earlier, later]
    edge_wire: np.ndarray              # (E, 2) (qubit, full gate index before the wire)

    def edge_mask(self, t: int) -> int:
        m = 0
        for e in self.tensor_edges[t]:
            m |= 1 << e
        return m

    def out_mask(self, t: int) -> int:
        m = 0
        for q in self.tensor_outputs[t]:
            m |= 1 << q
        return m


def network_structure(circ: Circuit) -> NetworkStructure:
    n = circ.n_qubits
    last = [-1] * n                    # tensor id of last two-qubit gate seen on q
    tensor_gate, tensor_qubits = [], []
    tensor_edges: List[List[int]] = []
    ends: List[Tuple[int, int]] = []
    wires: List[Tuple[int, int]] = []
    for gi, g in enumerate(circ.gates):
        if len(g.qubits) != 2:
            continue
        t = len(tensor_gate)
        tensor_gate.append(gi)
        tensor_qubits.append(g.qubits)
        tensor_edges.append([])
        for q in g.qubits:
            if last[q] >= 0:
                e = len(ends)
                ends.append((last[q], t))
                wires.append((q, int(tensor_gate[last[q]])))
                tensor_edges[last[q]].append(e)
                tensor_edges[t].append(e)
            last[q] = t
    if any(x < 0 for x in last):
        raise ValueError("every qubit needs at least one two-qubit gate")
    outputs: List[List[int]] = [[] for _ in tensor_gate]
    for q in range(n):
        outputs[last[q]].append(q)
    return NetworkStructure(
        n_qubits=n,
        n_tensors=len(tensor_gate),
        n_edges=len(ends),
        tensor_gate=np.asarray(tensor_gate, np.int64),
        tensor_qubits=np.asarray(tensor_qubits, np.int64).reshape(-1, 2),
        tensor_edges=tensor_edges,
        tensor_outputs=outputs,
        edge_ends=np.asarray(ends, np.int64).reshape(-1, 2),
        edge_wire=np.asarray(wires, np.int64).reshape(-1, 2),
    )
