"""The synthetic workloads, by name.

Seeds: circuit 1000+i, bitstrings 2000+i, tree search 3000+i for workload i.

* ``grid3x4_m8``   : 12 qubits, 3x4 grid, 8 cycles (ABCDCDAB), 34 fSim gates,
                     64 bitstrings, unsliced.
* ``grid5x6_m14``  : 30 qubits, 5x6 grid, 14 cycles, 171 fSim gates,
                     4096 bitstrings, 10 sliced bond edges (2^10 slices) chosen
                     with the largest per-instance intermediate capped at 2^28.
* ``grid6x7_m10``  : 42 qubits, 6x7 grid, 10 cycles (ABCDCDABAB), 178 fSim
                     gates, 1024 bitstrings, 14 sliced bond edges (2^14
                     slices).  At 16 cycles the seeded search's trees keep
                     per-slice intermediates of rank 39 after 14 slices
                     (~6e18 flops), beyond one GPU; 10 cycles gives rank 23.
* ``diamond53_m12``: 53 qubits, 54-site diamond with one dead site,
                     12 cycles, 258 fSim gates, 8192 bitstrings, sliced until
                     the largest per-instance intermediate has <= 2^32 entries.
"""

from dataclasses import dataclass
from typing import Optional

import numpy as np

from .bitstrings import uniform_bitstrings
from .circuit import Circuit, random_circuit
from .layouts import diamond_layout, grid_layout
from .network import NetworkStructure, network_structure
from .tree import ContractionTree, greedy_tree


@dataclass(frozen=True)
class WorkloadSpec:
    name: str
    index: int
    layout: str
    cycles: int
    k: int
    n_sliced: Optional[int]
    max_rank: Optional[int]
    trials: int = 16


WORKLOADS = {
    "grid3x4_m8": WorkloadSpec("grid3x4_m8", 1, "grid3x4", 8, 64, None, None),
    "grid5x6_m14": WorkloadSpec("grid5x6_m14", 2, "grid5x6", 14, 4096, 10, 28),
    "grid6x7_m10": WorkloadSpec("grid6x7_m10", 3, "grid6x7", 10, 1024, 14, None, trials=8),
    "diamond53_m12": WorkloadSpec("diamond53_m12", 4, "diamond53", 12, 8192, None, 32),
}


@dataclass
class Workload:
    spec: WorkloadSpec
    circuit: Circuit
    bits: np.ndarray
    struct: NetworkStructure
    tree: ContractionTree

    @property
    def name(self):
        return self.spec.name


def _layout(name):
    if name.startswith("grid"):
        r, c = name[4:].split("x")
        return grid_layout(int(r), int(c))
    if name == "diamond53":
        return diamond_layout()
    raise KeyError(name)


_CACHE = {}


def make_workload(name: str, k: Optional[int] = None, trials: Optional[int] = None) -> Workload:
    """Build (and memoise) a workload.  ``k`` and ``trials`` override the
    bitstring count and the number of greedy trials (smaller test cases)."""
    spec = WORKLOADS[name]
    key = (name, k, trials)
    if key in _CACHE:
        return _CACHE[key]
    kk = spec.k if k is None else k
    circ = random_circuit(_layout(spec.layout), spec.cycles, seed=1000 + spec.index)
    bits = uniform_bitstrings(circ.n_qubits, kk, seed=2000 + spec.index)
    struct = network_structure(circ)
    tree = greedy_tree(struct, kk, seed=3000 + spec.index,
                       trials=spec.trials if trials is None else trials,
                       n_sliced=spec.n_sliced, max_rank=spec.max_rank)
    w = Workload(spec, circ, bits, struct, tree)
    _CACHE[key] = w
    return w
