"""The synthetic workloads, by name.

Seeds: circuit 1000+i, bitstrings 2000+i, tree search 3000+i for workload i.

* ``grid3x4_m8``   : 12 qubits, 3x4 grid, 8 cycles (ABCDCDAB), 34 fSim gates,
                     64 bitstrings, unsliced.
* ``grid5x6_m14``  : 30 qubits, 5x6 grid, 14 cycles, 171 fSim gates,
                     4096 bitstrings, 10 sliced bond edges (2^10 slices) chosen
                     with the largest per-instance intermediate capped at 2^28.
* ``grid6x7_m10``  : 42 qubits, 6x7 grid, 10 cycles (ABCDCDABAB), 178 fSim
                     gates, 1024 bitstrings, 14 sliced bond edges (2^14
                     slices).  At 16 cycles the search's trees keep
                     per-slice intermediates of rank 35 or more after 14
                     slices, beyond one GPU; 10 cycles gives rank 23.
* ``diamond53_m12``: 53 qubits, 54-site diamond with one dead site,
                     12 cycles, 258 fSim gates, 8192 bitstrings, sliced until
                     the largest per-instance intermediate has <= 2^32 entries.
                     Its tree is the one stored in ``rqc/trees/``: the best
                     measured tree of the tree search
                     (``paper_2212_04749_gb300.treesearch``, its measured
                     climb over rotations), which needs no slicing (largest
                     intermediate 2^23); ``seeded_tree=True`` gives the
                     seeded random-greedy tree instead.
"""

from dataclasses import dataclass
from typing import Optional

import hashlib
import json
import os

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
    tree_file: Optional[str] = None  # stored tree (rqc/trees/), else the seeded search


WORKLOADS = {
    "grid3x4_m8": WorkloadSpec("grid3x4_m8", 1, "grid3x4", 8, 64, None, None),
    "grid5x6_m14": WorkloadSpec("grid5x6_m14", 2, "grid5x6", 14, 4096, 10, 28),
    "grid6x7_m10": WorkloadSpec("grid6x7_m10", 3, "grid6x7", 10, 1024, 14, None, trials=8),
    "diamond53_m12": WorkloadSpec("diamond53_m12", 4, "diamond53", 12, 8192, None, 32,
                                  tree_file="diamond53_m12.json"),
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
TREES = os.path.join(os.path.dirname(os.path.abspath(__file__)), "trees")


def circuit_digest(circ: Circuit) -> str:
    """Digest of a circuit's gate positions and names (what a tree of its
    network depends on)."""
    q0, q1, layer, _ = circ.to_arrays()
    h = hashlib.sha256()
    for a in (q0, q1, layer):
        h.update(np.ascontiguousarray(a).tobytes())
    h.update(",".join(g.kind for g in circ.gates).encode())
    return h.hexdigest()


def stored_tree(spec: WorkloadSpec, circ: Circuit) -> Optional[ContractionTree]:
    """The workload's stored tree, if it has one for exactly this circuit."""
    if not spec.tree_file:
        return None
    with open(os.path.join(TREES, spec.tree_file)) as f:
        rec = json.load(f)
    if rec["circuit_sha256"] != circuit_digest(circ):
        raise ValueError(f"{spec.tree_file} belongs to another circuit (the generators changed)")
    t = ContractionTree(ssa=np.asarray(rec["ssa"], np.int64))
    t.sliced = [int(e) for e in rec["sliced"]]
    return t


def make_workload(name: str, k: Optional[int] = None, trials: Optional[int] = None,
                  seeded_tree: bool = False) -> Workload:
    """Build (and memoise) a workload.  ``k`` and ``trials`` override the
    bitstring count and the number of greedy trials (smaller test cases; the
    seeded search then runs); ``seeded_tree`` ignores a stored tree."""
    spec = WORKLOADS[name]
    key = (name, k, trials, seeded_tree)
    if key in _CACHE:
        return _CACHE[key]
    kk = spec.k if k is None else k
    circ = random_circuit(_layout(spec.layout), spec.cycles, seed=1000 + spec.index)
    bits = uniform_bitstrings(circ.n_qubits, kk, seed=2000 + spec.index)
    struct = network_structure(circ)
    tree = None
    if not seeded_tree and k is None and trials is None:
        tree = stored_tree(spec, circ)
    if tree is None:
        tree = greedy_tree(struct, kk, seed=3000 + spec.index,
                           trials=spec.trials if trials is None else trials,
                           n_sliced=spec.n_sliced, max_rank=spec.max_rank)
    w = Workload(spec, circ, bits, struct, tree)
    _CACHE[key] = w
    return w
