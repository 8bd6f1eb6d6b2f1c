"""Seeded synthetic inputs for multiple-amplitude tensor network contraction.

This package only *generates inputs*: random quantum circuits of the
Sycamore family (SM Sec. I), uniform bitstrings, the connectivity of the
fused tensor network those circuits define (SM Sec. II), and seeded
contraction trees / sliced-edge sets for that network.  It holds none of the
contraction arithmetic.  Both the CPU oracle (``oracle/``) and the CUDA
library (``paper_2212_04749_gb300``) consume what it produces; neither of
them is imported here.
"""

from .gates import SQRT_X, SQRT_Y, SQRT_W, fsim
from .layouts import Layout, grid_layout, diamond_layout, pattern_sequence
from .circuit import Circuit, Gate, random_circuit
from .bitstrings import uniform_bitstrings
from .network import NetworkStructure, network_structure
from .tree import ContractionTree, greedy_tree, choose_slices
from .configs import WORKLOADS, Workload, make_workload

__all__ = [
    "SQRT_X", "SQRT_Y", "SQRT_W", "fsim",
    "Layout", "grid_layout", "diamond_layout", "pattern_sequence",
    "Circuit", "Gate", "random_circuit",
    "uniform_bitstrings",
    "NetworkStructure", "network_structure",
    "ContractionTree", "greedy_tree", "choose_slices",
    "WORKLOADS", "Workload", "make_workload",
]
