"""Qubit layouts and the four two-qubit layer patterns A, B, C, D (SM Sec. I).

The paper's pattern figure did not survive, so the geometry below is a
documented choice that keeps the one rule the text states: every
nearest-neighbour pair receives exactly one two-qubit gate in each block of
four cycles that contains all of A, B, C and D, and each pattern is a
matching (no qubit appears twice in one layer).

* Rectangular r x c grid, site (i, j) -> qubit i*c + j.
  A: horizontal (i,j)-(i,j+1) with i+j even; B: horizontal with i+j odd;
  C: vertical (i,j)-(i+1,j) with i+j even;   D: vertical with i+j odd.
* 54-site diamond (Sycamore-like): sites (i, j), i in 0..8, j in 0..5.
  Couplers: vertical (i,j)-(i+1,j); diagonal (i,j)-(i+1,j+1) for even i and
  (i,j)-(i+1,j-1) for odd i.  Site (0,0) is dead, leaving 53 qubits and 86
  couplers.  A: vertical, i even; B: vertical, i odd; C: diagonal, i even;
  D: diagonal, i odd.

Cycle sequences follow the 8-periodic prefix ABCDCDAB ABCDCDAB ... so that
depth 8 is ABCDCDAB and depth 12 is ABCDCDABABCD, as in the paper.
"""

from dataclasses import dataclass
from typing import Dict, List, Tuple

_PERIOD = "ABCDCDAB"


def pattern_sequence(cycles: int) -> str:
    """Pattern letter of each cycle: the first ``cycles`` letters of the
    repeated ABCDCDAB sequence (depth 8 -> ABCDCDAB, 12 -> ABCDCDABABCD)."""
    return "".join(_PERIOD[t % len(_PERIOD)] for t in range(cycles))


@dataclass(frozen=True)
class Layout:
    name: str
    n_qubits: int
    patterns: Dict[str, Tuple[Tuple[int, int], ...]]  # letter -> couplers (a<b)

    @property
    def couplers(self) -> List[Tuple[int, int]]:
        out = []
        for p in "ABCD":
            out.extend(self.patterns[p])
        return sorted(out)


def grid_layout(rows: int, cols: int) -> Layout:
    def q(i, j):
        return i * cols + j

    pats = {p: [] for p in "ABCD"}
    for i in range(rows):
        for j in range(cols):
            if j + 1 < cols:
                pats["A" if (i + j) % 2 == 0 else "B"].append((q(i, j), q(i, j + 1)))
            if i + 1 < rows:
                pats["C" if (i + j) % 2 == 0 else "D"].append((q(i, j), q(i + 1, j)))
    return Layout(
        name=f"grid{rows}x{cols}",
        n_qubits=rows * cols,
        patterns={p: tuple(sorted(v)) for p, v in pats.items()},
    )


def diamond_layout() -> Layout:
    rows, cols = 9, 6
    dead = {(0, 0)}
    ids = {}
    for i in range(rows):
        for j in range(cols):
            if (i, j) not in dead:
                ids[(i, j)] = len(ids)

    pats = {p: [] for p in "ABCD"}

    def add(p, s, t):
        if s in ids and t in ids:
            a, b = ids[s], ids[t]
            pats[p].append((min(a, b), max(a, b)))

    for i in range(rows - 1):
        for j in range(cols):
            add("A" if i % 2 == 0 else "B", (i, j), (i + 1, j))
            if i % 2 == 0:
                if j + 1 < cols:
                    add("C", (i, j), (i + 1, j + 1))
            else:
                if j - 1 >= 0:
                    add("D", (i, j), (i + 1, j - 1))
    return Layout(
        name="diamond53",
        n_qubits=len(ids),
        patterns={p: tuple(sorted(v)) for p, v in pats.items()},
    )
