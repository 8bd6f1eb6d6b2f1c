"""Seeded contraction-tree search and sliced-edge selection.

The paper searches contraction orders with KaHyPar using the
multiple-amplitude cost of Eq. (1) as the loss (main text; SM Sec. IV.A).
KaHyPar is not available here, so trees come from a seeded random-greedy
search whose merge score is the *multiple-amplitude* size of the merged
tensor: a node holding output legs of j qubits is stored once per distinct
projection of the bitstrings onto those j qubits, whose expected count for
k uniform bitstrings is 2^j (1 - (1 - 2^-j)^k).  That makes the greedy push
the bright tensors (the ones carrying output legs) towards the end of the
order, where the reuse tree branches.

Sliced edges are chosen greedily afterwards (first-level slicing, SM
Sec. IV.B): each pick is a bond edge of a largest intermediate that keeps
the estimated total cost lowest.

These are input generators: the costs here are estimates used to rank
candidate orders, nothing more.

Tree format: an SSA pair list ``ssa`` of shape (T-1, 2); leaves are
0..T-1 (tensor ids of :mod:`rqc.network`), pair i creates node T+i, and the
root is node 2T-2.
"""

import heapq
import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from .network import NetworkStructure


def expected_width(j: int, k: int) -> float:
    """Expected number of distinct projections of k uniform bitstrings onto
    j qubits: 2^j (1 - (1 - 2^-j)^k)."""
    if j == 0:
        return 1.0
    p = 2.0 ** (-j)
    return (2.0 ** j) * (-math.expm1(k * math.log1p(-p)))


def _popcount(x: int) -> int:
    return x.bit_count()


@dataclass
class TreeCost:
    flops: float                 # estimated multiple-amplitude flops (8 per complex MAC)
    flops_single: float          # single-amplitude flops of one slice, times the slice count
    max_rank: int                # largest per-instance intermediate rank
    peak_bytes: float            # largest single node's bytes (all instances, complex64)
    node_rank: List[int] = field(default_factory=list)
    node_width: List[float] = field(default_factory=list)


@dataclass
class ContractionTree:
    ssa: np.ndarray              # (T-1, 2) int32
    sliced: List[int] = field(default_factory=list)

    @property
    def n_leaves(self) -> int:
        return self.ssa.shape[0] + 1


def node_masks(struct: NetworkStructure, ssa):
    """Per node: open bond-edge mask, output-qubit mask, touched-edge mask."""
    T = struct.n_tensors
    I = [struct.edge_mask(t) for t in range(T)]
    O = [struct.out_mask(t) for t in range(T)]
    X = list(I)
    for a, b in np.asarray(ssa):
        a, b = int(a), int(b)
        I.append(I[a] ^ I[b])
        O.append(O[a] | O[b])
        X.append(X[a] | X[b])
    return I, O, X


def estimate_cost(struct: NetworkStructure, ssa, k: int, sliced: Optional[List[int]] = None) -> TreeCost:
    S = 0
    for e in sliced or []:
        S |= 1 << e
    n_sl = _popcount(S)
    I, O, X = node_masks(struct, ssa)
    T = struct.n_tensors
    flops = 0.0
    flops_single = 0.0
    max_rank = 0
    peak = 0.0
    ranks, widths = [], []
    for v in range(len(I)):
        rank = _popcount(I[v] & ~S)
        w = (2.0 ** _popcount(X[v] & S)) * expected_width(_popcount(O[v]), k)
        ranks.append(rank)
        widths.append(w)
        max_rank = max(max_rank, rank)
        peak = max(peak, w * (2.0 ** rank) * 8.0)
        if v >= T:
            a, b = (int(x) for x in ssa[v - T])
            macs = 2.0 ** _popcount((I[a] | I[b]) & ~S)
            flops += 8.0 * w * macs
            flops_single += 8.0 * macs * (2.0 ** n_sl)
    return TreeCost(flops, flops_single, max_rank, peak, ranks, widths)


def _greedy_once(struct: NetworkStructure, k: int, rng, temperature: float) -> np.ndarray:
    T = struct.n_tensors
    I = {t: struct.edge_mask(t) for t in range(T)}
    O = {t: struct.out_mask(t) for t in range(T)}
    owners = {e: [int(a), int(b)] for e, (a, b) in enumerate(struct.edge_ends)}

    def lsize(t_I, t_O):
        return math.log2(expected_width(_popcount(t_O), k)) + _popcount(t_I)

    ls = {t: lsize(I[t], O[t]) for t in range(T)}
    heap = []
    pushed = set()
    counter = 0

    def push(a, b):
        nonlocal counter
        key = (min(a, b), max(a, b))
        if key in pushed:
            return
        pushed.add(key)
        new_ls = lsize(I[a] ^ I[b], O[a] | O[b])
        score = new_ls - math.log2(2.0 ** ls[a] + 2.0 ** ls[b])
        if temperature > 0:
            score += temperature * float(-math.log(-math.log(rng.random() + 1e-300) + 1e-300))
        heapq.heappush(heap, (score, counter, key[0], key[1]))
        counter += 1

    for e, (a, b) in owners.items():
        push(a, b)

    alive = set(range(T))
    ssa = []
    nxt = T
    while len(alive) > 1:
        pair = None
        while heap:
            _, _, a, b = heapq.heappop(heap)
            if a in alive and b in alive:
                pair = (a, b)
                break
        if pair is None:  # disconnected remainder: join the two smallest
            srt = sorted(alive, key=lambda t: ls[t])
            pair = (srt[0], srt[1])
        a, b = pair
        v = nxt
        nxt += 1
        I[v] = I[a] ^ I[b]
        O[v] = O[a] | O[b]
        ls[v] = lsize(I[v], O[v])
        alive.discard(a)
        alive.discard(b)
        alive.add(v)
        ssa.append((a, b))
        m = I[v]
        while m:
            low = m & -m
            e = low.bit_length() - 1
            m ^= low
            own = owners[e]
            own[:] = [v if x in (a, b) else x for x in own]
            other = own[0] if own[1] == v else own[1]
            if other != v:
                push(v, other)
    return np.asarray(ssa, dtype=np.int32).reshape(-1, 2)


def _sweep_once(struct: NetworkStructure, k: int, rng, temperature: float, start: int) -> np.ndarray:
    """One random-greedy *sweep*: a single intermediate grows from tensor
    ``start`` by absorbing, at each step, the neighbouring tensor that gives
    the smallest multiple-amplitude size (Gumbel-perturbed when
    ``temperature`` > 0).  The result is a linear order, the form the paper
    states its contraction orders in (a sequence T1 T2 T3 ... of tensors
    absorbed one after the other)."""
    T = struct.n_tensors
    I = [struct.edge_mask(t) for t in range(T)]
    O = [struct.out_mask(t) for t in range(T)]
    nbr = [set() for _ in range(T)]
    for a, b in struct.edge_ends:
        nbr[int(a)].add(int(b))
        nbr[int(b)].add(int(a))

    def lsize(tI, tO):
        return math.log2(expected_width(_popcount(tO), k)) + _popcount(tI)

    bI, bO = I[start], O[start]
    cur, nxt = start, T
    done = {start}
    front = set(nbr[start])
    ssa = []
    while len(done) < T:
        if not front:  # disconnected remainder
            front = set(range(T)) - done
        best = None
        for t in sorted(front):
            s = lsize(bI ^ I[t], bO | O[t])
            if temperature > 0:
                s -= temperature * float(-math.log(-math.log(rng.random() + 1e-300) + 1e-300))
            if best is None or s < best[0]:
                best = (s, t)
        t = best[1]
        ssa.append((cur, t))
        cur, nxt = nxt, nxt + 1
        bI ^= I[t]
        bO |= O[t]
        done.add(t)
        front |= nbr[t]
        front -= done
    return np.asarray(ssa, dtype=np.int32).reshape(-1, 2)


def candidate_trees(struct: NetworkStructure, k: int, seed: int, trials: int = 16,
                    temperature: float = 0.5) -> List[np.ndarray]:
    """``trials`` random-greedy sweeps plus ``trials`` random-greedy pairwise
    orders (trial 0 of each is deterministic), sorted by the estimated
    multiple-amplitude flops, best first."""
    out = []
    T = struct.n_tensors
    for trial in range(trials):
        rng = np.random.default_rng([seed, trial])
        start = int(rng.integers(0, T))
        temp = temperature if trial > 0 else 0.0
        for ssa in (_sweep_once(struct, k, rng, temp, start),
                    _greedy_once(struct, k, rng, temp)):
            c = estimate_cost(struct, ssa, k)
            out.append(((c.flops, c.max_rank), len(out), ssa))
    out.sort(key=lambda x: (x[0], x[1]))
    return [x[2] for x in out]


def greedy_tree(struct: NetworkStructure, k: int, seed: int, trials: int = 16,
                temperature: float = 0.5, n_sliced: Optional[int] = None,
                max_rank: Optional[int] = None, keep: int = 4) -> ContractionTree:
    """Seeded tree + sliced edges: the ``keep`` best candidate trees are each
    sliced with :func:`choose_slices`; the winner is the one that meets the
    rank cap (if any) with the lowest estimated flops after slicing."""
    cands = candidate_trees(struct, k, seed, trials, temperature)
    if n_sliced is None and max_rank is None:
        return ContractionTree(ssa=cands[0])
    best, best_key = None, None
    for ssa in cands[:keep]:
        tr = ContractionTree(ssa=ssa)
        tr.sliced = choose_slices(struct, tr, k, n_sliced, max_rank)
        c = estimate_cost(struct, ssa, k, tr.sliced)
        key = (max_rank is not None and c.max_rank > max_rank, c.flops)
        if best is None or key < best_key:
            best, best_key = tr, key
    return best


def choose_slices(struct: NetworkStructure, tree: ContractionTree, k: int,
                  n_sliced: Optional[int] = None, max_rank: Optional[int] = None) -> List[int]:
    """Greedy first-level slicing.  While the largest per-instance
    intermediate has rank > ``max_rank``, pick among the bond edges of the
    largest intermediates; once under the cap (or with no cap), pick among
    all bond edges, keeping the cap.  Each pick minimises the estimated total
    flops.  Stops after ``n_sliced`` edges when that is given (the cap then
    only steers the picks), else as soon as the cap holds."""
    if n_sliced is None and max_rank is None:
        return []
    I, _, _ = node_masks(struct, tree.ssa)
    all_edges = (1 << struct.n_edges) - 1
    sliced: List[int] = []
    S = 0
    while True:
        cur = estimate_cost(struct, tree.ssa, k, sliced)
        top = max(cur.node_rank)
        capped = max_rank is None or top <= max_rank
        if (n_sliced is not None and len(sliced) >= n_sliced) or (n_sliced is None and capped):
            break
        if not capped or max_rank is None:
            cand = 0
            for v, r in enumerate(cur.node_rank):
                if r == top:
                    cand |= I[v] & ~S
        else:
            cand = all_edges & ~S
        limit = top if max_rank is None else max(max_rank, top)
        best_e, best_f = None, None
        m = cand
        while m:
            low = m & -m
            e = low.bit_length() - 1
            m ^= low
            c = estimate_cost(struct, tree.ssa, k, sliced + [e])
            if c.max_rank > limit:
                continue
            if best_f is None or c.flops < best_f:
                best_e, best_f = e, c.flops
        if best_e is None:
            break
        sliced.append(best_e)
        S |= 1 << best_e
    return sorted(sliced)


def refine_slices(struct: NetworkStructure, tree: ContractionTree, k: int, sliced: List[int],
                  max_rank: Optional[int] = None, rounds: int = 2, max_evals: int = 4000) -> List[int]:
    """Local search over the sliced-edge set: replace one sliced edge by an
    unsliced bond edge whenever that lowers the estimated multiple-amplitude
    cost summed over all slices (Eq. (1)) and keeps the largest per-instance
    rank within ``max_rank`` (or within the current largest rank).  Every
    unsliced edge is a candidate; first improvement, at most ``max_evals``
    cost evaluations."""
    cur = sorted(sliced)
    best = estimate_cost(struct, tree.ssa, k, cur)
    cap = best.max_rank if max_rank is None else max(max_rank, best.max_rank)
    evals = 0
    for _ in range(rounds):
        improved = False
        for i in range(len(cur)):
            for e in range(struct.n_edges):
                if e in cur:
                    continue
                if evals >= max_evals:
                    return cur
                trial = sorted(cur[:i] + [e] + cur[i + 1:])
                c = estimate_cost(struct, tree.ssa, k, trial)
                evals += 1
                if c.max_rank <= cap and c.flops < best.flops * (1.0 - 1e-9):
                    best, cur = c, trial
                    improved = True
        if not improved:
            break
    return cur
