"""Independent pairwise tensor-network contractor (test only).

Builds the *unfused* network of a circuit straight from its gate list
(SM Sec. II): a rank-1 |0> vector per qubit, a rank-2 tensor per
single-qubit gate, a rank-4 tensor per two-qubit gate and a rank-1 <b_q|
projection per output leg.  Labels are wire segments: a new segment starts
after every gate on a qubit.

First-level slicing (SM Sec. IV.B) fixes the value of a chosen wire: the
segment of qubit q right after the two-qubit gate with full-gate-list index
g.  The j-th sliced wire of a list takes the value (s >> j) & 1 in slice s;
a slice's partial amplitude is the contraction with those values fixed, and
the amplitude is the sum of the partials over all slices.

Contraction order.  Every unfused node is first assigned to a two-qubit
gate (|0> and single-qubit gates go to the next two-qubit gate on their
qubit; gates after the last two-qubit gate and the output projection go to
the last one) and each group is contracted to one tensor.  The groups are
then contracted pairwise following an SSA tree over two-qubit-gate ids
(the same tree format the library takes).  Each pairwise step is a plain
``numpy.tensordot`` in complex128.  Intermediate results are kept in a
dictionary keyed by (node, projection of the bitstring onto the node's
output qubits, values of the sliced wires inside the node): a dynamic cache
of the kind the paper contrasts its static reuse tree with (main text,
multiple-amplitude section), so that shared sub-networks are contracted
once.  The cache changes which contractions are repeated, never their
arithmetic.
"""

from typing import Dict, List, Sequence, Tuple

import numpy as np

_E = (np.array([1.0, 0.0], np.complex128), np.array([0.0, 1.0], np.complex128))


def _contract(a, b):
    """Pairwise contraction of labelled tensors over their shared labels."""
    ta, la = a
    tb, lb = b
    shared = [x for x in la if x in lb]
    ia = [la.index(x) for x in shared]
    ib = [lb.index(x) for x in shared]
    out = np.tensordot(ta, tb, axes=(ia, ib))
    labels = tuple(x for x in la if x not in shared) + tuple(x for x in lb if x not in shared)
    return out, labels


def _fix(node, label, value):
    t, l = node
    if label not in l:
        return node
    ax = l.index(label)
    return np.take(t, value, axis=ax), tuple(x for x in l if x != label)


class UnfusedNetwork:
    """Unfused network of a circuit with open output legs."""

    def __init__(self, circ):
        n = circ.n_qubits
        self.n = n
        counter = [0]

        def seg():
            counter[0] += 1
            return counter[0] - 1

        two_q = [gi for gi, g in enumerate(circ.gates) if len(g.qubits) == 2]
        self.tensor_of_gate = {gi: t for t, gi in enumerate(two_q)}
        per_qubit_2q = [[] for _ in range(n)]
        for gi in two_q:
            for q in circ.gates[gi].qubits:
                per_qubit_2q[q].append(gi)
        if any(len(x) == 0 for x in per_qubit_2q):
            raise ValueError("every qubit needs a two-qubit gate")

        def group_for(q, gi):
            nxt = [x for x in per_qubit_2q[q] if x > gi]
            return self.tensor_of_gate[nxt[0] if nxt else per_qubit_2q[q][-1]]

        self.nodes: List[Tuple[np.ndarray, tuple]] = []
        self.group: List[int] = []
        self.wire_after: Dict[Tuple[int, int], int] = {}
        cur = [seg() for _ in range(n)]
        for q in range(n):
            self.nodes.append((_E[0].copy(), (cur[q],)))
            self.group.append(group_for(q, -1))
        for gi, g in enumerate(circ.gates):
            m = np.asarray(g.matrix, np.complex128)
            if len(g.qubits) == 1:
                (q,) = g.qubits
                new = seg()
                self.nodes.append((m.copy(), (new, cur[q])))
                self.group.append(group_for(q, gi))
                cur[q] = new
            else:
                a, b = g.qubits
                na, nb = seg(), seg()
                self.nodes.append((m.reshape(2, 2, 2, 2).copy(), (na, nb, cur[a], cur[b])))
                self.group.append(self.tensor_of_gate[gi])
                self.wire_after[(a, gi)] = na
                self.wire_after[(b, gi)] = nb
                cur[a], cur[b] = na, nb
        self.out_label = list(cur)
        self.out_group = [per_qubit_2q[q][-1] for q in range(n)]
        self.out_group = [self.tensor_of_gate[x] for x in self.out_group]
        self.n_groups = len(two_q)

    def contract_all_open(self):
        """Plain contraction of the whole network with every output leg
        open (no projection), in gate order: returns the state vector with
        qubit 0 as the most significant index.  Small n only."""
        acc = None
        for node in self.nodes:
            acc = node if acc is None else _contract(acc, node)
        t, l = acc
        perm = [l.index(x) for x in self.out_label]
        return np.transpose(t, perm).reshape(-1)


def _group_tensor(net: UnfusedNetwork, t, bits_row, fixed: Dict[int, int]):
    acc = None
    for i, g in enumerate(net.group):
        if g != t:
            continue
        node = net.nodes[i]
        for lab, val in fixed.items():
            node = _fix(node, lab, val)
        acc = node if acc is None else _contract(acc, node)
    for q in range(net.n):
        if net.out_group[q] == t:
            acc = _contract(acc, (_E[int(bits_row[q])], (net.out_label[q],)))
    return acc


def partial_amplitudes(circ, ssa: np.ndarray, bits: np.ndarray,
                       sliced_wires: Sequence[Tuple[int, int]] = (),
                       slices: Sequence[int] = (0,)) -> np.ndarray:
    """Partial amplitudes, complex128 array (len(slices), k).

    ``sliced_wires[j] = (q, g)``: the wire of qubit q right after the
    two-qubit gate with full gate index g; slice s fixes it to (s >> j) & 1.
    With no sliced wires and ``slices=(0,)`` the result is the amplitude.
    """
    net = UnfusedNetwork(circ)
    T = net.n_groups
    ssa = np.asarray(ssa, np.int64).reshape(-1, 2)
    if ssa.shape[0] != T - 1:
        raise ValueError("tree size does not match the number of two-qubit gates")
    labels = [net.wire_after[(int(q), int(g))] for (q, g) in sliced_wires]

    # per node: output qubits and sliced wires inside the subtree
    outs: List[Tuple[int, ...]] = []
    touched: List[Tuple[int, ...]] = []
    for t in range(T):
        outs.append(tuple(q for q in range(net.n) if net.out_group[q] == t))
        labs = set()
        for i, g in enumerate(net.group):
            if g == t:
                labs.update(net.nodes[i][1])
        touched.append(tuple(j for j, lab in enumerate(labels) if lab in labs))
    children = []
    for a, b in ssa:
        a, b = int(a), int(b)
        children.append((a, b))
        outs.append(tuple(sorted(outs[a] + outs[b])))
        touched.append(tuple(sorted(set(touched[a]) | set(touched[b]))))
    root = 2 * T - 2

    bits = np.asarray(bits, np.uint8)
    k = bits.shape[0]
    result = np.zeros((len(slices), k), np.complex128)
    memo: Dict[Tuple[int, tuple, tuple], Tuple[np.ndarray, tuple]] = {}

    def value(v, brow, svals):
        key = (v, tuple(int(brow[q]) for q in outs[v]), tuple(svals[j] for j in touched[v]))
        hit = memo.get(key)
        if hit is not None:
            return hit
        if v < T:
            fixed = {labels[j]: svals[j] for j in touched[v]}
            res = _group_tensor(net, v, brow, fixed)
        else:
            a, b = children[v - T]
            res = _contract(value(a, brow, svals), value(b, brow, svals))
        memo[key] = res
        return res

    import sys
    old = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old, 4 * T + 100))
    try:
        for si, s in enumerate(slices):
            svals = tuple((int(s) >> j) & 1 for j in range(len(labels)))
            for b in range(k):
                t, l = value(root, bits[b], svals)
                assert l == ()
                result[si, b] = complex(t)
            # entries that depend on the slice are not reused by other slices
            for key in [key for key in memo if key[2]]:
                del memo[key]
    finally:
        sys.setrecursionlimit(old)
    return result
