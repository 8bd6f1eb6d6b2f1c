"""Write stored expected values computed by the CPU oracle only.

    python tests/golden/make_golden.py grid5x6_m14     # all amplitudes, state vector
    python tests/golden/make_golden.py diamond53_m12   # 320 sampled amplitudes, TN oracle
    python tests/golden/make_golden.py grid6x7_m10     # 32 slices x 16 bitstrings, TN oracle

``<workload>_sv.txt``: one line per bitstring (input order) with the real
and imaginary parts of <b|U|0^n> from the complex128 state-vector oracle.
``<workload>_sample.json`` / ``<workload>_slices.json``: amplitudes or
per-slice partial amplitudes from the complex128 tensor-network oracle, with
the inputs they belong to (bitstring rows, and for slices the contraction
tree, the sliced edges and the slice ids, stored so that a test uses exactly
these even if a tree search elsewhere breaks a tie differently).  Every
file holds a SHA-256 of the generated circuit and bitstrings, so a test can
tell when the input generators have drifted and the file must be
regenerated.
"""

import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import sv  # noqa: E402
from rqc.bitstrings import uniform_bitstrings  # noqa: E402
from rqc.circuit import random_circuit  # noqa: E402
from rqc.configs import WORKLOADS, _layout  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def workload_inputs(name):
    spec = WORKLOADS[name]
    circ = random_circuit(_layout(spec.layout), spec.cycles, seed=1000 + spec.index)
    bits = uniform_bitstrings(circ.n_qubits, spec.k, seed=2000 + spec.index)
    return circ, bits


def input_digest(circ, bits) -> str:
    """Digest of the discrete inputs (gate positions, gate names, bitstrings);
    the gate entries follow from the names, and leaving the floats out keeps
    the digest identical across host architectures."""
    q0, q1, layer, _ = circ.to_arrays()
    h = hashlib.sha256()
    for a in (q0, q1, layer, np.ascontiguousarray(bits, np.uint8)):
        h.update(np.ascontiguousarray(a).tobytes())
    h.update(",".join(g.kind for g in circ.gates).encode())
    return h.hexdigest()


def path_for(name):
    return os.path.join(HERE, f"{name}_sv.txt")


def write(name):
    circ, bits = workload_inputs(name)
    t = time.time()
    amps = sv.amplitudes(circ, bits)
    dt = time.time() - t
    with open(path_for(name), "w") as f:
        f.write(f"# workload {name}: amplitudes <b|U|0^n> from oracle/sv.c (complex128)\n")
        f.write(f"# n_qubits {circ.n_qubits} k {bits.shape[0]} gates {len(circ.gates)}\n")
        f.write(f"# inputs_sha256 {input_digest(circ, bits)}\n")
        f.write(f"# oracle wall time {dt:.1f} s\n")
        for a in amps:
            f.write(f"{a.real:.17e} {a.imag:.17e}\n")
    return path_for(name)


def read(name):
    digest = None
    rows = []
    with open(path_for(name)) as f:
        for line in f:
            if line.startswith("# inputs_sha256"):
                digest = line.split()[2]
            elif not line.startswith("#"):
                re, im = line.split()
                rows.append(complex(float(re), float(im)))
    return digest, np.asarray(rows, np.complex128)


def sample_path(name):
    return os.path.join(HERE, f"{name}_sample.json")


def slices_path(name):
    return os.path.join(HERE, f"{name}_slices.json")


def _rows(k, n, seed):
    rng = np.random.default_rng(seed)
    return sorted(int(x) for x in rng.choice(k, size=n, replace=False))


def write_sample(name, n=320):
    """Amplitudes of n seeded bitstring rows from the unsliced TN oracle."""
    from oracle import tn
    from rqc.configs import make_workload
    w = make_workload(name)
    rows = _rows(w.bits.shape[0], n, seed=5000 + w.spec.index)
    t = time.time()
    amps = tn.partial_amplitudes(w.circuit, w.tree.ssa, w.bits[rows])[0]
    rec = {"workload": name, "inputs_sha256": input_digest(w.circuit, w.bits), "rows": rows,
           "amplitudes": [[a.real, a.imag] for a in amps], "oracle": "oracle/tn.py (complex128)",
           "oracle_wall_s": time.time() - t}
    with open(sample_path(name), "w") as f:
        json.dump(rec, f)
    return sample_path(name)


def write_slices(name, n_slices=32, n_rows=16):
    """Per-slice partial amplitudes of seeded slices x bitstring rows."""
    from oracle import tn
    from rqc.configs import make_workload
    w = make_workload(name)
    rows = _rows(w.bits.shape[0], n_rows, seed=5000 + w.spec.index)
    rng = np.random.default_rng(6000 + w.spec.index)
    n_sl = len(w.tree.sliced)
    slice_ids = sorted(int(x) for x in rng.choice(1 << n_sl, size=n_slices, replace=False))
    wires = [tuple(int(x) for x in w.struct.edge_wire[e]) for e in w.tree.sliced]
    t = time.time()
    parts = tn.partial_amplitudes(w.circuit, w.tree.ssa, w.bits[rows], wires, slice_ids)
    rec = {"workload": name, "inputs_sha256": input_digest(w.circuit, w.bits), "rows": rows,
           "tree_ssa": np.asarray(w.tree.ssa).tolist(), "sliced_edges": [int(e) for e in w.tree.sliced],
           "slice_ids": slice_ids, "partials": [[[p.real, p.imag] for p in r] for r in parts],
           "oracle": "oracle/tn.py (complex128)", "oracle_wall_s": time.time() - t}
    with open(slices_path(name), "w") as f:
        json.dump(rec, f)
    return slices_path(name)


def read_json(path):
    with open(path) as f:
        rec = json.load(f)
    for key in ("amplitudes", "partials"):
        if key in rec:
            a = np.asarray(rec[key], np.float64)
            rec[key] = a[..., 0] + 1j * a[..., 1]
    return rec


if __name__ == "__main__":
    for name in sys.argv[1:] or ["grid5x6_m14"]:
        if name == "diamond53_m12":
            print(write_sample(name))
        elif name == "grid6x7_m10":
            print(write_slices(name))
        else:
            print(write(name))
