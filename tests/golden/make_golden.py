"""Write stored expected values computed by the CPU oracle only.

    python tests/golden/make_golden.py grid5x6_m14

writes ``tests/golden/<workload>_sv.txt``: one line per bitstring (input
order) with the real and imaginary parts of <b|U|0^n> from the complex128
state-vector oracle.  The header holds a SHA-256 of the generated circuit
and bitstrings, so a test can tell when the input generators have drifted
and the file must be regenerated.
"""

import hashlib
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


if __name__ == "__main__":
    for name in sys.argv[1:] or ["grid5x6_m14"]:
        print(write(name))
