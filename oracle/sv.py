"""ctypes front end of the oracle's C state-vector simulator (test only).

amp_b = <b| U |0^n>, U the ordered product of the circuit's gates
(SM Sec. II).  Qubit q is bit (n-1-q) of the basis index.
"""

import ctypes
import os

import numpy as np

from .build import build

_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        for fn in (_lib.oracle_sv_state, _lib.oracle_sv_amplitudes):
            fn.restype = ctypes.c_int
    return _lib


def _arrays(circ):
    q0, q1, _, m = circ.to_arrays()
    return (np.ascontiguousarray(q0, np.int32), np.ascontiguousarray(q1, np.int32),
            np.ascontiguousarray(m, np.float64))


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def state(circ) -> np.ndarray:
    """Full final state, complex128 of length 2^n."""
    lib = _load()
    q0, q1, m = _arrays(circ)
    n = circ.n_qubits
    psi = np.empty(2 * (1 << n), np.float64)
    rc = lib.oracle_sv_state(ctypes.c_int(n), ctypes.c_int(len(q0)), _ptr(q0), _ptr(q1),
                             _ptr(m), _ptr(psi))
    if rc != 0:
        raise RuntimeError(f"oracle_sv_state failed: {rc}")
    return psi.view(np.complex128)


def amplitudes(circ, bits: np.ndarray) -> np.ndarray:
    """Amplitudes of the rows of ``bits`` (k x n uint8), complex128 (k,)."""
    lib = _load()
    q0, q1, m = _arrays(circ)
    bits = np.ascontiguousarray(bits, np.uint8)
    k = bits.shape[0]
    out = np.empty(2 * k, np.float64)
    rc = lib.oracle_sv_amplitudes(ctypes.c_int(circ.n_qubits), ctypes.c_int(len(q0)), _ptr(q0),
                                  _ptr(q1), _ptr(m), _ptr(bits), ctypes.c_int64(k), _ptr(out))
    if rc != 0:
        raise RuntimeError(f"oracle_sv_amplitudes failed: {rc}")
    return out.view(np.complex128)


def completion_bits(bits: np.ndarray, open_qubits) -> np.ndarray:
    """Correlated batches (SM Sec. II: some output indices left open): every
    row of ``bits`` (k x n) expanded into its 2^r completions, r open qubits
    q_0 < ... < q_{r-1}: row p * 2^r + x is row p with qubit q_i set to bit
    r - 1 - i of x (k 2^r x n uint8)."""
    bits = np.ascontiguousarray(bits, np.uint8)
    oq = sorted(int(q) for q in open_qubits)
    r = len(oq)
    out = np.repeat(bits, 1 << r, axis=0)
    x = np.tile(np.arange(1 << r), bits.shape[0])
    for i, q in enumerate(oq):
        out[:, q] = (x >> (r - 1 - i)) & 1
    return out


def correlated_amplitudes(circ, bits: np.ndarray, open_qubits) -> np.ndarray:
    """Amplitudes of every completion of every row, complex128 (k 2^r,),
    in completion_bits order."""
    return amplitudes(circ, completion_bits(bits, open_qubits))


def threads() -> int:
    """Threads OpenMP will use (OMP_NUM_THREADS, else all host cores)."""
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v else (os.cpu_count() or 1)
