"""Seeded bitstrings standing in for the experimental Sycamore samples.

The paper's workload is three million bitstrings measured on the device;
those are not available here.  Uniform random bitstrings reproduce the
reuse-tree widths the paper prints (its Table S2 values sit within about
1 % of the uniform-occupancy prediction 2^j (1 - (1 - 2^-j)^k)), so they
stand in for them.

Layout: uint8 array of shape (k, n), entry [b, q] in {0, 1} is the value of
qubit q (column q) in bitstring b.
"""

import numpy as np


def uniform_bitstrings(n_qubits: int, k: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2, size=(k, n_qubits), dtype=np.uint8)


def bitstrings_from_indices(indices, n_qubits: int) -> np.ndarray:
    """Bitstrings for computational-basis indices, with qubit 0 as the most
    significant bit of the index (index = sum_q b_q 2^(n-1-q))."""
    idx = np.asarray(indices, dtype=np.uint64)
    shifts = np.arange(n_qubits - 1, -1, -1, dtype=np.uint64)
    return ((idx[:, None] >> shifts[None, :]) & np.uint64(1)).astype(np.uint8)


def bitstring_indices(bits: np.ndarray) -> np.ndarray:
    """Inverse of :func:`bitstrings_from_indices`."""
    b = np.asarray(bits, dtype=np.uint64)
    n = b.shape[1]
    shifts = np.arange(n - 1, -1, -1, dtype=np.uint64)
    return (b << shifts[None, :]).sum(axis=1, dtype=np.uint64)
