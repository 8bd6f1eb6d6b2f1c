"""Linear XEB fidelity and the Porter-Thomas law (test only).

The paper gives the density of x = N p for bitstrings sampled at fidelity F,
P(x|F) = (F x + 1 - F) e^{-x} (Eq. fxeb), but not the estimator.  Its mean
is E[x] = 2F + (1 - F) = 1 + F, so the estimator consistent with that law
is the linear XEB  F = N <p> - 1 = (2^n / k) sum_b |amp_b|^2 - 1.
"""

import numpy as np


def linear_xeb(amps: np.ndarray, n_qubits: int) -> float:
    a = np.asarray(amps, np.complex128)
    p = a.real * a.real + a.imag * a.imag
    return float((2.0 ** n_qubits) * p.mean() - 1.0)


def porter_thomas_pdf(x, fidelity: float):
    """Eq. (fxeb): density of x = N p at XEB fidelity F."""
    x = np.asarray(x, np.float64)
    return (fidelity * x + 1.0 - fidelity) * np.exp(-x)


def porter_thomas_cdf(x, fidelity: float):
    """Integral of Eq. (fxeb) from 0 to x: 1 - (1 + F x) e^{-x}."""
    x = np.asarray(x, np.float64)
    return 1.0 - (1.0 + fidelity * x) * np.exp(-x)
