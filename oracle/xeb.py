"""Linear XEB fidelity, the Porter-Thomas law and the maximum-likelihood fit
of the fidelity to it (test infrastructure only: imported by the tests and
the benchmark's CPU reference).

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


# Maximum-likelihood fit of F to Eq. (fxeb) ---------------------------------
#
# The log-likelihood of F for observed x_1..x_k under Eq. (fxeb) is
# l(F) = sum_b log(1 + F (x_b - 1)) - sum_b x_b; its derivative is
# sum_b g_b with g_b = (x_b - 1) / (1 + F (x_b - 1)), its second derivative
# -sum_b g_b^2 (< 0: l is concave, one maximum), and the Fisher information
# at the maximum, sum_b g_b^2, gives the standard error 1 / sqrt(.).


def x_values(amps: np.ndarray, n_qubits: int) -> np.ndarray:
    """x_b = 2^n |amp_b|^2, as re*re + im*im times 2^n (each operation rounded)."""
    a = np.asarray(amps, np.complex128)
    return (a.real * a.real + a.imag * a.imag) * (2.0 ** n_qubits)


def pt_moments(x: np.ndarray, fidelity: float) -> np.ndarray:
    """[sum g, sum g^2, sum log(1 + F (x - 1)), sum x, sum x^2]."""
    x = np.asarray(x, np.float64)
    d = 1.0 + fidelity * (x - 1.0)
    g = (x - 1.0) / d
    return np.array([g.sum(), (g * g).sum(), np.log(d).sum(), x.sum(), (x * x).sum()])


def pt_fit(x: np.ndarray, start: float = 0.0, iters: int = 100, tol: float = 1e-14) -> dict:
    """Newton's method on l(F), kept inside [0, 1 - 1e-12]; returns F, its
    standard error, the linear XEB and its standard error."""
    x = np.asarray(x, np.float64)
    k = x.size
    f = min(max(start, 0.0), 1.0 - 1e-12)
    it = 0
    for it in range(1, iters + 1):
        s = pt_moments(x, f)
        step = s[0] / s[1]
        nf = min(max(f + step, 0.0), 1.0 - 1e-12)
        done = abs(nf - f) <= tol
        f = nf
        if done:
            break
    s = pt_moments(x, f)
    mean = s[3] / k
    var = max(s[4] / k - mean * mean, 0.0)
    return {"fidelity": f, "stderr": 1.0 / np.sqrt(s[1]), "loglik": s[2] - s[3],
            "linear": mean - 1.0, "linear_stderr": np.sqrt(var / k), "iterations": it}


def pt_histogram(x: np.ndarray, x_max: float, nbins: int) -> np.ndarray:
    """Counts of floor(x / (x_max / nbins)) for bins 0..nbins-1, then x >= x_max."""
    q = np.floor(np.asarray(x, np.float64) / (x_max / nbins))
    j = np.where(q < nbins, q, nbins).astype(np.int64)
    return np.bincount(j, minlength=nbins + 1)
