"""Fidelity estimates from device amplitudes: the linear XEB with its
standard error, and the maximum-likelihood fit of the fidelity to the
Porter-Thomas mixture of Eq. (fxeb) with its error bar, plus a histogram of
x = 2^n |amp|^2 for comparing with that law.

With x_b = 2^n |amp_b|^2, bitstrings drawn at fidelity F have the density
p(x) = e^-x (1 + F (x - 1)).  The log-likelihood of F is concave; Newton's
method on it needs sum g and sum g^2 with g = (x - 1) / (1 + F (x - 1)), which
the library's k_pt_moments kernel reduces on the device in FP64 (one launch
per iteration); the scalar update runs here.  The error bar is the inverse
square root of the Fisher information sum g^2 at the maximum.
"""

import math

import numpy as np

from . import tn


def porter_thomas_fit(amps, k, n_qubits, stream=None, iters=60, tol=1e-13):
    """amps: device complex128 amplitudes (2k doubles, a torch CUDA tensor).
    Returns a dict: fidelity (maximum likelihood, kept in [0, 1 - 1e-12]),
    stderr, loglik (up to the constant), linear (N <p> - 1), linear_stderr,
    iterations."""
    import torch

    out = torch.empty(5, dtype=torch.float64, device=amps.device)

    def moments(f):
        tn.tn_pt_moments(amps, k, n_qubits, f, out, stream=stream)
        return out.cpu().numpy()  # synchronises with the launch

    top = 1.0 - 1e-12
    s = moments(0.0)
    mean = s[3] / k
    f = min(max(mean - 1.0, 0.0), top)  # start at the linear estimate
    it = 0
    for it in range(1, iters + 1):
        s = moments(f)
        nf = min(max(f + s[0] / s[1], 0.0), top)
        done = abs(nf - f) <= tol
        f = nf
        if done:
            break
    s = moments(f)
    var = max(s[4] / k - mean * mean, 0.0)
    return {"fidelity": float(f), "stderr": float(1.0 / math.sqrt(s[1])), "loglik": float(s[2] - s[3]),
            "linear": float(mean - 1.0), "linear_stderr": float(math.sqrt(var / k)), "iterations": it}


def porter_thomas_histogram(amps, k, n_qubits, x_max=8.0, nbins=64, stream=None):
    """Counts of x = 2^n |amp|^2 in nbins equal bins over [0, x_max), then
    the count at or above x_max (numpy int64, nbins + 1 entries)."""
    import torch

    counts = torch.zeros(nbins + 1, dtype=torch.int64, device=amps.device)
    tn.tn_pt_histogram(amps, k, n_qubits, x_max, nbins, counts, stream=stream)
    return counts.cpu().numpy()


def porter_thomas_expected(nbins, x_max, k, fidelity):
    """Expected counts of the histogram's bins under Eq. (fxeb) at `fidelity`
    (the last entry: x >= x_max), from the law's distribution function
    1 - (1 + F x) e^-x."""
    edges = np.linspace(0.0, x_max, nbins + 1)
    cdf = 1.0 - (1.0 + fidelity * edges) * np.exp(-edges)
    return k * np.append(np.diff(cdf), 1.0 - cdf[-1])
