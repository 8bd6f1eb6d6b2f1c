"""Fidelity analysis on the GPU (linear XEB error bar, maximum-likelihood fit
to the Porter-Thomas mixture of Eq. (fxeb), histogram of x = N |amp|^2)
against the float64 oracle on the same amplitudes, and on amplitudes the
library contracted for bitstrings drawn from the exact distribution and
uniformly.

Tolerances: the device sums run in FP64 in another order than numpy's
(relative error ~1e-15 per sum), held to 1e-11; the fitted F follows the
sums, held to 1e-9; histogram bins are integer decisions taken by the same
correctly rounded FP64 operations on both sides, compared exactly.
"""

import numpy as np
import pytest

from gpu_helpers import require_cuda, run_plan
from oracle import sv
from oracle import xeb as oxeb

pytestmark = pytest.mark.gpu


def _amps(k, n, seed):
    # Porter-Thomas-like amplitudes: complex normal, |amp|^2 of mean 2^-n
    rng = np.random.default_rng(seed)
    return (rng.normal(size=k) + 1j * rng.normal(size=k)) * np.sqrt(0.5 / 2 ** n)


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, np.complex128).view(np.float64)).cuda()


@pytest.mark.parametrize("k", [1, 1000, 300001])
def test_moments_match_oracle(k):
    torch, tn = require_cuda()
    n = 24
    a = _amps(k, n, 1)
    d = _dev(torch, a)
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    for f in (0.0, 0.37, 0.99):
        tn.tn_pt_moments(d, k, n, f, out)
        got = out.cpu().numpy()
        ref = oxeb.pt_moments(oxeb.x_values(a, n), f)
        assert np.all(np.abs(got - ref) <= 1e-11 * np.maximum(np.abs(ref), 1.0)), (f, got, ref)


def test_fit_matches_oracle_and_histogram_is_exact():
    torch, tn = require_cuda()
    from paper_2212_04749_gb300 import xeb
    n, k = 30, 200000
    rng = np.random.default_rng(4)
    # a mixture at F = 0.4: ideal samples have |amp|^2 size-biased (x e^-x)
    x = np.where(rng.random(k) < 0.4, rng.gamma(2.0, 1.0, k), rng.exponential(1.0, k))
    a = np.sqrt(x / 2 ** n) * np.exp(2j * np.pi * rng.random(k))
    d = _dev(torch, a)
    got = xeb.porter_thomas_fit(d, k, n)
    ref = oxeb.pt_fit(oxeb.x_values(a, n), start=got["linear"])
    assert abs(got["fidelity"] - ref["fidelity"]) < 1e-9
    assert abs(got["stderr"] - ref["stderr"]) < 1e-9 * ref["stderr"]
    assert abs(got["linear"] - ref["linear"]) < 1e-12
    assert abs(got["fidelity"] - 0.4) < 4 * got["stderr"]
    for x_max, nbins in ((8.0, 64), (5.0, 7), (1e-3, 1), (40.0, 8192)):
        h = xeb.porter_thomas_histogram(d, k, n, x_max=x_max, nbins=nbins)
        assert np.array_equal(h, oxeb.pt_histogram(oxeb.x_values(a, n), x_max, nbins)), (x_max, nbins)
    e = xeb.porter_thomas_expected(64, 8.0, k, got["fidelity"])
    h = xeb.porter_thomas_histogram(d, k, n)
    assert np.all(np.abs(h - e) < 5 * np.sqrt(e) + 5)


def test_fit_on_contracted_amplitudes():
    # 20 qubits, 20 cycles: bitstrings drawn from the exact output
    # distribution (oracle state vector) give F = 1, uniform ones F = 0,
    # each within 4 standard errors, from amplitudes the library contracted
    torch, tn = require_cuda()
    from paper_2212_04749_gb300 import xeb
    from rqc import grid_layout, network_structure, random_circuit
    from rqc.bitstrings import bitstrings_from_indices
    from rqc.tree import candidate_trees
    c = random_circuit(grid_layout(4, 5), 20, seed=77)
    psi = sv.state(c)
    p = np.abs(psi) ** 2
    rng = np.random.default_rng(9)
    k = 3000
    for f_true, idx in ((1.0, rng.choice(p.size, size=k, p=p / p.sum())), (0.0, rng.integers(0, p.size, size=k))):
        bits = bitstrings_from_indices(idx, 20)
        ssa = candidate_trees(network_structure(c), k, seed=2, trials=1)[0]
        amps, _ = run_plan(c, bits, ssa, [], precision="fp32")
        d = _dev(torch, amps)
        r = xeb.porter_thomas_fit(d, k, 20)
        print(f"F_true {f_true}: fit {r['fidelity']:.4f} +- {r['stderr']:.4f}, "
              f"linear {r['linear']:.4f} +- {r['linear_stderr']:.4f}")
        assert abs(r["fidelity"] - f_true) < 4 * r["stderr"] + 1e-6
        assert abs(r["linear"] - f_true) < 4 * r["linear_stderr"]
