"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the property it checks.  None of them re-derives the
oracle's own formula: brute force uses per-gate full matrices, the
projector pin inserts |s><s| into a state-vector run, the closed forms are
written independently, and the planted-mistake tests show that a plausible
slip in the oracle (a transposed gate, the wrong bit order, a wire sliced
on the wrong side of a gate) fails a pin.
"""

import numpy as np
import pytest

from oracle import brute, mlp, sv, tn, xeb
from rqc import grid_layout, make_workload, network_structure, random_circuit
from rqc.bitstrings import bitstrings_from_indices, uniform_bitstrings
from rqc.circuit import Circuit, Gate, inverse_circuit, product_circuit
from rqc.tree import ContractionTree, candidate_trees, choose_slices


def _all_bits(n):
    return bitstrings_from_indices(np.arange(1 << n, dtype=np.uint64), n)


SMALL = [(grid_layout(2, 3), 8, 5), (grid_layout(3, 3), 6, 11), (grid_layout(2, 5), 10, 2)]


# P1: brute force ------------------------------------------------------------
@pytest.mark.parametrize("layout,cycles,seed", SMALL)
def test_sv_matches_brute_force_unitary(layout, cycles, seed):
    c = random_circuit(layout, cycles, seed)
    a = brute.amplitudes(c)
    assert np.max(np.abs(sv.state(c) - a)) < 1e-13
    u = brute.unitary(c)
    assert np.allclose(u.conj().T @ u, np.eye(u.shape[0]), atol=1e-12)


@pytest.mark.parametrize("layout,cycles,seed", SMALL)
def test_tn_matches_brute_force(layout, cycles, seed):
    c = random_circuit(layout, cycles, seed)
    n = c.n_qubits
    s = network_structure(c)
    ssa = candidate_trees(s, 1 << n, seed=seed, trials=2)[0]
    amps = tn.partial_amplitudes(c, ssa, _all_bits(n))[0]
    assert np.max(np.abs(amps - brute.amplitudes(c))) < 1e-13
    # a second, unrelated order gives the same numbers (c10)
    ssa2 = candidate_trees(s, 1, seed=seed + 100, trials=3)[-1]
    amps2 = tn.partial_amplitudes(c, ssa2, _all_bits(n))[0]
    assert np.max(np.abs(amps2 - amps)) < 1e-13


def test_tn_open_network_is_the_state():
    c = random_circuit(grid_layout(2, 3), 6, 3)
    net = tn.UnfusedNetwork(c)
    assert np.max(np.abs(net.contract_all_open() - brute.amplitudes(c))) < 1e-13


# P2: norm -------------------------------------------------------------------
@pytest.mark.parametrize("rows,cols,cycles", [(3, 4, 8), (4, 5, 12)])
def test_norm_is_one(rows, cols, cycles):
    psi = sv.state(random_circuit(grid_layout(rows, cols), cycles, seed=rows * cols))
    assert abs(np.vdot(psi, psi).real - 1.0) < 1e-12


# P3: circuit followed by its inverse ---------------------------------------
def test_circuit_then_inverse_returns_to_zero_state():
    c = inverse_circuit(random_circuit(grid_layout(3, 4), 8, seed=1001))
    zero = np.zeros((1, 12), np.uint8)
    assert abs(sv.amplitudes(c, zero)[0] - 1.0) < 1e-12
    s = network_structure(c)
    ssa = candidate_trees(s, 1, seed=4, trials=2)[0]
    assert abs(tn.partial_amplitudes(c, ssa, zero)[0, 0] - 1.0) < 1e-12


# P4: product state closed form ---------------------------------------------
def test_product_circuit_closed_form():
    c = product_circuit(6, 4, seed=9)
    mats = {q: np.eye(2, dtype=complex) for q in range(6)}
    for g in c.gates:
        (q,) = g.qubits
        mats[q] = g.matrix @ mats[q]
    bits = uniform_bitstrings(6, 20, seed=1)
    expect = np.array([np.prod([mats[q][b[q], 0] for q in range(6)]) for b in bits])
    assert np.max(np.abs(sv.amplitudes(c, bits) - expect)) < 1e-14


# P5/P6: Porter-Thomas and XEB (Eq. fxeb) -----------------------------------
def _deep_state():
    return sv.state(random_circuit(grid_layout(4, 5), 20, seed=77))


def test_porter_thomas_at_zero_fidelity():
    psi = _deep_state()
    n = 20
    x = np.sort((2 ** n) * np.abs(psi) ** 2)
    emp = np.arange(1, x.size + 1) / x.size
    d = np.max(np.abs(emp - xeb.porter_thomas_cdf(x, 0.0)))
    assert d < 5e-3, d
    # a shallow circuit is far from the law: the test discriminates
    shallow = sv.state(random_circuit(grid_layout(4, 5), 2, seed=77))
    xs = np.sort((2 ** n) * np.abs(shallow) ** 2)
    ds = np.max(np.abs(emp - xeb.porter_thomas_cdf(xs, 0.0)))
    assert ds > 0.05


def test_porter_thomas_cdf_at_fidelity_one_and_a_mixture():
    # Eq. (fxeb) at F = 1 is the law of x for bitstrings drawn from the exact
    # output distribution (size-biased Porter-Thomas, x e^-x); at F = 0.3 it
    # is the 0.3 / 0.7 mixture of exact and uniform draws.  The CDF must
    # match both empirical laws, vanish at 0, and differentiate to the pdf.
    psi = _deep_state()
    n, k = 20, 40000
    p = np.abs(psi) ** 2
    rng = np.random.default_rng(11)
    exact = rng.choice(p.size, size=k, p=p / p.sum())
    uni = rng.integers(0, p.size, size=k)
    emp = np.arange(1, k + 1) / k
    for f, idx in ((1.0, exact), (0.3, np.where(rng.random(k) < 0.3, exact, uni))):
        x = np.sort((2 ** n) * p[idx])
        d = np.max(np.abs(emp - xeb.porter_thomas_cdf(x, f)))
        assert d < 1.63 / np.sqrt(k) + 5e-3, (f, d)  # KS 1 % level plus the finite-n law's deviation
        # the wrong fidelity is rejected by the same statistic
        assert np.max(np.abs(emp - xeb.porter_thomas_cdf(x, 0.0 if f > 0.5 else 1.0))) > 0.05
    assert xeb.porter_thomas_cdf(0.0, 0.7) == 0.0
    xs = np.linspace(0.05, 8.0, 50)
    h = 1e-6
    for f in (0.0, 0.4, 1.0):
        dcdf = (xeb.porter_thomas_cdf(xs + h, f) - xeb.porter_thomas_cdf(xs - h, f)) / (2 * h)
        assert np.max(np.abs(dcdf - xeb.porter_thomas_pdf(xs, f))) < 1e-8


def test_xeb_of_exact_samples_and_of_uniform_bitstrings():
    psi = _deep_state()
    n, k = 20, 20000
    p = np.abs(psi) ** 2
    rng = np.random.default_rng(5)
    idx = rng.choice(p.size, size=k, p=p / p.sum())
    f_exact = xeb.linear_xeb(psi[idx], n)
    assert abs(f_exact - 1.0) < 4 * np.sqrt(2.0 / k), f_exact
    uni = rng.integers(0, p.size, size=k)
    f_uni = xeb.linear_xeb(psi[uni], n)
    assert abs(f_uni) < 4 * np.sqrt(1.0 / k), f_uni
    # samples at fidelity F follow Eq. (fxeb): their mean x is 1 + F
    mix = np.where(rng.random(k) < 0.3, idx, uni)
    assert abs(xeb.linear_xeb(psi[mix], n) - 0.3) < 4 * np.sqrt(2.0 / k)


def test_fidelity_fit_two_point_closed_form():
    # for x = {a, b} the score (a-1)/(1+F(a-1)) + (b-1)/(1+F(b-1)) vanishes
    # at F = -(a + b - 2) / (2 (a - 1)(b - 1)); a = 0.5, b = 3 gives 3/4,
    # where each term of the Fisher information is 0.64
    r = xeb.pt_fit(np.array([0.5, 3.0]))
    assert abs(r["fidelity"] - 0.75) < 1e-12
    assert abs(r["stderr"] - 1.0 / np.sqrt(1.28)) < 1e-12
    assert abs(r["linear"] - 0.75) < 1e-15  # mean(x) - 1
    # other pairs against the same closed form
    for a, b in ((0.2, 2.5), (0.9, 1.7), (0.05, 6.0)):
        want = -(a + b - 2) / (2 * (a - 1) * (b - 1))
        if 0.0 < want < 1.0:
            assert abs(xeb.pt_fit(np.array([a, b]))["fidelity"] - want) < 1e-10


def test_fidelity_fit_recovers_the_mixture_fidelity():
    # x drawn from Eq. (fxeb): with probability F from x e^-x (Gamma(2)),
    # else from e^-x; the fit lands within 4 of its standard errors, and the
    # error bar matches the spread of the linear estimator's theory
    rng = np.random.default_rng(11)
    k = 200000
    for f in (0.0, 0.05, 0.3, 0.8):
        ideal = rng.random(k) < f
        x = np.where(ideal, rng.gamma(2.0, 1.0, k), rng.exponential(1.0, k))
        r = xeb.pt_fit(x, start=0.5)
        assert abs(r["fidelity"] - f) < 4 * r["stderr"] + 1e-9, (f, r)
        assert abs(r["linear"] - f) < 4 * r["linear_stderr"], (f, r)
        assert 0.5 / np.sqrt(k) < r["stderr"] < 2.0 / np.sqrt(k)
        # the likelihood is largest at the fit
        best = r["loglik"]
        for g in (max(r["fidelity"] - 0.01, 0.0), min(r["fidelity"] + 0.01, 0.99)):
            m = xeb.pt_moments(x, g)
            assert m[2] - m[3] <= best + 1e-6


def test_histogram_bins_and_counts():
    x = np.array([0.0, 0.49, 0.5, 0.99, 1.0, 7.99, 8.0, 100.0])
    h = xeb.pt_histogram(x, 8.0, 16)  # width 0.5
    assert h.sum() == x.size and h[0] == 2 and h[1] == 2 and h[2] == 1 and h[15] == 1 and h[16] == 2
    rng = np.random.default_rng(3)
    k = 100000
    y = rng.exponential(1.0, k)
    counts = xeb.pt_histogram(y, 6.0, 24)
    edges = np.linspace(0, 6.0, 25)
    expect = k * np.append(np.diff(1 - np.exp(-edges)), np.exp(-6.0))
    assert np.all(np.abs(counts - expect) < 5 * np.sqrt(expect) + 5)


def test_porter_thomas_pdf_normalised_and_mean():
    x = np.linspace(0, 60, 600001)
    for f in (0.0, 0.002, 0.5, 1.0):
        pdf = xeb.porter_thomas_pdf(x, f)
        assert abs(np.trapezoid(pdf, x) - 1) < 1e-6
        assert abs(np.trapezoid(x * pdf, x) - (1 + f)) < 1e-6


# Slicing: projector pin and slicing invariance (P7) -----------------------
def _with_projectors(circ, wires, values):
    """The circuit with |v><v| inserted on each sliced wire (q, g), right
    after two-qubit gate g."""
    out = Circuit(n_qubits=circ.n_qubits, name=circ.name + "_proj")
    for gi, g in enumerate(circ.gates):
        out.gates.append(g)
        for (q, gg), v in zip(wires, values):
            if gg == gi:
                P = np.zeros((2, 2), complex)
                P[v, v] = 1.0
                out.gates.append(Gate((q,), P, g.layer, "proj"))
    return out


def _sliced_case():
    w = make_workload("grid3x4_m8")
    sl = choose_slices(w.struct, w.tree, 64, n_sliced=3)
    wires = [tuple(int(x) for x in w.struct.edge_wire[e]) for e in sl]
    return w, wires


def test_sliced_partials_equal_projected_state_vector():
    w, wires = _sliced_case()
    parts = tn.partial_amplitudes(w.circuit, w.tree.ssa, w.bits, wires, range(8))
    for s in range(8):
        vals = [(s >> j) & 1 for j in range(3)]
        ref = sv.amplitudes(_with_projectors(w.circuit, wires, vals), w.bits)
        assert np.max(np.abs(parts[s] - ref)) < 1e-14
    assert np.max(np.abs(parts)) > 1e-3


def test_slicing_invariance_sum_over_slices():
    w, wires = _sliced_case()
    parts = tn.partial_amplitudes(w.circuit, w.tree.ssa, w.bits, wires, range(8))
    amps = sv.amplitudes(w.circuit, w.bits)
    assert np.max(np.abs(parts.sum(axis=0) - amps)) < 1e-14
    assert np.max(np.abs(tn.partial_amplitudes(w.circuit, w.tree.ssa, w.bits)[0] - amps)) < 1e-14


def test_tn_matches_sv_on_the_12_qubit_workload():
    w = make_workload("grid3x4_m8")
    amps = sv.amplitudes(w.circuit, w.bits)
    parts = tn.partial_amplitudes(w.circuit, w.tree.ssa, w.bits)
    rel = np.linalg.norm(parts[0] - amps) / np.linalg.norm(amps)
    assert rel < 1e-13
    # this 8-cycle circuit is shallow for 12 qubits: report, do not demand, PT
    f = xeb.linear_xeb(amps, 12)
    assert abs(f) < 1.0


# Planted mistakes: each one fails a pin ------------------------------------
def _mutate(circ, fn):
    out = Circuit(n_qubits=circ.n_qubits, name=circ.name + "_mut")
    out.gates = [Gate(g.qubits, fn(g), g.layer, g.kind) for g in circ.gates]
    return out


def test_planted_transposed_two_qubit_gate_fails_brute_force():
    c = random_circuit(grid_layout(2, 3), 8, 5)
    bad = _mutate(c, lambda g: g.matrix.T.copy() if len(g.qubits) == 2 and g.layer == 3 else g.matrix)
    # fSim at Delta = 0 is symmetric; make the slip visible with a 1q gate too
    bad = _mutate(bad, lambda g: g.matrix.T.copy() if len(g.qubits) == 1 else g.matrix)
    assert np.max(np.abs(sv.state(bad) - brute.amplitudes(c))) > 1e-3


def test_planted_reversed_bit_order_fails_brute_force():
    c = random_circuit(grid_layout(2, 3), 8, 5)
    n = c.n_qubits
    bits = _all_bits(n)
    good = sv.amplitudes(c, bits)
    bad = sv.amplitudes(c, bits[:, ::-1])
    assert np.max(np.abs(good - brute.amplitudes(c))) < 1e-13
    assert np.max(np.abs(bad - brute.amplitudes(c))) > 1e-3


def test_planted_wrong_slice_wire_fails_projector_pin():
    w, wires = _sliced_case()
    # the slip: slicing the wire *before* the gate instead of after it
    net = tn.UnfusedNetwork(w.circuit)
    q, g = wires[0]
    prev = [gi for gi in range(g) if len(w.circuit.gates[gi].qubits) == 2 and q in w.circuit.gates[gi].qubits]
    if not prev:
        pytest.skip("first sliced wire has no earlier two-qubit gate")
    bad_wires = [(q, prev[-1])] + wires[1:]
    parts_bad = tn.partial_amplitudes(w.circuit, w.tree.ssa, w.bits, bad_wires, range(8))
    vals = [0, 0, 0]
    ref = sv.amplitudes(_with_projectors(w.circuit, wires, vals), w.bits)
    assert np.max(np.abs(parts_bad[0] - ref)) > 1e-4
    # ... although slicing invariance alone would not notice it
    amps = sv.amplitudes(w.circuit, w.bits)
    assert np.max(np.abs(parts_bad.sum(axis=0) - amps)) < 1e-13
    assert net.n_groups == 34


# cost-model network (oracle/mlp.py) ------------------------------------------
def _mlp_case(d=5, h=7, n=11, seed=3):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.7, mlp.n_params(d, h))
    X = rng.normal(0, 1, (n, d))
    t = rng.normal(0, 1, n)
    return p, X, t


def test_mlp_gradient_matches_central_differences():
    d, h = 5, 7
    p, X, t = _mlp_case(d, h)
    g, L = mlp.grad(p, X, t, d, h)
    assert abs(L - mlp.loss(p, X, t, d, h)) < 1e-14
    eps = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = eps
        fd[i] = (mlp.loss(p + e, X, t, d, h) - mlp.loss(p - e, X, t, d, h)) / (2 * eps)
    assert np.max(np.abs(fd - g)) <= 1e-7 * max(1.0, np.max(np.abs(g)))


def test_mlp_forward_hand_evaluated():
    # D = 2, H = 2, evaluated by hand (x -> z1 -> a1 -> z2 -> a2 -> y):
    #   x = (3, 1):  z1 = (2, 2.5), z2 = (5, 3),   y = 2*5 - 3 + 0.25 = 7.25
    #   x = (0, 1):  z1 = (-1, 1), a1 = (0, 1), z2 = (1.5, 2), y = 3 - 2 + 0.25 = 1.25
    #   x = (-2, 0): z1 = (-2, -2), a1 = 0, z2 = (0.5, 0), y = 1 + 0.25 = 1.25
    p = mlp.pack([[1, -1], [0.5, 2]], [0, -1], [[1, 1], [-1, 2]], [0.5, 0], [2, -1], 0.25)
    y = mlp.forward(p, [[3, 1], [0, 1], [-2, 0]], 2, 2)
    np.testing.assert_allclose(y, [7.25, 1.25, 1.25], rtol=0, atol=1e-15)


def test_mlp_first_adam_step_moves_by_lr_times_sign():
    # after one step the bias-corrected ratio m_hat / sqrt(v_hat) is g / |g|
    d, h = 5, 7
    p, X, t = _mlp_case(d, h)
    g, _ = mlp.grad(p, X, t, d, h)
    lr = 1e-3
    p1, m, v = mlp.adam_step(p, g, np.zeros_like(p), np.zeros_like(p), 1, lr)
    big = np.abs(g) > 1e-4
    np.testing.assert_allclose((p - p1)[big], lr * np.sign(g[big]), rtol=1e-4)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_planted_missing_relu_mask_fails_finite_differences():
    # the backward pass with relu'(z2) dropped is a plausible slip: the
    # finite-difference pin must catch it
    d, h = 5, 7
    p, X, t = _mlp_case(d, h)
    W1, b1, W2, b2, w3, b3 = mlp.unpack(p, d, h)
    y, (Xk, z1, a1, z2, a2) = mlp.forward(p, X, d, h, keep=True)
    dy = 2.0 * (y - t) / X.shape[0]
    dz2_wrong = np.outer(dy, w3)  # mask missing
    g_wrong_W2 = dz2_wrong.T @ a1
    assert np.any(z2 <= 0)
    off = h * d + h  # W2 block of the flat parameter vector
    eps = 1e-6
    fd = np.empty(h * h)
    for i in range(h * h):
        e = np.zeros_like(p)
        e[off + i] = eps
        fd[i] = (mlp.loss(p + e, X, t, d, h) - mlp.loss(p - e, X, t, d, h)) / (2 * eps)
    # the pin's tolerance (as in the finite-difference test) rejects it
    assert np.max(np.abs(fd - g_wrong_W2.ravel())) > 1e-7 * max(1.0, np.max(np.abs(fd))) * 100


# Correlated batches and perfect samples from them ------------------------
def test_correlated_amplitudes_cover_the_state():
    # every closed assignment of 10 qubits with 3 left open: the completions
    # enumerate every basis state once, so they reproduce the brute-force
    # unitary's column (independent of the state-vector code) and sum to 1
    c = random_circuit(grid_layout(2, 5), 6, seed=8)
    n, oq = 10, [1, 4, 9]
    closed = [q for q in range(n) if q not in oq]
    base = np.zeros((1 << len(closed), n), np.uint8)
    for r in range(base.shape[0]):
        for i, q in enumerate(closed):
            base[r, q] = (r >> (len(closed) - 1 - i)) & 1
    amps = sv.correlated_amplitudes(c, base, oq)
    full = brute.unitary(c)[:, 0]
    rows = sv.completion_bits(base, oq)
    idx = (rows.astype(np.int64) << np.arange(n - 1, -1, -1)).sum(axis=1)
    assert np.allclose(amps, full[idx], atol=1e-13)
    assert abs(np.sum(np.abs(amps) ** 2) - 1.0) < 1e-12
    assert sorted(idx.tolist()) == list(range(1 << n))
    # the completion that equals the row itself is the row's own amplitude
    own = sv.amplitudes(c, base)  # base rows hold 0 at the open qubits: completion 0
    assert np.allclose(amps.reshape(-1, 8)[:, 0], own)


def test_sample_completions_rule_and_frequencies():
    from oracle.sampling import sample_completions
    a = np.array([0.5, 0.5j])  # |a|^2 = 1/4 each (exact): total 1/2
    for u, want in ((0.0, 0), (0.49, 0), (0.5, 1), (0.51, 1), (0.999, 1)):
        # u = 1/2: the running sum 1/4 does not exceed the threshold 1/4
        assert sample_completions(a, 1, np.array([u]))[0] == want, u
    z = np.array([0.0, 0.0, 0.6, 0.8])  # zeros are never drawn
    assert sample_completions(z, 2, np.array([0.0]))[0] == 2
    rng = np.random.default_rng(2)
    amps = rng.normal(size=(1, 16)) + 1j * rng.normal(size=(1, 16))
    p = np.abs(amps[0]) ** 2 / np.sum(np.abs(amps) ** 2)
    k = 200000
    picks = sample_completions(np.repeat(amps, k, axis=0).ravel(), 4, rng.random(k))
    freq = np.bincount(picks, minlength=16) / k
    assert np.all(np.abs(freq - p) < 5 * np.sqrt(p * (1 - p) / k) + 1e-4)
