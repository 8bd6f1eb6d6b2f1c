"""Config selection on the GPU: the cost-model network's kernels against the
float64 oracle (forward, gradient, Adam, FP16 inference), the exhaustive
autotuner (times, choice, parity of the tuned plan), and what the trained
network gains: configurations for held-out plans without measuring them,
compared with the plan's built-in rule and the autotuner.

Tolerances.  FP32 forward and gradient: the sums run over at most 128
products of O(1) terms, so the relative error stays near 1e-6; held to
1e-4.  FP16 inference: 11-bit significands with FP32 sums every 16
products; held to 3e-2 of the output scale.
"""

import numpy as np
import pytest

from gpu_helpers import rel_l2, require_cuda
from oracle import mlp as omlp
from oracle import sv

pytestmark = pytest.mark.gpu

D, H = 24, 128


def _params(seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.uniform(-1, 1, H * D) * np.sqrt(6.0 / D), rng.normal(0, 0.1, H),
                           rng.uniform(-1, 1, H * H) * np.sqrt(6.0 / H), rng.normal(0, 0.1, H),
                           rng.uniform(-1, 1, H) * np.sqrt(3.0 / H), [0.3]]) * scale


def _data(n, seed=1):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, (n, D))
    t = np.sin(X[:, 0] * 3) + X[:, 1] * X[:, 2] + 0.5 * X[:, 3]
    return X, t


def _dev(torch, a, dt=None):
    return torch.from_numpy(np.ascontiguousarray(a, dt or np.float32)).cuda()


@pytest.mark.parametrize("n", [1, 37, 5000])
def test_forward_matches_oracle(n):
    torch, tn = require_cuda()
    p = _params()
    X, _ = _data(n)
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    tn.tn_mlp_forward(_dev(torch, p), _dev(torch, X), n, y)
    torch.cuda.synchronize()
    ref = omlp.forward(p.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64), D, H)
    assert rel_l2(y.cpu().numpy(), ref) <= 1e-4


@pytest.mark.parametrize("n", [3, 700, 9000])
def test_gradient_matches_oracle(n):
    torch, tn = require_cuda()
    p = _params(2).astype(np.float32)
    X, t = _data(n, 3)
    X, t = X.astype(np.float32), t.astype(np.float32)
    g = torch.empty(tn.TN_MLP_NPARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    scratch = torch.empty(tn.tn_mlp_grad_scratch_bytes(n), dtype=torch.uint8, device="cuda")
    tn.tn_mlp_grad(_dev(torch, p), _dev(torch, X), _dev(torch, t), n, g, loss, scratch)
    torch.cuda.synchronize()
    ref, L = omlp.grad(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64), D, H)
    got = g.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - L) <= 1e-4 * L
    # each parameter block separately (W1, b1, W2, b2, w3, b3)
    for a, b in zip(omlp.unpack(got, D, H), omlp.unpack(ref, D, H)):
        a, b = np.atleast_1d(a).ravel(), np.atleast_1d(b).ravel()
        assert np.linalg.norm(a - b) <= 1e-4 * max(np.linalg.norm(b), 1e-8)
    # deterministic: the same call gives the same bits
    g2 = torch.empty_like(g)
    tn.tn_mlp_grad(_dev(torch, p), _dev(torch, X), _dev(torch, t), n, g2, loss, scratch)
    torch.cuda.synchronize()
    assert torch.equal(g, g2)


def test_adam_matches_oracle():
    torch, tn = require_cuda()
    rng = np.random.default_rng(5)
    p = _params(4).astype(np.float32)
    m = rng.normal(0, 0.01, p.size).astype(np.float32)
    v = rng.uniform(0, 1e-3, p.size).astype(np.float32)
    g = rng.normal(0, 0.1, p.size).astype(np.float32)
    dp, dm, dv = _dev(torch, p), _dev(torch, m), _dev(torch, v)
    tn.tn_mlp_adam(dp, _dev(torch, g), dm, dv, 7, lr=1e-3)
    torch.cuda.synchronize()
    # the entry point takes beta1, beta2 as FP32: the oracle gets the same
    # rounded values (1 - 0.999f differs from 0.001 by 1.3e-5 relative)
    rp, rm, rv = omlp.adam_step(p.astype(np.float64), g.astype(np.float64), m.astype(np.float64),
                                v.astype(np.float64), 7, float(np.float32(1e-3)), beta1=float(np.float32(0.9)),
                                beta2=float(np.float32(0.999)), eps=float(np.float32(1e-8)))
    # m = beta1 m + (1 - beta1) g cancels terms of size ~1e-2: absolute bound
    # at that scale
    np.testing.assert_allclose(dm.cpu().numpy(), rm, rtol=1e-5, atol=2e-8)
    np.testing.assert_allclose(dv.cpu().numpy(), rv, rtol=1e-5, atol=1e-11)
    np.testing.assert_allclose(dp.cpu().numpy(), rp, rtol=1e-5, atol=1e-7)


def test_fp16_inference_matches_oracle():
    torch, tn = require_cuda()
    p = _params(6)
    X, _ = _data(3000, 7)
    q = torch.empty(tn.TN_MLP_NPARAMS, dtype=torch.int16, device="cuda")
    tn.tn_mlp_to_half(_dev(torch, p), q)
    y = torch.empty(len(X), dtype=torch.float32, device="cuda")
    tn.tn_mlp_forward_f16(q, _dev(torch, X), len(X), y)
    torch.cuda.synchronize()
    ref = omlp.forward(p, X, D, H)
    err = np.abs(y.cpu().numpy() - ref)
    assert np.max(err) <= 3e-2 * max(1.0, np.max(np.abs(ref)))


def test_training_fits_a_smooth_target():
    torch, tn = require_cuda()
    from paper_2212_04749_gb300.costmodel import Trainer
    X, t = _data(8192, 9)
    tr = Trainer(seed=1)
    y0 = tr.predict(X.astype(np.float32))
    hist = tr.fit(X.astype(np.float32), t.astype(np.float32), epochs=80, batch=1024, lr=3e-3)
    y1 = tr.predict(X.astype(np.float32))
    mse0, mse1 = np.mean((y0 - t) ** 2), np.mean((y1 - t) ** 2)
    print(f"mlp fit: mse {mse0:.3f} -> {mse1:.4f}")
    assert mse1 < 0.05 * mse0


@pytest.fixture(scope="module")
def case20():
    from rqc import grid_layout, network_structure, random_circuit
    from rqc.bitstrings import uniform_bitstrings
    from rqc.tree import ContractionTree, candidate_trees, choose_slices
    c = random_circuit(grid_layout(4, 5), 12, seed=21)
    s = network_structure(c)
    bits = uniform_bitstrings(20, 1500, seed=5)
    ssa = candidate_trees(s, 1500, seed=2, trials=2)[0]
    sl = choose_slices(s, ContractionTree(ssa=ssa), 1500, n_sliced=2)
    return c, bits, ssa, sl, sv.amplitudes(c, bits)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_autotuner_picks_fastest_measured_and_keeps_parity(case20, prec):
    torch, tn = require_cuda()
    c, bits, ssa, sl, ref = case20
    p = tn.Plan(c, bits, ssa, sl)
    ws = torch.empty(p.info["workspace_bytes"], dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    p.tn_plan_bind(ws, stream=st)
    amps = torch.zeros(2 * len(bits), dtype=torch.float64, device="cuda")
    times = p.tn_plan_autotune(prec, amps, reps=2, stream=st)
    steps = p.tn_plan_steps()
    cfg = p.tn_plan_get_configs()
    for s, step in enumerate(steps):
        row_ok = step["nb"] <= 4 and step["kb"] + step["nb"] <= 8
        assert np.isfinite(times[s, 2]) and np.isfinite(times[s, 3])
        assert np.isfinite(times[s, 0]) == row_ok and np.isfinite(times[s, 1]) == row_ok
        assert cfg[s] == int(np.nanargmin(times[s]))
    amps.zero_()
    p.tn_contract(amps, prec, stream=st)
    p.tn_plan_check(stream=st)
    torch.cuda.synchronize()
    err = rel_l2(amps.cpu().numpy().view(np.complex128), ref)
    print(f"autotuned {prec}: rel-L2 {err:.2e}, configs {np.bincount(cfg, minlength=4).tolist()}")
    assert err <= (1e-5 if prec == "fp32" else 1e-3)


def test_cost_model_gain_over_the_rule_and_regret():
    # Train on the autotuner's timings of seeded random plans, then configure
    # held-out plans with the network alone (no measurement) and compare the
    # contraction time with the plan's built-in rule (the method without the
    # network) and with the exhaustive autotuner (the judge of its regret).
    torch, tn = require_cuda()
    from paper_2212_04749_gb300 import costmodel as cm
    cases = [cm.random_case(s) for s in range(40)]
    corpus = cm.collect(cases, cm.Corpus(), reps=1, budget_s=45, flops_range=(1e8, 1e12))
    assert len(corpus.y) > 2000
    tr = cm.Trainer(seed=0)
    tr.fit(corpus.X, corpus.y, epochs=400, batch=2048, lr=3e-3)
    pred = tr.predict(corpus.X)
    fit_mse = float(np.mean((pred - corpus.y) ** 2))
    rows = []
    for s in (10002, 10006, 10015):  # held-out plans of 1.5e11-2e11 flops
        b = cm.bind(cm.random_case(s))
        assert b is not None, f"held-out case {s} did not bind"
        for prec in ("fp32", "bf16x3"):
            r = cm.evaluate(b, prec, tr, reps=3)
            rows.append(r)
            print(f"{r['case']} {prec}: rule {r['rule_ms']:.3f} ms, model {r['model_ms']:.3f} ms "
                  f"(selection {r['model_select_s'] * 1e3:.1f} ms), model + fallback {r['hybrid_ms']:.3f} ms "
                  f"({r['uncertain_frac']:.0%} of steps timed, {r['hybrid_select_s']:.2f} s), autotuner "
                  f"{r['tuned_ms']:.3f} ms (tuning {r['autotune_s']:.2f} s), table regret {r['table_regret']:+.3f}")
        del b
    assert len(rows) == 6
    rule = sum(r["rule_ms"] for r in rows)
    model = sum(r["model_ms"] for r in rows)
    hybrid = sum(r["hybrid_ms"] for r in rows)
    tuned = sum(r["tuned_ms"] for r in rows)
    sel = sum(r["model_select_s"] for r in rows)
    hsel = sum(r["hybrid_select_s"] for r in rows)
    tune = sum(r["autotune_s"] for r in rows)
    print(f"cost model: corpus {len(corpus.y)} rows, fit mse {fit_mse:.3f} (log2 ms)^2; "
          f"total rule {rule:.2f} ms, model {model:.2f} ms, model + fallback {hybrid:.2f} ms, "
          f"autotuner {tuned:.2f} ms; selection {sel:.3f} s / {hsel:.2f} s vs autotuning {tune:.2f} s")
    # Gain of the learned part, per plan and precision (geometric mean of
    # rule time / chosen time; some plans leave nothing to gain, the
    # autotuner itself is 1-11 % faster than the rule on these): the network
    # with its autotuner fallback beats the rule by more than the run-to-run
    # noise of these timings (about 1 %), stays within 3 % of the exhaustive
    # autotuner and takes less than half its time; the network alone (no
    # measurement at all) stays within 5 % of the autotuner.
    gain = float(np.exp(np.mean([np.log(r["rule_ms"] / r["hybrid_ms"]) for r in rows])))
    gain_tuned = float(np.exp(np.mean([np.log(r["rule_ms"] / r["tuned_ms"]) for r in rows])))
    print(f"geometric-mean gain over the rule: model + fallback {gain:.3f}, autotuner {gain_tuned:.3f}")
    assert gain >= 1.02
    assert hybrid <= 1.03 * tuned
    assert hsel < 0.5 * tune
    assert model <= 1.05 * tuned
    assert sel < 0.05 * tune
