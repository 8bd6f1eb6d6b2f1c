"""The larger workloads against stored CPU-oracle values.

* grid6x7_m10 (42 qubits, 10 cycles, 2^14 slices): 32 seeded slices x 16
  seeded bitstrings of per-slice partial amplitudes from the complex128
  tensor-network oracle, in FP32, BF16x3 and TF32.
* diamond53_m12 (53 qubits, 12 cycles, 8192 bitstrings): the full
  contraction on the GPU, 16 seeded amplitudes compared with the oracle.
"""

import importlib.util
import os

import numpy as np
import pytest

from gpu_helpers import rel_l2, run_plan, run_slices
from rqc import make_workload

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "bf16x3": 1e-3, "tf32": 1e-2}


def _mg():
    spec = importlib.util.spec_from_file_location(
        "make_golden", os.path.join(os.path.dirname(__file__), "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    return mg


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "tf32"])
def test_grid6x7_sampled_slices(prec):
    mg = _mg()
    rec = mg.read_json(mg.slices_path("grid6x7_m10"))
    w = make_workload("grid6x7_m10")
    assert rec["inputs_sha256"] == mg.input_digest(w.circuit, w.bits)
    bits = w.bits[rec["rows"]]
    got = run_slices(w.circuit, bits, rec["tree_ssa"], rec["sliced_edges"], rec["slice_ids"], precision=prec)
    err = rel_l2(got, rec["partials"])
    print(f"grid6x7_m10 {prec}: rel-L2 over {got.size} partials {err:.3e}")
    assert err <= TOL[prec], err


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_diamond53_sampled_amplitudes(prec):
    mg = _mg()
    rec = mg.read_json(mg.sample_path("diamond53_m12"))
    w = make_workload("diamond53_m12")
    assert rec["inputs_sha256"] == mg.input_digest(w.circuit, w.bits)
    got, p = run_plan(w.circuit, w.bits, w.tree.ssa, w.tree.sliced, precision=prec, workspace_limit=160 << 30)
    err = rel_l2(got[rec["rows"]], rec["amplitudes"])
    print(f"diamond53_m12 {prec}: rel-L2 over {len(rec['rows'])} sampled amplitudes {err:.3e}")
    assert err <= TOL[prec], err


@pytest.mark.parametrize("config", [0, 1])
def test_diamond53_small_rank_steps_on_the_row_kernel(config):
    # every step the per-row kernel can take runs on it, under either
    # schedule (blocks of up to 64 or 4 row passes), among them K = N = 16
    # steps with groups of one and of several instances; FP32 against the
    # stored oracle sample
    mg = _mg()
    rec = mg.read_json(mg.sample_path("diamond53_m12"))
    w = make_workload("diamond53_m12")
    fits = lambda st: st["nb"] <= 4 and st["kb"] + st["nb"] <= 8  # noqa: E731
    got, p = run_plan(w.circuit, w.bits, w.tree.ssa, w.tree.sliced, precision="fp32",
                      force_config=lambda st: config if fits(st) else None, workspace_limit=160 << 30)
    big = [s for s in p.tn_plan_steps() if s["kb"] == 4 and s["nb"] == 4 and s["mb"] >= 7]
    assert big and any(s["n_inst"] > s["n_groups"] for s in big)
    err = rel_l2(got[rec["rows"]], rec["amplitudes"])
    print(f"diamond53_m12 fp32, row kernel (configuration {config}): rel-L2 {err:.3e}")
    assert err <= TOL["fp32"], err


@pytest.mark.parametrize("pairs", [True, False])
def test_diamond53_column_tile_pairs(pairs):
    # every tensor-core step with N >= 64 per instance and K >= 256 on
    # configuration 2 (a row tile's column tiles back to back): with pairs
    # on, BF16x3 steps whose B is packed walk the column tiles two at a
    # time, one MMA of N = 256 into both accumulators (N = 64: two instances
    # of a group, a group of odd size ending with a pad tile); off, one at a
    # time; both against the stored oracle sample
    mg = _mg()
    rec = mg.read_json(mg.sample_path("diamond53_m12"))
    w = make_workload("diamond53_m12")
    wide = lambda st: st["nb"] >= 6 and st["kb"] >= 8 and st["mb"] >= 6  # noqa: E731
    got, p = run_plan(w.circuit, w.bits, w.tree.ssa, w.tree.sliced, precision="bf16x3",
                      force_config=lambda st: 2 if wide(st) else None, tc_pairs=pairs,
                      workspace_limit=160 << 30)
    kinds = p.tn_plan_step_times()[1]
    steps = [s for s, k in zip(p.tn_plan_steps(), kinds) if k == 2 and wide(s)]
    # several groups and several K chunks among them; N = 64 steps whose
    # groups are not all of even size (pad tiles)
    assert any(s["n_groups"] > 1 for s in steps) and any(s["kb"] >= 6 for s in steps)
    assert any(s["nb"] == 6 and s["n_inst"] % 2 and s["n_inst"] >= 8 * s["n_groups"] for s in steps)
    err = rel_l2(got[rec["rows"]], rec["amplitudes"])
    print(f"diamond53_m12 bf16x3, column-tile pairs {pairs}: {len(steps)} wide steps, rel-L2 {err:.3e}")
    assert err <= TOL["bf16x3"], err
