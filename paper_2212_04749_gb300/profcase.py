"""Run one contraction of a seeded plan, for profilers (ncu) and timing.

    python -m paper_2212_04749_gb300.profcase --case 10002 --precision bf16x3 --reps 1
    python -m paper_2212_04749_gb300.profcase --workload grid3x4_m8 --fuse 1

--case picks a seeded random circuit and tree (costmodel.random_case), whose
plans stay within a few GB of workspace, so that full ncu captures of the
library's kernels stay small; --workload picks a named workload.
"""

import argparse
import sys


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", type=int, default=10002)
    ap.add_argument("--workload", default=None)
    ap.add_argument("--precision", default="bf16x3", choices=["fp32", "tf32", "bf16x3"])
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--fuse", type=int, default=0)
    ap.add_argument("--ws-gib", type=float, default=4.0)
    ap.add_argument("--list-steps", action="store_true", help="print each step's shape, bytes and flops")
    args = ap.parse_args()
    import torch
    from . import builder, costmodel, tn
    builder.build()
    tn.load()
    case = costmodel.workload_case(args.workload) if args.workload else costmodel.random_case(args.case)
    p = tn.Plan(case.circuit, case.bits, case.ssa, case.sliced, workspace_limit=int(args.ws_gib * 2 ** 30),
                fuse=args.fuse)
    ws = torch.empty(p.info["workspace_bytes"], dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    p.tn_plan_bind(ws, stream=st)
    amps = torch.zeros(2 * max(p.k, 1), dtype=torch.float64, device="cuda")
    for _ in range(args.reps):
        p.tn_contract(amps, args.precision, stream=st)
    torch.cuda.synchronize()
    p.tn_plan_check(stream=st)
    print(f"ok {case.name} workspace {p.info['workspace_bytes']} bytes, {p.info['n_steps']} steps")
    if args.list_steps:
        # the steps in launch order with their shapes and algorithmic bytes
        # and flops per launch (one slice batch), to match profiler records
        ms, kinds = p.tn_plan_step_times()
        for s, st in enumerate(p.tn_plan_steps()):
            print(f"step {s} family {int(kinds[s])} mb {st['mb']} kb {st['kb']} nb {st['nb']} "
                  f"inst {st['n_inst']} groups {st['n_groups']} inst_b {st['n_inst_b']} runs {st['runs']:.0f} "
                  f"bytes {st['bytes']:.0f} flops {st['flops']:.0f}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
