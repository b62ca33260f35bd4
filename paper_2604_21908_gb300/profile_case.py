"""Small, self-contained GPU cases for profiling one batch of two-site updates.

`python -m paper_2604_21908_gb300.profile_case --chi 64 --batch 4` loads the seeded peaked
MPO with every interior bond at `chi` (the saturated regime of the perturbed hidden-
permutation workloads), then applies one wave of `batch` two-site updates with Haar
operators on disjoint interior bonds through the C ABI, `--repeat` times, and prints the
per-kernel-class launches, milliseconds and algorithmic TFLOP/s.  Every launch runs the
same kernels as a contraction wave: merge GEMM, gate, accumulator set-up, Jacobi,
truncation, split.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2604_21908_gb300 import binding  # noqa: E402
from paper_2604_21908_gb300 import workloads as W  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--chi", type=int, default=64)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--eps", type=float, default=1e-10)
    ap.add_argument("--precision", type=int, default=0, help="0 FP64 merges, 1 complex 3xTF32 tensor-core merges")
    ap.add_argument("--pre-sweeps", type=int, default=0, help="cap on FP32 preconditioning sweeps (0: default)")
    args = ap.parse_args()
    n = 2 * args.batch + 8
    B, lam = W.peaked_saturated_state(n, args.chi, seed=1)
    rng = W.rng_for(12, 0)
    ops = np.array([W.haar_unitary(rng, 16) for _ in range(args.batch)])
    bonds = [4 + 2 * k for k in range(args.batch)]
    kw = {"precondition_sweeps": args.pre_sweeps} if args.pre_sweeps > 0 else {}
    ctx = binding.Context(eps=args.eps, chi_max=args.chi, precision=args.precision, **kw)
    c = ctx.load_gates(n, np.zeros((0, 2), np.int32), np.zeros((0, 4, 4), complex))
    c.reset_timers(True)
    for _ in range(args.repeat):
        c.set_state(B, lam)
        chi = c.apply_updates(bonds, ops)
    la, ms, fl = c.timers()
    names = ["merge_gate", "jacobi", "truncate", "split", "other"]
    st = c.stats()
    out = {"chi": args.chi, "batch": args.batch, "precision": args.precision, "repeat": args.repeat, "counts": chi.tolist(),
           "sweeps": {"fp64": st["max_sweeps"], "fp32": st["max_sweeps_fp32"], "fallbacks": st["fallbacks"]},
           "kernels": {nm: {"launches": int(la[k]), "ms": float(ms[k]),
                            "tflops_per_s": float(fl[k] / (ms[k] * 1e9)) if ms[k] > 0 else None}
                       for k, nm in enumerate(names)}}
    print(json.dumps(out))
    c.close()
    ctx.close()


if __name__ == "__main__":
    main()
