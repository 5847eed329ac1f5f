"""Writes oracle/counts.json: iteration counts of the oracle's own solves of
the benchmark workloads, computed by the oracle alone.

The CPU baseline of the benchmark times a bounded sample of the oracle's plain
FP64 BiCGStab (a few iterations at full size) and scales it to a whole solve;
the scale is the number of iterations the oracle needs for that solve, stored
here.  Run: python oracle/measure_counts.py   (32^4 takes a few minutes)
"""

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
import synth  # noqa: E402

WORKLOADS = {
    # name: (dims, eps, kappa, c_sw, gauge seed, source seed, tol)
    "32^4 eps=0.3 kappa=0.125": ((32, 32, 32, 32), 0.3, 0.125, 1.0, 1, 2, 1e-10),
    "16^4 eps=0.3 kappa=0.12": ((16, 16, 16, 16), 0.3, 0.12, 1.0, 1, 2, 1e-10),
    "8^4 eps=0.3 kappa=0.12": ((8, 8, 8, 8), 0.3, 0.12, 1.0, 1, 2, 1e-10),
}


def main():
    path = os.path.join(HERE, "counts.json")
    out = json.load(open(path)) if os.path.exists(path) else {}
    only = sys.argv[1:]
    for name, (dims, eps, kappa, csw, gs, ss, tol) in WORKLOADS.items():
        if only and not any(o in name for o in only):
            continue
        U = synth.gauge_field(dims, eps, gs)
        eta = synth.gaussian_source(dims, ss)
        op = oracle.Op(dims, (1, 1, 1, -1), U, kappa, csw)
        t0 = time.time()
        phi, info = op.solve(eta, tol)
        out[name] = {"plain_bicgstab": info, "seconds": time.time() - t0, "threads": oracle.get_threads(),
                     "true_rel_residual": op.true_residual(eta, phi)}
        print(name, out[name], flush=True)
    json.dump(out, open(path, "w"), indent=1)


if __name__ == "__main__":
    main()
