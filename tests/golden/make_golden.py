"""Write tests/golden/full_size_oracle.json from the FP64 oracle alone.

For each full-size workload it stores the oracle's MINRES iteration count, its
true relative residual, the 2-norm of each solution block and the solution at
a fixed set of sampled indices.  The GPU tests compare against these values.
Run:  python tests/golden/make_golden.py   (tens of minutes on a CPU)
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import sg_inputs as si  # noqa: E402
from oracle.solve import solve  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "full_size_oracle.json")


def sample_indices(N, count=256, seed=0):
    return np.sort(np.random.default_rng(seed).choice(N, size=min(count, N), replace=False))


def record(pr):
    t0 = time.time()
    res = solve(pr)
    F = pr.kkt_size // 3
    idx = sample_indices(pr.kkt_size)
    return {
        "name": pr.name,
        "iterations": int(res.iterations),
        "status": res.status,
        "rel_true": float(res.rel_true),
        "block_norms": [float(np.linalg.norm(res.x[b * F:(b + 1) * F])) for b in range(3)],
        "sample_idx": idx.tolist(),
        "sample_val": [float(v) for v in res.x[idx]],
        "oracle_seconds": time.time() - t0,
    }


def main():
    out = {}
    if os.path.exists(OUT):
        out = json.load(open(OUT))
    jobs = [("steady_128_beta%g" % b, lambda b=b: si.steady_128(b)) for b in si.STEADY_128_BETAS]
    jobs.append(("time_64", si.time_64))
    for key, mk in jobs:
        if key in out and "--force" not in sys.argv:
            continue
        pr = mk()
        out[key] = record(pr)
        print(key, out[key]["iterations"], out[key]["rel_true"], f"{out[key]['oracle_seconds']:.0f}s", flush=True)
        json.dump(out, open(OUT, "w"), indent=1)


if __name__ == "__main__":
    main()
