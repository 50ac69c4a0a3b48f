"""Writes tests/golden/quality_reference.json: the constrained optimum of Eq. (optim1)
on the paper-setting test set (Sec. VI-A: 5,000 i.i.d. CN(0,1) channels C^{8x64},
gamma = 10 dB, sigma_nu = 1), from the FP64 oracle's long-run ADMM solve (O3), and the
metrics the paper reports for it (Sec. VI-B: PCG, sum rate).  These are the "target"
values of the quality reproduction (the paper's CVXPY optimum is replaced by O3).

Calls only the oracle and the seeded channel generator.  Run from the repository root:
    python tests/golden/make_quality_reference.py
"""
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2304_12745_gb300 import channels as ch  # noqa: E402


def main():
    oracle.build()
    H = ch.paper_set("test").astype(np.complex128)
    B, K, M = H.shape
    t = np.full((B, K), math.sqrt(10.0))
    t0 = time.time()
    W, iters, st = oracle.batch_admm(H, t, rho=1.0, max_iter=200000, tol=1e-10,
                                     nthreads=os.cpu_count() or 1)
    assert np.all(st == oracle.OK), "ADMM did not converge on every test channel"
    pcg = np.array([oracle.pcg(H[b], t[b], W[b]) for b in range(B)])
    rsum = np.array([oracle.sum_rate(H[b], W[b], 1.0) for b in range(B)])
    out = {
        "_about": "Constrained optimum of Eq. (optim1) on the paper-setting test set, by the "
                  "FP64 oracle's ADMM (O3, tolerance 1e-10); written by "
                  "tests/golden/make_quality_reference.py",
        "test_set": {"name": "test", "B": B, "K": K, "M": M, "seed": ch.PAPER_SETS["test"][1],
                     "channels": "i.i.d. CN(0,1), paper_set('test')", "t": "sqrt(10) per user"},
        "pcg_mean": float(pcg.mean()), "pcg_std": float(pcg.std()),
        "sum_rate_mean": float(rsum.mean()),
        "admm_iterations_mean": float(iters.mean()), "admm_iterations_max": int(iters.max()),
        "seconds": round(time.time() - t0, 1),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "quality_reference.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
