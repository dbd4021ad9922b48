"""Writes oracle_pcg_iterations_c<id>.json: iterations the oracle's FP64 block-Jacobi PCG
needs to reach relative residual 1e-8 on a workload (calls only oracle/ and the input
generator).  Used to scale the CPU baseline's timed sample to a whole solve.

Usage: python tests/golden/make_oracle_iterations.py [config_id ...]   (default: 2)
"""

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import model, solve  # noqa: E402


def main(ids):
    for cid in ids:
        p = synth.config_problem(cid)
        L = model.laplacian_from_csr(p.graph.rowptr, p.graph.col, p.graph.val, p.n)
        A = model.powerlaw_mixing(p.nu, p.beta)
        b = model.rhs(p.D, p.Yobs[0], A)
        t0 = time.perf_counter()
        x, it, rel, secs = solve.pcg_block_jacobi(L, p.D, p.tau, p.kappa, A, b, eps=1e-8)
        true_rel = solve.relres(L, p.D, p.tau, p.kappa, A, x, b)
        out = {"config": cid, "workload": p.name, "iterations": it, "recursive_relres": rel,
               "true_relres": true_rel, "seconds": secs,
               "method": "oracle.solve.pcg_block_jacobi, eps=1e-8, x0=0, FP64"}
        with open(os.path.join(HERE, f"oracle_pcg_iterations_c{cid}.json"), "w") as f:
            json.dump(out, f, indent=1)
        print(out, f"({time.perf_counter() - t0:.0f} s)")


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [2])
