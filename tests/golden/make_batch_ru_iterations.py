"""Write tests/golden/batch512_ru_oracle.json: the oracle's own fp32 Jacobi-PCG with fp64
reliable updates (reading R8: update threshold tol_in = 0.1, at most 30 updates) for
every member of the 512-system batch workload (2-D 5-/9-point anisotropic Laplacians,
side uniform in [32, 512], eps log-uniform in [1e-3, 1]; member i has x* = xstar(n_i, i),
b = A x*, x0 = 0, tol 1e-8, at most 20000 inner iterations).  Calls only oracle/ and the
input generators:

    python tests/golden/make_batch_ru_iterations.py [--procs P]

The GPU test of the full-size fp32 batch reads the stored counts; nothing here is
produced by the CUDA path.
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "batch512_ru_oracle.json")
COUNT, SEED, TOL, TOL_IN, MAXIT, MAX_UPDATES = 512, 0, 1e-8, 0.1, 20000, 30


def member(i):
    import cgproblems as gen
    import oracle
    side, pts, eps = gen.batch_members(COUNT, SEED)[i]
    A = gen.lap2d(side, pts, eps)
    b = oracle.spmv(A, gen.xstar(A.n, i))
    t0 = time.time()
    s = oracle.pcg_ru(A, b, tol=TOL, tol_in=TOL_IN, maxit=MAXIT, max_updates=MAX_UPDATES, precond=1)
    return i, {"side": side, "points": pts, "eps": eps, "n": A.n, "nnz": A.nnz, "status": s.status,
               "iters": s.iters, "updates": s.restarts, "relres_true": s.relres_true,
               "oracle_s": round(time.time() - t0, 2)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    import cgproblems as gen
    params = gen.batch_members(COUNT, SEED)
    order = sorted(range(COUNT), key=lambda i: -params[i][0])   # largest first
    out = {}
    with mp.get_context("spawn").Pool(args.procs) as pool:
        for i, rec in pool.imap_unordered(member, order):
            out[i] = rec
            if len(out) % 32 == 0:
                print(f"{len(out)}/{COUNT}", flush=True)
    data = {"count": COUNT, "seed": SEED, "tol": TOL, "tol_in": TOL_IN, "maxit": MAXIT,
            "max_updates": MAX_UPDATES, "precond": "jacobi", "precision": "fp32 + fp64 reliable updates",
            "members": [out[i] for i in range(COUNT)]}
    with open(OUT + ".tmp", "w") as f:
        json.dump(data, f, indent=0)
    os.replace(OUT + ".tmp", OUT)
    tot = sum(m["n"] * m["iters"] for m in data["members"])
    print("sum n*iters", tot, "sum oracle s", sum(m["oracle_s"] for m in data["members"]))


if __name__ == "__main__":
    main()
