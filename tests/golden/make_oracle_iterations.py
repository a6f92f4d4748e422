"""Write tests/golden/oracle_iterations.json: the oracle's own iteration counts and
residuals on the benchmark workloads (full size).  Calls only oracle/ and the input
generators; run once per change of the oracle or the generators:

    python tests/golden/make_oracle_iterations.py [workload ...]

The GPU tests and the benchmark's CPU-baseline leg read the stored counts; nothing
here is produced by the CUDA path.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import cgproblems as gen  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(HERE, "oracle_iterations.json")

Q1_1024 = {"s": 1024, "sigma_a": 1.5, "theta": 0.7, "eps": 0.01, "seed": 3}
WEIGHTS = os.path.join(ROOT, "paper_2608_09647_gb300", "fsai_q1aniso_bf16.npy")

# name: (builder, kwargs, solver, precond, tol, maxit, tol_in); precond 2 = learned FSAI
CASES = {
    "poisson2d_64": ("lap2d", {"N": 64}, "pcg", 0, 1e-8, 1000, None),
    "poisson3d_256": ("lap3d7", {"N": 256}, "pcg", 1, 1e-8, 10000, None),
    "diffusion27_160_fp64": ("diff3d27", {"N": 160, "sigma": 1.0, "seed": 0}, "pcg", 1, 1e-10,
                             100000, None),
    "diffusion27_160": ("diff3d27", {"N": 160, "sigma": 1.0, "seed": 0}, "ir", 1, 1e-10, 100000,
                        1e-4),
    "diffusion27_160_ru": ("diff3d27", {"N": 160, "sigma": 1.0, "seed": 0}, "ru", 1, 1e-10, 100000,
                           0.1),
    "q1aniso_1024_jacobi_fp64": ("q1aniso", Q1_1024, "pcg", 1, 1e-8, 200000, None),
    "q1aniso_1024_learned": ("q1aniso", Q1_1024, "ir", 2, 1e-8, 200000, 1e-4),
    "q1aniso_1024_learned_ru": ("q1aniso", Q1_1024, "ru", 2, 1e-8, 200000, 0.1),
    "q1aniso_1024_learned_fp64": ("q1aniso", Q1_1024, "pcg", 2, 1e-8, 200000, None),
    "graph_spd_12m": ("graph_spd", {"n": 12_000_000, "dmax": 600, "seed": 0}, "pcg", 1, 1e-8, 20000, None),
}


def run(name):
    builder, kw, solver, precond, tol, maxit, tol_in = CASES[name]
    t0 = time.time()
    A = getattr(gen, builder)(**kw)
    xs = gen.xstar(A.n, 0)
    b = oracle.spmv(A, xs)
    t1 = time.time()
    if precond == 2:  # the learned FSAI factor of the committed weights, by the oracle's MLP
        from oracle import fsai
        bits = np.load(WEIGHTS)
        g = fsai.learned(A, (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64))
        if solver == "pcg":
            s = fsai.pcg(A, g, b, tol=tol, maxit=maxit)
        else:
            s = fsai.pcg_ir(A, g, b, tol=tol, tol_in=tol_in, maxit=maxit, carry=solver == "ru")
    elif solver == "pcg":
        s = oracle.pcg(A, b, tol=tol, maxit=maxit, precond=precond)
    elif solver == "ru":
        s = oracle.pcg_ru(A, b, tol=tol, tol_in=tol_in, maxit=maxit, precond=precond)
    else:
        s = oracle.pcg_ir(A, b, tol=tol, tol_in=tol_in, maxit=maxit, precond=precond)
    t2 = time.time()
    rec = {"n": A.n, "nnz": A.nnz, "solver": solver, "precond": precond, "tol": tol,
           "maxit": maxit, "tol_in": tol_in, "status": s.status, "iters": s.iters,
           "restarts": s.restarts, "relres_true": s.relres_true,
           "xerr_vs_xstar": float(np.linalg.norm(s.x - xs) / np.linalg.norm(xs)),
           "oracle_solve_s": round(t2 - t1, 1), "setup_s": round(t1 - t0, 1)}
    return rec


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        rec = run(name)
        data = json.load(open(OUT)) if os.path.exists(OUT) else {}
        data[name] = rec
        with open(OUT + ".tmp", "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(OUT + ".tmp", OUT)
        print(name, rec, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(CASES))
