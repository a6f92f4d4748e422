"""Training and evaluation driver of the learned FSAI preconditioner.

The host only orders the work: every step runs in libcg's kernels (features and
MLP forward/backward on the tensor cores, Kaporin and residual-history loss,
Adam).  Training data are the matrices themselves and residual vectors that
Jacobi-PCG produces on them (cg_solve stopped after a few iteration counts).

    python -m paper_2608_09647_gb300.fsai_train --train 2000 --test 200 --out fsai.json

trains on seeded rotated-anisotropy Q1 matrices and compares learned FSAI with
Jacobi and classic FSAI on held-out ones (iterations and time to 1e-8; fp32 inner
iterations with fp64 reliable updates by default).  ``--params FILE.npy`` skips
training and evaluates stored weights (fp32 values, or bf16 bit patterns as
uint16).  Not in the paper.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import (CG_MLP_HIDDEN, CG_MLP_INPUTS, CG_MLP_PARAMS, CG_OK, CG_NOT_CONVERGED, CG_PREC_FP32_IR,
               CG_PREC_FP32_RU, CG_PREC_FP64,
               CG_PRECOND_FSAI, CG_PRECOND_JACOBI, CGError, cg_adam_step, cg_create, cg_destroy,
               cg_fsai_classic, cg_fsai_load, cg_fsai_loss_grad, cg_get_solve_info, cg_last_error, cg_solve,
               cg_spmv)


def init_params(seed: int) -> np.ndarray:
    """He-normal hidden layers, zero biases and a zero output layer: the untrained
    network gives G = D^-1/2, Jacobi."""
    rng = np.random.default_rng(seed)
    w1 = rng.normal(0.0, math.sqrt(2.0 / CG_MLP_INPUTS), (CG_MLP_HIDDEN, CG_MLP_INPUTS))
    w2 = rng.normal(0.0, math.sqrt(2.0 / CG_MLP_HIDDEN), (CG_MLP_HIDDEN, CG_MLP_HIDDEN))
    z = np.zeros(CG_MLP_HIDDEN)
    p = np.concatenate([w1.ravel(), z, w2.ravel(), z, z, [0.0]]).astype(np.float32)
    assert p.size == CG_MLP_PARAMS
    return p


class Problem:
    """A matrix on the device with its handle, right-hand side and residual history."""

    def __init__(self, A, seed: int, snapshots=(2, 8, 32)):
        import torch
        self.A = A
        self.dev = tuple(torch.from_numpy(a).cuda() for a in (A.rowptr, A.colind, A.vals))
        self.h = cg_create(A.n, *self.dev)
        xs = torch.from_numpy(np.random.default_rng(seed).uniform(-1.0, 1.0, A.n)).cuda()
        self.b = torch.empty_like(xs)
        cg_spmv(self.h, xs, self.b)
        self.resid = self.residual_history(snapshots) if snapshots else None

    def residual_history(self, ks):
        """r = b - A x after k Jacobi-PCG iterations from x = 0, for each k."""
        import torch
        out = []
        for k in ks:
            x = torch.zeros_like(self.b)
            st, _, _ = cg_solve(self.h, self.b, x, 0.0, int(k), CG_PRECOND_JACOBI)
            if st not in (CG_OK, CG_NOT_CONVERGED):
                raise CGError(st, cg_last_error(self.h))
            ax = torch.empty_like(x)
            cg_spmv(self.h, x, ax)
            r = self.b - ax
            if float(torch.linalg.vector_norm(r)) > 0:
                out.append(r)
        return torch.stack(out) if out else None

    def fresh(self):
        """Another handle on the same device matrix and right-hand side (no factor)."""
        P = Problem.__new__(Problem)
        P.A, P.dev, P.b, P.resid = self.A, self.dev, self.b, self.resid
        P.h = cg_create(self.A.n, *self.dev)
        return P

    def close(self):
        cg_destroy(self.h)


def train(problems, epochs: int = 20, lr: float = 1e-3, lam: float = 0.1, seed: int = 0, log=None):
    """Adam on the summed per-matrix losses, one matrix per step, matrices in a
    seeded order each epoch.  Returns (fp32 parameter tensor, per-epoch mean loss)."""
    import torch
    params = torch.from_numpy(init_params(seed)).cuda()
    grad = torch.zeros_like(params)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    rng = np.random.default_rng(seed + 1)
    step = 0
    history = []
    for ep in range(epochs):
        losses = []
        for k in rng.permutation(len(problems)):
            P = problems[k]
            st, loss = cg_fsai_loss_grad(P.h, params, grad, P.resid, lam)
            if st != CG_OK:
                raise CGError(st, cg_last_error(P.h))
            step += 1
            st = cg_adam_step(params, grad, m, v, step, lr)
            if st != CG_OK:
                raise CGError(st, "cg_adam_step")
            losses.append(loss)
        history.append(float(np.mean(losses)))
        if log:
            log(f"epoch {ep + 1}/{epochs}: mean loss {history[-1]:.6f}")
    torch.cuda.synchronize()
    return params, history


def solve_stats(P, precond, tol=1e-8, maxit=100000, precision=CG_PREC_FP32_IR, reps=1):
    """(iterations, seconds of device time per solve) of one preconditioned solve."""
    import torch
    best = None
    for _ in range(reps):
        x = torch.zeros_like(P.b)
        st, it, rel = cg_solve(P.h, P.b, x, tol, maxit, precond, precision)
        if st != CG_OK:
            raise CGError(st, cg_last_error(P.h))
        info = cg_get_solve_info(P.h)
        t = info["kernel_ms"] / 1e3
        best = (it, t, rel, info["precond_used"]) if best is None or t < best[1] else best
    return best


def compare(problems, params, tol=1e-8, precision=CG_PREC_FP32_IR, reps=2):
    """Per matrix: Jacobi, classic FSAI and learned FSAI iterations, solve times
    (device time of the solve launch) and factor setup times (host wall time of
    cg_fsai_classic / cg_fsai_load, which synchronise), each factor on a handle of
    its own so that both setups include the pattern build."""
    rows = []
    params = params.detach().cpu().numpy() if hasattr(params, "detach") else params
    for P in problems:
        r = {"n": P.A.n, "name": P.A.name}
        r["jacobi_iters"], r["jacobi_s"], _, _ = solve_stats(P, CG_PRECOND_JACOBI, tol, precision=precision, reps=reps)
        # the plain fp64 Jacobi-PCG baseline (auto loop form)
        r["jacobi64_iters"], r["jacobi64_s"], _, _ = solve_stats(P, CG_PRECOND_JACOBI, tol, precision=CG_PREC_FP64,
                                                                 reps=reps)
        t0 = time.perf_counter()
        if cg_fsai_classic(P.h) != CG_OK:
            raise CGError(-1, cg_last_error(P.h))
        r["classic_setup_s"] = time.perf_counter() - t0
        r["classic_iters"], r["classic_s"], _, _ = solve_stats(P, CG_PRECOND_FSAI, tol, precision=precision, reps=reps)
        L = P.fresh()
        t0 = time.perf_counter()
        if cg_fsai_load(L.h, params) != CG_OK:
            raise CGError(-1, cg_last_error(L.h))
        r["learned_setup_s"] = time.perf_counter() - t0
        r["learned_iters"], r["learned_s"], _, used = solve_stats(L, CG_PRECOND_FSAI, tol, precision=precision,
                                                                  reps=reps)
        L.close()
        assert used == CG_PRECOND_FSAI
        rows.append(r)
    return rows


def summarize(rows):
    def q(vals):
        v = np.asarray(vals, dtype=np.float64)
        return {"median": float(np.median(v)), "q1": float(np.quantile(v, 0.25)), "q3": float(np.quantile(v, 0.75))}
    out = {}
    for a, b in (("learned", "jacobi"), ("learned", "classic"), ("classic", "jacobi")):
        out[f"{a}_vs_{b}_iters"] = q([r[f"{a}_iters"] / r[f"{b}_iters"] for r in rows])
        out[f"{a}_vs_{b}_time"] = q([r[f"{a}_s"] / r[f"{b}_s"] for r in rows])
    # against plain fp64 Jacobi-PCG, in time to tolerance (the iteration counts differ in kind
    # when the compared solve refines)
    out["learned_vs_jacobi64_time"] = q([r["learned_s"] / r["jacobi64_s"] for r in rows])
    out["learned_setup_plus_solve_vs_jacobi64_time"] = q([(r["learned_s"] + r["learned_setup_s"]) / r["jacobi64_s"]
                                                          for r in rows])
    return out


def load_params(path: str) -> np.ndarray:
    """fp32 parameters from an .npy file of fp32 values or of bf16 bit patterns (uint16)."""
    w = np.load(path)
    if w.dtype == np.uint16:
        w = (w.astype(np.uint32) << 16).view(np.float32)
    w = np.ascontiguousarray(w, dtype=np.float32).ravel()
    if w.size != CG_MLP_PARAMS:
        raise ValueError(f"{path}: {w.size} parameters, expected {CG_MLP_PARAMS}")
    return w


def q1_problem(index: int, seed: int, side_lo: int, side_hi: int, snapshots=(2, 8, 32)):
    import cgproblems as gen
    side, theta, eps, mseed = gen.q1_params(index, seed, side_lo, side_hi)
    A = gen.q1aniso(side, 1.5, theta, eps, mseed)
    return Problem(A, mseed, snapshots)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lam", type=float, default=0.1)
    ap.add_argument("--train-sides", type=int, nargs=2, default=(32, 96))
    ap.add_argument("--test-sides", type=int, nargs=2, default=(256, 1024))
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=None)
    ap.add_argument("--precision", choices=["fp32_ru", "fp32_ir", "fp64"], default="fp32_ru")
    ap.add_argument("--params", default=None, help="evaluate these weights instead of training")
    args = ap.parse_args()
    t0 = time.time()
    if args.params:
        params, hist = load_params(args.params), []
        t1 = t2 = time.time()
    else:
        tr = [q1_problem(i, args.seed, *args.train_sides) for i in range(args.train)]
        t1 = time.time()
        params, hist = train(tr, args.epochs, args.lr, args.lam, args.seed, log=print)
        t2 = time.time()
        for P in tr:
            P.close()
    rows = []
    prec = {"fp32_ru": CG_PREC_FP32_RU, "fp32_ir": CG_PREC_FP32_IR, "fp64": CG_PREC_FP64}[args.precision]
    for i in range(args.test):  # one held-out matrix at a time (they reach 10^6 rows)
        P = q1_problem(args.train + i, args.seed, *args.test_sides, snapshots=())
        rows += compare([P], params, precision=prec)
        P.close()
    t3 = time.time()
    summary = summarize(rows)
    # held-out matrices are q1_params indices train .. train + test - 1 either way
    res = {"train": args.train, "trained_here": not args.params, "test": args.test, "epochs": args.epochs,
           "lr": args.lr, "lam": args.lam, "precision": args.precision, "params": args.params,
           "train_sides": list(args.train_sides), "test_sides": list(args.test_sides), "loss_history": hist,
           "seconds": {"setup": t1 - t0, "train": t2 - t1, "evaluate": t3 - t2}, "summary": summary,
           "per_matrix": rows}
    print(json.dumps(summary, indent=1))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)
        if not args.params:
            np.save(args.out.rsplit(".", 1)[0] + "_params.npy", params.cpu().numpy())


if __name__ == "__main__":
    main()
