"""GPU parity of the learned FSAI factor: MLP inference (cg_fsai_load), the training
loss and gradient (cg_fsai_loss_grad) and Adam (cg_adam_step) against the fp64 oracle
(oracle/fsai.py) on the same bf16-rounded parameters and inputs, and a training run
that shows what the network gains over Jacobi.

Tolerances: the kernels sum in fp32 on the tensor cores where the oracle sums in fp64,
and both round h1, dz2 and dz1 to bf16, so a rare fp32/fp64 difference flips one
rounding: G and the gradient are compared norm-wise at 1e-3 relative (the bar the
method sets for the learned part), the loss at 1e-5 relative."""
import numpy as np
import pytest

import cgproblems as gen
import oracle
from oracle import fsai
from helpers import to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2608_09647_gb300 as cg  # noqa: E402
from paper_2608_09647_gb300 import fsai_train  # noqa: E402


def params_with_output(seed, scale):
    p = fsai.init_params(seed).astype(np.float64)
    rng = np.random.default_rng(seed + 100)
    p[-65:] = rng.normal(0.0, scale, 65)
    p[2048:2112] = rng.normal(0.0, 0.1, 64)        # b1
    p[6208:6272] = rng.normal(0.0, 0.1, 64)        # b2
    return p.astype(np.float32)


def bf16_params(p32):
    return fsai.bf16(np.asarray(p32, dtype=np.float64))


MATS = [("q1_30", lambda: gen.q1aniso(30, 1.5, 0.8, 0.03, 21)),
        ("q1_47", lambda: gen.q1aniso(47, 1.5, 2.2, 0.3, 22)),
        ("lap9_25", lambda: gen.lap2d(25, 9, 0.01))]


@pytest.mark.parametrize("name,make", MATS, ids=[m[0] for m in MATS])
def test_inference_matches_oracle(name, make):
    A = make()
    p = params_with_output(3, 0.05)
    h = cg.cg_create(A.n, *to_device(A))
    assert cg.cg_fsai_load(h, p) == cg.CG_OK, cg.cg_last_error(h)
    st, g, kind = cg.cg_fsai_get_factor(h)
    assert st == cg.CG_OK and kind == 2
    g = g.cpu().numpy()
    ref = fsai.learned(A, bf16_params(p), round_bf16=True)
    assert np.linalg.norm(g - ref) <= 1e-3 * np.linalg.norm(ref)
    assert np.max(np.abs(g - ref)) <= 1e-3 * np.max(np.abs(ref))


def test_zero_output_layer_gives_jacobi_on_the_gpu():
    A = gen.q1aniso(40, 1.5, 1.3, 0.02, 7)
    h = cg.cg_create(A.n, *to_device(A))
    assert cg.cg_fsai_load(h, fsai.init_params(9)) == cg.CG_OK
    g = cg.cg_fsai_get_factor(h)[1].cpu().numpy()
    trp, tci, _ = fsai.tril(A)
    rows = np.repeat(np.arange(A.n), np.diff(trp))
    jac = np.where(rows == tci, 1.0 / np.sqrt(fsai.diag(A))[rows], 0.0)
    assert np.max(np.abs(g - jac)) <= 1e-15 * np.max(jac)
    b = oracle.spmv(A, gen.xstar(A.n, 3))
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st, it, _ = cg.cg_solve(h, bd, x, 1e-9, 5000, cg.CG_PRECOND_FSAI)
    ref = oracle.pcg(A, b, tol=1e-9, maxit=5000, precond=1)
    assert st == cg.CG_OK and abs(it - ref.iters) <= max(3, 0.02 * ref.iters)


@pytest.mark.parametrize("with_resid", [False, True], ids=["kaporin", "kaporin+residuals"])
@pytest.mark.parametrize("name,make", MATS, ids=[m[0] for m in MATS])
def test_loss_and_gradient_match_oracle(name, make, with_resid):
    A = make()
    p = params_with_output(5, 0.05)
    h = cg.cg_create(A.n, *to_device(A))
    R = np.random.default_rng(8).normal(size=(3, A.n)) if with_resid else None
    pd = torch.from_numpy(p).cuda()
    gd = torch.full_like(pd, float("nan"))
    st, loss = cg.cg_fsai_loss_grad(h, pd, gd, None if R is None else torch.from_numpy(R).cuda(), 0.1)
    assert st == cg.CG_OK, cg.cg_last_error(h)
    L, grad = fsai.loss_and_grad(A, bf16_params(p), R, 0.1, round_bf16=True)
    assert abs(loss - L) <= 1e-5 * abs(L), (loss, L)
    gg = gd.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(gg))
    assert np.linalg.norm(gg - grad) <= 1e-3 * np.linalg.norm(grad), np.linalg.norm(gg - grad) / np.linalg.norm(grad)
    # each parameter block on its own, so a wrong block cannot hide behind a large one
    for a, b in ((0, 2048), (2048, 2112), (2112, 6208), (6208, 6272), (6272, 6336), (6336, 6337)):
        assert np.linalg.norm(gg[a:b] - grad[a:b]) <= 2e-3 * np.linalg.norm(grad[a:b]) + 1e-12, (a, b)
    # the same inputs give the same bits
    gd2 = torch.zeros_like(pd)
    st, loss2 = cg.cg_fsai_loss_grad(h, pd, gd2, None if R is None else torch.from_numpy(R).cuda(), 0.1)
    assert loss2 == loss and torch.equal(gd, gd2)


def test_adam_step_matches_oracle():
    rng = np.random.default_rng(2)
    n = 6337
    p = rng.normal(size=n).astype(np.float32)
    g = rng.normal(size=n).astype(np.float32)
    m = rng.normal(0, 0.1, n).astype(np.float32)
    v = rng.uniform(0, 0.1, n).astype(np.float32)
    pd, gd, md, vd = (torch.from_numpy(a.copy()).cuda() for a in (p, g, m, v))
    assert cg.cg_adam_step(pd, gd, md, vd, 7, lr=1e-3) == cg.CG_OK
    # the kernel works in fp32: give the oracle the same fp32 hyperparameters
    f = lambda x: float(np.float32(x))
    p1, m1, v1 = fsai.adam(p.astype(np.float64), g.astype(np.float64), m.astype(np.float64),
                           v.astype(np.float64), 7, lr=f(1e-3), b1=f(0.9), b2=f(0.999), eps=f(1e-8))
    assert np.allclose(pd.cpu().numpy(), p1, rtol=1e-6, atol=1e-6)
    assert np.allclose(md.cpu().numpy(), m1, rtol=1e-5, atol=1e-7)
    assert np.allclose(vd.cpu().numpy(), v1, rtol=1e-5, atol=1e-9)


def test_training_gains_over_jacobi():
    """Train on small rotated-anisotropy Q1 matrices, then on held-out larger ones the
    learned factor must need fewer iterations than Jacobi (median ratio < 0.8), and its
    loss must have dropped below the starting (Jacobi) loss."""
    train = [fsai_train.q1_problem(i, 5, 24, 48) for i in range(48)]
    params, hist = fsai_train.train(train, epochs=4, lr=3e-3, lam=0.1, seed=3)
    assert hist[-1] < hist[0]
    for P in train:
        P.close()
    test = [fsai_train.q1_problem(1000 + i, 5, 96, 160, snapshots=()) for i in range(6)]
    rows = fsai_train.compare(test, params, tol=1e-8, reps=1)
    ratios = [r["learned_iters"] / r["jacobi_iters"] for r in rows]
    assert np.median(ratios) < 0.8, rows
    for r in rows:
        assert r["classic_iters"] < r["jacobi_iters"]
