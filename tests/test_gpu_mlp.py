"""GPU parity of the learned FSAI factor: MLP inference (cg_fsai_load), the training
loss and gradient (cg_fsai_loss_grad) and Adam (cg_adam_step) against the fp64 oracle
(oracle/fsai.py) on the same bf16-rounded parameters and inputs, and a training run
that shows what the network gains over Jacobi.

Tolerances, element by element: a bound on |gpu - oracle| for every entry of G and
every parameter of the gradient, from a first-order error analysis of where the two
sides can differ (helper functions below).  The kernels sum in fp32 (tensor cores) where
the oracle sums in fp64, and form the features in fp32; both round the features, h1, dz2
and dz1 to bf16 (F4, F7).
  * An fp32 sum is within EPS_SUM (layers) or EPS_GRAD (a gradient summed over all
    entries) of its magnitude, the sum of the absolute values of its terms.
  * A bf16 rounding can come out one step (2^-8 of the value) apart only where the value
    lies within that error of a rounding boundary ("flippable"; found by rounding value
    - err and value + err); a ReLU or a backward mask only where the pre-activation lies
    within that error of zero.  In the forward pass a ReLU is continuous, so only the
    roundings count; in the backward pass a mask flip moves one term by its whole size.
  * The effect of every flippable rounding or mask is propagated to G and to each
    parameter with absolute values, as are the fp32 errors; the resulting changes of G
    are carried into dLoss/dG (Kaporin term and residual term) to first order.
  * A gradient sums the contributions of thousands of entries.  Each entry's error is
    bounded by b_e (worst case: its fp32 noise and every rounding or mask that may flip
    there); these errors have independent signs across entries (a flip goes either
    way), so they are combined by Hoeffding's inequality, 6 sqrt(sum_e b_e^2), exceeded
    with probability below 3e-8 per parameter.  Each entry of G keeps its worst case.
Most entries have nothing flippable and get a bound of about 2^-18 of their magnitude;
the loss is checked at 1e-5 relative, the norms of G and the gradient at 1e-3."""
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


EPS_SUM = 2.0 ** -18    # fp32 sum of a layer (32 or 64 terms), relative to its magnitude
EPS_FEAT = 2.0 ** -20   # a feature formed in fp32, relative to its value
EPS_GRAD = 2.0 ** -16   # fp32 sum of a gradient over all entries and CTA partials
STEP = 2.0 ** -8        # one bf16 step, relative to the value


def flippable(v, err):
    """Where two values within err of v can round to different bf16 values."""
    return fsai.bf16(v - err) != fsai.bf16(v + err)


def forward_analysis(A, params):
    """Oracle forward pass with the per-entry error bound of its output o and the pieces
    the backward bound needs."""
    Wr = [fsai.bf16(v) for v in fsai.unpack(params)]
    aW1, ab1, aW2, ab2, aW3, ab3 = (np.abs(v) for v in Wr)
    Fr = fsai.features(A)
    o, cache = fsai.mlp_forward(params, Fr, True)
    X, z1, h1, z2, h2 = cache[:5]
    aX, ah1, ah2 = np.abs(X), np.abs(h1), np.abs(h2)
    m1 = aX @ aW1.T + ab1                      # magnitude of z1
    m2 = ah1 @ aW2.T + ab2                     # magnitude of z2 (given h1)
    act1, act2 = z1 > 0, z2 > 0
    # flippable roundings and their size: features, then h1 (after a feature flip z1
    # moves by |W1| dX, which can in turn push h1 across a boundary)
    dX = flippable(Fr, EPS_FEAT * np.abs(Fr)) * STEP * aX
    nz1 = EPS_SUM * m1                          # fp32 noise of z1
    fz1 = dX @ aW1.T                            # z1 moved by feature flips
    fh1 = act1 * (fz1 + flippable(z1, nz1 + fz1) * STEP * ah1)   # h1 flips (+ carried)
    nz2 = EPS_SUM * m2 + (act1 * nz1) @ aW2.T   # noise of z2 (and h2: ReLU is 1-Lipschitz)
    fz2 = fh1 @ aW2.T
    no = EPS_SUM * (ah2 @ aW3 + ab3) + nz2 @ aW3 + 2.0 ** -23 * np.abs(o)
    fo = fz2 @ aW3
    return dict(o=o, X=X, z1=z1, h1=h1, z2=z2, h2=h2, W2=Wr[2], W3=Wr[4], m1=m1, m2=m2,
                dX=dX, ez1=nz1 + fz1, dh1=fh1, ez2=nz2 + fz2, nz2=nz2, fz2=fz2,
                eo=no + fo, no=no, fo=fo)


def g_bound(A, fw, part="eo"):
    """Bound on |G_gpu - G_oracle| per tril(A) entry: o / sqrt(A_jj) off the diagonal,
    softplus(o + c0) / sqrt(A_ii) on it (slope at most 1).  part: "eo" all, "no" the
    fp32 noise, "fo" the flips."""
    _, tci, _ = fsai.tril(A)
    return fw[part] / np.sqrt(fsai.diag(A)[tci])


def dgrad_bound(A, g, eg, R, lam):
    """dLoss/dG (oracle) and a first-order bound on its change when G moves by eg."""
    trp, tci, _ = fsai.tril(A)
    rows = np.repeat(np.arange(A.n), np.diff(trp))
    S_A = A.to_scipy().tocsr()
    aA = abs(S_A)
    G = fsai.g_matrix(A, g)
    aG, E = abs(G), fsai.g_matrix(A, eg)
    _, dG = fsai.kaporin(A, g)
    n = A.n
    GA = (G @ S_A).tocsr()
    quad = np.asarray(GA.multiply(G).sum(axis=1)).ravel()
    S = quad.mean()
    EA = (E @ aA).tocsr()
    dS = 2.0 / n * float(np.asarray(EA.multiply(aG).sum()))       # change of S
    ed = 2.0 / (n * S) * np.asarray(EA[rows, tci]).ravel() \
        + 2.0 / (n * S * S) * np.abs(np.asarray(GA[rows, tci]).ravel()) * dS
    on = rows == tci
    gd = g[on]
    ed[on] += 2.0 / n * eg[on] / (gd * gd)
    if R is not None:
        k = len(R)
        dR = np.zeros_like(ed)
        for r in np.atleast_2d(R):
            rn2 = float(r @ r)
            u = G @ r
            e = S_A @ (G.T @ u) - r
            Ae = S_A @ e
            GAe = G @ Ae
            du = E @ np.abs(r)
            dv = E.T @ np.abs(u) + aG.T @ du
            dAe = aA @ (aA @ dv)
            dGAe = E @ np.abs(Ae) + aG @ dAe
            dR += 2.0 / rn2 * (du[rows] * np.abs(Ae[tci]) + np.abs(u[rows]) * dAe[tci]
                               + dGAe[rows] * np.abs(r[tci]))
        dG = dG + lam * fsai.residual_term(A, g, R)[1]
        ed = ed + lam * dR / k
    return dG, ed


def grad_bound(A, params, R, lam):
    """Bound on |grad_gpu - grad_oracle| per parameter (module docstring)."""
    fw = forward_analysis(A, params)
    o = fw["o"]
    g, dgdo = fsai.g_from_output(A, o)
    trp, tci, _ = fsai.tril(A)
    rows = np.repeat(np.arange(A.n), np.diff(trp))
    sq = np.sqrt(fsai.diag(A)[rows])
    on = rows == tci
    parts = {}
    for part in ("no", "fo"):       # dout error from G's noise, from G's flips
        dG, edG = dgrad_bound(A, g, g_bound(A, fw, part), R, lam)
        parts[part] = edG * np.abs(dgdo) + np.abs(dG) * np.where(on, 0.25 * fw[part] / sq, 0.0)
    D = dG * dgdo
    aD = np.abs(D)
    nD = parts["no"] + 2.0 ** -23 * aD          # noise (fp32 store of dout included)
    fD = parts["fo"]
    X, z1, h1, z2, h2 = (fw[k] for k in ("X", "z1", "h1", "z2", "h2"))
    aX, ah1, ah2 = np.abs(X), np.abs(h1), np.abs(h2)
    aW2, aW3 = np.abs(fw["W2"]), np.abs(fw["W3"])
    act1, act2 = z1 > 0, z2 > 0
    # dz2 = dout W3 (second mask): noise n*, flips f*; rounded to bf16 for the products
    dz2 = np.outer(D, fw["W3"]) * act2
    mask2 = np.abs(z2) <= fw["ez2"]
    ndz2 = act2 * np.outer(nD, aW3)
    fdz2 = act2 * np.outer(fD, aW3) + mask2 * np.outer(aD + nD + fD, aW3)
    fdz2 = fdz2 + flippable(dz2, ndz2 + fdz2 + 2.0 ** -22 * np.abs(dz2)) * STEP * (np.abs(dz2) + ndz2 + fdz2)
    adz2r = np.abs(fsai.bf16(dz2))
    dh1 = fsai.bf16(dz2) @ fw["W2"]
    ndh1 = ndz2 @ aW2 + EPS_SUM * (adz2r @ aW2)
    fdh1 = fdz2 @ aW2
    dz1 = dh1 * act1
    mask1 = np.abs(z1) <= fw["ez1"]
    ndz1 = act1 * ndh1
    fdz1 = act1 * fdh1 + mask1 * (np.abs(dh1) + ndh1 + fdh1)
    fdz1 = fdz1 + flippable(dz1, ndz1 + fdz1 + 2.0 ** -22 * np.abs(dz1)) * STEP * (np.abs(dz1) + ndz1 + fdz1)
    adz1r = np.abs(fsai.bf16(dz1))
    fh1, fX = fw["dh1"], fw["dX"]
    nh2, fh2 = fw["nz2"], fw["fz2"]

    # per-entry bounds of a product term u_e a_e (weight gradients): |du| (|a| + |da|)
    # + |u| |da| <= sqrt(2 (du^2 (|a| + da)^2 + u^2 da^2)), summed over e by Hoeffding
    def hoeff_w(du, a, u, da):
        return 6.0 * np.sqrt(2.0 * ((du * du).T @ ((a + da) ** 2) + (u * u).T @ (da * da)))

    edz1, edz2 = ndz1 + fdz1, ndz2 + fdz2
    eh2, eD = nh2 + fh2, nD + fD
    tW1 = EPS_GRAD * (adz1r.T @ aX) + hoeff_w(edz1, aX, adz1r, fX)
    tb1 = EPS_GRAD * np.abs(dz1).sum(0) + 6.0 * np.sqrt((edz1 * edz1).sum(0))
    tW2 = EPS_GRAD * (adz2r.T @ ah1) + hoeff_w(edz2, ah1, adz2r, fh1)
    tb2 = EPS_GRAD * np.abs(dz2).sum(0) + 6.0 * np.sqrt((edz2 * edz2).sum(0))
    tW3 = EPS_GRAD * (ah2.T @ aD) + hoeff_w(eh2, aD[:, None], ah2, eD[:, None])[:, 0]
    tb3 = EPS_GRAD * aD.sum() + 6.0 * np.sqrt(np.sum(eD * eD))
    return fsai.pack(tW1, tb1, tW2, tb2, tW3, tb3)


def check_elementwise(got, ref, tol, what):
    err = np.abs(got - ref)
    bad = err > tol
    assert not np.any(bad), (what, int(np.argmax(err / (tol + 1e-300))),
                             float(np.max(err / (tol + 1e-300))), int(bad.sum()))


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
    check_elementwise(g, ref, g_bound(A, forward_analysis(A, bf16_params(p))), "G")


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
    # every parameter on its own against its own scale (the kernel's gradient is fp32:
    # its rounding, 2^-24 relative, sits well inside the 1e-5 bound)
    check_elementwise(gg, grad, grad_bound(A, bf16_params(p), R, 0.1), "gradient")
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
