"""GPU parity of eot_backward and of the autograd function built on it, through
the C ABI. Gradients of the EOT value (envelope theorem, Appx. A; s_C constant):
dC = P, dx_i = 2 s_C sum_j P_ij (x_i - y_j), dy_j = 2 s_C sum_i P_ij (y_j - x_i),
dr = u / gamma, dc = v / gamma, compared with the oracle's, which a CPU test pins
to finite differences of the oracle's own solves.

Tolerances: dX, dY are written in FP32, so one output rounding (2^-24) plus the
FP32 exponent and the compensated FP32 sums (about 1e-7 relative each) give a
relative error of a few 1e-7; the tests allow 1e-5 on the mixed path (below the
1e-4 gradient target) and 1e-6 on the FP64 path (output rounding only)."""
import numpy as np
import pytest

from oracle import eot_oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_02067_gb300 import Handle, build
    build()
    h = Handle(0, 64, 64)
    yield h
    h.close()


def t(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device=DEV, dtype=dtype)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def cloud(seed, n, m, d):
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 1, size=(n, d)).astype(np.float32)
    Y = (rng.normal(0, 1, size=(m, d)) + 0.2).astype(np.float32)
    r = rng.dirichlet(np.ones(n)) * 0.999 + 0.001 / n
    c = rng.dirichlet(np.ones(m)) * 0.999 + 0.001 / m
    return X, Y, r / r.sum(), c / c.sum()


def point_grads_gpu(H, prob, u, v, g, n, m, d):
    dX = torch.full((n, d), float("nan"), dtype=torch.float32, device=DEV)
    dY = torch.full((m, d), float("nan"), dtype=torch.float32, device=DEV)
    dr = torch.full((n,), float("nan"), dtype=torch.float64, device=DEV)
    dc = torch.full((m,), float("nan"), dtype=torch.float64, device=DEV)
    H.eot_backward(prob, t(u), t(v), g, 1.0, dX=dX, dY=dY, dr=dr, dc=dc)
    return dX.cpu().numpy(), dY.cpu().numpy(), dr.cpu().numpy(), dc.cpu().numpy()


@pytest.mark.parametrize("n,m,d", [(1, 1, 2), (300, 257, 3), (129, 700, 8), (250, 200, 16),
                                   (300, 280, 64)])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_point_backward_matches_oracle(H, n, m, d, prec):
    from paper_2504_02067_gb300 import Problem
    X, Y, r, c = cloud(5 * n + m + d, n, m, d)
    sC = O.sqeuclid_scale(X, Y)
    C64 = sC * O.sqeuclid(X, Y)
    g = 512.0
    u = np.log(r) + np.random.default_rng(2).normal(0, 0.3, n) + 7.0
    v = np.log(c) - O.lse_c(u[:, None] - g * C64)
    prob = Problem(X=t(X, torch.float32), Y=t(Y, torch.float32), precision=prec, cost_scale=sC)
    dX, dY, dr, dc = point_grads_gpu(H, prob, u, v, g, n, m, d)
    rX, rY = O.eot_grads_points(u, v, g, X, Y, sC)
    tol = 1e-5 if prec == "mixed" else 1e-6
    assert rel(dX, rX) <= tol
    assert rel(dY, rY) <= tol
    assert np.array_equal(dr, u / g) or rel(dr, u / g) <= 1e-15
    assert rel(dc, v / g) <= 1e-15


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_point_backward_is_gauge_invariant(H, prec):
    """(u + k, v - k) leaves P unchanged (Sec. 2.1), so dX and dY must not move
    beyond rounding, even for |k| far above the exponent range of FP32."""
    from paper_2504_02067_gb300 import Problem
    n, m, d = 400, 350, 3
    X, Y, r, c = cloud(31, n, m, d)
    sC = O.sqeuclid_scale(X, Y)
    C64 = sC * O.sqeuclid(X, Y)
    g = 1024.0
    u = np.log(r) + 1.0
    v = np.log(c) - O.lse_c(u[:, None] - g * C64)
    prob = Problem(X=t(X, torch.float32), Y=t(Y, torch.float32), precision=prec, cost_scale=sC)
    dX0, dY0, _, _ = point_grads_gpu(H, prob, u, v, g, n, m, d)
    rX, rY = O.eot_grads_points(u, v, g, X, Y, sC)
    for k in (-3.0e4, 2.5e5):
        dX, dY, _, _ = point_grads_gpu(H, prob, u + k, v - k, g, n, m, d)
        tol = 1e-5 if prec == "mixed" else 1e-6
        assert rel(dX, rX) <= tol and rel(dY, rY) <= tol
        assert rel(dX, dX0) <= tol and rel(dY, dY0) <= tol


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_dense_backward_matches_plan(H, prec):
    from paper_2504_02067_gb300 import Problem
    n, m = 333, 517
    p = W.random_dense_problem(3, n, m)
    C = p["C"].astype(np.float32) if prec == "mixed" else p["C"]
    C64 = C.astype(np.float64)
    g = 256.0
    u = np.log(p["r"]) + np.random.default_rng(4).normal(0, 0.3, n) - 40.0
    v = np.log(p["c"]) - O.lse_c(u[:, None] - g * C64)
    prob = Problem(t(C, torch.float32 if prec == "mixed" else torch.float64), precision=prec)
    dC = torch.full((n, m), float("nan"), dtype=torch.float32, device=DEV)
    H.eot_backward(prob, t(u), t(v), g, 2.0, dC=dC)
    P = O.plan(u, v, g, C64)
    got = dC.cpu().numpy().astype(np.float64)
    big = P > 1e-30
    tol = 1e-6 if prec == "mixed" else 2 ** -23
    assert np.abs(got[big] - 2.0 * P[big]).max() <= tol * 2.0 * P.max()
    assert (np.abs(got[big] / (2.0 * P[big]) - 1.0)).max() <= 1e-5


def _lse_expanded(A, B, w, K):
    """LSE_j(w_j - K |a_i - b_j|^2) for every row a_i, in row chunks."""
    A = A.astype(np.float64)
    B = B.astype(np.float64)
    bb = (B * B).sum(1)
    out = np.empty(A.shape[0])
    for k in range(0, A.shape[0], 1024):
        a = A[k:k + 1024]
        T = w[None, :] - K * ((a * a).sum(1)[:, None] + bb[None, :] - 2.0 * a @ B.T)
        mx = T.max(1)
        out[k:k + 1024] = mx + np.log(np.exp(T - mx[:, None]).sum(1))
    return out


def test_point_backward_full_size_sampled(H):
    """n = m = 16384 points in d = 64 (two 8-component Gaussian mixtures): one
    backward at the full size; 64 sampled rows of dX and 64 columns of dY are
    formed exactly by the oracle from those rows / columns alone."""
    from paper_2504_02067_gb300 import Problem
    p = W.gmm_problem_d64(0)
    X, Y = p["X"], p["Y"]
    n, d = X.shape
    rng = np.random.default_rng(12)
    sC = 1.0 / 2048.0  # a fixed normalisation, passed to both sides
    g = 1024.0
    # potentials with mass 1/n in every column: one half-step of Sinkhorn each
    # way (distances by the GEMM expansion: these only choose the inputs)
    u = -np.log(n) - _lse_expanded(X, Y, np.zeros(n), g * sC)
    v = -np.log(n) - _lse_expanded(Y, X, u, g * sC)
    prob = Problem(X=t(X, torch.float32), Y=t(Y, torch.float32), precision="mixed", cost_scale=sC)
    dX, dY, _, _ = point_grads_gpu(H, prob, u, v, g, n, n, d)
    rows = np.sort(rng.choice(n, 64, replace=False))
    X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
    for k in range(0, 64, 16):
        ii = rows[k:k + 16]
        Cr = sC * O.sqeuclid_rows(X, Y, ii)              # [16, m]
        Pr = np.exp(u[ii, None] + v[None, :] - g * Cr)
        ref = 2 * sC * (Pr.sum(1)[:, None] * X64[ii] - Pr @ Y64)
        assert rel(dX[ii], ref) <= 1e-5
        Cc = sC * O.sqeuclid_rows(Y, X, ii)              # columns ii: [16, n]
        Pc = np.exp(v[ii, None] + u[None, :] - g * Cc)
        ref = 2 * sC * (Pc.sum(1)[:, None] * Y64[ii] - Pc @ X64)
        assert rel(dY[ii], ref) <= 1e-5


def _fd_check(H, X, Y, r, c, sC, prec, gamma_f, tol_final, h):
    """Central difference of the GPU value along the gradient direction, with the
    FP32-rounded perturbation actually applied, against <grad, delta>."""
    from paper_2504_02067_gb300 import EOTFunction, default_params
    prm = default_params(gamma_f=gamma_f, tol_final=tol_final)
    Xt = t(X, torch.float32).requires_grad_(True)
    Yt = t(Y, torch.float32).requires_grad_(True)
    rt, ct = t(r).requires_grad_(True), t(c).requires_grad_(True)
    val, u, v = EOTFunction.apply(H, None, Xt, Yt, rt, ct, prm, prec, sC)
    val.backward()
    gX = Xt.grad.double().cpu().numpy()
    gY = Yt.grad.double().cpu().numpy()
    dirX = gX / np.abs(gX).max()
    dirY = gY / np.abs(gY).max()
    Xp, Xm = (X + h * dirX).astype(np.float32), (X - h * dirX).astype(np.float32)
    Yp, Ym = (Y + h * dirY).astype(np.float32), (Y - h * dirY).astype(np.float32)
    with torch.no_grad():
        Fp = EOTFunction.apply(H, None, t(Xp, torch.float32), t(Yp, torch.float32), t(r), t(c),
                               prm, prec, sC)[0].item()
        Fm = EOTFunction.apply(H, None, t(Xm, torch.float32), t(Ym, torch.float32), t(r), t(c),
                               prm, prec, sC)[0].item()
    dX = Xp.astype(np.float64) - Xm.astype(np.float64)
    dY = Yp.astype(np.float64) - Ym.astype(np.float64)
    pred = float((gX * dX).sum() + (gY * dY).sum())
    return val.item(), u, v, rt.grad.cpu().numpy(), ct.grad.cpu().numpy(), gX, gY, (Fp - Fm), pred


def test_eot_function_fd_and_oracle_fp64(H):
    """Uniform points in the unit square, gamma_f = 2^8, FP64 solved to marginal
    L1 1e-6: the autograd gradient equals the oracle's at the oracle's own
    (Sinkhorn to 1e-13) solution within 1e-4 relative, and so does the central
    difference of the GPU value along the gradient."""
    p = W.uniform_points_problem(8, 200, 180)
    X, Y, r, c = p["X"], p["Y"], p["r"], p["c"]
    sC = O.sqeuclid_scale(X, Y)
    val, u, v, gr, gc, gX, gY, fd, pred = _fd_check(H, X, Y, r, c, sC, "fp64", 256.0, 1e-6, 1e-3)
    C64 = sC * O.sqeuclid(X, Y)
    ru, rv = O.sinkhorn_log(C64, r, c, 256.0)
    rX, rY = O.eot_grads_points(ru, rv, 256.0, X, Y, sC)
    assert rel(gX, rX) <= 1e-4 and rel(gY, rY) <= 1e-4
    # the value is stationary in (u, v): second order in the 1e-6 marginal error
    assert abs(val - O.eot_value(ru, rv, 256.0, C64)) <= 1e-8 * abs(val)
    # dr, dc agree with u*/gamma, v*/gamma up to the gauge constant
    assert rel(gr - gr.mean(), (ru - ru.mean()) / 256.0) <= 1e-4
    assert rel(gc - gc.mean(), (rv - rv.mean()) / 256.0) <= 1e-4
    assert abs(fd - pred) <= 1e-4 * abs(pred)


def test_eot_function_fd_d64_mixed(H):
    """The config of the differentiation workload at n = m = 2048: 8-component
    Gaussian mixtures in d = 64, uniform weights, gamma_f = 2^10, mixed
    precision solved to marginal L1 1e-6; central difference of the value
    along the gradient within 1e-4 relative."""
    p = W.gmm_problem_d64(1, n=2048)
    X, Y, r, c = p["X"], p["Y"], p["r"], p["c"]
    sC = O.sqeuclid_scale(X, Y)
    val, u, v, gr, gc, gX, gY, fd, pred = _fd_check(H, X, Y, r, c, sC, "mixed", 1024.0, 1e-6, 1e-3)
    C64 = sC * O.sqeuclid(X, Y)
    err = O.marginal_l1_error(u.cpu().numpy(), v.cpu().numpy(), 1024.0, C64, r, c)
    assert err <= 1e-6
    rX, rY = O.eot_grads_points(u.cpu().numpy(), v.cpu().numpy(), 1024.0, X, Y, sC)
    assert rel(gX, rX) <= 1e-5 and rel(gY, rY) <= 1e-5
    assert abs(fd - pred) <= 1e-4 * abs(pred), (fd, pred)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_eot_value_is_the_dual_value_and_the_primal_at_the_optimum(H, prec):
    """eot_value returns (<r, u> + <c, v> - sum P + 1) / gamma on the device (Eq.
    sinkhorn-dual) at any (u, v): against the oracle's formula at the same point
    (relative 1e-12 in FP64, 1e-7 mixed: sum P carries the FP32 sweep's relative
    error, about 1e-7); and at a tight optimum it equals the primal value
    <P, C> - H(P) / gamma (strong duality, Sec. 2.1) to the same tolerances."""
    from paper_2504_02067_gb300 import Problem
    X, Y, r, c = cloud(91, 400, 350, 3)
    sC = O.sqeuclid_scale(X, Y)
    C64 = sC * O.sqeuclid(X, Y)
    g = 256.0 if prec == "fp64" else float(np.float32(256.0))
    prob = Problem(X=t(X, torch.float32), Y=t(Y, torch.float32), r=t(r), c=t(c), precision=prec, cost_scale=sC)
    rng = np.random.default_rng(5)
    u0 = np.log(r) + rng.normal(0, 0.2, 400) + 3.0
    v0 = np.log(c) - O.lse_c(u0[:, None] - g * C64)
    tol = 1e-12 if prec == "fp64" else 1e-7
    us, vs = O.sinkhorn_log(C64, r, c, g, tol=1e-14, max_iter=200000)
    for (u, v) in ((u0, v0), (us, vs)):
        val = torch.empty((), dtype=torch.float64, device=DEV)
        H.eot_value(prob, t(u), t(v), g, val)
        ref = (r @ u + c @ v - O.plan(u, v, g, C64).sum() + 1.0) / g
        assert abs(val.item() - ref) <= tol * abs(ref), (val.item(), ref)
    primal = O.primal_value(O.plan(us, vs, g, C64), C64, g)
    assert abs(val.item() - primal) <= max(tol, 1e-11) * abs(primal)


def test_backward_reads_the_gradient_scale_on_the_device(H):
    """grad_scale_dev (a device scalar, e.g. the incoming autograd gradient)
    multiplies every output as the host grad_scale does (a power of two, so both
    orders of the products are exact and the outputs bit-identical)."""
    from paper_2504_02067_gb300 import Problem
    X, Y, r, c = cloud(92, 300, 257, 3)
    sC = O.sqeuclid_scale(X, Y)
    C64 = sC * O.sqeuclid(X, Y)
    g = 512.0
    u = np.log(r) + 2.0
    v = np.log(c) - O.lse_c(u[:, None] - g * C64)
    prob = Problem(X=t(X, torch.float32), Y=t(Y, torch.float32), precision="fp64", cost_scale=sC)
    outs = []
    for host, dev in ((-0.5, None), (1.0, t(np.array(-0.5)))):
        dX = torch.empty(300, 3, dtype=torch.float32, device=DEV)
        dY = torch.empty(257, 3, dtype=torch.float32, device=DEV)
        dr = torch.empty(300, dtype=torch.float64, device=DEV)
        dc = torch.empty(257, dtype=torch.float64, device=DEV)
        H.eot_backward(prob, t(u), t(v), g, host, dX=dX, dY=dY, dr=dr, dc=dc, grad_scale_dev=dev)
        outs.append([x.cpu().numpy() for x in (dX, dY, dr, dc)])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
