"""GPU parity of the point-cloud path (cost C_ij = s_C |x_i - y_j|^2 formed on the
fly, never stored) against the FP64 oracle, through the C ABI. Inputs are seeded
and come from workloads/ or the oracle."""
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


def cloud(seed, n, m, d):
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 1, size=(n, d)).astype(np.float32)
    Y = (rng.normal(0, 1, size=(m, d)) + 0.3).astype(np.float32)
    r = rng.dirichlet(np.ones(n)) * 0.999 + 0.001 / n
    c = rng.dirichlet(np.ones(m)) * 0.999 + 0.001 / m
    return X, Y, r / r.sum(), c / c.sum()


def gam(g, prec):
    return float(np.float32(g)) if prec != "fp64" else g


@pytest.mark.parametrize("n,m,d", [(1, 1, 2), (37, 53, 3), (300, 517, 2), (1000, 700, 3),
                                   (129, 300, 8), (200, 150, 64), (129, 300, 17), (300, 517, 33),
                                   (1000, 700, 64)])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_point_marginals(H, n, m, d, prec):
    from paper_2504_02067_gb300 import Problem
    X, Y, r, c = cloud(n * 3 + m + d, n, m, d)
    sC = O.sqeuclid_scale(X, Y)
    C64 = sC * O.sqeuclid(X, Y)
    g = gam(256.0, prec)
    u = np.log(r) + np.random.default_rng(1).normal(0, 0.3, n) + 10.0
    v = np.log(c) - O.lse_c(u[:, None] - g * C64)
    prob = Problem(X=t(X, torch.float32), Y=t(Y, torch.float32), precision=prec, cost_scale=sC)
    rr, cc, lr, lc, tot = H.marginals(prob, t(u), t(v), g)
    P = O.plan(u, v, g, C64)
    tol = 1e-6 if prec == "mixed" else 1e-11
    assert np.abs(rr.cpu().numpy() - O.row_sum(P)).sum() <= tol
    assert np.abs(cc.cpu().numpy() - O.col_sum(P)).sum() <= tol
    assert abs(tot.item() - P.sum()) <= tol


def test_library_cost_scale_equals_oracle(H):
    """With cost_scale <= 0 the library computes s_C = 1 / max |x_i - y_j|^2 itself;
    in FP64 the marginals then match the oracle's (own s_C) to 1e-11, which needs
    the two normalisations to agree to ~1e-13."""
    from paper_2504_02067_gb300 import Problem
    X, Y, r, c = cloud(7, 900, 1100, 3)
    sC = O.sqeuclid_scale(X, Y)
    C64 = sC * O.sqeuclid(X, Y)
    g = 1024.0
    u = np.log(r) + 5.0
    v = np.log(c) - O.lse_c(u[:, None] - g * C64)
    prob = Problem(X=t(X, torch.float32), Y=t(Y, torch.float32), precision="fp64", cost_scale=0.0)
    rr, cc, _, _, _ = H.marginals(prob, t(u), t(v), g)
    P = O.plan(u, v, g, C64)
    assert np.abs(rr.cpu().numpy() - O.row_sum(P)).sum() <= 1e-11
    assert np.abs(cc.cpu().numpy() - O.col_sum(P)).sum() <= 1e-11


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_point_hvp(H, prec):
    from paper_2504_02067_gb300 import Problem
    n, m, d = 400, 333, 3
    X, Y, r, c = cloud(11, n, m, d)
    sC = O.sqeuclid_scale(X, Y)
    C64 = sC * O.sqeuclid(X, Y)
    g = gam(512.0, prec)
    u = np.log(r) + 3.0
    v = np.log(c) - O.lse_c(u[:, None] - g * C64)
    rng = np.random.default_rng(3)
    du, dv = rng.normal(size=n), rng.normal(size=m)
    prob = Problem(X=t(X, torch.float32), Y=t(Y, torch.float32), precision=prec, cost_scale=sC)
    ou, ov, rr, cc = H.hvp(prob, t(u), t(v), g, 0.9, t(du), t(dv))
    ru, rv, _, _ = O.hvp(u, v, g, C64, du, dv, 0.9)
    ref = np.concatenate([ru, rv])
    got = np.concatenate([ou.cpu().numpy(), ov.cpu().numpy()])
    tol = 1e-6 if prec == "mixed" else 1e-11
    assert np.abs(got - ref).sum() <= tol * np.abs(ref).sum()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_point_newton_solve(H, prec):
    from paper_2504_02067_gb300 import Problem
    n, m, d = 256, 256, 2
    X, Y, r, c = cloud(21, n, m, d)
    sC = O.sqeuclid_scale(X, Y)
    C64 = sC * O.sqeuclid(X, Y)
    g = 64.0
    u = np.log(r) + 2.0
    v = np.log(c) - O.lse_c(u[:, None] - g * C64)
    P = O.plan(u, v, g, C64)
    rP = O.row_sum(P)
    rt = rP * (1 + 0.02 * np.random.default_rng(22).normal(size=n))
    rt /= rt.sum()
    gu = rP - rt
    gl1 = np.abs(gu).sum()
    eta = max(gl1, 0.8 * 1e-4 / gl1)
    ref = O.newton_solve(P, gu, gl1, eta, 0.0)
    prob = Problem(X=t(X, torch.float32), Y=t(Y, torch.float32), precision=prec, cost_scale=sC)
    du, dv, rho, it = H.newton_solve(prob, t(u), t(v), g, t(rt), eta, 0.0)
    du = du.cpu().numpy()
    assert rho == pytest.approx(ref.rho)
    diff = du - ref.d_u
    tol = 1e-5 if prec == "mixed" else 1e-9
    assert np.abs(diff - diff.mean()).sum() <= tol * np.abs(ref.d_u).sum()
    assert np.abs(O.F_r_apply(P, 1.0, du) + gu).sum() <= eta * gl1 * (1 + 1e-6)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_point_solve_uniform_square(H, prec):
    """Uniform points in the unit square with Dirichlet weights (the many-small-
    problems regime), gamma_f = 2^12, to marginal L1 <= 1e-6 (oracle-checked), and
    the transport cost within 1e-6 relative of the oracle's run of the same
    algorithm on the same temperature sequence (every gamma rounded to FP32 on the
    mixed path, reading G11 / R12), as the cost comparison of reading (c) asks."""
    from paper_2504_02067_gb300 import Problem, default_params
    p = W.uniform_points_problem(5, 700, 600)
    sC = O.sqeuclid_scale(p["X"], p["Y"])
    C64 = sC * O.sqeuclid(p["X"], p["Y"])
    prob = Problem(X=t(p["X"], torch.float32), Y=t(p["Y"], torch.float32), r=t(p["r"]),
                   c=t(p["c"]), precision=prec, cost_scale=sC)
    u, v, st = H.solve(prob, default_params(gamma_i=16.0, gamma_f=4096.0))
    u, v = u.cpu().numpy(), v.cpu().numpy()
    err = O.marginal_l1_error(u, v, 4096.0, C64, p["r"], p["c"])
    assert err <= 1e-6, (err, st)
    rg = (lambda g: float(np.float32(g))) if prec == "mixed" else None
    ref = O.mdot(C64, p["r"], p["c"], gamma_i=16.0, gamma_f=4096.0, tol_final=1e-6, round_gamma=rg)
    assert ref.ok
    cost_ref = O.transport_cost(ref.u, ref.v, 4096.0, C64)
    assert abs(O.transport_cost(u, v, 4096.0, C64) - cost_ref) <= 1e-6 * cost_ref
    assert st["stages"] == ref.stages


def test_point_marginals_n2pow20_sampled(H):
    """n = m = 2^20 RGB clouds (d = 3): one row and one column LSE sweep of the full
    problem; 256 sampled rows and columns compared with the oracle, which forms
    those rows and columns exactly in FP64."""
    from paper_2504_02067_gb300 import Problem
    p = W.colour_problem(0)
    X, Y = p["X"], p["Y"]
    n = X.shape[0]
    rng = np.random.default_rng(9)
    i_s = np.sort(rng.choice(n, 256, replace=False))
    sC = 1.0 / 3.0  # RGB cube: a fixed normalisation, passed to both sides
    g = float(np.float32(1024.0))
    u = np.full(n, -np.log(n))
    v = np.full(n, -np.log(n)) + rng.normal(0, 0.5, n)
    prob = Problem(X=t(X, torch.float32), Y=t(Y, torch.float32), precision="mixed", cost_scale=sC)
    rr, cc, lr, lc, _ = H.marginals(prob, t(u), t(v), g)
    lr = lr.cpu().numpy()
    lc = lc.cpu().numpy()
    ref_lr = np.empty(len(i_s))
    ref_lc = np.empty(len(i_s))
    for k in range(0, len(i_s), 16):  # 16 rows of 2^20 entries at a time
        rows = i_s[k:k + 16]
        Cr = sC * O.sqeuclid_rows(X, Y, rows)
        ref_lr[k:k + 16] = u[rows] + O.lse_r(v[None, :] - g * Cr)
        Cc = sC * O.sqeuclid_rows(Y, X, rows)
        ref_lc[k:k + 16] = v[rows] + O.lse_r(u[None, :] - g * Cc)
    # relative error of the marginal entries (log difference) below 1e-6
    assert np.abs(lr[i_s] - ref_lr).max() <= 1e-6
    assert np.abs(lc[i_s] - ref_lc).max() <= 1e-6


@pytest.mark.parametrize("d,shift", [(17, 0.0), (64, 0.0), (64, 1000.0)])
def test_point_tensor_core_path_matches_simt(H, d, shift, monkeypatch):
    """For d >= 17 the mixed path forms x.y on the tensor cores from exact 8-bit
    digit slices (levels summed exactly in FP32); EOT_TC=0 selects the SIMT
    compensated distance instead. Both must match the oracle within the mixed
    tolerance, and each other within twice that; also for clouds moved 1000 away
    from the origin (the kernels centre both sets on a common point)."""
    from paper_2504_02067_gb300 import Problem
    n, m = 700, 650
    X, Y, r, c = cloud(77 + d, n, m, d)
    # far from the origin relative to their extent (the expansion must not care)
    X, Y = (X + np.float32(shift)).astype(np.float32), (Y + np.float32(shift)).astype(np.float32)
    sC = O.sqeuclid_scale(X, Y)
    C64 = sC * O.sqeuclid(X, Y)
    g = gam(1024.0, "mixed")
    u = np.log(r) + np.random.default_rng(4).normal(0, 0.3, n) + 2.0
    v = np.log(c) - O.lse_c(u[:, None] - g * C64)
    P = O.plan(u, v, g, C64)
    out = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("EOT_TC", flag)
        prob = Problem(X=t(X, torch.float32), Y=t(Y, torch.float32), precision="mixed", cost_scale=sC)
        rr, cc, _, _, _ = H.marginals(prob, t(u), t(v), g)
        out[flag] = (rr.cpu().numpy(), cc.cpu().numpy())
        assert np.abs(out[flag][0] - O.row_sum(P)).sum() <= 1e-6
        assert np.abs(out[flag][1] - O.col_sum(P)).sum() <= 1e-6
    assert np.abs(out["1"][0] - out["0"][0]).sum() <= 2e-6


def test_tensor_core_sweeps_full_size_sampled(H):
    """The d = 64 workload at full size (n = m = 16384, 8-component mixtures, the
    tensor-core sweeps with grids of 128 x chunks): row and column LSE sweeps
    (eot_marginals) and both weighted sweeps of the Hessian-vector product
    (eot_hvp: r(P) du + P dv and P^T du + c(P) dv), on 256 sampled rows and 256
    sampled columns that the oracle forms exactly in FP64. The inputs are seeded
    and made like a solve's: from v around -log m, one row fix and one column fix
    (u, then v, such that every row, then every column, of P has mass near 1/n,
    from approximate LSEs of the expansion |x|^2 + |y|^2 - 2 x.y, used only to
    pick the inputs). Tolerances: log-marginal error <= 1e-6; HVP entries within
    1e-5 of the sum of the absolute terms."""
    from paper_2504_02067_gb300 import Problem
    p = W.gmm_problem_d64(0)
    X, Y = p["X"], p["Y"]
    n, m = X.shape[0], Y.shape[0]
    sC = O.sqeuclid_scale(X, Y)
    g = float(np.float32(1024.0))
    rng = np.random.default_rng(17)
    v = np.full(m, -np.log(m)) + rng.normal(0, 0.5, m)
    X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
    y2 = (Y64 * Y64).sum(1)
    u = np.empty(n)
    for a in range(0, n, 2048):
        xa = X64[a:a + 2048]
        D = np.maximum((xa * xa).sum(1)[:, None] + y2[None, :] - 2.0 * xa @ Y64.T, 0.0)
        u[a:a + 2048] = -np.log(n) - O.lse_r(v[None, :] - g * sC * D)
    x2 = (X64 * X64).sum(1)
    for b in range(0, m, 2048):
        yb = Y64[b:b + 2048]
        D = np.maximum((yb * yb).sum(1)[:, None] + x2[None, :] - 2.0 * yb @ X64.T, 0.0)
        v[b:b + 2048] = -np.log(m) - O.lse_r(u[None, :] - g * sC * D)
    du = rng.normal(size=n)
    dv = rng.normal(size=m)
    s = 0.9
    prob = Problem(X=t(X, torch.float32), Y=t(Y, torch.float32), precision="mixed", cost_scale=sC)
    _, _, lr, lc, _ = H.marginals(prob, t(u), t(v), g)
    ou, ov, rr, cc = H.hvp(prob, t(u), t(v), g, s, t(du), t(dv))
    lr, lc, ou, ov = (x.cpu().numpy() for x in (lr, lc, ou, ov))
    rows = np.sort(rng.choice(n, 256, replace=False))
    cols = np.sort(rng.choice(m, 256, replace=False))
    for k in range(0, 256, 16):
        ri = rows[k:k + 16]
        Cr = sC * O.sqeuclid_rows(X, Y, ri)
        Pr = np.exp(u[ri, None] + v[None, :] - g * Cr)
        assert np.abs(lr[ri] - (u[ri] + O.lse_r(v[None, :] - g * Cr))).max() <= 1e-6
        ref = Pr.sum(1) * du[ri] + s * Pr @ dv
        scale = Pr.sum(1) * np.abs(du[ri]) + s * Pr @ np.abs(dv)
        assert np.all(np.abs(ou[ri] - ref) <= 1e-5 * scale)
        cj = cols[k:k + 16]
        Cc = sC * O.sqeuclid_rows(Y, X, cj)  # rows j of C^T
        Pc = np.exp(v[cj, None] + u[None, :] - g * Cc)
        assert np.abs(lc[cj] - (v[cj] + O.lse_r(u[None, :] - g * Cc))).max() <= 1e-6
        ref = s * Pc @ du + Pc.sum(1) * dv[cj]
        scale = s * Pc @ np.abs(du) + Pc.sum(1) * np.abs(dv[cj])
        assert np.all(np.abs(ov[cj] - ref) <= 1e-5 * scale)
