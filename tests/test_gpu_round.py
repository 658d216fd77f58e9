"""GPU parity of eot_round (the Round step closing Alg. 1, Altschuler, Weed and
Rigollet 2017, Alg. 2, kept implicit) against the oracle's round_to_polytope on
the explicit plan, through the C ABI. Both sides evaluate in FP64, so the plans
agree to a few ulps of the largest entry and the costs to ~1e-13 relative."""
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


def near_feasible(seed, n, m, gamma, C64, zero_rows=0):
    """Potentials a few Sinkhorn half-steps from feasible: c(P) = c exactly (column
    fix), r(P) off by the perturbation; optional zero entries in r."""
    rng = np.random.default_rng(seed)
    r = rng.dirichlet(np.ones(n))
    c = rng.dirichlet(np.ones(m))
    if zero_rows:
        r[rng.choice(n, zero_rows, replace=False)] = 0.0
        r /= r.sum()
    u = np.log(np.maximum(r, 1e-200)) + rng.normal(0, 0.05, n)
    v = np.log(c) - O.lse_c(u[:, None] - gamma * C64)
    return u, v, r, c


def gpu_round(H, prob, u, v, gamma, n, m):
    uo = torch.empty(n, dtype=torch.float64, device=DEV)
    vo = torch.empty(m, dtype=torch.float64, device=DEV)
    ao = torch.empty(n, dtype=torch.float64, device=DEV)
    bo = torch.empty(m, dtype=torch.float64, device=DEV)
    cost, corr = H.eot_round(prob, t(u), t(v), gamma, uo, vo, ao, bo)
    return cost, corr, uo.cpu().numpy(), vo.cpu().numpy(), ao.cpu().numpy(), bo.cpu().numpy()


def implicit_plan(uo, vo, a, b, gamma, C64):
    P = O.plan(uo, vo, gamma, C64)
    s = np.abs(a).sum()
    return P + np.outer(a, b) / s if s > 0 else P


def check_against_oracle(cost, corr, uo, vo, a, b, u, v, r, c, gamma, C64):
    ref = O.round_to_polytope(O.plan(u, v, gamma, C64), r, c)
    G = implicit_plan(uo, vo, a, b, gamma, C64)
    assert np.abs(G - ref).max() <= 1e-13 * ref.max()
    cref = (ref * C64).sum()
    assert abs(cost - cref) <= 1e-12 * abs(cref) + 1e-300
    assert abs(cost - (G * C64).sum()) <= 1e-12 * abs(cref) + 1e-300
    # Round's output lies in U(r, c) (Altschuler et al., Lemma 7)
    assert np.abs(G.sum(1) - r).sum() <= 1e-14 * max(1, len(r) ** 0.5)
    assert np.abs(G.sum(0) - c).sum() <= 1e-14 * max(1, len(c) ** 0.5)
    return ref


@pytest.mark.parametrize("n,m", [(1, 1), (1, 7), (9, 1), (31, 129), (300, 517), (1000, 1024)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_round_dense_matches_oracle(H, n, m, prec):
    from paper_2504_02067_gb300 import Problem
    rng = np.random.default_rng(n * 7 + m)
    C = rng.uniform(0, 1, size=(n, m))
    if prec == "mixed":
        C = C.astype(np.float32)
    C64 = C.astype(np.float64)
    gamma = 64.0
    u, v, r, c = near_feasible(3, n, m, gamma, C64)
    prob = Problem(t(C, torch.float32 if prec == "mixed" else torch.float64), t(r), t(c),
                   precision="mixed" if prec == "mixed" else "fp64")
    cost, corr, uo, vo, a, b = gpu_round(H, prob, u, v, gamma, n, m)
    check_against_oracle(cost, corr, uo, vo, a, b, u, v, r, c, gamma, C64)
    x = np.minimum(r / O.plan(u, v, gamma, C64).sum(1), 1.0)
    assert np.allclose(uo, u + np.log(x), rtol=0, atol=1e-12)
    assert abs(corr - np.abs(a).sum()) <= 1e-15


@pytest.mark.parametrize("d", [3, 17])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_round_points_matches_oracle(H, d, prec):
    from paper_2504_02067_gb300 import Problem
    p = W.uniform_points_problem(40 + d, 257, 300, d=d)
    sC = O.sqeuclid_scale(p["X"], p["Y"])
    C64 = sC * O.sqeuclid(p["X"], p["Y"])
    gamma = 256.0
    u, v, r, c = near_feasible(d, 257, 300, gamma, C64)
    prob = Problem(X=t(p["X"], torch.float32), Y=t(p["Y"], torch.float32), r=t(r), c=t(c),
                   precision=prec, cost_scale=sC)
    cost, corr, uo, vo, a, b = gpu_round(H, prob, u, v, gamma, 257, 300)
    check_against_oracle(cost, corr, uo, vo, a, b, u, v, r, c, gamma, C64)


def test_round_zero_marginal_entries_and_feasible_input(H):
    """Zero entries of r give x_i = 0 (u_out = -inf, empty rows); a plan already in
    U(r, c) (separable cost C_ij = f_i + g_j, whose plan is r c^T at any gamma for
    the right potentials) rounds to itself with a = 0."""
    from paper_2504_02067_gb300 import Problem
    n, m, gamma = 50, 40, 32.0
    rng = np.random.default_rng(9)
    C = rng.uniform(0, 1, size=(n, m))
    u, v, r, c = near_feasible(5, n, m, gamma, C, zero_rows=4)
    prob = Problem(t(C), t(r), t(c), precision="fp64")
    cost, corr, uo, vo, a, b = gpu_round(H, prob, u, v, gamma, n, m)
    assert np.all(np.isneginf(uo[r == 0])) and np.all(np.isfinite(uo[r > 0]))
    check_against_oracle(cost, corr, uo, vo, a, b, u, v, r, c, gamma, C)
    f, g = rng.uniform(0, 1, n), rng.uniform(0, 1, m)
    Cs = f[:, None] + g[None, :]
    r2, c2 = rng.dirichlet(np.ones(n)), rng.dirichlet(np.ones(m))
    us, vs = np.log(r2) + gamma * f, np.log(c2) + gamma * g
    prob2 = Problem(t(Cs), t(r2), t(c2), precision="fp64")
    cost2, corr2, uo2, vo2, a2, b2 = gpu_round(H, prob2, us, vs, gamma, n, m)
    assert corr2 <= 1e-15
    assert abs(cost2 - (np.outer(r2, c2) * Cs).sum()) <= 1e-13


def test_round_after_solve_full_size(H):
    """The 64 x 64 grid workload solved to 1e-6 in mixed precision, then rounded:
    the rounded plan is in U(r, c), its cost is within the Altschuler bound
    (||P_round - P||_1 <= 2 marginal error, times max C = 1) of the unrounded
    cost, and it equals the oracle's Round on the explicit plan."""
    from paper_2504_02067_gb300 import Problem, default_params
    p = W.grid_problem_4096(0)
    C64 = p["C"].astype(np.float64)
    gf = 4096.0
    prob = Problem(t(p["C"], torch.float32), t(p["r"]), t(p["c"]))
    u, v, st = H.solve(prob, default_params(gamma_i=16.0, gamma_f=gf))
    u, v = u.cpu().numpy(), v.cpu().numpy()
    cost, corr, uo, vo, a, b = gpu_round(H, prob, u, v, gf, 4096, 4096)
    r, c = p["r"], p["c"]
    ref = O.round_to_polytope(O.plan(u, v, gf, C64), r, c)
    cref = (ref * C64).sum()
    assert abs(cost - cref) <= 1e-12 * cref
    c0 = O.transport_cost(u, v, gf, C64)
    err = O.marginal_l1_error(u, v, gf, C64, r, c)
    assert abs(cost - c0) <= 2 * err + 1e-15
    assert corr <= err + 1e-15
    rows = np.random.default_rng(0).choice(4096, 64, replace=False)
    G = O.plan(uo[rows], vo, gf, C64[rows]) + np.outer(a[rows], b) / np.abs(a).sum()
    assert np.abs(G - ref[rows]).max() <= 1e-13 * ref.max()
