"""GPU parity of eot_solve_batched (many point-cloud problems in one persistent
launch) against the FP64 oracle, through the C ABI. Inputs: uniform points in
the unit square with Dirichlet(1) weights (the many-small-problems workload),
squared-Euclidean cost normalised per problem."""
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


def make(ps, prec, scale=True):
    from paper_2504_02067_gb300 import Problem
    out = []
    for p in ps:
        sC = O.sqeuclid_scale(p["X"], p["Y"]) if scale else 0.0
        out.append(Problem(X=t(p["X"], torch.float32), Y=t(p["Y"], torch.float32), r=t(p["r"]),
                           c=t(p["c"]), precision=prec, cost_scale=sC))
    return out


def small_batch():
    sizes = [(40, 55), (300, 260), (128, 128), (77, 300), (250, 90), (1, 5), (6, 1)]
    return [W.uniform_points_problem(100 + k, n, m) for k, (n, m) in enumerate(sizes)]


def test_batched_fp64_follows_oracle_step_by_step(H):
    """FP64: each problem of the batch takes the oracle's path (same stages,
    Newton steps and line-search trials; the same CG iteration count up to a
    stop moved by rounding: the kernels form (gamma s_C) D with one rounding, the
    oracle gamma (s_C D)). Both stop at the same projection tolerance on their own
    rounding paths, so the plans agree within 2 tol_final in L1 and the transport
    costs within 1e-6 relative. One-row / one-column members get the product
    plan's potentials (equal to the oracle's within 1e-12)."""
    from paper_2504_02067_gb300 import default_params, solve_batched
    ps = small_batch()
    probs = make(ps, "fp64")
    gf = 1024.0
    us, vs, st, stats = solve_batched(H, probs, default_params(gamma_i=16.0, gamma_f=gf))
    assert st == [0] * len(ps)
    for p, u, v, s in zip(ps, us, vs, stats):
        C64 = O.sqeuclid_scale(p["X"], p["Y"]) * O.sqeuclid(p["X"], p["Y"])
        ref = O.mdot(C64, p["r"], p["c"], gamma_i=16.0, gamma_f=gf)
        assert (s["stages"], s["newton_steps"], s["ls_trials"]) == \
            (ref.stages, ref.newton_steps, ref.ls_trials)
        assert abs(s["cg_iters"] - ref.cg_iters) <= 2 + 0.005 * ref.cg_iters
        uu, vv = u.cpu().numpy(), v.cpu().numpy()
        P = O.plan(uu, vv, gf, C64)
        Pr = O.plan(ref.u, ref.v, gf, C64)
        assert np.abs(P - Pr).sum() <= 2e-6
        cr = (Pr * C64).sum()
        assert abs((P * C64).sum() - cr) <= 1e-6 * cr + 1e-15
        if min(P.shape) == 1:
            assert np.abs(uu - ref.u).max() <= 1e-12 and np.abs(vv - ref.v).max() <= 1e-12
        assert O.marginal_l1_error(uu, vv, gf, C64, p["r"], p["c"]) <= 1e-6


def test_batched_mixed_reaches_tolerance(H):
    """Mixed precision: every problem reaches marginal L1 <= 1e-6 as the oracle
    measures it, its reported error (evaluated with FP32 plan entries, whose L1
    norms carry a floor of a few 1e-8 per entry error: 2.5e-7 allowed) agrees with
    the oracle's, and its transport cost is the oracle's (tight Sinkhorn at
    gamma_f) within 1e-6 relative."""
    from paper_2504_02067_gb300 import default_params, solve_batched
    ps = small_batch()
    probs = make(ps, "mixed")
    gf = float(np.float32(1024.0))
    us, vs, st, stats = solve_batched(H, probs, default_params(gamma_i=16.0, gamma_f=gf))
    assert st == [0] * len(ps)
    for p, u, v, s in zip(ps, us, vs, stats):
        C64 = O.sqeuclid_scale(p["X"], p["Y"]) * O.sqeuclid(p["X"], p["Y"])
        u, v = u.cpu().numpy(), v.cpu().numpy()
        err = O.marginal_l1_error(u, v, gf, C64, p["r"], p["c"])
        assert err <= 1e-6, (err, s)
        assert abs(s["marg_err_l1"] - err) <= 2.5e-7
        ru, rv = O.sinkhorn_log(C64, p["r"], p["c"], gf)
        cref = O.transport_cost(ru, rv, gf, C64)
        assert abs(O.transport_cost(u, v, gf, C64) - cref) <= 1e-6 * cref + 1e-12


def test_batched_matches_single_problem_solver(H):
    """Same problems through eot_solve one at a time (FP64): identical step
    counts; potentials agree modulo the gauge within 1e-9."""
    from paper_2504_02067_gb300 import default_params, solve_batched
    ps = small_batch()[:4]
    probs = make(ps, "fp64")
    prm = default_params(gamma_i=16.0, gamma_f=512.0)
    us, vs, st, stats = solve_batched(H, probs, prm)
    assert st == [0] * len(ps)
    for q, u, v, s in zip(probs, us, vs, stats):
        u1, v1, s1 = H.solve(q, default_params(gamma_i=16.0, gamma_f=512.0))
        assert (s["stages"], s["newton_steps"], s["cg_iters"], s["ls_trials"]) == \
            (s1["stages"], s1["newton_steps"], s1["cg_iters"], s1["ls_trials"])
        du = (u - u1).cpu().numpy()
        dv = (v - v1).cpu().numpy()
        k = (du.mean() - dv.mean()) / 2
        assert np.abs(du - k).max() <= 1e-9 and np.abs(dv + k).max() <= 1e-9


def test_batched_degenerate_and_failing_members(H):
    """d = 1 and d = 4, n = m = 1, a library-computed s_C, and one member whose r
    does not sum to 1: that member reports INVALID_ARG, the others still solve."""
    from paper_2504_02067_gb300 import Problem, default_params, solve_batched
    rng = np.random.default_rng(5)
    ps = [W.uniform_points_problem(7, 90, 70, d=1), W.uniform_points_problem(8, 60, 80, d=4),
          W.uniform_points_problem(9, 1, 1), W.uniform_points_problem(10, 50, 40)]
    bad = dict(ps[3])
    bad["r"] = bad["r"] * 1.01
    ps.append(bad)
    probs = make(ps[:2], "mixed") + make(ps[2:], "mixed", scale=False)
    gf = float(np.float32(512.0))
    us, vs, st, stats = solve_batched(H, probs, default_params(gamma_i=16.0, gamma_f=gf))
    assert st[:4] == [0, 0, 0, 0] and st[4] == 1
    for p, u, v in zip(ps[:4], us, vs):
        C64 = O.sqeuclid_scale(p["X"], p["Y"]) * O.sqeuclid(p["X"], p["Y"])
        assert O.marginal_l1_error(u.cpu().numpy(), v.cpu().numpy(), gf, C64, p["r"], p["c"]) <= 1e-6
    del rng


def test_batched_rejects_unsupported(H):
    from paper_2504_02067_gb300 import EotError, Problem, default_params, solve_batched
    p = W.uniform_points_problem(3, 20, 20)
    X5 = np.zeros((20, 5), np.float32)
    q = Problem(X=t(X5, torch.float32), Y=t(X5, torch.float32), r=t(p["r"]), c=t(p["c"]),
                precision="mixed", cost_scale=1.0)
    with pytest.raises(EotError):
        solve_batched(H, [q], default_params())
    dense = Problem(t(np.ones((20, 20)), torch.float32), t(p["r"]), t(p["c"]), precision="mixed")
    with pytest.raises(EotError):
        solve_batched(H, [dense], default_params())
    plain = make([p], "plain_fp32")
    with pytest.raises(EotError):
        solve_batched(H, plain, default_params())


def test_batched_many_problems_workload(H):
    """The batching workload: 256 problems, n = m uniform in [256, 4096], points
    uniform in the unit square, Dirichlet(1) weights, gamma_f = 2^12, mixed
    precision, one launch. Every problem must report success and marginal
    L1 <= 1e-6; for six problems (the three smallest, three of mid size) the
    oracle recomputes that error exactly."""
    from paper_2504_02067_gb300 import default_params, solve_batched
    sizes = W.batch_sizes(0)
    ps = [W.uniform_points_problem(1000 + k, int(n)) for k, n in enumerate(sizes)]
    probs = make(ps, "mixed", scale=False)
    gf = 4096.0
    us, vs, st, stats = solve_batched(H, probs, default_params(gamma_i=16.0, gamma_f=gf))
    assert st == [0] * len(ps)
    assert max(s["marg_err_l1"] for s in stats) <= 1e-6
    order = np.argsort(sizes)
    for k in list(order[:3]) + list(order[120:123]):
        p = ps[k]
        C64 = O.sqeuclid_scale(p["X"], p["Y"]) * O.sqeuclid(p["X"], p["Y"])
        err = O.marginal_l1_error(us[k].cpu().numpy(), vs[k].cpu().numpy(), gf, C64, p["r"], p["c"])
        assert err <= 1e-6, (k, err, stats[k])
    G, ro, groups = H.batch_last_config()
    assert G in (1, 2, 4, 8) and ro in (1, 2, 4) and groups >= 1
