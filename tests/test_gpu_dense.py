"""GPU parity of the dense-cost path against the FP64 oracle, through the C ABI.

Tolerances: marginal L1 <= 1e-6, relative transport cost <= 1e-6;
the FP64 path is held to ~1e-12 on single sweeps. Inputs are seeded and come
from workloads/ or the oracle, never from the CUDA path."""
import math

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


def near_feasible(seed, n, m, gamma, C64):
    """u, v with sum P = 1 and c(P) = c (oracle column fix), r, c Dirichlet."""
    rng = np.random.default_rng(seed)
    r = rng.dirichlet(np.ones(n)) * 0.999 + 0.001 / n
    c = rng.dirichlet(np.ones(m)) * 0.999 + 0.001 / m
    u = np.log(r) + rng.normal(0, 0.3, n) + 5.0 * gamma / 4096
    v = np.log(c) - O.lse_c(u[:, None] - gamma * C64)
    return u, v, r, c


SIZES = [(1, 1), (7, 5), (31, 129), (128, 128), (300, 517), (784, 784), (1000, 1024)]


def make_dense(seed, n, m, f32):
    rng = np.random.default_rng(seed)
    C = rng.uniform(0, 1, size=(n, m))
    if f32:
        C = C.astype(np.float32)
    return C


@pytest.mark.parametrize("n,m", SIZES)
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_marginals(H, n, m, prec):
    from paper_2504_02067_gb300 import Problem
    f32 = prec == "mixed"
    C = make_dense(n * 7 + m, n, m, f32)
    gamma = float(np.float32(2.0 ** 10)) if f32 else 2.0 ** 10
    C64 = C.astype(np.float64)
    u, v, _, _ = near_feasible(n + m, n, m, gamma, C64)
    prob = Problem(t(C, torch.float32 if f32 else torch.float64), precision=prec)
    r, c, lr, lc, tot = H.marginals(prob, t(u), t(v), gamma)
    P = O.plan(u, v, gamma, C64)
    rr, cr = O.row_sum(P), O.col_sum(P)
    er = np.abs(r.cpu().numpy() - rr).sum()
    ec = np.abs(c.cpu().numpy() - cr).sum()
    tol = 1e-6 if f32 else 1e-12
    assert er <= tol and ec <= tol, (er, ec)
    np.testing.assert_allclose(lr.cpu().numpy(), np.log(rr), atol=50 * tol)
    assert abs(tot.item() - P.sum()) <= tol


@pytest.mark.parametrize("n,m", [(7, 5), (128, 128), (300, 517), (1000, 1024)])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_hvp_and_null_vector(H, n, m, prec):
    from paper_2504_02067_gb300 import Problem
    f32 = prec == "mixed"
    C = make_dense(3 * n + m, n, m, f32)
    C64 = C.astype(np.float64)
    gamma = float(np.float32(2.0 ** 12)) if f32 else 2.0 ** 12
    u, v, _, _ = near_feasible(n * m, n, m, gamma, C64)
    rng = np.random.default_rng(5)
    du, dv = rng.normal(size=n), rng.normal(size=m)
    prob = Problem(t(C, torch.float32 if f32 else torch.float64), precision=prec)
    tol = 1e-6 if f32 else 1e-12
    for s in (1.0, math.sqrt(0.75)):
        ou, ov, r, c = H.hvp(prob, t(u), t(v), gamma, s, t(du), t(dv))
        ru, rv, rr, cr = O.hvp(u, v, gamma, C64, du, dv, s)
        ref = np.concatenate([ru, rv])
        got = np.concatenate([ou.cpu().numpy(), ov.cpu().numpy()])
        assert np.abs(got - ref).sum() <= tol * np.abs(ref).sum(), np.abs(got - ref).sum()
        assert np.abs(r.cpu().numpy() - rr).sum() <= tol
    # K1: the Hessian (s = 1) annihilates (1, -1)  (Sec. 2.1 footnote)
    ou, ov, r, c = H.hvp(prob, t(u), t(v), gamma, 1.0, t(np.ones(n)), t(-np.ones(m)))
    assert (ou.abs().sum() + ov.abs().sum()).item() <= 2 * tol


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_newton_solve_matches_oracle(H, prec):
    """Alg. 2 on the GPU vs the oracle at the same (u, v): same rho sequence end,
    CG iteration count within one, direction within tolerance."""
    from paper_2504_02067_gb300 import Problem
    f32 = prec == "mixed"
    n = m = 256
    rng = np.random.default_rng(11)
    C = rng.uniform(0, 1, size=(n, m))
    if f32:
        C = C.astype(np.float32)
    C64 = C.astype(np.float64)
    gamma = 64.0
    u, v, r, c = near_feasible(12, n, m, gamma, C64)
    P = O.plan(u, v, gamma, C64)
    rP = O.row_sum(P)
    rt = rP * (1 + 0.02 * rng.normal(size=n))
    rt /= rt.sum()
    gu = rP - rt
    gl1 = np.abs(gu).sum()
    eta = max(gl1, 0.8 * 1e-4 / gl1)
    ref = O.newton_solve(P, gu, gl1, eta, 0.0)
    prob = Problem(t(C, torch.float32 if f32 else torch.float64), precision=prec)
    du, dv, rho, it = H.newton_solve(prob, t(u), t(v), gamma, t(rt), eta, 0.0)
    du = du.cpu().numpy()
    assert rho == pytest.approx(ref.rho)
    assert abs(it - ref.cg_iters) <= 1 + ref.cg_solves
    tol = 1e-5 if f32 else 1e-9
    # Compare modulo the gauge direction 1: F_r(rho) 1 = (1 - rho) r(P), so the
    # CG solution is most sensitive along 1, and (k 1, -k 1) leaves P unchanged.
    # the library returns d_u modulo the gauge: <r(P), d_u> = 0
    ref_du = ref.d_u - (rP @ ref.d_u) / rP.sum()
    diff = du - ref_du
    kappa = diff.mean()
    assert np.abs(diff - kappa).sum() <= tol * np.abs(ref_du).sum()
    assert abs(kappa) <= (1e-4 if f32 else 1e-9) * np.abs(ref_du).mean()
    np.testing.assert_allclose(dv.cpu().numpy() + kappa, -(P.T @ ref_du) / O.col_sum(P),
                               atol=tol * np.abs(ref_du).max())
    # the forcing test of Alg. 2 holds for the GPU direction, checked in FP64
    assert np.abs(O.F_r_apply(P, 1.0, du) + gu).sum() <= eta * gl1 * (1 + 1e-6)


def test_solve_small_fp64_matches_oracle(H):
    from paper_2504_02067_gb300 import Problem, default_params
    rng = np.random.default_rng(21)
    n, m = 60, 50
    C = rng.uniform(0, 1, size=(n, m))
    r, c = rng.dirichlet(np.ones(n)), rng.dirichlet(np.ones(m))
    ref = O.mdot(C, r, c, gamma_i=16.0, gamma_f=1024.0, tol_final=1e-9)
    prob = Problem(t(C), t(r), t(c))
    u, v, st = H.solve(prob, default_params(gamma_i=16.0, gamma_f=1024.0, tol_final=1e-9))
    u, v = u.cpu().numpy(), v.cpu().numpy()
    assert O.marginal_l1_error(u, v, 1024.0, C, r, c) <= 1e-9
    assert st["marg_err_l1"] <= 1e-9
    c_gpu = O.transport_cost(u, v, 1024.0, C)
    c_ref = O.transport_cost(ref.u, ref.v, 1024.0, C)
    assert abs(c_gpu - c_ref) <= 1e-6 * c_ref
    assert st["stages"] == ref.stages


@pytest.mark.parametrize("seed", [0, 1])
def test_solve_grid784_fp64(H, seed):
    """28 x 28 grid, float64 cost, gamma_f = 2^12, to marginal L1 <= 1e-6 (oracle-checked)."""
    from paper_2504_02067_gb300 import Problem, default_params
    p = W.grid_problem_784(seed)
    prob = Problem(t(p["C"]), t(p["r"]), t(p["c"]))
    u, v, st = H.solve(prob, default_params(gamma_i=16.0, gamma_f=4096.0))
    u, v = u.cpu().numpy(), v.cpu().numpy()
    err = O.marginal_l1_error(u, v, 4096.0, p["C"], p["r"], p["c"])
    assert err <= 1e-6, err
    assert abs(st["marg_err_l1"] - err) <= 1e-9


@pytest.mark.parametrize("kind", ["sqeuclid", "l1"])
def test_solve_grid4096_mixed(H, kind):
    """64 x 64 grid, float32 cost in HBM, gamma_f = 2^14, mixed precision, to marginal
    L1 <= 1e-6 as evaluated by the FP64 oracle on the float32 cost."""
    from paper_2504_02067_gb300 import Problem, default_params
    p = W.grid_problem_4096(0, kind)
    prob = Problem(t(p["C"], torch.float32), t(p["r"]), t(p["c"]))
    u, v, st = H.solve(prob, default_params(gamma_i=16.0, gamma_f=16384.0))
    u, v = u.cpu().numpy(), v.cpu().numpy()
    g = float(np.float32(16384.0))
    err = O.marginal_l1_error(u, v, g, p["C"].astype(np.float64), p["r"], p["c"])
    assert err <= 1e-6, (err, st)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("kappa", [0.0, 700.0, -3.0e4, 2.0e5])
def test_marginals_large_potentials_gauge(H, prec, kappa):
    """Potentials of magnitude ~gamma from a zero-bin grid problem, shifted along the
    gauge direction (u + k, v - k), which leaves P unchanged (Sec. 2.1 footnote):
    the LSE sweeps must return the oracle's marginals of the unshifted point."""
    from paper_2504_02067_gb300 import Problem
    p = W.grid_problem_4096(3, "sqeuclid", side=32)
    C = p["C"] if prec == "mixed" else p["C"].astype(np.float64)
    C64 = C.astype(np.float64)
    gamma = 4096.0
    r, c = p["r"] * 0.999 + 0.001 / 1024, p["c"] * 0.999 + 0.001 / 1024
    u, v = O.sinkhorn_log(C64, r, c, gamma, tol=1e-30, max_iter=25)
    assert np.abs(u).max() > 100
    P = O.plan(u, v, gamma, C64)
    prob = Problem(t(C, torch.float32 if prec == "mixed" else torch.float64), precision=prec)
    rr, cc, lr, lc, tot = H.marginals(prob, t(u + kappa), t(v - kappa), gamma)
    tol = 1e-6 if prec == "mixed" else 1e-11
    assert np.abs(rr.cpu().numpy() - O.row_sum(P)).sum() <= tol
    assert np.abs(cc.cpu().numpy() - O.col_sum(P)).sum() <= tol
    assert abs(tot.item() - P.sum()) <= tol


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_grid4096_matches_oracle_trace(H, prec):
    """Full-size 64 x 64 grid workload against the oracle's recorded run
    (tests/golden/grid4096_oracle_trace.json, written by make_grid4096_oracle_trace.py
    from oracle/ only): the FP64 path reproduces the oracle's schedule and operation
    counts exactly; both paths reach marginal L1 <= 1e-6 and the oracle's transport
    cost to 1e-6 relative, all evaluated in FP64 by the oracle."""
    import json
    import os
    from paper_2504_02067_gb300 import Problem, default_params
    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                      "grid4096_oracle_trace.json")))["sqeuclid"]
    p = W.grid_problem_4096(0, "sqeuclid")
    C64 = p["C"].astype(np.float64)
    Cdev = t(C64) if prec == "fp64" else t(p["C"], torch.float32)
    prob = Problem(Cdev, t(p["r"]), t(p["c"]))
    u, v, st = H.solve(prob, default_params(gamma_i=16.0, gamma_f=16384.0))
    u, v = u.cpu().numpy(), v.cpu().numpy()
    if prec == "fp64":
        for k in ("stages", "newton_steps", "cg_iters", "ls_trials", "sinkhorn_iters"):
            assert st[k] == ref[k], (k, st[k], ref[k])
    else:
        assert st["stages"] == ref["stages"]
        assert abs(st["cg_iters"] - ref["cg_iters"]) <= 0.02 * ref["cg_iters"]
    assert O.marginal_l1_error(u, v, 16384.0, C64, p["r"], p["c"]) <= 1e-6
    cost = O.transport_cost(u, v, 16384.0, C64)
    assert abs(cost - ref["transport_cost"]) <= 1e-6 * ref["transport_cost"]


def test_graph_and_direct_programs_agree(monkeypatch):
    """Each stage of eot_solve (and each eot_newton_solve) is a device-controlled
    program: one CUDA graph with conditional nodes by default, or, with
    EOT_GRAPH=0, the same kernels in the same order launched directly with the
    host reading every loop flag. Both must give bit-identical Newton directions,
    potentials and counters, and the same kernel-launch count."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_02067_gb300 import Handle, Problem, default_params
    n, m = 600, 512
    rng = np.random.default_rng(41)
    C = rng.uniform(0, 1, size=(n, m)).astype(np.float32)
    C64 = C.astype(np.float64)
    gamma = 64.0
    u, v, r, c = near_feasible(42, n, m, gamma, C64)
    rP = O.row_sum(O.plan(u, v, gamma, C64))
    rt = rP * (1 + 0.02 * rng.normal(size=n))
    rt /= rt.sum()
    gl1 = np.abs(rP - rt).sum()
    eta = max(gl1, 0.8 * 1e-4 / gl1)
    out = {}
    for mode in ("", "0"):
        if mode:
            monkeypatch.setenv("EOT_GRAPH", mode)
        else:
            monkeypatch.delenv("EOT_GRAPH", raising=False)
        h = Handle(0, 64, 64)
        try:
            prob = Problem(t(C, torch.float32), r=t(r), c=t(c), precision="mixed")
            du, dv, rho, it = h.newton_solve(prob, t(u), t(v), gamma, t(rt), eta, 0.0)
            l0 = h.launches()
            uu, vv, st = h.solve(prob, default_params(gamma_i=16.0, gamma_f=1024.0, tol_final=1e-6))
            out[mode] = (du.cpu().numpy(), dv.cpu().numpy(), rho, it, uu.cpu().numpy(), vv.cpu().numpy(), st,
                         h.launches() - l0)
        finally:
            h.close()
    a, b = out[""], out["0"]
    assert a[2] == b[2] and a[3] == b[3]
    for k in (0, 1, 4, 5):
        assert np.array_equal(a[k], b[k]), k
    for key in ("stages", "newton_steps", "cg_iters", "cg_solves", "ls_trials", "sinkhorn_iters", "sweeps_total",
                "sweeps_cg", "sweeps_newton", "sweeps_linesearch", "sweeps_sinkhorn", "sweeps_stage",
                "marg_err_l1", "final_rho"):
        assert a[6][key] == b[6][key], key
    assert a[6]["marg_err_l1"] <= 1e-6
    assert a[7] == b[7] and a[7] > 0


def test_stage_records_match_oracle_and_schedule(H):
    """Per-stage records of eot_solve (Alg. 1's loop) against the oracle's mdot on
    the same FP64 problem: the same temperatures, tolerances, Newton steps and CG
    iterations per stage and the same delta_min (Eq. delta_k-ratio); and, from the
    records alone, AdjustSchedule's rule (Sec. 3.3: q <- min(2, q^2) above 0.95,
    sqrt(q) below 0.8) and gamma^(t+1) = min(q gamma^(t), gamma_f) (Alg. 1)."""
    from paper_2504_02067_gb300 import Problem, default_params
    rng = np.random.default_rng(23)
    n, m = 120, 100
    C = rng.uniform(0, 1, size=(n, m))
    r, c = rng.dirichlet(np.ones(n)), rng.dirichlet(np.ones(m))
    gi, gf = 16.0, 4096.0
    ref = O.mdot(C, r, c, gamma_i=gi, gamma_f=gf, tol_final=1e-8)
    prob = Problem(t(C), t(r), t(c))
    u, v, st = H.solve(prob, default_params(gamma_i=gi, gamma_f=gf, tol_final=1e-8))
    recs = st["stage_records"]
    assert len(recs) == st["stages"] == ref.stages == len(ref.records)
    for g, o in zip(recs, ref.records):
        assert g["gamma"] == o["gamma"]
        assert g["eps"] == pytest.approx(o["eps"], rel=1e-12)
        assert g["newton_steps"] == o["newton_steps"] and abs(g["ls_trials"] - o["ls_trials"]) <= 1
        assert abs(g["cg_iters"] - o["cg_iters"]) <= 2  # a CG stop moved by summation rounding
        if math.isinf(o["delta_min"]):
            assert math.isinf(g["delta_min"])
        else:
            # measured: up to 2e-4 relative in the last stages (FP64 summation order,
            # amplified by the conditioning at large gamma, and a CG stop moved by one)
            assert g["delta_min"] == pytest.approx(o["delta_min"], rel=1e-3), (g, o)
        assert g["q_next"] == o["q_next"]
    q = 2.0
    for k, g in enumerate(recs):
        d = g["delta_min"]
        q = min(2.0, q * q) if d > 0.95 else (math.sqrt(q) if d < 0.8 else q)
        assert g["q_next"] == q
        if k + 1 < len(recs):
            assert recs[k + 1]["gamma"] == min(q * g["gamma"], gf)
    assert recs[0]["gamma"] == gi and recs[-1]["gamma"] == gf
    assert sum(g["cg_iters"] for g in recs) == st["cg_iters"]
    assert sum(g["newton_steps"] for g in recs) == st["newton_steps"]
    # every sweep is in one stage except the final marginal evaluation (a row and a column LSE)
    assert sum(g["sweeps"] for g in recs) + 2 == st["sweeps_total"]
    assert st["sweeps_total"] == (st["sweeps_cg"] + st["sweeps_newton"] + st["sweeps_linesearch"]
                                  + st["sweeps_sinkhorn"] + st["sweeps_stage"] + 2)


# ---------------- the plain FP32 comparator (EOT_PREC_PLAIN_FP32) ----------------
# Plain FP32 rounds every potential to FP32 and forms t = fma(-gamma, C, a + b) in
# FP32 with no shift and no split (the comparator of the metric). Each P_ij then
# carries a relative error of about 2^-24 (|u_i| + |v_j| + |u_i + v_j| + |t_ij|)
# from the roundings plus 2^-22 from ex2.approx, so the stated tolerance is
#     ||out - ref||_1 <= 2^-20 (max|u| + max|v| + gamma max C) ||ref||_1,
# 16 times the first-order bound, with the FP32 sums' rounding far below it.

def plain_tol(u, v, gamma, C64):
    return 2.0 ** -20 * (np.abs(u).max() + np.abs(v).max() + gamma * C64.max())


@pytest.mark.parametrize("n,m", [(7, 5), (128, 128), (300, 517), (1000, 1024)])
def test_plain_fp32_marginals_and_hvp(H, n, m):
    from paper_2504_02067_gb300 import Problem
    C = make_dense(11 * n + m, n, m, True)
    C64 = C.astype(np.float64)
    gamma = float(np.float32(2.0 ** 8))
    u, v, _, _ = near_feasible(n + 3 * m, n, m, gamma, C64)
    prob = Problem(t(C, torch.float32), precision="plain_fp32")
    tol = plain_tol(u, v, gamma, C64)
    r, c, lr, lc, tot = H.marginals(prob, t(u), t(v), gamma)
    P = O.plan(u, v, gamma, C64)
    rr, cr = O.row_sum(P), O.col_sum(P)
    assert np.abs(r.cpu().numpy() - rr).sum() <= tol * rr.sum()
    assert np.abs(c.cpu().numpy() - cr).sum() <= tol * cr.sum()
    assert abs(tot.item() - P.sum()) <= tol * P.sum()
    rng = np.random.default_rng(9)
    du, dv = rng.normal(size=n), rng.normal(size=m)
    ou, ov, _, _ = H.hvp(prob, t(u), t(v), gamma, 0.9, t(du), t(dv))
    ru, rv, _, _ = O.hvp(u, v, gamma, C64, du, dv, 0.9)
    ref = np.concatenate([ru, rv])
    got = np.concatenate([ou.cpu().numpy(), ov.cpu().numpy()])
    scale = np.concatenate([rr * np.abs(du) + 0.9 * P @ np.abs(dv), 0.9 * P.T @ np.abs(du) + cr * np.abs(dv)])
    assert np.abs(got - ref).sum() <= tol * scale.sum()


def test_plain_fp32_solve_floor_on_the_grid_workload(H):
    """The plain FP32 comparator on the 64 x 64 grid workload (gamma 2^4 -> 2^14):
    at tol_final = 1e-6 it stops with a documented cap status (its FP32 exponent
    cannot resolve the marginals at gamma = 2^14: reading R20) and leaves its last
    iterate in (u, v) and the stage it stopped in in the stats; the FP64 oracle
    evaluates that iterate's marginal L1 error at that stage's temperature (the
    floor), which stays above 1e-6. At gamma_f = 2^8 (exponents 64 times
    smaller) and tol_final = 1e-4 the same path reaches its target as the oracle
    measures it, within the factor 2 its own FP32 evaluation of the stopping
    test allows."""
    from paper_2504_02067_gb300 import EotError, Problem, default_params
    p = W.grid_problem_4096(0, "sqeuclid")
    C64 = p["C"].astype(np.float64)
    prob = Problem(t(p["C"], torch.float32), t(p["r"]), t(p["c"]), precision="plain_fp32")
    g = float(np.float32(16384.0))
    u = torch.empty(4096, dtype=torch.float64, device=DEV)
    v = torch.empty(4096, dtype=torch.float64, device=DEV)
    with pytest.raises(EotError) as ex:
        H.eot_solve(prob, default_params(gamma_i=16.0, gamma_f=16384.0, tol_final=1e-6), u, v)
    assert ex.value.status in (3, 4, 5, 6, 7)  # CG_MAXITER, LINESEARCH, MAXSTAGES, MAXNEWTON, RANGE
    st = ex.value.stats  # the work done before the cap: the stage it stopped in
    assert st["stages"] >= 1 and np.isnan(st["marg_err_l1"])
    g_last = st["final_gamma"]
    assert g_last <= g
    floor = O.marginal_l1_error(u.cpu().numpy(), v.cpu().numpy(), g_last, C64, p["r"], p["c"])
    assert np.isfinite(floor) and floor > 1e-6
    st = H.eot_solve(prob, default_params(gamma_i=16.0, gamma_f=256.0, tol_final=1e-4), u, v).as_dict()
    err = O.marginal_l1_error(u.cpu().numpy(), v.cpu().numpy(), 256.0, C64, p["r"], p["c"])
    assert err <= 2e-4, (err, st["marg_err_l1"])


def test_cluster_and_ticketed_column_half_agree(monkeypatch):
    """The CG column half of FP32 dense costs runs as thread-block clusters whose
    CTAs combine their column sums in distributed shared memory; EOT_CG_CLUSTER=0
    selects the ticketed combine through global partials. Both take the same
    Alg. 2 / Alg. 1 path: the same rho and CG count (within one) for a Newton
    step whose row-block counts differ (600 x 512: R = 8 clustered, more
    ticketed), and on the 64 x 64 grid workload the same stages and potentials
    to rounding, both at marginal L1 <= 1e-6 as the oracle measures it."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_02067_gb300 import Handle, Problem, default_params
    n, m = 600, 512
    rng = np.random.default_rng(43)
    C = rng.uniform(0, 1, size=(n, m)).astype(np.float32)
    C64 = C.astype(np.float64)
    gamma = 64.0
    u, v, r, c = near_feasible(44, n, m, gamma, C64)
    rP = O.row_sum(O.plan(u, v, gamma, C64))
    rt = rP * (1 + 0.02 * rng.normal(size=n))
    rt /= rt.sum()
    gl1 = np.abs(rP - rt).sum()
    eta = max(gl1, 0.8 * 1e-4 / gl1)
    p = W.grid_problem_4096(0, "sqeuclid")
    g = float(np.float32(16384.0))
    out = {}
    for mode in ("8", "0"):
        monkeypatch.setenv("EOT_CG_CLUSTER", mode)
        h = Handle(0, 64, 64)
        try:
            prob = Problem(t(C, torch.float32), r=t(r), c=t(c), precision="mixed")
            du, dv, rho, it = h.newton_solve(prob, t(u), t(v), gamma, t(rt), eta, 0.0)
            gp = Problem(t(p["C"], torch.float32), t(p["r"]), t(p["c"]))
            uu, vv, st = h.solve(gp, default_params(gamma_i=16.0, gamma_f=16384.0))
            out[mode] = (du.cpu().numpy(), rho, it, uu.cpu().numpy(), vv.cpu().numpy(), st)
        finally:
            h.close()
    a, b = out["8"], out["0"]
    assert a[1] == b[1] and abs(a[2] - b[2]) <= 1
    d = a[0] - b[0]
    assert np.abs(d - d.mean()).sum() <= 1e-5 * np.abs(b[0]).sum()
    for k in (3, 4):
        e = a[k] - b[k]
        assert np.abs(e - e.mean()).max() <= 1e-9 * (1.0 + np.abs(b[k]).max()), k
    assert a[5]["stages"] == b[5]["stages"]
    assert abs(a[5]["cg_iters"] - b[5]["cg_iters"]) <= 0.01 * b[5]["cg_iters"]
    for x in (a, b):
        err = O.marginal_l1_error(x[3], x[4], g, p["C"].astype(np.float64), p["r"], p["c"])
        assert err <= 1e-6, err
