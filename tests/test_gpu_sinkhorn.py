"""GPU parity of MDOT with Sinkhorn projections (the comparison method of Sec. 4,
eot_params.projector = EOT_PROJECT_SINKHORN) against the FP64 oracle's
mdot(..., projector="sinkhorn"), through the C ABI."""
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


@pytest.mark.parametrize("seed", [0, 1])
def test_sinkhorn_projector_fp64_grid784(H, seed):
    """28 x 28 grid, FP64 cost, gamma_f = 2^10: the same stages as the oracle and
    the same Sinkhorn iteration count up to one per stage (a stopping test that
    rounding moves across eps); both stop inside the projection tolerance, so the
    plans agree within 2 tol_final in L1 and the costs within 1e-6 relative."""
    from paper_2504_02067_gb300 import PROJECT_SINKHORN, Problem, default_params
    p = W.grid_problem_784(seed)
    gf = 1024.0
    ref = O.mdot(p["C"], p["r"], p["c"], gamma_i=16.0, gamma_f=gf, projector="sinkhorn")
    prob = Problem(t(p["C"]), t(p["r"]), t(p["c"]))
    u, v, st = H.solve(prob, default_params(gamma_i=16.0, gamma_f=gf, projector=PROJECT_SINKHORN))
    u, v = u.cpu().numpy(), v.cpu().numpy()
    assert st["stages"] == ref.stages and st["newton_steps"] == 0 and st["cg_iters"] == 0
    assert abs(st["sinkhorn_iters"] - ref.sinkhorn_iters) <= ref.stages
    err = O.marginal_l1_error(u, v, gf, p["C"], p["r"], p["c"])
    assert err <= 1e-6 and abs(st["marg_err_l1"] - err) <= 1e-9
    P, Pr = O.plan(u, v, gf, p["C"]), O.plan(ref.u, ref.v, gf, p["C"])
    assert np.abs(P - Pr).sum() <= 2e-6
    cr = (Pr * p["C"]).sum()
    assert abs((P * p["C"]).sum() - cr) <= 1e-6 * cr


def test_sinkhorn_projector_mixed_grid4096(H):
    """64 x 64 grid, FP32 cost, gamma_f = 2^12, mixed precision: MDOT-Sinkhorn
    reaches marginal L1 <= 1e-6 (as the oracle evaluates it) and the transport
    cost of the Newton-projected solve within 1e-6 relative (the same unique
    optimum of the regularised problem)."""
    from paper_2504_02067_gb300 import PROJECT_SINKHORN, Problem, default_params
    p = W.grid_problem_4096(0)
    gf = 4096.0
    prob = Problem(t(p["C"], torch.float32), t(p["r"]), t(p["c"]))
    u, v, st = H.solve(prob, default_params(gamma_i=16.0, gamma_f=gf, projector=PROJECT_SINKHORN))
    u1, v1, st1 = H.solve(prob, default_params(gamma_i=16.0, gamma_f=gf))
    C64 = p["C"].astype(np.float64)
    u, v, u1, v1 = (x.cpu().numpy() for x in (u, v, u1, v1))
    err = O.marginal_l1_error(u, v, gf, C64, p["r"], p["c"])
    assert err <= 1e-6, (err, st)
    assert st["newton_steps"] == 0 and st["sinkhorn_iters"] > st1["cg_iters"]
    c0, c1 = O.transport_cost(u, v, gf, C64), O.transport_cost(u1, v1, gf, C64)
    assert abs(c0 - c1) <= 1e-6 * c1


def test_projector_argument_checks(H):
    from paper_2504_02067_gb300 import (PROJECT_SINKHORN, EotError, Problem, default_params,
                                        solve_batched)
    p = W.uniform_points_problem(3, 20, 20)
    C = O.sqeuclid(p["X"], p["Y"])
    prob = Problem(t(C), t(p["r"]), t(p["c"]))
    with pytest.raises(EotError):
        H.solve(prob, default_params(projector=7))
    with pytest.raises(EotError):
        H.solve(prob, default_params(projector=PROJECT_SINKHORN, max_sinkhorn=-1))
    q = Problem(X=t(p["X"], torch.float32), Y=t(p["Y"], torch.float32), r=t(p["r"]), c=t(p["c"]),
                precision="mixed", cost_scale=1.0)
    with pytest.raises(EotError):
        solve_batched(H, [q], default_params(projector=PROJECT_SINKHORN))
