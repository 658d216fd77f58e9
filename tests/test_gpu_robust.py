"""Failure handling of the dense path through the C ABI: invalid arguments and
parameters, marginals off the simplex, and caps forced tiny each return their
documented status (no abort, no fault), and the handle keeps working afterwards.
Degenerate shapes (one row, one column) return the potentials of r c^T, the
only plan in U(r, c) (Sec. 2.1), as the oracle does."""
import math

import numpy as np
import pytest

from oracle import eot_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
INVALID_ARG, CG_MAXITER, MAXSTAGES, MAXNEWTON = 1, 3, 5, 6


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_02067_gb300 import Handle, build
    build()
    h = Handle(0, 64, 64)
    yield h
    h.close()


def t(x, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device=DEV, dtype=dtype or torch.float64)


def problem(seed=23, n=120, m=100):
    rng = np.random.default_rng(seed)
    C = rng.uniform(0, 1, size=(n, m))
    return C, rng.dirichlet(np.ones(n)), rng.dirichlet(np.ones(m))


def status_of(fn):
    from paper_2504_02067_gb300 import EotError
    with pytest.raises(EotError) as e:
        fn()
    return e.value.status


def test_invalid_gamma_and_params(H):
    from paper_2504_02067_gb300 import Problem, default_params
    C, r, c = problem()
    prob = Problem(t(C), t(r), t(c))
    u, v = t(np.log(r)), t(np.log(c))
    for g in (0.0, -1.0, float("nan"), float("inf"), 2.0 ** 19):
        assert status_of(lambda: H.marginals(prob, u, v, g)) == INVALID_ARG
    for bad in (dict(w_r=0.6), dict(w_r=0.25), dict(p=0.5), dict(q1=1.0), dict(max_ls=0),
                dict(max_stages=0), dict(tol_final=0.0), dict(gamma_f=float("nan"))):
        assert status_of(lambda: H.solve(prob, default_params(**bad))) == INVALID_ARG, bad


def test_marginals_off_the_simplex(H):
    """r, c must be finite, non-negative and sum to 1 (the transport polytope of Sec. 2.1)."""
    from paper_2504_02067_gb300 import Problem, default_params
    C, r, c = problem()
    for rr, cc in ((2.0 * r, c), (r, c * (1 - 1e-3)), (np.where(np.arange(len(r)) == 3, -r[3], r) * 1.0, c)):
        rr = rr / rr.sum() if rr.min() < 0 else rr  # the negative case keeps sum 1
        prob = Problem(t(C), t(rr), t(cc))
        assert status_of(lambda: H.solve(prob, default_params())) == INVALID_ARG
    rn = r.copy()
    rn[5] = float("nan")
    prob = Problem(t(C), t(rn), t(c))
    assert status_of(lambda: H.solve(prob, default_params())) == INVALID_ARG


def test_caps_return_their_status_and_the_handle_recovers(H):
    """max_stages, max_newton and max_cg forced to 1 on a problem whose solve needs
    more (its first stage takes two Newton steps, later linear CG solves take
    many iterations); then the same handle solves the problem normally."""
    from paper_2504_02067_gb300 import Problem, default_params
    C, r, c = problem()
    prob = Problem(t(C), t(r), t(c))
    kw = dict(gamma_i=16.0, gamma_f=4096.0, tol_final=1e-8)
    assert status_of(lambda: H.solve(prob, default_params(max_stages=1, **kw))) == MAXSTAGES
    assert status_of(lambda: H.solve(prob, default_params(max_newton=1, **kw))) == MAXNEWTON
    assert status_of(lambda: H.solve(prob, default_params(max_cg=1, **kw))) == CG_MAXITER
    u, v, st = H.solve(prob, default_params(**kw))
    assert O.marginal_l1_error(u.cpu().numpy(), v.cpu().numpy(), 4096.0, C, r, c) <= 1e-8


def test_gamma_i_above_gamma_f_is_one_stage(H):
    """gamma^(1) = min(gamma_i, gamma_f) (Alg. 1): a single projection at gamma_f."""
    from paper_2504_02067_gb300 import Problem, default_params
    C, r, c = problem(seed=29, n=80, m=90)
    prob = Problem(t(C), t(r), t(c))
    u, v, st = H.solve(prob, default_params(gamma_i=256.0, gamma_f=64.0))
    assert st["stages"] == 1 and st["final_gamma"] == 64.0
    assert O.marginal_l1_error(u.cpu().numpy(), v.cpu().numpy(), 64.0, C, r, c) <= 1e-6


@pytest.mark.parametrize("shape", [(1, 37), (41, 1)])
def test_one_row_or_column_is_the_independence_coupling(H, shape):
    from paper_2504_02067_gb300 import Problem, default_params
    n, m = shape
    rng = np.random.default_rng(n + m)
    C = rng.uniform(0, 1, size=(n, m))
    r = rng.dirichlet(np.ones(n)) if n > 1 else np.ones(1)
    c = rng.dirichlet(np.ones(m)) if m > 1 else np.ones(1)
    prob = Problem(t(C), t(r), t(c))
    u, v, st = H.solve(prob, default_params(gamma_i=16.0, gamma_f=1024.0))
    ref = O.mdot(C, r, c, gamma_i=16.0, gamma_f=1024.0)
    np.testing.assert_allclose(u.cpu().numpy(), ref.u, rtol=0, atol=1e-12)
    np.testing.assert_allclose(v.cpu().numpy(), ref.v, rtol=0, atol=1e-12)
    P = O.plan(u.cpu().numpy(), v.cpu().numpy(), 1024.0, C)
    np.testing.assert_allclose(P, np.outer(r, c), rtol=1e-12, atol=1e-15)
    assert st["stages"] == 0 and math.isfinite(st["marg_err_l1"])


def test_wall_clock_budget_stops_the_solve(H):
    """eot_params.max_seconds: a budget that has run out before the first Newton
    step stops eot_solve with EOT_ERR_TIME_LIMIT, leaves the last iterate and the
    work done so far, and the handle solves normally afterwards."""
    from paper_2504_02067_gb300 import EotError, Problem, default_params
    rng = np.random.default_rng(3)
    n, m = 200, 150
    C = rng.uniform(0, 1, size=(n, m)).astype(np.float32)
    r, c = rng.dirichlet(np.ones(n)), rng.dirichlet(np.ones(m))
    prob = Problem(t(C, torch.float32), t(r), t(c))
    u = torch.empty(n, dtype=torch.float64, device=DEV)
    v = torch.empty(m, dtype=torch.float64, device=DEV)
    with pytest.raises(EotError) as ex:
        H.eot_solve(prob, default_params(gamma_f=4096.0, max_seconds=1e-9), u, v)
    assert ex.value.status == 11
    assert ex.value.stats["stages"] >= 1 and np.isnan(ex.value.stats["marg_err_l1"])
    assert torch.isfinite(u).all() and torch.isfinite(v).all()
    st = H.eot_solve(prob, default_params(gamma_f=4096.0, max_seconds=600.0), u, v).as_dict()
    assert st["marg_err_l1"] <= 1e-6
