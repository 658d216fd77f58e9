"""Integer outputs of the plan through the C ABI, compared bit-exactly with the
FP64 oracle on the same seeded inputs: the row argmax of P (lowest index on
ties) and the support counts #{j : P_ij > tau} (reading G12; the decisions are
taken on the FP64 exponent in a fixed order of rounded operations, Sec. 2.1
Eq. lagrangian-closed-form). Dense FP32 / FP64 costs and point clouds, ragged
sizes, forced ties, entries exactly on the threshold, and the full-size
workloads on sampled rows."""
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


def run_int(H, prob, u, v, gamma, log_tau):
    n = prob.n
    idx = torch.full((n,), -7, dtype=torch.int64, device=DEV)
    cnt = torch.full((n,), -7, dtype=torch.int64, device=DEV)
    tot = torch.full((1,), -7, dtype=torch.int64, device=DEV)
    H.eot_plan_argmax(prob, t(v), gamma, idx)
    H.eot_plan_support(prob, t(u), t(v), gamma, log_tau, cnt, tot)
    torch.cuda.synchronize()
    return idx.cpu().numpy(), cnt.cpu().numpy(), int(tot.item())


def dense_case(seed, n, m, f32, ties):
    rng = np.random.default_rng(seed)
    C = rng.uniform(0, 1, size=(n, m))
    if f32:
        C = C.astype(np.float32)
    u = rng.normal(0, 0.5, n) - math.log(n)
    v = rng.normal(0, 0.5, m) - math.log(m)
    if ties and m >= 4:
        # duplicated columns with equal v: exact ties wherever they hold the max
        C[:, m - 1] = C[:, 1]
        v[m - 1] = v[1]
        C[:, m // 2] = C[:, 0]
        v[m // 2] = v[0]
        # a row whose best entries are an exact tie
        C[0, :] = 1.0
        C[0, 2] = C[0, m - 2] = 0.0
        v[2] = v[m - 2] = 0.25
    return C, u, v


@pytest.mark.parametrize("n,m", [(1, 1), (7, 5), (31, 129), (300, 517), (1000, 1024)])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_dense_argmax_and_support_bit_exact(H, n, m, prec):
    from paper_2504_02067_gb300 import Problem
    f32 = prec == "mixed"
    C, u, v = dense_case(n * 31 + m, n, m, f32, ties=True)
    C64 = C.astype(np.float64)
    gamma = 64.0
    t_all = (u[:, None] + v[None, :]) - gamma * C64
    log_tau = float(np.quantile(t_all, 0.7)) if t_all.size > 1 else float(t_all.flat[0]) - 1.0
    prob = Problem(t(C, torch.float32 if f32 else torch.float64), precision=prec)
    idx, cnt, tot = run_int(H, prob, u, v, gamma, log_tau)
    ref_idx = O.plan_row_argmax(v, gamma, C64)
    ref_cnt = O.plan_support_counts(u, v, gamma, C64, log_tau)
    assert np.array_equal(idx, ref_idx)
    assert np.array_equal(cnt, ref_cnt)
    assert tot == int(ref_cnt.sum())
    if m >= 4 and n >= 1:
        assert idx[0] == 2  # exact tie between columns 2 and m - 2: the lower index


def test_dense_threshold_entry_is_excluded(H):
    """An entry lying exactly on the threshold (t_ij = log tau) is not counted
    (the test is strict), on both sides."""
    from paper_2504_02067_gb300 import Problem
    C, u, v = dense_case(5, 200, 300, True, ties=False)
    C64 = C.astype(np.float64)
    gamma = 128.0
    t_all = (u[:, None] + v[None, :]) - gamma * C64
    log_tau = float(t_all[17, 33])
    prob = Problem(t(C, torch.float32), precision="mixed")
    _, cnt, tot = run_int(H, prob, u, v, gamma, log_tau)
    ref = O.plan_support_counts(u, v, gamma, C64, log_tau)
    assert np.array_equal(cnt, ref)
    assert ref[17] == int((t_all[17] > log_tau).sum())


@pytest.mark.parametrize("n,m,d", [(1, 1, 2), (37, 53, 3), (300, 517, 2), (129, 300, 17), (200, 150, 64),
                                   (1000, 700, 64)])
def test_point_argmax_and_support_bit_exact(H, n, m, d):
    from paper_2504_02067_gb300 import Problem
    rng = np.random.default_rng(n + 7 * m + d)
    X = rng.normal(0, 1, size=(n, d)).astype(np.float32)
    Y = (rng.normal(0, 1, size=(m, d)) + 0.3).astype(np.float32)
    if m >= 3:
        Y[m - 1] = Y[1]  # duplicated points: exact ties when v agrees
    sC = O.sqeuclid_scale(X, Y)
    C64 = sC * O.sqeuclid_ordered(X, Y)
    u = rng.normal(0, 0.5, n)
    v = rng.normal(0, 0.5, m)
    if m >= 3:
        v[m - 1] = v[1]
    gamma = 256.0
    t_all = (u[:, None] + v[None, :]) - gamma * C64
    log_tau = float(np.quantile(t_all, 0.9)) if t_all.size > 1 else float(t_all.flat[0]) - 1.0
    prob = Problem(X=t(X, torch.float32), Y=t(Y, torch.float32), precision="mixed", cost_scale=sC)
    idx, cnt, tot = run_int(H, prob, u, v, gamma, log_tau)
    assert np.array_equal(idx, O.plan_row_argmax(v, gamma, C64))
    ref_cnt = O.plan_support_counts(u, v, gamma, C64, log_tau)
    assert np.array_equal(cnt, ref_cnt)
    assert tot == int(ref_cnt.sum())
    if m >= 3:
        assert not np.any(idx == m - 1)


def test_argmax_recovers_assignment_from_a_solve(H):
    """Uniform marginals, gamma_f = 2^12: the solved plan concentrates on the
    optimal assignment (Birkhoff), so the GPU row argmax at the GPU's potentials
    equals the oracle's argmax at the same potentials and, with a clear optimum,
    the permutation that brute force finds."""
    import itertools
    from paper_2504_02067_gb300 import Problem, default_params
    n = 7
    rng = np.random.default_rng(12)
    C = rng.uniform(0, 1, size=(n, n))
    C /= C.max()
    perms = list(itertools.permutations(range(n)))
    costs = np.array([C[np.arange(n), list(p)].sum() for p in perms])
    order = np.argsort(costs)
    assert costs[order[1]] - costs[order[0]] > 1e-3
    best = np.array(perms[order[0]])
    w = np.full(n, 1.0 / n)
    prob = Problem(t(C), t(w), t(w), precision="fp64")
    u, v, st = H.solve(prob, default_params(gamma_i=16.0, gamma_f=4096.0, tol_final=1e-7))
    idx = torch.empty(n, dtype=torch.int64, device=DEV)
    H.eot_plan_argmax(prob, v, 4096.0, idx)
    idx = idx.cpu().numpy()
    assert np.array_equal(idx, O.plan_row_argmax(v.cpu().numpy(), 4096.0, C))
    assert np.array_equal(idx, best)


def test_full_size_workloads_sampled_rows(H):
    """At the benchmark sizes: the 64 x 64 grid (n = m = 4096, FP32 cost) in full,
    and the d = 64 clouds (n = m = 16384) on 256 sampled rows, against the
    oracle's decisions on the same rows."""
    from paper_2504_02067_gb300 import Problem
    p = W.grid_problem_4096(0, "sqeuclid")
    C64 = p["C"].astype(np.float64)
    rng = np.random.default_rng(3)
    u = np.log(p["r"] + 1e-9) + rng.normal(0, 0.1, 4096)
    v = np.log(p["c"] + 1e-9) + rng.normal(0, 0.1, 4096)
    g = 16384.0
    t_row = (u[:, None] + v[None, :]) - g * C64
    log_tau = float(np.quantile(t_row, 0.999))
    prob = Problem(t(p["C"], torch.float32), precision="mixed")
    idx, cnt, tot = run_int(H, prob, u, v, g, log_tau)
    assert np.array_equal(idx, O.plan_row_argmax(v, g, C64))
    ref_cnt = O.plan_support_counts(u, v, g, C64, log_tau)
    assert np.array_equal(cnt, ref_cnt) and tot == int(ref_cnt.sum())
    del t_row

    q = W.gmm_problem_d64(0)
    X, Y = q["X"], q["Y"]
    n = X.shape[0]
    sC = O.sqeuclid_scale(X, Y)
    u = np.full(n, -math.log(n)) + rng.normal(0, 0.5, n)
    v = np.full(n, -math.log(n)) + rng.normal(0, 0.5, n)
    g = 1024.0
    rows = np.sort(rng.choice(n, 256, replace=False))
    Cs = sC * O.sqeuclid_ordered(X[rows], Y)
    ts = (u[rows, None] + v[None, :]) - g * Cs
    log_tau = float(np.quantile(ts, 0.99))
    probp = Problem(X=t(X, torch.float32), Y=t(Y, torch.float32), precision="mixed", cost_scale=sC)
    idx, cnt, _ = run_int(H, probp, u, v, g, log_tau)
    assert np.array_equal(idx[rows], O.plan_row_argmax(v, g, Cs))
    assert np.array_equal(cnt[rows], O.plan_support_counts(u[rows], v, g, Cs, log_tau))
