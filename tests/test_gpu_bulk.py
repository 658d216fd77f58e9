"""GPU parity of the bulk-copy (TMA ring) sweeps against the FP64 oracle.

With EOT_BULK=1 (set for this module), dense FP32 costs with at least 2^20
entries and 16-byte rows run their row and column sweeps through the bulk-copy
kernels: the shapes below cover a ragged
last column strip, rows longer than one 16 KB stage, fewer rows than SMs (idle
consumer warps), column vectors too large for six ring warps (four-warp
variant) and for any ring (register-load fallback inside the same solve).
Tolerance: marginal L1 <= 1e-6 in mixed precision, as for the other sweeps."""
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
    import os
    from paper_2504_02067_gb300 import Handle, build
    build()
    old = os.environ.get("EOT_BULK")
    os.environ["EOT_BULK"] = "1"
    h = Handle(0, 64, 64)
    yield h
    h.close()
    if old is None:
        del os.environ["EOT_BULK"]
    else:
        os.environ["EOT_BULK"] = old


def t(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device=DEV, dtype=dtype)


def near_feasible(seed, n, m, gamma, C64):
    rng = np.random.default_rng(seed)
    r = rng.dirichlet(np.ones(n)) * 0.999 + 0.001 / n
    c = rng.dirichlet(np.ones(m)) * 0.999 + 0.001 / m
    u = np.log(r) + rng.normal(0, 0.3, n) + 5.0 * gamma / 4096
    v = np.log(c) - O.lse_c(u[:, None] - gamma * C64)
    return u, v, r, c


# (n, m): ragged strip; multi-stage rows (four ring warps); one row per CTA and
# 12000 columns; a square 2^20; the 64 x 64 grid size
BULK_SIZES = [(1500, 1100), (300, 8200), (100, 12000), (1024, 1024), (2048, 4096)]


@pytest.mark.parametrize("n,m", BULK_SIZES)
def test_bulk_marginals_match_oracle(H, n, m):
    from paper_2504_02067_gb300 import Problem
    rng = np.random.default_rng(n * 3 + m)
    C = rng.uniform(0, 1, size=(n, m)).astype(np.float32)
    C64 = C.astype(np.float64)
    gamma = float(np.float32(2.0 ** 10))
    u, v, _, _ = near_feasible(n + 2 * m, n, m, gamma, C64)
    prob = Problem(t(C, torch.float32), precision="mixed")
    r, c, lr, lc, tot = H.marginals(prob, t(u), t(v), gamma)
    P = O.plan(u, v, gamma, C64)
    rr, cr = O.row_sum(P), O.col_sum(P)
    assert np.abs(r.cpu().numpy() - rr).sum() <= 1e-6
    assert np.abs(c.cpu().numpy() - cr).sum() <= 1e-6
    np.testing.assert_allclose(lr.cpu().numpy(), np.log(rr), atol=5e-5)
    np.testing.assert_allclose(lc.cpu().numpy(), np.log(cr), atol=5e-5)
    assert abs(tot.item() - P.sum()) <= 1e-6


def test_bulk_and_register_load_sweeps_agree(monkeypatch):
    """The same marginals through the bulk-copy kernels and, with EOT_BULK=0, the
    register-load kernels (separate handles): both within the mixed tolerance of
    each other."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_02067_gb300 import Handle, Problem
    n, m = 1500, 1100
    rng = np.random.default_rng(77)
    C = rng.uniform(0, 1, size=(n, m)).astype(np.float32)
    gamma = float(np.float32(2.0 ** 12))
    u, v, _, _ = near_feasible(78, n, m, gamma, C.astype(np.float64))
    out = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("EOT_BULK", flag)
        h = Handle(0, 64, 64)
        try:
            prob = Problem(t(C, torch.float32), precision="mixed")
            r, c, _, _, _ = h.marginals(prob, t(u), t(v), gamma)
            out[flag] = (r.cpu().numpy(), c.cpu().numpy())
        finally:
            h.close()
    assert np.abs(out["1"][0] - out["0"][0]).sum() <= 1e-6
    assert np.abs(out["1"][1] - out["0"][1]).sum() <= 1e-6


@pytest.mark.parametrize("kappa", [0.0, -3.0e4, 2.0e5])
def test_bulk_lse_large_potentials_gauge(H, kappa):
    """Potentials of magnitude ~gamma (a zero-bin grid problem at gamma = 4096)
    shifted along the gauge direction: the online max of the bulk LSE sweeps is
    raised lazily as in the register-load kernels and the marginals are those of
    the unshifted point."""
    from paper_2504_02067_gb300 import Problem
    p = W.grid_problem_4096(5, "l1", side=48)
    C64 = p["C"].astype(np.float64)
    gamma = 4096.0
    r, c = p["r"] * 0.999 + 0.001 / C64.shape[0], p["c"] * 0.999 + 0.001 / C64.shape[1]
    u, v = O.sinkhorn_log(C64, r, c, gamma, tol=1e-30, max_iter=25)
    assert np.abs(u).max() > 100
    P = O.plan(u, v, gamma, C64)
    prob = Problem(t(p["C"], torch.float32), precision="mixed")
    rr, cc, lr, lc, tot = H.marginals(prob, t(u + kappa), t(v - kappa), gamma)
    assert np.abs(rr.cpu().numpy() - O.row_sum(P)).sum() <= 1e-6
    assert np.abs(cc.cpu().numpy() - O.col_sum(P)).sum() <= 1e-6
    assert abs(tot.item() - P.sum()) <= 1e-6


@pytest.mark.parametrize("n,m", [(1024, 1024), (300, 8200)])
def test_bulk_newton_solve_matches_oracle(H, n, m):
    """Alg. 2 (set-up sweeps, the CG halves in the captured graph, d_v) through
    the bulk kernels: rho, CG count within one per solve, direction modulo gauge."""
    from paper_2504_02067_gb300 import Problem
    rng = np.random.default_rng(n + m)
    C = rng.uniform(0, 1, size=(n, m)).astype(np.float32)
    C64 = C.astype(np.float64)
    gamma = 64.0
    u, v, r, c = near_feasible(abs(n - m), n, m, gamma, C64)
    P = O.plan(u, v, gamma, C64)
    rP = O.row_sum(P)
    rt = rP * (1 + 0.02 * rng.normal(size=n))
    rt /= rt.sum()
    gu = rP - rt
    gl1 = np.abs(gu).sum()
    eta = max(gl1, 0.8 * 1e-4 / gl1)
    ref = O.newton_solve(P, gu, gl1, eta, 0.0)
    prob = Problem(t(C, torch.float32), precision="mixed")
    du, dv, rho, it = H.newton_solve(prob, t(u), t(v), gamma, t(rt), eta, 0.0)
    du = du.cpu().numpy()
    assert rho == pytest.approx(ref.rho)
    assert abs(it - ref.cg_iters) <= 1 + ref.cg_solves
    ref_du = ref.d_u - (rP @ ref.d_u) / rP.sum()
    diff = du - ref_du
    kappa = diff.mean()
    assert np.abs(diff - kappa).sum() <= 1e-5 * np.abs(ref_du).sum()
    np.testing.assert_allclose(dv.cpu().numpy() + kappa, -(P.T @ ref_du) / O.col_sum(P),
                               atol=1e-5 * np.abs(ref_du).max())
    assert np.abs(O.F_r_apply(P, 1.0, du) + gu).sum() <= eta * gl1 * (1 + 1e-6)


def test_bulk_solve_reaches_tolerance(H):
    """A full solve of a 1200 x 1100 point problem (L1 cost, Dirichlet weights) in
    mixed precision reaches marginal L1 <= 1e-6 as the oracle evaluates it in
    FP64 (transport-cost parity at full size: test_gpu_dense's 64 x 64 grid
    trace, which also runs through these kernels)."""
    from paper_2504_02067_gb300 import Problem, default_params
    rng = np.random.default_rng(5)
    n, m = 1200, 1100
    x = rng.uniform(0, 1, size=(n, 2))
    y = rng.uniform(0, 1, size=(m, 2))
    C64 = np.abs(x[:, None, :] - y[None, :, :]).sum(-1)
    C = (C64 / C64.max()).astype(np.float32)
    C64 = C.astype(np.float64)
    r = rng.dirichlet(np.ones(n))
    c = rng.dirichlet(np.ones(m))
    gf = 1024.0
    prob = Problem(t(C, torch.float32), t(r), t(c))
    u, v, st = H.solve(prob, default_params(gamma_i=16.0, gamma_f=gf, tol_final=1e-6))
    u, v = u.cpu().numpy(), v.cpu().numpy()
    assert st["cg_iters"] > 0
    assert O.marginal_l1_error(u, v, gf, C64, r, c) <= 1e-6
