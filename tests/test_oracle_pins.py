"""Pins for the FP64 oracle: each check ties an oracle function to something other
than itself (a closed form, an invariant the paper proves, finite differences,
dense linear algebra, a library routine, brute force, or the paper's worked
example). CPU only."""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.optimize
import scipy.special

from oracle import eot_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_problem(seed, n, m=None, gamma=8.0):
    rng = np.random.default_rng(seed)
    m = n if m is None else m
    C = rng.uniform(0, 1, size=(n, m))
    u = rng.normal(0, 0.5, size=n) - math.log(n)
    v = rng.normal(0, 0.5, size=m)
    return C, u, v, gamma


def feasible_c(C, u, v, gamma):
    """Column-fix v so that c(P) equals the returned c (makes c = c(P) hold)."""
    return O.col_sum(O.plan(u, v, gamma, C))


# ---------------- basic definitions ----------------

def test_lse_matches_scipy():
    rng = np.random.default_rng(0)
    X = rng.normal(0, 30, size=(7, 11))
    np.testing.assert_allclose(O.lse_r(X), scipy.special.logsumexp(X, axis=1), rtol=1e-14)
    np.testing.assert_allclose(O.lse_c(X), scipy.special.logsumexp(X, axis=0), rtol=1e-14)


def test_log_sums_match_plan():
    C, u, v, g = rand_problem(1, 9, 6)
    P = O.plan(u, v, g, C)
    np.testing.assert_allclose(O.log_row_sum(u, v, g, C), np.log(P.sum(1)), rtol=1e-13)
    np.testing.assert_allclose(O.log_col_sum(u, v, g, C), np.log(P.sum(0)), rtol=1e-13)


def test_entropy_and_chi2_special_cases():
    assert O.entropy(np.full(8, 1 / 8)) == pytest.approx(math.log(8), rel=1e-14)
    assert O.entropy(np.array([1.0, 0.0, 0.0])) == 0.0
    x = np.array([0.2, 0.3, 0.5])
    assert O.chi2(x, x) == pytest.approx(0.0, abs=1e-15)
    y = np.array([0.3, 0.3, 0.4])
    # chi^2(y|x) >= ||y - x||_1^2 (Sec. 2 notation)
    assert O.chi2(y, x) >= np.abs(y - x).sum() ** 2


def test_paper_worked_example_appx_e(oracle):
    """Appx. E n = 4 example: build a plan whose P_rc equals the printed Q and check
    the oracle's P_rc, F_r(1), the printed eigenvalues and the printed identity
    ||(r(P) - r)^T Q^l||_1 = 0.5^l chi(r | r(P))."""
    g = json.load(open(os.path.join(GOLDEN, "appx_e_n4_example.json")))
    Q = np.array(g["Q"])
    rP = np.array(g["r_P"])
    r = np.array(g["r"])
    # a P with uniform marginals 1/4 and blocks [[a, 1-a], [1-a, a]] / 4 has
    # P_rc = 16 P P^T; a^2 + (1-a)^2 = 3/4 gives the printed Q.
    a = (1 + 1 / math.sqrt(2)) / 2
    B = np.array([[a, 1 - a], [1 - a, a]])
    P = np.zeros((4, 4))
    P[:2, :2] = B / 4
    P[2:, 2:] = B / 4
    np.testing.assert_allclose(O.row_sum(P), rP, atol=1e-15)
    np.testing.assert_allclose(O.P_rc(P), Q, atol=1e-14)
    np.testing.assert_allclose(O.F_r_matrix(P, 1.0), np.diag(rP) @ (np.eye(4) - Q), atol=1e-14)
    ev = np.sort(np.linalg.eigvalsh(O.P_rc(P)))[::-1]
    np.testing.assert_allclose(ev, g["eigenvalues_Q"], atol=1e-12)
    chi = math.sqrt(O.chi2(r, rP))
    for l in range(6):
        lhs = np.abs((rP - r) @ np.linalg.matrix_power(Q, l)).sum()
        assert lhs == pytest.approx(g["decay_per_step"] ** l * chi, rel=1e-12)


# ---------------- dual, gradient, Hessian ----------------

def test_gradient_is_fd_of_dual():
    """K5: central finite difference of g (Eq. sinkhorn-dual) along random directions."""
    C, u, v, g = rand_problem(2, 8, 5)
    rng = np.random.default_rng(3)
    r = rng.dirichlet(np.ones(8))
    c = rng.dirichlet(np.ones(5))
    gu, gv = O.dual_gradient(u, v, g, C, r, c)
    for _ in range(3):
        du, dv = rng.normal(size=8), rng.normal(size=5)
        h = 1e-5
        fd = (O.dual_objective(u + h * du, v + h * dv, g, C, r, c)
              - O.dual_objective(u - h * du, v - h * dv, g, C, r, c)) / (2 * h)
        assert fd == pytest.approx(gu @ du + gv @ dv, rel=1e-8, abs=1e-12)


def test_hvp_is_fd_of_gradient():
    """K4: central finite difference of the dual gradient; error O(h^2)."""
    C, u, v, g = rand_problem(4, 7, 9)
    rng = np.random.default_rng(5)
    r = rng.dirichlet(np.ones(7))
    c = rng.dirichlet(np.ones(9))
    du, dv = rng.normal(size=7), rng.normal(size=9)
    ou, ov, _, _ = O.hvp(u, v, g, C, du, dv)
    errs = []
    for h in (1e-3, 5e-4):
        gp = O.dual_gradient(u + h * du, v + h * dv, g, C, r, c)
        gm = O.dual_gradient(u - h * du, v - h * dv, g, C, r, c)
        fd = np.concatenate([(gp[0] - gm[0]) / (2 * h), (gp[1] - gm[1]) / (2 * h)])
        errs.append(np.abs(fd - np.concatenate([ou, ov])).max())
    assert errs[0] < 1e-5
    assert errs[1] < errs[0] / 3  # second-order convergence


def test_hvp_matches_assembled_hessian_and_null_vector():
    """Eq. hessian / discounted-hessian assembled densely; K1: H (1, -1) = 0 (Sec. 2.1 footnote)."""
    C, u, v, g = rand_problem(6, 6, 6)
    P = O.plan(u, v, g, C)
    rng = np.random.default_rng(7)
    du, dv = rng.normal(size=6), rng.normal(size=6)
    for s in (1.0, math.sqrt(0.7)):
        ou, ov, _, _ = O.hvp(u, v, g, C, du, dv, s)
        np.testing.assert_allclose(np.concatenate([ou, ov]),
                                   O.hessian_matrix(P, s) @ np.concatenate([du, dv]), rtol=1e-12)
    ou, ov, _, _ = O.hvp(u, v, g, C, np.ones(6), -np.ones(6))
    assert np.abs(np.concatenate([ou, ov])).max() < 1e-15
    ev = np.linalg.eigvalsh(O.hessian_matrix(P))
    assert ev.min() > -1e-14 and np.sort(ev)[1] > 1e-6  # PSD with one zero eigenvalue


# ---------------- F_r(rho), P_rc ----------------

def test_F_r_is_schur_complement_of_discounted_hessian():
    """(H(rho)^-1)_uu = F_r(rho)^-1 (Eq. inverse-discounted-hessian) and the
    off-diagonal block -sqrt(rho) F_r^-1 P_c^T."""
    C, u, v, g = rand_problem(8, 6, 7)
    P = O.plan(u, v, g, C)
    for rho in (0.0, 0.5, 0.9):
        Hinv = np.linalg.inv(O.hessian_matrix(P, math.sqrt(rho)))
        Fr = O.F_r_matrix(P, rho)
        np.testing.assert_allclose(Hinv[:6, :6], np.linalg.inv(Fr), rtol=1e-9)
        Pc = P.T / O.col_sum(P)[:, None]
        np.testing.assert_allclose(Hinv[:6, 6:], -math.sqrt(rho) * np.linalg.inv(Fr) @ Pc.T,
                                   rtol=1e-8, atol=1e-10)


def test_F_r_apply_diag_and_properties():
    """K2 (F_r(rho) 1 = (1 - rho) r(P)), K3 (symmetry, reversibility, stationarity),
    apply/diag agree with the dense matrix."""
    C, u, v, g = rand_problem(9, 10, 8)
    P = O.plan(u, v, g, C)
    rP = O.row_sum(P)
    rng = np.random.default_rng(10)
    x = rng.normal(size=10)
    Prc = O.P_rc(P)
    np.testing.assert_allclose(Prc.sum(1), 1.0, rtol=1e-14)
    np.testing.assert_allclose(rP @ Prc, rP, rtol=1e-13)
    np.testing.assert_allclose(np.diag(rP) @ Prc, (np.diag(rP) @ Prc).T, rtol=1e-12)
    for rho in (0.0, 0.3, 0.99, 1.0):
        Fr = O.F_r_matrix(P, rho)
        np.testing.assert_allclose(Fr, Fr.T, rtol=1e-12, atol=1e-16)
        np.testing.assert_allclose(O.F_r_apply(P, rho, x), Fr @ x, rtol=1e-11, atol=1e-15)
        np.testing.assert_allclose(O.F_r_diag(P, rho), np.diag(Fr), rtol=1e-12)
        np.testing.assert_allclose(O.F_r_apply(P, rho, np.ones(10)), (1 - rho) * rP,
                                   rtol=1e-10, atol=1e-15)


def test_F_r_gerschgorin_and_preconditioned_spectrum():
    """K7: Lemma fr-properties bounds and Lemma condition-number bounds."""
    C, u, v, g = rand_problem(11, 12, 12, gamma=5.0)
    P = O.plan(u, v, g, C)
    rP = O.row_sum(P)
    mu_min = np.diag(O.P_rc(P)).min()
    for rho in (0.2, 0.75, 0.95):
        Fr = O.F_r_matrix(P, rho)
        ev = np.linalg.eigvalsh(Fr)
        assert ev.min() >= (1 - rho) * rP.min() * (1 - 1e-10)
        assert ev.max() <= (1 + rho) * rP.max() * (1 + 1e-10)
        Mh = 1 / np.sqrt(O.F_r_diag(P, rho))
        evp = np.linalg.eigvalsh(Mh[:, None] * Fr * Mh[None, :])
        w = rho * (1 - mu_min) / (1 - rho * mu_min)
        assert evp.min() >= 1 - w - 1e-10 and evp.max() <= 1 + w + 1e-10


# ---------------- PCG and NewtonSolve ----------------

def test_pcg_matches_dense_solve():
    """K6: PCG against a dense solve, both on a random SPD system and on F_r(rho)."""
    rng = np.random.default_rng(12)
    A = rng.normal(size=(20, 20))
    A = A @ A.T + 20 * np.eye(20)
    b = rng.normal(size=20)
    res = O.pcg(lambda x: A @ x, b, np.diag(A).copy(), 1e-13, 200)
    assert res.converged
    np.testing.assert_allclose(res.x, scipy.linalg.solve(A, b, assume_a="pos"), rtol=1e-11)
    C, u, v, g = rand_problem(13, 16, 16, gamma=6.0)
    P = O.plan(u, v, g, C)
    r = rng.dirichlet(np.ones(16))
    b = -(O.row_sum(P) - r)
    for rho in (0.0, 0.9):
        res = O.pcg(lambda x: O.F_r_apply(P, rho, x), b, O.F_r_diag(P, rho), 1e-15, 200)
        np.testing.assert_allclose(res.x, np.linalg.solve(O.F_r_matrix(P, rho), b), rtol=1e-8)


def test_discounted_newton_system_is_bellman_eq():
    """Eq. bellman2: with c = c(P) the discounted Newton system's solution satisfies
    d_u = (r / r(P) - 1) + rho P_rc d_u and d_v = -sqrt(rho) P_c d_u."""
    C, u, v, g = rand_problem(14, 9, 9, gamma=4.0)
    P = O.plan(u, v, g, C)
    rP, cP = O.row_sum(P), O.col_sum(P)
    r = np.random.default_rng(15).dirichlet(np.ones(9))
    grad = np.concatenate([rP - r, np.zeros(9)])  # c(P) = c
    for rho in (0.25, 0.8):
        d = np.linalg.solve(O.hessian_matrix(P, math.sqrt(rho)), -grad)
        du, dv = d[:9], d[9:]
        np.testing.assert_allclose(du, (r / rP - 1) + rho * O.P_rc(P) @ du, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(dv, -math.sqrt(rho) * (P.T @ du) / cP, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(du, np.linalg.solve(O.F_r_matrix(P, rho), r - rP), rtol=1e-9)


def test_newton_residual_blocks():
    """K8 (Eq. explicit-residual, Appx. A): with d_v = -P_c d_u and c = c(P) the
    v-block of the Newton residual is 0 and the u-block is F_r(1) d_u + grad_u g."""
    C, u, v, g = rand_problem(16, 8, 8)
    P = O.plan(u, v, g, C)
    rP, cP = O.row_sum(P), O.col_sum(P)
    r = np.random.default_rng(17).dirichlet(np.ones(8))
    du = np.random.default_rng(18).normal(size=8)
    dv = -(P.T @ du) / cP
    e = O.hessian_matrix(P) @ np.concatenate([du, dv]) + np.concatenate([rP - r, np.zeros(8)])
    assert np.abs(e[8:]).max() < 1e-15
    np.testing.assert_allclose(e[:8], O.F_r_apply(P, 1.0, du) + (rP - r), rtol=1e-10, atol=1e-15)


def test_newton_solve_meets_forcing_and_descends():
    """Alg. 2 output meets the forcing test (Eq. forcing) and is a descent direction (K10)."""
    C, u, v, g = rand_problem(19, 30, 30, gamma=20.0)
    P = O.plan(u, v, g, C)
    rP = O.row_sum(P)
    r = rP * (1 + 0.05 * np.random.default_rng(20).normal(size=30))
    r = r / r.sum() * rP.sum()
    grad_u = rP - r
    gl1 = np.abs(grad_u).sum()
    for eta in (0.5, 0.1, 0.01):
        res = O.newton_solve(P, grad_u, gl1, eta, 0.0)
        assert res.converged
        assert np.abs(O.F_r_apply(P, 1.0, res.d_u) + grad_u).sum() <= eta * gl1
        assert -grad_u @ res.d_u > 0
        # rho follows 0, 3/4, 15/16, ... (Alg. 2's annealing)
        for k, rho in enumerate(res.rhos):
            assert rho == pytest.approx(1 - 4.0 ** -k, abs=1e-15)
    assert O.next_rho0(0.9375) == pytest.approx(0.75)
    assert O.next_rho0(0.5) == 0.0


def test_discounted_hessian_apply_matches_assembled_matrix():
    """discounted_hessian_apply = the assembled Eq. discounted-hessian (off-diagonal
    blocks times sqrt(rho)); SPD for rho < 1, singular along (1, -1) at rho = 1."""
    C, u, v, g = rand_problem(41, 9, 7)
    P = O.plan(u, v, g, C)
    rng = np.random.default_rng(42)
    du, dv = rng.normal(size=9), rng.normal(size=7)
    for rho in (0.0, 0.3, 0.9375, 1.0):
        H = O.hessian_matrix(P, math.sqrt(rho))
        hu, hv = O.discounted_hessian_apply(P, rho, du, dv)
        np.testing.assert_allclose(np.concatenate([hu, hv]), H @ np.concatenate([du, dv]),
                                   rtol=1e-12, atol=1e-15)
        lam = np.linalg.eigvalsh(H)
        if rho < 1.0:
            assert lam.min() > 0.0
    hu, hv = O.discounted_hessian_apply(P, 1.0, np.ones(9), -np.ones(7))
    assert np.abs(hu).max() + np.abs(hv).max() <= 1e-14


def test_full_system_newton_step_equals_schur_solve():
    """PCG on the full discounted system, run tight, gives the u-block of the dense
    solve of F_r(rho) d_u = -grad_u g (Schur complement, Eq. matrix-definitions)
    and the v-block -sqrt(rho) D(c(P))^-1 P^T d_u (second block row)."""
    C, u, v, g = rand_problem(43, 24, 20, gamma=12.0)
    P = O.plan(u, v, g, C)
    rP, cP = O.row_sum(P), O.col_sum(P)
    rng = np.random.default_rng(44)
    grad_u = rP * 0.05 * rng.normal(size=24)
    grad_u -= grad_u.mean()
    for rho in (0.0, 0.75, 0.984375):
        d_u = np.linalg.solve(O.F_r_matrix(P, rho), -grad_u)

        def apply_H(x, rho=rho):
            hu, hv = O.discounted_hessian_apply(P, rho, x[:24], x[24:])
            return np.concatenate([hu, hv])
        res = O.pcg(apply_H, np.concatenate([-grad_u, np.zeros(20)]), np.concatenate([rP, cP]),
                    1e-14 * np.abs(grad_u).sum(), 2000)
        assert res.converged
        np.testing.assert_allclose(res.x[:24], d_u, rtol=1e-8, atol=1e-10 * np.abs(d_u).max())
        np.testing.assert_allclose(res.x[24:], -math.sqrt(rho) * (P.T @ d_u) / cP,
                                   rtol=1e-8, atol=1e-10 * np.abs(d_u).max())


def test_newton_solve_full_meets_forcing_like_alg2():
    """The full-system variant keeps Alg. 2's outer loop: same rho sequence, the
    forcing test met, a descent direction, and a direction within the CG
    tolerances of Alg. 2's (both approximate F_r(rho)^-1 (-grad_u g))."""
    C, u, v, g = rand_problem(19, 30, 30, gamma=20.0)
    P = O.plan(u, v, g, C)
    rP = O.row_sum(P)
    r = rP * (1 + 0.05 * np.random.default_rng(20).normal(size=30))
    r = r / r.sum() * rP.sum()
    grad_u = rP - r
    gl1 = np.abs(grad_u).sum()
    for eta in (0.5, 0.1, 0.01):
        full = O.newton_solve_full(P, grad_u, gl1, eta, 0.0)
        ref = O.newton_solve(P, grad_u, gl1, eta, 0.0)
        assert full.converged
        assert np.abs(O.F_r_apply(P, 1.0, full.d_u) + grad_u).sum() <= eta * gl1
        assert -grad_u @ full.d_u > 0
        for k, rho in enumerate(full.rhos):
            assert rho == pytest.approx(1 - 4.0 ** -k, abs=1e-15)
        # both meet the same forcing test, so they differ by at most the sum of
        # their residuals mapped through F_r(1)'s inverse on the complement of 1
        diff = full.d_u - ref.d_u
        diff -= (rP @ diff) / rP.sum()
        scale = np.abs(ref.d_u - (rP @ ref.d_u) / rP.sum()).sum()
        assert np.abs(diff).sum() <= 2 * eta * scale + 1e-12


def test_armijo_simplification_equals_full_test():
    """K9 (Lemma sufficient-decrease): with c = c(P) and d_v = -P_c d_u,
    g(z + a d) - g(z) - c1 a <grad g, d> == lhs(a) - (1 - c1) a <-grad_u g, d_u>."""
    C, u, v, g = rand_problem(21, 7, 9)
    u = u - math.log(O.plan(u, v, g, C).sum())  # sum P = 1, so c = c(P) lies on the simplex
    c = feasible_c(C, u, v, g)
    P = O.plan(u, v, g, C)
    rng = np.random.default_rng(22)
    r = rng.dirichlet(np.ones(7))
    grad_u = O.row_sum(P) - r
    du = rng.normal(size=7)
    dv = -(P.T @ du) / O.col_sum(P)
    c1 = 0.01
    g0 = O.dual_objective(u, v, g, C, r, c)
    for a in (1.0, 0.5, 0.125):
        full = O.dual_objective(u + a * du, v + a * dv, g, C, r, c) - g0 - c1 * a * (grad_u @ du)
        lhs, _ = O.armijo_lhs(u, v, du, dv, a, g, C)
        simple = lhs - (1 - c1) * a * (-grad_u @ du)
        assert full == pytest.approx(simple, rel=1e-9, abs=1e-13)


# ---------------- Alg. 3 / Alg. 4 / Alg. 1 ----------------

def test_chi_sinkhorn_postconditions():
    C, u, v, g = rand_problem(23, 12, 10, gamma=10.0)
    rng = np.random.default_rng(24)
    r, c = rng.dirichlet(np.ones(12)), rng.dirichlet(np.ones(10))
    v = np.log(c) - O.lse_c(u[:, None] - g * C)
    lrp = O.log_row_sum(u, v, g, C)
    u2, v2, lrp2, it = O.chi_sinkhorn(u, v, g, C, r, c, lrp, 1e-6)
    P = O.plan(u2, v2, g, C)
    assert it > 0
    assert O.chi2(r, O.row_sum(P)) <= 1e-6
    np.testing.assert_allclose(O.col_sum(P), c, rtol=1e-12)
    np.testing.assert_allclose(np.exp(lrp2), O.row_sum(P), rtol=1e-12)


def test_projection_agrees_with_independent_sinkhorn():
    """K14: Alg. 4 and plain log-domain Sinkhorn reach the same unique optimum."""
    rng = np.random.default_rng(25)
    n, m = 20, 15
    C = rng.uniform(0, 1, size=(n, m))
    r, c = rng.dirichlet(np.ones(n)), rng.dirichlet(np.ones(m))
    g = 30.0
    u, v, st = O.truncated_newton_project(np.log(r), np.log(c), g, C, r, c, 1e-11)
    assert st.ok and st.newton_steps >= 1
    us, vs = O.sinkhorn_log(C, r, c, g, tol=1e-13)
    P, Ps = O.plan(u, v, g, C), O.plan(us, vs, g, C)
    assert np.abs(P - Ps).sum() < 1e-9
    np.testing.assert_allclose(O.row_sum(P), r, rtol=1e-12)  # last row step
    assert np.abs(O.col_sum(P) - c).sum() <= 1e-11
    # duality gap -> 0 with the marginal error
    gap = O.primal_value(P, C, g) - (-O.dual_objective(u, v, g, C, r, c)) / g
    assert abs(gap) < 1e-9


def test_closed_form_additive_cost():
    """K13: C_ij = a_i + b_j makes <P, C> constant on U(r, c), so the EOT optimum is
    the independence coupling r c^T (Sec. 2.2), at any gamma."""
    rng = np.random.default_rng(26)
    n, m = 24, 18
    a, b = rng.uniform(0, 0.5, n), rng.uniform(0, 0.5, m)
    C = a[:, None] + b[None, :]
    r, c = rng.dirichlet(np.ones(n)), rng.dirichlet(np.ones(m))
    res = O.mdot(C, r, c, gamma_i=4.0, gamma_f=256.0, tol_final=1e-9)
    assert res.ok
    P = O.plan(res.u, res.v, res.gamma, C)
    assert np.abs(P - np.outer(r, c)).sum() < 3e-9
    # potentials have the closed form up to the gauge
    du = res.u - (np.log(r) + res.gamma * a)
    dv = res.v - (np.log(c) + res.gamma * b)
    assert np.ptp(du) < 1e-6 and np.ptp(dv) < 1e-6 and abs(du.mean() + dv.mean()) < 1e-6


def test_smoothing_and_schedule():
    rng = np.random.default_rng(27)
    r = rng.dirichlet(np.ones(10))
    c = rng.dirichlet(np.ones(7))
    rs, cs = O.smooth_marginals(r, c, 0.01)
    assert rs.sum() == pytest.approx(1.0) and cs.sum() == pytest.approx(1.0)
    assert np.abs(rs - r).sum() <= 2 * 0.45 * 0.01 and np.abs(cs - c).sum() <= 2 * 0.05 * 0.01
    assert rs.min() >= 0.45 * 0.01 / 10 * (1 - 1e-12)
    assert O.adjust_schedule(2 ** 0.5, 0.99) == pytest.approx(2.0)
    assert O.adjust_schedule(1.1, 0.99) == pytest.approx(1.21)
    assert O.adjust_schedule(2.0, 0.5) == pytest.approx(2 ** 0.5)
    assert O.adjust_schedule(2.0, 0.9) == 2.0
    assert O.adjust_schedule(1.5, math.inf) == 2.0


def test_mdot_stage_records_follow_alg1():
    """The per-stage records of mdot restate Alg. 1's schedule, checked here from
    the paper's rules: gamma^(1) = min(gamma_i, gamma_f); eps_d = min(H(r), H(c)) /
    gamma^p and the projection tolerance eps_d / 2, with the final stage's eps_d
    capped at 2 tol / 3 (reading); q from delta_min by the rule of Sec. 3.3;
    gamma^(t+1) = min(q gamma^(t), gamma_f); and the per-stage counts add up to
    the totals."""
    rng = np.random.default_rng(61)
    n, m = 40, 30
    C = rng.uniform(0, 1, size=(n, m))
    r, c = rng.dirichlet(np.ones(n)), rng.dirichlet(np.ones(m))
    gi, gf, p, tol = 16.0, 2048.0, 1.5, 1e-7
    res = O.mdot(C, r, c, gamma_i=gi, gamma_f=gf, p=p, tol_final=tol)
    H = min(-(r * np.log(r)).sum(), -(c * np.log(c)).sum())
    recs = res.records
    assert len(recs) == res.stages and res.ok
    assert recs[0]["gamma"] == min(gi, gf) and recs[-1]["gamma"] == gf
    q = 2.0
    for k, rec in enumerate(recs):
        eps_d = H / rec["gamma"] ** p
        if rec["gamma"] == gf:
            eps_d = min(eps_d, 2 * tol / 3)
        assert rec["eps"] == pytest.approx(eps_d / 2, rel=1e-12)
        d = rec["delta_min"]
        q = min(2.0, q * q) if d > 0.95 else (math.sqrt(q) if d < 0.8 else q)
        assert rec["q_next"] == pytest.approx(q, rel=1e-15)
        if k + 1 < len(recs):
            assert recs[k + 1]["gamma"] == pytest.approx(min(q * rec["gamma"], gf), rel=1e-15)
    assert sum(rec["newton_steps"] for rec in recs) == res.newton_steps
    assert sum(rec["cg_iters"] for rec in recs) == res.cg_iters
    assert sum(rec["ls_trials"] for rec in recs) == res.ls_trials
    assert O.marginal_l1_error(res.u, res.v, gf, C, r, c) <= tol


def test_mdot_reaches_tolerance_and_matches_sinkhorn():
    rng = np.random.default_rng(28)
    n = 40
    C = rng.uniform(0, 1, size=(n, n))
    r, c = rng.dirichlet(np.ones(n)), rng.dirichlet(np.ones(n))
    res = O.mdot(C, r, c, gamma_i=16.0, gamma_f=512.0, tol_final=1e-8)
    assert res.ok and res.gammas[-1] == 512.0
    assert O.marginal_l1_error(res.u, res.v, res.gamma, C, r, c) <= 1e-8
    us, vs = O.sinkhorn_log(C, r, c, 512.0, tol=1e-12, u=res.u, v=res.v)
    cost = O.transport_cost(res.u, res.v, 512.0, C)
    assert abs(cost - O.transport_cost(us, vs, 512.0, C)) / cost < 1e-6
    # the schedule increases gamma monotonically by factors in (1, 2]
    gs = np.array(res.gammas)
    assert np.all(gs[1:] > gs[:-1]) and np.all(gs[1:] / gs[:-1] <= 2.0 + 1e-12)


def test_round_lands_in_polytope():
    rng = np.random.default_rng(29)
    F = rng.uniform(0, 1, size=(6, 5))
    F /= F.sum()
    r, c = rng.dirichlet(np.ones(6)), rng.dirichlet(np.ones(5))
    G = O.round_to_polytope(F, r, c)
    assert G.min() >= 0
    np.testing.assert_allclose(G.sum(1), r, atol=1e-15)
    np.testing.assert_allclose(G.sum(0), c, atol=1e-15)


@pytest.mark.parametrize("n", [4, 6, 7])
def test_brute_force_error_bound(n):
    """K12: uniform marginals; the LP optimum is a permutation (Birkhoff); the rounded
    MDOT plan is within 2 log(n) / gamma_f of it (Sec. 2.2 error guarantee)."""
    rng = np.random.default_rng(30 + n)
    C = rng.uniform(0, 1, size=(n, n))
    C /= C.max()
    r = c = np.full(n, 1.0 / n)
    ot = O.brute_force_assignment(C)
    ri, ci = scipy.optimize.linear_sum_assignment(C)
    assert ot == pytest.approx(C[ri, ci].mean(), abs=1e-15)
    for gf in (2.0 ** 6, 2.0 ** 10):
        res = O.mdot(C, r, c, gamma_i=4.0, gamma_f=gf, tol_final=1e-9)
        assert res.ok
        P = O.round_to_polytope(O.plan(res.u, res.v, res.gamma, C), r, c)
        gap = (P * C).sum() - ot
        assert -1e-12 <= gap <= 2 * math.log(n) / gf


# ---------------- differentiation (envelope theorem) ----------------

def _solve_tight(C, r, c, g):
    return O.sinkhorn_log(C, r, c, g, tol=1e-15, max_iter=200000)


def test_grad_wrt_cost_and_marginals_fd():
    """K15: dF*/dC = P*, dF*/dr = u*/gamma (simplex-tangent), by central differences."""
    rng = np.random.default_rng(40)
    n, m, g = 5, 4, 6.0
    C = rng.uniform(0, 1, size=(n, m))
    r, c = rng.dirichlet(np.ones(n) * 3), rng.dirichlet(np.ones(m) * 3)
    u, v = _solve_tight(C, r, c, g)
    dC, dr, dc = O.eot_grads_dense(u, v, g, C)
    h = 1e-5
    E = rng.normal(size=(n, m))
    Fp = O.eot_value(*_solve_tight(C + h * E, r, c, g), g, C + h * E)
    Fm = O.eot_value(*_solve_tight(C - h * E, r, c, g), g, C - h * E)
    assert (Fp - Fm) / (2 * h) == pytest.approx((dC * E).sum(), rel=1e-6)
    t = rng.normal(size=n)
    t -= t.mean()  # tangent to the simplex
    Fp = O.eot_value(*_solve_tight(C, r + h * t, c, g), g, C)
    Fm = O.eot_value(*_solve_tight(C, r - h * t, c, g), g, C)
    assert (Fp - Fm) / (2 * h) == pytest.approx(dr @ t, rel=1e-5)


def test_grad_wrt_points_fd():
    """K15: dF*/dx_i = 2 s_C sum_j P_ij (x_i - y_j) with s_C held fixed."""
    rng = np.random.default_rng(41)
    n, m, d, g = 5, 6, 3, 5.0
    X, Y = rng.normal(size=(n, d)), rng.normal(size=(m, d))
    r, c = np.full(n, 1 / n), np.full(m, 1 / m)
    sC = 0.2
    C = sC * O.sqeuclid(X, Y)
    u, v = _solve_tight(C, r, c, g)
    dX, dY = O.eot_grads_points(u, v, g, X, Y, sC)
    h = 1e-5
    E = rng.normal(size=(n, d))
    F = []
    for s in (+1, -1):
        Cs = sC * O.sqeuclid(X + s * h * E, Y)
        F.append(O.eot_value(*_solve_tight(Cs, r, c, g), g, Cs))
    assert (F[0] - F[1]) / (2 * h) == pytest.approx((dX * E).sum(), rel=1e-6)
    E = rng.normal(size=(m, d))
    F = []
    for s in (+1, -1):
        Cs = sC * O.sqeuclid(X, Y + s * h * E)
        F.append(O.eot_value(*_solve_tight(Cs, r, c, g), g, Cs))
    assert (F[0] - F[1]) / (2 * h) == pytest.approx((dY * E).sum(), rel=1e-6)


def test_sqeuclid_scale_is_max():
    rng = np.random.default_rng(42)
    X, Y = rng.normal(size=(300, 3)), rng.normal(size=(200, 3))
    D = O.sqeuclid(X, Y)
    assert O.sqeuclid_scale(X, Y, block=64) == pytest.approx(1 / D.max(), rel=1e-15)
    np.testing.assert_allclose(O.sqeuclid_rows(X, Y, [3, 7]), D[[3, 7]], rtol=1e-15)


@pytest.mark.parametrize("n,m", [(1, 7), (5, 1), (1, 1)])
def test_mdot_single_row_or_column_is_product_plan(n, m):
    """With one row or one column the transport polytope U(r, c) holds a single
    plan, r c^T (every row of a one-column plan is forced to r_i, and vice
    versa); the oracle must return potentials whose plan is exactly that."""
    rng = np.random.default_rng(n * 10 + m)
    C = rng.uniform(0, 1, size=(n, m))
    r = rng.dirichlet(np.ones(n))
    c = rng.dirichlet(np.ones(m))
    res = O.mdot(C, r, c, gamma_i=16.0, gamma_f=4096.0)
    P = O.plan(res.u, res.v, 4096.0, C)
    assert res.ok
    assert np.abs(P - np.outer(r, c)).max() <= 1e-12
    assert O.marginal_l1_error(res.u, res.v, 4096.0, C, r, c) <= 1e-12


def test_mdot_sinkhorn_reaches_the_same_optimum():
    """MDOT with Sinkhorn projections (the paper's comparison) converges to the
    same unique plan as with TruncatedNewtonProject (Sec. 2.1: strictly convex
    problem), each within its marginal tolerance."""
    rng = np.random.default_rng(13)
    C = rng.uniform(0, 1, size=(40, 33))
    r = rng.dirichlet(np.ones(40))
    c = rng.dirichlet(np.ones(33))
    a = O.mdot(C, r, c, gamma_i=16.0, gamma_f=512.0, tol_final=1e-8)
    b = O.mdot(C, r, c, gamma_i=16.0, gamma_f=512.0, tol_final=1e-8, projector="sinkhorn")
    assert a.ok and b.ok and b.newton_steps == 0 and b.sinkhorn_iters > 0
    assert O.marginal_l1_error(b.u, b.v, 512.0, C, r, c) <= 1e-8
    Pa, Pb = O.plan(a.u, a.v, 512.0, C), O.plan(b.u, b.v, 512.0, C)
    assert np.abs(Pa - Pb).sum() <= 1e-6


# ---------------- integer outputs of the plan (row argmax, support) ----------------

def test_sqeuclid_ordered_exact_on_integer_points():
    """Integer coordinates make every difference, square and partial sum exact in
    FP64, so the ordered distance must equal the exact integer distance; on
    general points it agrees with the vectorised distance to rounding."""
    rng = np.random.default_rng(70)
    Xi = rng.integers(-1000, 1000, size=(9, 5))
    Yi = rng.integers(-1000, 1000, size=(7, 5))
    exact = np.array([[sum(int(a - b) ** 2 for a, b in zip(x, y)) for y in Yi] for x in Xi])
    D = O.sqeuclid_ordered(Xi.astype(np.float32), Yi.astype(np.float32))
    assert np.array_equal(D, exact.astype(np.float64))
    X = rng.normal(size=(11, 33)).astype(np.float32)
    Y = rng.normal(size=(13, 33)).astype(np.float32)
    np.testing.assert_allclose(O.sqeuclid_ordered(X, Y), O.sqeuclid(X, Y), rtol=1e-14)


def test_row_argmax_is_argmax_of_the_plan_and_breaks_ties_low():
    """The argmax of v_j - gamma C_ij equals the argmax of the formed plan P_ij
    (exp is increasing and u_i is constant along a row) where the maximum is not
    within rounding of a tie; duplicated columns give exact ties, which go to
    the lower index."""
    C, u, v, g = rand_problem(71, 40, 57, gamma=64.0)
    C[:, 20] = C[:, 9]
    v[20] = v[9]
    idx = O.plan_row_argmax(v, g, C)
    P = O.plan(u, v, g, C)
    t = v[None, :] - g * C
    srt = np.sort(t, axis=1)
    clear = srt[:, -1] - srt[:, -2] > 1e-9
    assert np.array_equal(idx[clear], np.argmax(P, axis=1)[clear])
    # rows whose maximum is the duplicated pair report the lower index 9, never 20
    assert not np.any(idx == 20)
    tied = np.argmax(t[:, [9, 20]].max(axis=1)[:, None] >= t, axis=1)
    assert np.sum(idx == 9) >= 0 and np.all((idx != 9) | (tied >= 0))
    # a brute-force scan in Python: first index of the maximum
    for i in range(C.shape[0]):
        best, bj = -math.inf, -1
        for j in range(C.shape[1]):
            if t[i, j] > best:
                best, bj = t[i, j], j
        assert idx[i] == bj


def test_row_argmax_recovers_the_optimal_assignment():
    """Uniform marginals at a large gamma: the EOT plan concentrates on the LP
    optimum, a permutation (Birkhoff; Sec. 2.2's error bound), so the row argmax
    is that permutation when it is unique (checked by brute force)."""
    n = 6
    rng = np.random.default_rng(72)
    C = rng.uniform(0, 1, size=(n, n))
    C /= C.max()
    r = c = np.full(n, 1.0 / n)
    ri, ci = scipy.optimize.linear_sum_assignment(C)
    costs = sorted(C[np.arange(n), list(p)].sum() for p in __import__("itertools").permutations(range(n)))
    assert costs[1] - costs[0] > 1e-3  # a unique optimum with a margin
    res = O.mdot(C, r, c, gamma_i=4.0, gamma_f=2.0 ** 12, tol_final=1e-9)
    idx = O.plan_row_argmax(res.v, res.gamma, C)
    assert np.array_equal(idx[ri], ci)


def test_support_counts_match_thresholded_plan():
    """Counts of the exponent test equal counts of the formed plan above tau away
    from rounding ties, are monotone in tau, give m per row at log tau = -inf and
    0 above the largest entry, and exclude an entry lying exactly on the threshold."""
    C, u, v, g = rand_problem(73, 50, 61, gamma=32.0)
    P = O.plan(u, v, g, C)
    t = (u[:, None] + v[None, :]) - g * C
    for q in (0.1, 0.5, 0.9):
        lt = float(np.quantile(t, q))
        near = np.abs(t - lt) < 1e-9
        cnt = O.plan_support_counts(u, v, g, C, lt)
        ref = (P > math.exp(lt)).sum(axis=1)
        ok_rows = ~near.any(axis=1)
        assert np.array_equal(cnt[ok_rows], ref[ok_rows])
    assert np.all(O.plan_support_counts(u, v, g, C, -math.inf) == C.shape[1])
    assert np.all(O.plan_support_counts(u, v, g, C, float(t.max())) == 0)
    c1 = O.plan_support_counts(u, v, g, C, float(np.quantile(t, 0.3)))
    c2 = O.plan_support_counts(u, v, g, C, float(np.quantile(t, 0.6)))
    assert np.all(c1 >= c2)
    on = float(t[3, 7])
    assert O.plan_support_counts(u, v, g, C, on)[3] == int((t[3] > on).sum())
