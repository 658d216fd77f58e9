"""Plain FP64 CPU oracle for entropic optimal transport solved by the truncated
Newton method of Kemertas, Farahmand and Jepson, "A Truncated Newton Method for
Optimal Transport" (ICLR 2025, arXiv 2504.02067).

THIS MODULE IS TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the
benchmark's CPU-baseline leg may import it. The product (the CUDA library and its
Python binding) never calls it, and it shares no code with the product.

Everything here is float64 numpy, written for a reader to check against the
paper by eye: no blocking, no fusion, no reordering beyond the definitions.
Notation follows the paper: the plan is P(u, v; gamma) = exp(u 1^T + 1 v^T - gamma C)
(Sec. 2.1, Eq. lagrangian-closed-form), gamma is the INVERSE temperature, and
potentials are log-domain (u, not u / gamma).

Readings of places where the paper is silent or ambiguous are marked "Reading".
Each function is pinned by a test in tests/test_oracle_*.py against something
other than itself (closed forms, invariants, finite differences, brute force,
dense linear algebra, the paper's worked example).
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# Plan, marginals, LSE (Sec. 2 "Notation and Definitions"; Eq. lagrangian-closed-form)
# --------------------------------------------------------------------------


def plan(u, v, gamma, C):
    """P_ij = exp(u_i + v_j - gamma C_ij)  (Sec. 2.1, Eq. lagrangian-closed-form)."""
    return np.exp(u[:, None] + v[None, :] - gamma * C)


def row_sum(P):
    """r(P) = P 1  (Sec. 2, notation)."""
    return P.sum(axis=1)


def col_sum(P):
    """c(P) = P^T 1  (Sec. 2, notation)."""
    return P.sum(axis=0)


def lse_r(X):
    """LSE_r(X) = log(exp{X} 1), row-wise log-sum-exp (Sec. 2, notation).

    Written with the usual max shift, which is the same number mathematically.
    """
    m = X.max(axis=1)
    return m + np.log(np.exp(X - m[:, None]).sum(axis=1))


def lse_c(X):
    """LSE_c(X) = log(exp{X^T} 1), column-wise log-sum-exp (Sec. 2, notation)."""
    return lse_r(X.T)


def log_row_sum(u, v, gamma, C):
    """log r(P) = u + LSE_r(1 v^T - gamma C)  (Alg. 3 / Alg. 4, row update)."""
    return u + lse_r(v[None, :] - gamma * C)


def log_col_sum(u, v, gamma, C):
    """log c(P) = v + LSE_c(u 1^T - gamma C)  (Alg. 4, line-search column sums)."""
    return v + lse_c(u[:, None] - gamma * C)


def entropy(x):
    """Shannon entropy H(x) = -sum_i x_i log x_i with 0 log 0 = 0 (Sec. 2)."""
    x = np.asarray(x, dtype=np.float64)
    nz = x > 0
    return float(-(x[nz] * np.log(x[nz])).sum())


def chi2(y, x):
    """chi^2(y | x) = <x, (y / x)^2> - 1  (Sec. 2, notation)."""
    return float((x * (y / x) ** 2).sum() - 1.0)


# --------------------------------------------------------------------------
# Dual objective, gradient, Hessian (Sec. 2.1, Eq. sinkhorn-dual and Eq. hessian)
# --------------------------------------------------------------------------


def dual_objective(u, v, gamma, C, r, c):
    """g(u, v; gamma) = sum_ij P_ij - 1 - <u, r> - <v, c>  (Sec. 2.1, Eq. sinkhorn-dual)."""
    P = plan(u, v, gamma, C)
    return float(P.sum() - 1.0 - u @ r - v @ c)


def dual_gradient(u, v, gamma, C, r, c):
    """grad_u g = r(P) - r, grad_v g = c(P) - c  (Sec. 2.1, text after Eq. sinkhorn-dual)."""
    P = plan(u, v, gamma, C)
    return row_sum(P) - r, col_sum(P) - c


def hessian_matrix(P, s=1.0):
    """The 2n x 2n (discounted) dual Hessian.

    s = 1 gives Eq. hessian; s = sqrt(rho) gives Eq. discounted-hessian (Sec. 3.1).
    """
    n, m = P.shape
    H = np.zeros((n + m, n + m))
    H[:n, :n] = np.diag(row_sum(P))
    H[:n, n:] = s * P
    H[n:, :n] = s * P.T
    H[n:, n:] = np.diag(col_sum(P))
    return H


def hvp(u, v, gamma, C, du, dv, s=1.0):
    """Hessian-vector product [D(r(P)) du + s P dv ; s P^T du + D(c(P)) dv].

    Eq. hessian (s = 1) and Eq. discounted-hessian (s = sqrt(rho)), Sec. 2.1 / 3.1.
    Returns (out_u, out_v, r(P), c(P)).
    """
    P = plan(u, v, gamma, C)
    rP, cP = row_sum(P), col_sum(P)
    return rP * du + s * (P @ dv), s * (P.T @ du) + cP * dv, rP, cP


# --------------------------------------------------------------------------
# The n-variable system F_r(rho) (Sec. 3.1, Eq. matrix-definitions)
# --------------------------------------------------------------------------


def P_rc(P):
    """P_rc = P_r P_c = D(r(P))^-1 P D(c(P))^-1 P^T  (Eq. matrix-definitions)."""
    rP, cP = row_sum(P), col_sum(P)
    return (P / rP[:, None]) @ (P.T / cP[:, None])


def F_r_matrix(P, rho):
    """F_r(rho) = D(r(P)) (I - rho P_rc)  (Eq. matrix-definitions), as a dense matrix."""
    rP = row_sum(P)
    return np.diag(rP) @ (np.eye(P.shape[0]) - rho * P_rc(P))


def F_r_apply(P, rho, x):
    """F_r(rho) x = r(P) * x - rho P (P^T x / c(P)).

    The same operator as F_r_matrix, using D(r(P)) P_rc = P D(c(P))^-1 P^T
    (proof of Lemma fr-properties, Appx. A).
    """
    rP, cP = row_sum(P), col_sum(P)
    return rP * x - rho * (P @ ((P.T @ x) / cP))


def F_r_diag(P, rho):
    """Jacobi preconditioner M = diag(F_r(rho)): r(P)_i - rho sum_j P_ij^2 / c(P)_j.

    Lemma condition-number (Appx. A) uses M = D(diag(F_r(rho))).
    """
    rP, cP = row_sum(P), col_sum(P)
    return rP - rho * ((P * P) @ (1.0 / cP))


# --------------------------------------------------------------------------
# Diagonally preconditioned linear CG (Thm. convergence-alg1; Lemma conv-cg)
# --------------------------------------------------------------------------


@dataclass
class CGResult:
    x: np.ndarray
    iters: int
    res_l1: float
    converged: bool


def pcg(apply_A, b, M, tol_l1, max_iter):
    """Jacobi-preconditioned linear conjugate gradient started at x = 0.

    Standard PCG (the method of Shewchuk 1994, cited for Lemma conv-cg). It stops
    when the L1 norm of the recursively updated residual b - A x is <= tol_l1
    (Sec. 3.1: CG terminates on the L1 norm of the residual).
    """
    x = np.zeros_like(b)
    res = b.copy()
    if np.abs(res).sum() <= tol_l1:
        return CGResult(x, 0, float(np.abs(res).sum()), True)
    z = res / M
    p = z.copy()
    rz = res @ z
    for k in range(1, max_iter + 1):
        q = apply_A(p)
        alpha = rz / (p @ q)
        x = x + alpha * p
        res = res - alpha * q
        res_l1 = float(np.abs(res).sum())
        if res_l1 <= tol_l1:
            return CGResult(x, k, res_l1, True)
        z = res / M
        rz_new = res @ z
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return CGResult(x, max_iter, float(np.abs(res).sum()), False)


# --------------------------------------------------------------------------
# Algorithm 2: NewtonSolve, with the adaptive rho_0 of Appx. B
# --------------------------------------------------------------------------


@dataclass
class NewtonResult:
    d_u: np.ndarray
    rho: float  # the rho of the last CG solve (or rho0 if no CG solve ran)
    cg_iters: int
    cg_solves: int
    rhos: list
    converged: bool


def newton_solve(P, grad_u, grad_l1, eta, rho0=0.0, max_cg=None):
    """Algorithm 2 (NewtonSolve), Sec. 3.1, started from rho0 (Appx. B).

    grad_u   = r(P) - r (the u-block of the dual gradient);
    grad_l1  = ||grad g||_1 (equals ||grad_u g||_1 when c(P) = c, Alg. 4);
    eta      = forcing parameter.
    The discount starts at rho0 and the direction at -D(r(P))^-1 grad_u g; while
    the undiscounted residual ||F_r(1) d_u + grad_u g||_1 exceeds eta ||grad g||_1,
    d_u is replaced by a linear CG solve of F_r(rho) d_u = -grad_u g (from 0, to
    tolerance eta / 4) and 1 - rho is divided by 4.
    Reading: the CG tolerance eta/4 is relative, ||res||_1 <= (eta/4)||grad g||_1
    (Thm. residual uses the same scale). Reading (Appx. B): the returned rho is
    the one the last CG solve used, so that the next call starts from
    max(0, 1 - 4 (1 - rho)), "the second last annealing step".
    """
    n = P.shape[0]
    if max_cg is None:
        max_cg = 4 * n
    rP = row_sum(P)
    rho = rho0
    rho_last = rho0
    d_u = -grad_u / rP
    total = 0
    solves = 0
    rhos = []
    while np.abs(F_r_apply(P, 1.0, d_u) + grad_u).sum() > eta * grad_l1:
        M = F_r_diag(P, rho)
        res = pcg(lambda x: F_r_apply(P, rho, x), -grad_u, M, (eta / 4.0) * grad_l1, max_cg)
        d_u = res.x
        total += res.iters
        solves += 1
        rhos.append(rho)
        rho_last = rho
        if not res.converged:
            return NewtonResult(d_u, rho_last, total, solves, rhos, False)
        rho = 1.0 - (1.0 - rho) / 4.0
        if solves > 60:  # 1 - rho below 4^-60: cannot make progress in FP64
            return NewtonResult(d_u, rho_last, total, solves, rhos, False)
    return NewtonResult(d_u, rho_last, total, solves, rhos, True)


def discounted_hessian_apply(P, rho, du, dv):
    """The discounted Hessian of Eq. discounted-hessian (off-diagonal blocks
    scaled by sqrt(rho)) applied to (du, dv), Sec. 3.1."""
    s = np.sqrt(rho)
    return row_sum(P) * du + s * (P @ dv), s * (P.T @ du) + col_sum(P) * dv


def newton_solve_full(P, grad_u, grad_l1, eta, rho0=0.0, max_cg=None):
    """NewtonSolve with each linear solve on the full discounted system.

    The outer loop is Algorithm 2's (rho annealed 1 - rho <- (1 - rho) / 4, the
    same test ||F_r(1) d_u + grad_u g||_1 <= eta ||grad g||_1, Sec. 3.1), but
    each LinearCGSolve runs PCG on the (n + m)-variable system of the discounted
    Hessian (Eq. discounted-hessian),
        [D(r(P)) d_u + sqrt(rho) P d_v ; sqrt(rho) P^T d_u + D(c(P)) d_v] = [-grad_u g ; 0],
    with the diagonal preconditioner (r(P), c(P)), from 0, to an L1 residual
    <= (eta / 4) ||grad g||_1, and keeps its u-block. Eliminating d_v from the
    second block row leaves F_r(rho) d_u = -grad_u g (the Schur complement,
    Eq. matrix-definitions), so in exact arithmetic both solves give the same
    d_u; each iteration applies one two-sided product (one pass over P) where
    Alg. 2's CG applies F_r(rho) (two passes). A different Krylov iteration, to
    be measured against Algorithm 2, not substituted for it.
    """
    n, m = P.shape
    if max_cg is None:
        max_cg = 4 * (n + m)
    rP, cP = row_sum(P), col_sum(P)
    rho = rho0
    rho_last = rho0
    d_u = -grad_u / rP
    total = 0
    solves = 0
    rhos = []
    b = np.concatenate([-grad_u, np.zeros(m)])
    M = np.concatenate([rP, cP])
    while np.abs(F_r_apply(P, 1.0, d_u) + grad_u).sum() > eta * grad_l1:
        def apply_H(x, rho=rho):
            hu, hv = discounted_hessian_apply(P, rho, x[:n], x[n:])
            return np.concatenate([hu, hv])
        res = pcg(apply_H, b, M, (eta / 4.0) * grad_l1, max_cg)
        d_u = res.x[:n]
        total += res.iters
        solves += 1
        rhos.append(rho)
        rho_last = rho
        if not res.converged:
            return NewtonResult(d_u, rho_last, total, solves, rhos, False)
        rho = 1.0 - (1.0 - rho) / 4.0
        if solves > 60:
            return NewtonResult(d_u, rho_last, total, solves, rhos, False)
    return NewtonResult(d_u, rho_last, total, solves, rhos, True)


def next_rho0(rho_last):
    """rho_0^new = max(0, 1 - 4 (1 - rho^old))  (Appx. B, Eq. for rho_0^new)."""
    return max(0.0, 1.0 - 4.0 * (1.0 - rho_last))


# --------------------------------------------------------------------------
# Algorithm 3: ChiSinkhorn
# --------------------------------------------------------------------------


def chi_sinkhorn(u, v, gamma, C, r, c, log_rP, eps_chi, max_iter=100000):
    """Algorithm 3 (ChiSinkhorn), Sec. 3.1.

    while chi^2(r | r(P)) > eps_chi:
        u <- u + log r - log r(P)
        v <- log c - LSE_c(u 1^T - gamma C)
        log r(P) <- u + LSE_r(1 v^T - gamma C)
    Returns (u, v, log r(P), iterations).
    """
    it = 0
    while chi2(r, np.exp(log_rP)) > eps_chi and it < max_iter:
        u = u + np.log(r) - log_rP
        v = np.log(c) - lse_c(u[:, None] - gamma * C)
        log_rP = log_row_sum(u, v, gamma, C)
        it += 1
    return u, v, log_rP, it


def sinkhorn_project(u, v, gamma, C, r, c, eps, max_iter=1_000_000):
    """Sinkhorn as the Bregman projection of Alg. 1 (MDOT-Sinkhorn, the paper's
    main comparison, Sec. 4): the column fix, then alternating row and column
    fixes while ||grad g||_1 = ||r - r(P)||_1 > eps, then the same last row step
    as Alg. 4. Returns (u, v, ProjectStats) with sinkhorn_iters counted."""
    st = ProjectStats()
    log_r, log_c = np.log(r), np.log(c)
    v = log_c - lse_c(u[:, None] - gamma * C)
    log_rP = log_row_sum(u, v, gamma, C)
    grad_l1 = float(np.abs(r - np.exp(log_rP)).sum())
    while grad_l1 > eps:
        if st.sinkhorn_iters >= max_iter:
            st.ok = False
            break
        u = u + log_r - log_rP
        v = log_c - lse_c(u[:, None] - gamma * C)
        log_rP = log_row_sum(u, v, gamma, C)
        grad_l1 = float(np.abs(r - np.exp(log_rP)).sum())
        st.sinkhorn_iters += 1
    u = u + log_r - log_rP
    return u, v, st


# --------------------------------------------------------------------------
# Algorithm 4: TruncatedNewtonProject
# --------------------------------------------------------------------------


@dataclass
class ProjectStats:
    newton_steps: int = 0
    cg_iters: int = 0
    sinkhorn_iters: int = 0
    ls_trials: int = 0
    deltas: list = field(default_factory=list)
    rho_last: float = 0.0
    ok: bool = True


def armijo_lhs(u, v, d_u, d_v, alpha, gamma, C):
    """||c(P(alpha))||_1 - 1 with log c(P(alpha)) = v + a d_v + LSE_c((u + a d_u) 1^T - gamma C).

    Alg. 4, line-search lines; Lemma sufficient-decrease (Appx. A) shows this
    equals the Armijo test on g when c(P) = c. Returns (lhs, log c(P(alpha))).
    """
    log_cPa = log_col_sum(u + alpha * d_u, v + alpha * d_v, gamma, C)
    return float(np.exp(log_cPa).sum() - 1.0), log_cPa


def truncated_newton_project(u, v, gamma, C, r, c, eps, rho_last=0.0,
                             max_newton=200, max_ls=40, max_cg=None, newton=None):
    """Algorithm 4 (TruncatedNewtonProject), Sec. 3.2, projecting onto U(r, c) to tolerance eps.

    Opening: the column fix v <- log c - LSE_c(u 1^T - gamma C) (so c(P) = c), then
    log r(P) <- u + LSE_r(1 v^T - gamma C). While ||grad g||_1 = ||r - r(P)||_1 > eps:
    ChiSinkhorn with eps_chi = eps^(2/5); the forcing parameter
    eta <- max(||grad g||_1, 0.8 eps / ||grad g||_1); d_u <- NewtonSolve(grad_u g,
    P_rc, r(P), eta) and d_v <- -P_c d_u; a backtracking line search on the Armijo
    test (factor 0.5, c_1 = 0.01); the update u <- u + alpha d_u, v <- v + alpha d_v
    and the column fix v <- v + log c - log c(P); log r(P) at the new point.
    Closing: one last row step u <- u + log r - log r(P).
    rho_last carries the adaptive discount of Appx. B between NewtonSolve calls
    (0 before the first call). Reading: a NewtonSolve call that runs no CG solve
    leaves rho_last unchanged. newton: the NewtonSolve used for d_u
    (newton_solve, Algorithm 2, by default; newton_solve_full for the variant
    whose linear solves run on the full discounted system).
    delta_k (Eq. delta_k-ratio) is recorded for every Newton step.
    """
    st = ProjectStats(rho_last=rho_last)
    log_r, log_c = np.log(r), np.log(c)
    v = log_c - lse_c(u[:, None] - gamma * C)
    log_rP = log_row_sum(u, v, gamma, C)
    grad_l1 = float(np.abs(r - np.exp(log_rP)).sum())
    while grad_l1 > eps:
        if st.newton_steps >= max_newton:
            st.ok = False
            break
        u, v, log_rP, it = chi_sinkhorn(u, v, gamma, C, r, c, log_rP, eps ** 0.4)
        st.sinkhorn_iters += it
        rP = np.exp(log_rP)
        grad_u = rP - r
        grad_l1 = float(np.abs(grad_u).sum())
        if grad_l1 <= eps:
            break
        eta = max(grad_l1, 0.8 * eps / grad_l1)
        P = plan(u, v, gamma, C)
        nres = (newton or newton_solve)(P, grad_u, grad_l1, eta, next_rho0(st.rho_last), max_cg)
        st.cg_iters += nres.cg_iters
        if nres.cg_solves:
            st.rho_last = nres.rho
        if not nres.converged:
            st.ok = False
        # Reading: the direction is taken modulo the gauge (u + k 1, v - k 1 give
        # the same P, Sec. 2.1): d_u <- d_u - k 1 with k = <r(P), d_u> / sum r(P).
        # (d_u - k 1, d_v + k 1) moves P, g and every later iterate exactly as
        # (d_u, d_v) does; a large k only costs precision in d_v = -P_c d_u.
        d_u = nres.d_u - (rP @ nres.d_u) / rP.sum()
        d_v = -(P.T @ d_u) / col_sum(P)
        slope = float(-grad_u @ d_u)  # <-grad_u g, d_u>
        # Reading: the test's left side is taken relative to its computed value at
        # alpha = 0, which is 0 in exact arithmetic (c(P) = c after the column fixes,
        # sum c = 1); measuring it removes the rounding offset of sum P - 1, which
        # near the final tolerance can exceed the sufficient decrease itself.
        lhs0, _ = armijo_lhs(u, v, d_u, d_v, 0.0, gamma, C)
        alpha = 1.0
        lhs, log_cPa = armijo_lhs(u, v, d_u, d_v, alpha, gamma, C)
        lhs -= lhs0
        st.ls_trials += 1
        while lhs > 0.99 * alpha * slope:
            alpha *= 0.5
            if st.ls_trials >= max_ls * (st.newton_steps + 1):
                st.ok = False
                break
            lhs, log_cPa = armijo_lhs(u, v, d_u, d_v, alpha, gamma, C)
            lhs -= lhs0
            st.ls_trials += 1
        u = u + alpha * d_u
        v = v + alpha * d_v
        v = v + log_c - log_cPa
        log_rP = log_row_sum(u, v, gamma, C)
        new_l1 = float(np.abs(r - np.exp(log_rP)).sum())
        st.deltas.append((grad_l1 - new_l1) / ((1.0 - eta) * grad_l1))
        grad_l1 = new_l1
        st.newton_steps += 1
        if not st.ok:
            break
    u = u + log_r - log_rP
    return u, v, st


# --------------------------------------------------------------------------
# Algorithm 1: MDOT with adaptive q (Sec. 3.3) and asymmetric smoothing (Sec. 3.4)
# --------------------------------------------------------------------------


def smooth_marginals(r, c, eps_d, w_r=0.45):
    """Asymmetric smoothing (Sec. 3.4):
    r~ = (1 - w_r eps_d) r + (w_r eps_d / n) 1,  c~ = (1 - w_c eps_d) c + (w_c eps_d / n) 1,
    with w_r + w_c = 1/2 (combined mixing weight eps_d / 2, Sec. 2.2).
    Reading: w_r = 0.45 (Table 2's best column equals Table 1's adaptive run).
    Reading: the uniform term of c~ uses the length of c.
    """
    w_c = 0.5 - w_r
    n, m = r.shape[0], c.shape[0]
    return ((1.0 - w_r * eps_d) * r + (w_r * eps_d / n),
            (1.0 - w_c * eps_d) * c + (w_c * eps_d / m))


def adjust_schedule(q, delta_min):
    """AdjustSchedule (Sec. 3.3): q <- min(2, q^2) if delta_min > 0.95;
    q <- sqrt(q) if delta_min < 0.8; else unchanged.
    Reading: a stage without Newton steps has delta_min = +inf.
    """
    if delta_min > 0.95:
        return min(2.0, q * q)
    if delta_min < 0.8:
        return math.sqrt(q)
    return q


@dataclass
class SolveResult:
    u: np.ndarray
    v: np.ndarray
    gamma: float
    stages: int
    newton_steps: int
    cg_iters: int
    sinkhorn_iters: int
    ls_trials: int
    gammas: list
    ok: bool
    records: list = field(default_factory=list)  # one dict per stage (Alg. 1 loop)


def mdot(C, r, c, gamma_i=2.0 ** 4, gamma_f=2.0 ** 12, p=1.5, q1=2.0, w_r=0.45,
         tol_final=1e-6, round_gamma=None, max_stages=200, max_newton=200, max_cg=None,
         projector="newton", newton=None):
    """Algorithm 1 (MDOT) driving Algorithm 4, Sec. 2.2 and Sec. 3.

    It starts at gamma^(1) = min(gamma_i, gamma_f) with q^(1) = q and gamma^(0) = 0.
    Each stage t: done when gamma^(t) = gamma_f; eps_d = min(H(r), H(c)) / gamma^p;
    r~, c~ = SmoothMarginals(r, c, eps_d); at t = 1 the potentials start at
    (log r~, log c~); z^(t) <- BregmanProject(z^(t), gamma, C, r~, c~, eps_d / 2);
    q <- AdjustSchedule(q); gamma^(t+1) = min(q gamma^(t), gamma_f); the next stage
    starts from the extrapolation z^(t) + (gamma^(t+1) - gamma^(t)) /
    (gamma^(t) - gamma^(t-1)) (z^(t) - z^(t-1)). Output: the last projected z.
    Reading: in the final stage eps_d <- min(eps_d, 2 tol_final / 3). Smoothing
    moves r and c by at most 2 (w_r + w_c) eps_d = eps_d in L1, and the projection
    to eps_d / 2 followed by the last row step leaves ||c(P) - c~||_1 <= eps_d / 2,
    so the marginal L1 error against the unsmoothed r, c is <= 1.5 eps_d <= tol_final.
    Reading: round_gamma (e.g. a round-to-float32 map) is applied to every
    gamma^(t) so that a reduced-precision solver and this oracle see the same
    temperatures.
    projector="sinkhorn" replaces Alg. 4 by sinkhorn_project (MDOT-Sinkhorn); a
    stage then has no Newton steps, so AdjustSchedule sees delta_min = +inf.
    """
    rg = round_gamma or (lambda g: g)
    n, m = C.shape
    if n == 1 or m == 1:
        # Reading: with one row or one column U(r, c) = {r c^T}, and Alg. 1's
        # tolerance eps_d = min(H(r), H(c)) / gamma^p is 0, which no finite-
        # precision iteration meets. The potentials of r c^T at gamma_f are
        # returned directly (a zero mass is clamped to 1e-300).
        gf = rg(gamma_f)
        lr = np.log(np.maximum(r, 1e-300))
        lc = np.log(np.maximum(c, 1e-300))
        if n == 1:
            u, v = lr.copy(), lc + gf * C[0, :]
        else:
            u, v = lr + gf * C[:, 0], lc.copy()
        return SolveResult(u, v, gf, 0, 0, 0, 0, 0, [], True)
    H = min(entropy(r), entropy(c))
    gamma_f = rg(gamma_f)
    gamma = rg(min(gamma_i, gamma_f))
    gamma_prev = 0.0
    q = q1
    z_prev = None
    z = None
    rho_last = 0.0
    t = 1
    totals = dict(newton=0, cg=0, sk=0, ls=0)
    gammas = []
    records = []
    ok = True
    while True:
        done = gamma == gamma_f
        eps_d = H / gamma ** p
        if done:
            eps_d = min(eps_d, 2.0 * tol_final / 3.0)
        rs, cs = smooth_marginals(r, c, eps_d, w_r)
        if t == 1:
            z = (np.log(rs), np.log(cs))
            z_prev = z
        if projector == "sinkhorn":
            u, v, st = sinkhorn_project(z[0], z[1], gamma, C, rs, cs, eps_d / 2.0)
        else:
            u, v, st = truncated_newton_project(z[0], z[1], gamma, C, rs, cs, eps_d / 2.0,
                                                rho_last, max_newton=max_newton, max_cg=max_cg,
                                                newton=newton)
        rho_last = st.rho_last
        ok = ok and st.ok
        totals["newton"] += st.newton_steps
        totals["cg"] += st.cg_iters
        totals["sk"] += st.sinkhorn_iters
        totals["ls"] += st.ls_trials
        gammas.append(gamma)
        z = (u, v)
        dmin = min(st.deltas) if st.deltas else math.inf
        q = adjust_schedule(q, dmin)
        records.append(dict(gamma=gamma, eps=eps_d / 2.0, delta_min=dmin, q_next=q,
                            newton_steps=st.newton_steps, cg_iters=st.cg_iters,
                            ls_trials=st.ls_trials, sinkhorn_iters=st.sinkhorn_iters))
        gamma_next = rg(min(q * gamma, gamma_f))
        ratio = (gamma_next - gamma) / (gamma - gamma_prev)
        z_next = (z[0] + ratio * (z[0] - z_prev[0]), z[1] + ratio * (z[1] - z_prev[1]))
        if done or t >= max_stages or not ok:
            ok = ok and done
            break
        z_prev, z = z, z_next
        gamma_prev, gamma = gamma, gamma_next
        t += 1
    return SolveResult(z[0], z[1], gamma, t, totals["newton"], totals["cg"], totals["sk"],
                       totals["ls"], gammas, ok, records)


# --------------------------------------------------------------------------
# Independent reference: plain log-domain Sinkhorn (special case of Alg. 3)
# --------------------------------------------------------------------------


def sinkhorn_log(C, r, c, gamma, tol=1e-13, max_iter=1_000_000, u=None, v=None):
    """Alternating log-domain Sinkhorn at fixed gamma (no annealing), run until
    ||grad g||_1 <= tol. Its limit is the unique EOT optimum (Sec. 2.1)."""
    n, m = C.shape
    u = np.log(r) if u is None else u
    v = np.log(c) if v is None else v
    for it in range(max_iter):
        v = np.log(c) - lse_c(u[:, None] - gamma * C)
        u = np.log(r) - lse_r(v[None, :] - gamma * C)
        if it % 10 == 0:
            P = plan(u, v, gamma, C)
            if np.abs(col_sum(P) - c).sum() <= tol:
                break
    return u, v


# --------------------------------------------------------------------------
# Results derived from a solution
# --------------------------------------------------------------------------


def marginal_l1_error(u, v, gamma, C, r, c):
    """||r(P) - r||_1 + ||c(P) - c||_1 of the unrounded plan."""
    P = plan(u, v, gamma, C)
    return float(np.abs(row_sum(P) - r).sum() + np.abs(col_sum(P) - c).sum())


def transport_cost(u, v, gamma, C):
    """<P, C> of the unrounded plan."""
    return float((plan(u, v, gamma, C) * C).sum())


def primal_value(P, C, gamma):
    """<P, C> - H(P) / gamma with H(P) = -sum P log P  (Eq. sinkhorn-primal)."""
    nz = P > 0
    return float((P * C).sum() + (P[nz] * np.log(P[nz])).sum() / gamma)


def round_to_polytope(F, r, c):
    """Round(F, r, c): Algorithm 2 of Altschuler, Weed and Rigollet (2017), which
    Alg. 1 applies to its output. Scales rows down to r, then columns down to c, then adds
    the rank-one correction err_r err_c^T / ||err_r||_1."""
    x = np.minimum(r / row_sum(F), 1.0)
    F = F * x[:, None]
    y = np.minimum(c / col_sum(F), 1.0)
    F = F * y[None, :]
    er = r - row_sum(F)
    ec = c - col_sum(F)
    s = np.abs(er).sum()
    if s > 0:
        F = F + np.outer(er, ec) / s
    return F


def gauge_fix(u, v):
    """Shift (u + k, v - k) so that sum(u) = sum(v); P is unchanged (Sec. 2.1 footnote)."""
    k = (v.sum() - u.sum()) / (u.shape[0] + v.shape[0])
    return u + k, v - k


# --------------------------------------------------------------------------
# Costs
# --------------------------------------------------------------------------


def sqeuclid(X, Y):
    """D_ij = |x_i - y_j|^2 in float64 from the given points."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    return ((X[:, None, :] - Y[None, :, :]) ** 2).sum(axis=2)


def sqeuclid_rows(X, Y, rows):
    """Selected rows of D, D_ij = |x_i - y_j|^2, for sampled checks at large n."""
    X = np.asarray(X, dtype=np.float64)[rows]
    Y = np.asarray(Y, dtype=np.float64)
    out = np.empty((X.shape[0], Y.shape[0]))
    for k, x in enumerate(X):
        out[k] = ((Y - x[None, :]) ** 2).sum(axis=1)
    return out


def sqeuclid_scale(X, Y, block=4096):
    """s_C = 1 / max_ij |x_i - y_j|^2 (cost normalised to max 1, Sec. 4.1)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    best = 0.0
    for a in range(0, X.shape[0], block):
        Xa = X[a:a + block]
        d = (Xa * Xa).sum(1)[:, None] + (Y * Y).sum(1)[None, :] - 2.0 * Xa @ Y.T
        i, j = np.unravel_index(np.argmax(d), d.shape)
        # re-evaluate the arg-max pair (and its neighbours in value) exactly
        cand = np.argsort(d.ravel())[-8:]
        for idx in cand:
            ii, jj = np.unravel_index(idx, d.shape)
            best = max(best, float(((Xa[ii] - Y[jj]) ** 2).sum()))
    return 1.0 / best


# --------------------------------------------------------------------------
# Differentiation of the EOT value (envelope theorem on the Lagrangian, Appx. A)
# --------------------------------------------------------------------------


def eot_value(u, v, gamma, C):
    """F* = <P*, C> - H(P*) / gamma at the optimum, computed from the plan."""
    return primal_value(plan(u, v, gamma, C), C, gamma)


def eot_grads_dense(u, v, gamma, C):
    """dF*/dC = P*, dF*/dr = u*/gamma, dF*/dc = v*/gamma (up to constants that
    vanish on simplex-tangent directions)."""
    return plan(u, v, gamma, C), u / gamma, v / gamma


def eot_grads_points(u, v, gamma, X, Y, s_C):
    """For C_ij = s_C |x_i - y_j|^2 with s_C held constant:
    dF*/dx_i = 2 s_C sum_j P_ij (x_i - y_j),  dF*/dy_j = 2 s_C sum_i P_ij (y_j - x_i)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    C = s_C * sqeuclid(X, Y)
    P = plan(u, v, gamma, C)
    rP, cP = row_sum(P), col_sum(P)
    dX = 2.0 * s_C * (rP[:, None] * X - P @ Y)
    dY = 2.0 * s_C * (cP[:, None] * Y - P.T @ X)
    return dX, dY


# --------------------------------------------------------------------------
# Integer outputs of the plan: row argmax and support (Reading G12 of the
# readings list: lowest index on ties, compared bit-exactly). The decisions are
# taken on the FP64 exponent in a fixed order of rounded operations.
# --------------------------------------------------------------------------


def sqeuclid_ordered(X, Y):
    """D_ij = sum_k (x_ik - y_jk)^2 in float64 with the coordinates added in order
    k = 0, 1, ..., d - 1, every difference, square and partial sum rounded on its
    own (numpy elementwise operations: no fused multiply-add, no pairwise
    reordering). This is the fixed evaluation order of the integer outputs."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    D = np.zeros((X.shape[0], Y.shape[0]))
    for k in range(X.shape[1]):
        diff = X[:, k][:, None] - Y[:, k][None, :]
        D = D + diff * diff
    return D


def plan_row_argmax(v, gamma, C):
    """argmax_j P_ij for every row i, P = P(u, v; gamma) (Eq. lagrangian-closed-form).
    u_i is constant along row i and exp is increasing, so the argmax is that of
    t_ij = v_j - gamma C_ij (the product and the difference each rounded).
    Ties go to the lowest index (np.argmax returns the first occurrence)."""
    t = v[None, :] - gamma * C
    return np.argmax(t, axis=1).astype(np.int64)


def plan_support_counts(u, v, gamma, C, log_tau):
    """#{j : P_ij > tau} for every row i, decided on the exponent:
    (u_i + v_j) - gamma C_ij > log tau (each operation rounded, in that order)."""
    t = (u[:, None] + v[None, :]) - gamma * C
    return (t > log_tau).sum(axis=1).astype(np.int64)


# --------------------------------------------------------------------------
# Brute force (Birkhoff: the LP optimum over U(1/n, 1/n) is a permutation)
# --------------------------------------------------------------------------


def brute_force_assignment(C):
    """min over permutations sigma of (1/n) sum_i C_{i sigma(i)}; n <= 8."""
    n = C.shape[0]
    best = math.inf
    for perm in itertools.permutations(range(n)):
        best = min(best, C[np.arange(n), list(perm)].sum() / n)
    return best
