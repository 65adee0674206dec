"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test ties an oracle function to something other than itself:
closed forms, invariants, brute force with a pseudoinverse, an independent
factorisation route, printed values of the paper, or finite differences.
Runs on the CPU only (no GPU marker).
"""
import math
import os

import numpy as np
import pytest

from oracle import feti_oracle as O
from paper_2502_08382_gb300.problems import make_config, make_problem, make_W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.fixture(scope="module")
def cfg1():
    return make_config(1)


@pytest.fixture(scope="module")
def tiny_el():
    return make_problem(dim=3, physics="elasticity", cuts=[[2, 3]] * 3, material="density", seed=3)


# ------------------------------------------------------------- generator pins


@pytest.mark.parametrize("row", _golden("multiplier_counts.txt"))
def test_multiplier_counts(row):
    k, nlam, mmin, mmax = map(int, row)
    P = make_config(k)
    assert P.n_lambda == nlam
    ms = [s.m for s in P.subs]
    assert min(ms) == mmin and max(ms) == mmax


def test_gluing_structure(cfg1):
    """Each B row holds one signed unit; every multiplier is either a Dirichlet
    row (one +1 entry) or a gluing row (+1 on the lower id, -1 on the higher)
    between copies of the same global DOF (eqs. 2-3, Total FETI)."""
    P = cfg1
    entries = [[] for _ in range(P.n_lambda)]
    for i, s in enumerate(P.subs):
        assert np.all(np.diff(s.B_lambda) > 0)
        assert set(np.unique(s.B_sign)) <= {-1.0, 1.0}
        for lam, dof, sg in zip(s.B_lambda, s.B_dof, s.B_sign):
            entries[lam].append((i, int(s.l2g[dof]), sg))
    dirichlet = set(P.dirichlet_dofs.tolist())
    for e in entries:
        assert len(e) in (1, 2)
        if len(e) == 1:
            assert e[0][2] == 1.0 and e[0][1] in dirichlet
        else:
            (i, g1, s1), (j, g2, s2) = sorted(e)
            assert i < j and g1 == g2 and s1 == 1.0 and s2 == -1.0


def test_kernel_basis(cfg1, tiny_el):
    for P in (cfg1, tiny_el):
        for s in P.subs:
            K = O.K_dense(s)
            assert np.allclose(K, K.T, atol=0)
            assert np.abs(K @ s.R).max() <= 1e-12 * np.abs(K).max()


# ------------------------------------------------------------- regularisation


@pytest.mark.parametrize("which", ["heat", "elasticity"])
def test_generalised_inverse(which, cfg1, tiny_el):
    """K K_reg^{-1} K = K (the defining property of K^+, eq. 5) with exactly
    d penalised DOFs.  A 9-DOF (three whole nodes) penalty breaks it."""
    P = cfg1 if which == "heat" else tiny_el
    for s in P.subs[:4]:
        K = O.K_dense(s)
        Kr = O.K_reg(s, K)
        err = np.linalg.norm(K @ np.linalg.solve(Kr, K) - K) / np.linalg.norm(K)
        assert err < 1e-12
    if which == "elasticity":
        s = P.subs[0]
        K = O.K_dense(s)
        nodes = sorted(set(int(x) // 3 for x in s.fix_dofs))
        all9 = np.array([3 * q + c for q in nodes for c in range(3)])
        Kr = K.copy()
        Kr[all9, all9] += O.rho_pen(K)
        err = np.linalg.norm(K @ np.linalg.solve(Kr, K) - K) / np.linalg.norm(K)
        assert err > 1e-6


# ------------------------------------------------------------- local dual operator


def test_F_two_routes(cfg1, tiny_el):
    """Cholesky route (eq. 9) and Schur-complement route (eq. 13) agree."""
    for P in (cfg1, tiny_el):
        for s in P.subs[:4]:
            F1 = O.local_F(s)
            F2 = O.local_F_schur(s)
            assert np.linalg.norm(F1 - F2) <= 1e-12 * np.linalg.norm(F1)


def test_F_symmetric_psd(cfg1, tiny_el):
    for P in (cfg1, tiny_el):
        for s in P.subs[:4]:
            F = O.local_F(s)
            assert np.allclose(F, F.T, rtol=0, atol=1e-14 * np.abs(F).max())
            ev = np.linalg.eigvalsh(F)
            assert ev.min() >= -1e-12 * ev.max()


@pytest.mark.parametrize("dim,phys,ne", [(2, "heat", 2), (2, "heat", 3), (3, "heat", 2), (3, "elasticity", 2),
                                         (3, "elasticity", 3)])
def test_F_pinv_brute_force(dim, phys, ne):
    """Projected F from K_reg^{-1} equals projected F from the Moore-Penrose
    pseudoinverse: any two generalised inverses differ by terms in R, which
    P_i = I - G_i G_i^+ (G_i = B_i R_i) annihilates."""
    P = make_problem(dim=dim, physics=phys, cuts=[[ne, ne]] * dim, material="lognormal", sigma=0.7, seed=11)
    for s in P.subs:
        B = O.B_dense(s)
        K = O.K_dense(s)
        Freg = O.local_F(s)
        Fpinv = B @ np.linalg.pinv(K, rcond=1e-12) @ B.T
        G = B @ s.R
        Pi = np.eye(s.m) - G @ np.linalg.pinv(G)
        a = Pi @ Freg @ Pi
        b = Pi @ Fpinv @ Pi
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b)


def test_F_explicit_vs_implicit_application(cfg1):
    """Explicit F_i p (eq. 12) equals the right-to-left application
    B (K_reg^{-1} (B^T p)) with a sparse LU of K_reg (eq. 11)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    for s in cfg1.subs[:3]:
        p = np.random.default_rng(5).normal(size=s.m)
        Kr = sp.csc_matrix(O.K_reg(s))
        z = spla.splu(Kr).solve(O.B_dense(s).T @ p)
        q_impl = O.B_dense(s) @ z
        q_expl = O.local_F(s) @ p
        assert np.linalg.norm(q_impl - q_expl) <= 1e-12 * np.linalg.norm(q_expl)


# ------------------------------------------------------------- global solve


def test_closed_form_poisson(cfg1):
    """Workload 1: -u'' = 1, u(0) = 0, natural elsewhere gives u = x - x^2/2;
    Q1 with consistent load is nodally exact for this y-independent solution."""
    X = cfg1.global_solution_coords()[:, 0]
    exact = X - X ** 2 / 2
    um = O.monolithic_solve(cfg1)
    assert np.abs(um - exact).max() < 1e-12
    res = O.feti_solve(cfg1, tol=1e-12)
    for s, u in zip(cfg1.subs, res["u"]):
        assert np.abs(u - exact[s.l2g]).max() < 1e-10 * 0.5


def test_feti_matches_monolithic_lognormal():
    P = make_problem(dim=2, physics="heat", cuts=[[6, 7, 5]] * 2, material="lognormal", sigma=1.0, seed=2)
    um = O.monolithic_solve(P)
    res = O.feti_solve(P, tol=1e-13)
    err = max(np.abs(u - um[s.l2g]).max() for s, u in zip(P.subs, res["u"]))
    assert err <= 1e-10 * np.abs(um).max()


def test_feti_matches_monolithic_elasticity():
    P = make_problem(dim=3, physics="elasticity", cuts=[[3, 2]] * 3, material="const", seed=0)
    um = O.monolithic_solve(P)
    res = O.feti_solve(P, tol=1e-13)
    err = max(np.abs(u - um[s.l2g]).max() for s, u in zip(P.subs, res["u"]))
    assert err <= 1e-10 * np.abs(um).max()


def test_pcpg_invariants(cfg1):
    """G^T lambda_k = e at every iterate (the projector keeps the
    solvability condition, eq. 4), and B u = c at convergence (eq. 3)."""
    Fs = [O.local_F(s) for s in cfg1.subs]
    lam, its, info = O.pcpg(cfg1, Fs, tol=1e-12, history=True)
    e = info["e"]
    for h in info["hist"]:
        assert np.abs(h).max() <= 1e-12 * max(1.0, np.abs(e).max())
    alpha = O.alpha_from_lambda(cfg1, Fs, lam, info["P"], info["d"])
    us = O.primal_solution(cfg1, lam, alpha)
    Bu = np.zeros(cfg1.n_lambda)
    for s, u in zip(cfg1.subs, us):
        np.add.at(Bu, s.B_lambda, s.B_sign * u[s.B_dof])
    assert np.abs(Bu - cfg1.c).max() < 1e-10


# ------------------------------------------------------------- sensitivities


def test_gradient_vs_central_fd(tiny_el):
    """dL/drho_e from -<Z^T dK_e Z, W> against central differences
    (h = 1e-6) of L = <W_i, F_i> with rho_pen frozen.  The numerator
    L(rho + h) - L(rho - h) is taken through the resolvent identity
    (loss_difference, pinned against the plain difference below): subtracting
    two loss values of size ~1e2-1e5 loses about seven digits at h = 1e-6,
    which leaves the plain quotient only ~1e-6 accurate."""
    P = tiny_el
    Ws = make_W(P, seed=0)
    rng = np.random.default_rng([0, 4])
    for si in (0, 5):
        s = P.subs[si]
        rho = O.rho_pen(O.K_dense(s))
        elems = rng.choice(s.elem_dofs.shape[0], size=4, replace=False)
        g = O.gradient_sub(s, Ws[si], P.K_ref, elems=elems, Kr=O.K_reg(s, rho=rho))
        for k, e in enumerate(elems):
            th = (s.elem_coef[e] / 1.0) ** (1.0 / 3.0)  # rho_e with E_e = rho_e^3
            hh = 1e-6
            Kp = O.perturbed_K_reg(s, e, (th + hh) ** 3 - th ** 3, P.K_ref, rho)
            Km = O.perturbed_K_reg(s, e, (th - hh) ** 3 - th ** 3, P.K_ref, rho)
            dc = (th + hh) ** 3 - (th - hh) ** 3
            fd = O.loss_difference(s, Ws[si], Kp, Km, e, dc, P.K_ref) / (2 * hh)
            assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd))
            plain = (O.loss_sub(s, Ws[si], Kp) - O.loss_sub(s, Ws[si], Km)) / (2 * hh)
            assert abs(plain - g[k]) <= 1e-4 * max(1.0, abs(plain))


def test_loss_difference_identity(tiny_el):
    """The resolvent form of L(K+) - L(K-) equals the plain difference of the
    two losses on a step large enough for the plain difference to be exact
    to ~1e-10."""
    P = tiny_el
    Ws = make_W(P, seed=2)
    s = P.subs[3]
    rho = O.rho_pen(O.K_dense(s))
    e = 5
    dc = 0.05 * s.elem_coef[e]
    Kp = O.perturbed_K_reg(s, e, dc, P.K_ref, rho)
    Km = O.perturbed_K_reg(s, e, -dc, P.K_ref, rho)
    a = O.loss_difference(s, Ws[3], Kp, Km, e, 2 * dc, P.K_ref)
    b = O.loss_sub(s, Ws[3], Kp) - O.loss_sub(s, Ws[3], Km)
    assert abs(a - b) <= 1e-9 * abs(b)


def test_loss_difference_lowrank_matches_two_factorisations(tiny_el):
    """The Woodbury form (one factorisation, element-rank update) gives the same
    L(K+) - L(K-) as the resolvent form with two factorisations, at a large step
    (where both are checked against the plain difference) and at h = 1e-6 in
    rho_e with E_e = rho_e^3 (the central-difference step), on elements of
    several subdomains."""
    import scipy.linalg as sla
    P = tiny_el
    Ws = make_W(P, seed=2)
    for si, e in ((3, 5), (0, 0), (7, 11)):
        s = P.subs[si]
        rho = O.rho_pen(O.K_dense(s))
        cho = sla.cho_factor(O.K_reg(s), lower=True)
        th = s.elem_coef[e] ** (1.0 / 3.0)
        for dp, dm in ((0.05 * s.elem_coef[e], -0.05 * s.elem_coef[e]),
                       ((th + 1e-6) ** 3 - th ** 3, (th - 1e-6) ** 3 - th ** 3)):
            Kp = O.perturbed_K_reg(s, e, dp, P.K_ref, rho)
            Km = O.perturbed_K_reg(s, e, dm, P.K_ref, rho)
            a = O.loss_difference(s, Ws[si], Kp, Km, e, dp - dm, P.K_ref)
            b = O.loss_difference_lowrank(s, Ws[si], cho, e, dp, dm, P.K_ref)
            assert abs(a - b) <= 1e-9 * abs(a), (si, e, a, b)


def test_schur_boundary_and_dirichlet_preconditioner(tiny_el, cfg1):
    """S_i (Schur complement of K_i onto the B-touched DOFs T) is symmetric PSD,
    annihilates the rigid modes restricted to T (K R = 0 and the interior
    rows of K R = 0 give S R_T = 0), and is the minimum energy over interior
    extensions: v_T^T S v_T = min_{v_I} v^T K v, with any other v_I giving
    more.  The scaled Dirichlet M is symmetric PSD, and the PCPG it
    preconditions reaches the unpreconditioned solution in fewer iterations."""
    rng = np.random.default_rng(21)
    for s in (tiny_el.subs[0], tiny_el.subs[5], cfg1.subs[6]):
        K = O.K_dense(s)
        T, S = O.schur_boundary(s, K)
        assert np.allclose(S, S.T, atol=1e-12 * np.abs(S).max())
        assert np.linalg.eigvalsh(S).min() >= -1e-10 * np.abs(S).max()
        if s.R.shape[1]:
            assert np.abs(S @ s.R[T]).max() <= 1e-9 * np.abs(S).max() * np.abs(s.R).max()
        I = np.setdiff1d(np.arange(s.n), T)
        vT = rng.normal(size=T.size)
        vI = -np.linalg.solve(K[np.ix_(I, I)], K[np.ix_(I, T)] @ vT)
        v = np.zeros(s.n)
        v[T], v[I] = vT, vI
        e_min = v @ K @ v
        assert abs(vT @ S @ vT - e_min) <= 1e-10 * abs(e_min)
        v[I] += 1e-3 * rng.normal(size=I.size)
        assert v @ K @ v > e_min
    M = O.dirichlet_M(cfg1)
    assert np.allclose(M, M.T, atol=1e-12 * np.abs(M).max())
    assert np.linalg.eigvalsh(M).min() >= -1e-10 * np.abs(M).max()
    plain = O.feti_solve(cfg1, tol=1e-12)
    res = O.feti_solve(cfg1, tol=1e-12, precond="dirichlet")
    assert res["iterations"] < plain["iterations"], (res["iterations"], plain["iterations"])
    err = max(np.abs(a - b).max() for a, b in zip(res["u"], plain["u"]))
    assert err <= 1e-10 * max(np.abs(u).max() for u in plain["u"])


# ------------------------------------------------------------- paper's printed numbers


@pytest.mark.parametrize("row", _golden("break_even_fig4.txt"))
def test_break_even_formula(row):
    from paper_2502_08382_gb300.metrics import break_even
    name = row[0]
    pe, ae, pi, ai, n = map(float, row[1:])
    assert break_even(pe, ae, pi, ai) == int(n), name


def test_Gt_times_and_residuals(cfg1):
    """G^T lam without forming G equals the dense G^T lam; the FETI equation
    residuals vanish for the oracle's own converged solve and do not for a
    perturbed multiplier vector."""
    lam = np.random.default_rng(3).normal(size=cfg1.n_lambda)
    assert np.allclose(O.Gt_times(cfg1, lam), O.G_matrix(cfg1).T @ lam, rtol=0, atol=1e-12)
    res = O.feti_solve(cfg1, tol=1e-12)
    fwd, bwd, Bu = O.feti_equation_residuals(cfg1, res["lam"], res["u"])
    assert fwd.max() < 1e-12 and bwd.max() < 1e-13 and np.abs(Bu).max() < 1e-10
    assert np.all(bwd <= fwd)
    fwd2, bwd2, Bu2 = O.feti_equation_residuals(cfg1, res["lam"] + 1e-3 * lam, res["u"])
    assert fwd2.max() > 1e-6 and bwd2.max() > 1e-8


def test_pcpg_degenerate_initial_guess():
    """One Q1 element as one subdomain, u = 0 on x = 0: the two Dirichlet
    multipliers and the constant kernel make lambda_I = G (G^T G)^{-1} e the
    exact dual solution, so w_0 is rounding noise.  The rounding floor of the
    stopping rule ends the iteration at once, and the primal solution equals
    the monolithic one."""
    P = make_problem(dim=2, physics="heat", cuts=[[1], [1]], material="const", seed=0)
    res = O.feti_solve(P, tol=1e-12, maxit=50)
    assert res["iterations"] == 0
    um = O.monolithic_solve(P)
    assert np.abs(res["u"][0] - um[P.subs[0].l2g]).max() <= 1e-12 * np.abs(um).max()


def test_pcpg_warm_start(cfg1):
    """A warm start lambda_I + P lambda_g (Algorithm 2's next step) keeps
    G^T lambda = e from the first iterate; started from the dual solution it
    stops at once; a guess in range(G) is removed by the projector, so the
    iterates are those of the cold start; a guess near the solution converges
    to the same (unique) lambda and primal solution in fewer iterations."""
    Fs = [O.local_F(s) for s in cfg1.subs]
    lam, its, info = O.pcpg(cfg1, Fs, tol=1e-12)
    e = info["e"]
    sc = np.linalg.norm(lam)
    lam0, its0, _ = O.pcpg(cfg1, Fs, tol=1e-12, lam_guess=lam)
    assert its0 == 0 and np.linalg.norm(lam0 - lam) <= 1e-11 * sc
    G = info["G"]
    rng = np.random.default_rng([5, 1])
    lam_g, its_g, _ = O.pcpg(cfg1, Fs, tol=1e-12, lam_guess=G @ rng.normal(size=G.shape[1]))
    assert its_g == its and np.linalg.norm(lam_g - lam) <= 1e-10 * sc
    noise = rng.normal(size=cfg1.n_lambda)
    guess = lam + 1e-6 * sc * noise / np.linalg.norm(noise)
    lam_w, its_w, info_w = O.pcpg(cfg1, Fs, tol=1e-12, lam_guess=guess, history=True)
    for h in info_w["hist"]:
        assert np.abs(h).max() <= 1e-12 * max(1.0, np.abs(e).max())
    assert 0 < its_w < its
    assert np.linalg.norm(lam_w - lam) <= 1e-9 * sc
    res = O.feti_solve(cfg1, tol=1e-12, lam_guess=guess)
    um = O.monolithic_solve(cfg1)
    err = max(np.abs(u - um[s.l2g]).max() for s, u in zip(cfg1.subs, res["u"]))
    assert err <= 1e-10 * np.abs(um).max()


def _global_B_and_K(problem):
    """Global B (n_lambda x sum n_i) and block-diagonal K, assembled densely."""
    ntot = sum(s.n for s in problem.subs)
    B = np.zeros((problem.n_lambda, ntot))
    K = np.zeros((ntot, ntot))
    off = 0
    for s in problem.subs:
        lam = np.asarray(s.B_lambda, dtype=np.int64)
        np.add.at(B, (lam, off + np.asarray(s.B_dof)), s.B_sign)
        K[off:off + s.n, off:off + s.n] = O.K_dense(s)
        off += s.n
    return B, K


def test_lumped_preconditioner(cfg1):
    """M = sum_i B_i K_i B_i^T equals the global product B K B^T (block-diagonal
    K, dense B), is symmetric positive semidefinite, and the preconditioned
    PCPG reaches the same dual solution (unique: B has full row rank) and the
    monolithic primal solution, keeping G^T lambda_k = e."""
    M = O.lumped_M(cfg1)
    B, K = _global_B_and_K(cfg1)
    assert np.abs(M - B @ K @ B.T).max() <= 1e-12 * np.abs(M).max()
    assert np.abs(M - M.T).max() == 0.0
    assert np.linalg.eigvalsh(M).min() >= -1e-10 * np.abs(M).max()
    Fs = [O.local_F(s) for s in cfg1.subs]
    lam0, its0, _ = O.pcpg(cfg1, Fs, tol=1e-12)
    lam1, its1, info = O.pcpg(cfg1, Fs, tol=1e-12, M=M, history=True)
    for h in info["hist"]:
        assert np.abs(h).max() <= 1e-12 * max(1.0, np.abs(info["e"]).max())
    assert np.linalg.norm(lam1 - lam0) <= 1e-9 * np.linalg.norm(lam0)
    res = O.feti_solve(cfg1, tol=1e-12, precond="lumped")
    um = O.monolithic_solve(cfg1)
    err = max(np.abs(u - um[s.l2g]).max() for s, u in zip(cfg1.subs, res["u"]))
    assert err <= 1e-10 * np.abs(um).max()


def test_q_recurrence_reading(cfg1):
    """Reading C20: the CUDA path carries q_k = F p_k as F w_k + beta q_{k-1} and
    z_k = (G^T G)^{-1} G^T r_k as z_k - delta (G^T G)^{-1} G^T q_k.  Written out
    here in FP64 (test code, not the oracle), its iterates follow the oracle's
    literal Algorithm 1 (M = I) to rounding and stop at the same iteration."""
    Fs = [O.local_F(s) for s in cfg1.subs]
    lam_ref, its_ref, info = O.pcpg(cfg1, Fs, tol=1e-10)
    G, d, e, P = info["G"], info["d"], info["e"], info["P"]
    F = lambda v: O.apply_F(cfg1, Fs, v)
    lam = G @ P.coarse_solve(e)
    Flam = F(lam)
    r = d - Flam
    floor = 64.0 * np.finfo(np.float64).eps * (np.linalg.norm(d) + np.linalg.norm(Flam))
    z = P.coarse_solve(G.T @ r)
    w = r - G @ z
    nw0 = np.linalg.norm(w)
    p = np.zeros_like(w)
    q = np.zeros_like(w)
    wy, beta, k = float(w @ w), 0.0, 0
    while k < 5000:
        f = F(w)                       # the apply streams F against w_k
        q = f + beta * q               # q_k = F p_k
        p = w + beta * p
        delta = wy / float(p @ q)
        lam = lam + delta * p
        r = r - delta * q
        z = z - delta * P.coarse_solve(G.T @ q)
        w = r - G @ z
        wy_new = float(w @ w)
        beta, wy = wy_new / wy, wy_new
        k += 1
        if np.sqrt(wy) <= max(1e-10 * nw0, floor):
            break
    assert k == its_ref
    assert np.linalg.norm(lam - lam_ref) <= 1e-9 * np.linalg.norm(lam_ref)
    assert np.linalg.norm(G.T @ lam - e) <= 1e-12 * max(1.0, np.linalg.norm(e))


def test_scaled_lumped_preconditioner(tiny_el, cfg1):
    """B B^T from the subdomain rows equals the global dense product; on
    gluing-only multipliers it is 2 I; the scaled lumped M is symmetric PSD
    and equals the global W B K B^T W; the preconditioned PCPG reaches the
    same dual and primal solution in fewer iterations than M = I (workload 1:
    57 -> 31; 3D elasticity: 363 -> 58 at tol 1e-10)."""
    for P in (cfg1, tiny_el):
        B, K = _global_B_and_K(P)
        BB = O.BBt(P)
        assert np.abs(BB - B @ B.T).max() == 0.0
        W = np.linalg.inv(B @ B.T)
        M = O.scaled_lumped_M(P)
        assert np.abs(M - W @ B @ K @ B.T @ W).max() <= 1e-12 * np.abs(M).max()
        assert np.abs(M - M.T).max() <= 1e-12 * np.abs(M).max()
        assert np.linalg.eigvalsh((M + M.T) / 2).min() >= -1e-10 * np.abs(M).max()
        Fs = [O.local_F(s) for s in P.subs]
        lam0, its0, _ = O.pcpg(P, Fs, tol=1e-10)
        lam1, its1, _ = O.pcpg(P, Fs, tol=1e-10, M=M)
        assert its1 < its0, (its0, its1)
        assert np.linalg.norm(lam1 - lam0) <= 1e-8 * np.linalg.norm(lam0)
    owners = np.zeros(cfg1.n_lambda, dtype=int)
    for s in cfg1.subs:
        np.add.at(owners, np.asarray(s.B_lambda), 1)
    BB = O.BBt(cfg1)
    two = np.flatnonzero(owners == 2)
    # a gluing multiplier between two subdomains only: B B^T row = 2 on the diagonal
    assert np.all(np.diag(BB)[two] == 2.0)
    res = O.feti_solve(cfg1, tol=1e-12, precond="lumped")
    um = O.monolithic_solve(cfg1)
    err = max(np.abs(u - um[s.l2g]).max() for s, u in zip(cfg1.subs, res["u"]))
    assert err <= 1e-10 * np.abs(um).max()


# ------------------------------------------------------------- e, d and Z


def test_e_vector_closed_form(cfg1, tiny_el):
    """e = R^T f (eq. 7) against the integrals of the load (consistent loads of bilinear / trilinear elements
    reproduce constants and linear functions).  Heat with f = 1 and R = 1: each subdomain's area, 1/16 on
    workload 1.  Elasticity with the body force (0, 0, -1): (0, 0, -volume) for the translations and zero for
    the rotations, whose moments are taken about the subdomain's centroid."""
    e = O.e_vector(cfg1)
    assert e.shape == (16,)
    assert np.abs(e - 1.0 / 16.0).max() <= 1e-15
    e = O.e_vector(tiny_el).reshape(-1, 6)
    for s, ei in zip(tiny_el.subs, e):
        ext = s.coords.max(axis=0) - s.coords.min(axis=0)
        vol = float(np.prod(ext))
        want = np.array([0.0, 0.0, -vol, 0.0, 0.0, 0.0])
        assert np.abs(ei - want).max() <= 1e-14 * max(1.0, vol), (ei, want)


def test_d_vector_routes_and_sign(cfg1):
    """d = B K^+ f - c (eq. 7): against a sparse LU solve of K_reg (an independent factorisation of the same
    generalised inverse), and, with the load removed and c nonzero, exactly -c."""
    import copy

    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    d = O.d_vector(cfg1)
    dd = -np.asarray(cfg1.c, dtype=np.float64).copy()
    for s in cfg1.subs:
        x = spla.splu(sp.csc_matrix(O.K_reg(s))).solve(s.f)
        np.add.at(dd, np.asarray(s.B_lambda, dtype=np.int64), s.B_sign * x[s.B_dof])
    assert np.linalg.norm(d - dd) <= 1e-12 * np.linalg.norm(d)
    P0 = copy.deepcopy(cfg1)
    for s in P0.subs:
        s.f = np.zeros_like(s.f)
    P0.c = np.random.default_rng(5).standard_normal(P0.n_lambda)
    assert np.array_equal(O.d_vector(P0), -P0.c)


def test_local_Z_against_schur_route(cfg1, tiny_el):
    """Z_i = K_reg^{-1} B_i^T (the adjoint's Z): B_i Z_i equals F_i of the Schur-complement route (eq. 13, LU
    solves on the interior block, no Cholesky)."""
    for P in (cfg1, tiny_el):
        for s in P.subs[:4]:
            Z = O.local_Z(s)
            assert Z.shape == (s.n, s.m)
            Fs = O.local_F_schur(s)
            assert np.linalg.norm(O.B_dense(s) @ Z - Fs) <= 1e-12 * np.linalg.norm(Fs)
