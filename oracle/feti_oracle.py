"""Plain FP64 CPU oracle for the FETI dual-operator path.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import or call
this module: only the tests, the smoke check and the CPU-baseline leg of the
benchmark do.  It shares no code with the CUDA library; its only input is the
seeded problem description built by ``paper_2502_08382_gb300.problems``
(duck-typed here: subdomains with CSR K, B rows, R, f, fix DOFs, l2g).

Every function restates a definition of the paper (arXiv 2502.08382) in
dense NumPy/SciPy with no blocking or reordering beyond the definition:

  regularisation  K_reg = K + rho * sum_{j in fix} e_j e_j^T,  rho = max diag K
                  (Sec. III: K^+ = K_reg^{-1}, "analytic regularisation")
  local operator  F_i = B_i K_reg,i^{-1} B_i^T                (eq. 9 / eq. 12)
  Schur route     F_i = B_T S^{-1} B_T^T, S = Schur complement of K_reg onto
                  the DOFs B touches                          (eq. 13)
  dual data       G = B R, e = R^T f, d = B K^+ f - c         (eqs. 6-7)
  FETI residuals  K_i u_i + B_i^T lambda - f_i and B u - c     (eq. 3)
  projector       P = I - G (G^T G)^{-1} G^T                  (Sec. II)
  PCPG            Algorithm 1, lambda_I = G (G^T G)^{-1} e, M = I or a given
                  matrix (the lumped M = sum_i B_i K_i B_i^T, its B B^T
                  scaled form, and the scaled Dirichlet form with the Schur
                  complements S_i of K_i onto the B-touched DOFs, are
                  provided; the paper leaves M open),
                  optionally warm-started from
                  lambda_I + P lambda_g (Algorithm 2's next step)
  recovery        alpha (eq. 8), u = K^+ (f - B^T lambda) + R alpha (eq. 5)
  monolithic      K~ u~ = f~ with Dirichlet DOFs eliminated     (eq. 1)
  sensitivity     dL/dtheta_e = -<Z^T dK_e Z, W>, Z = K_reg^{-1} B^T
                  (derivative of the inverse; rho held fixed); exact loss
                  differences for central differences, by the resolvent
                  identity or by the Woodbury identity of a rank-k update

Parity pins for each function live in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# ---------------------------------------------------------------- subdomain


def K_dense(sub) -> np.ndarray:
    return sp.csr_matrix((sub.K_val, sub.K_col, sub.K_rowptr), shape=(sub.n, sub.n)).toarray()


def B_dense(sub) -> np.ndarray:
    B = np.zeros((sub.m, sub.n))
    B[np.arange(sub.m), sub.B_dof] = sub.B_sign
    return B


def rho_pen(K: np.ndarray) -> float:
    """Fixing-node penalty: the largest diagonal entry of K_i."""
    return float(np.max(np.diag(K)))


def K_reg(sub, K: np.ndarray | None = None, rho: float | None = None) -> np.ndarray:
    """K_reg = K + rho * sum_{j in fix} e_j e_j^T (Sec. III, analytic regularisation)."""
    if K is None:
        K = K_dense(sub)
    if rho is None:
        rho = rho_pen(K)
    Kr = K.copy()
    fx = np.asarray(sub.fix_dofs, dtype=np.int64)
    Kr[fx, fx] += rho
    return Kr


def local_F(sub, Kr: np.ndarray | None = None) -> np.ndarray:
    """F_i = B_i K_reg^{-1} B_i^T via a dense Cholesky solve (eq. 9)."""
    if Kr is None:
        Kr = K_reg(sub)
    B = B_dense(sub)
    c = sla.cho_factor(Kr, lower=True)
    Z = sla.cho_solve(c, B.T)
    F = B @ Z
    return 0.5 * (F + F.T)


def local_F_schur(sub, Kr: np.ndarray | None = None) -> np.ndarray:
    """Independent route (eq. 13): with T the DOFs touched by B_i and I the
    rest, (K_reg^{-1})_TT = S^{-1}, S = K_TT - K_TI K_II^{-1} K_IT.  Uses LU
    solves (numpy.linalg.solve), not the Cholesky path of local_F."""
    if Kr is None:
        Kr = K_reg(sub)
    T = np.unique(sub.B_dof)
    I = np.setdiff1d(np.arange(sub.n), T)
    KTT = Kr[np.ix_(T, T)]
    if I.size:
        KTI = Kr[np.ix_(T, I)]
        KII = Kr[np.ix_(I, I)]
        S = KTT - KTI @ np.linalg.solve(KII, KTI.T)
    else:
        S = KTT
    BT = np.zeros((sub.m, T.size))
    BT[np.arange(sub.m), np.searchsorted(T, sub.B_dof)] = sub.B_sign
    F = BT @ np.linalg.solve(S, BT.T)
    return 0.5 * (F + F.T)


def local_Z(sub, Kr: np.ndarray | None = None) -> np.ndarray:
    """Z_i = K_reg^{-1} B_i^T (n x m)."""
    if Kr is None:
        Kr = K_reg(sub)
    return sla.cho_solve(sla.cho_factor(Kr, lower=True), B_dense(sub).T)


# ---------------------------------------------------------------- global dual data


def apply_F(problem, Fs, p: np.ndarray) -> np.ndarray:
    """q = F p = sum_i B~_i^T F_i B~_i p: gather p on each subdomain's
    multipliers, multiply, and add back (Algorithm 2, scatter/apply/gather)."""
    q = np.zeros(problem.n_lambda)
    for sub, F in zip(problem.subs, Fs):
        lam = np.asarray(sub.B_lambda, dtype=np.int64)
        np.add.at(q, lam, F @ p[lam])
    return q


def G_matrix(problem) -> np.ndarray:
    """G = B R (n_lambda x sum d_i), column block i = B_i R_i (eqs. 6-7)."""
    dtot = sum(s.d for s in problem.subs)
    G = np.zeros((problem.n_lambda, dtot))
    off = 0
    for s in problem.subs:
        lam = np.asarray(s.B_lambda, dtype=np.int64)
        G[lam, off:off + s.d] += s.B_sign[:, None] * s.R[s.B_dof, :]
        off += s.d
    return G


def Gt_times(problem, lam: np.ndarray) -> np.ndarray:
    """G^T lam = (R_i^T B_i^T lam)_i without forming G (G = B R, eqs. 6-7):
    the subdomain's multipliers, signed, summed onto their DOFs, then R_i^T."""
    out = []
    for s in problem.subs:
        v = np.zeros(s.n)
        np.add.at(v, s.B_dof, s.B_sign * lam[np.asarray(s.B_lambda, dtype=np.int64)])
        out.append(s.R.T @ v)
    return np.concatenate(out) if out else np.zeros(0)


def feti_equation_residuals(problem, lam, us):
    """Residuals of the FETI system (eq. 3) for a computed (lambda, u).  Per
    subdomain, for the primal rows K_i u_i + B_i^T lambda - f_i:
      forward   ||K_i u_i + B_i^T lambda - f_i|| / ||f_i - B_i^T lambda||,
      backward  ||K_i u_i + B_i^T lambda - f_i|| / (||K_i||_F ||u_i|| + ||f_i - B_i^T lambda||)
    (the normwise backward error, the quantity a backward-stable solve bounds
    by a small multiple of the unit roundoff); and the gluing / Dirichlet rows
    B u - c.  Returns (forward, backward, B u - c)."""
    fwd, bwd = [], []
    Bu = -np.asarray(problem.c, dtype=np.float64).copy()
    for s, u in zip(problem.subs, us):
        K = sp.csr_matrix((s.K_val, s.K_col, s.K_rowptr), shape=(s.n, s.n))
        btl = np.zeros(s.n)
        np.add.at(btl, s.B_dof, s.B_sign * lam[np.asarray(s.B_lambda, dtype=np.int64)])
        rhs = s.f - btl
        res = np.linalg.norm(K @ u - rhs)
        fwd.append(res / max(np.linalg.norm(rhs), 1e-300))
        scale = sp.linalg.norm(K) * np.linalg.norm(u) + np.linalg.norm(rhs)
        bwd.append(res / max(scale, 1e-300))
        np.add.at(Bu, np.asarray(s.B_lambda, dtype=np.int64), s.B_sign * u[s.B_dof])
    return np.asarray(fwd), np.asarray(bwd), Bu


def e_vector(problem) -> np.ndarray:
    """e = R^T f (eq. 7)."""
    return np.concatenate([s.R.T @ s.f for s in problem.subs])


def d_vector(problem, Krs=None) -> np.ndarray:
    """d = B K^+ f - c (eq. 7)."""
    d = -np.asarray(problem.c, dtype=np.float64).copy()
    for i, s in enumerate(problem.subs):
        Kr = K_reg(s) if Krs is None else Krs[i]
        x = sla.cho_solve(sla.cho_factor(Kr, lower=True), s.f)
        np.add.at(d, np.asarray(s.B_lambda, dtype=np.int64), s.B_sign * x[s.B_dof])
    return d


def lumped_M(problem) -> np.ndarray:
    """Lumped preconditioner M = sum_i B_i K_i B_i^T for Algorithm 1 (the
    paper leaves M open): each subdomain's stiffness on its B-touched DOFs,
    signed as B_i, added at its multipliers.  Dense n_lambda x n_lambda."""
    M = np.zeros((problem.n_lambda, problem.n_lambda))
    for s in problem.subs:
        lam = np.asarray(s.B_lambda, dtype=np.int64)
        Ks = K_dense(s)[np.ix_(s.B_dof, s.B_dof)]
        np.add.at(M, (lam[:, None], lam[None, :]), s.B_sign[:, None] * s.B_sign[None, :] * Ks)
    return M


def BBt(problem) -> np.ndarray:
    """B B^T (dense n_lambda x n_lambda): multipliers a, b couple when a
    subdomain has rows for both on the same DOF (signs multiplied)."""
    out = np.zeros((problem.n_lambda, problem.n_lambda))
    for s in problem.subs:
        lam = np.asarray(s.B_lambda, dtype=np.int64)
        same = (np.asarray(s.B_dof)[:, None] == np.asarray(s.B_dof)[None, :]).astype(np.float64)
        np.add.at(out, (lam[:, None], lam[None, :]), s.B_sign[:, None] * s.B_sign[None, :] * same)
    return out


def scaled_lumped_M(problem) -> np.ndarray:
    """Lumped preconditioner with the B B^T scaling of the multipliers,
    M = (B B^T)^{-1} (sum_i B_i K_i B_i^T) (B B^T)^{-1}: for gluing rows
    between two subdomains it halves each side, for chained rows at cross
    points it distributes them consistently, for Dirichlet rows it keeps 1."""
    W = np.linalg.inv(BBt(problem))
    return W @ lumped_M(problem) @ W


def schur_boundary(sub, K: np.ndarray | None = None):
    """S_i = K_TT - K_TI K_II^{-1} K_IT, the Schur complement of the
    unregularised K_i onto the DOFs T that B_i touches (I: the others), by a
    dense LU solve.  Returns (T, S)."""
    if K is None:
        K = K_dense(sub)
    T = np.unique(sub.B_dof)
    I = np.setdiff1d(np.arange(sub.n), T)
    S = K[np.ix_(T, T)].copy()
    if I.size:
        KTI = K[np.ix_(T, I)]
        S -= KTI @ np.linalg.solve(K[np.ix_(I, I)], KTI.T)
    return T, 0.5 * (S + S.T)


def dirichlet_M(problem) -> np.ndarray:
    """Dirichlet preconditioner with the B B^T scaling, M = W (sum_i B_i S~_i B_i^T) W,
    W = (B B^T)^{-1}, S~_i = S_i on the DOFs B_i touches and zero elsewhere (the
    paper leaves M open; this is the Dirichlet counterpart of scaled_lumped_M,
    with the interior condensed instead of dropped).  Dense n_lambda x n_lambda."""
    M = np.zeros((problem.n_lambda, problem.n_lambda))
    for s in problem.subs:
        T, S = schur_boundary(s)
        lam = np.asarray(s.B_lambda, dtype=np.int64)
        pos = np.searchsorted(T, s.B_dof)
        np.add.at(M, (lam[:, None], lam[None, :]), s.B_sign[:, None] * s.B_sign[None, :] * S[np.ix_(pos, pos)])
    W = np.linalg.inv(BBt(problem))
    return W @ M @ W


class Projector:
    """P = I - G (G^T G)^{-1} G^T (Sec. II)."""

    def __init__(self, G: np.ndarray):
        self.G = G
        self.GtG = G.T @ G
        self.c = sla.cho_factor(self.GtG, lower=True)

    def coarse_solve(self, b):
        return sla.cho_solve(self.c, b)

    def __call__(self, x):
        return x - self.G @ self.coarse_solve(self.G.T @ x)


def pcpg(problem, Fs, tol=1e-10, maxit=5000, G=None, d=None, e=None, history=False, lam_guess=None, M=None):
    """Algorithm 1 (PCPG) with lambda_I = G (G^T G)^{-1} e and the
    preconditioner M (a dense matrix; None: M = I), y = P M w.
    Stops when ||w_k|| <= tol * ||w_0||, or when ||w_k|| has reached the
    rounding level of the residual, ||w_k|| <= 64 eps (||d|| + ||F lambda_I||)
    (Algorithm 1 only says "until convergence"; without the floor a problem
    whose lambda_I already solves the dual problem could never stop, since
    w_0 is then rounding noise).
    lam_guess (a warm start, e.g. the previous step of Algorithm 2): the
    iteration starts from lambda_I + P lam_guess, which keeps G^T lambda = e;
    w_0 and the floor above stay those of lambda_I, so the stopping rule asks
    for the same accuracy as a cold start.  Returns (lambda, iterations, info)."""
    if G is None:
        G = G_matrix(problem)
    if e is None:
        e = e_vector(problem)
    if d is None:
        d = d_vector(problem)
    P = Projector(G)
    Fop = lambda v: apply_F(problem, Fs, v)
    lam = G @ P.coarse_solve(e)
    Flam = Fop(lam)
    r = d - Flam
    floor = 64.0 * np.finfo(np.float64).eps * (np.linalg.norm(d) + np.linalg.norm(Flam))
    w = P(r)
    nw0 = float(np.linalg.norm(w))
    if lam_guess is not None:
        lam = lam + P(np.asarray(lam_guess, dtype=np.float64))
        r = d - Fop(lam)
        w = P(r)
    hist = [G.T @ lam - e] if history else None
    Mop = (lambda v: v) if M is None else (lambda v: M @ v)
    y = P(Mop(w))       # y = P M w
    p = y.copy()
    wy = float(w @ y)
    k = 0
    if np.linalg.norm(w) <= max(tol * nw0, floor):
        return lam, 0, dict(P=P, G=G, d=d, e=e, hist=hist)
    while k < maxit:
        q = Fop(p)
        delta = wy / float(p @ q)
        lam = lam + delta * p
        r = r - delta * q
        w = P(r)
        y = P(Mop(w))
        wy_new = float(w @ y)
        beta = wy_new / wy
        p = y + beta * p
        wy = wy_new
        k += 1
        if history:
            hist.append(G.T @ lam - e)
        if np.linalg.norm(w) <= max(tol * nw0, floor):
            break
    return lam, k, dict(P=P, G=G, d=d, e=e, hist=hist)


def alpha_from_lambda(problem, Fs, lam, P: Projector, d) -> np.ndarray:
    """alpha = -(G^T G)^{-1} G^T (d - F lambda) (eq. 8)."""
    return -P.coarse_solve(P.G.T @ (d - apply_F(problem, Fs, lam)))


def primal_solution(problem, lam, alpha, Krs=None):
    """u_i = K_reg,i^{-1} (f_i - B_i^T lambda_i) + R_i alpha_i (eq. 5)."""
    us = []
    off = 0
    for i, s in enumerate(problem.subs):
        Kr = K_reg(s) if Krs is None else Krs[i]
        rhs = s.f.copy()
        np.add.at(rhs, s.B_dof, -s.B_sign * lam[np.asarray(s.B_lambda, dtype=np.int64)])
        u = sla.cho_solve(sla.cho_factor(Kr, lower=True), rhs) + s.R @ alpha[off:off + s.d]
        off += s.d
        us.append(u)
    return us


def feti_solve(problem, tol=1e-10, maxit=5000, lam_guess=None, precond=None):
    """Whole FETI solve in FP64: F_i, PCPG (warm-started from lam_guess if
    given; precond "lumped" for M = scaled_lumped_M, else M = I), alpha, u_i."""
    Krs = [K_reg(s) for s in problem.subs]
    Fs = [local_F(s, Kr) for s, Kr in zip(problem.subs, Krs)]
    G = G_matrix(problem)
    d = d_vector(problem, Krs)
    e = e_vector(problem)
    M = (scaled_lumped_M(problem) if precond == "lumped" else dirichlet_M(problem) if precond == "dirichlet"
         else None)
    lam, its, info = pcpg(problem, Fs, tol=tol, maxit=maxit, G=G, d=d, e=e, lam_guess=lam_guess, M=M)
    alpha = alpha_from_lambda(problem, Fs, lam, info["P"], d)
    us = primal_solution(problem, lam, alpha, Krs)
    return dict(lam=lam, alpha=alpha, u=us, iterations=its, Fs=Fs, G=G, d=d, e=e)


# ---------------------------------------------------------------- monolithic FEM


def monolithic_solve(problem) -> np.ndarray:
    """Solve K~ u~ = f~ (eq. 1): subdomain matrices summed on shared DOFs,
    Dirichlet DOFs eliminated (u = 0 there)."""
    N = problem.n_global_dofs
    rows, cols, vals = [], [], []
    f = np.zeros(N)
    for s in problem.subs:
        Kc = sp.csr_matrix((s.K_val, s.K_col, s.K_rowptr), shape=(s.n, s.n)).tocoo()
        rows.append(s.l2g[Kc.row]); cols.append(s.l2g[Kc.col]); vals.append(Kc.data)
        np.add.at(f, s.l2g, s.f)
    K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    free = np.setdiff1d(np.arange(N), problem.dirichlet_dofs)
    u = np.zeros(N)
    u[free] = spla.spsolve(K[free][:, free].tocsc(), f[free])
    return u


# ---------------------------------------------------------------- sensitivity


def loss_sub(sub, W, Kr=None) -> float:
    """L_i = <W_i, F_i>."""
    return float(np.sum(W * local_F(sub, Kr)))


def gradient_sub(sub, W, dK_ref, elems=None, Kr=None) -> np.ndarray:
    """dL_i/dtheta_e = -<Z^T dK_e Z, W> with dK_e = dcoef_e * dK_ref on the
    element's DOFs and Z = K_reg^{-1} B^T (rho_pen held at its base value).
    Written as -sum_{a,b} (dK_e)_{ab} (Z W)_{b,:} . Z_{a,:}."""
    Z = local_Z(sub, Kr)
    Y = Z @ W
    if elems is None:
        elems = np.arange(sub.elem_dofs.shape[0])
    g = np.zeros(len(elems))
    for k, e in enumerate(elems):
        dofs = sub.elem_dofs[e]
        dKe = sub.elem_dcoef[e] * dK_ref
        g[k] = -np.sum(dKe * (Z[dofs, :] @ Y[dofs, :].T))
    return g


def loss_difference(sub, W, Kp, Km, e, dcoef, K_ref) -> float:
    """L(K_+) - L(K_-) for L = <W, B K^{-1} B^T>, where K_+ and K_- differ
    only on element e by dcoef * K_ref, through the resolvent identity
    K_+^{-1} - K_-^{-1} = -K_+^{-1} (K_+ - K_-) K_-^{-1}:
    -<W, Z_+[dofs_e]^T (dcoef K_ref) Z_-[dofs_e]>.  The same difference as
    subtracting two loss values (and as subtracting the two matrices), written
    so that no digits are lost to cancellation at small steps (h = 1e-6)."""
    Zp = local_Z(sub, Kp)
    Zm = local_Z(sub, Km)
    dofs = sub.elem_dofs[e]
    return float(-np.sum(W * (Zp[dofs].T @ (dcoef * K_ref) @ Zm[dofs])))


def loss_difference_lowrank(sub, W, cho, e, d_plus, d_minus, K_ref) -> float:
    """L(K_+) - L(K_-) for L = <W, B K^{-1} B^T> with K_+- = K + d_+- U K_ref U^T
    (U selects element e's DOFs), from ONE factorisation `cho` of K
    (scipy cho_factor of K_reg, rho held fixed).  The Woodbury identity for a
    low-rank update, (K + U C U^T)^{-1} = K^{-1} - K^{-1} U C (I + U^T K^{-1} U C)^{-1}
    U^T K^{-1} (valid for a singular C such as an element stiffness), gives
    B K_+-^{-1} B^T = F - Z_e M(d) Z_e^T with Z_e = B K^{-1} U (m x k) and
    M(d) = d C (I + d S C)^{-1}, S = U^T K^{-1} U, so
    L(K_+) - L(K_-) = -<W, Z_e (M(d_+) - M(d_-)) Z_e^T>.
    The same number as loss_difference (two factorisations), at the cost of k
    solves with an existing factor; no digits are lost to cancellation."""
    dofs = np.asarray(sub.elem_dofs[e], dtype=np.int64)
    k = dofs.size
    E = np.zeros((sub.n, k))
    E[dofs, np.arange(k)] = 1.0
    X = sla.cho_solve(cho, E)                    # K^{-1} U
    S = X[dofs, :]
    Ze = sub.B_sign[:, None] * X[sub.B_dof, :]   # B K^{-1} U
    C = np.asarray(K_ref, dtype=np.float64)

    def M(d):
        return d * C @ np.linalg.inv(np.eye(k) + d * S @ C)

    D = M(d_plus) - M(d_minus)
    return float(-np.sum(W * (Ze @ D @ Ze.T)))


def perturbed_K_reg(sub, e, dtheta_coef, K_ref, rho):
    """K_reg with element e's coefficient changed by dtheta_coef (rho fixed)."""
    K = K_dense(sub)
    dofs = sub.elem_dofs[e]
    K[np.ix_(dofs, dofs)] += dtheta_coef * K_ref
    return K_reg(sub, K, rho)
