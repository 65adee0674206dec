"""Parity at the benchmark's full size and launch configuration (workload 2:
32 x 32 subdomains of 64 x 64 Q1 elements, 4225 DOFs each, n_lambda = 130 048).

The oracle cannot form all 1024 dense F_i quickly, so the checks sample:
  * F_i of seeded subdomains against B K_reg^{-1} B^T (dense Cholesky);
  * q = F p on every multiplier of seeded subdomains: such a multiplier
    touches the subdomain and at most one neighbour, so q there is the sum of
    oracle F_j p_j over that small set;
and for the solve use properties that hold at any size: the FETI equations
(eq. 3) K_i u_i + B_i^T lambda = f_i on sampled subdomains and B u = c on
all multipliers, plus the solvability condition G^T lambda = e (eq. 4).
The solve runs in the configuration bench.py times (split-bf16 tensor-core
TRSM updates and SYRK, FP32 F tiles, FP64 residual recomputed after every 1e4
drop with a restart of the search direction, tol 1e-10); its solution is also
compared with the plain FP64 path's at 1e-10."""
import types

import numpy as np
import pytest

from bounds import F_bar, apply_scale, gamma
from oracle import feti_oracle as O
from paper_2502_08382_gb300.problems import make_config, seeded_vector

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


@pytest.fixture(scope="module")
def workload2():
    return make_config(2)


def _neighbourhood(P, i):
    owners = {}
    for j, s in enumerate(P.subs):
        for lam in s.B_lambda:
            owners.setdefault(int(lam), []).append(j)
    near = sorted({j for lam in P.subs[i].B_lambda for j in owners[int(lam)]})
    return near


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
def test_workload2_full_sampled(torch_cuda, workload2, prec):
    torch = torch_cuda
    from paper_2502_08382_gb300 import feti
    P = workload2
    op = feti.FetiOperator(P, prec=prec, tol=1e-10, maxit=5000, refine_every=10 if prec != "fp64" else 0)
    op.assemble()
    rng = np.random.default_rng([0, 9])
    picks = [int(x) for x in rng.choice(P.nsub, 3, replace=False)] + [0, P.nsub - 1]
    cache = {}

    def F_or(j):
        if j not in cache:
            cache[j] = O.local_F(P.subs[j])
        return cache[j]

    worst = 0.0
    for i in picks:
        Fo = F_or(i)
        err = np.linalg.norm(op.get_F(i) - Fo) / np.linalg.norm(Fo)
        worst = max(worst, err)
        assert err <= F_bar(prec, Fo, P.subs[i].n), (i, err)
    print(f"workload 2 {prec}: sampled F_i max relative error {worst:.3e}")

    p = seeded_vector(P.n_lambda, 11)
    q = op.apply(torch.from_numpy(p).cuda()).cpu().numpy()
    for i in picks[:2]:
        near = _neighbourhood(P, i)
        sub_P = types.SimpleNamespace(subs=[P.subs[j] for j in near], n_lambda=P.n_lambda)
        qo = O.apply_F(sub_P, [F_or(j) for j in near], p)
        lam = np.asarray(P.subs[i].B_lambda, dtype=np.int64)
        err = np.linalg.norm(q[lam] - qo[lam]) / np.linalg.norm(qo[lam])
        bar = F_bar(prec, F_or(i), P.subs[i].n)
        assert err <= bar, (i, err)
        # element by element on the subdomain's multipliers (FP32 tiles: the apply's own accumulation on top)
        tau = bar + (0.0 if prec == "fp64" else gamma(2 * max(P.subs[j].m for j in near), 2.0 ** -24))
        scale = apply_scale(sub_P.subs, [F_or(j) for j in near], p, P.n_lambda)[lam]
        assert np.all(np.abs(q[lam] - qo[lam]) <= tau * scale), (i, np.max(np.abs(q[lam] - qo[lam]) / scale))
    op.close()


def check_primal(P, lam, alpha, us, sample, info, label):
    """The FETI equations (eq. 3) at full size, on every subdomain where cheap and densely on a sample:
      * B u - c = P (d - F lambda) (eqs. 5, 8): the projected FP64 residual, which the stopping rule bounds
        by tol ||P r_0||;
      * primal rows K_i u_i + B_i^T lambda = f_i: normwise backward error at most 3 n_i eps (the bound of a
        backward-stable Cholesky solve, K_reg = L L^T with ||L|| ||L^T|| ~ ||K||), and a forward residual
        ||K_i u_i + B_i^T lambda - f_i|| / ||f_i - B_i^T lambda|| at most ten times that of the oracle's dense
        FP64 Cholesky solve from the same lambda and alpha;
      * u_i itself against that oracle solution, 1e-10 relative."""
    import types
    alpha = np.asarray(alpha)
    aoff = np.cumsum([0] + [s.d for s in P.subs])
    fwd, bwd, Bu = O.feti_equation_residuals(P, lam, us)
    bound = 2e-10 * info["initial_residual"] + 1e-13 * np.linalg.norm(np.concatenate(us))
    sub_P = types.SimpleNamespace(subs=[P.subs[j] for j in sample], c=np.zeros(P.n_lambda), n_lambda=P.n_lambda)
    a_s = np.concatenate([alpha[aoff[j]:aoff[j + 1]] for j in sample])
    uo = O.primal_solution(sub_P, lam, a_s)
    fwd_o, _, _ = O.feti_equation_residuals(sub_P, lam, uo)
    uerr = max(np.linalg.norm(us[j] - u) / np.linalg.norm(u) for j, u in zip(sample, uo))
    nmax = max(s.n for s in P.subs)
    print(f"{label}: {info['iterations']} iterations; primal backward error max {bwd.max():.2e} "
          f"(bar {3 * nmax * EPS:.2e}); forward residual max {fwd.max():.2e}; sampled forward "
          f"{fwd[sample].max():.2e} vs oracle {fwd_o.max():.2e}; sampled u vs oracle {uerr:.2e}; "
          f"||Bu - c|| {np.linalg.norm(Bu):.3e} (bound {bound:.3e})")
    assert all(b <= 3 * s.n * EPS for b, s in zip(bwd, P.subs)), bwd.max()
    assert np.all(fwd[sample] <= 10 * fwd_o), (fwd[sample], fwd_o)
    assert uerr <= 1e-10, uerr
    assert np.linalg.norm(Bu) <= bound, (np.linalg.norm(Bu), bound)


def test_workload2_full_solve_properties(torch_cuda, workload2):
    """The benchmark's solve (mixed precision with FP64 refinement) satisfies
    the FETI equations at full size and matches the plain FP64 path's solution."""
    torch = torch_cuda
    from paper_2502_08382_gb300 import feti
    P = workload2
    op = feti.FetiOperator(P, prec="split_bf16", tol=1e-10, maxit=5000, refine_drop=1e-4, refine_restart=True)
    op.assemble()
    lam, alpha, u, info = op.solve()
    op.close()
    op64 = feti.FetiOperator(P, prec="fp64", tol=1e-10, maxit=5000)
    op64.assemble()
    lam64, alpha64, u64, info64 = op64.solve()
    op64.close()
    assert info["converged"], info
    assert info64["converged"], info64
    du = (torch.linalg.norm(u - u64) / torch.linalg.norm(u64)).item()
    print(f"workload 2: u mixed vs FP64 path {du:.2e} ({info['iterations']} / {info64['iterations']} iterations)")
    assert du <= 1e-10, du
    lam = lam.cpu().numpy()
    u = u.cpu().numpy()
    us, off = [], 0
    for s in P.subs:
        us.append(u[off:off + s.n])
        off += s.n
    gte = O.Gt_times(P, lam) - O.e_vector(P)
    assert np.abs(gte).max() <= 1e-10 * max(1.0, np.abs(O.e_vector(P)).max())
    rng = np.random.default_rng([0, 10])
    sample = sorted(int(x) for x in rng.choice(P.nsub, 16, replace=False))
    check_primal(P, lam, alpha.cpu().numpy(), us, sample, info, "workload 2")
