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
The operator runs in the configuration bench.py times (split-bf16 SYRK,
FP32 F tiles, FP64 residual recomputed after every 1e3 drop, tol 1e-10)."""
import types

import numpy as np
import pytest

from oracle import feti_oracle as O
from paper_2502_08382_gb300.problems import make_config, seeded_vector

pytestmark = pytest.mark.gpu

MIXED_TOL = {"tf32": 1e-2, "split_bf16": 1e-4, "fp64": 1e-12}


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
        worst = max(worst, np.linalg.norm(op.get_F(i) - Fo) / np.linalg.norm(Fo))
    print(f"workload 2 {prec}: sampled F_i max relative error {worst:.3e}")
    assert worst <= MIXED_TOL[prec], worst

    p = seeded_vector(P.n_lambda, 11)
    q = op.apply(torch.from_numpy(p).cuda()).cpu().numpy()
    for i in picks[:2]:
        near = _neighbourhood(P, i)
        sub_P = types.SimpleNamespace(subs=[P.subs[j] for j in near], n_lambda=P.n_lambda)
        qo = O.apply_F(sub_P, [F_or(j) for j in near], p)
        lam = np.asarray(P.subs[i].B_lambda, dtype=np.int64)
        err = np.linalg.norm(q[lam] - qo[lam]) / np.linalg.norm(qo[lam])
        assert err <= MIXED_TOL[prec], (i, err)
    op.close()


def test_workload2_full_solve_properties(torch_cuda, workload2):
    """The benchmark's solve (mixed precision with FP64 refinement) satisfies
    the FETI equations at full size."""
    from paper_2502_08382_gb300 import feti
    P = workload2
    op = feti.FetiOperator(P, prec="split_bf16", tol=1e-10, maxit=5000, refine_drop=1e-3, refine_restart=True)
    op.assemble()
    lam, alpha, u, info = op.solve()
    lam = lam.cpu().numpy()
    u = u.cpu().numpy()
    op.close()
    assert info["converged"], info
    us, off = [], 0
    for s in P.subs:
        us.append(u[off:off + s.n])
        off += s.n
    gte = O.Gt_times(P, lam) - O.e_vector(P)
    assert np.abs(gte).max() <= 1e-10 * max(1.0, np.abs(O.e_vector(P)).max())
    rng = np.random.default_rng([0, 10])
    sample = sorted(int(x) for x in rng.choice(P.nsub, 16, replace=False))
    sub_P = types.SimpleNamespace(subs=[P.subs[j] for j in sample], c=np.zeros(P.n_lambda), n_lambda=P.n_lambda)
    prim, _ = O.feti_equation_residuals(sub_P, lam, [us[j] for j in sample])
    _, Bu = O.feti_equation_residuals(P, lam, us)
    # B u - c = d - F lambda + G alpha = P (d - F lambda) (eqs. 5, 8): the projected FP64
    # residual, which the stopping rule bounds by tol * ||P r_0||
    bound = 2e-10 * info["initial_residual"] + 1e-13 * np.linalg.norm(np.concatenate(us))
    print(f"primal residual max {prim.max():.2e}, ||Bu - c|| {np.linalg.norm(Bu):.3e}, "
          f"tol ||P r_0|| {1e-10 * info['initial_residual']:.3e}, iterations {info['iterations']}")
    assert prim.max() <= 1e-10, prim.max()
    assert np.linalg.norm(Bu) <= bound, (np.linalg.norm(Bu), bound)
