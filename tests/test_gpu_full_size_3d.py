"""Parity at full size for the 3D workloads, in the configuration bench.py
times (split-bf16 tensor-core TRSM updates and SYRK, FP32 F tiles, FP64
refinement after every 1e4 drop with a restart, tol 1e-10):

  * workload 3: 3D elasticity, 8^3 = 512 subdomains of 6591 DOFs;
  * workload 4: 3D heat, 1000 uneven subdomains (729 to 15 625 nodes).

The oracle cannot form every dense F_i quickly, so the checks sample:
  * F_i of seeded subdomains against B K_reg^{-1} B^T (dense Cholesky);
  * the apply on a vector supported on the Dirichlet multipliers of one
    subdomain at x = 0: those multipliers have that subdomain as their only
    owner, so q = F p equals F_i p_i on its multipliers and is zero elsewhere;
and for the solve, properties that hold at any size: G^T lambda = e (eq. 4),
the FETI equations (eq. 3) on every subdomain, and B u = c within the
projected FP64 residual the stopping rule bounds."""
import numpy as np
import pytest

from bounds import SPLIT_BAR, apply_scale, gamma
from oracle import feti_oracle as O
from paper_2502_08382_gb300.problems import make_config
from test_gpu_full_size import check_primal

pytestmark = pytest.mark.gpu

TOL_F = SPLIT_BAR  # split bf16 (tests/bounds.py)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def _single_owner_subdomain(P):
    """A subdomain with multipliers owned by it alone (Dirichlet rows), and those multipliers."""
    owners = np.zeros(P.n_lambda, dtype=np.int64)
    for s in P.subs:
        np.add.at(owners, np.asarray(s.B_lambda, dtype=np.int64), 1)
    best, best_rows = None, None
    for i, s in enumerate(P.subs):
        rows = np.flatnonzero(owners[np.asarray(s.B_lambda, dtype=np.int64)] == 1)
        if rows.size >= 8 and (best is None or s.n < P.subs[best].n):
            best, best_rows = i, rows
    assert best is not None
    return best, best_rows


@pytest.mark.parametrize("config", [3, 4])
def test_full_size_3d(torch_cuda, config):
    torch = torch_cuda
    from paper_2502_08382_gb300 import feti
    P = make_config(config)
    op = feti.FetiOperator(P, prec="split_bf16", tol=1e-10, maxit=5000, refine_drop=1e-4, refine_restart=True)
    op.assemble()
    i_dir, rows = _single_owner_subdomain(P)
    by_size = sorted(range(P.nsub), key=lambda i: P.subs[i].n)
    rng = np.random.default_rng([config, 12])
    picks = sorted({i_dir, by_size[0], by_size[len(by_size) // 2],
                    int(rng.choice(by_size[: len(by_size) // 2 + 1]))})
    Fo = {}
    for i in picks:
        Fo[i] = O.local_F(P.subs[i])
        err = np.linalg.norm(op.get_F(i) - Fo[i]) / np.linalg.norm(Fo[i])
        print(f"workload {config}: F_{i} (n = {P.subs[i].n}, m = {P.subs[i].m}) relative error {err:.3e}")
        assert err <= TOL_F, (i, err)

    s = P.subs[i_dir]
    lam_i = np.asarray(s.B_lambda, dtype=np.int64)
    p = np.zeros(P.n_lambda)
    p[lam_i[rows]] = rng.standard_normal(rows.size)
    q = op.apply(torch.from_numpy(p).cuda()).cpu().numpy()
    qi = Fo[i_dir] @ p[lam_i]
    assert np.linalg.norm(q[lam_i] - qi) <= TOL_F * np.linalg.norm(qi)
    scale = apply_scale([s], [Fo[i_dir]], p, P.n_lambda)[lam_i]
    tau = TOL_F + gamma(2 * s.m, 2.0 ** -24)
    assert np.all(np.abs(q[lam_i] - qi) <= tau * scale), np.max(np.abs(q[lam_i] - qi) / np.maximum(scale, 1e-300))
    outside = np.ones(P.n_lambda, dtype=bool)
    outside[lam_i] = False
    assert np.all(q[outside] == 0.0)

    lam, alpha, u, info = op.solve()
    lam = lam.cpu().numpy()
    u = u.cpu().numpy()
    op.close()
    assert info["converged"], info
    us, off = [], 0
    for sd in P.subs:
        us.append(u[off:off + sd.n])
        off += sd.n
    e = O.e_vector(P)
    assert np.abs(O.Gt_times(P, lam) - e).max() <= 1e-10 * max(1.0, np.abs(e).max())
    check_primal(P, lam, alpha.cpu().numpy(), us, picks, info, f"workload {config}")
