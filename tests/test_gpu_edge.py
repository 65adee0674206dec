"""Edge and degenerate cases of the CUDA path against the oracle.

* a one-element, one-subdomain problem (n = 4, m = 2, d = 1);
* a non-floating subdomain (d = 0, no regularisation): K_0 made SPD by a
  reaction term, so F_0 = B K_0^{-1} B^T and the FETI solve must match the
  monolithic solve of the same modified problem;
* no coarse space at all (every subdomain non-floating, G empty, P = I);
* apply of the zero vector (exact zeros) and of unit vectors (columns of F);
* Algorithm 2's multi-step use: new K values with the same pattern, then
  re-assembly;
* a non-SPD K_i: assembly reports FETI_ERR_NOT_SPD and the context stays
  unusable (sticky error) without faulting.
"""
import dataclasses

import numpy as np
import pytest
import scipy.sparse as sp

from bounds import F_bar
from oracle import feti_oracle as O
from paper_2502_08382_gb300.problems import make_problem, seeded_vector

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def _op(P, prec="fp64", **kw):
    from paper_2502_08382_gb300 import feti
    op = feti.FetiOperator(P, prec=prec, **kw)
    op.assemble()
    return op


def _split(P, u):
    out, off = [], 0
    for s in P.subs:
        out.append(u[off:off + s.n])
        off += s.n
    return out


def _non_floating(P, i, react=0.1):
    """Copy of P with subdomain i given K_i + react * I (SPD, d = 0)."""
    s = P.subs[i]
    K = sp.csr_matrix((s.K_val, s.K_col, s.K_rowptr), shape=(s.n, s.n)) + react * sp.identity(s.n, format="csr")
    K.sort_indices()
    s2 = dataclasses.replace(s, K_rowptr=K.indptr.astype(np.int64), K_col=K.indices.astype(np.int32),
                             K_val=K.data.copy(), R=np.zeros((s.n, 0)), fix_dofs=np.zeros(0, dtype=np.int32))
    subs = list(P.subs)
    subs[i] = s2
    return dataclasses.replace(P, subs=subs)


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
def test_single_element_single_subdomain(torch_cuda, prec):
    torch = torch_cuda
    P = make_problem(dim=2, physics="heat", cuts=[[1], [1]], material="const", seed=0)
    s = P.subs[0]
    assert (s.n, s.m, s.d) == (4, 2, 1)
    op = _op(P, prec=prec, tol=1e-12, maxit=50, refine_every=2 if prec != "fp64" else 0)
    Fo = O.local_F(s)
    tol = 1e-12 if prec == "fp64" else 1e-4
    assert np.linalg.norm(op.get_F(0) - Fo) <= tol * np.linalg.norm(Fo)
    lam, alpha, u, info = op.solve()
    um = O.monolithic_solve(P)
    op.close()
    # lambda_I already solves this dual problem: the rounding floor of the stopping rule ends it at once
    assert info["converged"] and info["iterations"] == 0, info
    assert np.abs(u.cpu().numpy() - um[s.l2g]).max() <= 1e-10 * max(1.0, np.abs(um).max())


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_non_floating_subdomain(torch_cuda, prec):
    P = _non_floating(make_problem(dim=2, physics="heat", cuts=[[5, 6]] * 2, material="lognormal", sigma=0.7,
                                   seed=3), 2)
    assert P.subs[2].d == 0
    op = _op(P, prec=prec, tol=1e-12, maxit=500, refine_every=5 if prec != "fp64" else 0)
    for i, s in enumerate(P.subs):
        Fo = O.local_F(s)
        # derived bars (tests/bounds.py): 1e-12 for FP64, the TF32 SYRK rounding bound otherwise
        assert np.linalg.norm(op.get_F(i) - Fo) <= F_bar(prec, Fo, s.n) * np.linalg.norm(Fo), i
    lam, alpha, u, info = op.solve()
    assert alpha.numel() == sum(s.d for s in P.subs)
    us = _split(P, u.cpu().numpy())
    um = O.monolithic_solve(P)
    op.close()
    assert info["converged"], info
    err = max(np.abs(ui - um[s.l2g]).max() for s, ui in zip(P.subs, us))
    assert err <= 1e-10 * np.abs(um).max(), err


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
def test_no_coarse_space(torch_cuda, prec):
    P = make_problem(dim=2, physics="heat", cuts=[[5, 6]] * 2, material="lognormal", sigma=0.7, seed=3)
    for i in range(len(P.subs)):
        P = _non_floating(P, i)
    assert all(s.d == 0 for s in P.subs)
    kw = dict(tol=1e-12, maxit=500)
    if prec != "fp64":
        kw.update(refine_drop=1e-3, refine_restart=True)
    op = _op(P, prec=prec, **kw)
    lam, alpha, u, info = op.solve()
    ref = O.feti_solve(P, tol=1e-13)
    um = O.monolithic_solve(P)
    op.close()
    assert info["converged"], info
    assert alpha.numel() == 0
    sc = np.linalg.norm(ref["lam"])
    assert np.linalg.norm(lam.cpu().numpy() - ref["lam"]) <= 1e-9 * sc
    us = _split(P, u.cpu().numpy())
    err = max(np.abs(ui - um[s.l2g]).max() for s, ui in zip(P.subs, us))
    assert err <= 1e-10 * np.abs(um).max(), err


def test_apply_zero_and_unit_vectors(torch_cuda):
    torch = torch_cuda
    P = make_problem(dim=3, physics="heat", cuts=[[4, 5]] * 3, material="lognormal", sigma=0.5, seed=4)
    op = _op(P)
    z = op.apply(torch.zeros(P.n_lambda, dtype=torch.float64, device="cuda")).cpu().numpy()
    assert np.all(z == 0.0)
    Fs = [O.local_F(s) for s in P.subs]
    for lam in (0, P.n_lambda // 2, P.n_lambda - 1):
        e = np.zeros(P.n_lambda)
        e[lam] = 1.0
        q = op.apply(torch.from_numpy(e).cuda()).cpu().numpy()
        qo = O.apply_F(P, Fs, e)
        assert np.linalg.norm(q - qo) <= 1e-12 * np.linalg.norm(qo)
    op.close()


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
def test_update_values_and_reassemble(torch_cuda, prec):
    """Algorithm 2: K values change between steps, the pattern does not."""
    torch = torch_cuda
    P = make_problem(dim=2, physics="heat", cuts=[[6, 5, 7]] * 2, material="lognormal", sigma=1.0, seed=6)
    op = _op(P, prec=prec)
    rng = np.random.default_rng([6, 2])
    new = {}
    for i in (1, 4, 7):
        s = P.subs[i]
        coef = rng.uniform(0.5, 2.0, size=s.elem_dofs.shape[0])
        from paper_2502_08382_gb300.problems import subdomain_K_values
        new[i] = dataclasses.replace(s, K_val=subdomain_K_values(P, i, s.elem_coef * coef))
        op.update_values(i, new[i].K_val)
    op.assemble()
    subs = [new.get(i, s) for i, s in enumerate(P.subs)]
    P2 = dataclasses.replace(P, subs=subs)
    tol = 1e-12 if prec == "fp64" else 1e-4
    Fs = []
    for i, s in enumerate(P2.subs):
        Fo = O.local_F(s)
        Fs.append(Fo)
        assert np.linalg.norm(op.get_F(i) - Fo) <= tol * np.linalg.norm(Fo), i
    p = seeded_vector(P.n_lambda, 2)
    q = op.apply(torch.from_numpy(p).cuda()).cpu().numpy()
    qo = O.apply_F(P2, Fs, p)
    op.close()
    assert np.linalg.norm(q - qo) <= tol * np.linalg.norm(qo)


def test_not_spd_is_reported(torch_cuda):
    torch = torch_cuda
    from paper_2502_08382_gb300 import feti
    P = make_problem(dim=2, physics="heat", cuts=[[4, 4]] * 2, material="const", seed=0)
    s = P.subs[1]
    bad = dataclasses.replace(s, K_val=-s.K_val)
    P2 = dataclasses.replace(P, subs=[P.subs[0], bad] + list(P.subs[2:]))
    op = feti.FetiOperator(P2, prec="fp64")
    with pytest.raises(feti.FetiError) as ei:
        op.assemble()
    assert ei.value.status == 3  # FETI_ERR_NOT_SPD
    with pytest.raises(feti.FetiError) as ei2:
        op.apply(torch.zeros(P.n_lambda, dtype=torch.float64, device="cuda"))
    assert ei2.value.status == 6  # FETI_ERR_STATE (sticky)
    op.close()
