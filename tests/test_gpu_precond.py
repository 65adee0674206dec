"""The preconditioners on the CUDA path, against the oracle's preconditioned
Algorithm 1 and the monolithic FEM solve:
  * lumped (options.precond = 1): M = W (sum_i B_i K_i B_i^T) W, W = (B B^T)^{-1};
  * Dirichlet (options.precond = 2, with the Schur-complement assembly route):
    M = W (sum_i B_i S_i B_i^T) W with S_i the Schur complement of K_i onto the
    DOFs B_i touches, taken from a factorisation of K_i stopped at its root
    front and applied as tiles like F_i."""
import dataclasses

import numpy as np
import pytest

from oracle import feti_oracle as O
from paper_2502_08382_gb300.problems import make_config, make_problem, subdomain_K_values

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


CASES = {
    "cfg1": lambda: make_config(1),
    "heat2d_lognormal": lambda: make_problem(dim=2, physics="heat", cuts=[[6, 7, 5]] * 2, material="lognormal",
                                             sigma=1.0, seed=2),
    "elast3d_small": lambda: make_problem(dim=3, physics="elasticity", cuts=[[3, 2]] * 3, material="const", seed=0),
}


def _solve(P, prec, precond, route="syrk"):
    from paper_2502_08382_gb300 import feti
    kw = dict(tol=1e-12, maxit=3000, precond=precond, route=route)
    if prec != "fp64":
        kw.update(refine_drop=1e-4, refine_restart=True)
    op = feti.FetiOperator(P, prec=prec, **kw)
    op.assemble()
    lam, alpha, u, info = op.solve()
    out = lam.cpu().numpy(), u.cpu().numpy(), info
    op.close()
    return out


def _split(P, u):
    out, off = [], 0
    for s in P.subs:
        out.append(u[off:off + s.n])
        off += s.n
    return out


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
@pytest.mark.parametrize("name", list(CASES))
def test_lumped_solve_matches_monolithic(torch_cuda, name, prec):
    P = CASES[name]()
    lam, u, info = _solve(P, prec, "lumped")
    lam0, u0, info0 = _solve(P, prec, "none")
    um = O.monolithic_solve(P)
    Fs = [O.local_F(s) for s in P.subs]
    _, its_o, _ = O.pcpg(P, Fs, tol=1e-12, M=O.scaled_lumped_M(P))
    print(f"{name} {prec}: iterations lumped {info['iterations']} (oracle {its_o}), none {info0['iterations']}")
    assert info["converged"], info
    err = max(np.abs(ui - um[s.l2g]).max() for s, ui in zip(P.subs, _split(P, u)))
    assert err <= 1e-10 * np.abs(um).max(), err
    e = O.e_vector(P)
    assert np.abs(O.Gt_times(P, lam) - e).max() <= 1e-10 * max(1.0, np.abs(e).max())
    assert np.linalg.norm(lam - lam0) <= 1e-8 * np.linalg.norm(lam0)
    if prec == "fp64":
        # the same Algorithm 1 as the oracle, up to rounding (q_k by recurrence, reading C20)
        assert abs(info["iterations"] - its_o) <= 2, (info["iterations"], its_o)
    assert info["iterations"] <= info0["iterations"], (info["iterations"], info0["iterations"])


def test_lumped_values_follow_new_K(torch_cuda):
    """Algorithm 2's next step: new K values, re-assembly; the preconditioner's
    values are summed again from the new K (same iterations as the oracle's
    preconditioned solve of the new problem, same solution)."""
    from paper_2502_08382_gb300 import feti
    P = CASES["heat2d_lognormal"]()
    op = feti.FetiOperator(P, prec="fp64", tol=1e-12, maxit=3000, precond="lumped")
    op.assemble()
    rng = np.random.default_rng([7, 3])
    subs = []
    for i, s in enumerate(P.subs):
        coef = s.elem_coef * rng.uniform(0.2, 5.0, size=s.elem_dofs.shape[0])
        subs.append(dataclasses.replace(s, elem_coef=coef, K_val=subdomain_K_values(P, i, coef)))
        op.update_values(i, subs[-1].K_val)
    P2 = dataclasses.replace(P, subs=subs)
    op.assemble()
    lam, alpha, u, info = op.solve()
    u = u.cpu().numpy()
    op.close()
    Fs = [O.local_F(s) for s in P2.subs]
    _, its_o, _ = O.pcpg(P2, Fs, tol=1e-12, M=O.scaled_lumped_M(P2))
    um = O.monolithic_solve(P2)
    assert info["converged"], info
    assert abs(info["iterations"] - its_o) <= 2, (info["iterations"], its_o)
    err = max(np.abs(ui - um[s.l2g]).max() for s, ui in zip(P2.subs, _split(P2, u)))
    assert err <= 1e-10 * np.abs(um).max(), err


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
@pytest.mark.parametrize("name", list(CASES))
def test_dirichlet_solve_matches_monolithic(torch_cuda, name, prec):
    P = CASES[name]()
    lam, u, info = _solve(P, prec, "dirichlet", route="schur")
    lam0, u0, info0 = _solve(P, prec, "none")
    um = O.monolithic_solve(P)
    Fs = [O.local_F(s) for s in P.subs]
    _, its_o, _ = O.pcpg(P, Fs, tol=1e-12, M=O.dirichlet_M(P))
    _, its_l, _ = O.pcpg(P, Fs, tol=1e-12, M=O.scaled_lumped_M(P))
    print(f"{name} {prec}: iterations Dirichlet {info['iterations']} (oracle {its_o}; lumped oracle {its_l}), "
          f"none {info0['iterations']}")
    assert info["converged"], info
    err = max(np.abs(ui - um[s.l2g]).max() for s, ui in zip(P.subs, _split(P, u)))
    assert err <= 1e-10 * np.abs(um).max(), err
    e = O.e_vector(P)
    assert np.abs(O.Gt_times(P, lam) - e).max() <= 1e-10 * max(1.0, np.abs(e).max())
    assert np.linalg.norm(lam - lam0) <= 1e-8 * np.linalg.norm(lam0)
    if prec == "fp64":
        assert abs(info["iterations"] - its_o) <= 2, (info["iterations"], its_o)
    assert info["iterations"] <= info0["iterations"], (info["iterations"], info0["iterations"])


def test_dirichlet_needs_schur_route(torch_cuda):
    from paper_2502_08382_gb300 import feti
    with pytest.raises(feti.FetiError):
        feti.FetiOperator(CASES["cfg1"](), prec="fp64", precond="dirichlet")


def test_dirichlet_values_follow_new_K(torch_cuda):
    """Algorithm 2's next step with the Dirichlet preconditioner: after new K values the re-assembly (replayed from
    its CUDA graph) factors the new K up to the root front again, so S_i follows K: the iterations match the
    oracle's Dirichlet-preconditioned solve of the new problem, and so does the solution."""
    from paper_2502_08382_gb300 import feti
    P = CASES["heat2d_lognormal"]()
    op = feti.FetiOperator(P, prec="fp64", tol=1e-12, maxit=3000, precond="dirichlet", route="schur")
    op.assemble()
    op.assemble()  # the second assembly is the graph replay
    rng = np.random.default_rng([7, 5])
    subs = []
    for i, s in enumerate(P.subs):
        coef = s.elem_coef * rng.uniform(0.2, 5.0, size=s.elem_dofs.shape[0])
        subs.append(dataclasses.replace(s, elem_coef=coef, K_val=subdomain_K_values(P, i, coef)))
        op.update_values(i, subs[-1].K_val)
    P2 = dataclasses.replace(P, subs=subs)
    op.assemble()
    lam, alpha, u, info = op.solve()
    u = u.cpu().numpy()
    op.close()
    Fs = [O.local_F(s) for s in P2.subs]
    _, its_o, _ = O.pcpg(P2, Fs, tol=1e-12, M=O.dirichlet_M(P2))
    um = O.monolithic_solve(P2)
    assert info["converged"], info
    assert abs(info["iterations"] - its_o) <= 2, (info["iterations"], its_o)
    err = max(np.abs(ui - um[s.l2g]).max() for s, ui in zip(P2.subs, _split(P2, u)))
    assert err <= 1e-10 * np.abs(um).max(), err
