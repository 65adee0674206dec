"""Algorithm 2's multi-step use on the CUDA path: new K values with the same
pattern (feti_update_values), re-assembly, and a PCPG warm-started from the
previous step's multipliers (feti_solve_warm), against the oracle's solve of
the new problem."""
import dataclasses

import numpy as np
import pytest

from oracle import feti_oracle as O
from paper_2502_08382_gb300.problems import make_problem, subdomain_K_values

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def _next_step(P, seed, spread=0.001):
    """Every subdomain's element coefficients scaled by U[1 - spread, 1 + spread]."""
    rng = np.random.default_rng([seed, 7])
    subs = []
    for s in P.subs:
        coef = s.elem_coef * rng.uniform(1.0 - spread, 1.0 + spread, size=s.elem_dofs.shape[0])
        subs.append(dataclasses.replace(s, elem_coef=coef, K_val=subdomain_K_values(P, len(subs), coef)))
    return dataclasses.replace(P, subs=subs)


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
def test_warm_started_next_step(torch_cuda, prec):
    from paper_2502_08382_gb300 import feti
    P = make_problem(dim=2, physics="heat", cuts=[[6, 5, 7]] * 2, material="lognormal", sigma=1.0, seed=6)
    kw = dict(tol=1e-10, maxit=2000)
    if prec != "fp64":
        kw.update(refine_drop=1e-3, refine_restart=True)
    op = feti.FetiOperator(P, prec=prec, **kw)
    op.assemble()
    lam1, _, _, info1 = op.solve()
    assert info1["converged"], info1
    P2 = _next_step(P, 1)
    for i, s in enumerate(P2.subs):
        op.update_values(i, s.K_val)
    op.assemble()
    lam_c, _, u_c, info_c = op.solve()
    lam_w, _, u_w, info_w = op.solve(lambda_guess=lam1)
    ref = O.feti_solve(P2, tol=1e-12)
    lam_exact, _, _, info_x = op.solve(lambda_guess=torch_cuda.from_numpy(ref["lam"]).cuda())
    op.close()
    assert info_c["converged"] and info_w["converged"], (info_c, info_w)
    print(f"{prec}: cold {info_c['iterations']} iterations, warm {info_w['iterations']}, "
          f"from the exact solution {info_x['iterations']}")
    assert info_w["iterations"] < info_c["iterations"]
    assert info_x["iterations"] <= 1
    sc = np.linalg.norm(ref["lam"])
    for lam in (lam_c, lam_w, lam_exact):
        assert np.linalg.norm(lam.cpu().numpy() - ref["lam"]) <= 1e-7 * sc
    um = np.concatenate(ref["u"])
    for u in (u_c, u_w):
        assert np.abs(u.cpu().numpy() - um).max() <= 1e-9 * np.abs(um).max()
    Gte = O.Gt_times(P2, lam_w.cpu().numpy()) - O.e_vector(P2)
    assert np.abs(Gte).max() <= 1e-10 * max(1.0, np.abs(O.e_vector(P2)).max())
