"""The Schur-complement assembly route (options.assembly_route = 1): the DOFs
B_i touches are ordered last as one root supernode, so the factorisation's
root front is the Schur complement S_i of the interior onto them, its factor
L_T gives F_i = (L_T^{-1} D_i)^T (L_T^{-1} D_i), and the pruned TRSM and SYRK
run on that one dense block.  Same F_i (the same K_reg) as the SYRK path, so
the same bars against the oracle; same solution."""
import numpy as np
import pytest

from bounds import F_bar
from oracle import feti_oracle as O
from paper_2502_08382_gb300.problems import make_config, make_problem, seeded_vector

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
    "heat3d_ragged": lambda: make_problem(dim=3, physics="heat", cuts=[[5, 9, 7]] * 3, material="lognormal",
                                          sigma=0.5, seed=1),
    "elast3d_2x2x2": lambda: make_problem(dim=3, physics="elasticity", cuts=[[4, 6]] * 3, material="density",
                                          seed=2),
}


@pytest.mark.parametrize("prec", ["fp64", "split_bf16", "tf32"])
@pytest.mark.parametrize("name", list(CASES))
def test_schur_route_F_and_apply(torch_cuda, name, prec):
    torch = torch_cuda
    from paper_2502_08382_gb300 import feti
    P = CASES[name]()
    op = feti.FetiOperator(P, prec=prec, route="schur")
    op.assemble()
    worst = 0.0
    Fs = []
    for i, s in enumerate(P.subs):
        Fo = O.local_F(s)
        Fs.append(Fo)
        err = np.linalg.norm(op.get_F(i) - Fo) / np.linalg.norm(Fo)
        worst = max(worst, err / F_bar(prec, Fo, s.n))
        assert err <= F_bar(prec, Fo, s.n), (i, err)
    p = seeded_vector(P.n_lambda, 6)
    q = op.apply(torch.from_numpy(p).cuda()).cpu().numpy()
    op.close()
    qo = O.apply_F(P, Fs, p)
    bar = max(F_bar(prec, F, s.n) for s, F in zip(P.subs, Fs))
    print(f"{name} {prec}: Schur route F_i at most {worst:.3f} of the bar")
    assert np.linalg.norm(q - qo) <= bar * np.linalg.norm(qo)


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
def test_schur_route_solve(torch_cuda, prec):
    from paper_2502_08382_gb300 import feti
    P = make_problem(dim=2, physics="heat", cuts=[[6, 7, 5]] * 2, material="lognormal", sigma=1.0, seed=2)
    kw = dict(tol=1e-12, maxit=3000, route="schur")
    if prec != "fp64":
        kw.update(refine_drop=1e-4, refine_restart=True)
    op = feti.FetiOperator(P, prec=prec, **kw)
    op.assemble()
    lam, alpha, u, info = op.solve()
    u = u.cpu().numpy()
    op.close()
    um = O.monolithic_solve(P)
    assert info["converged"], info
    off, err = 0, 0.0
    for s in P.subs:
        err = max(err, np.abs(u[off:off + s.n] - um[s.l2g]).max())
        off += s.n
    assert err <= 1e-10 * np.abs(um).max(), err


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
@pytest.mark.parametrize("name", ["cfg1", "heat3d_ragged", "elast3d_2x2x2"])
def test_trsm_path_route_F(torch_cuda, name, prec):
    """Route 2: F_i = B_i P^T L^{-T} X_i from the FP64 backward solve (stored in the precision's tiles): the FP64
    path within 1e-12 of the oracle, the FP32 tiles within their rounding (the split-bf16 bar covers it)."""
    from paper_2502_08382_gb300 import feti
    P = CASES[name]()
    op = feti.FetiOperator(P, prec=prec, route="trsm")
    op.assemble()
    assert op.stats()["assembly_route"] == 2
    for i, s in enumerate(P.subs):
        Fo = O.local_F(s)
        err = np.linalg.norm(op.get_F(i) - Fo) / np.linalg.norm(Fo)
        assert err <= F_bar(prec, Fo, s.n), (i, err)
    op.assemble()  # a second assembly on the same route
    Fo = O.local_F(P.subs[0])
    assert np.linalg.norm(op.get_F(0) - Fo) <= F_bar(prec, Fo, P.subs[0].n) * np.linalg.norm(Fo)
    op.close()


def test_autotuned_route(torch_cuda):
    """Route 3 times the SYRK path against the TRSM path at the first assembly and keeps the faster; whichever it
    keeps, F_i and the solution are right, and later assemblies stay on it."""
    from paper_2502_08382_gb300 import feti
    P = CASES["heat3d_ragged"]()
    op = feti.FetiOperator(P, prec="fp64", route="auto", tol=1e-12, maxit=2000)
    op.assemble()
    st = op.stats()
    assert st["assembly_route"] in (0, 2) and st["route_ms"][0] > 0 and st["route_ms"][2] > 0, st
    first = st["assembly_route"]
    for i, s in enumerate(P.subs):
        Fo = O.local_F(s)
        assert np.linalg.norm(op.get_F(i) - Fo) <= 1e-12 * np.linalg.norm(Fo), i
    op.assemble()
    assert op.stats()["assembly_route"] == first
    lam, alpha, u, info = op.solve()
    u = u.cpu().numpy()
    op.close()
    um = O.monolithic_solve(P)
    assert info["converged"], info
    off, err = 0, 0.0
    for s in P.subs:
        err = max(err, np.abs(u[off:off + s.n] - um[s.l2g]).max())
        off += s.n
    assert err <= 1e-10 * np.abs(um).max(), err


def test_schur_route_recompute_X(torch_cuda):
    """recompute_X with the Schur route: X_i released after each assembly and allocated again; the same F_i."""
    from paper_2502_08382_gb300 import feti
    P = CASES["elast3d_2x2x2"]()
    a = feti.FetiOperator(P, prec="split_bf16", route="schur")
    a.assemble()
    b = feti.FetiOperator(P, prec="split_bf16", route="schur", recompute_X=True)
    b.assemble()
    b.assemble()
    for i in range(P.nsub):
        assert np.array_equal(a.get_F(i), b.get_F(i)), i
    a.close()
    b.close()
