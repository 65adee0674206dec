"""The batched Cholesky's two work splits (options.chol_split): one subdomain
per CTA, or subtree tasks (a heavy subtree of the supernodal tree factored by
a CTA of its own, its root's update block handed to the parent task through
global memory, the parent task waiting, bounded, for its children).  Each
supernode's arithmetic and the order of its children's extend-adds are the
same either way, so the factor, and with it F_i, must agree bit for bit; the
split must actually create tasks on the 3D cases; and F_i meets the oracle's
bar.  The Dirichlet preconditioner's factorisation (stopped at the root
front) runs through the same tasks."""
import numpy as np
import pytest

from bounds import F_bar
from oracle import feti_oracle as O
from paper_2502_08382_gb300.problems import make_config, make_problem

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
    # one large subdomain (11^3 nodes, 3993 DOFs) beside seven smaller ones
    "elast3d_one_large": lambda: make_problem(dim=3, physics="elasticity", cuts=[[10, 4]] * 3,
                                              material="density", seed=3),
    "heat3d_ragged": lambda: make_problem(dim=3, physics="heat", cuts=[[5, 9, 7]] * 3, material="lognormal",
                                          sigma=0.5, seed=1),
}


def _assemble(P, prec, route, split):
    from paper_2502_08382_gb300 import feti
    op = feti.FetiOperator(P, prec=prec, route=route, chol_split=split)
    op.assemble()
    op.assemble()  # a second assembly replays the captured graph with the same split
    Fs = [op.get_F(i) for i in range(P.nsub)]
    st = op.stats()
    op.close()
    return Fs, st


@pytest.mark.parametrize("route", ["syrk", "schur"])
@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
@pytest.mark.parametrize("name", list(CASES))
def test_subtree_tasks_same_factor(torch_cuda, name, prec, route):
    P = CASES[name]()
    Fw, sw = _assemble(P, prec, route, "whole")
    Ft, stt = _assemble(P, prec, route, "tasks")
    assert sw["chol_tasks"] == P.nsub
    # the 2D case's subtrees are all warp-sized (nothing to split); the 3D ones have tasks
    assert stt["chol_tasks"] >= P.nsub
    if P.dim == 3:
        assert stt["chol_tasks"] > P.nsub, stt["chol_tasks"]
    for i in range(P.nsub):
        assert np.array_equal(Fw[i], Ft[i]), i
    worst = 0.0
    for i, s in enumerate(P.subs):
        Fo = O.local_F(s)
        err = np.linalg.norm(Ft[i] - Fo) / np.linalg.norm(Fo)
        worst = max(worst, err / F_bar(prec, Fo, s.n))
        assert err <= F_bar(prec, Fo, s.n), (i, err)
    print(f"{name} {prec} {route}: {stt['chol_tasks']} Cholesky tasks for {P.nsub} subdomains, "
          f"F_i at most {worst:.3f} of the bar, Cholesky {sw['t_chol_ms']:.2f} ms whole, "
          f"{stt['t_chol_ms']:.2f} ms tasks")


def test_subtree_tasks_dirichlet(torch_cuda):
    from paper_2502_08382_gb300 import feti
    P = CASES["elast3d_one_large"]()
    um = O.monolithic_solve(P)
    its = []
    for split in ("whole", "tasks"):
        op = feti.FetiOperator(P, prec="fp64", tol=1e-12, maxit=3000, precond="dirichlet", route="schur",
                               chol_split=split)
        op.assemble()
        lam, alpha, u, info = op.solve()
        u = u.cpu().numpy()
        op.close()
        assert info["converged"], info
        off, err = 0, 0.0
        for s in P.subs:
            err = max(err, np.abs(u[off:off + s.n] - um[s.l2g]).max())
            off += s.n
        assert err <= 1e-10 * np.abs(um).max(), (split, err)
        its.append(info["iterations"])
    assert its[0] == its[1], its


def test_autotuned_split_reports_its_choice(torch_cuda):
    from paper_2502_08382_gb300 import feti
    P = CASES["elast3d_one_large"]()
    op = feti.FetiOperator(P, prec="fp64")
    op.assemble()
    st = op.stats()
    F0 = op.get_F(0)
    op.close()
    assert st["chol_tasks"] >= P.nsub
    Fo = O.local_F(P.subs[0])
    assert np.linalg.norm(F0 - Fo) <= F_bar("fp64", Fo, P.subs[0].n) * np.linalg.norm(Fo)


@pytest.mark.parametrize("route", ["syrk", "schur"])
@pytest.mark.parametrize("name", ["elast3d_one_large", "cfg3_2x2x2"])
def test_tensor_core_cholesky(torch_cuda, name, route):
    """The large fronts' rank-128 updates on the tensor cores (exact bf16 slicing, options.chol_tc = 0) against
    the FP64-pipe Cholesky (chol_tc = 1): F_i within the FP64 bar of the oracle either way, and the two within
    the same bar of each other."""
    from paper_2502_08382_gb300 import feti
    P = make_config(3, nsub_axis=2) if name == "cfg3_2x2x2" else CASES[name]()
    Fs = {}
    for tc in (True, False):
        op = feti.FetiOperator(P, prec="fp64", route=route, chol_tc=tc)
        op.assemble()
        Fs[tc] = [op.get_F(i) for i in range(P.nsub)]
        op.close()
    worst = 0.0
    for i, s in enumerate(P.subs):
        Fo = O.local_F(s)
        bar = F_bar("fp64", Fo, s.n)
        for tc in (True, False):
            err = np.linalg.norm(Fs[tc][i] - Fo) / np.linalg.norm(Fo)
            assert err <= bar, (tc, i, err)
        d = np.linalg.norm(Fs[True][i] - Fs[False][i]) / np.linalg.norm(Fo)
        worst = max(worst, np.linalg.norm(Fs[True][i] - Fo) / np.linalg.norm(Fo) / bar)
        assert d <= bar, (i, d)
    print(f"{name} {route}: tensor-core Cholesky F_i at most {worst:.3f} of the FP64 bar")


@pytest.mark.parametrize("front", [128, 256])
@pytest.mark.parametrize("name", ["elast3d_one_large", "cfg3_2x2x2"])
def test_tensor_core_cholesky_front_threshold(torch_cuda, name, front):
    """options.chol_tc_front hands narrower fronts (with all their ancestors) to the tensor-core kernel: its
    time share grows, and F_i stays within the FP64 bar of the oracle."""
    from paper_2502_08382_gb300 import feti
    P = make_config(3, nsub_axis=2) if name == "cfg3_2x2x2" else CASES[name]()
    op = feti.FetiOperator(P, prec="fp64", chol_tc_front=front)
    op.assemble()
    st = op.stats()
    Fs = [op.get_F(i) for i in range(P.nsub)]
    op.close()
    assert st["t_chol_tc_ms"] > 0.0, st["t_chol_tc_ms"]
    worst = 0.0
    for i, s in enumerate(P.subs):
        Fo = O.local_F(s)
        err = np.linalg.norm(Fs[i] - Fo) / np.linalg.norm(Fo)
        bar = F_bar("fp64", Fo, s.n)
        worst = max(worst, err / bar)
        assert err <= bar, (i, err)
    print(f"{name} front {front}: F_i at most {worst:.3f} of the FP64 bar, Cholesky {st['t_chol_ms']:.2f} ms "
          f"({st['t_chol_tc_ms']:.2f} ms tensor-core kernel)")
