"""GPU parity of the CUDA path against the FP64 CPU oracle (through the C ABI)."""
import numpy as np
import pytest

from bounds import F_bar, apply_scale, gamma, tf32_vs_split_bar
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


def _op(P, prec="fp64", **kw):
    from paper_2502_08382_gb300 import feti
    op = feti.FetiOperator(P, prec=prec, **kw)
    op.assemble()
    return op


CASES = {
    "cfg1": lambda: make_config(1),
    "cfg2_2x2": lambda: make_config(2, nsub_axis=2),
    "heat3d_ragged": lambda: make_problem(dim=3, physics="heat", cuts=[[5, 9, 7]] * 3, material="lognormal",
                                          sigma=0.5, seed=1),
    "elast3d_2x2x2": lambda: make_problem(dim=3, physics="elasticity", cuts=[[4, 6]] * 3, material="density",
                                          seed=2),
    "cfg3_2x2x2": lambda: make_config(3, nsub_axis=2),
}


@pytest.mark.parametrize("name", list(CASES))
def test_F_fp64_matches_oracle(torch_cuda, name):
    """Plain FP64 path: F_i within 1e-12 relative Frobenius of B K_reg^{-1} B^T."""
    P = CASES[name]()
    op = _op(P)
    idx = range(P.nsub) if P.nsub <= 27 else np.random.default_rng(0).choice(P.nsub, 8, replace=False)
    worst = 0.0
    for i in idx:
        s = P.subs[i]
        Fo = O.local_F(s)
        Fg = op.get_F(int(i))
        worst = max(worst, np.linalg.norm(Fg - Fo) / np.linalg.norm(Fo))
    op.close()
    assert worst <= 1e-12, worst


@pytest.mark.parametrize("name", ["cfg1", "cfg2_2x2", "heat3d_ragged", "elast3d_2x2x2"])
def test_apply_fp64_matches_oracle(torch_cuda, name):
    torch = torch_cuda
    P = CASES[name]()
    op = _op(P)
    Fs = [O.local_F(s) for s in P.subs]
    for seed in (0, 1):
        p = seeded_vector(P.n_lambda, seed)
        q = op.apply(torch.from_numpy(p).cuda()).cpu().numpy()
        qo = O.apply_F(P, Fs, p)
        assert np.linalg.norm(q - qo) <= 1e-12 * np.linalg.norm(qo)
        # element by element: |q_j - qo_j| <= 1e-12 s_j (componentwise scale of F p)
        scale = apply_scale(P.subs, Fs, p, P.n_lambda)
        assert np.all(np.abs(q - qo) <= 1e-12 * scale), np.max(np.abs(q - qo) / np.maximum(scale, 1e-300))
    # bitwise determinism run to run
    p = torch.from_numpy(seeded_vector(P.n_lambda, 3)).cuda()
    a = op.apply(p).cpu().numpy()
    b = op.apply(p).cpu().numpy()
    assert np.array_equal(a, b)
    op.close()


# Mixed precision: pruned TRSM with split-bf16 tensor-core panel updates, then a
# tensor-core SYRK (split bf16, or TF32 on X rounded to TF32), F_i stored as FP32
# tiles.  The bars follow the rounding model in tests/bounds.py: split bf16 is held
# to the FP32-level SPLIT_BAR, TF32 to its derived SYRK bound on top of it.


@pytest.mark.parametrize("prec", ["tf32", "split_bf16"])
@pytest.mark.parametrize("name", ["cfg1", "heat3d_ragged", "elast3d_2x2x2", "cfg3_2x2x2"])
def test_F_mixed_matches_oracle(torch_cuda, name, prec):
    P = CASES[name]()
    op = _op(P, prec=prec)
    idx = range(P.nsub) if P.nsub <= 27 else range(8)
    worst, worst_ratio = 0.0, 0.0
    for i in idx:
        s = P.subs[i]
        Fo = O.local_F(s)
        Fg = op.get_F(int(i))
        err = np.linalg.norm(Fg - Fo) / np.linalg.norm(Fo)
        bar = F_bar(prec, Fo, s.n)
        worst = max(worst, err)
        worst_ratio = max(worst_ratio, err / bar)
        assert err <= bar, (i, err, bar)
    op.close()
    print(f"{name} {prec}: max relative Frobenius error of F_i = {worst:.3e} ({worst_ratio:.2f} of its bar)")


@pytest.mark.parametrize("name", ["cfg1", "heat3d_ragged", "elast3d_2x2x2", "cfg3_2x2x2"])
def test_F_tf32_syrk_within_rounding_bound(torch_cuda, name):
    """Both mixed modes run the same TRSM, so F_tf32 - F_split is the SYRK rounding alone:
    ||F_tf32 - F_split||_F <= (c_tf32 + c_split) tr(F) (tests/bounds.py)."""
    P = CASES[name]()
    a = _op(P, prec="tf32")
    b = _op(P, prec="split_bf16")
    idx = range(P.nsub) if P.nsub <= 27 else range(8)
    worst = 0.0
    for i in idx:
        Ft, Fs = a.get_F(int(i)), b.get_F(int(i))
        bar = tf32_vs_split_bar(Fs, P.subs[i].n)
        worst = max(worst, np.linalg.norm(Ft - Fs) / bar)
        assert np.linalg.norm(Ft - Fs) <= bar, (i, np.linalg.norm(Ft - Fs), bar)
    a.close()
    b.close()
    print(f"{name}: ||F_tf32 - F_split|| at most {worst:.3f} of the derived bound")


@pytest.mark.parametrize("prec", ["tf32", "split_bf16"])
def test_apply_mixed_matches_oracle(torch_cuda, prec):
    torch = torch_cuda
    P = CASES["heat3d_ragged"]()
    op = _op(P, prec=prec)
    Fs = [O.local_F(s) for s in P.subs]
    p = seeded_vector(P.n_lambda, 4)
    q = op.apply(torch.from_numpy(p).cuda()).cpu().numpy()
    qo = O.apply_F(P, Fs, p)
    op.close()
    bar = max(F_bar(prec, F, s.n) for s, F in zip(P.subs, Fs))
    assert np.linalg.norm(q - qo) <= bar * np.linalg.norm(qo)
    # element by element, with the FP32 apply's own accumulation (m_i terms) on top
    tau = bar + gamma(2 * max(s.m for s in P.subs), 2.0 ** -24)
    scale = apply_scale(P.subs, Fs, p, P.n_lambda)
    assert np.all(np.abs(q - qo) <= tau * scale), np.max(np.abs(q - qo) / np.maximum(scale, 1e-300))


# ---------------------------------------------------------------- implicit operator and solve


@pytest.mark.parametrize("name", ["cfg1", "heat3d_ragged", "elast3d_2x2x2"])
def test_implicit_apply_matches_oracle(torch_cuda, name):
    """FP64 implicit operator B L^-T L^-1 B^T p (eq. 11) against B K_reg^-1 B^T p."""
    torch = torch_cuda
    P = CASES[name]()
    op = _op(P)
    Fs = [O.local_F(s) for s in P.subs]
    p = seeded_vector(P.n_lambda, 5)
    q = op.apply_implicit(torch.from_numpy(p).cuda()).cpu().numpy()
    qo = O.apply_F(P, Fs, p)
    op.close()
    assert np.linalg.norm(q - qo) <= 1e-12 * np.linalg.norm(qo)


def _split_u(P, u):
    out, off = [], 0
    for s in P.subs:
        out.append(u[off:off + s.n])
        off += s.n
    return out


def test_solve_closed_form_poisson(torch_cuda):
    """Workload 1 solved on the GPU reproduces u = x - x^2/2 (FP64 path)."""
    P = make_config(1)
    op = _op(P, tol=1e-12, maxit=1000)
    lam, alpha, u, info = op.solve()
    X = P.global_solution_coords()[:, 0]
    exact = X - X ** 2 / 2
    us = _split_u(P, u.cpu().numpy())
    op.close()
    assert info["converged"], info
    err = max(np.abs(ui - exact[s.l2g]).max() for s, ui in zip(P.subs, us))
    assert err <= 1e-10 * 0.5, err


@pytest.mark.parametrize("prec,kref", [("fp64", 0), ("split_bf16", 10), ("tf32", 5)])
@pytest.mark.parametrize("name", ["heat2d_lognormal", "elast3d_small"])
def test_solve_matches_monolithic(torch_cuda, name, prec, kref):
    """FETI solution (PCPG + FP64 refinement, alpha, u) against the monolithic
    FEM solve to 1e-10 relative."""
    if name == "heat2d_lognormal":
        P = make_problem(dim=2, physics="heat", cuts=[[6, 7, 5]] * 2, material="lognormal", sigma=1.0, seed=2)
    else:
        P = make_problem(dim=3, physics="elasticity", cuts=[[3, 2]] * 3, material="const", seed=0)
    um = O.monolithic_solve(P)
    op = _op(P, prec=prec, tol=1e-12, maxit=3000, refine_every=kref)
    lam, alpha, u, info = op.solve()
    us = _split_u(P, u.cpu().numpy())
    # the multipliers keep the solvability condition G^T lambda = e (eq. 4)
    G = O.G_matrix(P)
    e = O.e_vector(P)
    gte = G.T @ lam.cpu().numpy() - e
    op.close()
    print(f"{name} {prec}: iterations {info['iterations']} refinements {info['refinements']}")
    assert info["converged"], info
    err = max(np.abs(ui - um[s.l2g]).max() for s, ui in zip(P.subs, us))
    assert err <= 1e-10 * np.abs(um).max(), err
    assert np.abs(gte).max() <= 1e-10 * max(1.0, np.abs(e).max())
