"""FP64 adjoint kernel (dL/dtheta_e for L = sum_i <W_i, F_i>) against the
oracle's gradient, the oracle's central differences (rho_pen frozen) and the
autograd wrapper."""
import numpy as np
import pytest

from oracle import feti_oracle as O
from paper_2502_08382_gb300.problems import make_problem, make_W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def _problem():
    return make_problem(dim=3, physics="elasticity", cuts=[[3, 4]] * 3, material="density", seed=5)


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
def test_adjoint_matches_oracle_gradient(torch_cuda, prec):
    """The adjoint is FP64 in every precision mode (Z recomputed with FP64 L)."""
    from paper_2502_08382_gb300 import feti
    P = _problem()
    Ws = make_W(P, seed=0)
    op = feti.FetiOperator(P, prec=prec, with_elements=True)
    op.assemble()
    g = op.adjoint(Ws).cpu().numpy()
    op.close()
    off = 0
    worst = 0.0
    for i, s in enumerate(P.subs):
        ne = s.elem_dofs.shape[0]
        go = O.gradient_sub(s, Ws[i], P.K_ref)
        worst = max(worst, np.linalg.norm(g[off:off + ne] - go) / np.linalg.norm(go))
        off += ne
    assert worst <= 1e-10, worst


def test_adjoint_vs_central_differences(torch_cuda):
    """Central differences h = 1e-6 of L_i = <W_i, F_i> in rho_e (E_e = rho_e^3,
    rho_pen frozen at its base value) on 50 random elements, to 1e-6 relative.
    The difference L(rho + h) - L(rho - h) is evaluated through the resolvent
    identity (oracle.loss_difference): subtracting two loss values of size
    ~1e5 would lose ~7 digits at h = 1e-6."""
    from paper_2502_08382_gb300 import feti
    P = _problem()
    Ws = make_W(P, seed=0)
    op = feti.FetiOperator(P, prec="fp64", with_elements=True)
    op.assemble()
    g = op.adjoint(Ws).cpu().numpy()
    op.close()
    rng = np.random.default_rng([0, 4])
    offs = np.concatenate([[0], np.cumsum([s.elem_dofs.shape[0] for s in P.subs])])
    picks = rng.choice(offs[-1], size=50, replace=False)
    for ge in picks:
        i = int(np.searchsorted(offs, ge, side="right") - 1)
        e = int(ge - offs[i])
        s = P.subs[i]
        rho = O.rho_pen(O.K_dense(s))
        th = s.elem_coef[e] ** (1.0 / 3.0)
        h = 1e-6
        Kp = O.perturbed_K_reg(s, e, (th + h) ** 3 - th ** 3, P.K_ref, rho)
        Km = O.perturbed_K_reg(s, e, (th - h) ** 3 - th ** 3, P.K_ref, rho)
        fd = O.loss_difference(s, Ws[i], Kp, Km, e, (th + h) ** 3 - (th - h) ** 3, P.K_ref) / (2 * h)
        assert abs(fd - g[ge]) <= 1e-6 * max(1.0, abs(fd)), (ge, fd, g[ge])


def test_autograd_function(torch_cuda):
    """torch.autograd through FetiWeightedTrace gives dL/dcoef_e; with
    coef = rho^3 the chain rule reproduces the oracle's dL/drho_e."""
    torch = torch_cuda
    from paper_2502_08382_gb300 import feti
    P = _problem()
    Ws = make_W(P, seed=1)
    op = feti.FetiOperator(P, prec="fp64", with_elements=True, unit_scale=True)
    rho0 = np.concatenate([s.elem_coef ** (1.0 / 3.0) for s in P.subs])
    rho = torch.tensor(rho0, dtype=torch.float64, requires_grad=True)
    L = feti.weighted_trace(rho ** 3, op, Ws)
    L.backward()
    g = rho.grad.numpy()
    Lo = sum(O.loss_sub(s, W) for s, W in zip(P.subs, Ws))
    op.close()
    assert abs(L.item() - Lo) <= 1e-10 * abs(Lo)
    off = 0
    for i, s in enumerate(P.subs):
        ne = s.elem_dofs.shape[0]
        go = O.gradient_sub(s, Ws[i], P.K_ref)  # uses elem_dcoef = 3 rho^2
        assert np.linalg.norm(g[off:off + ne] - go) <= 1e-10 * np.linalg.norm(go)
        off += ne


def test_adjoint_forms_batches_and_recompute(torch_cuda):
    """The same gradient from (a) the compact dK_e = scale_e K_ref form, (b) one
    dK_e matrix per element, (c) a work budget that forces one subdomain per
    batch, and (d) recompute_X (X_i released after the assembly and after the
    adjoint, recomputed from L_i): (a), (c), (d) bitwise (each output is formed
    by the same arithmetic in the same order), (b) to rounding."""
    from paper_2502_08382_gb300 import feti
    P = _problem()
    Ws = make_W(P, seed=3)
    ref = feti.FetiOperator(P, prec="split_bf16", with_elements=True)
    ref.assemble()
    g_a = ref.adjoint(Ws).cpu().numpy()
    g_a2 = ref.adjoint(Ws).cpu().numpy()
    ref.close()
    per = feti.FetiOperator(P, prec="split_bf16", with_elements=True, per_element=True)
    per.assemble()
    g_b = per.adjoint(Ws).cpu().numpy()
    per.close()
    one = feti.FetiOperator(P, prec="split_bf16", with_elements=True, adjoint_work_bytes=1)
    one.assemble()
    g_c = one.adjoint(Ws).cpu().numpy()
    one.close()
    rec = feti.FetiOperator(P, prec="split_bf16", with_elements=True, recompute_X=True)
    rec.assemble()
    F0 = rec.get_F(2)
    rec.assemble()  # X_i re-allocated and recomputed
    assert np.array_equal(rec.get_F(2), F0)
    g_d = rec.adjoint(Ws).cpu().numpy()
    g_d2 = rec.adjoint(Ws).cpu().numpy()
    rec.close()
    assert np.array_equal(g_a, g_a2)
    assert np.array_equal(g_a, g_c)
    assert np.array_equal(g_a, g_d) and np.array_equal(g_a, g_d2)
    assert np.linalg.norm(g_b - g_a) <= 1e-13 * np.linalg.norm(g_a)


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
def test_weighted_trace_matches_oracle(torch_cuda, prec):
    """feti_weighted_trace against sum_i <W_i, F_i> of the oracle's F_i; the bar is
    sum_i ||W_i||_F ||F_i||_F times the F bar of the precision."""
    from bounds import F_bar
    from paper_2502_08382_gb300 import feti
    P = _problem()
    Ws = make_W(P, seed=4)
    op = feti.FetiOperator(P, prec=prec)
    op.assemble()
    L = op.weighted_trace(Ws).item()
    L2 = op.weighted_trace(Ws).item()
    op.close()
    Fs = [O.local_F(s) for s in P.subs]
    Lo = sum(float(np.sum(W * F)) for W, F in zip(Ws, Fs))
    bar = sum(np.linalg.norm(W) * np.linalg.norm(F) * F_bar(prec, F, s.n) for W, F, s in zip(Ws, Fs, P.subs))
    assert L == L2
    assert abs(L - Lo) <= bar, (L, Lo, bar)
