"""Workload 5 at full size: 3D elasticity sensitivity, 6 x 6 x 6 = 216
subdomains of 16^3 Hex8 elements (14 739 DOFs each, m_i 2451..4902,
n_lambda = 473 832), densities rho_e ~ U[0.1, 1] with E_e = rho_e^3, nu = 0.3,
clamped at x = 0.

The loss L = sum_i <W_i, F_i> and its gradient run through the autograd
function (forward: FP64 feti_assemble with X_i released afterwards
(recompute_X) and feti_weighted_trace; backward: the batched FP64 adjoint,
X_i recomputed from L_i).  The oracle factorises three subdomains densely
(the smallest and the largest m_i and a seeded one), so W_i is the seeded
symmetric N(0, 1) matrix on those and zero elsewhere:
  * F_i of those subdomains against B K_reg^{-1} B^T (1e-12 relative);
  * L against sum <W_i, F_i> of the oracle's F_i;
  * dL/drho_e on every element of those subdomains against the oracle's
    gradient (1e-10 relative), and exactly zero on every other element;
  * central differences (h = 1e-6, rho_pen frozen) on 50 seeded elements of
    those subdomains, the loss difference taken through the Woodbury form of
    the element-rank update (one factorisation per subdomain), 1e-6 relative.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import feti_oracle as O
from paper_2502_08382_gb300.problems import make_config, make_W_sub

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def test_workload5_full_size_sensitivity(torch_cuda):
    torch = torch_cuda
    from paper_2502_08382_gb300 import feti
    P = make_config(5)
    assert P.nsub == 216 and P.n_lambda == 473832
    ms = np.array([s.m for s in P.subs])
    rng = np.random.default_rng([0, 13])
    picks = sorted({int(np.argmin(ms)), int(np.argmax(ms)), int(rng.integers(P.nsub))})
    Ws = {i: make_W_sub(P.subs[i].m, 0, i) for i in picks}
    # W on the device (sum m_i^2 values, zero outside the picked subdomains), built in place
    woff = np.concatenate([[0], np.cumsum(ms.astype(np.int64) ** 2)])
    Wd = torch.zeros(int(woff[-1]), dtype=torch.float64, device="cuda")
    for i in picks:
        Wd[int(woff[i]):int(woff[i + 1])] = torch.from_numpy(Ws[i].ravel()).cuda()
    op = feti.FetiOperator(P, prec="fp64", with_elements=True, unit_scale=True, recompute_X=True)
    rho0 = np.concatenate([s.elem_coef ** (1.0 / 3.0) for s in P.subs])
    rho = torch.tensor(rho0, dtype=torch.float64, requires_grad=True)
    L = feti.weighted_trace(rho ** 3, op, Wd)
    L.backward()
    g = rho.grad.numpy()
    Fg = {i: op.get_F(i) for i in picks}
    op.close()

    offs = np.concatenate([[0], np.cumsum([s.elem_dofs.shape[0] for s in P.subs])])
    mask = np.ones(offs[-1], dtype=bool)
    for i in picks:
        mask[offs[i]:offs[i + 1]] = False
    assert np.all(g[mask] == 0.0)

    Lo = 0.0
    cho = {}
    for i in picks:
        s = P.subs[i]
        Kr = O.K_reg(s)
        cho[i] = sla.cho_factor(Kr, lower=True)
        Fo = O.local_F(s, Kr)
        err = np.linalg.norm(Fg[i] - Fo) / np.linalg.norm(Fo)
        print(f"workload 5: F_{i} (m = {s.m}) relative error {err:.2e}")
        assert err <= 1e-12, (i, err)
        Lo += float(np.sum(Ws[i] * Fo))
        go = O.gradient_sub(s, Ws[i], P.K_ref, Kr=Kr)
        gi = g[offs[i]:offs[i + 1]]
        gerr = np.linalg.norm(gi - go) / np.linalg.norm(go)
        print(f"workload 5: dL/drho on the {s.elem_dofs.shape[0]} elements of subdomain {i}: relative error "
              f"{gerr:.2e}")
        assert gerr <= 1e-10, (i, gerr)
    Lbar = sum(np.linalg.norm(Ws[i]) * np.linalg.norm(Fg[i]) for i in picks) * 1e-12
    assert abs(L.item() - Lo) <= Lbar, (L.item(), Lo)

    # central differences on 50 seeded elements of the factorised subdomains (C12: purpose 4)
    pool = np.concatenate([np.arange(offs[i], offs[i + 1]) for i in picks])
    fd_pick = np.random.default_rng([0, 4]).choice(pool, size=50, replace=False)
    worst = 0.0
    for ge in fd_pick:
        i = int(np.searchsorted(offs, ge, side="right") - 1)
        e = int(ge - offs[i])
        s = P.subs[i]
        th = s.elem_coef[e] ** (1.0 / 3.0)
        h = 1e-6
        dL = O.loss_difference_lowrank(s, Ws[i], cho[i], e, (th + h) ** 3 - th ** 3, (th - h) ** 3 - th ** 3,
                                       P.K_ref)
        fd = dL / (2 * h)
        rel = abs(fd - g[ge]) / max(1.0, abs(fd))
        worst = max(worst, rel)
        assert rel <= 1e-6, (ge, fd, g[ge])
    print(f"workload 5: central differences on 50 elements, worst relative difference {worst:.2e}")
