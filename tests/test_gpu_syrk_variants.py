"""The three split-bf16 SYRK kernels (options.syrk_kernel): all threads load
and one issues, 64-deep chunks in the 128-byte swizzle, one CTA per SM (0);
warp-specialised producers / issuer / epilogue (1); as 0 with 32-deep chunks in
the 64-byte swizzle and two CTAs per SM (2).  Each issues the same MMAs in the
same order (zero chunks beyond a supernode's width add exact zeros), so F_i
agrees bit for bit between them, and each meets the oracle's bar."""
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
    "cfg2_2x2": lambda: make_config(2, nsub_axis=2),
    "elast3d_2x2x2": lambda: make_problem(dim=3, physics="elasticity", cuts=[[4, 6]] * 3, material="density",
                                          seed=2),
    "cfg3_2x2x2": lambda: make_config(3, nsub_axis=2),
}


@pytest.mark.parametrize("name", list(CASES))
def test_syrk_kernels_agree(torch_cuda, name):
    from paper_2502_08382_gb300 import feti
    P = CASES[name]()
    Fs = []
    for v in range(3):
        op = feti.FetiOperator(P, prec="split_bf16", syrk_kernel=v)
        op.assemble()
        assert op.stats()["syrk_variant"] == v
        Fs.append([op.get_F(i) for i in range(P.nsub)])
        op.close()
    for v in (1, 2):
        for i in range(P.nsub):
            assert np.array_equal(Fs[0][i], Fs[v][i]), (v, i)
    idx = range(P.nsub) if P.nsub <= 8 else np.random.default_rng(0).choice(P.nsub, 8, replace=False)
    for i in idx:
        s = P.subs[i]
        Fo = O.local_F(s)
        err = np.linalg.norm(Fs[2][i] - Fo) / np.linalg.norm(Fo)
        assert err <= F_bar("split_bf16", Fo, s.n), (i, err)
