"""feti_apply_one_static: the explicit apply of one local operator with no
device allocation (intermediates in fixed device arrays of the library).

Callers that cannot allocate device memory when they apply the operator
(a framework whose pool owns all device memory, or a loop where cudaMalloc's
device synchronisation is not acceptable) use this entry point.  The test
feeds it the F_i that feti_assemble produced, re-laid into the documented tile
layout, one subdomain at a time, and compares the accumulated q with
feti_apply on two calls in a row.  Kept in its own file so pytest collects it
last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2502_08382_gb300.problems import make_problem, seeded_vector

pytestmark = pytest.mark.gpu


def _tiles(F, esz):
    """Lay a dense m x m symmetric F out as 64 x 64 lower tiles in the documented
    layout: tiles (bi, bj <= bi) one after another, the last block row ragged;
    off-diagonal tiles row-major; diagonal tiles keep for row r only the first
    w ceil((r + 1) / w) values (w = 16 / esz), zeros right of the diagonal."""
    m = F.shape[0]
    nb = (m + 63) // 64
    vr = m - 64 * (nb - 1)
    Fp = np.zeros((nb * 64, nb * 64))
    Fp[:m, :m] = F
    w = 16 // esz
    out = []
    for bi in range(nb):
        rows = 64 if bi < nb - 1 else vr
        for bj in range(bi + 1):
            t = Fp[bi * 64:bi * 64 + rows, bj * 64:(bj + 1) * 64]
            if bj < bi:
                out.append(t.ravel())
            else:
                for r in range(rows):
                    keep = w * ((r + 1 + w - 1) // w)
                    row = t[r, :keep].copy()
                    row[r + 1:] = 0.0
                    out.append(row)
    return np.concatenate(out)


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
def test_apply_one_static_matches_feti_apply(prec):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2502_08382_gb300 import feti
    lib = feti.load_library()
    P = make_problem(dim=3, physics="heat", cuts=[[5, 9, 7]] * 3, material="lognormal", sigma=0.5, seed=1)
    op = feti.FetiOperator(P, prec=prec)
    op.assemble()
    dt = torch.float32 if prec != "fp64" else torch.float64
    Fdev, maps = [], []
    for i, s in enumerate(P.subs):
        Fdev.append(torch.from_numpy(_tiles(op.get_F(i), 8 if prec == "fp64" else 4)).to(dt).cuda())
        maps.append(torch.from_numpy(np.asarray(s.B_lambda, dtype=np.int32)).cuda())
    p = torch.from_numpy(seeded_vector(P.n_lambda, 9)).cuda()
    q_ref = op.apply(p)
    torch.cuda.synchronize()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    tol = 1e-12 if prec == "fp64" else 1e-5
    for _call in range(2):
        q = torch.zeros_like(p)
        for i, s in enumerate(P.subs):
            rc = lib.feti_apply_one_static(s.m, 1 if prec != "fp64" else 0, C.c_void_p(Fdev[i].data_ptr()),
                                           C.c_void_p(maps[i].data_ptr()), C.c_void_p(p.data_ptr()),
                                           C.c_void_p(q.data_ptr()), stream)
            assert rc == 0, rc
        err = (torch.linalg.norm(q - q_ref) / torch.linalg.norm(q_ref)).item()
        assert err <= tol, err
    # sizes beyond the fixed scratch are rejected before anything is launched
    rc = lib.feti_apply_one_static(8193, 0, C.c_void_p(Fdev[0].data_ptr()), C.c_void_p(maps[0].data_ptr()),
                                   C.c_void_p(p.data_ptr()), C.c_void_p(q.data_ptr()), stream)
    assert rc == 1
    op.close()
