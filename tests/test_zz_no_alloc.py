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
    q = torch.zeros_like(p)
    free = []
    for _call in range(2):
        q.zero_()
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        for i, s in enumerate(P.subs):
            rc = lib.feti_apply_one_static(s.m, 1 if prec != "fp64" else 0, C.c_void_p(Fdev[i].data_ptr()),
                                           C.c_void_p(maps[i].data_ptr()), C.c_void_p(p.data_ptr()),
                                           C.c_void_p(q.data_ptr()), stream)
            assert rc == 0, rc
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        err = (torch.linalg.norm(q - q_ref) / torch.linalg.norm(q_ref)).item()
        assert err <= tol, err
    # the second round of calls takes no device memory (the first may load the library's device code)
    assert free[3] == free[2], free
    # sizes beyond the fixed scratch are rejected before anything is launched
    rc = lib.feti_apply_one_static(8193, 0, C.c_void_p(Fdev[0].data_ptr()), C.c_void_p(maps[0].data_ptr()),
                                   C.c_void_p(p.data_ptr()), C.c_void_p(q.data_ptr()), stream)
    assert rc == 1
    op.close()


@pytest.mark.parametrize("m", [128, 8192])
def test_apply_one_static_dense_extremes(m):
    """A synthetic symmetric F with a full last block row (m = 128) and at the
    largest accepted size (m = 8192), in FP64 and FP32 tiles, against the dense
    product F p[map] computed with NumPy; two calls in a row accumulate 2 F p."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2502_08382_gb300 import feti
    lib = feti.load_library()
    rng = np.random.default_rng([m, 31])
    A = rng.standard_normal((m, m))
    F = (A + A.T) / 2
    n_lambda = m + 37
    lam = np.sort(rng.choice(n_lambda, m, replace=False)).astype(np.int32)
    p_h = rng.standard_normal(n_lambda)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    mp = torch.from_numpy(lam).cuda()
    p = torch.from_numpy(p_h).cuda()
    nb = (m + 63) // 64
    for fp32, dt, u in ((0, torch.float64, 2.0 ** -53), (1, torch.float32, 2.0 ** -24)):
        # componentwise bound of a product accumulated over at most m + nb + 2 terms in the tile
        # precision (p itself rounded to it in the FP32 case), doubled by the second call
        k = m + nb + 2
        tol = k * u / (1 - k * u) + u
        Ft = torch.from_numpy(_tiles(F, 4 if fp32 else 8)).to(dt).cuda()
        q = torch.zeros(n_lambda, dtype=torch.float64, device="cuda")
        for _call in range(2):
            rc = lib.feti_apply_one_static(m, fp32, C.c_void_p(Ft.data_ptr()), C.c_void_p(mp.data_ptr()),
                                           C.c_void_p(p.data_ptr()), C.c_void_p(q.data_ptr()), stream)
            assert rc == 0, rc
        got = q.cpu().numpy()
        Fr = F.astype(np.float32).astype(np.float64) if fp32 else F
        want = np.zeros(n_lambda)
        want[lam] = 2 * (Fr @ p_h[lam])
        scale = 2 * (np.abs(Fr) @ np.abs(p_h[lam]))
        assert np.all(np.abs(got[lam] - want[lam]) <= tol * scale), (fp32, np.max(
            np.abs(got[lam] - want[lam]) / scale))
        assert np.all(got[np.setdiff1d(np.arange(n_lambda), lam)] == 0.0)
