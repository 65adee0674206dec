"""Host-side checks that need no GPU.

* The C-ABI library loads and exports every entry point that the public
  header declares (no compute call is made).
* The host symbolic analysis (nested-dissection ordering, elimination tree,
  relaxed supernodes; the once-per-pattern step the paper keeps on the CPU)
  is checked against brute-force symbolic elimination of the permuted
  pattern: every fill entry of L lies in the supernode's own columns or in
  an ancestor supernode, the rows below each supernode are exactly the
  union of its columns' pattern and its children's rows, and the reported
  sizes and Cholesky flop count follow from (width, rows below).
"""
import os
import re

import numpy as np
import pytest

from paper_2502_08382_gb300 import build_lib, feti
from paper_2502_08382_gb300.problems import make_problem

HEADER = os.path.join(os.path.dirname(__file__), "..", "include", "feti.h")


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return feti.load_library()


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(feti_[A-Za-z_0-9]+)\s*\(", txt)))


def test_header_exports(lib):
    names = _declared()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(feti.EXPORTS)
    assert lib.feti_version().decode()


def _pattern(sub):
    n = sub.n
    A = np.zeros((n, n), dtype=bool)
    for r in range(n):
        A[r, sub.K_col[sub.K_rowptr[r]:sub.K_rowptr[r + 1]]] = True
    return A


def _brute_fill(A):
    """Structure of the Cholesky factor by plain symbolic elimination."""
    M = A.copy()
    n = M.shape[0]
    for k in range(n):
        rows = np.nonzero(M[k + 1:, k])[0] + k + 1
        if rows.size:
            M[np.ix_(rows, rows)] = True
    return np.tril(M)


CASES = [
    dict(dim=2, physics="heat", cuts=[[16, 16]] * 2, material="const", seed=0),
    dict(dim=2, physics="heat", cuts=[[9, 13]] * 2, material="lognormal", sigma=1.0, seed=4),
    dict(dim=3, physics="heat", cuts=[[5, 7]] * 3, material="lognormal", sigma=0.5, seed=1),
    dict(dim=3, physics="elasticity", cuts=[[4, 3]] * 3, material="const", seed=0),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("use_coords", [True, False])
def test_symbolic_vs_brute_force(lib, case, use_coords):
    P = make_problem(**CASES[case])
    for sub in P.subs[:2]:
        info = feti.analyse(sub, leaf_dofs=16, use_coords=use_coords)
        n = sub.n
        perm = info["perm"]
        assert sorted(perm.tolist()) == list(range(n))
        c0, w, par, r = info["sn_c0"], info["sn_w"], info["sn_parent"], info["sn_r"]
        ns = len(c0)
        assert c0[0] == 0 and np.all(c0[1:] == c0[:-1] + w[:-1]) and c0[-1] + w[-1] == n
        assert np.all((par == -1) | (par > np.arange(ns)))
        assert int(info["nroots"]) == int((par < 0).sum())
        col2sn = np.repeat(np.arange(ns), w)

        A = _pattern(sub)[np.ix_(perm, perm)]
        Lb = _brute_fill(A)
        anc = []
        for s in range(ns):
            a, t = set(), par[s]
            while t >= 0:
                a.add(int(t))
                t = par[t]
            anc.append(a)
        kids = [[] for _ in range(ns)]
        for s in range(ns):
            if par[s] >= 0:
                kids[par[s]].append(s)
        rows = [None] * ns
        for s in range(ns):
            end = c0[s] + w[s]
            own = set()
            for j in range(c0[s], end):
                fill = np.nonzero(Lb[end:, j])[0] + end
                # fill of column j lies in ancestor supernodes (etree property)
                assert all(int(col2sn[i]) in anc[s] for i in fill), (s, j)
                own.update(np.nonzero(A[end:, j])[0] + end)
            for c in kids[s]:
                own.update(i for i in rows[c] if i >= end)
            rows[s] = own
            assert len(own) == r[s], (s, len(own), r[s])
            # the exact fill of the supernode's columns is covered
            cover = set()
            for j in range(c0[s], end):
                cover.update(np.nonzero(Lb[end:, j])[0] + end)
            assert cover <= own

        wf, rf = w.astype(float), r.astype(float)
        assert info["Lsize"] == float(np.sum(wf * (wf + rf)))
        assert info["nnzL"] == float(np.sum(wf * (wf + 1) / 2 + wf * rf))
        assert info["nnzL"] >= float(Lb.sum())
        fl = 0.0
        for ws, rs in zip(w, r):
            for k in range(ws):
                rem = ws + rs - k - 1
                fl += 1 + rem + rem * (rem + 1)
        assert info["chol_flops"] == pytest.approx(fl, rel=1e-12)
        assert info["max_front"] == float(np.max(w + r)) and info["max_width"] == float(np.max(w))
        assert info["m"] == sub.m


@pytest.mark.parametrize("case", range(len(CASES)))
def test_trsm_syrk_counts(lib, case):
    """The algorithmic TRSM and SYRK flop counts that the rooflines divide by, recomputed from the plan:
    column j of X = L^{-1} P B^T starts in the supernode holding its permuted DOF and reaches every supernode
    on the path to the root, so J_s counts the columns starting in the subtree of s; TRSM = sum_s J_s (w_s^2 +
    2 w_s r_s), SYRK = sum_s w_s J_s (J_s + 1), X = sum_s ceil8(w_s) J_s stored values (rows padded to 8).  The SYRK count is
    bounded by the suffix model sum_{a <= b} 2 (n - max(s_a, s_b)) and the TRSM count by the model that
    counts each supernode's triangle twice, sum_s J_s 2 w_s (w_s + r_s)."""
    P = make_problem(**CASES[case])
    for sub in P.subs[:3]:
        info = feti.analyse(sub, leaf_dofs=16)
        n = sub.n
        perm = info["perm"]
        iperm = np.empty(n, dtype=np.int64)
        iperm[perm] = np.arange(n)
        w, par, r = info["sn_w"].astype(np.int64), info["sn_parent"], info["sn_r"].astype(np.int64)
        col2sn = np.repeat(np.arange(len(w)), w)
        J = np.zeros(len(w), dtype=np.int64)
        start = iperm[np.asarray(sub.B_dof, dtype=np.int64)]
        for p0 in start:
            t = int(col2sn[p0])
            while t >= 0:
                J[t] += 1
                t = int(par[t])
        trsm = float(np.sum(J * (w * w + 2 * w * r)))
        syrk = float(np.sum(w * J * (J + 1)))
        xs = float(np.sum(((w + 7) // 8 * 8) * J))
        assert info["trsm_flops"] == pytest.approx(trsm, rel=1e-12)
        assert info["syrk_flops"] == pytest.approx(syrk, rel=1e-12)
        assert info["Xsize"] == xs
        sa = np.sort(start)
        m = len(sa)
        # sum over a <= b of 2 (n - max(s_a, s_b)): with sorted starts, pair (a, b <= a) has max s_a
        suffix = float(np.sum(2.0 * (n - sa) * (np.arange(m) + 1)))
        assert syrk <= suffix
        assert trsm <= float(np.sum(J * 2 * w * (w + r))) <= 2 * trsm


def test_nested_dissection_reduces_fill(lib):
    """On a 64 x 64 Q1 grid (the 2D heat subdomain) the exact fill of the
    nested-dissection order is well below the banded fill of the natural
    lexicographic order, and relaxed amalgamation stores a bounded number of
    explicit zeros on top of it."""
    P = make_problem(dim=2, physics="heat", cuts=[[64, 64]] * 2, material="const", seed=0)
    sub = P.subs[0]
    A = _pattern(sub)
    nat = float(_brute_fill(A).sum())
    info = feti.analyse(sub, leaf_dofs=16, use_coords=True)
    perm = info["perm"]
    nd = float(_brute_fill(A[np.ix_(perm, perm)]).sum())
    assert nd < 0.5 * nat
    assert nd <= info["nnzL"] < 1.5 * nd


# ---------------------------------------------------------------- input validation (host fault injection)
#
# feti_create validates every input on the host before it touches the GPU,
# so malformed problems are rejected with FETI_ERR_ARG and a message here,
# without a device.  Each case corrupts one field of a valid problem.


def _create_status(P, corrupt):
    import ctypes as C
    lib = feti.load_library()
    m = feti._Marshal(P)
    corrupt(m)
    h = C.c_void_p()
    opt = feti.FetiOptions()
    rc = lib.feti_create(C.byref(m.prob), C.byref(opt), C.byref(h))
    msg = lib.feti_last_error(h).decode() if h else ""
    if h:
        lib.feti_destroy(h)
    return rc, msg


def _set_int(arr_ptr, idx, val):
    arr_ptr[idx] = val


BAD_INPUTS = {
    "no_subdomains": (lambda m: setattr(m.prob, "nsub", 0), ""),
    "nfix_ne_d": (lambda m: setattr(m.subs[0], "nfix", 0), "nfix must equal d"),
    "B_two_entries": (lambda m: _set_int(m.subs[1].B_rowptr, 1, 2), "exactly one entry"),
    "B_not_unit": (lambda m: _set_int(m.subs[0].B_val, 0, 0.5), "+1 or -1"),
    "B_lambda_order": (lambda m: _set_int(m.subs[0].B_lambda, 1, -5), "strictly increasing"),
    "K_col_range": (lambda m: _set_int(m.subs[2].K_col, 3, 10 ** 6), "out of range"),
    "K_unsorted": (lambda m: (_set_int(m.subs[0].K_col, 1, m.subs[0].K_col[0])), "sorted and unique"),
    "fix_range": (lambda m: _set_int(m.subs[0].fix_dofs, 0, -1), "fix DOF out of range"),
    "B_dof_range": (lambda m: _set_int(m.subs[3].B_col, 0, 10 ** 6), "B column out of range"),
}


def test_create_rejects_bad_options(lib):
    """Unknown precision or preconditioner codes are rejected on the host."""
    import ctypes as C
    P = make_problem(dim=2, physics="heat", cuts=[[3, 4]] * 2, material="const", seed=0)
    for field, val, words in (("prec", 7, "bad precision"), ("precond", 5, "bad preconditioner")):
        m = feti._Marshal(P)
        opt = feti.FetiOptions()
        setattr(opt, field, val)
        h = C.c_void_p()
        rc = lib.feti_create(C.byref(m.prob), C.byref(opt), C.byref(h))
        msg = lib.feti_last_error(h).decode() if h else ""
        if h:
            lib.feti_destroy(h)
        assert rc == 1 and words in msg, (field, rc, msg)


@pytest.mark.parametrize("name", list(BAD_INPUTS))
def test_create_rejects_malformed_input(lib, name):
    P = make_problem(dim=2, physics="heat", cuts=[[3, 4]] * 2, material="const", seed=0)
    corrupt, words = BAD_INPUTS[name]
    rc, msg = _create_status(P, corrupt)
    assert rc == 1, (rc, msg)  # FETI_ERR_ARG
    assert words in msg, msg


def test_apply_one_static_rejects_sizes_on_host(lib):
    """Sizes beyond the fixed scratch (and non-positive ones) are rejected
    before any device work is issued."""
    import ctypes as C
    one = C.c_void_p(16)
    for m in (0, -3, 8193, 1 << 20):
        assert lib.feti_apply_one_static(m, 1, one, one, one, one, None) == 1
    assert lib.feti_apply_one_static(64, 1, None, one, one, one, None) == 1


def test_lumped_plan_matches_oracle(lib):
    """The host plan of the lumped preconditioner (no device): W against the
    oracle's (B B^T)^{-1}, the summed M_core contributions against the
    oracle's sum_i B_i K_i B_i^T, and W M_core W against its scaled form."""
    from oracle import feti_oracle as O
    for P in (make_problem(dim=2, physics="heat", cuts=[[4, 5, 3]] * 2, material="lognormal", sigma=1.0, seed=3),
              make_problem(dim=3, physics="elasticity", cuts=[[2, 3]] * 3, material="density", seed=3)):
        pl = feti.lumped_plan(P)
        n = P.n_lambda
        W = np.zeros((n, n))
        for a in range(n):
            for k in range(pl["w_off"][a], pl["w_off"][a + 1]):
                W[a, pl["w_col"][k]] = pl["w_val"][k]
        Kall = np.concatenate([s.K_val for s in P.subs])
        Mc = np.zeros((n, n))
        for a in range(n):
            for e in range(pl["m_off"][a], pl["m_off"][a + 1]):
                c0, c1 = pl["c_off"][e], pl["c_off"][e + 1]
                Mc[a, pl["m_col"][e]] = np.sum(pl["c_sign"][c0:c1] * Kall[pl["c_kidx"][c0:c1]])
        Wo = np.linalg.inv(O.BBt(P))
        Mo = O.lumped_M(P)
        assert np.abs(W - Wo).max() <= 1e-12 * np.abs(Wo).max()
        assert np.abs(Mc - Mo).max() <= 1e-12 * np.abs(Mo).max()
        So = O.scaled_lumped_M(P)
        assert np.abs(W @ Mc @ W - So).max() <= 1e-12 * np.abs(So).max()
