"""Seeded synthetic FETI problems on structured meshes (inputs only).

This module builds the *inputs* of the dual-operator path and nothing else:
per-subdomain stiffness matrices K_i (full symmetric CSR), gluing matrices
B_i (one signed unit per row), kernel bases R_i, load vectors f_i, fixing
DOFs, element data for sensitivities, and the bookkeeping a monolithic FEM
solve needs (local-to-global maps, Dirichlet DOFs).  It contains none of the
method's arithmetic (no regularisation, factorisation, dual operator, PCPG).
Both the CUDA path and the CPU oracle consume its output, so it is the one
module they share.

Mesh/physics readings (paper Sec. V uses triangles/tetrahedra; the workloads
here are Q1 quads and Hex8 bricks on the unit square/cube):
  * heat: K_e = k_e * int grad N . grad N, full Gauss integration (2 points
    per axis), consistent load f = 1;
  * elasticity: isotropic, E_e, nu = 0.3, Voigt strain (xx,yy,zz,yz,xz,xy),
    consistent body force (0, 0, -1).
Gluing follows Total FETI (Sec. II, eqs. 2-3): Dirichlet DOFs become rows of
B with c = 0 on the lowest-numbered subdomain owning the node; a node shared
by k subdomains gets k-1 chained rows between consecutive sorted subdomain
ids, +1 on the lower id and -1 on the higher.  Multipliers are ordered by
(global node, chain position, component) with the Dirichlet rows first.
Random streams: numpy default_rng([seed, purpose]) with purpose 0 =
conductivity, 1 = cuts, 2 = densities, 3 = W_i, 4 = element picks.
"""
from __future__ import annotations

import dataclasses
import functools
import itertools
from typing import List, Optional, Sequence

import numpy as np
import scipy.linalg
import scipy.sparse as sp

# --------------------------------------------------------------------------
# reference element matrices (unit coefficient) by Gauss quadrature


def _gauss2():
    g = 1.0 / np.sqrt(3.0)
    return np.array([-g, g]), np.array([1.0, 1.0])


@functools.lru_cache(maxsize=None)
def _corners(dim):
    # itertools.product varies the last axis fastest; reverse so x is fastest.
    c = np.array(list(itertools.product((-1.0, 1.0), repeat=dim)))[:, ::-1]
    return np.ascontiguousarray(c)


def _shape_grads(dim, xi):
    """dN_a/dxi_k at reference point xi for the 2^dim corner nodes."""
    c = _corners(dim)
    n = c.shape[0]
    N = np.ones(n)
    dN = np.ones((n, dim))
    for k in range(dim):
        fk = 0.5 * (1.0 + c[:, k] * xi[k])
        N = N * fk
    for k in range(dim):
        for a in range(n):
            v = 0.5 * c[a, k]
            for l in range(dim):
                if l != k:
                    v *= 0.5 * (1.0 + c[a, l] * xi[l])
            dN[a, k] = v
    return N, dN


@functools.lru_cache(maxsize=None)
def ref_heat(dim, h):
    """Unit-conductivity element matrix and unit-source load of a cube of side h."""
    pts, wts = _gauss2()
    n = 2 ** dim
    K = np.zeros((n, n))
    f = np.zeros(n)
    jac = (h / 2.0) ** dim
    for idx in itertools.product(range(2), repeat=dim):
        xi = np.array([pts[i] for i in idx])
        w = np.prod([wts[i] for i in idx])
        N, dN = _shape_grads(dim, xi)
        G = dN * (2.0 / h)
        K += w * jac * (G @ G.T)
        f += w * jac * N
    K.setflags(write=False)
    f.setflags(write=False)
    return K, f


@functools.lru_cache(maxsize=None)
def ref_elasticity(h, nu):
    """Unit-modulus Hex8 element matrix (24x24, DOF = 3*node + comp) and the
    consistent load of a unit body force per component (8 nodes)."""
    pts, wts = _gauss2()
    E = 1.0
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    K = np.zeros((24, 24))
    fN = np.zeros(8)
    jac = (h / 2.0) ** 3
    for idx in itertools.product(range(2), repeat=3):
        xi = np.array([pts[i] for i in idx])
        w = np.prod([wts[i] for i in idx])
        N, dN = _shape_grads(3, xi)
        G = dN * (2.0 / h)  # 8 x 3
        Bm = np.zeros((6, 24))
        for a in range(8):
            gx, gy, gz = G[a]
            Bm[0, 3 * a + 0] = gx
            Bm[1, 3 * a + 1] = gy
            Bm[2, 3 * a + 2] = gz
            Bm[3, 3 * a + 1] = gz
            Bm[3, 3 * a + 2] = gy
            Bm[4, 3 * a + 0] = gz
            Bm[4, 3 * a + 2] = gx
            Bm[5, 3 * a + 0] = gy
            Bm[5, 3 * a + 1] = gx
        K += w * jac * (Bm.T @ D @ Bm)
        fN += w * jac * N
    K = 0.5 * (K + K.T)
    K.setflags(write=False)
    fN.setflags(write=False)
    return K, fN


# --------------------------------------------------------------------------
# data containers


@dataclasses.dataclass
class Subdomain:
    n: int                      # DOFs
    K_rowptr: np.ndarray        # int64 [n+1]
    K_col: np.ndarray           # int32 [nnz], sorted per row
    K_val: np.ndarray           # float64 [nnz], full symmetric
    B_lambda: np.ndarray        # int32 [m], global multiplier id of row r (increasing)
    B_dof: np.ndarray           # int32 [m], local DOF touched by row r
    B_sign: np.ndarray          # float64 [m], +1 / -1
    R: np.ndarray               # float64 [n, d] kernel basis (column j = R[:, j])
    f: np.ndarray               # float64 [n]
    fix_dofs: np.ndarray        # int32 [d]
    coords: np.ndarray          # float64 [n, 3] coordinates of each DOF's node
    l2g: np.ndarray             # int64 [n] global DOF of each local DOF
    elem_dofs: np.ndarray       # int32 [nelem, edofs]
    elem_coef: np.ndarray       # float64 [nelem] material coefficient multiplying K_ref
    elem_dcoef: np.ndarray      # float64 [nelem] d(coef)/d(theta_e)
    elem_global: np.ndarray     # int64 [nelem] global element id
    shape: tuple                # elements per axis

    @property
    def m(self):
        return int(self.B_lambda.shape[0])

    @property
    def d(self):
        return int(self.R.shape[1])

    @property
    def nnz(self):
        return int(self.K_col.shape[0])

    def B_rowptr(self):
        return np.arange(self.m + 1, dtype=np.int64)

    def K_dense(self):
        return sp.csr_matrix((self.K_val, self.K_col, self.K_rowptr), shape=(self.n, self.n)).toarray()

    def B_dense(self):
        Bd = np.zeros((self.m, self.n))
        Bd[np.arange(self.m), self.B_dof] = self.B_sign
        return Bd


@dataclasses.dataclass
class Problem:
    name: str
    dim: int
    physics: str                # "heat" | "elasticity"
    dpn: int                    # DOFs per node
    h: float
    n_global_dofs: int
    dirichlet_dofs: np.ndarray  # global DOFs fixed to 0
    subs: List[Subdomain]
    n_lambda: int
    c: np.ndarray               # float64 [n_lambda]
    K_ref: np.ndarray           # reference element matrix (unit coefficient)
    elem_global_shape: tuple    # global elements per axis
    seed: int

    @property
    def nsub(self):
        return len(self.subs)

    def global_solution_coords(self):
        """Coordinates of every global DOF's node (for closed-form checks)."""
        out = np.zeros((self.n_global_dofs, 3))
        for s in self.subs:
            out[s.l2g] = s.coords
        return out


# --------------------------------------------------------------------------
# builders


def _random_cuts(total, count, lo, hi, rng):
    """Seeded subdomain widths: count iid integers in [lo, hi] redrawn until
    they sum to total (one draw of `count` values per attempt)."""
    if count * lo > total or count * hi < total:
        raise ValueError("cut range cannot reach the total")
    for _ in range(1_000_000):
        w = rng.integers(lo, hi + 1, size=count)
        if int(w.sum()) == total:
            return [int(x) for x in w]
    raise RuntimeError("cut sampling did not converge")


@functools.lru_cache(maxsize=64)
def _local_pattern(shape, dpn):
    """CSR pattern of a box subdomain and the position of every element-matrix
    entry in it.  Returns (rowptr, col, pos[nelem, edofs, edofs], elem_dofs)."""
    dim = len(shape)
    nn = [e + 1 for e in shape]
    corners = _corners(dim).astype(np.int64)
    c01 = (corners + 1) // 2  # 0/1 offsets, x fastest
    # element origins, x fastest
    grids = np.meshgrid(*[np.arange(e) for e in shape], indexing="ij")
    org = np.stack([g.ravel(order="F") for g in grids], axis=1)  # x fastest
    strides = np.cumprod([1] + nn[:-1])
    enodes = ((org[:, None, :] + c01[None, :, :]) * strides[None, None, :]).sum(-1)  # nelem x 2^dim
    edofs = (enodes[:, :, None] * dpn + np.arange(dpn)[None, None, :]).reshape(enodes.shape[0], -1)
    n = int(np.prod(nn)) * dpn
    ne, ed = edofs.shape
    rows = np.repeat(edofs, ed, axis=1).ravel()
    cols = np.tile(edofs, (1, ed)).ravel()
    key = np.unique(rows * n + cols)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, (key // n) + 1, 1)
    rowptr = np.cumsum(rowptr)
    col = (key % n).astype(np.int32)
    pos = np.searchsorted(key, rows * n + cols).reshape(ne, ed, ed)
    for a in (rowptr, col, pos, edofs):
        a.setflags(write=False)
    return rowptr, col, pos, edofs.astype(np.int32)


def make_problem(*, dim: int, physics: str, cuts: Sequence[Sequence[int]],
                 material: str = "const", sigma: float = 1.0, nu: float = 0.3,
                 seed: int = 0, name: str = "custom") -> Problem:
    """Build a box of elements cut into subdomains.

    cuts[k] lists the element widths of the subdomains along axis k.
    material: "const" (coefficient 1), "lognormal" (k_e = exp(N(0, sigma^2))),
    "density" (rho_e ~ U[0.1, 1], E_e = rho_e^3; theta_e = rho_e).
    """
    assert dim in (2, 3) and physics in ("heat", "elasticity")
    dpn = 1 if physics == "heat" else dim
    assert not (physics == "elasticity" and dim != 3)
    NE = [int(sum(c)) for c in cuts]
    assert len(set(NE)) == 1, "the domain is the unit square/cube: equal element counts per axis"
    h = 1.0 / NE[0]
    NN = [e + 1 for e in NE]
    nglob_nodes = int(np.prod(NN))
    gstr = np.cumprod([1] + NN[:-1])
    estr = np.cumprod([1] + NE[:-1])
    nelem_glob = int(np.prod(NE))

    if physics == "heat":
        K_ref, f_ref = ref_heat(dim, h)
    else:
        K_ref, fN = ref_elasticity(h, nu)

    # per-element coefficients over the global element grid (x fastest)
    if material == "const":
        coef = np.ones(nelem_glob)
        dcoef = np.zeros(nelem_glob)
    elif material == "lognormal":
        rng = np.random.default_rng([seed, 0])
        g = rng.normal(0.0, sigma, size=nelem_glob)
        coef = np.exp(g)
        dcoef = coef.copy()  # d/d(log k) -- not used by the sensitivity workload
    elif material == "density":
        rng = np.random.default_rng([seed, 2])
        rho = rng.uniform(0.1, 1.0, size=nelem_glob)
        coef = rho ** 3
        dcoef = 3.0 * rho ** 2
    else:
        raise ValueError(material)

    offs = [np.concatenate([[0], np.cumsum(c)]).astype(np.int64) for c in cuts]
    nsub_axis = [len(c) for c in cuts]
    subs: List[Subdomain] = []
    owners = []  # (global node, sub, local node)
    for sidx in itertools.product(*[range(k) for k in nsub_axis[::-1]]):
        sidx = sidx[::-1]  # x fastest subdomain numbering
        shape = tuple(int(cuts[k][sidx[k]]) for k in range(dim))
        org = [int(offs[k][sidx[k]]) for k in range(dim)]
        rowptr, col, pos, edofs = _local_pattern(shape, dpn)
        nn = [e + 1 for e in shape]
        nloc_nodes = int(np.prod(nn))
        n = nloc_nodes * dpn
        # local node -> global node
        lg = np.meshgrid(*[np.arange(x) for x in nn], indexing="ij")
        lidx = np.stack([g.ravel(order="F") for g in lg], axis=1)  # x fastest
        gnode = ((lidx + np.array(org)[None, :]) * gstr[None, :]).sum(1)
        xyz = np.zeros((nloc_nodes, 3))
        xyz[:, :dim] = (lidx + np.array(org)[None, :]) * h
        # local elements -> global elements
        le = np.meshgrid(*[np.arange(x) for x in shape], indexing="ij")
        leidx = np.stack([g.ravel(order="F") for g in le], axis=1)
        gelem = ((leidx + np.array(org)[None, :]) * estr[None, :]).sum(1)
        ce = coef[gelem]
        vals = np.bincount(pos.ravel(), weights=(ce[:, None, None] * K_ref[None]).ravel(),
                           minlength=col.shape[0])
        # consistent load
        f = np.zeros(n)
        if physics == "heat":
            np.add.at(f, edofs.ravel(), np.tile(f_ref, edofs.shape[0]))
        else:
            zdofs = edofs.reshape(edofs.shape[0], 8, 3)[:, :, 2]
            np.add.at(f, zdofs.ravel(), np.tile(-fN, edofs.shape[0]))
        # kernel basis and fixing DOFs (centre node, plus two offset nodes in elasticity)
        coords = np.repeat(xyz, dpn, axis=0)
        centre = [x // 2 for x in nn]
        cnode = int(sum(centre[k] * int(np.prod(nn[:k])) for k in range(dim)))
        if physics == "heat":
            R = np.ones((n, 1))
            fix = np.array([cnode], dtype=np.int32)
        else:
            xc = xyz.mean(axis=0)
            rel = xyz - xc[None, :]
            R = np.zeros((n, 6))
            for k in range(3):
                R[k::3, k] = 1.0
            # rotations about z, x, y
            R[0::3, 3] = -rel[:, 1]; R[1::3, 3] = rel[:, 0]
            R[1::3, 4] = -rel[:, 2]; R[2::3, 4] = rel[:, 1]
            R[0::3, 5] = rel[:, 2];  R[2::3, 5] = -rel[:, 0]
            n2 = cnode + max(1, nn[0] // 4)
            n3 = cnode + max(1, nn[1] // 4) * nn[0]
            fix9 = np.array([3 * q + c for q in (cnode, n2, n3) for c in range(3)])
            _, _, piv = scipy.linalg.qr(R[fix9, :].T, pivoting=True)
            fix = np.sort(fix9[piv[:6]]).astype(np.int32)
        l2g = (np.repeat(gnode, dpn) * dpn + np.tile(np.arange(dpn), nloc_nodes)).astype(np.int64)
        sid = len(subs)
        owners.append(np.stack([gnode, np.full(nloc_nodes, sid), np.arange(nloc_nodes)], axis=1))
        subs.append(Subdomain(
            n=n, K_rowptr=rowptr.copy(), K_col=col.copy(), K_val=vals,
            B_lambda=None, B_dof=None, B_sign=None, R=R, f=f, fix_dofs=fix,
            coords=coords, l2g=l2g, elem_dofs=edofs.copy(), elem_coef=ce.copy(),
            elem_dcoef=dcoef[gelem].copy(), elem_global=gelem.astype(np.int64), shape=shape))

    # ---- gluing and Dirichlet rows (Total FETI) ----
    own = np.concatenate(owners)
    order = np.lexsort((own[:, 1], own[:, 0]))
    own = own[order]
    gn = own[:, 0]
    bounds = np.flatnonzero(np.diff(gn)) + 1
    starts = np.concatenate([[0], bounds])
    ends = np.concatenate([bounds, [gn.shape[0]]])
    counts = ends - starts
    # x-coordinate index of each global node (Dirichlet: x = 0)
    gx = gn % NN[0]
    rows_sub, rows_dof, rows_sign, rows_lam = [], [], [], []
    lam = 0
    # vectorised emission: per global node, Dirichlet rows then chain rows
    is_dir = gx[starts] == 0
    n_rows_node = (counts - 1 + is_dir.astype(np.int64)) * dpn
    lam_start = np.concatenate([[0], np.cumsum(n_rows_node)])
    n_lambda = int(lam_start[-1])
    # Dirichlet rows
    di = np.flatnonzero(is_dir)
    for comp in range(dpn):
        lid = lam_start[di] + comp
        r = own[starts[di]]
        rows_lam.append(lid); rows_sub.append(r[:, 1]); rows_dof.append(r[:, 2] * dpn + comp)
        rows_sign.append(np.ones(di.shape[0]))
    # chain rows
    maxk = int(counts.max())
    for k in range(maxk - 1):
        sel = np.flatnonzero(counts > k + 1)
        base = lam_start[sel] + is_dir[sel].astype(np.int64) * dpn + k * dpn
        a = own[starts[sel] + k]
        b = own[starts[sel] + k + 1]
        for comp in range(dpn):
            lid = base + comp
            rows_lam += [lid, lid]
            rows_sub += [a[:, 1], b[:, 1]]
            rows_dof += [a[:, 2] * dpn + comp, b[:, 2] * dpn + comp]
            rows_sign += [np.ones(sel.shape[0]), -np.ones(sel.shape[0])]
    L = np.concatenate(rows_lam)
    S = np.concatenate(rows_sub)
    Dd = np.concatenate(rows_dof)
    Sg = np.concatenate(rows_sign)
    o = np.lexsort((L, S))
    L, S, Dd, Sg = L[o], S[o], Dd[o], Sg[o]
    sb = np.searchsorted(S, np.arange(len(subs) + 1))
    for i, s in enumerate(subs):
        a, b = sb[i], sb[i + 1]
        s.B_lambda = L[a:b].astype(np.int32)
        s.B_dof = Dd[a:b].astype(np.int32)
        s.B_sign = Sg[a:b].astype(np.float64)
    dir_nodes = gn[starts[di]]
    dirichlet = (np.repeat(dir_nodes, dpn) * dpn + np.tile(np.arange(dpn), dir_nodes.shape[0])).astype(np.int64)
    return Problem(name=name, dim=dim, physics=physics, dpn=dpn, h=h,
                   n_global_dofs=nglob_nodes * dpn, dirichlet_dofs=np.sort(dirichlet),
                   subs=subs, n_lambda=n_lambda, c=np.zeros(n_lambda), K_ref=np.asarray(K_ref),
                   elem_global_shape=tuple(NE), seed=seed)


# --------------------------------------------------------------------------
# the five workloads (and same-shape smaller copies)

CONFIG_NAMES = {
    1: "2D Poisson Q1, 4x4 subdomains of 16x16 elements, FP64",
    2: "2D heat Q1 lognormal(sigma=1), 32x32 subdomains of 64x64 elements",
    3: "3D elasticity Hex8, 8x8x8 subdomains of 12^3 elements",
    4: "3D heat Hex8 lognormal(sigma=0.5), 120^3 box cut 10x10x10 (8..24 per axis)",
    5: "3D elasticity sensitivity Hex8, 6x6x6 subdomains of 16^3, rho~U[0.1,1], E=rho^3",
}


def make_config(k: int, nsub_axis: Optional[int] = None, seed: int = 0) -> Problem:
    """Workload k (1..5).  nsub_axis overrides the subdomain count per axis
    (same subdomain shape and material law) for smaller copies."""
    if k == 1:
        q = nsub_axis or 4
        return make_problem(dim=2, physics="heat", cuts=[[16] * q] * 2, material="const",
                            seed=seed, name=f"cfg1_poisson2d_{q}x{q}x16")
    if k == 2:
        q = nsub_axis or 32
        return make_problem(dim=2, physics="heat", cuts=[[64] * q] * 2, material="lognormal",
                            sigma=1.0, seed=seed, name=f"cfg2_heat2d_{q}x{q}x64")
    if k == 3:
        q = nsub_axis or 8
        return make_problem(dim=3, physics="elasticity", cuts=[[12] * q] * 3, material="const",
                            seed=seed, name=f"cfg3_elast3d_{q}^3x12")
    if k == 4:
        q = nsub_axis or 10
        total = 12 * q
        rng = np.random.default_rng([seed, 1])
        cuts = [_random_cuts(total, q, 8, 24, rng) for _ in range(3)]
        return make_problem(dim=3, physics="heat", cuts=cuts, material="lognormal", sigma=0.5,
                            seed=seed, name=f"cfg4_heat3d_uneven_{q}^3")
    if k == 5:
        q = nsub_axis or 6
        return make_problem(dim=3, physics="elasticity", cuts=[[16] * q] * 3, material="density",
                            seed=seed, name=f"cfg5_elast3d_sens_{q}^3x16")
    raise ValueError(k)


def subdomain_K_values(problem: Problem, i: int, elem_coef: np.ndarray) -> np.ndarray:
    """CSR values of K_i for per-element coefficients elem_coef (K_e = coef_e K_ref)."""
    s = problem.subs[i]
    _, col, pos, _ = _local_pattern(tuple(s.shape), problem.dpn)
    return np.bincount(pos.ravel(), weights=(np.asarray(elem_coef)[:, None, None] * problem.K_ref[None]).ravel(),
                       minlength=col.shape[0])


def make_W_sub(m: int, seed: int, i: int) -> np.ndarray:
    """Symmetric N(0,1) weight W_i (m x m) of subdomain i: upper triangle incl.
    the diagonal drawn row by row from default_rng([seed, 3, i]) and mirrored
    (one stream per subdomain, so any subset can be drawn on its own)."""
    rng = np.random.default_rng([seed, 3, i])
    iu = np.triu_indices(m)
    W = np.zeros((m, m))
    W[iu] = rng.normal(0.0, 1.0, size=iu[0].shape[0])
    return W + np.triu(W, 1).T


def make_W(problem: Problem, seed: int = 0, only=None) -> List[np.ndarray]:
    """W_i of every subdomain (make_W_sub); with `only` (subdomain indices) the
    others are zero matrices."""
    keep = None if only is None else set(int(i) for i in only)
    return [make_W_sub(s.m, seed, i) if keep is None or i in keep else np.zeros((s.m, s.m))
            for i, s in enumerate(problem.subs)]


def seeded_vector(n: int, seed: int, purpose: int = 7) -> np.ndarray:
    """A seeded N(0,1) test vector (e.g. a dual vector p for F.p parity)."""
    return np.random.default_rng([seed, purpose]).normal(0.0, 1.0, size=n)
