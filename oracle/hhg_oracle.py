"""Plain CPU FP64 oracle: HHG refinement, P1 assembly, FMG (Alg. 4), estimator, marking, 2D and 3D
red-green refinement (Alg. 3), adjoint gradients.

TEST INFRASTRUCTURE ONLY -- imported by tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; never by the product path.

Paper: B. Mann, U. Ruede, "kl-refinement: An adaptive mesh refinement scheme for
hierarchical hybrid grids" (arXiv 2508.06049).

What each part follows
----------------------
* Sec. 2 (HHG construction): every macro element of the coarse mesh T_0 is refined
  uniformly L times, red refinement for triangles, Bey's rule for tetrahedra.
  Here this is done literally, element by element, recursively.  A node is keyed
  by its integer barycentric weights over the macro vertices (weights sum to 2^l),
  which makes nodes on shared macro edges/faces/vertices coincide without any
  structured indexing.
* Sec. 4.4, Eq. (4.15): A_l u_l = b_l, P1 Lagrange elements for the Poisson /
  piecewise-constant-coefficient diffusion problem of Eq. (5.1), assembled
  element by element (stiffness k_T int grad phi_i . grad phi_j, mass int phi_i phi_j).
  b_l = M_l f_l with f_l = f at the level-l nodes; Dirichlet nodes fixed to g.
* Sec. 4.4, Alg. 4 (FMG): for l = 0..L, nu V-cycles on level l, then
  u_{l+1} <- I u_l and w_l <- u_{l+1}.  The V-cycle (pre-smooth, residual,
  restriction = I^T, coarse correction, prolongation, post-smooth) and the
  smoother ordering are not spelled out in the paper; the readings taken are:
    - Gauss-Seidel sweep = ordered stage list: macro vertices; macro-edge
      interior nodes with even, then odd, edge-local index (counted from the
      endpoint with the smaller global id); (3D) macro-face interior nodes by
      colour (a + 2b) mod 3 in face-local coordinates (vertices sorted by global
      id); macro-cell interior nodes by colour (alpha . p) mod m with alpha, m
      chosen per macro from its interior stencil (red-black where the diagonal
      couplings vanish).  Inside one stage all nodes are updated from the values
      at the start of the stage.  The three face colours form one block in which
      every macro face is smoothed on its own: Gauss-Seidel over the face's nodes
      in colour order, with all nodes outside the face (including the nodes of
      other faces next to a shared macro edge) at their values from the start of
      the block.
    - Coarse solve: exact dense Cholesky solve (the limit of the paper's CG).
    - I = linear interpolation on the nested meshes, restriction = I^T.
* Sec. 4.4, Alg. 4 (ErrorEstimate) and Eqs. (4.5), (4.6), (4.14): e~_l = u_L - I w_l,
  theta~_l = ||e~_l|| / ||e~_{l-1}||, eta_j = theta~_l^j ||e~_l|| with l = L-j,
  L2 norms through the mass matrix; local eta_T = ||e~_{L-1}||_{L2(T)} over the
  micro elements inside macro T.  The Remark in Sec. 4: the energy norm (stiffness
  matrix in place of the mass matrix) and a goal-oriented local seminorm
  ||G(v|_T)||, here G(v|_T) = sqrt(w_T) v|_T with per-macro weights w_T.
* Theorem 4.1 / Corollaries 4.3-4.4: effectivity constants.
* Sec. 3 and Sec. 5.1: marking of a top fraction of macro elements; 2D red-green
  refinement with greens reverted before the next step; Alg. 3 (3D red-green: red
  by Bey's rule, the face and tet closure rules, three green types).
* No paper counterpart: gradients of J(u) = u^T M_S u with respect to the nodal source
  and the per-macro coefficients, by an exact adjoint solve (implicit differentiation).

No kernel blocking, fusion or reordering beyond the definitions above.

Pins: every function here is checked against facts that do not come from this file
(closed forms, invariants, brute force, the paper's printed constants, finite
differences, planted mistakes) in tests/test_oracle_pins.py, test_oracle_norms.py,
test_oracle_rg_adjoint.py and test_rg3d.py; none is parity-unpinned.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg
import scipy.sparse as sp

# Sentinel global id used to pad node keys (sorts after every real vertex id).
_PAD = np.int64(1 << 40)


# --------------------------------------------------------------------------------------
# Refinement rules (Sec. 2): children given as index lists into [vertices..., midpoints...]
# --------------------------------------------------------------------------------------

def _red_children_2d():
    # vertices 0,1,2 ; midpoints 3=(0,1) 4=(1,2) 5=(2,0)
    """Red refinement of a triangle (Sec. 2): its three edges and four children, as indices into
    [vertices 0..2, edge midpoints 3..5]."""
    edges = [(0, 1), (1, 2), (2, 0)]
    children = [(0, 3, 5), (3, 1, 4), (5, 4, 2), (4, 5, 3)]
    return edges, children


def _bey_children_3d():
    # vertices 0..3 ; midpoints 4=(0,1) 5=(0,2) 6=(0,3) 7=(1,2) 8=(1,3) 9=(2,3)
    # Bey's rule: four corner tets and the interior octahedron cut along x02-x13.
    """Bey's rule for a tetrahedron (Sec. 2): its six edges and eight children (four corner tets and
    the inner octahedron cut along the x02-x13 diagonal), as indices into [vertices, midpoints]."""
    edges = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    children = [
        (0, 4, 5, 6), (4, 1, 7, 8), (5, 7, 2, 9), (6, 8, 9, 3),
        (4, 5, 6, 8), (4, 5, 7, 8), (5, 6, 8, 9), (5, 7, 8, 9),
    ]
    return edges, children


def _refine_weights(W, dim):
    """One uniform refinement of micro elements given by integer weight vectors (Sec. 2).

    W has shape (nE, d+1, d+1): W[e, a] is the weight vector of vertex a of element e
    over the d+1 vertices of its macro element (weights sum to 2^l).  Returns the
    children's weights (sum 2^(l+1)) and the (vertex, midpoint) bookkeeping needed
    for the interpolation operator.
    """
    edges, children = (_red_children_2d() if dim == 2 else _bey_children_3d())
    nE = W.shape[0]
    pts = [2 * W[:, a, :] for a in range(dim + 1)]
    for (a, b) in edges:
        pts.append(W[:, a, :] + W[:, b, :])
    P = np.stack(pts, axis=1)  # (nE, d+1+n_edges, d+1)
    C = np.stack([P[:, list(ch), :] for ch in children], axis=1)  # (nE, nchild, d+1, d+1)
    return C.reshape(nE * len(children), dim + 1, dim + 1), edges


# --------------------------------------------------------------------------------------
# Node keys
# --------------------------------------------------------------------------------------

def _canonical_keys(wts, macro, cells):
    """Canonical key rows for points with integer weights `wts` (N, d+1) over macro `macro`, so that
    nodes on shared macro primitives coincide (Sec. 2).

    Key = (global vertex id, weight) pairs with nonzero weight, sorted by global id,
    padded with (_PAD, 0).  Shape (N, 2(d+1)) int64.
    """
    gids = cells[macro].astype(np.int64)  # (N, d+1)
    g = np.where(wts > 0, gids, _PAD)
    w = np.where(wts > 0, wts, 0).astype(np.int64)
    order = np.argsort(g, axis=1, kind="stable")
    g = np.take_along_axis(g, order, axis=1)
    w = np.take_along_axis(w, order, axis=1)
    key = np.empty((wts.shape[0], 2 * wts.shape[1]), dtype=np.int64)
    key[:, 0::2] = g
    key[:, 1::2] = w
    return key


# --------------------------------------------------------------------------------------
# Element matrices (P1)
# --------------------------------------------------------------------------------------

def _element_matrices(X):
    """P1 stiffness (unit coefficient) and mass matrices of Eq. 5.1 for simplices X (nE, d+1, d).

    Stiffness K_ab = |E| grad(phi_a) . grad(phi_b); mass M_ab = |E| (1 + delta_ab) / ((d+1)(d+2)).
    """
    nE, dp1, d = X.shape
    J = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))  # columns = edge vectors, (nE, d, d)
    det = np.linalg.det(J)
    vol = np.abs(det) / math.factorial(d)
    Jinv = np.linalg.inv(J)  # rows = gradients of barycentric coords 1..d
    G = np.empty((nE, dp1, d))
    G[:, 1:, :] = Jinv
    G[:, 0, :] = -Jinv.sum(axis=1)
    K = vol[:, None, None] * np.einsum("eak,ebk->eab", G, G)
    Mref = (np.ones((dp1, dp1)) + np.eye(dp1)) / ((d + 1) * (d + 2))
    M = vol[:, None, None] * Mref[None, :, :]
    return K, M, vol


def _assemble(elems, Ke, n):
    """Sparse global matrix summed element by element from element matrices (the assembly of the
    P1 system A_l u_l = b_l, Eq. 4.15)."""
    dp1 = elems.shape[1]
    rows = np.repeat(elems, dp1, axis=1).ravel()
    cols = np.tile(elems, (1, dp1)).ravel()
    return sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(n, n))


# --------------------------------------------------------------------------------------
# Coarse topology
# --------------------------------------------------------------------------------------

def _faces_of(cells, dim):
    """Facets (sorted vertex tuples) of each cell, the macro primitives of Sec. 2: edges in 2D,
    triangles in 3D."""
    from itertools import combinations
    out = []
    for c in cells:
        out.append([tuple(sorted(f)) for f in combinations([int(v) for v in c], dim)])
    return out


@dataclass
class Level:
    """One level T_l of the HHG (Sec. 2): nodes, micro elements, the assembled A_l and M_l (Eq. 4.15),
    Dirichlet flags, the smoother's stages (Alg. 4) and the interpolation P from level l-1 (Sec. 4.4)."""
    l: int
    keys: np.ndarray          # (N, 2(d+1)) canonical node keys
    x: np.ndarray             # (N, d) coordinates
    elems: np.ndarray         # (nE, d+1) node ids
    emacro: np.ndarray        # (nE,) macro id of each micro element
    Ke: np.ndarray            # (nE, d+1, d+1) stiffness element matrices (with k_T)
    Me: np.ndarray            # (nE, d+1, d+1) mass element matrices
    A: sp.csr_matrix = None
    M: sp.csr_matrix = None
    dirichlet: np.ndarray = None
    free: np.ndarray = None
    stages: list = field(default_factory=list)
    stage_rows: list = field(default_factory=list)
    stage_diag: list = field(default_factory=list)
    # 3D face block (stages face_first .. face_first+2): each face stage's rows split into the
    # couplings to nodes of the same macro face (current values) and all others (values frozen
    # at the start of the block)
    face_first: int = -1
    stage_rows_same: list = field(default_factory=list)
    stage_rows_other: list = field(default_factory=list)
    P: sp.csr_matrix = None   # interpolation from level l-1 to l (l >= 1)


class Hierarchy:
    """Nested P1 meshes T_0 ... T_L of an HHG (Sec. 2), assembled explicitly.

    coords (nV, d), cells (nC, d+1) 0-based; dirichlet: per-vertex flags or None (= all
    boundary vertices); k: per-cell coefficient or None (= 1).
    """

    def __init__(self, coords, cells, L, dirichlet=None, k=None):
        coords = np.asarray(coords, dtype=np.float64)
        cells = np.asarray(cells, dtype=np.int64)
        self.dim = d = coords.shape[1]
        if d not in (2, 3) or cells.shape[1] != d + 1:
            raise ValueError("need triangles in 2D or tetrahedra in 3D")
        self.coords, self.cells, self.L = coords, cells, int(L)
        self.n_cells = len(cells)
        self.k = np.ones(self.n_cells) if k is None else np.asarray(k, dtype=np.float64)
        self._topology(dirichlet)
        self.levels = []
        W = np.repeat(np.eye(d + 1, dtype=np.int64)[None], self.n_cells, axis=0)
        macro = np.arange(self.n_cells)
        prev = None
        for l in range(self.L + 1):
            if l > 0:
                Wc, macro_c = W, macro
                W, edges = _refine_weights(W, d)
                nchild = W.shape[0] // Wc.shape[0]
                macro = np.repeat(macro_c, nchild)
            lev = self._build_level(l, W, macro)
            if l > 0:
                lev.P = self._interpolation(lev, prev, Wc, macro_c, edges)
            self.levels.append(lev)
            prev = lev
        self._colouring()
        for lev in self.levels:
            self._stages(lev)

    # ---- topology and boundary (Sec. 2: macro primitives) ----
    def _topology(self, dirichlet):
        """Boundary macro primitives of T_0 (Sec. 2: vertices, edges, faces) and the Dirichlet flag of
        each macro vertex (every boundary vertex unless flags are given)."""
        d = self.dim
        facets = _faces_of(self.cells, d)
        count = {}
        for fl in facets:
            for f in fl:
                count[f] = count.get(f, 0) + 1
        self.boundary_facets = {f for f, c in count.items() if c == 1}
        bverts = set()
        bedges = set()
        for f in self.boundary_facets:
            bverts.update(f)
            if d == 2:
                bedges.add(f)
            else:
                bedges.update({(f[0], f[1]), (f[0], f[2]), (f[1], f[2])})
        self.boundary_edges = bedges
        if dirichlet is None:
            vflag = np.zeros(len(self.coords), dtype=bool)
            vflag[list(bverts)] = True
        else:
            vflag = np.asarray(dirichlet).astype(bool).copy()
        self.vflag = vflag
        self.cell_of_vertex_set = {tuple(sorted(int(v) for v in c)): t for t, c in enumerate(self.cells)}

    def _node_dirichlet(self, keys):
        """A node is a Dirichlet node when it lies on a boundary macro primitive whose vertices are all
        Dirichlet (the boundary of the HHG primitives, Sec. 2)."""
        d = self.dim
        g = keys[:, 0::2]
        s = (g != _PAD).sum(axis=1)
        out = np.zeros(len(keys), dtype=bool)
        for i in np.nonzero(s <= d)[0]:
            sup = tuple(int(v) for v in g[i, : s[i]])
            if len(sup) == 1:
                out[i] = self.vflag[sup[0]]
            elif len(sup) == 2:
                out[i] = sup in self.boundary_edges and all(self.vflag[v] for v in sup)
            else:  # face interior (3D only: s <= d)
                out[i] = sup in self.boundary_facets and all(self.vflag[v] for v in sup)
        return out

    def _build_level(self, l, W, macro):
        """Level l (Sec. 2): nodes de-duplicated through their canonical keys, coordinates, element
        matrices with k_T (Eq. 5.1) and the assembled A_l, M_l of Eq. 4.15."""
        d = self.dim
        nE = W.shape[0]
        flat_w = W.reshape(nE * (d + 1), d + 1)
        flat_m = np.repeat(macro, d + 1)
        keys_all = _canonical_keys(flat_w, flat_m, self.cells)
        keys, inv = _unique_rows(keys_all)
        elems = inv.reshape(nE, d + 1)
        # coordinates from the canonical key: sum_a w_a X_{g_a} / 2^l
        g = keys[:, 0::2]
        w = keys[:, 1::2].astype(np.float64)
        gsafe = np.where(g == _PAD, 0, g)
        x = np.einsum("na,nak->nk", w, self.coords[gsafe]) / float(2 ** l)
        X = x[elems]
        K, Mm, _ = _element_matrices(X)
        K = K * self.k[macro][:, None, None]
        lev = Level(l=l, keys=keys, x=x, elems=elems, emacro=macro, Ke=K, Me=Mm)
        n = len(keys)
        lev.A = _assemble(elems, K, n)
        lev.M = _assemble(elems, Mm, n)
        lev.dirichlet = self._node_dirichlet(keys)
        lev.free = ~lev.dirichlet
        return lev

    def _interpolation(self, fine, coarse, Wc, macro_c, edges):
        """Linear interpolation I_{l-1}^{l}: old nodes copied, edge midpoints averaged (Sec. 4.4)."""
        d = self.dim
        nEc = Wc.shape[0]
        rows, cols, vals = [], [], []
        # coarse node ids of coarse element vertices
        cvert = coarse.elems  # (nEc, d+1)
        # fine keys of doubled coarse vertices
        kv = _canonical_keys((2 * Wc).reshape(-1, d + 1), np.repeat(macro_c, d + 1), self.cells)
        fid_v = _lookup(fine.keys, kv)
        rows.append(fid_v)
        cols.append(cvert.ravel())
        vals.append(np.ones(len(fid_v)))
        for (a, b) in edges:
            km = _canonical_keys(Wc[:, a, :] + Wc[:, b, :], macro_c, self.cells)
            fid = _lookup(fine.keys, km)
            for c in (a, b):
                rows.append(fid)
                cols.append(cvert[:, c])
                vals.append(np.full(nEc, 0.5))
        rows = np.concatenate(rows)
        cols = np.concatenate(cols)
        vals = np.concatenate(vals)
        # each (fine, coarse) pair is defined once, even if several coarse elements share it
        pair, _ = _unique_rows(np.stack([rows, cols, (vals * 2).astype(np.int64)], axis=1))
        P = sp.csr_matrix((pair[:, 2] / 2.0, (pair[:, 0], pair[:, 1])),
                          shape=(len(fine.keys), len(coarse.keys)))
        return P

    # ---- smoother stage ordering (reading of "Gauss-Seidel", Sec. 5) ----
    def _colouring(self):
        """Per macro (alpha_T, m_T) for the macro-cell interior colours (smoother reading of Alg. 4).

        Decided from the interior couplings of macro T on level 2 (the interior stencil is
        the same on every level): m=2 with the first alpha in a fixed candidate list for
        which alpha . d is odd for every lattice direction d with a nonzero coupling;
        otherwise m=3, alpha=(1,2) in 2D and m=4, alpha=(1,2,3) in 3D.
        """
        d = self.dim
        self.alpha = np.zeros((self.n_cells, d), dtype=np.int64)
        self.mcol = np.zeros(self.n_cells, dtype=np.int64)
        cands = ([(1, 1), (1, 0), (0, 1)] if d == 2 else
                 [(1, 1, 1), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1)])
        fallback = ((1, 2), 3) if d == 2 else ((1, 2, 3), 4)
        if self.L < 2:
            for t in range(self.n_cells):
                self.alpha[t], self.mcol[t] = fallback
            return
        lev = self.levels[2]
        loc = self._local_coords(lev.keys)  # (N, macro, p) for interior nodes
        A = lev.A
        done = np.zeros(self.n_cells, dtype=bool)
        for i in np.nonzero(loc[0] >= 0)[0]:
            t = loc[0][i]
            if done[t]:
                continue
            done[t] = True
            row = A.getrow(i)
            offs = [(j, v) for j, v in zip(row.indices, row.data) if j != i]
            vmax = max(abs(v) for _, v in offs)
            dirs = []
            for j, v in offs:
                if abs(v) > 1e-12 * vmax:
                    dirs.append(self._local_p(lev.keys[j], t) - loc[1][i])
            chosen = None
            for a in cands:
                if all((int(np.dot(a, dd)) % 2) != 0 for dd in dirs):
                    chosen = (a, 2)
                    break
            if chosen is None:
                chosen = fallback
            self.alpha[t], self.mcol[t] = chosen

    def _local_p(self, key, t):
        """Lattice coordinates (Sec. 2) of a node, given by key, in macro t: its weights on
        cells[t][1..d]."""
        g = key[0::2]
        w = key[1::2]
        p = np.zeros(self.dim, dtype=np.int64)
        for a in range(1, self.dim + 1):
            hit = np.nonzero(g == self.cells[t][a])[0]
            p[a - 1] = w[hit[0]] if len(hit) else 0
        return p

    def _local_coords(self, keys):
        """For macro-cell interior nodes: (macro id, lattice coordinates of Sec. 2); -1 elsewhere."""
        d = self.dim
        g = keys[:, 0::2]
        w = keys[:, 1::2]
        s = (g != _PAD).sum(axis=1)
        macro = np.full(len(keys), -1, dtype=np.int64)
        p = np.zeros((len(keys), d), dtype=np.int64)
        inner = np.nonzero(s == d + 1)[0]
        if len(inner) == 0:
            return macro, p
        sets, inv = _unique_rows(g[inner])
        tmap = np.array([self.cell_of_vertex_set[tuple(int(v) for v in row)] for row in sets])
        t = tmap[inv]
        macro[inner] = t
        for a in range(1, d + 1):
            target = self.cells[t, a][:, None]
            p[inner, a - 1] = (w[inner] * (g[inner] == target)).sum(axis=1)
        return macro, p

    def _stages(self, lev):
        """The ordered stage list of one Gauss-Seidel sweep on this level (the smoother of Alg. 4, in the
        reading stated in the module docstring), with each stage's rows and diagonal."""
        d = self.dim
        keys = lev.keys
        g = keys[:, 0::2]
        w = keys[:, 1::2]
        s = (g != _PAD).sum(axis=1)
        free = lev.free
        stage_of = np.full(len(keys), -1, dtype=np.int64)
        # stage ids: 0 vertex, 1/2 edge even/odd, then faces (3D: 3 colours), then cells
        stage_of[(s == 1)] = 0
        e = s == 2
        stage_of[e] = 1 + (w[e, 1] % 2)  # weight on the larger-id endpoint
        base = 3
        if d == 3:
            f = s == 3
            stage_of[f] = base + (w[f, 1] + 2 * w[f, 2]) % 3
            base += 3
        macro, p = self._local_coords(keys)
        c = macro >= 0
        if c.any():
            col = (np.einsum("nk,nk->n", p[c], self.alpha[macro[c]])) % self.mcol[macro[c]]
            stage_of[c] = base + col
        n_stages = base + int(self.mcol.max())
        # macro face of each face-interior node (its three vertex ids), -1 elsewhere
        face_of = np.full(len(keys), -1, dtype=np.int64)
        if d == 3:
            f = s == 3
            if f.any():
                _, fid = np.unique(np.sort(g[f][:, :3], axis=1), axis=0, return_inverse=True)
                face_of[f] = fid.ravel()
            lev.face_first = 3
        lev.stages = []
        diag = lev.A.diagonal()
        for st in range(n_stages):
            idx = np.nonzero((stage_of == st) & free)[0]
            lev.stages.append(idx)
            rows = lev.A[idx]
            lev.stage_rows.append(rows)
            lev.stage_diag.append(diag[idx])
            if d == 3 and 3 <= st < 6:
                coo = rows.tocoo()
                same = face_of[coo.col] == face_of[idx[coo.row]]
                shape = rows.shape
                lev.stage_rows_same.append(sp.csr_matrix((coo.data[same], (coo.row[same], coo.col[same])), shape=shape))
                lev.stage_rows_other.append(
                    sp.csr_matrix((coo.data[~same], (coo.row[~same], coo.col[~same])), shape=shape))


def _row_hash(keys):
    """64-bit hash of each key row for the node de-duplication of Sec. 2 (collisions are checked by
    the callers)."""
    h = np.full(len(keys), np.uint64(1469598103934665603))
    with np.errstate(over="ignore"):
        for c in range(keys.shape[1]):
            h = (h ^ keys[:, c].astype(np.uint64)) * np.uint64(1099511628211)
            h ^= h >> np.uint64(29)
    return h


def _unique_rows(keys):
    """Unique key rows (ordered by hash) and the inverse map, for the node de-duplication of Sec. 2;
    exact (hash collisions rejected)."""
    h = _row_hash(keys)
    uh, first, inv = np.unique(h, return_index=True, return_inverse=True)
    uniq = keys[first]
    if not np.array_equal(uniq[inv], keys):
        raise AssertionError("node-key hash collision")
    return uniq, inv.ravel()


def _lookup(keys_unique, q):
    """Row indices of the rows of q inside `keys_unique` (as produced by _unique_rows; node
    de-duplication, Sec. 2)."""
    hk = _row_hash(keys_unique)
    order = np.argsort(hk)
    pos = np.searchsorted(hk[order], _row_hash(q))
    pos = np.minimum(pos, len(order) - 1)
    idx = order[pos]
    if not np.array_equal(keys_unique[idx], q):
        raise AssertionError("query keys not all present on the level")
    return idx


# --------------------------------------------------------------------------------------
# Level data: right-hand sides and Dirichlet values (Sec. 4.4, Eq. (4.15); Eq. (5.1))
# --------------------------------------------------------------------------------------

def inject_from_finest(h: Hierarchy, vL: np.ndarray, l: int) -> np.ndarray:
    """Values at level-l nodes taken from a level-L nodal vector (the nodes are nested, Sec. 2:
    key * 2^(L-l))."""
    if l == h.L:
        return np.asarray(vL, dtype=np.float64).copy()
    keys = h.levels[l].keys.copy()
    keys[:, 1::2] *= 2 ** (h.L - l)
    return np.asarray(vL)[_lookup(h.levels[h.L].keys, keys)]


def nodal(h: Hierarchy, fn, l: int) -> np.ndarray:
    """A nodal vector on level l (f_l or g_l of Sec. 4.4) from a callable of x (N, d) or a level-L
    nodal array."""
    if callable(fn):
        return np.asarray(fn(h.levels[l].x), dtype=np.float64)
    return inject_from_finest(h, fn, l)


class Problem:
    """The right-hand sides b_l of Eq. 4.15 (Sec. 4.4) and Dirichlet values g_l for every level of a
    hierarchy.  The paper does not say how the coarse levels' right-hand sides are formed; two
    readings are offered:
      rhs="injected" (default): b_l = M_l f_l with f_l the values of f at the level-l nodes;
      rhs="restricted": b_L = M_L f_L and b_l = I_l^T b_{l+1} for l < L (I = the interpolation of
        Sec. 4.4), i.e. the load vector of the level-L interpolant of f tested with the level-l hat
        functions (each of which is a combination of level-L hat functions)."""

    def __init__(self, h: Hierarchy, f, g, rhs: str = "injected"):
        self.h = h
        if rhs == "injected":
            self.b = [lev.M @ nodal(h, f, lev.l) for lev in h.levels]
        elif rhs == "restricted":
            b = [None] * (h.L + 1)
            b[h.L] = h.levels[h.L].M @ nodal(h, f, h.L)
            for l in range(h.L, 0, -1):
                b[l - 1] = h.levels[l].P.T @ b[l]
            self.b = b
        else:
            raise ValueError("rhs must be 'injected' or 'restricted'")
        self.g = [nodal(h, g, lev.l) for lev in h.levels]
        lev0 = h.levels[0]
        F = np.nonzero(lev0.free)[0]
        self.coarse_free = F
        A0 = lev0.A[F][:, F].toarray()
        self.coarse_factor = scipy.linalg.cho_factor(A0, lower=True) if len(F) else None


# --------------------------------------------------------------------------------------
# Smoother, V-cycle, FMG (Alg. 4)
# --------------------------------------------------------------------------------------

def smooth(lev: Level, u: np.ndarray, rhs: np.ndarray) -> None:
    """One Gauss-Seidel sweep of Alg. 4 as the ordered stage list; Jacobi inside a stage (in place).

    3D face block: the three face colours update each macro face's nodes by Gauss-Seidel over the
    face (its own nodes at their current values), with every node outside the face taken at its
    value from the start of the block (the faces are independent of each other inside the block)."""
    u0 = None
    for s in range(len(lev.stages)):
        idx = lev.stages[s]
        if lev.face_first >= 0 and s == lev.face_first:
            u0 = u.copy()
        if len(idx) == 0:
            continue
        if lev.face_first >= 0 and lev.face_first <= s < lev.face_first + 3:
            q = s - lev.face_first
            r = rhs[idx] - lev.stage_rows_same[q] @ u - lev.stage_rows_other[q] @ u0
        else:
            r = rhs[idx] - lev.stage_rows[s] @ u
        u[idx] += r / lev.stage_diag[s]


def residual(lev: Level, u: np.ndarray, rhs: np.ndarray) -> np.ndarray:
    """r = rhs - A u on free nodes, zero on Dirichlet nodes (V-cycle of Alg. 4)."""
    r = rhs - lev.A @ u
    r[lev.dirichlet] = 0.0
    return r


def coarse_solve(prob: Problem, u: np.ndarray, rhs: np.ndarray) -> None:
    """u <- u + A_ff^{-1} (rhs - A u)_f on level 0 (Alg. 4): exact, the converged limit of the CG that
    Sec. 5.4 runs."""
    lev0 = prob.h.levels[0]
    F = prob.coarse_free
    if len(F) == 0:
        return
    r = (rhs - lev0.A @ u)[F]
    u[F] += scipy.linalg.cho_solve(prob.coarse_factor, r)


def vcycle(prob: Problem, l: int, u: np.ndarray, rhs: np.ndarray, pre: int = 2, post: int = 1) -> None:
    """One V(pre, post)-cycle on level l for A_l u = rhs (in place) (Alg. 4)."""
    h = prob.h
    if l == 0:
        coarse_solve(prob, u, rhs)
        return
    lev = h.levels[l]
    for _ in range(pre):
        smooth(lev, u, rhs)
    r = residual(lev, u, rhs)
    rc = lev.P.T @ r                      # restriction = transpose of interpolation
    uc = np.zeros(len(h.levels[l - 1].keys))
    vcycle(prob, l - 1, uc, rc, pre, post)
    corr = lev.P @ uc
    u[lev.free] += corr[lev.free]
    for _ in range(post):
        smooth(lev, u, rhs)


def fmg(prob: Problem, nu: int = 2, pre: int = 2, post: int = 1, n_extra: int = 0):
    """Alg. 4 FMG: returns (u_L, [w_0 .. w_{L-1}], [u_0 .. u_L] after their V-cycles).

    w_l is the prolongated level-l solution stored on level l+1 (before the level-(l+1)
    V-cycles).  n_extra additional V-cycles on level L do not update w (Sec. 5).
    """
    h = prob.h
    L = h.L
    u = np.where(h.levels[0].dirichlet, prob.g[0], 0.0)
    ws, us = [], []
    for l in range(L + 1):
        for _ in range(nu):
            vcycle(prob, l, u, prob.b[l], pre, post)
        us.append(u.copy())
        if l < L:
            fine = h.levels[l + 1]
            u = fine.P @ u
            u[fine.dirichlet] = prob.g[l + 1][fine.dirichlet]
            ws.append(u.copy())
    for _ in range(n_extra):
        vcycle(prob, L, u, prob.b[L], pre, post)
    return u, ws, us


# --------------------------------------------------------------------------------------
# Error estimator (Alg. 4 ErrorEstimate; Eqs. (4.5), (4.6), (4.10), (4.14))
# --------------------------------------------------------------------------------------

def local_mass_sq(lev: Level, e: np.ndarray, n_cells: int) -> np.ndarray:
    """Per macro T: e^T M_{l,T} e, summing the element mass forms of the micro elements inside T (the
    local indicator of Eq. 4.14)."""
    ee = e[lev.elems]
    per_elem = np.einsum("ea,eab,eb->e", ee, lev.Me, ee)
    return np.bincount(lev.emacro, weights=per_elem, minlength=n_cells)


def local_energy_sq(lev: Level, e: np.ndarray, n_cells: int) -> np.ndarray:
    """Per macro T: e^T A_{l,T} e = int_T k |grad e|^2, summing the element stiffness forms (with
    k_T) of micro elements inside T, boundary nodes included (the energy norm of the Remark in
    Sec. 4)."""
    ee = e[lev.elems]
    per_elem = np.einsum("ea,eab,eb->e", ee, lev.Ke, ee)
    return np.bincount(lev.emacro, weights=per_elem, minlength=n_cells)


def prolong_to_finest(h: Hierarchy, v: np.ndarray, l: int) -> np.ndarray:
    """I_l^L v for a level-l nodal vector (interpolation, Sec. 4.4)."""
    for m in range(l + 1, h.L + 1):
        v = h.levels[m].P @ v
    return v


def estimate(h: Hierarchy, u_L: np.ndarray, ws, j: int = 1, norm: str = "l2", weights=None):
    """Alg. 4 ErrorEstimate with offset j (l = L - j), plus the local indicators.

    norm (Remark in Sec. 4): "l2" (the paper's choice, mass matrix), "energy" (the stiffness
    matrix in place of the mass matrix: int_T k |grad v|^2), or "goal": the local seminorm
    ||v||_T^2 = w_T ||v||_{L2(T)}^2 of the piecewise constant goal operator G(v|_T) = sqrt(w_T) v|_T
    with per-macro weights w_T >= 0 (e.g. the indicator of a subregion made of macro cells); the
    global values are the sums of the weighted local squares.

    Returns a dict with
      err_l, err_lm1  : ||e~_l||, ||e~_{l-1}|| (L2 via the mass matrix)
      theta           : theta~_l = ||e~_l|| / ||e~_{l-1}||          (Eq. 4.5b)
      eta_j           : theta~_l^j ||e~_l||                          (Eq. 4.6)
      eta_T           : ||e~_{L-1}||_{L2(T)} per macro (eta'_{1,T}, Eq. 4.14, Sec. 4.4)
      eta_jT          : theta~_{l,T}^j ||e~_l||_T per macro          (Eq. 4.10)
      sq_l_T, sq_lm1_T: per-macro squared local norms of e~_l and e~_{l-1}
    """
    L = h.L
    l = L - j
    if not (1 <= l <= L - 1):
        raise ValueError("need 1 <= j <= L-1")
    levL = h.levels[L]
    e_l = u_L - prolong_to_finest(h, ws[l], l + 1)          # w_l lives on level l+1
    e_lm1 = u_L - prolong_to_finest(h, ws[l - 1], l)         # w_{l-1} lives on level l
    if norm not in ("l2", "energy", "goal"):
        raise ValueError("norm must be l2, energy or goal")
    form = local_energy_sq if norm == "energy" else local_mass_sq
    wT = np.ones(h.n_cells) if norm != "goal" else np.asarray(weights, dtype=np.float64)
    # clamped at 0: the energy form is only semidefinite (constants are in the kernel of A_T)
    sq_l = np.maximum(wT * form(levL, e_l, h.n_cells), 0.0)
    sq_lm1 = np.maximum(wT * form(levL, e_lm1, h.n_cells), 0.0)
    e_L1 = u_L - ws[L - 1]
    sq_T = np.maximum(wT * form(levL, e_L1, h.n_cells), 0.0)
    err_l = math.sqrt(sq_l.sum())
    err_lm1 = math.sqrt(sq_lm1.sum())
    theta = err_l / err_lm1 if err_lm1 > 0 else 0.0
    with np.errstate(divide="ignore", invalid="ignore"):
        theta_T = np.where(sq_lm1 > 0, np.sqrt(sq_l / sq_lm1), 0.0)
    return dict(err_l=err_l, err_lm1=err_lm1, theta=theta, eta_j=theta ** j * err_l,
                eta_T=np.sqrt(sq_T), eta_jT=theta_T ** j * np.sqrt(sq_l),
                sq_l_T=sq_l, sq_lm1_T=sq_lm1, sq_T=sq_T)


def l2_error_sq(h: Hierarchy, u_L: np.ndarray, u_exact) -> float:
    """||I u - u_L||_M^2 on level L with the nodal interpolant of the exact solution (the error
    measure of Sec. 5)."""
    lev = h.levels[h.L]
    e = u_exact(lev.x) - u_L
    return float(e @ (lev.M @ e))


# --------------------------------------------------------------------------------------
# Theorem 4.1 and Corollaries 4.3 / 4.4 (effectivity constants)
# --------------------------------------------------------------------------------------

def theorem41_constants(theta: float, j: int, eps: float = 0.0):
    """(C1, C2) of Theorem 4.1 with theta_eps = (1+eps) theta."""
    te = (1.0 + eps) * theta
    c1 = (1.0 + eps) ** (-j) * (1.0 - te ** j) ** (j + 1) / (1.0 + te ** (j + 1)) ** j
    c2 = (1.0 + eps) ** j * (1.0 + te ** j) ** (j + 1) / (1.0 - te ** (j + 1)) ** j
    return c1, c2


def corollary_dgamma_bounds(theta_min: float, theta_max: float, j: int, eps: float = 0.0):
    """Upper bounds on the local effectivity spread for eta_{j,T} (Cor. 4.3) and eta'_{j,T} (Cor. 4.4).

    theta_max is the already (1+eps)-inflated worst local factor, as in the paper.
    """
    tx = theta_max
    scaled = ((1.0 + eps) ** (2 * j) * ((1.0 + tx ** (j + 1)) / (1.0 - tx ** (j + 1))) ** j
              * ((1.0 + tx ** j) / (1.0 - tx ** j)) ** (j + 1))
    unscaled = (theta_min ** (-j) + 1.0) / (tx ** (-j) - 1.0)
    return scaled, unscaled


# --------------------------------------------------------------------------------------
# Marking (Sec. 5.1: mark a fixed fraction of the macro elements with the largest indicator)
# --------------------------------------------------------------------------------------

def mark_top_fraction(eta: np.ndarray, fraction: float) -> np.ndarray:
    """Marking of Sec. 5.1 as a boolean mask: n = max(1, ceil(fraction * N - 1e-9)); eta* = n-th
    largest value (ties ordered by index); mark every T with eta_T >= (1 - 1e-8) eta*."""
    eta = np.asarray(eta, dtype=np.float64)
    N = len(eta)
    if N == 0:
        return np.zeros(0, dtype=bool)
    n = max(1, int(math.ceil(fraction * N - 1e-9)))
    n = min(n, N)
    order = sorted(range(N), key=lambda i: (-eta[i], i))
    star = eta[order[n - 1]]
    return eta >= (1.0 - 1e-8) * star


# --------------------------------------------------------------------------------------
# 2D red-green refinement of the macro mesh (Sec. 3), greens reverted before each step
# --------------------------------------------------------------------------------------

class RG2D:
    """Red-green refinement of a triangle mesh, written out from Sec. 3's description.

    red   : split a triangle (v0,v1,v2) into 4 through its edge midpoints m01, m12, m20;
            children (v0,m01,m20), (m01,v1,m12), (m20,m12,v2), (m12,m20,m01).
    green : bisect a triangle with exactly one split edge from the opposite vertex a:
            with (a,b,c) the rotation of (v0,v1,v2) that starts at a, children (a,b,m), (a,m,c).
    One step (marked = flags on the current conforming mesh):
      1. revert every green pair to its parent; a marked green child marks the parent;
      2. red-refine the marked triangles, then repeat: red-refine every triangle that has
         two or more split edges, or a split edge whose half is split again, until none;
      3. green-bisect every triangle with exactly one split edge.
    An edge (a,b) is split when its midpoint vertex exists.  New midpoints are numbered in
    creation order: triangles in list order, edges (v0v1, v1v2, v2v0).  Refined triangles
    are replaced in place by their children, so the cell order is deterministic.
    """

    def __init__(self, coords, cells):
        self.coords = [tuple(float(c) for c in p) for p in np.asarray(coords, dtype=np.float64)]
        # entries: (v0, v1, v2, green_parent or None, child index)
        self.tris = [(int(a), int(b), int(c), None, -1) for a, b, c in np.asarray(cells)]
        self.mid = {}

    def mesh(self):
        """The current conforming mesh (coords, cells) of the red-green refinement (Sec. 3)."""
        return (np.array(self.coords, dtype=np.float64),
                np.array([t[:3] for t in self.tris], dtype=np.int32).reshape(-1, 3))

    def _midpoint(self, a, b, create):
        """Midpoint vertex of edge (a, b), created on request in creation order (Sec. 3)."""
        key = (min(a, b), max(a, b))
        m = self.mid.get(key)
        if m is None and create:
            pa, pb = self.coords[a], self.coords[b]
            self.coords.append(((pa[0] + pb[0]) * 0.5, (pa[1] + pb[1]) * 0.5))
            m = len(self.coords) - 1
            self.mid[key] = m
        return m

    def _red(self, t):
        """Red refinement of one triangle into four through its edge midpoints (Sec. 3)."""
        v0, v1, v2 = t
        m01 = self._midpoint(v0, v1, True)
        m12 = self._midpoint(v1, v2, True)
        m20 = self._midpoint(v2, v0, True)
        return [(v0, m01, m20), (m01, v1, m12), (m20, m12, v2), (m12, m20, m01)]

    def _split_info(self, t):
        """Split edges of a triangle and whether a split edge's half is split again (the closure
        condition of step 2, Sec. 3)."""
        v = t
        split = []
        over = False
        for e in range(3):
            a, b = v[e], v[(e + 1) % 3]
            m = self._midpoint(a, b, False)
            if m is not None:
                split.append(e)
                if self._midpoint(a, m, False) is not None or self._midpoint(m, b, False) is not None:
                    over = True
        return split, over

    def refine(self, marked):
        """One red-green step on the current mesh (Sec. 3): steps 1-3 of the class docstring."""
        marked = np.asarray(marked).astype(bool)
        if len(marked) != len(self.tris):
            raise ValueError("one flag per current cell")
        # 1. revert greens
        R, flags = [], []
        i = 0
        while i < len(self.tris):
            v0, v1, v2, parent, ci = self.tris[i]
            if parent is not None:
                nxt = self.tris[i + 1]
                if ci != 0 or nxt[3] != parent or nxt[4] != 1:
                    raise AssertionError("green pair not adjacent")
                R.append(parent)
                flags.append(bool(marked[i] or marked[i + 1]))
                i += 2
            else:
                R.append((v0, v1, v2))
                flags.append(bool(marked[i]))
                i += 1
        # 2. red refinement and closure
        while any(flags):
            newR = []
            for t, fl in zip(R, flags):
                newR.extend(self._red(t) if fl else [t])
            R = newR
            flags = []
            for t in R:
                split, over = self._split_info(t)
                flags.append(len(split) >= 2 or over)
        # 3. green closure
        out = []
        for t in R:
            split, _ = self._split_info(t)
            if len(split) == 1:
                e = split[0]
                a = t[(e + 2) % 3]
                b = t[e]
                c = t[(e + 1) % 3]
                m = self._midpoint(b, c, False)
                out.append((a, b, m, t, 0))
                out.append((a, m, c, t, 1))
            else:
                out.append((t[0], t[1], t[2], None, -1))
        self.tris = out


_TET_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
_TET_FACES = ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3))


class RG3D:
    """Red-green refinement of a tetrahedral mesh following Alg. 3 (Sec. 3).

    A tet is stored by its four vertex ids (its slots 0..3); an edge (a,b) is split when its
    midpoint vertex exists.  One step (marked = flags on the current conforming mesh):
      1. revert every green family to its parent; a marked green child marks the parent;
      2. repeat: red-refine the flagged tets (Bey's eight children, x_ab = midpoint of slots a, b:
         (x0,x01,x02,x03), (x01,x1,x12,x13), (x02,x12,x2,x23), (x03,x13,x23,x3), (x01,x02,x03,x13),
         (x02,x01,x12,x13), (x02,x03,x13,x23), (x12,x02,x13,x23) -- the sixth and eighth with two
         slots swapped so that every child keeps the parent's orientation); then split the third
         edge of every face with exactly two split edges, until no such face is left; flag the
         tets with more than three split edges, or a split edge whose half is split again, or a
         fully split face one of whose midlines is split -- until nothing is flagged;
      3. green closure of every tet with one to three split edges (after step 2 these are one
         edge, two opposite edges, or the three edges of one face):
           one edge (slots i<j, midpoint m): T with slot j := m, T with slot i := m;
           two opposite edges: the one-edge rule on the first (in edge order
             01,02,03,12,13,23), then on the second inside each half (four children);
           one face (slots a<b<c, midpoints m_ab, m_bc, m_ca): T with (b, c) := (m_ab, m_ca),
             T with (a, c) := (m_ab, m_bc), T with (a, b) := (m_ca, m_bc), and T with
             (a, b, c) := (m_bc, m_ca, m_ab) (four children; all keep the orientation).
    New vertices are numbered in creation order: tets in list order, edges in the order above,
    faces in the order 012, 013, 023, 123.  Refined tets are replaced in place by their children.
    """

    def __init__(self, coords, cells):
        self.coords = [tuple(float(c) for c in p) for p in np.asarray(coords, dtype=np.float64)]
        # entries: (vertex 4-tuple, green parent 4-tuple or None, child index, children in family)
        self.tets = [(tuple(int(v) for v in c), None, -1, 0) for c in np.asarray(cells)]
        self.mid = {}

    def mesh(self):
        """The current conforming mesh (coords, cells) of the 3D red-green refinement (Alg. 3)."""
        return (np.array(self.coords, dtype=np.float64),
                np.array([t[0] for t in self.tets], dtype=np.int32).reshape(-1, 4))

    def _midpoint(self, a, b, create):
        """Midpoint vertex of edge (a, b), created on request in creation order (Alg. 3)."""
        key = (min(a, b), max(a, b))
        m = self.mid.get(key)
        if m is None and create:
            pa, pb = self.coords[a], self.coords[b]
            self.coords.append(((pa[0] + pb[0]) * 0.5, (pa[1] + pb[1]) * 0.5, (pa[2] + pb[2]) * 0.5))
            m = len(self.coords) - 1
            self.mid[key] = m
        return m

    def _red(self, t):
        """Red refinement of one tet by Bey's rule with orientation-keeping children (Alg. 3, Sec. 2)."""
        x = {}
        for a, b in _TET_EDGES:
            x[(a, b)] = self._midpoint(t[a], t[b], True)
        x0, x1, x2, x3 = t
        x01, x02, x03, x12, x13, x23 = (x[e] for e in _TET_EDGES)
        return [(x0, x01, x02, x03), (x01, x1, x12, x13), (x02, x12, x2, x23), (x03, x13, x23, x3),
                (x01, x02, x03, x13), (x02, x01, x12, x13), (x02, x03, x13, x23), (x12, x02, x13, x23)]

    def _split_edges(self, t):
        """Indices (edge order 01, 02, 03, 12, 13, 23) of a tet's split edges (Alg. 3)."""
        return [e for e, (a, b) in enumerate(_TET_EDGES) if self._midpoint(t[a], t[b], False) is not None]

    def _over(self, t):
        """True when a split edge's half is split again, or a fully split face has a split midline
        (the red conditions of Alg. 3 beyond the count of split edges)."""
        for a, b in _TET_EDGES:
            m = self._midpoint(t[a], t[b], False)
            if m is not None and (self._midpoint(t[a], m, False) is not None or
                                  self._midpoint(m, t[b], False) is not None):
                return True
        for f in _TET_FACES:
            ms = [self._midpoint(t[f[0]], t[f[1]], False), self._midpoint(t[f[1]], t[f[2]], False),
                  self._midpoint(t[f[2]], t[f[0]], False)]
            if all(m is not None for m in ms):
                for i in range(3):
                    if self._midpoint(ms[i], ms[(i + 1) % 3], False) is not None:
                        return True
        return False

    def _close_faces(self, tets):
        """Split the third edge of every face with exactly two split edges until none is left (the face
        rule of Alg. 3)."""
        changed = True
        while changed:
            changed = False
            for t in tets:
                for f in _TET_FACES:
                    edges = [(t[f[0]], t[f[1]]), (t[f[1]], t[f[2]]), (t[f[0]], t[f[2]])]
                    have = [self._midpoint(a, b, False) is not None for a, b in edges]
                    if sum(have) == 2:
                        a, b = edges[have.index(False)]
                        self._midpoint(a, b, True)
                        changed = True

    def _green(self, t, split):
        """Children of a tet with one split edge, two opposite split edges, or the three split edges of
        one face (the three green types of Alg. 3), by slot substitution."""
        def sub(tt, slot, v):
            tt = list(tt)
            tt[slot] = v
            return tuple(tt)
        if len(split) == 1:
            i, j = _TET_EDGES[split[0]]
            m = self._midpoint(t[i], t[j], False)
            return [sub(t, j, m), sub(t, i, m)]
        if len(split) == 2:
            (i, j), (k, l) = _TET_EDGES[split[0]], _TET_EDGES[split[1]]
            m1 = self._midpoint(t[i], t[j], False)
            m2 = self._midpoint(t[k], t[l], False)
            out = []
            for half in (sub(t, j, m1), sub(t, i, m1)):
                out.extend([sub(half, l, m2), sub(half, k, m2)])
            return out
        # three edges of one face
        for f in _TET_FACES:
            fe = {_TET_EDGES.index((f[0], f[1])), _TET_EDGES.index((f[1], f[2])), _TET_EDGES.index((f[0], f[2]))}
            if fe == set(split):
                a, b, c = f
                mab = self._midpoint(t[a], t[b], False)
                mbc = self._midpoint(t[b], t[c], False)
                mca = self._midpoint(t[c], t[a], False)
                return [sub(sub(t, b, mab), c, mca), sub(sub(t, a, mab), c, mbc), sub(sub(t, a, mca), b, mbc),
                        sub(sub(sub(t, a, mbc), b, mca), c, mab)]
        raise AssertionError("split pattern is not a green type")

    def refine(self, marked):
        """One red-green step on the current mesh (Alg. 3): steps 1-3 of the class docstring."""
        marked = np.asarray(marked).astype(bool)
        if len(marked) != len(self.tets):
            raise ValueError("one flag per current cell")
        # 1. revert greens
        R, flags = [], []
        i = 0
        while i < len(self.tets):
            v, parent, ci, nch = self.tets[i]
            if parent is not None:
                fam = self.tets[i:i + nch]
                if ci != 0 or len(fam) != nch or any(f[1] != parent or f[2] != q for q, f in enumerate(fam)):
                    raise AssertionError("green family not contiguous")
                R.append(parent)
                flags.append(bool(marked[i:i + nch].any()))
                i += nch
            else:
                R.append(v)
                flags.append(bool(marked[i]))
                i += 1
        # 2. red refinement and closure
        while True:
            newR = []
            for t, fl in zip(R, flags):
                newR.extend(self._red(t) if fl else [t])
            R = newR
            self._close_faces(R)
            flags = [len(self._split_edges(t)) > 3 or self._over(t) for t in R]
            if not any(flags):
                break
        # 3. green closure
        out = []
        for t in R:
            split = self._split_edges(t)
            if split:
                ch = self._green(t, split)
                out.extend((c, t, q, len(ch)) for q, c in enumerate(ch))
            else:
                out.append((t, None, -1, 0))
        self.tets = out


# --------------------------------------------------------------------------------------
# Adjoint of the discrete solve: gradients of J(u) = u^T M_S u (no counterpart in the paper)
# --------------------------------------------------------------------------------------

def exact_solve(prob: Problem) -> np.ndarray:
    """Exact discrete solution u_L of A_L u = b_L (Eq. 4.15) with Dirichlet values g_L, by sparse LU
    (the pins' reference)."""
    import scipy.sparse.linalg as spla
    h = prob.h
    lev = h.levels[h.L]
    F = np.nonzero(lev.free)[0]
    D = np.nonzero(lev.dirichlet)[0]
    u = np.zeros(len(lev.keys))
    u[D] = prob.g[h.L][D]
    rhs = prob.b[h.L][F] - lev.A[F][:, D] @ u[D]
    u[F] = spla.spsolve(lev.A[F][:, F].tocsc(), rhs)
    return u


def adjoint_gradients(h: Hierarchy, u_L: np.ndarray, in_S: np.ndarray):
    """J = sum_{T in S} u^T M_{L,T} u and its gradients w.r.t. nodal f and per-macro k_T (no
    counterpart in the paper).

    Solves A_ff lam_f = 2 (M_S u)_f (lam = 0 on Dirichlet nodes) exactly, then
      dJ/df = M_L lam          (b_L = M_L f_L),
      dJ/dk_T = -lam^T A_T^(1) u  (A_L = sum_T k_T A_T^(1)).
    """
    import scipy.sparse.linalg as spla
    lev = h.levels[h.L]
    in_S = np.asarray(in_S, dtype=bool)
    J = float(local_mass_sq(lev, u_L, h.n_cells)[in_S].sum())
    ee = u_L[lev.elems]
    sel = in_S[lev.emacro]
    g = np.zeros(len(lev.keys))
    np.add.at(g, lev.elems[sel].ravel(), 2.0 * np.einsum("eab,eb->ea", lev.Me[sel], ee[sel]).ravel())
    F = np.nonzero(lev.free)[0]
    lam = np.zeros(len(lev.keys))
    lam[F] = spla.spsolve(lev.A[F][:, F].tocsc(), g[F])
    grad_f = lev.M @ lam
    ll = lam[lev.elems]
    unit = lev.Ke / h.k[lev.emacro][:, None, None]
    per_elem = np.einsum("ea,eab,eb->e", ll, unit, ee)
    grad_k = -np.bincount(lev.emacro, weights=per_elem, minlength=h.n_cells)
    return J, grad_f, grad_k, lam
