"""Oracle, part 1: finite-element operators of the periodic cell problem, assembled in FP64.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, links or calls this module; only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` do.

What is computed (definitions, no blocking or fusion):

* Sec. 3, Eq. Du_mat / Eq. grad_componets: the gradient matrix D with entries dphi_I/dx_beta at the
  quadrature points, in Mandel form for elasticity (Eq. mandel_grad) and plain d-vector form for the
  scalar problem (App. A, Eq. Dt_mat).
* Sec. 3, Eq. W_mat and Eq. global_sum: quadrature weights w^Q (Fig. 3: two P1 triangles per pixel
  with w = V_p / 2; bilinear/trilinear elements with 2^d Gauss points, w = V_p / 2^d; the 3-D
  counterpart of Fig. 3 b, six P1 tetrahedra per voxel with one point each, w = V_p / 6).
* Sec. 3.1, Eq. lin_system: K = D^T W C D and, for the linear problem at u_(0) = 0,
  b = -D^T W C e.  Assembled as a scipy CSR matrix over element matrices
  K_e = sum_q w_q B_q^T C_e B_q with periodic node wrap.
* Sec. 2 (average strain definition) with the quadrature of Eq. global_sum: the volume average of
  flux / stress, <sigma> = (1/|Y|) sum_Q w_Q C_Q (e + (D u)_Q).

Conventions (readings of the paper where it is silent): unit cell [0, 1]^d, grid of n_x x n_y
(x n_z) nodes, node (i, j, k) at h * (i, j, k), voxel (i, j, k) with corner nodes (i + a, j + b,
k + c) mod n; node flat index i + n_x (j + n_y k); DOF index comp * N + node (component-blocked,
the paper's u = [u_1; u_2] ordering of Eq. Du_mat).  Mandel order (11, 22, 12) in 2-D and
(11, 22, 33, 23, 13, 12) in 3-D with sqrt(2) on shear strains.  P1 pixels are split along the
(0, 0)-(1, 1) diagonal; P1 voxels into the six tetrahedra that share the (0, 0, 0)-(1, 1, 1)
diagonal, one per order in which a path from (0, 0, 0) to (1, 1, 1) steps along x, y and z.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.sparse as sp

ELEMS = ("p1tri2_2d", "q1_2d", "hex8_3d", "p1tri4_2d", "p1tet6_3d")


# ----------------------------------------------------------------------------------------------
# grid bookkeeping
# ----------------------------------------------------------------------------------------------
class Grid:
    """Periodic regular grid: ``shape`` = (n_z, n_y, n_x) in 3-D or (n_y, n_x) in 2-D."""

    def __init__(self, shape, elem: str, physics: str):
        assert elem in ELEMS and physics in ("scalar", "elastic")
        self.shape = tuple(int(s) for s in shape)
        self.dim = len(self.shape)
        assert (self.dim == 3) == (elem in ("hex8_3d", "p1tet6_3d"))
        self.elem, self.physics = elem, physics
        self.n_xyz = self.shape[::-1]                       # (n_x, n_y[, n_z])
        self.h = np.array([1.0 / n for n in self.n_xyz])     # unit cell
        self.vp = float(np.prod(self.h))                     # pixel / voxel volume
        self.N = int(np.prod(self.shape))                    # nodes == voxels (one-node stencil)
        self.c = 1 if physics == "scalar" else self.dim      # DOF per node
        self.m = self.dim if physics == "scalar" else self.dim * (self.dim + 1) // 2
        self.corners = list(itertools.product((0, 1), repeat=self.dim))  # (a, b[, c]) per x, y, z
        # local corner ordering: a + 2 b (+ 4 c)
        self.corners = sorted(self.corners, key=lambda t: sum(v << i for i, v in enumerate(t)))
        self.ne = len(self.corners)
        # two-node stencil (Fig. 3 c): a corner node and a centre node per pixel, four P1 triangles;
        # the DOF vector is [corner values; centre values] (node type as the outer block, like a
        # component), scalar physics only
        self.nn = 2 if elem == "p1tri4_2d" else 1
        if self.nn == 2:
            assert physics == "scalar"
            self.c = 2              # DOF blocks of N values (node types)
            self.ne = 5             # element DOFs: 4 corners + centre

    def node_index(self, ijk):
        """Flat node index of integer coordinates (tuple of arrays, x first), wrapped periodically."""
        idx = 0
        stride = 1
        for ax, n in enumerate(self.n_xyz):
            idx = idx + np.mod(ijk[ax], n) * stride
            stride *= n
        return idx

    def element_nodes(self):
        """(N_elem, n_e) array: global node of each local corner of each voxel."""
        coords = np.meshgrid(*[np.arange(n) for n in self.n_xyz], indexing="ij")
        base = [c.transpose(*range(self.dim)[::-1]).ravel() for c in coords]  # x-fastest flattening
        out = np.empty((self.N, len(self.corners)), dtype=np.int64)
        for a, off in enumerate(self.corners):
            out[:, a] = self.node_index([base[ax] + off[ax] for ax in range(self.dim)])
        return out

    def element_dofs(self):
        """(N_elem, c * n_e) DOF map, element DOF order (component j, corner a) -> j * n_e + a.
        Two-node stencil: the 4 corner DOFs then the pixel's centre DOF (N + pixel)."""
        nodes = self.element_nodes()
        if self.nn == 2:
            return np.concatenate([nodes, self.N + np.arange(self.N)[:, None]], axis=1)
        return np.concatenate([j * self.N + nodes for j in range(self.c)], axis=1)


# ----------------------------------------------------------------------------------------------
# element gradients at the quadrature points (Sec. 3, Fig. 3)
# ----------------------------------------------------------------------------------------------
def _p1_gradients(verts):
    """Gradients of the d + 1 P1 basis functions of a simplex with vertices ``verts`` ((d+1) x d)."""
    k = verts.shape[0]
    A = np.column_stack([np.ones(k), verts])          # rows [1, x, y(, z)]; phi_i = coefficients
    coef = np.linalg.inv(A)                           # column i: coefficients of phi_i
    return coef[1:, :]                                # (d, d + 1): d phi_i / d x_beta


def quadrature(grid: Grid):
    """List of (dN, w) per quadrature point of one voxel: dN is (d, n_e) = dphi_a/dx_beta."""
    h, d = grid.h, grid.dim
    pts = []
    if grid.elem == "p1tri4_2d":
        # Fig. 3 c: triangles (edge, centre) for the bottom, right, top and left edges, w = V_p / 4
        corner_xy = {off: np.array(off, dtype=float) * h for off in grid.corners}
        centre = 0.5 * h
        for e0, e1 in (((0, 0), (1, 0)), ((1, 0), (1, 1)), ((1, 1), (0, 1)), ((0, 1), (0, 0))):
            g = _p1_gradients(np.array([corner_xy[e0], corner_xy[e1], centre]))
            dN = np.zeros((2, 5))
            dN[:, grid.corners.index(e0)] = g[:, 0]
            dN[:, grid.corners.index(e1)] = g[:, 1]
            dN[:, 4] = g[:, 2]
            pts.append((dN, grid.vp / 4.0))
    elif grid.elem == "p1tet6_3d":
        # six tetrahedra (0,0,0) -> +e_p -> +e_q -> (1,1,1), one per order (p, q, r) of the axes
        corner_xyz = {off: np.array(off, dtype=float) * h for off in grid.corners}
        for order in itertools.permutations(range(3)):
            path = [(0, 0, 0)]
            for ax in order:
                nxt = list(path[-1])
                nxt[ax] = 1
                path.append(tuple(nxt))
            g = _p1_gradients(np.array([corner_xyz[t] for t in path]))
            dN = np.zeros((3, grid.ne))
            for col, t in enumerate(path):
                dN[:, grid.corners.index(t)] = g[:, col]
            pts.append((dN, grid.vp / 6.0))
    elif grid.elem == "p1tri2_2d":
        corner_xy = {off: np.array(off, dtype=float) * h for off in grid.corners}
        for tri in (((0, 0), (1, 0), (1, 1)), ((0, 0), (1, 1), (0, 1))):
            g = _p1_gradients(np.array([corner_xy[t] for t in tri]))
            dN = np.zeros((2, grid.ne))
            for col, t in enumerate(tri):
                dN[:, grid.corners.index(t)] = g[:, col]
            pts.append((dN, grid.vp / 2.0))
    else:
        # multilinear shape functions on [-1, 1]^d, Gauss points +-1/sqrt(3), weight 1 each
        g = 1.0 / math.sqrt(3.0)
        for xi in itertools.product((-g, g), repeat=d):
            dN = np.zeros((d, grid.ne))
            for a, off in enumerate(grid.corners):
                s = [2 * o - 1 for o in off]
                for beta in range(d):
                    val = 1.0
                    for ax in range(d):
                        val *= (s[ax] if ax == beta else (1.0 + s[ax] * xi[ax]))
                    dN[beta, a] = val / (2 ** d) * (2.0 / h[beta])
            pts.append((dN, grid.vp / (2 ** d)))
    return pts


_SHEAR_PAIRS = {2: [(0, 1)], 3: [(1, 2), (0, 2), (0, 1)]}


def b_matrix(grid: Grid, dN):
    """B_q mapping element DOFs to the gradient (scalar, d rows) or Mandel strain (m rows)."""
    d, ne = grid.dim, grid.ne
    if grid.physics == "scalar":
        return dN.copy()
    B = np.zeros((grid.m, d * ne))
    for i in range(d):                                   # normal strains eps_ii = d_i u_i
        B[i, i * ne:(i + 1) * ne] = dN[i]
    r2 = math.sqrt(2.0) / 2.0                            # Mandel: sqrt(2) * eps_ij = (d_j u_i + d_i u_j) / sqrt(2)
    for row, (i, j) in enumerate(_SHEAR_PAIRS[d], start=d):
        B[row, i * ne:(i + 1) * ne] += r2 * dN[j]
        B[row, j * ne:(j + 1) * ne] += r2 * dN[i]
    return B


def element_B(grid: Grid):
    """[(B_q, w_q)] for one voxel."""
    return [(b_matrix(grid, dN), w) for dN, w in quadrature(grid)]


def element_stiffness(grid: Grid, C):
    """K_e = sum_q w_q B_q^T C B_q for a voxel of uniform material C (Eq. lin_system, per element)."""
    return sum(w * B.T @ C @ B for B, w in element_B(grid))


def element_load(grid: Grid, C, e):
    """f_e = sum_q w_q B_q^T C e: the element part of D^T W C e."""
    return sum(w * B.T @ (C @ e) for B, w in element_B(grid))


# ----------------------------------------------------------------------------------------------
# global operators
# ----------------------------------------------------------------------------------------------
def assemble_K(grid: Grid, phases, moduli):
    """Global stiffness K = D^T W C D (CSR, FP64) with material C = moduli[phase] per voxel."""
    phases = np.asarray(phases).ravel()
    dofs = grid.element_dofs()
    Ke = np.stack([element_stiffness(grid, C) for C in moduli])          # (P, k, k)
    vals = Ke[phases]                                                   # (N_e, k, k)
    k = dofs.shape[1]
    rows = np.repeat(dofs, k, axis=1).ravel()
    cols = np.tile(dofs, (1, k)).ravel()
    n = grid.c * grid.N
    return sp.coo_matrix((vals.ravel(), (rows, cols)), shape=(n, n)).tocsr()


def assemble_rhs(grid: Grid, phases, moduli, e):
    """b = -D^T W C e for the macroscopic gradient / strain e (linear problem, u_(0) = 0)."""
    phases = np.asarray(phases).ravel()
    dofs = grid.element_dofs()
    fe = np.stack([element_load(grid, C, np.asarray(e, float)) for C in moduli])  # (P, k)
    b = np.zeros(grid.c * grid.N)
    np.add.at(b, dofs.ravel(), -fe[phases].ravel())
    return b


def stiffness_rows(grid: Grid, phases, moduli, u, dof_rows):
    """(K u)[dof_rows] computed element by element, without assembling K.

    For each requested DOF (component j at node n) the 2^d voxels that contain n contribute the
    matching row of their element matrix times their element DOF vector.
    """
    phases = np.asarray(phases).ravel()
    dof_rows = np.asarray(dof_rows, dtype=np.int64)
    comp, node = dof_rows // grid.N, dof_rows % grid.N
    Ke = np.stack([element_stiffness(grid, C) for C in moduli])
    # node coordinates
    coords, rem = [], node.copy()
    for n in grid.n_xyz:
        coords.append(rem % n)
        rem //= n
    out = np.zeros(dof_rows.shape)
    for a, off in enumerate(grid.corners):
        # the voxel whose corner a is this node
        vox = grid.node_index([coords[ax] - off[ax] for ax in range(grid.dim)])
        vcoords = [coords[ax] - off[ax] for ax in range(grid.dim)]
        edofs = []
        for j in range(grid.c):
            for b_, off2 in enumerate(grid.corners):
                edofs.append(j * grid.N + grid.node_index([vcoords[ax] + off2[ax] for ax in range(grid.dim)]))
        edofs = np.stack(edofs, axis=1)                                  # (S, k)
        row_local = comp * grid.ne + a
        Krow = Ke[phases[vox], row_local, :]                            # (S, k)
        out += np.einsum("sk,sk->s", Krow, u[edofs])
    return out


def mean_flux(grid: Grid, phases, moduli, e, u):
    """<sigma> = (1/|Y|) sum_Q w_Q C_Q (e + (D u)_Q), |Y| = 1 (Sec. 2 average; Eq. global_sum)."""
    phases = np.asarray(phases).ravel()
    dofs = grid.element_dofs()
    ue = u[dofs]                                                        # (N_e, k)
    acc = np.zeros(grid.m)
    for B, w in element_B(grid):
        strain = np.asarray(e, float)[None, :] + ue @ B.T               # (N_e, m)
        for p, C in enumerate(moduli):
            sel = phases == p
            if np.any(sel):
                acc += w * (strain[sel] @ C.T).sum(axis=0)
    return acc


def energy(grid: Grid, phases, moduli, e_i, u_i, e_j, u_j):
    """sum_Q w_Q (e_i + (D u_i)_Q)^T C_Q (e_j + (D u_j)_Q): the bilinear form of the cell energy of
    Sec. 2 (strain e + grad u, stress C times it) with the quadrature of Eq. global_sum.  At the
    solutions of the loads e_i, e_j it equals |Y| e_i^T C_eff e_j (Hill-Mandel)."""
    phases = np.asarray(phases).ravel()
    dofs = grid.element_dofs()
    ui, uj = u_i[dofs], u_j[dofs]
    acc = 0.0
    for B, w in element_B(grid):
        si = np.asarray(e_i, float)[None, :] + ui @ B.T
        sj = np.asarray(e_j, float)[None, :] + uj @ B.T
        for p, C in enumerate(moduli):
            sel = phases == p
            if np.any(sel):
                acc += w * float(np.einsum("qa,ab,qb->", si[sel], C, sj[sel]))
    return acc


def mean_material(grid: Grid, phases, moduli):
    """C_mean = (1/|Y|) sum_Q C(x_Q) w_Q (Sec. 6.2 reference-material choice)."""
    phases = np.asarray(phases).ravel()
    counts = np.bincount(phases, minlength=len(moduli)).astype(float)
    volume = grid.vp * grid.N  # |Y|: 1 on the unit cell, the cell volume when grid.h is scaled
    return np.einsum("p,pij->ij", counts * grid.vp / volume, np.asarray(moduli, float))
