"""Pins of the FP64 CPU oracle against facts fixed by the paper and by the mathematics.

Each test checks the oracle against something other than itself: textbook closed forms, the
closed-form Fourier symbol of the tensor-product elements, exact laminate results, invariants
(homogeneous material, symmetry, Voigt/Reuss bounds, Hill-Mandel energy identity, element-by-
element eigenvalue bounds of Sec. 4.3), one-iteration convergence for C = s C_ref (Sec. 4.3) and
brute force on tiny grids.  No GPU needed.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import fem, solvers
from paper_2203_02962_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


def _rand_spd(m, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, m))
    return scale * (A @ A.T + m * np.eye(m))


def _mandel_tensor(C):
    """Full 4th-order tensor C_ijkl (3-D or 2-D) from a Mandel matrix, written out for the test."""
    m = C.shape[0]
    d = 3 if m == 6 else 2
    pairs = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)] if d == 3 else [(0, 0), (1, 1), (0, 1)]
    w = [1.0 if i == j else math.sqrt(2.0) for i, j in pairs]
    T = np.zeros((d, d, d, d))
    for I_, (i, j) in enumerate(pairs):
        for J_, (k, l) in enumerate(pairs):
            v = C[I_, J_] / (w[I_] * w[J_])
            for a, b in ((i, j), (j, i)):
                for c, e in ((k, l), (l, k)):
                    T[a, b, c, e] = v
    return T


def _mandel_vec(E):
    d = E.shape[0]
    s2 = math.sqrt(2.0)
    if d == 2:
        return np.array([E[0, 0], E[1, 1], s2 * E[0, 1]])
    return np.array([E[0, 0], E[1, 1], E[2, 2], s2 * E[1, 2], s2 * E[0, 2], s2 * E[0, 1]])


# ------------------------------------------------------------------------------------------------
# element level: closed forms and patch tests
# ------------------------------------------------------------------------------------------------
def test_p1_scalar_is_five_point_laplacian():
    """Two P1 triangles per pixel, isotropic k: the assembled stencil is k * (4, -1, -1, -1, -1)."""
    k = 2.5
    g = fem.Grid((6, 6), "p1tri2_2d", "scalar")
    K = fem.assemble_K(g, np.zeros(g.N, int), [k * np.eye(2)]).toarray()
    for node in (0, 7, 35):
        i, j = node % 6, node // 6
        expect = np.zeros(g.N)
        expect[node] = 4 * k
        for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            expect[((i + di) % 6) + 6 * ((j + dj) % 6)] -= k
        np.testing.assert_allclose(K[node], expect, atol=1e-13)


def test_p1tet6_scalar_is_seven_point_laplacian():
    """Six tetrahedra per voxel along the (0,0,0)-(1,1,1) diagonal, identity conductivity, cubic voxels:
    K is the 7-point Laplacian times h (textbook stencil; the face- and body-diagonal couplings of the
    six tetrahedra cancel), and the reference symbol of an elastic material is real (the split is
    symmetric under the point reflection through the voxel centre)."""
    n = 4
    g = fem.Grid((n, n, n), "p1tet6_3d", "scalar")
    K = fem.assemble_K(g, np.zeros(g.N, int), [np.eye(3)]).toarray()
    h = g.h[0]
    L = np.zeros_like(K)
    for node in range(g.N):
        x, y, z = node % n, (node // n) % n, node // (n * n)
        L[node, node] = 6.0 * h
        for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
            L[node, ((x + dx) % n) + n * (((y + dy) % n) + n * ((z + dz) % n))] -= h
    np.testing.assert_allclose(K, L, atol=1e-14)
    ge = fem.Grid((4, 6, 4), "p1tet6_3d", "elastic")
    Sh = solvers.kref_symbol(ge, _rand_spd(6, 7))
    assert np.abs(np.imag(Sh)).max() <= 1e-14 * np.abs(Sh).max()


def test_hex8_scalar_element_closed_form():
    """Q1 3-D Laplacian element matrix: h*k*(1/3 diag, 0 edge, -1/12 face/body diagonal)."""
    n, k = 4, 3.0
    g = fem.Grid((n, n, n), "hex8_3d", "scalar")
    Ke = fem.element_stiffness(g, k * np.eye(3))
    h = 1.0 / n
    for a, oa in enumerate(g.corners):
        for b, ob in enumerate(g.corners):
            dist = sum(x != y for x, y in zip(oa, ob))
            expect = {0: 1 / 3, 1: 0.0, 2: -1 / 12, 3: -1 / 12}[dist] * h * k
            assert abs(Ke[a, b] - expect) < 1e-14


def test_q1_2d_scalar_element_closed_form():
    """Q1 2-D Laplacian element: (1/6) * [4 -1 -2 -1] pattern (diag, edge, diagonal), h-free."""
    g = fem.Grid((5, 5), "q1_2d", "scalar")
    Ke = fem.element_stiffness(g, np.eye(2))
    for a, oa in enumerate(g.corners):
        for b, ob in enumerate(g.corners):
            dist = sum(x != y for x, y in zip(oa, ob))
            assert abs(Ke[a, b] - {0: 4 / 6, 1: -1 / 6, 2: -2 / 6}[dist]) < 1e-14


@pytest.mark.parametrize("elem,shape", [("hex8_3d", (3, 4, 5)), ("q1_2d", (4, 5)), ("p1tri2_2d", (4, 5)),
                                        ("p1tet6_3d", (3, 4, 5))])
@pytest.mark.parametrize("physics", ["scalar", "elastic"])
def test_patch_linear_field(elem, shape, physics):
    """A linear nodal field has the exact constant gradient / Mandel strain at every quadrature point,
    and its element energy is V * eps^T C eps (patch test; pins D and the Mandel sqrt(2) factors)."""
    g = fem.Grid(shape, elem, physics)
    rng = np.random.default_rng(1)
    d = g.dim
    h = g.h
    X = np.array([[off[ax] * h[ax] for ax in range(d)] for off in g.corners])  # (ne, d)
    if physics == "scalar":
        gvec = rng.standard_normal(d)
        ue = X @ gvec
        target = gvec
    else:
        G = rng.standard_normal((d, d))       # u_i = sum_j G_ij x_j
        ue = np.concatenate([X @ G[i] for i in range(d)])
        E = 0.5 * (G + G.T)
        target = _mandel_vec(E)
    for B, w in fem.element_B(g):
        np.testing.assert_allclose(B @ ue, target, atol=1e-12)
    C = _rand_spd(g.m, 3)
    Ke = fem.element_stiffness(g, C)
    np.testing.assert_allclose(ue @ Ke @ ue, g.vp * target @ C @ target, rtol=1e-12)
    # constant fields (translations) are in the kernel
    for j in range(g.c):
        t = np.zeros(g.c * g.ne)
        t[j * g.ne:(j + 1) * g.ne] = 1.0
        np.testing.assert_allclose(Ke @ t, 0.0, atol=1e-12)


def test_hex8_elastic_rigid_rotations():
    """Infinitesimal rotations u = W x (W skew) produce zero strain: 6 null modes of K_e in 3-D."""
    g = fem.Grid((3, 3, 3), "hex8_3d", "elastic")
    Ke = fem.element_stiffness(g, I.isotropic_elastic_mandel(1.0, 0.3))
    ev = np.linalg.eigvalsh(Ke)
    assert np.sum(np.abs(ev) < 1e-12 * ev.max()) == 6


# ------------------------------------------------------------------------------------------------
# Algorithm 2: symbol of K_ref against its closed form; pseudo-inverse action
# ------------------------------------------------------------------------------------------------
def _closed_form_hex8(shape, A4, h):
    """K_hat_ab(k) = sum_ij A_{i a j b} S_ij, S_ii = k_i prod m_j, S_ij = sin_i sin_j prod m_k.

    1-D factors on a periodic line of spacing h: stiffness (2 - 2 cos t)/h, mass h (2 + cos t)/3,
    first-derivative coupling sin t (up to a sign that cancels in S_ij)."""
    d = len(shape)
    th = np.meshgrid(*[2 * np.pi * np.arange(n) / n for n in shape], indexing="ij")  # (z, y, x) order
    th = th[::-1]                                      # x, y, z
    hh = h
    kf = [(2 - 2 * np.cos(t)) / hh[i] for i, t in enumerate(th)]
    mf = [hh[i] * (2 + np.cos(t)) / 3 for i, t in enumerate(th)]
    sf = [np.sin(t) for t in th]
    S = np.empty((d, d) + tuple(shape))
    for i in range(d):
        for j in range(d):
            if i == j:
                val = kf[i].copy()
                for l in range(d):
                    if l != i:
                        val = val * mf[l]
            else:
                val = sf[i] * sf[j]
                for l in range(d):
                    if l not in (i, j):
                        val = val * mf[l]
            S[i, j] = val
    if A4.ndim == 2:       # scalar conductivity A_ij
        return np.einsum("ij,ij...->...", A4, S)[None, None]
    return np.einsum("iajb,ij...->ab...", A4, S)


def test_symbol_hex8_scalar_closed_form():
    shape = (4, 6, 8)  # (z, y, x)
    g = fem.Grid(shape, "hex8_3d", "scalar")
    A = _rand_spd(3, 5)
    Kh = solvers.kref_symbol(g, A)
    assert np.max(np.abs(Kh.imag)) < 1e-13 * np.max(np.abs(Kh.real))
    ref = _closed_form_hex8(shape, A, g.h)
    np.testing.assert_allclose(Kh.real, ref, atol=1e-12 * np.abs(ref).max())


def test_symbol_hex8_elastic_closed_form():
    shape = (4, 4, 6)
    g = fem.Grid(shape, "hex8_3d", "elastic")
    C = _rand_spd(6, 7)
    Kh = solvers.kref_symbol(g, C)
    assert np.max(np.abs(Kh.imag)) < 1e-13 * np.max(np.abs(Kh.real))
    ref = _closed_form_hex8(shape, _mandel_tensor(C), g.h)
    np.testing.assert_allclose(Kh.real, ref, atol=1e-12 * np.abs(ref).max())
    # k = 0 block is the zero matrix: d null eigenvalues (Sec. 5.3)
    assert np.max(np.abs(Kh[:, :, 0, 0, 0])) < 1e-12 * np.abs(ref).max()


def test_symbol_p1_isotropic_closed_form():
    shape = (6, 8)
    g = fem.Grid(shape, "p1tri2_2d", "scalar")
    k = 1.7
    Kh = solvers.kref_symbol(g, k * np.eye(2))[0, 0]
    t1 = 2 * np.pi * np.arange(8) / 8
    t2 = 2 * np.pi * np.arange(6) / 6
    hx, hy = 1 / 8, 1 / 6       # rectangular pixels: edge couplings scale with h_y/h_x and h_x/h_y
    ref = k * ((hy / hx) * (2 - 2 * np.cos(t1))[None, :] + (hx / hy) * (2 - 2 * np.cos(t2))[:, None])
    np.testing.assert_allclose(Kh, ref, atol=1e-12)


@pytest.mark.parametrize("elem,shape,physics", [("hex8_3d", (4, 6, 4), "elastic"),
                                                 ("hex8_3d", (6, 4, 8), "scalar"),
                                                 ("p1tri2_2d", (6, 8), "elastic"),
                                                 ("q1_2d", (6, 4), "scalar"),
                                                 ("p1tet6_3d", (4, 6, 4), "elastic"),
                                                 ("p1tet6_3d", (6, 4, 8), "scalar")])
def test_precond_is_pseudo_inverse(elem, shape, physics):
    """K_ref (K_ref^+ r) = r minus its mean per component, for a random r (Eq. M_inverse)."""
    g = fem.Grid(shape, elem, physics)
    C = _rand_spd(g.m, 11)
    Kref = fem.assemble_K(g, np.zeros(g.N, int), [C])
    Kinv = solvers.kref_pinv_symbol(solvers.kref_symbol(g, C))
    r = np.random.default_rng(2).standard_normal(g.c * g.N)
    z = solvers.apply_precond(g, Kinv, r)
    np.testing.assert_allclose(Kref @ z, solvers.project_mean_zero(g, r), atol=1e-11 * np.abs(r).max())
    # z is mean-zero per component (pseudo-inverse at k = 0)
    np.testing.assert_allclose(solvers.project_mean_zero(g, z), z, atol=1e-12)


# ------------------------------------------------------------------------------------------------
# invariants and exact results of the homogenised problem
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("elem,shape,physics", [("hex8_3d", (4, 4, 4), "elastic"),
                                                 ("p1tri2_2d", (8, 8), "scalar"),
                                                 ("q1_2d", (6, 6), "elastic"),
                                                 ("p1tet6_3d", (4, 4, 4), "elastic")])
def test_homogeneous_material(elem, shape, physics):
    g = fem.Grid(shape, elem, physics)
    C = _rand_spd(g.m, 4)
    ids = np.zeros(g.N, int)
    for e in np.eye(g.m):
        np.testing.assert_allclose(fem.assemble_rhs(g, ids, [C], e), 0.0, atol=1e-13)
    res = solvers.homogenise(g, ids, [C], np.eye(g.m), method="dense")
    np.testing.assert_allclose(res["fields"], 0.0, atol=1e-12)
    np.testing.assert_allclose(res["C_eff"], C, rtol=1e-13, atol=1e-13)


def test_laminate_scalar_exact():
    """Layers normal to x: C_eff = diag(harmonic, arithmetic[, arithmetic]) exactly (FE space holds the solution)."""
    layers = [0, 0, 1, 1, 1, 0, 2, 2]
    ks = [1.0, 10.0, 3.0]
    for elem, shape in (("hex8_3d", (2, 3, 8)), ("p1tri2_2d", (4, 8)), ("q1_2d", (4, 8)), ("p1tet6_3d", (2, 3, 8))):
        g = fem.Grid(shape, elem, "scalar")
        ids = I.laminate(shape, layers).ravel()
        mod = [k * np.eye(g.dim) for k in ks]
        res = solvers.homogenise(g, ids, mod, np.eye(g.dim), method="dense")
        kk = np.array([ks[p] for p in layers])
        expect = np.diag([1.0 / np.mean(1.0 / kk)] + [np.mean(kk)] * (g.dim - 1))
        np.testing.assert_allclose(res["C_eff"], expect, rtol=1e-11, atol=1e-12)


def test_laminate_elastic_exact():
    """Exact laminate formula derived here for layers normal to x, in Mandel coordinates.

    The fluctuation only produces the strain components that involve the normal (n-set: 11, 13,
    12); the t-set strains equal the macro strain and the n-set stresses are continuous, which gives
    C_eff = <C> - <C_:n C_nn^-1 C_n:> + <C_:n C_nn^-1> <C_nn^-1>^-1 <C_nn^-1 C_n:>."""
    layers = [0, 1, 1, 0, 0, 2]
    Cs = [_rand_spd(6, 20), _rand_spd(6, 21, 5.0), I.isotropic_elastic_mandel(7.0, 0.25)]
    ids = I.laminate((2, 2, 6), layers).ravel()
    res = solvers.homogenise(fem.Grid((2, 2, 6), "hex8_3d", "elastic"), ids, Cs, np.eye(6), method="dense")
    res_tet = solvers.homogenise(fem.Grid((2, 2, 6), "p1tet6_3d", "elastic"), ids, Cs, np.eye(6), method="dense")
    nset = [0, 4, 5]
    f = np.bincount(layers, minlength=3) / len(layers)
    avg = lambda fn: sum(f[p] * fn(Cs[p]) for p in range(3))
    inv_nn = lambda C: np.linalg.inv(C[np.ix_(nset, nset)])
    A = avg(lambda C: C)
    Bm = avg(lambda C: C[:, nset] @ inv_nn(C) @ C[nset, :])
    L = avg(lambda C: C[:, nset] @ inv_nn(C))
    M = avg(inv_nn)
    R = avg(lambda C: inv_nn(C) @ C[nset, :])
    expect = A - Bm + L @ np.linalg.inv(M) @ R
    np.testing.assert_allclose(res["C_eff"], expect, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(res_tet["C_eff"], expect, rtol=1e-10, atol=1e-10)


def _voigt_reuss_check(C_eff, moduli, ids):
    f = np.bincount(np.asarray(ids).ravel(), minlength=len(moduli)) / np.asarray(ids).size
    voigt = sum(fp * C for fp, C in zip(f, moduli))
    reuss = np.linalg.inv(sum(fp * np.linalg.inv(C) for fp, C in zip(f, moduli)))
    sym = 0.5 * (C_eff + C_eff.T)
    assert np.linalg.eigvalsh(voigt - sym).min() > -1e-10
    assert np.linalg.eigvalsh(sym - reuss).min() > -1e-10


def test_circle2d_invariants_and_solver_agreement():
    """32^2 P1 disc cell: dense-equivalent sparse LU, CG and PCG agree; C_eff symmetric, inside
    the Voigt/Reuss bounds; Hill-Mandel: e^T <sigma> = <(e + Du)^T C (e + Du)>."""
    w = I.workload_circle2d_32()
    g = fem.Grid((32, 32), "p1tri2_2d", "scalar")
    r_lu = solvers.homogenise(g, w["ids"], w["moduli"], w["loads"], method="sparse")
    r_cg = solvers.homogenise(g, w["ids"], w["moduli"], w["loads"], method="cg", tol=1e-14)
    r_pcg = solvers.homogenise(g, w["ids"], w["moduli"], w["loads"], method="pcg", tol=1e-13)
    np.testing.assert_allclose(r_cg["C_eff"], r_lu["C_eff"], rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(r_pcg["C_eff"], r_lu["C_eff"], rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(r_pcg["fields"], r_lu["fields"], atol=1e-11)
    C = r_lu["C_eff"]
    assert abs(C[0, 1]) < 1e-12 and abs(C[0, 0] - C[1, 1]) < 1e-12   # square symmetry of the disc
    _voigt_reuss_check(C, w["moduli"], w["ids"])
    # Hill-Mandel energy identity
    ids = w["ids"].ravel()
    dofs = g.element_dofs()
    for li, e in enumerate(w["loads"]):
        u = r_lu["fields"][li]
        energy = 0.0
        for B, wq in fem.element_B(g):
            strain = e[None, :] + u[dofs] @ B.T
            Cq = np.asarray(w["moduli"])[ids]
            energy += wq * np.einsum("ni,nij,nj->", strain, Cq, strain)
        assert abs(energy - e @ r_lu["mean_flux"][li]) < 1e-11


@pytest.mark.parametrize("elem,shape,physics", [("hex8_3d", (3, 2, 4), "elastic"),
                                                 ("hex8_3d", (2, 3, 4), "scalar"),
                                                 ("p1tri2_2d", (4, 6), "elastic"),
                                                 ("q1_2d", (3, 4), "scalar"),
                                                 ("p1tet6_3d", (3, 2, 4), "elastic")])
def test_brute_force_tiny(elem, shape, physics):
    """Tiny random grids: dense bordered solve == CG == PCG; residual K u - b vanishes."""
    g = fem.Grid(shape, elem, physics)
    rng = np.random.default_rng(9)
    ids = rng.integers(0, 3, g.N)
    mod = [_rand_spd(g.m, 30 + p, 10.0 ** p) for p in range(3)]
    K = fem.assemble_K(g, ids, mod)
    e = rng.standard_normal(g.m)
    b = fem.assemble_rhs(g, ids, mod, e)
    u_d = solvers.solve_dense(g, K, b)
    np.testing.assert_allclose(K @ u_d, b, atol=1e-11 * np.abs(b).max())
    u_c, _, _ = solvers.cg(K, b, tol=1e-15)
    Kinv = solvers.kref_pinv_symbol(solvers.kref_symbol(g, fem.mean_material(g, ids, mod)))
    res = solvers.pcg(lambda v: K @ v, lambda v: solvers.apply_precond(g, Kinv, v), b, 1e-14)
    scale = np.abs(u_d).max()
    np.testing.assert_allclose(solvers.project_mean_zero(g, u_c), u_d, atol=1e-10 * scale)
    np.testing.assert_allclose(solvers.project_mean_zero(g, res["x"]), u_d, atol=1e-10 * scale)
    # element-by-element stiffness rows agree with the assembled matrix
    rows = rng.integers(0, g.c * g.N, 17)
    np.testing.assert_allclose(fem.stiffness_rows(g, ids, mod, u_d, rows), (K @ u_d)[rows], atol=1e-12 * scale)


def test_one_iteration_when_reference_equals_material():
    """C = s * C_ref everywhere: M^-1 K = s I on the range, PCG converges in one step (Sec. 4.3)."""
    g = fem.Grid((4, 6, 4), "hex8_3d", "elastic")
    C_ref = _rand_spd(6, 40)
    K = fem.assemble_K(g, np.zeros(g.N, int), [3.5 * C_ref])
    Kinv = solvers.kref_pinv_symbol(solvers.kref_symbol(g, C_ref))
    b = solvers.project_mean_zero(g, np.random.default_rng(3).standard_normal(g.c * g.N))
    res = solvers.pcg(lambda v: K @ v, lambda v: solvers.apply_precond(g, Kinv, v), b, 1e-12)
    assert res["iters"] == 1
    np.testing.assert_allclose(res["alphas"][0], 1 / 3.5, rtol=1e-12)


def test_ritz_values_inside_element_bounds():
    """Sec. 4.3: the spectrum of K_ref^-1 K lies in [min_e lambda_min(C_ref^-1 C_e), max_e lambda_max];
    the CG-Lanczos Ritz values from the PCG coefficients must lie there too."""
    g = fem.Grid((6, 6, 6), "hex8_3d", "elastic")
    rng = np.random.default_rng(5)
    ids = rng.integers(0, 2, g.N)
    mod = [I.isotropic_elastic_mandel(1.0, 0.3), I.isotropic_elastic_mandel(20.0, 0.2)]
    C_ref = fem.mean_material(g, ids, mod)
    K = fem.assemble_K(g, ids, mod)
    Kinv = solvers.kref_pinv_symbol(solvers.kref_symbol(g, C_ref))
    b = fem.assemble_rhs(g, ids, mod, np.eye(6)[0])
    res = solvers.pcg(lambda v: K @ v, lambda v: solvers.apply_precond(g, Kinv, v), b, 1e-10)
    ritz = solvers.lanczos_ritz(res["alphas"], res["betas"])
    lam = [np.linalg.eigvals(np.linalg.solve(C_ref, C)).real for C in mod]
    lo, hi = min(l.min() for l in lam), max(l.max() for l in lam)
    assert ritz.min() >= lo * (1 - 1e-8) and ritz.max() <= hi * (1 + 1e-8)


def test_iterations_flat_under_refinement():
    """h-independent conditioning (Sec. 4.3): PCG iterations for the disc cell at fixed contrast
    stay within +-20 % when the grid is refined 32 -> 64 -> 128 (tol 1e-8)."""
    its = []
    for n in (32, 64, 128):
        g = fem.Grid((n, n), "p1tri2_2d", "scalar")
        ids = I.circle2d(n, 0.3)
        mod = [np.eye(2), 10.0 * np.eye(2)]
        res = solvers.homogenise(g, ids, mod, np.eye(2)[:1], method="pcg", tol=1e-8)
        its.append(res["iters"][0])
    assert max(its) <= 1.2 * min(its), its


def test_coated_sphere_bulk_modulus_golden():
    """Sec. 6.2 coated sphere (golden parameters): the neutral coated inclusion leaves the
    hydrostatic response of the K_eff matrix unchanged, so the cell bulk modulus is ~K_eff = 1.0
    (exact in the continuum, up to the voxelisation of the two spheres here)."""
    with open(os.path.join(HERE, "golden", "hashin_coated_sphere.json")) as fh:
        gd = json.load(fh)
    n = 16
    g = fem.Grid((n, n, n), "hex8_3d", "elastic")
    ids = I.coated_sphere(n, gd["r1"], gd["r2"]).ravel()
    mod = [I.bulk_shear_mandel(gd["K1"], gd["G1"]), I.bulk_shear_mandel(gd["K2"], gd["G2"]),
           I.bulk_shear_mandel(gd["K_eff"], gd["G_eff"])]
    e = np.array([1.0, 1.0, 1.0, 0, 0, 0]) / 3.0          # hydrostatic strain, trace 1
    res = solvers.homogenise(g, ids, mod, e[None, :], method="pcg", tol=1e-10)
    sig = res["mean_flux"][0]
    K_cell = sig[:3].mean()                                # mean normal stress / trace(e) = K
    assert abs(K_cell - gd["K_eff"]) < 0.1, K_cell
    # without the coating balance (core material everywhere inside r2) the response moves far away
    mod_bad = [mod[0], mod[0], mod[2]]
    sig_bad = solvers.homogenise(g, ids, mod_bad, e[None, :], method="pcg", tol=1e-8)["mean_flux"][0]
    assert abs(sig_bad[:3].mean() - gd["K_eff"]) > 0.3


@pytest.mark.parametrize("elem,shape,physics", [("hex8_3d", (4, 4, 4), "elastic"), ("p1tri2_2d", (6, 6), "scalar"),
                                                 ("q1_2d", (6, 4), "elastic"), ("hex8_3d", (4, 2, 6), "scalar")])
def test_element_eigenvalue_bounds_bracket_the_spectrum(elem, shape, physics):
    """Sec. 4.3: sorted per-node bounds bracket every eigenvalue of K_ref^-1 K on the mean-zero
    space: lower[j + c] <= lambda_j <= upper[j] (dense generalized eigenproblem on tiny grids)."""
    import scipy.linalg as sl
    g = fem.Grid(shape, elem, physics)
    rng = np.random.default_rng(17)
    ids = rng.integers(0, 3, g.N)
    if physics == "elastic":
        mod = [I.isotropic_elastic_mandel(E, nu, g.dim) for E, nu in ((1, 0.3), (30, 0.2), (5, 0.4))]
    else:
        mod = [k * np.eye(g.dim) for k in (1.0, 30.0, 5.0)]
    C_ref = fem.mean_material(g, ids, mod)
    K = fem.assemble_K(g, ids, mod).toarray()
    Kr = fem.assemble_K(g, np.zeros(g.N, int), [C_ref]).toarray()
    Q, _ = np.linalg.qr(solvers.constant_modes(g), mode="complete")
    B = Q[:, g.c:]
    lam = np.sort(sl.eigh(B.T @ K @ B, B.T @ Kr @ B, eigvals_only=True))
    lower, upper = solvers.eig_bounds(g, ids, mod, C_ref)
    n = lam.size
    assert np.all(lower[g.c:] <= lam + 1e-9) and np.all(lam <= upper[:n] + 1e-9)
    # the global bounds are the phase extremes
    assert lower[0] == min(sl.eigh(C, C_ref, eigvals_only=True).min() for C in mod)


def test_coated_sphere_balance_reproduces_printed_moduli():
    """Sec. 6.2 golden values: the neutral-inclusion balance at rho = 1e3 gives the printed K1, K2."""
    from paper_2203_02962_gb300 import coated_sphere
    with open(os.path.join(HERE, "golden", "hashin_coated_sphere.json")) as fh:
        gd = json.load(fh)
    (K1, G1), (K2, G2), (Ke, Ge) = coated_sphere.balanced_moduli(1e3)
    assert abs(K1 - gd["K1"]) < 5e-9 and abs(K2 - gd["K2"]) < 5e-7
    assert abs(G1 - gd["G1"]) < 5e-9 and abs(G2 - gd["G2"]) < 5e-7
    assert Ke == gd["K_eff"] and abs(Ge - gd["G_eff"]) < 1e-15


def test_energy_bilinear_form_pins():
    """fem.energy: at the exact solutions it is |Y| e_i^T C_eff e_j for every pair of loads (Hill-Mandel,
    bilinear); with zero fluctuations it is |Y| e^T <C> e; it is symmetric; and it is stationary at the
    solution: E(u + eps v) - E(u) = eps^2 v^T K v exactly."""
    g = fem.Grid((4, 3, 4), "hex8_3d", "elastic")
    rng = np.random.default_rng(17)
    ids = rng.integers(0, 2, g.N)
    mod = [_rand_spd(6, 40, 1.0), _rand_spd(6, 41, 20.0)]
    loads = np.eye(6)
    r = solvers.homogenise(g, ids, mod, loads, method="sparse")
    vol = g.vp * g.N
    u = r["fields"]
    for i in range(6):
        for j in range(6):
            Eij = fem.energy(g, ids, mod, loads[i], u[i], loads[j], u[j])
            assert abs(Eij - vol * r["C_eff"][i, j]) < 1e-10 * vol * np.abs(r["C_eff"]).max()
            assert abs(Eij - fem.energy(g, ids, mod, loads[j], u[j], loads[i], u[i])) < 1e-12
    e = rng.standard_normal(6)
    z = np.zeros(g.c * g.N)
    em = e @ fem.mean_material(g, ids, mod) @ e
    assert abs(fem.energy(g, ids, mod, e, z, e, z) - vol * em) < 1e-12 * abs(em)
    K = fem.assemble_K(g, ids, mod)
    v = rng.standard_normal(g.c * g.N)
    for eps in (1e-3, 1e-1):
        d = fem.energy(g, ids, mod, loads[2], u[2] + eps * v, loads[2], u[2] + eps * v) \
            - fem.energy(g, ids, mod, loads[2], u[2], loads[2], u[2])
        assert abs(d - eps * eps * v @ (K @ v)) < 1e-9 * max(1.0, eps * eps * abs(v @ (K @ v)))


# ------------------------------------------------------------------------------------------------
# two-node stencil (Fig. 3 c): corner + centre node per pixel, four P1 triangles
# ------------------------------------------------------------------------------------------------
def test_two_node_stencil_element_patch_test():
    """Every triangle reproduces the gradient of a linear field sampled at its corner and centre
    nodes exactly; the four weights sum to the pixel area."""
    g = fem.Grid((3, 4), "p1tri4_2d", "scalar")
    a = np.array([0.7, -1.3])
    hx, hy = g.h
    pos = {0: (0, 0), 1: (hx, 0), 2: (0, hy), 3: (hx, hy), 4: (hx / 2, hy / 2)}
    ve = np.array([a @ np.array(pos[i]) for i in range(5)])
    qp = fem.quadrature(g)
    assert len(qp) == 4 and abs(sum(w for _, w in qp) - g.vp) < 1e-15
    for dN, w in qp:
        assert np.allclose(dN @ ve, a, atol=1e-12)


def test_two_node_stencil_operator_and_rhs():
    g = fem.Grid((4, 6), "p1tri4_2d", "scalar")
    rng = np.random.default_rng(31)
    ids = rng.integers(0, 2, g.N)
    mod = [_rand_spd(2, 60, 1.0), _rand_spd(2, 61, 8.0)]
    K = fem.assemble_K(g, ids, mod)
    assert K.shape == (2 * g.N, 2 * g.N)
    assert abs(K - K.T).max() < 1e-13
    assert np.abs(K @ np.ones(2 * g.N)).max() < 1e-12          # one null vector: the constants
    ev = np.linalg.eigvalsh(K.toarray())
    assert (ev < 1e-10 * ev.max()).sum() == 1
    # homogeneous material: the constant flux has zero divergence, b = 0
    Kh = fem.assemble_rhs(g, np.zeros(g.N, int), [mod[1]], np.array([1.0, -0.5]))
    assert np.abs(Kh).max() < 1e-13


def test_two_node_stencil_laminate_exact():
    g = fem.Grid((4, 8), "p1tri4_2d", "scalar")
    layer = (np.arange(8) >= 3).astype(int)
    ids = np.broadcast_to(layer, (4, 8)).ravel()
    k = [1.0, 9.0]
    mod = [kk * np.eye(2) for kk in k]
    r = solvers.homogenise(g, ids, mod, np.eye(2), method="sparse")
    f = np.array([3 / 8, 5 / 8])
    harm = 1.0 / (f[0] / k[0] + f[1] / k[1])
    arith = f[0] * k[0] + f[1] * k[1]
    assert abs(r["C_eff"][0, 0] - harm) < 1e-12 and abs(r["C_eff"][1, 1] - arith) < 1e-12
    assert abs(r["C_eff"][0, 1]) < 1e-12 and abs(r["C_eff"][1, 0]) < 1e-12


def test_two_node_stencil_symbol_and_pseudo_inverse():
    """Algorithm 2 on the two-node stencil: Hermitian 2 x 2 blocks; the k = 0 block has exactly one
    null eigenvalue (d N_n = 2 blocks, d = 1 rigid mode) and needs a true pseudo-inverse; every
    other block is invertible; with C_ref = C PCG converges in one iteration."""
    g = fem.Grid((6, 8), "p1tri4_2d", "scalar")
    C = _rand_spd(2, 62, 3.0)
    Kh = solvers.kref_symbol(g, C)
    blocks = np.moveaxis(Kh.reshape(2, 2, -1), 2, 0)
    assert np.abs(blocks - np.conj(np.swapaxes(blocks, 1, 2))).max() < 1e-12 * np.abs(blocks).max()
    assert np.abs(blocks[:, 0, 1].imag).max() > 1e-3 * np.abs(blocks).max()   # the centre coupling is complex
    ev0 = np.linalg.eigvalsh(blocks[0])
    assert abs(ev0[0]) < 1e-12 * np.abs(blocks).max() and ev0[1] > 1e-3 * np.abs(blocks).max()
    evs = np.linalg.eigvalsh(blocks[1:])
    assert evs.min() > 1e-6 * np.abs(blocks).max()
    Kinv = solvers.kref_pinv_symbol(Kh)
    P0 = Kinv[:, :, 0, 0] @ Kh[:, :, 0, 0]
    assert np.allclose(P0, np.array([[0.5, -0.5], [-0.5, 0.5]]), atol=1e-12)   # projector off the constants
    K = fem.assemble_K(g, np.zeros(g.N, int), [C])
    rng = np.random.default_rng(5)
    b = solvers.project_mean_zero(g, rng.standard_normal(2 * g.N))
    res = solvers.pcg(lambda v: K @ v, lambda v: solvers.apply_precond(g, Kinv, v), b, 1e-12)
    assert res["iters"] == 1


def test_lanczos_ritz_values_are_the_spectrum_after_n_steps():
    """Sec. 4.3 (Ritz values from the CG coefficients): on a tiny SPD system A with SPD preconditioner M,
    n = dim PCG steps span the whole space, so the eigenvalues of the CG-Lanczos tridiagonal matrix
    equal the generalised eigenvalues of (A, M), i.e. the spectrum of M^-1 A.  A beta_j in place of
    sqrt(beta_j) off the diagonal, or a dropped beta_{j-1} / alpha_{j-1} term, breaks the equality."""
    import scipy.linalg as sl
    n = 7
    rng = np.random.default_rng(17)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.linspace(1.0, 9.0, n) ** 1.3) @ Q.T          # well-separated spectrum
    M = _rand_spd(n, 18) / n
    Minv = np.linalg.inv(M)
    b = rng.standard_normal(n)
    res = solvers.pcg(lambda v: A @ v, lambda v: Minv @ v, b, tol=0.0, maxiter=n)
    assert res["iters"] == n
    ritz = np.sort(solvers.lanczos_ritz(res["alphas"], res["betas"]))
    exact = np.sort(sl.eigh(A, M, eigvals_only=True))
    assert np.abs(ritz - exact).max() <= 1e-10 * exact.max()
    # after fewer steps the Ritz values interlace inside the spectrum (Cauchy interlacing)
    ritz3 = solvers.lanczos_ritz(res["alphas"][:3], res["betas"][:3])
    assert exact.min() * (1 - 1e-12) <= ritz3.min() and ritz3.max() <= exact.max() * (1 + 1e-12)


def test_mean_material_of_the_disc_cell_is_exact():
    """Sec. 6.2 C_mean (volume mean) for the 32 x 32 disc cell: 284 of 1024 pixels have k = 10, the rest
    k = 1, so C_mean = (1 + 9 * 284 / 1024) I = 3.49609375 I exactly in binary floating point."""
    w = I.workload_circle2d_32()
    g = fem.Grid((32, 32), "p1tri2_2d", "scalar")
    assert int((w["ids"] == 1).sum()) == 284
    Cm = fem.mean_material(g, w["ids"].ravel(), w["moduli"])
    assert np.array_equal(Cm, 3.49609375 * np.eye(2))
    # and for an anisotropic pair on a 3-D grid: the voxel-fraction weighted sum of the phase tensors
    g3 = fem.Grid((4, 4, 4), "hex8_3d", "elastic")
    ids = np.zeros(64, np.int64)
    ids[:16] = 1
    mod = [_rand_spd(6, 1), _rand_spd(6, 2)]
    assert np.allclose(fem.mean_material(g3, ids, mod), 0.75 * mod[0] + 0.25 * mod[1], rtol=0, atol=1e-14)


def test_mean_material_is_a_volume_mean_on_any_cell():
    """Sec. 6.2 C_mean = (1/|Y|) sum_Q C(x_Q) w_Q: the same phase fractions on a scaled (non-unit) cell give
    the same C_mean (a sum without the 1/|Y| would scale it by the cell volume)."""
    rng = np.random.default_rng(3)
    ids = rng.integers(0, 2, 4 * 6 * 8)
    mod = [_rand_spd(6, 4), _rand_spd(6, 5)]
    g = fem.Grid((4, 6, 8), "hex8_3d", "elastic")
    unit = fem.mean_material(g, ids, mod)
    g.h = np.array([1.0, 0.7, 0.5]) / np.array(g.n_xyz, float)
    g.vp = float(np.prod(g.h))
    f1 = (ids == 1).mean()
    assert np.allclose(fem.mean_material(g, ids, mod), unit, rtol=1e-14, atol=0)
    assert np.allclose(unit, (1 - f1) * mod[0] + f1 * mod[1], rtol=1e-14, atol=0)
