"""Oracle, part 2: the reference-material preconditioner and the linear solvers, FP64 on the CPU.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, links or calls this module; only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` do.

* Sec. 4.1, Eq. Kref: K_ref = D^T W C_ref D with spatially uniform C_ref.
* Sec. 5.2, Algorithm 2 and Fig. 5: for each DOF type beta, apply K_ref to the unit impulse at the
  first node of that type, giving the first columns of the blocks K_ref[alpha, beta]; their
  d-dimensional DFTs are the diagonals of the Fourier blocks.  Sec. 5.3, Eq. block_inversion: the
  c x c blocks are inverted one wavevector at a time, with the Moore-Penrose pseudo-inverse at the
  zero frequency.  DFT convention (a reading of the paper): unnormalised forward transform
  exp(-2 pi i k.x / n), inverse with 1/N, so that the block eigenvalues are the DFT of the first
  column (numpy.fft conventions).
* Sec. 4.2, Eq. M_inverse: K_ref^+ r = F^-1 [K_hat^+ (F r)] per component block.
* Sec. 4.1 with Saad's preconditioned CG (the symmetric PCG the paper solves): plain PCG, and
  the unpreconditioned CG the oracle uses to solve K u = b.  The stopping test is the paper's
  relative K_ref^-1-norm of the residual (Sec. 6, termination criteria), normalised by the
  right-hand side b (the same as r_0 for a zero initial guess).
* Uniqueness reading: K has the constants per component in its kernel, so the solution is the
  mean-zero one; the dense solve uses the bordered system [K Z; Z^T 0].
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem


# ----------------------------------------------------------------------------------------------
# Algorithm 2: Fourier blocks of K_ref and their (pseudo-)inverses
# ----------------------------------------------------------------------------------------------
def kref_symbol(grid: fem.Grid, C_ref):
    """K_hat[alpha, beta](k) for every wavevector: array (c, c, *grid.shape), complex.

    Follows Algorithm 2: impulse -> matrix-free-equivalent action of K_ref (here the assembled
    K_ref) -> DFT of each component block of the result.
    """
    Kref = fem.assemble_K(grid, np.zeros(grid.N, dtype=np.int64), [np.asarray(C_ref, float)])
    c, N = grid.c, grid.N
    out = np.empty((c, c) + grid.shape, dtype=np.complex128)
    for beta in range(c):
        imp = np.zeros(c * N)
        imp[beta * N] = 1.0                          # p = (beta - 1) N_p + 1 in 1-based indexing
        col = Kref @ imp                             # p-th column of K_ref
        for alpha in range(c):
            blk = col[alpha * N:(alpha + 1) * N].reshape(grid.shape)
            out[alpha, beta] = np.fft.fftn(blk)
    return out


def kref_pinv_symbol(K_hat, rel_tol=1e-12):
    """Per-wavevector inverse of the c x c blocks; Moore-Penrose pseudo-inverse at k = 0.

    The zero-frequency block carries the d rigid-body null eigenvalues (Sec. 5.3).  Its singular
    values are cut relative to the largest block norm over all wavevectors (``rel_tol``), not
    relative to the block itself: for the one-node stencils the block is zero up to rounding and
    a block-relative cut would invert that rounding noise.
    """
    c = K_hat.shape[0]
    shape = K_hat.shape[2:]
    blocks = np.moveaxis(K_hat.reshape(c, c, -1), 2, 0)          # (Np, c, c)
    inv = np.empty_like(blocks)
    inv[1:] = np.linalg.inv(blocks[1:])
    scale = np.abs(blocks).max()
    U, s, Vh = np.linalg.svd(blocks[0])
    keep = s > rel_tol * scale
    inv[0] = (Vh[keep].conj().T / s[keep]) @ U[:, keep].conj().T
    return np.moveaxis(inv, 0, 2).reshape((c, c) + shape)


def apply_precond(grid: fem.Grid, K_inv_hat, r):
    """z = K_ref^+ r = F^-1 K_hat^+ F r (Eq. M_inverse), r and z of length c * N."""
    c, N = grid.c, grid.N
    rh = np.stack([np.fft.fftn(r[a * N:(a + 1) * N].reshape(grid.shape)) for a in range(c)])
    zh = np.einsum("ab...,b...->a...", K_inv_hat, rh)
    return np.concatenate([np.fft.ifftn(zh[a]).real.ravel() for a in range(c)])


# ----------------------------------------------------------------------------------------------
# linear solvers
# ----------------------------------------------------------------------------------------------
def constant_modes(grid: fem.Grid):
    """Z: indicator columns of the constants per physical component (kernel of K): (c N, c), or for
    the two-node stencil the single column of ones (every node of the field at the same value)."""
    if getattr(grid, "nn", 1) == 2:
        return np.ones((grid.c * grid.N, 1))
    Z = np.zeros((grid.c * grid.N, grid.c))
    for j in range(grid.c):
        Z[j * grid.N:(j + 1) * grid.N, j] = 1.0
    return Z


def project_mean_zero(grid: fem.Grid, u):
    u = np.array(u, dtype=float, copy=True)
    if getattr(grid, "nn", 1) == 2:
        return u - u.mean()
    for j in range(grid.c):
        u[j * grid.N:(j + 1) * grid.N] -= u[j * grid.N:(j + 1) * grid.N].mean()
    return u


def solve_dense(grid: fem.Grid, K, b):
    """Mean-zero solution of K u = b from the dense bordered system (tiny grids only)."""
    Kd = K.toarray() if sp.issparse(K) else np.asarray(K)
    Z = constant_modes(grid)
    n, c = Kd.shape[0], Z.shape[1]
    A = np.zeros((n + c, n + c))
    A[:n, :n], A[:n, n:], A[n:, :n] = Kd, Z, Z.T
    rhs = np.concatenate([b, np.zeros(c)])
    return np.linalg.solve(A, rhs)[:n]


def solve_sparse(grid: fem.Grid, K, b):
    """Mean-zero solution of K u = b from the sparse bordered system (sparse LU)."""
    import scipy.sparse.linalg as spla
    Z = sp.csr_matrix(constant_modes(grid))
    A = sp.bmat([[K, Z], [Z.T, None]], format="csc")
    rhs = np.concatenate([b, np.zeros(Z.shape[1])])
    return spla.spsolve(A, rhs)[: K.shape[0]]


def cg(K, b, tol=1e-14, maxiter=100000, x0=None):
    """Unpreconditioned CG on K u = b; stops when ||r||_2 <= tol ||b||_2 or on stagnation.

    Returns (x, iterations, final relative residual).
    """
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=float)
    r = b - K @ x
    p = r.copy()
    rr = r @ r
    bb = b @ b
    if bb == 0.0:
        return x, 0, 0.0
    best, stall = np.inf, 0
    it = 0
    while it < maxiter:
        if np.sqrt(rr / bb) <= tol:
            break
        Kp = K @ p
        alpha = rr / (p @ Kp)
        x += alpha * p
        r -= alpha * Kp
        rr_new = r @ r
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
        rel = np.sqrt(rr / bb)
        if rel < 0.5 * best:
            best, stall = rel, 0
        else:
            stall += 1
            if stall > 2000:
                break
    return x, it, float(np.sqrt(rr / bb))


def pcg(K_apply, M_apply, b, tol, maxiter=10000, x0=None):
    """Preconditioned CG (symmetric form, Saad Sec. 9.2.1) with the paper's K_ref^-1-norm test.

    Stops when sqrt(<r, z>) <= tol * sqrt(<b, M^-1 b>), z = M^-1 r.  Returns a dict with the
    solution, the iteration count, the sqrt(<r,z>)/sqrt(<b,M^-1 b>) history and the CG
    coefficients alpha_j, beta_j (for the Lanczos/Ritz check).
    """
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=float)
    r = b - K_apply(x) if x0 is not None else b.copy()
    z = M_apply(r)
    p = z.copy()
    rz = r @ z
    zb = M_apply(b)
    bnorm = np.sqrt(b @ zb)
    hist, alphas, betas = [np.sqrt(max(rz, 0.0)) / bnorm if bnorm > 0 else 0.0], [], []
    it = 0
    while it < maxiter and bnorm > 0 and np.sqrt(max(rz, 0.0)) > tol * bnorm:
        Ap = K_apply(p)
        alpha = rz / (p @ Ap)
        x = x + alpha * p
        r = r - alpha * Ap
        z = M_apply(r)
        rz_new = r @ z
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
        it += 1
        alphas.append(alpha)
        betas.append(beta)
        hist.append(np.sqrt(max(rz, 0.0)) / bnorm)
    return dict(x=x, iters=it, hist=np.array(hist), alphas=np.array(alphas), betas=np.array(betas),
                bnorm=bnorm)


def lanczos_ritz(alphas, betas):
    """Eigenvalues of the CG-Lanczos tridiagonal matrix built from the PCG coefficients."""
    k = len(alphas)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    return np.linalg.eigvalsh(T)


# ----------------------------------------------------------------------------------------------
# homogenisation driver
# ----------------------------------------------------------------------------------------------
def homogenise(grid: fem.Grid, phases, moduli, loads, method="cg", tol=1e-14, C_ref=None,
               maxiter=100000):
    """Solve the cell problem for each load row of ``loads`` and return fields, <sigma>, C_eff.

    method: "dense" (bordered dense solve), "sparse" (bordered sparse LU), "cg" (unpreconditioned
    CG to ``tol``) or "pcg" (reference-material PCG to ``tol``).  C_eff = S E^-1 with the mean
    fluxes S and loads E as columns (only when E is square and invertible).
    """
    moduli = np.asarray(moduli, float)
    loads = np.atleast_2d(np.asarray(loads, float))
    K = fem.assemble_K(grid, phases, moduli)
    if method == "pcg":
        C_ref = fem.mean_material(grid, phases, moduli) if C_ref is None else np.asarray(C_ref)
        Kinv = kref_pinv_symbol(kref_symbol(grid, C_ref))
    fields, fluxes, iters = [], [], []
    for e in loads:
        b = fem.assemble_rhs(grid, phases, moduli, e)
        if method == "dense":
            u, it = solve_dense(grid, K, b), 0
        elif method == "sparse":
            u, it = solve_sparse(grid, K, b), 0
        elif method == "cg":
            u, it, _ = cg(K, b, tol=tol, maxiter=maxiter)
        elif method == "pcg":
            res = pcg(lambda v: K @ v, lambda v: apply_precond(grid, Kinv, v), b, tol, maxiter)
            u, it = res["x"], res["iters"]
        else:
            raise ValueError(method)
        u = project_mean_zero(grid, u)
        fields.append(u)
        fluxes.append(fem.mean_flux(grid, phases, moduli, e, u))
        iters.append(it)
    S = np.array(fluxes).T
    C_eff = S @ np.linalg.inv(loads.T) if loads.shape[0] == loads.shape[1] else None
    return dict(fields=np.array(fields), mean_flux=np.array(fluxes), C_eff=C_eff, iters=iters)


# ----------------------------------------------------------------------------------------------
# Sec. 4.3: element-by-element eigenvalue bounds of K_ref^-1 K
# ----------------------------------------------------------------------------------------------
def eig_bounds(grid: fem.Grid, phases, moduli, C_ref):
    """Sorted lower and upper bound sequences (length c N) of the eigenvalues of K_ref^-1 K.

    For each node I: lambda_I^L / lambda_I^U = min / max over the voxels in supp(phi_I) of the
    extreme generalized eigenvalues of (C_e, C_ref) (constant material per voxel, so one pair per
    voxel); each value counted once per DOF of the node (d times for elasticity) and sorted.
    """
    import scipy.linalg as sl
    phases = np.asarray(phases).ravel()
    lam = [sl.eigh(np.asarray(C, float), np.asarray(C_ref, float), eigvals_only=True) for C in moduli]
    lo_p = np.array([l.min() for l in lam])
    hi_p = np.array([l.max() for l in lam])
    en = grid.element_nodes()
    node_lo = np.full(grid.N, np.inf)
    node_hi = np.full(grid.N, -np.inf)
    for a in range(grid.ne):
        np.minimum.at(node_lo, en[:, a], lo_p[phases])
        np.maximum.at(node_hi, en[:, a], hi_p[phases])
    return np.sort(np.repeat(node_lo, grid.c)), np.sort(np.repeat(node_hi, grid.c))
