"""Oracle, part 4: Newton's method of Algorithm 1 for a nonlinear conductivity, FP64 on the CPU.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, links or calls this module; only
``tests/`` does.  It shares no code with the CUDA kernels.

* Sec. 3, nonlinear system: R(u) = D^T W q(e + D u) = 0 for the fluctuation u, with the flux q of
  the per-quadrature-point gradient g = e + D u (the scalar form of App. A).
* Sec. 3.1, Eq. lin_system: the Newton step solves K_t delta = -R with the tangent
  K_t = D^T W A D, A = dq/dg at every quadrature point.
* Algorithm 1: u_0 = 0; per step: flux and tangent, reference material = volume mean of the
  tangent (Sec. 6.2 C_mean, reassembled whenever the tangent changes), linear solve, update, and the
  Newton test ||D delta|| <= eta ||D u|| (Sec. 6, termination criteria).
* The law (the paper's own nonlinear law is defined in another paper, so any smooth monotone law
  serves): per phase p a regularised power law
      q(g) = k_p s^((n_p - 1) / 2) g,   s = 1 + |g|^2 / g0^2,
      A(g) = k_p s^((n_p - 1) / 2) (I + (n_p - 1) g g^T / (g0^2 s)),
  linear (q = k_p g) for n_p = 1.
Pinned by tests/test_oracle_pins_newton.py: the tangent against central differences of the flux and
of the residual, the linear case against the linear solve, a grid-aligned laminate against the exact
one-dimensional solution, and the quadratic convergence of the Newton increments.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem, solvers


def flux_tangent(g, k, n, g0):
    """q (..., d) and A (..., d, d) of the power law for gradients g (..., d); k and n broadcast
    against the leading axes of g."""
    g = np.asarray(g, float)
    k, n = np.asarray(k, float), np.asarray(n, float)
    s = 1.0 + (g * g).sum(axis=-1) / (g0 * g0)
    f = k * s ** ((n - 1.0) / 2.0)
    q = f[..., None] * g
    d = g.shape[-1]
    c = (n - 1.0) / (g0 * g0 * s)
    A = f[..., None, None] * (np.eye(d) + c[..., None, None] * g[..., :, None] * g[..., None, :])
    return q, A


def _per_voxel(phases, vals):
    return np.asarray(vals, float)[np.asarray(phases).ravel()]


def residual_tangent(grid: fem.Grid, phases, k, n, g0, e, u):
    """R(u) (c N), K_t (CSR), volume mean flux (d) and volume mean tangent (d x d)."""
    assert grid.physics == "scalar"
    kv, nv = _per_voxel(phases, k), _per_voxel(phases, n)
    dofs = grid.element_dofs()
    ue = u[dofs]
    nd = grid.c * grid.N
    R = np.zeros(nd)
    kdim = dofs.shape[1]
    Ke = np.zeros((dofs.shape[0], kdim, kdim))
    qsum = np.zeros(grid.m)
    Asum = np.zeros((grid.m, grid.m))
    for B, w in fem.element_B(grid):
        g = np.asarray(e, float)[None, :] + ue @ B.T                   # (N_e, d)
        q, A = flux_tangent(g, kv, nv, g0)
        np.add.at(R, dofs, w * q @ B)
        Ke += w * np.einsum("ia,nij,jb->nab", B, A, B)
        qsum += w * q.sum(axis=0)
        Asum += w * A.sum(axis=0)
    rows = np.repeat(dofs, kdim, axis=1).ravel()
    cols = np.tile(dofs, (1, kdim)).ravel()
    Kt = sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(nd, nd)).tocsr()
    vol = grid.vp * grid.N
    return R, Kt, qsum / vol, Asum / vol


def grad_norm2(grid: fem.Grid, u):
    """sum_Q w_Q |(D u)_Q|^2."""
    ue = u[grid.element_dofs()]
    return float(sum(w * ((ue @ B.T) ** 2).sum() for B, w in fem.element_B(grid)))


def newton(grid: fem.Grid, phases, k, n, g0, e, eta=1e-10, max_newton=30):
    """Algorithm 1 with exact (sparse direct, mean-zero) linear solves.

    Returns (u, mean flux, history) with history = [(||R_k||, ||D delta_k|| / ||D u_{k+1}||), ...]."""
    u = np.zeros(grid.c * grid.N)
    hist = []
    for _ in range(max_newton):
        R, Kt, _, _ = residual_tangent(grid, phases, k, n, g0, e, u)
        delta = solvers.solve_sparse(grid, Kt, -R)
        u = u + delta
        gu = grad_norm2(grid, u)
        ratio = np.sqrt(grad_norm2(grid, delta) / gu) if gu > 0 else 0.0
        hist.append((float(np.linalg.norm(R)), float(ratio)))
        if ratio <= eta:
            break
    _, _, qbar, _ = residual_tangent(grid, phases, k, n, g0, e, u)
    return u, qbar, hist


def laminate_flux(k, n, g0, fractions, E):
    """Exact mean flux of a laminate normal to x1 under the mean gradient (E, 0, 0): the layer
    gradients g_p (along x1) share one flux, q_p(g_p) = Q, and average to E.  Each q_p is strictly
    increasing in g, so Q follows from bisection on sum_p f_p g_p(Q) = E."""
    def g_of(Q, p):
        lo, hi = 0.0, 1.0
        f = lambda g: k[p] * (1 + g * g / (g0 * g0)) ** ((n[p] - 1) / 2) * g - abs(Q)
        while f(hi) < 0:
            hi *= 2.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if f(mid) < 0 else (lo, mid)
        return np.sign(Q) * 0.5 * (lo + hi)

    lo, hi = 0.0, 1.0
    while sum(fp * g_of(hi, p) for p, fp in enumerate(fractions)) < abs(E):
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if sum(fp * g_of(mid, p) for p, fp in enumerate(fractions)) < abs(E):
            lo = mid
        else:
            hi = mid
    return np.sign(E) * 0.5 * (lo + hi)
