"""Pins of the Newton oracle (oracle/newton.py, Algorithm 1 with a power-law conductivity): the
tangent against central differences, the linear limit against the linear solve, a grid-aligned
laminate against the exact one-dimensional solution, and quadratic convergence."""
import numpy as np

from oracle import fem, newton as NW, solvers


def test_flux_tangent_is_the_derivative_of_the_flux():
    rng = np.random.default_rng(0)
    g = rng.standard_normal((20, 3))
    k, n, g0 = 3.0, 0.6, 0.7
    _, A = NW.flux_tangent(g, k, n, g0)
    h = 1e-6
    for i in range(3):
        dg = np.zeros(3)
        dg[i] = h
        fd = (NW.flux_tangent(g + dg, k, n, g0)[0] - NW.flux_tangent(g - dg, k, n, g0)[0]) / (2 * h)
        assert np.abs(fd - A[:, :, i]).max() < 1e-7 * np.abs(A).max()
    assert np.abs(A - np.swapaxes(A, 1, 2)).max() < 1e-14
    q1, A1 = NW.flux_tangent(g, 2.5, 1.0, g0)      # n = 1: linear law
    assert np.allclose(q1, 2.5 * g) and np.allclose(A1, 2.5 * np.eye(3))


def test_residual_tangent_matches_central_differences():
    g = fem.Grid((3, 4, 4), "hex8_3d", "scalar")
    rng = np.random.default_rng(1)
    ids = rng.integers(0, 2, g.N)
    k, n, g0, e = [1.0, 5.0], [1.4, 0.6], 0.5, [0.7, -0.3, 0.2]
    u = 0.1 * rng.standard_normal(g.N)
    v = rng.standard_normal(g.N)
    _, Kt, _, _ = NW.residual_tangent(g, ids, k, n, g0, e, u)
    h = 1e-6
    fd = (NW.residual_tangent(g, ids, k, n, g0, e, u + h * v)[0]
          - NW.residual_tangent(g, ids, k, n, g0, e, u - h * v)[0]) / (2 * h)
    assert np.abs(fd - Kt @ v).max() < 1e-7 * np.abs(Kt @ v).max()
    assert abs((Kt - Kt.T)).max() < 1e-12


def test_linear_law_takes_one_newton_step_to_the_linear_solution():
    g = fem.Grid((4, 4, 4), "hex8_3d", "scalar")
    rng = np.random.default_rng(2)
    ids = rng.integers(0, 2, g.N)
    k = [1.0, 7.0]
    e = np.array([1.0, 0.0, 0.0])
    u, q, hist = NW.newton(g, ids, k, [1.0, 1.0], 0.5, e)
    lin = solvers.homogenise(g, ids, [ki * np.eye(3) for ki in k], e[None], method="sparse")
    assert np.abs(u - lin["fields"][0]).max() < 1e-12
    assert np.abs(q - lin["mean_flux"][0]).max() < 1e-12
    assert len(hist) == 2 and hist[1][1] < 1e-12


def test_laminate_matches_the_exact_one_dimensional_solution():
    g = fem.Grid((2, 2, 8), "hex8_3d", "scalar")
    ids = np.broadcast_to((np.arange(8) >= 3).astype(int), (2, 2, 8)).ravel()   # 3/8 phase 0, 5/8 phase 1
    k, n, g0 = [1.0, 10.0], [1.5, 0.6], 0.5
    for E in (0.3, 1.0, -2.0):
        _, q, _ = NW.newton(g, ids, k, n, g0, [E, 0.0, 0.0])
        ref = NW.laminate_flux(k, n, g0, [3 / 8, 5 / 8], E)
        assert abs(q[0] - ref) < 1e-10 * abs(ref) and abs(q[1]) < 1e-12 and abs(q[2]) < 1e-12


def test_newton_converges_quadratically():
    g = fem.Grid((6, 6, 6), "hex8_3d", "scalar")
    rng = np.random.default_rng(3)
    ids = (rng.random(g.N) < 0.3).astype(int)
    _, _, hist = NW.newton(g, ids, [1.0, 20.0], [1.6, 0.5], 0.4, [1.0, 0.5, 0.0], eta=1e-13)
    r = [h[1] for h in hist]
    assert r[-1] <= 1e-13
    # once in the basin, each increment ratio is bounded by a constant times the square of the previous
    tail = [(a, b) for a, b in zip(r[1:], r[2:]) if a < 1e-2 and b > 1e-15]
    assert tail and all(b <= 10.0 * a * a for a, b in tail), r
