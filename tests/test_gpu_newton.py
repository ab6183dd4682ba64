"""Newton's method of Algorithm 1 on the GPU (power-law conductivity, per-Gauss-point tangents,
preconditioner reassembled every step) against the FP64 Newton oracle (oracle/newton.py)."""
import numpy as np
import pytest

from oracle import fem, newton as NW
from paper_2203_02962_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _solver(shape, ids, k):
    from paper_2203_02962_gb300 import fehom
    mod = np.stack([I.isotropic_conductivity(kk, 3) for kk in k])
    return fehom.Solver("hex8_3d", "scalar", tuple(shape[::-1]), ids, mod)


@pytest.mark.parametrize("shape,seed", [((8, 8, 8), 0), ((6, 12, 16), 1)])
def test_newton_matches_oracle(shape, seed):
    rng = np.random.default_rng(seed)
    ids = (rng.random(shape) < 0.35).astype(np.uint8)
    k, n, g0, e = [1.0, 10.0], [1.5, 0.6], 0.5, [1.0, 0.5, -0.25]
    g = fem.Grid(shape, "hex8_3d", "scalar")
    u_ref, q_ref, hist = NW.newton(g, ids.ravel(), k, n, g0, e, eta=1e-10)
    s = _solver(shape, ids, k)
    out = s.newton_solve(e, n, g0, tol_cg=1e-13, eta=1e-10)
    assert out["converged"]
    assert abs(out["newton_iterations"] - len(hist)) <= 1, (out["increment"], hist)
    u = out["fields"].cpu().numpy()
    u_ref = u_ref - u_ref.mean()
    assert np.abs(u - u_ref).max() <= 1e-9 * np.abs(u_ref).max()
    assert np.abs(out["mean_flux"] - q_ref).max() <= 1e-11 * np.abs(q_ref).max()
    s.close()


def test_newton_linear_law_matches_the_linear_solve():
    shape = (8, 8, 8)
    ids = I.spheres3d(8, count=4, rmin=1.0, rmax=2.0, seed=3)
    k = [1.0, 30.0]
    s = _solver(shape, ids, k)
    out = s.newton_solve([0.0, 1.0, 0.0], [1.0, 1.0], 0.5, tol_cg=1e-13, eta=1e-10)
    s.precond_build()
    lin = s.solve(np.array([[0.0, 1.0, 0.0]]), tol=1e-13)
    assert out["newton_iterations"] == 2 and out["increment"][1] < 1e-10
    assert np.abs(out["mean_flux"] - lin["mean_flux"][0]).max() < 1e-11
    assert np.abs(out["fields"].cpu().numpy() - lin["fields"][0, 0].cpu().numpy()).max() < 1e-10
    s.close()


def test_newton_laminate_is_exact():
    shape = (2, 2, 8)
    ids = np.broadcast_to((np.arange(8) >= 3).astype(np.uint8), shape).copy()
    k, n, g0 = [1.0, 10.0], [1.5, 0.6], 0.5
    s = _solver(shape, ids, k)
    for E in (0.3, -2.0):
        out = s.newton_solve([E, 0.0, 0.0], n, g0, tol_cg=1e-13, eta=1e-11)
        ref = NW.laminate_flux(k, n, g0, [3 / 8, 5 / 8], E)
        assert abs(out["mean_flux"][0] - ref) < 1e-10 * abs(ref)
    s.close()


def test_newton_converges_quadratically_and_reassembles_the_reference():
    shape = (16, 16, 16)
    ids = I.spheres3d(16, count=8, rmin=1.5, rmax=3.0, seed=5)
    s = _solver(shape, ids, [1.0, 20.0])
    out = s.newton_solve([1.0, 0.5, 0.0], [1.6, 0.5], 0.4, tol_cg=1e-12, eta=1e-12)
    r = out["increment"]
    assert out["converged"] and r[-1] <= 1e-12
    tail = [(a, b) for a, b in zip(r[1:], r[2:]) if a < 1e-2 and b > 1e-14]
    assert tail and all(b <= 10.0 * a * a for a, b in tail), r
    assert all(p > 0 for p in out["pcg_per_step"])
    s.close()


def test_set_reference_changes_speed_not_answer():
    shape = (16, 16, 16)
    ids = I.spheres3d(16, count=8, rmin=1.5, rmax=3.0, seed=6)
    s = _solver(shape, ids, [1.0, 50.0])
    s.precond_build()
    a = s.solve(np.eye(3), tol=1e-12)
    s.set_reference(np.diag([1.0, 5.0, 20.0]))  # anisotropic: not a multiple of C_mean (a multiple would not change PCG)
    b = s.solve(np.eye(3), tol=1e-12, raise_on_failure=False)
    assert b["status"] == 7  # FEHOM_E_STATE: the preconditioner must be rebuilt first
    s.precond_build()
    b = s.solve(np.eye(3), tol=1e-12)
    assert np.abs(a["C_eff"] - b["C_eff"]).max() < 1e-9 * np.abs(a["C_eff"]).max()
    assert [i["iterations"] for i in a["info"]] != [i["iterations"] for i in b["info"]]
    s.close()
