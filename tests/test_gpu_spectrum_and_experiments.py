"""GPU checks of the spectral diagnostics (Sec. 4.3) and of the coated-sphere experiment (Sec. 6.2).

* fehom_eig_bounds against the oracle's element-by-element bounds (exact counts, values to 1e-12).
* The Ritz values of the GPU PCG (CG-Lanczos tridiagonal from fehom_pcg_coefficients) lie inside the
  bounds, as Sec. 4.3 guarantees for the spectrum of K_ref^+ K.
* The coated sphere: the volume-mean reference material needs no more PCG iterations than I_s, and
  the counts stay flat under grid refinement at fixed contrast (Sec. 6.2, Fig. 9 trends).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import fem, solvers  # noqa: E402
from paper_2203_02962_gb300 import inputs as I  # noqa: E402


def _solver(elem, physics, shape, ids, moduli, **kw):
    from paper_2203_02962_gb300 import fehom
    return fehom.Solver(elem, physics, tuple(shape[::-1]), ids, moduli, **kw)


@pytest.mark.parametrize("elem,physics,shape", [("hex8_3d", "elastic", (8, 12, 16)), ("p1tri2_2d", "scalar", (24, 32)),
                                                 ("hex8_3d", "scalar", (6, 8, 12))])
def test_eig_bounds_match_oracle(elem, physics, shape):
    g = fem.Grid(shape, elem, physics)
    rng = np.random.default_rng(21)
    ids = rng.integers(0, 3, size=shape).astype(np.uint8)
    if physics == "elastic":
        mod = np.stack([I.isotropic_elastic_mandel(E, nu, g.dim) for E, nu in ((1, 0.3), (40, 0.2), (6, 0.45))])
    else:
        mod = np.stack([k * np.eye(g.dim) for k in (1.0, 40.0, 6.0)])
    s = _solver(elem, physics, shape, ids, mod)
    lo, hi = s.eig_bounds()
    lo_ref, hi_ref = solvers.eig_bounds(g, ids.ravel(), mod, fem.mean_material(g, ids.ravel(), mod))
    assert lo.shape == lo_ref.shape and hi.shape == hi_ref.shape
    assert np.abs(lo - lo_ref).max() <= 1e-12 * hi_ref.max()
    assert np.abs(hi - hi_ref).max() <= 1e-12 * hi_ref.max()
    s.close()


def test_ritz_values_inside_bounds():
    n = 32
    ids = I.spheres3d(n, count=20, rmin=2.0, rmax=5.0, seed=5)
    mod = np.stack([I.isotropic_elastic_mandel(1.0, 0.3), I.isotropic_elastic_mandel(50.0, 0.2)])
    s = _solver("hex8_3d", "elastic", (n, n, n), ids, mod)
    s.precond_build()
    out = s.solve(np.eye(6)[:1], tol=1e-8)
    a, b = s.pcg_coefficients(0)
    assert len(a) == out["info"][0]["iterations"] and len(a) > 5
    ritz = solvers.lanczos_ritz(a, b)
    lo, hi = s.eig_bounds()
    assert ritz.min() >= lo.min() * (1 - 1e-8) and ritz.max() <= hi.max() * (1 + 1e-8)
    s.close()


def test_coated_sphere_reference_material_and_refinement():
    from paper_2203_02962_gb300 import coated_sphere
    rows = coated_sphere.run(sizes=[16, 32, 64], contrasts=[1e-2, 1e2], tol=1e-6)
    it = {(r["n"], r["rho"], r["ref"]): r["iterations"] for r in rows}
    assert all(r["converged"] for r in rows)
    for n in (16, 32, 64):
        for rho in (1e-2, 1e2):
            assert it[(n, rho, "C_mean")] <= it[(n, rho, "I_s")], it
    for rho in (1e-2, 1e2):
        assert it[(64, rho, "C_mean")] <= 1.3 * it[(32, rho, "C_mean")], it
