"""The oracle's C/OpenMP CG (oracle/csr_cg.c) against the numpy CG it restates and against direct solves.

The C version exists to time the oracle on all host cores; here it must take the same iterations as
``solvers.cg`` and reach the same mean-zero solution of K u = b (Sec. 3.1, Eq. lin_system) as the
sparse direct solve, with one thread and with several.  No GPU.
"""
import numpy as np
import pytest

from oracle import cg_native, fem, solvers
from paper_2203_02962_gb300 import inputs as I


@pytest.fixture(scope="module")
def lib():
    try:
        cg_native.build()
    except RuntimeError as e:  # pragma: no cover - no C compiler
        pytest.skip(str(e))
    return cg_native


@pytest.mark.parametrize("threads", [1, 3])
def test_native_cg_matches_numpy_cg_and_direct_solve(lib, threads):
    shape = (6, 8, 10)
    g = fem.Grid(shape, "hex8_3d", "elastic")
    rng = np.random.default_rng(4)
    ids = rng.integers(0, 2, g.N)
    mod = [I.isotropic_elastic_mandel(1.0, 0.3), I.isotropic_elastic_mandel(30.0, 0.2)]
    K = fem.assemble_K(g, ids, mod)
    b = fem.assemble_rhs(g, ids, mod, np.eye(6)[3])
    x_py, it_py, rel_py = solvers.cg(K, b, tol=1e-12)
    x_c, it_c, rel_c = lib.cg(K, b, tol=1e-12, threads=threads)
    assert abs(it_c - it_py) <= 1 and rel_c <= 1e-12
    u_ref = solvers.solve_sparse(g, K, b)
    u_c = solvers.project_mean_zero(g, x_c)
    assert np.abs(u_c - u_ref).max() <= 1e-9 * np.abs(u_ref).max()
    assert np.abs(solvers.project_mean_zero(g, x_py) - u_c).max() <= 1e-9 * np.abs(u_ref).max()


def test_native_cg_scalar_disc_and_zero_rhs(lib):
    w = I.workload_circle2d_32()
    g = fem.Grid((32, 32), "p1tri2_2d", "scalar")
    K = fem.assemble_K(g, w["ids"].ravel(), w["moduli"])
    ref = solvers.homogenise(g, w["ids"].ravel(), w["moduli"], w["loads"], method="sparse")
    for l, e in enumerate(w["loads"]):
        b = fem.assemble_rhs(g, w["ids"].ravel(), w["moduli"], e)
        x, it, rel = lib.cg(K, b, tol=1e-13)
        assert rel <= 1e-13 and it > 0
        assert np.abs(solvers.project_mean_zero(g, x) - ref["fields"][l]).max() <= 1e-10
    x, it, rel = lib.cg(K, np.zeros(g.N), tol=1e-8)
    assert it == 0 and rel == 0.0 and not x.any()
