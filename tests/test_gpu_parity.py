"""Parity of the CUDA path (called through the C ABI) with the FP64 CPU oracle.

Operator level: stiffness apply (S1/S3), right-hand side (S2), Algorithm 2 symbol (S4), the FFT
preconditioner (S5-S7), volume averages (S9), on grids that span several tiles with ragged tails.
Solve level (S8 + everything): C_eff and fields against the oracle's direct solve, iteration counts
against the oracle's PCG, batched vs one-by-one loads, mixed vs FP64.  Error paths return status
codes.  Tolerances: FP64 operators 1e-12 relative to the largest entry; FP32 operators 2e-5;
solves at tol 1e-12: C_eff 1e-10 relative, fields 1e-9 relative max-norm.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import fem, solvers  # noqa: E402
from paper_2203_02962_gb300 import inputs as I  # noqa: E402


def _torch():
    import torch
    return torch


def _fehom():
    from paper_2203_02962_gb300 import fehom
    return fehom


def _rand_spd(m, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, m))
    return scale * (A @ A.T + m * np.eye(m))


def _solver(elem, physics, shape, ids, moduli, **kw):
    return _fehom().Solver(elem, physics, tuple(shape[::-1]), ids, moduli, **kw)


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


OPERATOR_CASES = [
    # elem, physics, shape (z, y, x) or (y, x), materials, cell
    ("hex8_3d", "elastic", (12, 6, 48), "aniso", None),
    ("hex8_3d", "elastic", (12, 12, 48), "iso", (4.0, 1.0, 1.0)),     # cubic voxels -> isotropic fast path
    ("hex8_3d", "elastic", (24, 24, 24), "iso", None),
    ("hex8_3d", "scalar", (6, 12, 48), "aniso", None),
    ("hex8_3d", "scalar", (8, 8, 8), "iso", None),
    ("p1tri2_2d", "scalar", (24, 48), "aniso", None),
    ("p1tri2_2d", "elastic", (12, 96), "aniso", None),
    ("q1_2d", "scalar", (16, 48), "iso", None),
    ("q1_2d", "elastic", (6, 64), "aniso", None),
]


def _materials(physics, dim, kind, seed=0):
    m = dim if physics == "scalar" else dim * (dim + 1) // 2
    if kind == "aniso":
        return np.stack([_rand_spd(m, seed + p, 10.0 ** p) for p in range(3)])
    if physics == "scalar":
        return np.stack([I.isotropic_conductivity(k, dim) for k in (1.0, 30.0, 1000.0)])
    return np.stack([I.isotropic_elastic_mandel(E, nu, dim) for E, nu in ((1.0, 0.3), (100.0, 0.2), (7.0, 0.45))])


@pytest.mark.parametrize("elem,physics,shape,kind,cell", OPERATOR_CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_stiffness_apply(elem, physics, shape, kind, cell, precision):
    torch = _torch()
    g = fem.Grid(shape, elem, physics)
    if cell is not None:  # the oracle's grid is the unit cell: scale h by hand
        g.h = np.array(cell, float)[: g.dim] / np.array(g.n_xyz, float)
        g.vp = float(np.prod(g.h))
    rng = np.random.default_rng(1)
    ids = rng.integers(0, 3, size=shape).astype(np.uint8)
    mod = _materials(physics, g.dim, kind)
    K = fem.assemble_K(g, ids.ravel(), mod)
    x = rng.standard_normal(g.c * g.N)
    y_ref = K @ x
    s = _solver(elem, physics, shape, ids, mod, cell=cell)
    dt = torch.float64 if precision == "fp64" else torch.float32
    y = s.apply_stiffness(torch.tensor(x, dtype=dt, device="cuda"), precision).double().cpu().numpy()
    tol = 1e-12 if precision == "fp64" else 2e-5
    scale = np.abs(K).max() * np.abs(x).max() if precision == "mixed" else np.abs(y_ref).max()
    assert np.abs(y - y_ref).max() <= tol * scale
    s.close()


@pytest.mark.parametrize("elem,physics,shape,kind,cell", OPERATOR_CASES[::2])
def test_rhs_and_mean_flux(elem, physics, shape, kind, cell):
    torch = _torch()
    g = fem.Grid(shape, elem, physics)
    if cell is not None:
        g.h = np.array(cell, float)[: g.dim] / np.array(g.n_xyz, float)
        g.vp = float(np.prod(g.h))
    rng = np.random.default_rng(2)
    ids = rng.integers(0, 3, size=shape).astype(np.uint8)
    mod = _materials(physics, g.dim, kind)
    s = _solver(elem, physics, shape, ids, mod, cell=cell)
    e = rng.standard_normal(g.m)
    b = s.rhs(e).cpu().numpy()
    b_ref = fem.assemble_rhs(g, ids.ravel(), mod, e)
    assert _rel(b, b_ref) < 1e-12
    u = rng.standard_normal(g.c * g.N)
    fl = s.mean_flux(e, torch.tensor(u, device="cuda"))
    fl_ref = fem.mean_flux(g, ids.ravel(), mod, e, u) / (g.vp * g.N)
    assert _rel(fl, fl_ref) < 1e-12
    s.close()


PRECOND_CASES = [
    ("hex8_3d", "elastic", (6, 12, 24)),
    ("hex8_3d", "scalar", (12, 6, 48)),
    ("hex8_3d", "elastic", (16, 8, 32)),
    ("p1tri2_2d", "scalar", (24, 48)),
    ("q1_2d", "elastic", (3, 8)),
    ("p1tri2_2d", "elastic", (96, 12)),
]


@pytest.mark.parametrize("elem,physics,shape", PRECOND_CASES)
def test_symbol_and_preconditioner(elem, physics, shape):
    """Algorithm 2 table (half spectrum, packed, times 1/N) and z = K_ref^+ r against the oracle."""
    torch = _torch()
    g = fem.Grid(shape, elem, physics)
    rng = np.random.default_rng(3)
    ids = rng.integers(0, 2, size=shape).astype(np.uint8)
    mod = _materials(physics, g.dim, "aniso")[:2]
    C_ref = fem.mean_material(g, ids.ravel(), mod)
    s = _solver(elem, physics, shape, ids, mod)
    s.precond_build()
    Kinv = solvers.kref_pinv_symbol(solvers.kref_symbol(g, C_ref))   # (c, c, *shape) complex
    assert np.abs(Kinv.imag).max() < 1e-12 * np.abs(Kinv).max()
    tab = s.symbol_inverse()                                          # (ne, nz, ny, nxh)
    c = g.c
    pairs = {1: [(0, 0)], 2: [(0, 0), (1, 1), (0, 1)], 3: [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]}[c]
    nxh = g.n_xyz[0] // 2 + 1
    for e_, (i, j) in enumerate(pairs):
        ref = Kinv[i, j].real / g.N
        ref = ref.reshape((1,) * (3 - g.dim) + ref.shape)[..., :nxh]
        assert _rel(tab[e_], ref) < 1e-12
    r = rng.standard_normal(g.c * g.N)
    z_ref = solvers.apply_precond(g, Kinv, r)
    z = s.apply_precond(torch.tensor(r, device="cuda")).cpu().numpy()
    assert _rel(z, z_ref) < 1e-12
    z32 = s.apply_precond(torch.tensor(r, dtype=torch.float32, device="cuda"), "mixed").double().cpu().numpy()
    assert _rel(z32, z_ref) < 2e-5
    s.close()


@pytest.mark.parametrize("n", [128, 96, 64, 32])
@pytest.mark.parametrize("physics", ["elastic", "scalar"])
def test_fused_xy_passes_match_oracle(physics, n):
    """The fused x-y FFT passes (FP32, n x n planes, n = 16 x 8, 16 x 6, 16 x 4, 16 x 2 points):
    preconditioner apply against the oracle, and mixed-precision solves with and without them agree."""
    torch = _torch()
    shape = (6, n, n)
    g = fem.Grid(shape, "hex8_3d", physics)
    rng = np.random.default_rng(21)
    ids = (rng.random(shape) < 0.3).astype(np.uint8)
    mod = _materials(physics, 3, "iso")[:2]
    C_ref = fem.mean_material(g, ids.ravel(), mod)
    Kinv = solvers.kref_pinv_symbol(solvers.kref_symbol(g, C_ref))
    r = rng.standard_normal(g.c * g.N)
    z_ref = solvers.apply_precond(g, Kinv, r)
    outs = {}
    for fused in (1, 0):
        s = _solver("hex8_3d", physics, shape, ids, mod, precision="mixed", fft_xy=fused, autotune=False)
        s.precond_build()
        z32 = s.apply_precond(torch.tensor(r, dtype=torch.float32, device="cuda"), "mixed").double().cpu().numpy()
        assert _rel(z32, z_ref) < 2e-5, fused
        loads = np.eye(6 if physics == "elastic" else 3)
        outs[fused] = s.solve(loads, tol=1e-9, fields=None)
        assert s.fft_plan("mixed")["xy_fused"] == fused
        s.close()
    assert _rel(outs[1]["C_eff"], outs[0]["C_eff"]) < 1e-7


@pytest.mark.parametrize("shape", [(128, 128, 128), (96, 96, 96), (64, 64, 64), (32, 32, 32), (96, 16, 24),
                                   (256, 16, 24)])
@pytest.mark.parametrize("physics", ["elastic", "scalar"])
def test_register_split_last_axis_pass_matches_oracle(physics, shape):
    """The register-split last-axis pass (FP32, nz = 32, 64, 96, 128, 256) with the fused x-y passes where
    the planes are square: preconditioner apply against the oracle, and mixed solves with and without
    them agree."""
    torch = _torch()
    g = fem.Grid(shape, "hex8_3d", physics)
    rng = np.random.default_rng(23)
    ids = (rng.random(shape) < 0.3).astype(np.uint8)
    mod = _materials(physics, 3, "iso")[:2]
    C_ref = fem.mean_material(g, ids.ravel(), mod)
    Kinv = solvers.kref_pinv_symbol(solvers.kref_symbol(g, C_ref))
    r = rng.standard_normal(g.c * g.N)
    z_ref = solvers.apply_precond(g, Kinv, r)
    outs = {}
    for fused in (1, 0):
        s = _solver("hex8_3d", physics, shape, ids, mod, precision="mixed", fft_xy=fused, autotune=False)
        s.precond_build()
        z32 = s.apply_precond(torch.tensor(r, dtype=torch.float32, device="cuda"), "mixed").double().cpu().numpy()
        assert _rel(z32, z_ref) < 2e-5, fused
        plan = s.fft_plan("mixed")
        assert (plan["xy_fused"], plan["last_reg"]) == ((int(shape[1] == shape[2]), 1) if fused else (0, 0))
        loads = np.eye(6 if physics == "elastic" else 3)[:2]
        outs[fused] = s.solve(loads, tol=1e-8, fields=None)
        s.close()
    assert _rel(outs[1]["mean_flux"], outs[0]["mean_flux"]) < 1e-6
    for a, b in zip(outs[1]["info"], outs[0]["info"]):
        assert a["converged"] and abs(a["iterations"] - b["iterations"]) <= 3


def _small_elastic(n=16, seed=3):
    ids = I.spheres3d(n, count=8, rmin=2.0, rmax=3.5, seed=seed)
    mod = np.stack([I.isotropic_elastic_mandel(1.0, 0.3), I.isotropic_elastic_mandel(100.0, 0.2)])
    return ids, mod


def test_solve_circle2d_matches_oracle():
    w = I.workload_circle2d_32()
    g = fem.Grid((32, 32), "p1tri2_2d", "scalar")
    ref = solvers.homogenise(g, w["ids"], w["moduli"], w["loads"], method="sparse")
    s = _solver("p1tri2_2d", "scalar", (32, 32), w["ids"], w["moduli"])
    s.precond_build()
    out = s.solve(w["loads"], tol=1e-12)
    assert _rel(out["C_eff"], ref["C_eff"]) < 1e-10
    assert _rel(out["fields"].reshape(len(w["loads"]), -1).cpu().numpy(), ref["fields"]) < 1e-9
    assert _rel(out["mean_flux"], ref["mean_flux"]) < 1e-10
    assert all(i["converged"] for i in out["info"])
    s.close()


@pytest.mark.parametrize("physics", ["elastic", "scalar"])
def test_solve_3d_matches_oracle(physics):
    n = 16
    if physics == "elastic":
        ids, mod = _small_elastic(n)
    else:
        ids = I.grf_threshold((n, n, n), ell=3.0, seed=4)
        mod = np.stack([I.isotropic_conductivity(1.0, 3), I.isotropic_conductivity(1000.0, 3)])
    g = fem.Grid((n, n, n), "hex8_3d", physics)
    loads = np.eye(g.m)
    # sparse LU for the scalar cell; unpreconditioned CG to 1e-14 for elasticity (LU fill is slow there)
    ref = solvers.homogenise(g, ids, mod, loads, method="sparse" if physics == "scalar" else "cg", tol=1e-14)
    s = _solver("hex8_3d", physics, (n, n, n), ids, mod)
    s.precond_build()
    out = s.solve(loads, tol=1e-12)
    assert _rel(out["C_eff"], ref["C_eff"]) < 1e-10
    assert _rel(out["fields"].reshape(len(loads), -1).cpu().numpy(), ref["fields"]) < 1e-9
    s.close()


@pytest.mark.parametrize("shape", [(4, 4, 1024), (4, 1024, 4), (1024, 4, 4)])
def test_longest_axis_matches_oracle(shape):
    """Cells with one axis at the longest supported length (1024 points; 4 x 4 across it): the FP64 and
    FP32 stiffness, the Algorithm 2 preconditioner in both precisions and the solve of two loads
    against the oracle.  Along such an axis the FFT passes hold fewer lines per CTA to fit shared
    memory."""
    torch = _torch()
    g = fem.Grid(shape, "hex8_3d", "elastic")
    rng = np.random.default_rng(41)
    ids = (rng.random(shape) < 0.3).astype(np.uint8)
    mod = _materials("elastic", 3, "iso")[:2]
    K = fem.assemble_K(g, ids.ravel(), mod)
    x = rng.standard_normal(g.c * g.N)
    y_ref = K @ x
    C_ref = fem.mean_material(g, ids.ravel(), mod)
    Kinv = solvers.kref_pinv_symbol(solvers.kref_symbol(g, C_ref))
    z_ref = solvers.apply_precond(g, Kinv, x)
    s = _solver("hex8_3d", "elastic", shape, ids, mod)
    y = s.apply_stiffness(torch.tensor(x, device="cuda"), "fp64").cpu().numpy()
    assert np.abs(y - y_ref).max() <= 1e-12 * np.abs(y_ref).max()
    y32 = s.apply_stiffness(torch.tensor(x, dtype=torch.float32, device="cuda"), "mixed").double().cpu().numpy()
    assert np.abs(y32 - y_ref).max() <= 2e-5 * np.abs(K).max() * np.abs(x).max()
    # The reference symbol's smallest nonzero modes scale like (2 pi / n)^2 along an axis of n points, so
    # the rounding of the transforms reaches z amplified by (n / 128)^2 more than on the 128-point cells
    # the base tolerances below are set for (the stiffness is local and keeps its tolerances).
    f = (max(shape) / 128) ** 2
    s.precond_build()
    z = s.apply_precond(torch.tensor(x, device="cuda")).cpu().numpy()
    z32 = s.apply_precond(torch.tensor(x, dtype=torch.float32, device="cuda"), "mixed").double().cpu().numpy()
    loads = np.eye(6)[:2]
    ref = solvers.homogenise(g, ids, mod, loads, method="pcg", tol=1e-13)  # the oracle's own PCG
    out = s.solve(loads, tol=1e-12)
    s.close()
    errs = (_rel(z, z_ref), _rel(z32, z_ref), _rel(out["mean_flux"], ref["mean_flux"]),
            _rel(out["fields"].reshape(len(loads), -1).cpu().numpy(), ref["fields"]))
    assert all(i["converged"] for i in out["info"])
    assert errs[0] < 1e-12 * f and errs[1] < 2e-5 * f, errs
    assert errs[2] < 1e-10 * f and errs[3] < 1e-9 * f, errs


def test_iteration_counts_match_oracle_pcg():
    """Same algorithm, same stopping test: the GPU and oracle PCG stop at the same iteration (+-1)."""
    n = 16
    ids, mod = _small_elastic(n, seed=5)
    g = fem.Grid((n, n, n), "hex8_3d", "elastic")
    loads = np.eye(6)
    ref = solvers.homogenise(g, ids, mod, loads, method="pcg", tol=1e-6)
    s = _solver("hex8_3d", "elastic", (n, n, n), ids, mod)
    s.precond_build()
    out = s.solve(loads, tol=1e-6)
    its = [i["iterations"] for i in out["info"]]
    assert all(abs(a - b) <= 1 for a, b in zip(its, ref["iters"])), (its, ref["iters"])
    s.close()


def test_batched_loads_equal_one_by_one():
    n = 16
    ids, mod = _small_elastic(n, seed=6)
    s = _solver("hex8_3d", "elastic", (n, n, n), ids, mod)
    s.precond_build()
    loads = np.eye(6) + 0.1
    batch = s.solve(loads, tol=1e-8)
    for l in range(6):
        one = s.solve(loads[l:l + 1], tol=1e-8)
        assert one["info"][0]["iterations"] == batch["info"][l]["iterations"]
        assert _rel(one["fields"][0].cpu().numpy(), batch["fields"][l].cpu().numpy()) < 1e-13
    s.close()


def test_mixed_precision_matches_fp64():
    n = 16
    ids, mod = _small_elastic(n, seed=7)
    s64 = _solver("hex8_3d", "elastic", (n, n, n), ids, mod)
    s64.precond_build()
    o64 = s64.solve(np.eye(6), tol=1e-10)
    s32 = _solver("hex8_3d", "elastic", (n, n, n), ids, mod, precision="mixed")
    s32.precond_build()
    o32 = s32.solve(np.eye(6), tol=1e-10)
    assert _rel(o32["C_eff"], o64["C_eff"]) < 1e-7
    for inf in o32["info"]:
        assert inf["converged"] and inf["refinements"] >= 1
        assert inf["rel_residual_M"] <= 1e-10
    s64.close()
    s32.close()


def test_mixed_precision_matches_fp64_on_a_ragged_field_length():
    """Mixed and FP64 solves agree where the field length c N x loads is not a multiple of 4: the 16-byte
    precision casts of the refinement loop then finish the last elements one at a time (2-D P1
    conductivity on a 6 x 3 grid, one load: 18 values)."""
    shape = (3, 6)
    ids = np.array([[0, 1, 0, 0, 1, 1], [1, 0, 0, 1, 0, 0], [0, 0, 1, 1, 0, 1]], np.uint8)
    mod = _materials("scalar", 2, "iso")[:2]
    out = {}
    for prec in ("fp64", "mixed"):
        s = _solver("p1tri2_2d", "scalar", shape, ids, mod, precision=prec)
        s.precond_build()
        out[prec] = s.solve(np.eye(2)[:1], tol=1e-10)
        assert out[prec]["info"][0]["converged"]
        s.close()
    assert _rel(out["mixed"]["mean_flux"], out["fp64"]["mean_flux"]) < 1e-8
    assert _rel(out["mixed"]["fields"].cpu().numpy(), out["fp64"]["fields"].cpu().numpy()) < 1e-7


def test_graph_and_plain_launches_agree():
    n = 16
    ids, mod = _small_elastic(n, seed=8)
    # fixed launch plans: the plan tuner may pick different tilings (and so summation orders) per context
    a = _solver("hex8_3d", "elastic", (n, n, n), ids, mod, use_graph=True, autotune=False)
    b = _solver("hex8_3d", "elastic", (n, n, n), ids, mod, use_graph=False, autotune=False)
    a.precond_build()
    b.precond_build()
    oa, ob = a.solve(np.eye(6), tol=1e-8), b.solve(np.eye(6), tol=1e-8)
    assert [i["iterations"] for i in oa["info"]] == [i["iterations"] for i in ob["info"]]
    assert _rel(oa["fields"].cpu().numpy(), ob["fields"].cpu().numpy()) == 0.0
    a.close()
    b.close()


def test_warm_start_with_solution_converges_immediately():
    torch = _torch()
    n = 16
    ids, mod = _small_elastic(n, seed=9)
    s = _solver("hex8_3d", "elastic", (n, n, n), ids, mod)
    s.precond_build()
    o = s.solve(np.eye(6), tol=1e-10)
    w = s.solve(np.eye(6), tol=1e-8, x0=o["fields"].contiguous())
    assert all(i["iterations"] <= 1 for i in w["info"])
    assert _rel(w["C_eff"], o["C_eff"]) < 1e-9
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_warm_start_galerkin_scaling(precision):
    """x0 = 2.5 u*: the energy-optimal factor <b, x0> / <x0, K x0> is 1 / 2.5, so the scaled start is
    the solution; without the scaling PCG has to remove the excess.  A constant x0 (mean-free part 0)
    gets gamma = 0 and behaves like the zero guess."""
    n = 16
    ids, mod = _small_elastic(n, seed=11)
    ref = _solver("hex8_3d", "elastic", (n, n, n), ids, mod)
    ref.precond_build()
    o = ref.solve(np.eye(6), tol=1e-11)
    ref.close()
    u = o["fields"].contiguous()
    for scaled in (True, False):
        s = _solver("hex8_3d", "elastic", (n, n, n), ids, mod, precision=precision, x0_scaling=scaled)
        s.precond_build()
        w = s.solve(np.eye(6), tol=1e-6, x0=(2.5 * u).contiguous())
        its = [i["iterations"] for i in w["info"]]
        if scaled:
            assert max(its) <= 1, its
        else:
            assert min(its) > 1, its
        assert _rel(w["C_eff"], o["C_eff"]) < 1e-5
        cold = s.solve(np.eye(6), tol=1e-6)
        c = s.solve(np.eye(6), tol=1e-6, x0=(u * 0 + 3.0).contiguous())
        assert [i["iterations"] for i in c["info"]] == [i["iterations"] for i in cold["info"]]
        s.close()


def test_energy_form_c_eff():
    """Energy (Hill-Mandel) form of C_eff: equals the oracle's bilinear energy of the GPU's own fields at
    any accuracy, matches the exact C_eff when converged, is far closer to it than the stress average
    when loosely converged, and makes mixed and FP64 agree to 1e-7 at tol 1e-6."""
    n = 16
    ids, mod = _small_elastic(n, seed=14)
    g = fem.Grid((n, n, n), "hex8_3d", "elastic")
    exact = solvers.homogenise(g, ids.ravel(), mod, np.eye(6), method="cg", tol=1e-14)["C_eff"]
    s = _solver("hex8_3d", "elastic", (n, n, n), ids, mod)
    s.precond_build()
    loose = s.solve(np.eye(6), tol=1e-3)
    CE = s.effective_energy()
    u = loose["fields"].cpu().numpy()
    vol = g.vp * g.N
    ref = np.array([[fem.energy(g, ids.ravel(), mod, np.eye(6)[i], u[i].ravel(), np.eye(6)[j], u[j].ravel())
                     for j in range(6)] for i in range(6)]) / vol
    assert _rel(CE, 0.5 * (ref + ref.T)) < 1e-11
    assert np.abs(CE - exact).max() < 0.05 * np.abs(loose["C_eff"] - exact).max()
    s.solve(np.eye(6), tol=1e-12, fields=None)
    assert _rel(s.effective_energy(), exact) < 1e-10
    s.close()
    ce = {}
    for prec in ("fp64", "mixed"):
        t = _solver("hex8_3d", "elastic", (n, n, n), ids, mod, precision=prec)
        t.precond_build()
        t.solve(np.eye(6), tol=1e-6, fields=None)
        ce[prec] = t.effective_energy()
        t.close()
    assert _rel(ce["mixed"], ce["fp64"]) < 1e-7


def test_homogeneous_and_zero_load():
    C = _rand_spd(6, 12)
    ids = np.zeros((8, 8, 8), np.uint8)
    s = _solver("hex8_3d", "elastic", (8, 8, 8), ids, C[None])
    s.precond_build()
    out = s.solve(np.eye(6), tol=1e-10)
    assert _rel(out["C_eff"], C) < 1e-13
    assert np.abs(out["fields"].cpu().numpy()).max() < 1e-13
    z = s.solve(np.zeros((1, 6)), tol=1e-6)
    assert z["info"][0]["iterations"] == 0 and z["info"][0]["converged"]
    s.close()


def test_error_paths_return_status():
    fehom = _fehom()
    ids = np.zeros((8, 8, 8), np.uint8)
    mod = I.isotropic_elastic_mandel(1.0, 0.3)[None]
    with pytest.raises(fehom.FehomError) as e:
        _solver("hex8_3d", "elastic", (8, 8, 10), np.zeros((8, 8, 10), np.uint8), mod)
    assert e.value.status == 2
    with pytest.raises(fehom.FehomError) as e:
        _solver("hex8_3d", "elastic", (8, 8, 8), ids + 1, mod)            # id 1 >= n_phases
    assert e.value.status == 1
    bad = mod.copy()
    bad[0, 0, 0] = -5.0
    with pytest.raises(fehom.FehomError) as e:
        _solver("hex8_3d", "elastic", (8, 8, 8), ids, bad)
    assert e.value.status == 1
    s = _solver("hex8_3d", "elastic", (8, 8, 8), ids, mod)
    with pytest.raises(fehom.FehomError) as e:
        s.solve(np.eye(6), tol=1e-6)                                      # before precond_build
    assert e.value.status == 7
    s.close()
    ids2, mod2 = _small_elastic(16, seed=10)
    s = _solver("hex8_3d", "elastic", (16, 16, 16), ids2, mod2, max_iter=2)
    s.precond_build()
    out = s.solve(np.eye(6), tol=1e-10, raise_on_failure=False)
    assert out["status"] == 5
    assert all(i["iterations"] == 2 and not i["converged"] for i in out["info"])
    assert np.isfinite(out["C_eff"]).all()
    s.close()


def test_full_size_bench_config_sampled():
    """128^3 elastic spheres (the benchmark workload): sampled stiffness rows against the oracle's
    element-by-element rows; the FP64 solve's outputs satisfy properties that hold at any size."""
    torch = _torch()
    w = I.workload_spheres_elastic(128, seed=0)
    shape = (128, 128, 128)
    g = fem.Grid(shape, "hex8_3d", "elastic")
    s = _solver("hex8_3d", "elastic", shape, w["ids"], w["moduli"])
    rng = np.random.default_rng(11)
    x = rng.standard_normal(g.c * g.N)
    y = s.apply_stiffness(torch.tensor(x, device="cuda")).cpu().numpy()
    rows = rng.integers(0, g.c * g.N, 3000)
    y_ref = fem.stiffness_rows(g, w["ids"].ravel(), w["moduli"], x, rows)
    assert np.abs(y[rows] - y_ref).max() <= 1e-12 * np.abs(y_ref).max()
    s.precond_build()
    out = s.solve(w["loads"], tol=1e-6)
    C = out["C_eff"]
    assert all(i["converged"] for i in out["info"])
    assert np.abs(C - C.T).max() <= 1e-4 * np.abs(C).max()
    f = np.bincount(w["ids"].ravel(), minlength=2) / g.N
    voigt = sum(fp * Cp for fp, Cp in zip(f, w["moduli"]))
    reuss = np.linalg.inv(sum(fp * np.linalg.inv(Cp) for fp, Cp in zip(f, w["moduli"])))
    sym = 0.5 * (C + C.T)
    assert np.linalg.eigvalsh(voigt - sym).min() > 0 and np.linalg.eigvalsh(sym - reuss).min() > 0
    # the oracle's volume average of the GPU fields reproduces the GPU's mean stress
    u0 = out["fields"][0].reshape(-1).cpu().numpy()
    fl_ref = fem.mean_flux(g, w["ids"].ravel(), w["moduli"], w["loads"][0], u0) / (g.vp * g.N)
    assert _rel(out["mean_flux"][0], fl_ref) < 1e-12
    # true residual from the oracle at sampled DOFs: |b - K u| small relative to |b|
    b_rows = fem.assemble_rhs(g, w["ids"].ravel(), w["moduli"], w["loads"][0])
    r_rows = b_rows[rows] - fem.stiffness_rows(g, w["ids"].ravel(), w["moduli"], u0, rows)
    assert np.abs(r_rows).max() < 1e-3 * np.abs(b_rows).max()
    s.close()


def test_full_size_grf_scalar_512_mixed_and_fp64():
    """512^3 scalar conductivity, thresholded GRF, contrast 1000, three unit gradients (134M DOF):
    sampled stiffness rows against the oracle; FP64 and mixed solves to 1e-6 converge, give a symmetric
    C_eff inside the Voigt-Reuss bounds, and agree with each other."""
    torch = _torch()
    w = I.workload_grf_scalar(512)
    shape = (512, 512, 512)
    g = fem.Grid(shape, "hex8_3d", "scalar")
    ids = w["ids"].ravel()
    f = np.bincount(ids, minlength=2) / g.N
    voigt = sum(fp * Cp for fp, Cp in zip(f, w["moduli"]))
    reuss = np.linalg.inv(sum(fp * np.linalg.inv(Cp) for fp, Cp in zip(f, w["moduli"])))
    C = {}
    for prec in ("fp64", "mixed"):
        s = _solver("hex8_3d", "scalar", shape, w["ids"], w["moduli"], precision=prec)
        if prec == "fp64":
            rng = np.random.default_rng(5)
            x = rng.standard_normal(g.N)
            y = s.apply_stiffness(torch.tensor(x, device="cuda")).cpu().numpy()
            rows = rng.integers(0, g.N, 2000)
            y_ref = fem.stiffness_rows(g, ids, w["moduli"], x, rows)
            assert np.abs(y[rows] - y_ref).max() <= 1e-12 * np.abs(y_ref).max()
            del x, y
        s.precond_build()
        out = s.solve(w["loads"], tol=w["tol"], fields=None)
        assert all(i["converged"] for i in out["info"]), out["info"]
        assert all(i["rel_residual_2"] < 1e-4 for i in out["info"]), out["info"]
        C[prec] = out["C_eff"]
        sym = 0.5 * (C[prec] + C[prec].T)
        assert np.abs(C[prec] - C[prec].T).max() <= 1e-4 * np.abs(C[prec]).max()
        assert np.linalg.eigvalsh(voigt - sym).min() > 0 and np.linalg.eigvalsh(sym - reuss).min() > 0
        s.close()
    assert _rel(C["mixed"], C["fp64"]) < 1e-5


def test_autotuned_plans_are_valid_and_agree():
    """The FFT launch-plan tuner only changes tiling: results agree with the built-in plan."""
    n = 32
    ids, mod = _small_elastic(n, seed=12)
    outs, plans = [], []
    for tune in (True, False):
        for prec in ("fp64", "mixed"):
            s = _solver("hex8_3d", "elastic", (n, n, n), ids, mod, precision=prec, autotune=tune)
            s.precond_build()
            outs.append(s.solve(np.eye(6), tol=1e-9)["C_eff"])
            plans.append(s.fft_plan(prec))
            s.close()
    for p in plans[:2]:
        assert p["pairs"] in (4, 8, 16) and p["tc_y"] in (2, 4, 8, 16) and p["tc_last"] in (2, 4, 8, 16)
    for p in plans[2:]:
        assert p["pairs"] == 0 and p["tc_last"] == 0
    assert _rel(outs[0], outs[2]) < 1e-9 and _rel(outs[1], outs[3]) < 1e-8


def test_tuned_plans_are_shared_by_contexts_of_the_same_shape():
    """The launch-plan tuners time their candidates once per shape in a process: a second context of
    the same grid, field blocks, batch size and precision adopts the first one's plans (same choices
    and the same recorded timings) and reproduces its result bit for bit."""
    n = 48
    ids, mod = _small_elastic(n, seed=21)
    plans, fluxes = [], []
    for _ in range(2):
        s = _solver("hex8_3d", "elastic", (n, n, n), ids, mod, precision="mixed")
        s.precond_build()
        out = s.solve(np.eye(6)[:3], tol=1e-8)
        plans.append((s.fft_plan("mixed"), s.stencil_plan("mixed")))
        fluxes.append(np.asarray(out["mean_flux"]))
        s.close()
    (f0, s0), (f1, s1) = plans
    assert f0["pairs"] in (4, 8, 16) and all(m >= 0 for m in f0["ms"])
    assert f0 == f1 and s0 == s1
    assert np.array_equal(fluxes[0], fluxes[1])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_individual_solves(precision):
    """fehom_solve_batch (one graph, one branch per cell; cells of different sizes and contrasts)
    gives the per-cell results of separate fehom_solve calls."""
    fehom = _fehom()
    cells = I.workload_batched_spheres(count=4, sizes=(16, 24), seed0=30)
    def make():
        return [fehom.Solver("hex8_3d", "elastic", c["n"], c["ids"], c["moduli"], precision=precision, autotune=False)
                for c in cells]
    single = make()
    ref = []
    for sv in single:
        sv.precond_build()
        ref.append(sv.solve(np.eye(6), tol=1e-8, fields=None))
    solvers_b = make()
    for sv in solvers_b:
        sv.precond_build()
    batch = fehom.Batch(solvers_b)
    out = batch.solve(np.eye(6), tol=1e-8)
    tol = 1e-10 if precision == "fp64" else 1e-8
    for c in range(len(cells)):
        assert _rel(out["C_eff"][c], ref[c]["C_eff"]) < tol
        assert [i["iterations"] for i in out["info"][c]] == [i["iterations"] for i in ref[c]["info"]]
    # a second batch solve reuses the captured graph and gives the same answer
    out2 = batch.solve(np.eye(6), tol=1e-8)
    assert _rel(out2["C_eff"], out["C_eff"]) < tol
    batch.close()
    for sv in single + solvers_b:
        sv.close()


# ------------------------------------------------------------------------------------------------
# two-node stencil (Fig. 3 c): corner + centre node per pixel, four P1 triangles, Hermitian blocks
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(8, 16), (12, 48), (6, 96)])
def test_two_node_stencil_operators_match_oracle(shape):
    torch = _torch()
    g = fem.Grid(shape, "p1tri4_2d", "scalar")
    rng = np.random.default_rng(sum(shape))
    ids = rng.integers(0, 3, size=shape).astype(np.uint8)
    mod = _materials("scalar", 2, "aniso")
    s = _solver("p1tri4_2d", "scalar", shape, ids, mod)
    assert s.c == 2
    K = fem.assemble_K(g, ids.ravel(), mod)
    x = rng.standard_normal(2 * g.N)
    for prec, tol in (("fp64", 1e-12), ("mixed", 2e-5)):
        dt = torch.float64 if prec == "fp64" else torch.float32
        y = s.apply_stiffness(torch.tensor(x, dtype=dt, device="cuda"), prec).double().cpu().numpy()
        ref = K @ x
        assert _rel(y, ref) < tol, prec
    e = np.array([0.8, -0.3])
    b = s.rhs(e).cpu().numpy()
    assert _rel(b, fem.assemble_rhs(g, ids.ravel(), mod, e)) < 1e-12
    s.precond_build()
    C_ref = fem.mean_material(g, ids.ravel(), mod)
    Kinv = solvers.kref_pinv_symbol(solvers.kref_symbol(g, C_ref))
    tab = s.symbol_inverse()[:, 0]                                    # (4, ny, nxh)
    nxh = g.n_xyz[0] // 2 + 1
    ref01 = Kinv[0, 1][..., :nxh] / g.N
    assert _rel(tab[0], Kinv[0, 0].real[..., :nxh] / g.N) < 1e-12
    assert _rel(tab[1], Kinv[1, 1].real[..., :nxh] / g.N) < 1e-12
    assert _rel(tab[2] + 1j * tab[3], ref01) < 1e-12
    r = solvers.project_mean_zero(g, rng.standard_normal(2 * g.N))
    z_ref = solvers.apply_precond(g, Kinv, r)
    z = s.apply_precond(torch.tensor(r, device="cuda")).cpu().numpy()
    assert _rel(z, z_ref) < 1e-12
    z32 = s.apply_precond(torch.tensor(r, dtype=torch.float32, device="cuda"), "mixed").double().cpu().numpy()
    assert _rel(z32, z_ref) < 2e-5
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_two_node_stencil_solve_matches_oracle(precision):
    shape = (32, 32)
    g = fem.Grid(shape, "p1tri4_2d", "scalar")
    ids = I.circle2d(32, 0.3)
    mod = np.stack([I.isotropic_conductivity(1.0, 2), I.isotropic_conductivity(10.0, 2)])
    ref = solvers.homogenise(g, ids.ravel(), mod, np.eye(2), method="sparse")
    s = _solver("p1tri4_2d", "scalar", shape, ids, mod, precision=precision)
    s.precond_build()
    out = s.solve(np.eye(2), tol=1e-12)
    tol = 1e-10 if precision == "fp64" else 1e-8
    assert _rel(out["C_eff"], ref["C_eff"]) < tol
    u = out["fields"].cpu().numpy().reshape(2, -1)
    assert np.abs(u - ref["fields"]).max() < (1e-9 if precision == "fp64" else 1e-7) * np.abs(ref["fields"]).max()
    assert abs(u[0].sum()) < 1e-9  # the common mean of both node types is removed
    assert all(i["converged"] for i in out["info"])
    s.close()


def test_full_size_mixed_meets_fp64_energy_c_eff():
    """The benchmark workload (128^3 elasticity, 6 loads, tol 1e-6): the mixed-precision solve reaches
    the tolerance with an energy-form C_eff within 1e-7 of the FP64 solve's."""
    w = I.workload_spheres_elastic(128, seed=0)
    ce = {}
    for prec in ("fp64", "mixed"):
        s = _fehom().Solver("hex8_3d", "elastic", w["n"], w["ids"], w["moduli"], precision=prec)
        s.precond_build()
        out = s.solve(w["loads"], tol=w["tol"], fields=None)
        assert all(i["converged"] for i in out["info"])
        ce[prec] = s.effective_energy()
        s.close()
    assert _rel(ce["mixed"], ce["fp64"]) < 1e-7


@pytest.mark.parametrize("shape", [(12, 12, 48), (24, 24, 24), (6, 6, 96)])
def test_double_float_residual_update_matches_oracle(shape):
    """r_out = r_in - K d with K d in double-float arithmetic (isotropic phases, cubic voxels): against
    the oracle's assembled K at FP64-level accuracy, ||r_out||^2 in FP64, and <sigma> of d alone
    against the oracle's volume average.  The shapes span several 32 x 8 tiles with ragged edges."""
    torch = _torch()
    g = fem.Grid(shape, "hex8_3d", "elastic")
    cell = tuple(float(n) / 16.0 for n in shape[::-1])  # cubic voxels, h = 1/16 (x, y, z)
    g.h = np.array(cell) / np.array(g.n_xyz, float)
    g.vp = float(np.prod(g.h))
    rng = np.random.default_rng(21)
    ids = rng.integers(0, 3, size=shape).astype(np.uint8)
    mod = np.stack([I.isotropic_elastic_mandel(1.0, 0.3), I.isotropic_elastic_mandel(100.0, 0.2),
                    I.isotropic_elastic_mandel(7.0, 0.45)])
    K = fem.assemble_K(g, ids.ravel(), mod)
    d = rng.standard_normal(g.c * g.N).astype(np.float32)
    r_in = rng.standard_normal(g.c * g.N)
    ref = r_in - K @ d.astype(np.float64)
    s = _solver("hex8_3d", "elastic", shape, ids, mod, cell=cell)
    r_out, rn2, sig = s.residual_update(torch.tensor(d, device="cuda"), torch.tensor(r_in, device="cuda"))
    r_out = r_out.cpu().numpy()
    scale = np.abs(K).max() * np.abs(d).max()
    assert np.abs(r_out - ref).max() <= 1e-11 * scale
    assert abs(rn2 - float(ref @ ref)) <= 1e-10 * float(ref @ ref)
    sig_ref = fem.mean_flux(g, ids.ravel(), mod, np.zeros(6), d.astype(np.float64)) / (g.vp * g.N)
    assert np.abs(sig - sig_ref).max() <= 1e-11 * np.abs(sig_ref).max()
    # in place (r_out = r_in)
    r = torch.tensor(r_in, device="cuda")
    s.residual_update(torch.tensor(d, device="cuda"), r, r)
    assert np.abs(r.cpu().numpy() - ref).max() <= 1e-11 * scale
    s.close()


@pytest.mark.parametrize("shape", [(12, 12, 48), (6, 6, 96)])
def test_double_float_rhs_matches_oracle(shape):
    """b = -D^T W C e in double-float arithmetic (the mixed solve's right-hand side) against the oracle's
    assembled right-hand side, at FP64-level accuracy."""
    g = fem.Grid(shape, "hex8_3d", "elastic")
    cell = tuple(float(n) / 16.0 for n in shape[::-1])
    g.h = np.array(cell) / np.array(g.n_xyz, float)
    g.vp = float(np.prod(g.h))
    rng = np.random.default_rng(24)
    ids = rng.integers(0, 3, size=shape).astype(np.uint8)
    mod = np.stack([I.isotropic_elastic_mandel(1.0, 0.3), I.isotropic_elastic_mandel(100.0, 0.2),
                    I.isotropic_elastic_mandel(7.0, 0.45)])
    s = _solver("hex8_3d", "elastic", shape, ids, mod, cell=cell)
    for e in (np.eye(6)[3], rng.standard_normal(6)):
        b = s.rhs_df(e).cpu().numpy()
        b_ref = fem.assemble_rhs(g, ids.ravel(), mod, e)
        assert _rel(b, b_ref) < 1e-12
        assert _rel(b, s.rhs(e).cpu().numpy()) < 1e-12
    s.close()


def test_double_float_residual_update_full_size_sampled():
    """The 128^3 benchmark cell: the double-float update against the FP64 stiffness kernel everywhere
    (both are checked against the oracle's rows elsewhere) and against the oracle's rows on a sample."""
    torch = _torch()
    w = I.workload_spheres_elastic(128, seed=0)
    shape = (128, 128, 128)
    g = fem.Grid(shape, "hex8_3d", "elastic")
    s = _solver("hex8_3d", "elastic", shape, w["ids"], w["moduli"])
    rng = np.random.default_rng(22)
    d = torch.tensor(rng.standard_normal(g.c * g.N).astype(np.float32), device="cuda")
    r_in = torch.tensor(rng.standard_normal(g.c * g.N), device="cuda")
    r_out, _, _ = s.residual_update(d, r_in)
    kd = s.apply_stiffness(d.double())
    ref = (r_in - kd).cpu().numpy()
    out = r_out.cpu().numpy()
    scale = float(kd.abs().max())
    assert np.abs(out - ref).max() <= 1e-11 * scale
    rows = rng.integers(0, g.c * g.N, 2000)
    kd_rows = fem.stiffness_rows(g, w["ids"].ravel(), w["moduli"], d.double().cpu().numpy(), rows)
    assert np.abs(out[rows] - (r_in.cpu().numpy()[rows] - kd_rows)).max() <= 1e-11 * scale
    s.close()


def test_mixed_solve_double_float_residual_agrees_with_fp64_residual():
    """The mixed solve with refinement residuals updated in double-float arithmetic agrees with the one
    that recomputes b - K x by the FP64 stiffness: same iteration counts (within one), fields and C_eff."""
    n = 32
    ids, mod = _small_elastic(n, seed=23)
    out = {}
    for df in (True, False):
        s = _solver("hex8_3d", "elastic", (n, n, n), ids, mod, precision="mixed", residual_df=df)
        s.precond_build()
        o = s.solve(np.eye(6), tol=1e-6)
        out[df] = (o, s.effective_energy(), o["fields"].cpu().numpy())
        s.close()
    (a, ea, fa), (b, eb, fb) = out[True], out[False]
    assert all(i["converged"] for i in a["info"]) and all(i["converged"] for i in b["info"])
    for ia, ib in zip(a["info"], b["info"]):
        assert abs(ia["iterations"] - ib["iterations"]) <= 1 and ia["refinements"] == ib["refinements"]
    assert _rel(a["C_eff"], b["C_eff"]) < 1e-9
    assert _rel(ea, eb) < 1e-11
    assert np.abs(fa - fb).max() < 1e-8 * np.abs(fb).max()


def test_double_float_residual_rejects_unsupported_contexts():
    """Anisotropic phases (no isotropic table): FEHOM_E_UNSUPPORTED_SIZE, nothing written."""
    torch = _torch()
    shape = (8, 8, 8)
    ids = np.zeros(shape, np.uint8)
    s = _solver("hex8_3d", "elastic", shape, ids, _materials("elastic", 3, "aniso")[:1])
    d = torch.zeros(3 * 512, dtype=torch.float32, device="cuda")
    r = torch.ones(3 * 512, dtype=torch.float64, device="cuda")
    st = s.lib.fehom_residual_update(s.ctx, C.c_void_p(d.data_ptr()), C.c_void_p(r.data_ptr()),
                                     C.c_void_p(r.data_ptr()), None)
    assert st == 2  # FEHOM_E_UNSUPPORTED_SIZE
    assert float(r.min()) == 1.0 and float(r.max()) == 1.0
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_stencil_tile_heights_agree_with_oracle(precision):
    """The PCG stiffness apply with 8- and 16-row tiles (forced, and as picked by the stencil tuner) gives
    the oracle's C_eff on a grid whose y extent is ragged for the 16-row tiles (24 = 16 + 8) and whose x
    extent is ragged for the 32-node tile width (48 = 32 + 16)."""
    shape = (8, 24, 48)
    rng = np.random.default_rng(31)
    ids = rng.integers(0, 2, size=shape).astype(np.uint8)
    mod = np.stack([I.isotropic_elastic_mandel(1.0, 0.3), I.isotropic_elastic_mandel(20.0, 0.2)])
    cell = (48 / 16, 24 / 16, 8 / 16)  # cubic voxels: the isotropic fast path
    g = fem.Grid(shape, "hex8_3d", "elastic")
    g.h = np.array(cell) / np.array(g.n_xyz, float)
    g.vp = float(np.prod(g.h))
    # the oracle's averages are over the unit cell (|Y| = 1): divide by this cell's volume
    ref = solvers.homogenise(g, ids.ravel(), mod, np.eye(6), method="cg", tol=1e-13)["C_eff"] / (g.vp * g.N)
    tol, bound = (1e-10, 1e-9) if precision == "fp64" else (1e-8, 1e-7)
    for rows in (8, 16, 0):
        s = _solver("hex8_3d", "elastic", shape, ids, mod, precision=precision, cell=cell, stencil_rows=rows)
        s.precond_build()
        out = s.solve(np.eye(6), tol=tol)
        assert all(i["converged"] for i in out["info"])
        assert _rel(s.effective_energy(), ref) < bound
        used, staging, ms = s.stencil_plan(precision)
        assert used == (rows if rows else used) and used in (8, 16)
        if rows == 0:  # the tuner timed every candidate (TMA staging only for the FP32 kernels) and kept the fastest
            timed = [(m, (8, 0) if i == 0 else (16, 0) if i == 1 else (8, 3) if i == 2 else (16, 3))
                     for i, m in enumerate(ms) if m > 0]
            assert ms[0] > 0 and ms[1] > 0 and (precision == "fp64") == (ms[2] == 0 and ms[3] == 0)
            assert (used, staging) == min(timed)[1]
        else:
            assert staging == 0
        s.close()
