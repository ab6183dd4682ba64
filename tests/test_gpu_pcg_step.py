"""Element-wise parity of the fused kernels that one PCG iteration runs, against the FP64 oracle.

The solves check these kernels only through their results, and the mixed solve's FP64 refinement
hides an error of its FP32 operators (it would only cost iterations).  Here each half of an iteration
is called through the C ABI on its own, with the same instantiations the solve launches:

* the stiffness launch with the fused <p, K p> and alpha = rz / <p, K p> (Sec. 5.1; PCG of Sec. 4.1),
  FP64 and FP32, 8- and 16-row hex8 tiles, the FP32 plane staging by 16-byte row copies (x extent a
  multiple of 32) and by 4-byte entries, ragged y and x tails, isotropic and general materials, and the
  2-D pixel stencils;
* the preconditioner passes with their fused vector updates (Sec. 4.2 Eq. M_inverse, Sec. 5.3):
  r -= alpha Ap, z = K_ref^+ r, <r, z> (Parseval), beta, x += alpha p, p = z + beta p, and the first
  apply (p = z), for the generic Stockham passes, the fused x-y passes and the register-split
  last-axis pass.

Oracle side: the assembled K (``fem.assemble_K`` / ``fem.stiffness_rows``) and the FFT
preconditioner of Algorithm 2 (``solvers.kref_symbol``, ``kref_pinv_symbol``, ``apply_precond``), with
the vector updates of the PCG recurrence written out in FP64 on the same inputs.  Tolerances: FP64
1e-12 of the operand scale; FP32 2e-5 of the operand scale; dot products against the sum of the
magnitudes of their terms.
"""
import functools

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import fem, solvers  # noqa: E402
from paper_2203_02962_gb300 import inputs as I  # noqa: E402

TOL = {"fp64": 1e-12, "mixed": 2e-5}


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


def _materials(physics, dim, kind):
    m = dim if physics == "scalar" else dim * (dim + 1) // 2
    if kind == "aniso":
        return np.stack([_rand_spd(m, 7 + p, 10.0 ** p) for p in range(3)])
    if physics == "scalar":
        return np.stack([I.isotropic_conductivity(k, dim) for k in (1.0, 30.0, 1000.0)])
    return np.stack([I.isotropic_elastic_mandel(E, nu, dim) for E, nu in ((1.0, 0.3), (100.0, 0.2), (7.0, 0.45))])


@functools.lru_cache(maxsize=None)
def _case(elem, physics, shape, kind, cubic, seed=0):
    """ids, moduli, cell, the oracle grid (cell-scaled) and its assembled K."""
    g = fem.Grid(shape, elem, physics)
    cell = None
    if cubic:  # cubic voxels of edge 1/16: the isotropic fast path of the hex8 kernels
        cell = tuple(n / 16.0 for n in g.n_xyz)
        g.h = np.array(cell) / np.array(g.n_xyz, float)
        g.vp = float(np.prod(g.h))
    rng = np.random.default_rng(100 + seed + sum(shape))
    ids = rng.integers(0, 3, size=shape).astype(np.uint8)
    mod = _materials(physics, g.dim, kind)
    K = fem.assemble_K(g, ids.ravel(), mod)
    return ids, mod, cell, g, K


def _solver(elem, physics, shape, ids, mod, cell, **kw):
    return _fehom().Solver(elem, physics, tuple(shape[::-1]), ids, mod, cell=cell, **kw)


STIFFNESS_CASES = [
    # elem, physics, shape (z, y, x), material, cubic voxels
    ("hex8_3d", "elastic", (8, 16, 64), "iso", True),     # x a multiple of 32: 16-byte staging; full tiles
    ("hex8_3d", "elastic", (6, 24, 96), "iso", True),     # ragged y for the 16-row tiles
    ("hex8_3d", "elastic", (6, 12, 64), "iso", True),     # ragged y for both heights
    ("hex8_3d", "elastic", (6, 12, 64), "aniso", False),  # general material contraction
    ("hex8_3d", "elastic", (4, 12, 48), "iso", True),     # ragged x: 4-byte staging only
    ("hex8_3d", "scalar", (6, 12, 64), "aniso", False),
    ("hex8_3d", "scalar", (8, 12, 48), "iso", True),
]
PIXEL_CASES = [
    ("p1tri2_2d", "scalar", (24, 48), "aniso", False),
    ("p1tri2_2d", "elastic", (12, 96), "aniso", False),
    ("q1_2d", "elastic", (6, 64), "aniso", False),
    ("p1tri4_2d", "scalar", (12, 48), "aniso", False),
]


def _check_stiffness(s, g, K, precision, rows, staging, n_loads=2, seed=0):
    torch = _torch()
    rng = np.random.default_rng(seed)
    dt = torch.float64 if precision == "fp64" else torch.float32
    p = rng.standard_normal((n_loads, g.c * g.N))
    p = p.astype(np.float32).astype(np.float64) if precision == "mixed" else p
    rz = rng.uniform(0.5, 2.0, n_loads)
    ap, pap, alpha = s.pcg_apply_stiffness(torch.tensor(p.reshape(n_loads, g.c, g.N), dtype=dt, device="cuda"), rz,
                                           precision, rows=rows, staging=staging)
    ap = ap.double().cpu().numpy().reshape(n_loads, -1)
    absK = abs(K)
    tol = TOL[precision]
    for l in range(n_loads):
        ref = K @ p[l]
        scale = np.abs(ref).max() if precision == "fp64" else np.abs(K).max() * np.abs(p[l]).max()
        assert np.abs(ap[l] - ref).max() <= tol * scale, (l, np.abs(ap[l] - ref).max() / scale)
        pap_ref = p[l] @ ref
        mag = np.abs(p[l]) @ (absK @ np.abs(p[l]))
        assert abs(pap[l] - pap_ref) <= tol * mag, (l, pap[l], pap_ref)
        a_ref = rz[l] / pap_ref
        assert abs(alpha[l] - a_ref) <= 2.0 * tol * mag / pap_ref * a_ref


def _staging_applies(physics, shape, kind, cubic, precision, staging, rows):
    """Whether a staging mode of the FP32 hex8 PCG apply exists for a case (the others must be refused)."""
    if staging in (0, 1):
        return True
    return precision == "mixed" and shape[2] % 32 == 0


@pytest.mark.parametrize("elem,physics,shape,kind,cubic", STIFFNESS_CASES)
@pytest.mark.parametrize("precision,staging", [("fp64", 0), ("mixed", 0), ("mixed", 1), ("mixed", 2), ("mixed", 3)])
@pytest.mark.parametrize("rows", [8, 16])
def test_pcg_stiffness_hex8_matches_oracle(elem, physics, shape, kind, cubic, precision, staging, rows):
    """The hex8 PCG stiffness launch: K p and the fused <p, K p> and alpha, every tile height and staging
    (4-byte and 16-byte cp.async copies, one tensor-memory-accelerator box per plane); a staging that does not
    apply to the case is refused with FEHOM_E_UNSUPPORTED_SIZE."""
    ids, mod, cell, g, K = _case(elem, physics, shape, kind, cubic)
    s = _solver(elem, physics, shape, ids, mod, cell, precision=precision)
    if _staging_applies(physics, shape, kind, cubic, precision, staging, rows):
        _check_stiffness(s, g, K, precision, rows, staging, n_loads=2, seed=rows + staging)
    else:
        torch = _torch()
        p = torch.zeros((1, g.c, g.N), dtype=torch.float32, device="cuda")
        with pytest.raises(_fehom().FehomError) as ei:
            s.pcg_apply_stiffness(p, [1.0], precision, rows=rows, staging=staging)
        assert ei.value.status == 2
    s.close()


@pytest.mark.parametrize("elem,physics,shape,kind,cubic", PIXEL_CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pcg_stiffness_pixels_match_oracle(elem, physics, shape, kind, cubic, precision):
    """The 2-D PCG stiffness launches (P1, Q1, two-node stencil) with the fused <p, K p>."""
    ids, mod, cell, g, K = _case(elem, physics, shape, kind, cubic)
    s = _solver(elem, physics, shape, ids, mod, cell, precision=precision)
    _check_stiffness(s, g, K, precision, 0, 0, n_loads=3, seed=5)
    s.close()


def test_pcg_stiffness_skips_finished_loads_and_reports_breakdown():
    """A zero direction gives <p, K p> = 0: that load breaks down (FEHOM_E_BREAKDOWN, alpha 0) while the
    other load of the launch is still computed."""
    torch = _torch()
    ids, mod, cell, g, K = _case("hex8_3d", "elastic", (6, 12, 64), "iso", True)
    s = _solver("hex8_3d", "elastic", (6, 12, 64), ids, mod, cell, precision="mixed")
    rng = np.random.default_rng(3)
    p = np.zeros((2, g.c * g.N), np.float32)
    p[1] = rng.standard_normal(g.c * g.N)
    fe = _fehom()
    with pytest.raises(fe.FehomError) as ei:
        s.pcg_apply_stiffness(torch.tensor(p.reshape(2, g.c, g.N), device="cuda"), [1.0, 1.0], "mixed")
    assert ei.value.status == 6
    ap = torch.empty((2, g.c, g.N), dtype=torch.float32, device="cuda")
    pt = torch.tensor(p.reshape(2, g.c, g.N), device="cuda")
    import ctypes as C
    rz = np.ones(2)
    pap, al = np.zeros(2), np.zeros(2)
    dp = C.POINTER(C.c_double)
    st = s.lib.fehom_pcg_apply_stiffness(s.ctx, 1, 2, C.c_void_p(pt.data_ptr()), C.c_void_p(ap.data_ptr()),
                                         rz.ctypes.data_as(dp), 0, 0, pap.ctypes.data_as(dp), al.ctypes.data_as(dp))
    assert st == 6 and pap[0] == 0.0 and al[0] == 0.0
    ref = K @ p[1].astype(np.float64)
    assert np.abs(ap[1].double().cpu().numpy().ravel() - ref).max() <= 2e-5 * np.abs(K).max() * np.abs(p[1]).max()
    assert abs(pap[1] - p[1].astype(np.float64) @ ref) <= 2e-5 * abs(pap[1])
    s.close()


PRECOND_CASES = [
    # elem, physics, shape, fft_xy (0 = generic Stockham passes; 1 = register-split passes where supported)
    ("hex8_3d", "elastic", (6, 12, 24), 0),
    ("hex8_3d", "scalar", (12, 6, 48), 0),
    ("hex8_3d", "elastic", (6, 128, 128), 1),   # fused x-y passes, generic last axis
    ("hex8_3d", "scalar", (6, 128, 128), 1),
    ("hex8_3d", "scalar", (6, 96, 96), 1),      # fused x-y passes of 96 = 16 x 6 points
    ("hex8_3d", "elastic", (96, 16, 24), 1),    # register-split last axis (nz = 96), generic x and y
    ("hex8_3d", "elastic", (96, 96, 96), 1),    # both register-split passes at 96, 64 and 32 points
    ("hex8_3d", "scalar", (64, 64, 64), 1),
    ("hex8_3d", "elastic", (32, 32, 32), 1),
    ("hex8_3d", "elastic", (256, 16, 24), 1),   # last axis of 256 points (16 x 16)
    ("p1tri2_2d", "scalar", (24, 48), 0),
    ("q1_2d", "elastic", (12, 96), 0),
    ("p1tri4_2d", "scalar", (12, 48), 0),       # Hermitian 2 x 2 blocks
]


@functools.lru_cache(maxsize=None)
def _precond_case(elem, physics, shape):
    g = fem.Grid(shape, elem, physics)
    rng = np.random.default_rng(40 + sum(shape))
    ids = rng.integers(0, 2, size=shape).astype(np.uint8)
    mod = _materials(physics, g.dim, "aniso")[:2]
    C_ref = fem.mean_material(g, ids.ravel(), mod)
    Kinv = solvers.kref_pinv_symbol(solvers.kref_symbol(g, C_ref))
    return ids, mod, g, Kinv


def _check_precond_step(s, g, Kinv, precision, n_loads, seed, expect_plan=None):
    torch = _torch()
    rng = np.random.default_rng(seed)
    dt = torch.float64 if precision == "fp64" else torch.float32
    rnd = lambda: rng.standard_normal((n_loads, g.c * g.N))  # noqa: E731
    r, ap, x, p = rnd(), rnd(), rnd(), rnd()
    if precision == "mixed":
        r, ap, x, p = (v.astype(np.float32).astype(np.float64) for v in (r, ap, x, p))
    alpha = rng.uniform(0.2, 1.5, n_loads)
    rz = rng.uniform(1.0, 3.0, n_loads)
    dev = lambda v: torch.tensor(v.reshape(n_loads, g.c, g.N), dtype=dt, device="cuda")  # noqa: E731
    tol = TOL[precision]

    # the first apply of PCG: p = z = K_ref^+ r, <r, z>
    rt, pt = dev(r), dev(p)
    rz0, _ = s.pcg_precond_step(rt, pt, precision)
    z0 = pt.double().cpu().numpy().reshape(n_loads, -1)
    assert np.abs(rt.double().cpu().numpy().reshape(n_loads, -1) - r).max() == 0.0  # r untouched
    for l in range(n_loads):
        zr = solvers.apply_precond(g, Kinv, r[l])
        assert np.abs(z0[l] - zr).max() <= tol * np.abs(zr).max()
        assert abs(rz0[l] - r[l] @ zr) <= tol * abs(r[l] @ zr)

    # a full iteration's passes: r -= alpha Ap; z; <r, z>; beta; x += alpha p; p = z + beta p
    rt, apt, xt, pt = dev(r), dev(ap), dev(x), dev(p)
    rz_new, beta = s.pcg_precond_step(rt, pt, precision, ap=apt, x=xt, alpha=alpha, rz=rz)
    r1 = rt.double().cpu().numpy().reshape(n_loads, -1)
    x1 = xt.double().cpu().numpy().reshape(n_loads, -1)
    p1 = pt.double().cpu().numpy().reshape(n_loads, -1)
    for l in range(n_loads):
        r_ref = r[l] - alpha[l] * ap[l]
        sc = np.abs(r[l]).max() + alpha[l] * np.abs(ap[l]).max()
        assert np.abs(r1[l] - r_ref).max() <= tol * sc
        z = solvers.apply_precond(g, Kinv, r_ref)
        rzn = r_ref @ z
        assert abs(rz_new[l] - rzn) <= tol * abs(rzn), (l, rz_new[l], rzn)
        b_ref = rzn / rz[l]
        assert abs(beta[l] - b_ref) <= tol * abs(b_ref)
        x_ref = x[l] + alpha[l] * p[l]
        assert np.abs(x1[l] - x_ref).max() <= tol * (np.abs(x[l]).max() + alpha[l] * np.abs(p[l]).max())
        p_ref = z + b_ref * p[l]
        assert np.abs(p1[l] - p_ref).max() <= tol * (np.abs(z).max() + abs(b_ref) * np.abs(p[l]).max()), l
    if expect_plan is not None:
        plan = s.fft_plan(precision)
        assert (plan["xy_fused"], plan["last_reg"]) == expect_plan


RS_LENGTHS = (32, 64, 96, 128)


def _rs_plan(elem, shape, fft_xy, precision):
    """(fused x-y, register-split last axis) that fft_xy = 1 must give: FP32 hex8 fields whose x-y planes
    are n x n (n = 32, 64, 96 or 128), and whose z axis has 32, 64, 96, 128 or 256 points, with whole
    16-column groups."""
    if fft_xy != 1 or precision != "mixed" or elem != "hex8_3d":
        return (0, 0)
    nz, ny, nx = shape
    fused = int(nx == ny and nx in RS_LENGTHS)
    z_ok = nz in RS_LENGTHS or nz == 256
    last = int(z_ok and (ny * (nx // 2 + 1)) % 16 == 0)
    return (fused, last)


@pytest.mark.parametrize("elem,physics,shape,fft_xy", PRECOND_CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pcg_precond_step_matches_oracle(elem, physics, shape, fft_xy, precision):
    """The FFT passes of a PCG iteration with their fused updates, for two loads at once."""
    ids, mod, g, Kinv = _precond_case(elem, physics, shape)
    s = _fehom().Solver(elem, physics, tuple(shape[::-1]), ids, mod, precision=precision, fft_xy=fft_xy,
                        autotune=False)
    s.precond_build()
    _check_precond_step(s, g, Kinv, precision, n_loads=2, seed=sum(shape),
                        expect_plan=_rs_plan(elem, shape, fft_xy, precision))
    s.close()


def test_pcg_step_full_size_benchmark_cell():
    """128^3 elastic spheres, six loads (the benchmark launch): the FP32 PCG stiffness with both tile
    heights and every staging on 3000 sampled rows of the oracle's K, its fused <p, K p> against the dot
    of its own output; the FP32 preconditioner passes with the register-split x-y and last-axis passes
    (the solve's plan at this size) against the oracle's FFT preconditioner, and the generic passes."""
    torch = _torch()
    w = I.workload_spheres_elastic(128, seed=0)
    shape = (128, 128, 128)
    g = fem.Grid(shape, "hex8_3d", "elastic")
    rng = np.random.default_rng(77)
    L = 6
    p = rng.standard_normal((L, g.c * g.N)).astype(np.float32)
    rows = rng.integers(0, g.c * g.N, 3000)
    s = _fehom().Solver("hex8_3d", "elastic", w["n"], w["ids"], w["moduli"], precision="mixed", fft_xy=1,
                        autotune=False)
    pt = torch.tensor(p.reshape(L, g.c, g.N), device="cuda")
    ref_rows = [fem.stiffness_rows(g, w["ids"].ravel(), w["moduli"], p[l].astype(np.float64), rows) for l in (0, L - 1)]
    for tile_rows, staging in ((8, 0), (8, 1), (8, 2), (8, 3), (16, 0), (16, 1), (16, 2), (16, 3)):
        ap, pap, _ = s.pcg_apply_stiffness(pt, np.ones(L), "mixed", rows=tile_rows, staging=staging)
        apn = ap.double()
        dots = (apn * pt.double()).sum(dim=(1, 2)).cpu().numpy()
        mags = (apn.abs() * pt.double().abs()).sum(dim=(1, 2)).cpu().numpy()
        assert np.all(np.abs(pap - dots) <= 1e-9 * mags), (tile_rows, staging)
        apc = apn.cpu().numpy().reshape(L, -1)
        for j, l in enumerate((0, L - 1)):
            assert np.abs(apc[l][rows] - ref_rows[j]).max() <= 2e-5 * np.abs(ref_rows[j]).max()
    s.precond_build()
    C_ref = fem.mean_material(g, w["ids"].ravel(), w["moduli"])
    Kinv = solvers.kref_pinv_symbol(solvers.kref_symbol(g, C_ref))
    _check_precond_step(s, g, Kinv, "mixed", n_loads=2, seed=5, expect_plan=(1, 1))
    s.close()
    s = _fehom().Solver("hex8_3d", "elastic", w["n"], w["ids"], w["moduli"], precision="mixed", fft_xy=0,
                        autotune=False)
    s.precond_build()
    _check_precond_step(s, g, Kinv, "mixed", n_loads=2, seed=6, expect_plan=(0, 0))
    s.close()
