"""Seeded synthetic inputs: phase-id fields, phase moduli and macroscopic loads.

This module is shared by the CUDA path's tests and benchmark and by the oracle's tests.  It holds
none of the solver's arithmetic: it only draws microstructures (uint8 phase id per voxel, x
fastest, array shape ``(nz, ny, nx)`` or ``(ny, nx)``), builds per-phase material matrices in the
Mandel convention of Sec. 2 (Eq. mandel_grad and the matrix form of the stiffness that follows it),
and lists unit macroscopic loads.

Geometry convention: the cell is the unit cube [0, 1]^d, node (i, j, k) sits at h * (i, j, k) and
voxel (i, j, k) spans [i h, (i + 1) h] x ...; a voxel belongs to a shape when its centre lies
strictly inside it under the periodic minimum-image distance.
"""
from __future__ import annotations

import numpy as np

MANDEL_3D = ("11", "22", "33", "23", "13", "12")
MANDEL_2D = ("11", "22", "12")


# ----------------------------------------------------------------------------------------------
# material matrices
# ----------------------------------------------------------------------------------------------
def lame(E: float, nu: float) -> tuple[float, float]:
    """Lame constants (lambda, mu) of an isotropic solid from Young's modulus and Poisson ratio."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def isotropic_elastic_mandel(E: float, nu: float, dim: int = 3) -> np.ndarray:
    """Isotropic stiffness in Mandel form: C = lambda * J + 2 mu * I (J = ones on the normal block).

    2-D uses plane strain with the Mandel order (11, 22, 12); 3-D uses (11, 22, 33, 23, 13, 12).
    """
    lam, mu = lame(E, nu)
    m = 3 if dim == 2 else 6
    C = 2.0 * mu * np.eye(m)
    C[:dim, :dim] += lam
    return C


def bulk_shear_mandel(K: float, G: float, dim: int = 3) -> np.ndarray:
    """Isotropic stiffness in Mandel form from bulk and shear moduli (3-D: lambda = K - 2G/3)."""
    lam = K - 2.0 * G / 3.0 if dim == 3 else K - G
    m = 3 if dim == 2 else 6
    C = 2.0 * G * np.eye(m)
    C[:dim, :dim] += lam
    return C


def isotropic_conductivity(k: float, dim: int) -> np.ndarray:
    """Isotropic conductivity matrix k * I (d x d)."""
    return k * np.eye(dim)


def unit_loads(m: int) -> np.ndarray:
    """The m unit macroscopic gradients/strains (rows), Mandel components for elasticity."""
    return np.eye(m)


# ----------------------------------------------------------------------------------------------
# geometry helpers
# ----------------------------------------------------------------------------------------------
def _centres(shape):
    """Voxel-centre coordinates in voxel units, one array per axis, broadcast to ``shape``."""
    axes = [np.arange(s, dtype=np.float64) + 0.5 for s in shape]
    return np.meshgrid(*axes, indexing="ij")


def circle2d(n: int, radius: float = 0.3, inside: int = 1, outside: int = 0) -> np.ndarray:
    """Centred disc of radius ``radius`` (fraction of the cell edge) on an n x n pixel grid."""
    y, x = _centres((n, n))
    c = n / 2.0
    r = radius * n
    d2 = (x - c) ** 2 + (y - c) ** 2
    return np.where(d2 < r * r, inside, outside).astype(np.uint8)


def coated_sphere(n: int, r1: float = 0.2, r2: float = 0.4) -> np.ndarray:
    """Centred coated sphere (core id 0, coating id 1, matrix id 2) on an n^3 voxel grid (Sec. 6.2)."""
    z, y, x = _centres((n, n, n))
    c = n / 2.0
    d2 = ((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2) / (n * n)
    out = np.full((n, n, n), 2, dtype=np.uint8)
    out[d2 < r2 * r2] = 1
    out[d2 < r1 * r1] = 0
    return out


def laminate(shape, layer_phase) -> np.ndarray:
    """Grid-aligned laminate with layers normal to x (axis -1): ``layer_phase[i]`` for voxel column i."""
    layer_phase = np.asarray(layer_phase, dtype=np.uint8)
    assert layer_phase.shape == (shape[-1],)
    return np.broadcast_to(layer_phase, shape).copy()


def _periodic_d2(a, b, n):
    d = np.abs(a - b)
    d = np.minimum(d, n - d)
    return d * d


def spheres3d(n: int, count: int = 60, rmin: float = 8.0, rmax: float = 16.0, seed: int = 0,
              max_tries: int = 1_000_000) -> np.ndarray:
    """Random sequential addition of ``count`` non-overlapping periodic spheres (id 1) in a matrix (id 0).

    Radii ~ U[rmin, rmax] voxels, centres ~ U[0, n)^3; a sphere is accepted when its periodic
    centre distance to every placed sphere is at least the sum of the radii.
    """
    rng = np.random.default_rng(seed)
    centres, radii = [], []
    tries = 0
    while len(radii) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("spheres3d: could not place all spheres")
        r = rng.uniform(rmin, rmax)
        c = rng.uniform(0.0, n, size=3)
        ok = True
        for cc, rr in zip(centres, radii):
            d2 = sum(_periodic_d2(c[i], cc[i], n) for i in range(3))
            if d2 < (r + rr) ** 2:
                ok = False
                break
        if ok:
            centres.append(c)
            radii.append(r)
    out = np.zeros((n, n, n), dtype=np.uint8)
    for c, r in zip(centres, radii):
        # voxels whose centre may lie within r of c, per axis, wrapped periodically
        idx, d2 = [], []
        for ax in range(3):
            lo = int(np.floor(c[ax] - r - 1.0))
            hi = int(np.ceil(c[ax] + r + 1.0))
            span = np.arange(lo, hi + 1)
            if span.size > n:
                span = np.arange(n)
            w = np.mod(span, n)
            idx.append(w)
            d2.append(_periodic_d2(w + 0.5, c[ax], n))
        dd = d2[2][:, None, None] + d2[1][None, :, None] + d2[0][None, None, :]
        zz, yy, xx = np.ix_(idx[2], idx[1], idx[0])
        sub = out[zz, yy, xx]
        sub[dd < r * r] = 1
        out[zz, yy, xx] = sub
    return out


def grf_threshold(shape, ell: float = 16.0, seed: int = 0, fraction: float = 0.5) -> np.ndarray:
    """Periodic Gaussian random field thresholded to an exact volume fraction of phase 1.

    Seeded white noise is low-pass filtered by exp(-|k|^2 ell^2 / 2) (k in rad/voxel, ell in
    voxels); the ``fraction * size`` largest values become phase 1, ties broken by flat index.
    """
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(shape)
    ks = np.meshgrid(*[2.0 * np.pi * np.fft.fftfreq(s) for s in shape], indexing="ij")
    k2 = sum(k * k for k in ks)
    f = np.fft.ifftn(np.fft.fftn(w) * np.exp(-0.5 * k2 * ell * ell)).real
    flat = f.ravel()
    order = np.lexsort((np.arange(flat.size), flat))  # ascending value, ties by index
    out = np.zeros(flat.size, dtype=np.uint8)
    n1 = int(round(fraction * flat.size))
    if n1 > 0:
        out[order[flat.size - n1:]] = 1
    return out.reshape(shape)


# ----------------------------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------------------------
def workload_circle2d_32():
    """32 x 32 scalar P1 (2 triangles/pixel) cell: disc r = 0.3 L, conductivity 10 in 1."""
    ids = circle2d(32, 0.3)
    moduli = np.stack([isotropic_conductivity(1.0, 2), isotropic_conductivity(10.0, 2)])
    return dict(dim=2, n=(32, 32, 1), elem="p1tri2_2d", physics="scalar", ids=ids, moduli=moduli,
                loads=unit_loads(2), tol=1e-8)


def workload_spheres_elastic(n: int = 128, seed: int = 0, count: int = 60, rmin: float = 8.0,
                             rmax: float = 16.0):
    """n^3 hex8 elasticity: periodic spheres E = 100, nu = 0.2 in a matrix E = 1, nu = 0.3."""
    ids = spheres3d(n, count, rmin, rmax, seed)
    moduli = np.stack([isotropic_elastic_mandel(1.0, 0.3), isotropic_elastic_mandel(100.0, 0.2)])
    return dict(dim=3, n=(n, n, n), elem="hex8_3d", physics="elastic", ids=ids, moduli=moduli,
                loads=unit_loads(6), tol=1e-6)


def workload_grf_scalar(n: int = 512, seed: int = 0, ell: float = 16.0):
    """n^3 hex8 conductivity: thresholded periodic GRF (50 % vol.), conductivities 1 and 1000."""
    ids = grf_threshold((n, n, n), ell, seed)
    moduli = np.stack([isotropic_conductivity(1.0, 3), isotropic_conductivity(1000.0, 3)])
    return dict(dim=3, n=(n, n, n), elem="hex8_3d", physics="scalar", ids=ids, moduli=moduli,
                loads=unit_loads(3), tol=1e-6)


def random_field(shape, seed: int, dtype=np.float64) -> np.ndarray:
    """Seeded standard-normal test field (for operator-level parity tests)."""
    return np.random.default_rng(seed).standard_normal(shape).astype(dtype)


def hashin_coated_sphere_moduli():
    """Core / coating / matrix bulk and shear moduli of the coated-sphere example, contrast 1e3 (Sec. 6.2)."""
    K1, K2, Keff = 0.00132060, 1.3206033, 1.0
    G1, G2, Geff = 0.00079236, 0.7923620, 0.6
    return np.stack([bulk_shear_mandel(K1, G1), bulk_shear_mandel(K2, G2), bulk_shear_mandel(Keff, Geff)])



def workload_batched_spheres(count: int = 48, sizes=(32, 64, 96), seed0: int = 0):
    """Cells of uneven size for batched solves: ``count`` instances split evenly over ``sizes``;
    60 periodic spheres with radii U[n/16, n/8] (the 128^3 workload's statistics scaled to n), matrix
    E = 1, nu = 0.3, inclusions nu = 0.2 with a per-instance stiffness contrast 10^U[1, 3]."""
    out = []
    per = count // len(sizes)
    for i in range(count):
        n = sizes[min(i // per, len(sizes) - 1)]
        seed = seed0 + i
        rng = np.random.default_rng(10_000 + seed)
        contrast = 10.0 ** rng.uniform(1.0, 3.0)
        ids = spheres3d(n, 60, n / 16.0, n / 8.0, seed)
        moduli = np.stack([isotropic_elastic_mandel(1.0, 0.3), isotropic_elastic_mandel(contrast, 0.2)])
        out.append(dict(n=(n, n, n), ids=ids, moduli=moduli, contrast=contrast, seed=seed))
    return out


def workload_warmstart(n: int = 64, count: int = 4000, seed0: int = 0):
    """Scalar-conductivity cells for the learned warm start: even seeds draw 60 periodic spheres with
    radii U[n/16, n/8], odd seeds a Gaussian random field with correlation length n/16 voxels
    thresholded at 50 % volume; phase 1 has conductivity 10^U[1, 3] in a matrix of conductivity 1."""
    out = []
    for i in range(count):
        seed = seed0 + i
        rng = np.random.default_rng(20_000 + seed)
        contrast = 10.0 ** rng.uniform(1.0, 3.0)
        if seed % 2 == 0:
            ids = spheres3d(n, 60, n / 16.0, n / 8.0, seed)
            kind = "spheres"
        else:
            ids = grf_threshold((n, n, n), ell=n / 16.0, seed=seed)
            kind = "grf"
        moduli = np.stack([isotropic_conductivity(1.0, 3), isotropic_conductivity(contrast, 3)])
        out.append(dict(n=(n, n, n), ids=ids, moduli=moduli, contrast=contrast, seed=seed, kind=kind))
    return out
