"""Seeded synthetic inputs for 2-D deblurring: test images, Gaussian PSFs and
noise directions.

This module holds none of the deblurring method's arithmetic (no blur, no
Kronecker factors, no solver); it only draws the raw inputs.  Both the CUDA
path and the CPU oracle take their inputs from here, and each side forms the
observed data b = A x_true + e with its own operator (Section 5 of the paper:
b = A x_true + eps, noise level = ||eps||_2 / ||b_true||_2).

Conventions: an image X is n_r x n_c (row index i vertical, column index j
horizontal), stored as a float64 numpy array X[i, j]; vec(X) stacks columns
(Fortran order), Section 3.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 231_115_393


def phantom(n_r: int, n_c: int, n_shapes: int, rng: np.random.Generator) -> np.ndarray:
    """Piecewise-constant test image: ``n_shapes`` ellipses / axis-aligned
    rectangles painted in order on a zero background (later shapes overwrite
    earlier ones).  Centre ~ U over the image, semi-axes / half-sides
    ~ U[n/32, n/8] per axis, ellipse angle ~ U[0, pi), intensity ~ U[0, 1],
    ellipse vs rectangle by a fair coin."""
    X = np.zeros((n_r, n_c), dtype=np.float64)
    for _ in range(n_shapes):
        cy = rng.uniform(0.0, n_r)
        cx = rng.uniform(0.0, n_c)
        is_ellipse = rng.uniform() < 0.5
        hx = rng.uniform(n_c / 32.0, n_c / 8.0)
        hy = rng.uniform(n_r / 32.0, n_r / 8.0)
        theta = rng.uniform(0.0, np.pi)
        val = rng.uniform(0.0, 1.0)
        # only the pixels of a box that holds the whole shape are tested
        ry, rx = (max(hx, hy), max(hx, hy)) if is_ellipse else (hy, hx)
        i0, i1 = max(0, int(np.floor(cy - ry)) - 1), min(n_r, int(np.ceil(cy + ry)) + 2)
        j0, j1 = max(0, int(np.floor(cx - rx)) - 1), min(n_c, int(np.ceil(cx + rx)) + 2)
        if i0 >= i1 or j0 >= j1:
            continue
        ii, jj = np.meshgrid(np.arange(i0, i1, dtype=np.float64),
                             np.arange(j0, j1, dtype=np.float64), indexing="ij")
        dx = jj - cx
        dy = ii - cy
        if is_ellipse:
            u = (dx * np.cos(theta) + dy * np.sin(theta)) / hx
            v = (-dx * np.sin(theta) + dy * np.cos(theta)) / hy
            mask = u * u + v * v <= 1.0
        else:
            mask = (np.abs(dx) <= hx) & (np.abs(dy) <= hy)
        X[i0:i1, j0:j1][mask] = val
    return X


def gaussian_psf(n_r: int, n_c: int, c_r: int, c_c: int,
                 sigma_x: float, sigma_y: float, rho: float) -> np.ndarray:
    """Bivariate Gaussian point spread function on an n_r x n_c grid with
    0-based centre (c_r, c_c), normalised to sum 1.

    p[i, j] = exp(-1/2 d^T C^{-1} d), d = (j - c_c, i - c_r) (x horizontal =
    column offset, y vertical = row offset), C = [[sx^2, rho sx sy],
    [rho sx sy, sy^2]].  rho != 0 makes the PSF non-separable."""
    if not (-1.0 < rho < 1.0) or sigma_x <= 0 or sigma_y <= 0:
        raise ValueError("need sigma_x, sigma_y > 0 and |rho| < 1")
    dy = np.arange(n_r, dtype=np.float64)[:, None] - c_r
    dx = np.arange(n_c, dtype=np.float64)[None, :] - c_c
    q = (dx / sigma_x) ** 2 - 2.0 * rho * (dx / sigma_x) * (dy / sigma_y) + (dy / sigma_y) ** 2
    p = np.exp(-0.5 * q / (1.0 - rho * rho))
    return p / p.sum()


def separable_psf(n_r: int, n_c: int, c_r: int, c_c: int,
                  sigma_x: float, sigma_y: float) -> np.ndarray:
    """Axis-aligned Gaussian PSF (rho = 0): exactly rank one, p = u v^T."""
    return gaussian_psf(n_r, n_c, c_r, c_c, sigma_x, sigma_y, 0.0)


def noise_direction(n_r: int, n_c: int, rng: np.random.Generator) -> np.ndarray:
    """Standard normal n_r x n_c array g; the noise is e = nl * ||b_true|| * g / ||g||."""
    return rng.standard_normal((n_r, n_c))


@dataclass
class Problem:
    """One synthetic deblurring problem instance (raw inputs only)."""
    name: str
    n_r: int
    n_c: int
    center: tuple
    bc: str                      # "zero" | "reflexive"
    op_rank: int                 # Kronecker terms in A (0 = full)
    x_true: np.ndarray
    psf: np.ndarray
    noise_levels: list
    noise_dirs: list             # one standard-normal array per noise level
    lam: float | None = None     # fixed lambda, if the workload fixes one
    tol: float = 1e-6
    maxit: int = 100
    extra: dict = field(default_factory=dict)


# Workload recipes (shapes, sizes and value distributions of the paper's
# image-deblurring experiments, Section 5, scaled to the sizes studied here).
WORKLOADS = {
    # 64 x 64, FP64 throughout, full-rank (exact) Kronecker sum, zero BC.
    "deblur64_fp64": dict(n=64, shapes=12, sx=3.0, sy=1.5, rho=0.5, bc="zero",
                          op_rank=0, noise=[0.01], lam=0.01, tol=1e-8, maxit=50),
    # 256 x 256, reflexive BC, rank-3 operator, FP32 operator.
    "deblur256_fp32": dict(n=256, shapes=40, sx=4.0, sy=2.0, rho=0.6, bc="reflexive",
                           op_rank=3, noise=[0.01], lam=None, tol=1e-6, maxit=100),
    # 1024 x 1024, reflexive BC, rank-4 operator on tensor cores, two noise levels.
    "deblur1024_mixed": dict(n=1024, shapes=150, sx=6.0, sy=3.0, rho=0.7, bc="reflexive",
                             op_rank=4, noise=[0.005, 0.05], lam=None, tol=1e-6, maxit=100),
}
WORKLOAD_INDEX = {"deblur64_fp64": 0, "deblur256_fp32": 1, "deblur1024_mixed": 2}


def make_problem(name: str, n: int | None = None, seed: int | None = None) -> Problem:
    """Build the raw inputs of a named workload.  ``n`` overrides the image
    size for small test cases: the shape count scales with n, the PSF widths
    (a property of the optics) stay as in the workload."""
    w = WORKLOADS[name]
    n_full = w["n"]
    n = n_full if n is None else int(n)
    scale = n / n_full
    if seed is None:
        seed = SEED_BASE + WORKLOAD_INDEX[name]
    rng = np.random.default_rng(seed)
    shapes = max(1, int(round(w["shapes"] * scale))) if n != n_full else w["shapes"]
    x = phantom(n, n, shapes, rng)
    c = (n // 2, n // 2)
    sx, sy = w["sx"], w["sy"]
    psf = gaussian_psf(n, n, c[0], c[1], sx, sy, w["rho"])
    dirs = [noise_direction(n, n, rng) for _ in w["noise"]]
    return Problem(name=name, n_r=n, n_c=n, center=c, bc=w["bc"], op_rank=w["op_rank"],
                   x_true=x, psf=psf, noise_levels=list(w["noise"]), noise_dirs=dirs,
                   lam=w["lam"], tol=w["tol"], maxit=w["maxit"],
                   extra=dict(sigma_x=sx, sigma_y=sy, rho=w["rho"]))


# Batched workload: independent problems of uneven sizes, each with its own
# Gaussian PSF (sigma_x, sigma_y ~ U[1, 8], rho ~ U[-0.8, 0.8]), boundary
# condition (zero or reflexive, fair coin), noise level ~ U[0.1%, 5%] and
# GCV lambda; image shapes scale with the image side as in deblur1024_mixed.
BATCH_SIZES = [(128, 128), (256, 256), (384, 512), (512, 512), (768, 768), (1024, 1024)]
BATCH_INDEX = 3


def make_batch(n_problems: int = 64, sizes=None, seed: int | None = None, op_rank: int = 4) -> list:
    """``n_problems`` raw problem instances for the batched workload (one
    noise level each); ``sizes`` restricts the size set (smaller test runs)."""
    sizes = list(sizes or BATCH_SIZES)
    rng = np.random.default_rng(SEED_BASE + BATCH_INDEX if seed is None else seed)
    out = []
    for k in range(n_problems):
        n_r, n_c = sizes[int(rng.integers(len(sizes)))]
        sx, sy = rng.uniform(1.0, 8.0), rng.uniform(1.0, 8.0)
        rho = rng.uniform(-0.8, 0.8)
        bc = "zero" if rng.uniform() < 0.5 else "reflexive"
        nl = rng.uniform(0.001, 0.05)
        shapes = max(4, int(round(150 * np.sqrt(n_r * n_c) / 1024)))
        x = phantom(n_r, n_c, shapes, rng)
        c = (n_r // 2, n_c // 2)
        psf = gaussian_psf(n_r, n_c, c[0], c[1], sx, sy, rho)
        g = noise_direction(n_r, n_c, rng)
        out.append(Problem(name=f"batch{k}", n_r=n_r, n_c=n_c, center=c, bc=bc, op_rank=op_rank, x_true=x,
                           psf=psf, noise_levels=[nl], noise_dirs=[g], lam=None, tol=1e-7, maxit=500,
                           extra=dict(sigma_x=sx, sigma_y=sy, rho=rho)))
    return out


def random_matrix(m: int, n: int, seed: int) -> np.ndarray:
    """Seeded standard-normal matrix, for operator-level tests."""
    return np.random.default_rng(seed).standard_normal((m, n))
