"""CPU checks of the seeded input generators (paper_2311_15393_gb300/synth.py):
the image generator paints exactly what its description says, and the
batched workload draws its problems from the stated distributions,
reproducibly."""
import numpy as np

from paper_2311_15393_gb300 import synth


def _phantom_full_grid(n_r, n_c, n_shapes, rng):
    """The phantom's description evaluated on the whole grid for every shape
    (no bounding boxes): the reference the generator must equal."""
    X = np.zeros((n_r, n_c))
    ii, jj = np.meshgrid(np.arange(n_r, dtype=float), np.arange(n_c, dtype=float), indexing="ij")
    for _ in range(n_shapes):
        cy, cx = rng.uniform(0.0, n_r), rng.uniform(0.0, n_c)
        ell = rng.uniform() < 0.5
        hx, hy = rng.uniform(n_c / 32.0, n_c / 8.0), rng.uniform(n_r / 32.0, n_r / 8.0)
        th, val = rng.uniform(0.0, np.pi), rng.uniform(0.0, 1.0)
        dx, dy = jj - cx, ii - cy
        if ell:
            u = (dx * np.cos(th) + dy * np.sin(th)) / hx
            v = (-dx * np.sin(th) + dy * np.cos(th)) / hy
            m = u * u + v * v <= 1.0
        else:
            m = (np.abs(dx) <= hx) & (np.abs(dy) <= hy)
        X[m] = val
    return X


def test_phantom_equals_its_full_grid_definition():
    for seed, (n_r, n_c, k) in enumerate([(64, 64, 12), (48, 80, 20), (128, 96, 40)]):
        a = synth.phantom(n_r, n_c, k, np.random.default_rng(seed))
        b = _phantom_full_grid(n_r, n_c, k, np.random.default_rng(seed))
        assert np.array_equal(a, b)


def test_batch_draws_from_the_stated_distributions():
    probs = synth.make_batch(64)
    sizes = {(p.n_r, p.n_c) for p in probs}
    assert sizes <= set(synth.BATCH_SIZES) and len(sizes) >= 4
    assert {p.bc for p in probs} == {"zero", "reflexive"}
    for p in probs:
        e = p.extra
        assert 1.0 <= e["sigma_x"] <= 8.0 and 1.0 <= e["sigma_y"] <= 8.0 and -0.8 <= e["rho"] <= 0.8
        assert 0.001 <= p.noise_levels[0] <= 0.05
        assert p.psf.shape == (p.n_r, p.n_c) and abs(p.psf.sum() - 1.0) < 1e-12
        assert p.center == (p.n_r // 2, p.n_c // 2)
        assert p.x_true.shape == (p.n_r, p.n_c) and p.noise_dirs[0].shape == (p.n_r, p.n_c)


def test_batch_is_reproducible_and_seeded():
    a = synth.make_batch(5, sizes=[(128, 128)])
    b = synth.make_batch(5, sizes=[(128, 128)])
    c = synth.make_batch(5, sizes=[(128, 128)], seed=1)
    for p, q in zip(a, b):
        assert np.array_equal(p.x_true, q.x_true) and np.array_equal(p.psf, q.psf)
        assert p.noise_levels == q.noise_levels and p.bc == q.bc
    assert any(not np.array_equal(p.psf, q.psf) for p, q in zip(a, c))


def test_gaussian_psf_moments_fix_the_axes():
    """The PSF is the bivariate normal with sigma_x along the columns (x),
    sigma_y along the rows (y) and correlation rho, normalised to sum 1: on a
    grid reaching 20 sigma from the centre the sampled second moments about
    the centre equal the covariance [[sx^2, rho sx sy], [rho sx sy, sy^2]] (the
    grid sums of a Gaussian match its integrals to far below rounding), and
    the peak sits at the centre."""
    sx, sy, rho, n, c = 3.0, 1.5, 0.5, 128, (64, 60)
    P = synth.gaussian_psf(n, n, c[0], c[1], sx, sy, rho)
    assert abs(P.sum() - 1.0) < 1e-14
    assert np.unravel_index(np.argmax(P), P.shape) == c
    dy = np.arange(n)[:, None] - c[0]
    dx = np.arange(n)[None, :] - c[1]
    np.testing.assert_allclose([np.sum(P * dx * dx), np.sum(P * dy * dy), np.sum(P * dx * dy)],
                               [sx * sx, sy * sy, rho * sx * sy], rtol=1e-12)
    np.testing.assert_allclose([np.sum(P * dx), np.sum(P * dy)], [0.0, 0.0], atol=1e-12)
