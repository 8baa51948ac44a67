"""Seeded synthetic particle systems shared by the tests, the benchmark and
the oracle's callers.

This module only draws inputs; it holds none of the method's arithmetic.
Every generator returns float64 numpy arrays of shape ``(N, 3)``:
positions ``x``, force weights ``f``, dipole weights ``h`` and normals ``nu``
(the quantities of eq. (1.3)).  Seeds are explicit so that the CUDA path and
the oracle see bit-identical inputs.

Workloads (the paper's own test cases are synthetic, Section 6):

* ``uniform_cube``       -- N points uniform in [0, side]^3; f, h uniform in
                            [-1, 1]^3; nu uniform random unit vectors.
* ``density_cube``       -- test case 2: random Stokeslets in a cube of number
                            density N / L^3 = 2500, stresslet omitted (h = 0).
* ``icosahedral_sphere`` -- test case 1: centroids of an L-times refined
                            icosahedral triangulation (N = 20 * 4^L) projected
                            to the unit sphere; f, h and nu uniform in
                            [-1, 1]^3 (the reading under which the errors of
                            Table 1 are reproduced; ``normals=True`` gives the
                            outward normal instead).
* ``fibonacci_sphere``   -- quasi-uniform spherical Fibonacci lattice of any N,
                            f, h ~ N(0, 1)^3, nu = outward normal.
* ``gaussian_clusters``  -- 8 Gaussian blobs (sigma 0.05) centred at
                            {0.25, 0.75}^3.
* ``batch_sizes``        -- system sizes drawn log-uniform in [lo, hi].
"""
import numpy as np

SEED_BASE = 181112498


def _unit_vectors(rng, n):
    v = rng.standard_normal((n, 3))
    nrm = np.sqrt(np.sum(v * v, axis=1, keepdims=True))
    nrm[nrm == 0] = 1.0
    return v / nrm


def uniform_cube(N, seed, side=1.0, stresslet=True):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, side, size=(N, 3))
    f = rng.uniform(-1.0, 1.0, size=(N, 3))
    h = rng.uniform(-1.0, 1.0, size=(N, 3))
    nu = _unit_vectors(rng, N)
    if not stresslet:
        h[:] = 0.0
    return x, f, h, nu


def density_cube(N, seed, density=2500.0):
    """Test case 2 (Section 6.1.2): side L with N / L^3 = density, h = 0."""
    L = (N / density) ** (1.0 / 3.0)
    return uniform_cube(N, seed, side=L, stresslet=False)


def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    return v, f


def icosahedral_sphere(L, seed, normals=False):
    """Test case 1 (Section 6.1.1): N = 20 * 4^L particles on the unit sphere.

    Each face is split into four by its edge midpoints; new vertices are
    pushed onto the sphere at every level (geodesic refinement).  Particles
    are the face centroids projected onto the sphere.  f and h are uniform in
    [-1, 1]^3 as the paper states.  The paper does not say how nu was drawn
    for this test (Section 1 defines nu as a unit vector; Section 6 draws the
    weights as random numbers in [-1, 1]).  Components uniform in [-1, 1]
    (the default) reproduce the 18 errors of Table 1(a) within factors 0.87
    to 1.18 (geometric mean 1.02); random unit vectors within 0.98 to 1.51
    (mean 1.18); the outward normal (normals=True) gives errors ten times
    larger, because on a sphere the stresslet velocity of outward normals
    nearly cancels (its RMS is 50 times smaller than with random directions)
    while its truncation error does not.
    """
    v, faces = _icosahedron()
    for _ in range(L):
        e = np.concatenate([faces[:, [0, 1]], faces[:, [1, 2]], faces[:, [2, 0]]])
        e.sort(axis=1)
        uniq, inv = np.unique(e, axis=0, return_inverse=True)
        inv = inv.reshape(-1)
        mid = v[uniq[:, 0]] + v[uniq[:, 1]]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        base = v.shape[0]
        v = np.concatenate([v, mid])
        nf = faces.shape[0]
        m01 = base + inv[:nf]
        m12 = base + inv[nf:2 * nf]
        m20 = base + inv[2 * nf:]
        a, b, c = faces[:, 0], faces[:, 1], faces[:, 2]
        faces = np.concatenate([np.stack([a, m01, m20], 1), np.stack([m01, b, m12], 1),
                                np.stack([m20, m12, c], 1), np.stack([m01, m12, m20], 1)])
    cen = v[faces].mean(axis=1)
    x = cen / np.linalg.norm(cen, axis=1, keepdims=True)
    rng = np.random.default_rng(seed)
    N = x.shape[0]
    f = rng.uniform(-1.0, 1.0, size=(N, 3))
    h = rng.uniform(-1.0, 1.0, size=(N, 3))
    nu = x.copy() if normals else rng.uniform(-1.0, 1.0, size=(N, 3))
    return np.ascontiguousarray(x), f, h, nu


def fibonacci_sphere(N, seed):
    """Quasi-uniform points on the unit sphere; f, h ~ N(0,1)^3; nu = x."""
    i = np.arange(N, dtype=np.float64) + 0.5
    z = 1.0 - 2.0 * i / N
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = np.pi * (3.0 - 5.0 ** 0.5) * i
    x = np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((N, 3))
    h = rng.standard_normal((N, 3))
    return x, f, h, x.copy()


def gaussian_clusters(N, seed, sigma=0.05):
    """N points in 8 Gaussian blobs centred at {0.25, 0.75}^3 (not clipped)."""
    rng = np.random.default_rng(seed)
    centres = np.array([[a, b, c] for a in (0.25, 0.75) for b in (0.25, 0.75) for c in (0.25, 0.75)])
    which = np.arange(N) % 8
    x = centres[which] + sigma * rng.standard_normal((N, 3))
    f = rng.uniform(-1.0, 1.0, size=(N, 3))
    h = rng.uniform(-1.0, 1.0, size=(N, 3))
    nu = _unit_vectors(rng, N)
    return x, f, h, nu


def batch_sizes(nsys, seed, lo=10_000, hi=500_000):
    rng = np.random.default_rng(seed)
    return np.round(np.exp(rng.uniform(np.log(lo), np.log(hi), size=nsys))).astype(np.int64)


def sample_indices(N, count, seed):
    """Distinct target indices drawn without replacement (seeded)."""
    rng = np.random.default_rng(seed)
    count = min(int(count), int(N))
    return np.sort(rng.choice(N, size=count, replace=False))
