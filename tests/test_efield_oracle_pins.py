"""Pins of the electric-field / relaxation-time oracle (oracle/efield.py)
against closed forms and brute-force loops (no GPU)."""
import numpy as np

from oracle import efield as EF


def centres(n, h):
    return (np.arange(n) + 0.5) * h


def test_linear_potential_gives_its_gradient_everywhere():
    """phi = a + b x along one axis with Dirichlet faces holding phi's face
    values on that axis (Neumann on the others): the ghost 2g - phi_c is the
    linear extrapolation, so E = -b in every cell, 0 across."""
    shape = (6, 7, 8)
    h = 0.1
    b = np.array([0.7, -1.3, 2.1])  # d/dx, d/dy, d/dz
    z, y, x = [centres(m, h) for m in shape]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    L = (shape[2] * h, shape[1] * h, shape[0] * h)
    for axis in range(3):
        phi = 0.4 + b[axis] * (X, Y, Z)[axis]
        g = [0.0] * 6
        g[2 * axis] = 0.4
        g[2 * axis + 1] = 0.4 + b[axis] * L[axis]
        kinds = [1] * 6
        kinds[2 * axis] = kinds[2 * axis + 1] = 0
        E = EF.efield(phi, h, kinds, g)
        np.testing.assert_allclose(E[axis], -b[axis], rtol=1e-12)
        for other in range(3):
            if other != axis:
                np.testing.assert_allclose(E[other], 0.0, atol=1e-12)


def test_quadratic_potential_exact_inside():
    """Centred differences are exact for quadratics at interior cells."""
    shape = (7, 6, 9)
    h = 0.05
    z, y, x = [centres(m, h) for m in shape]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    phi = 1.0 + X * X - 2.0 * Y * Z + 0.5 * Z * Z
    E = EF.efield(phi, h, (1,) * 6, (0.0,) * 6)
    inner = np.s_[1:-1, 1:-1, 1:-1]
    np.testing.assert_allclose(E[0][inner], -2.0 * X[inner], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(E[1][inner], 2.0 * Z[inner], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(E[2][inner], 2.0 * Y[inner] - Z[inner], rtol=1e-10, atol=1e-12)


def brute(phi, h, kinds, vals, mask, J):
    nz, ny, nx = phi.shape
    E = np.zeros((3, nz, ny, nx))
    best = np.inf
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                if mask[k, j, i]:
                    continue
                c = (k, j, i)
                for ax, (d, fm, fp) in enumerate(((2, 0, 1), (1, 2, 3), (0, 4, 5))):
                    lo = list(c)
                    hi = list(c)
                    lo[d] -= 1
                    hi[d] += 1
                    n = phi.shape[d]
                    pm = phi[tuple(lo)] if lo[d] >= 0 else (
                        2 * vals[fm] - phi[c] if kinds[fm] == 0 else phi[c])
                    pp = phi[tuple(hi)] if hi[d] < n else (
                        2 * vals[fp] - phi[c] if kinds[fp] == 0 else phi[c])
                    E[ax][c] = (pm - pp) / (2 * h)
                jn = np.sqrt(sum(J[a][c] ** 2 for a in range(3)))
                en = np.sqrt(sum(E[a][c] ** 2 for a in range(3)))
                if jn > 0:
                    best = min(best, EF.EPS0 * en / jn)
    return E, best


def test_matches_brute_force_loops():
    rng = np.random.default_rng(3)
    shape = (4, 5, 6)
    h = 0.3
    phi = rng.standard_normal(shape)
    mask = np.zeros(shape, dtype=np.uint8)
    mask[1:3, 2, 2:4] = 1
    J = rng.standard_normal((3,) + shape)
    J[:, 0, 0, 0] = 0.0
    kinds = (0, 1, 1, 0, 0, 1)
    vals = (0.3, 0.0, 0.0, -0.7, 1.1, 0.0)
    E_ref, dt_ref = brute(phi, h, kinds, vals, mask, J)
    E = EF.efield(phi, h, kinds, vals, mask)
    np.testing.assert_allclose(E, E_ref, rtol=1e-14, atol=1e-14)
    assert EF.relaxation_time(E, J, mask) == dt_ref
    assert EF.relaxation_time(E, np.zeros_like(J), mask) == np.inf
