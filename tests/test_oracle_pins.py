"""Pins for the FP64 CPU oracle against what the mathematics fixes.

None of these compares the oracle with itself: each checks it against a closed
form, an independent direct solver (scipy.fft sine/cosine transforms, dense
numpy solves), a hand-derived fixture, a convergence order or an invariant.
The discretisation is the second-order cell-centred one of Sec. 2, items
(ii)-(iii), applied to Eq. 2 (Poisson) and Eq. 3 (screened Helmholtz).
"""
import os

import numpy as np
import pytest
import scipy.fft as sfft

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def lam(m, n, h):
    """Eigenvalue of the 1D cell-centred second difference, (4/h^2) sin^2(m pi / 2n)."""
    return 4.0 / h**2 * np.sin(m * np.pi / (2 * n)) ** 2


def cc(n):
    return np.arange(n) + 0.5


# ---------------------------------------------------------------- eigenmodes


def test_eigenmode_dirichlet_helmholtz():
    """Homogeneous Dirichlet faces: sin(k pi (i+1/2)/n) is an exact discrete
    eigenvector (ghost = -u); one mode's solution is f / (kappa^2 + sum lambda)."""
    nz, ny, nx = 12, 10, 8
    h = 0.1
    kx, ky, kz = 3, 2, 5
    kappa = 7.0
    mode = (np.sin(kz * np.pi * cc(nz) / nz)[:, None, None]
            * np.sin(ky * np.pi * cc(ny) / ny)[None, :, None]
            * np.sin(kx * np.pi * cc(nx) / nx)[None, None, :])
    lt = kappa**2 + lam(kx, nx, h) + lam(ky, ny, h) + lam(kz, nz, h)
    p = oracle.Problem((nz, ny, nx), h, alpha=kappa**2)
    u, cyc, rel, _ = p.solve(mode)
    assert rel < 1e-12
    np.testing.assert_allclose(u, mode / lt, rtol=0, atol=1e-12 * np.abs(mode / lt).max())


def test_eigenmode_mixed_neumann_dirichlet():
    """Neumann x/y faces (cos modes, ghost = u), Dirichlet z faces (sin modes)."""
    nz, ny, nx = 16, 12, 10
    h = 1.0 / 16
    kx, ky, kz = 0, 4, 3
    mode = (np.sin(kz * np.pi * cc(nz) / nz)[:, None, None]
            * np.cos(ky * np.pi * cc(ny) / ny)[None, :, None]
            * np.cos(kx * np.pi * cc(nx) / nx)[None, None, :])
    lt = lam(kx, nx, h) + lam(ky, ny, h) + lam(kz, nz, h)
    p = oracle.Problem((nz, ny, nx), h, bc_kind=(1, 1, 1, 1, 0, 0))
    r, _ = p.residual(mode, mode / lt)
    assert np.abs(r).max() < 1e-11 * np.abs(mode).max()
    u, _, rel, _ = p.solve(mode)
    np.testing.assert_allclose(u, mode / lt, atol=1e-11 * np.abs(mode / lt).max())


# -------------------------------------------------- fast direct solver (FFT)


def fft_solve(f, h, kind, alpha=0.0):
    """Exact discrete solve with homogeneous BCs per axis (kind per axis in
    (z, y, x) order: 'D' -> DST-II, 'N' -> DCT-II), independent of the oracle."""
    F = np.array(f, dtype=np.float64)
    lamtot = np.full(F.shape, alpha)
    for ax, k in enumerate(kind):
        n = F.shape[ax]
        if k == "D":
            F = sfft.dst(F, type=2, axis=ax, norm="ortho")
            l = lam(np.arange(1, n + 1), n, h)
        else:
            F = sfft.dct(F, type=2, axis=ax, norm="ortho")
            l = lam(np.arange(n), n, h)
        shp = [1, 1, 1]
        shp[ax] = n
        lamtot = lamtot + l.reshape(shp)
    F = F / lamtot
    for ax, k in enumerate(kind):
        F = (sfft.idst if k == "D" else sfft.idct)(F, type=2, axis=ax, norm="ortho")
    return F


@pytest.mark.parametrize("shape", [(16, 24, 32), (32, 32, 32)])
def test_gap_poisson_matches_fft_solver(shape):
    """Gap BCs (phi = 0 at z = 0, 1 at z = 1, Neumann sides), random charge.
    Exact discrete solution = linear ramp (reproduced exactly by the scheme)
    plus the DST(z)/DCT(y,x) solve of the charge term."""
    nz, ny, nx = shape
    h = 1.0 / nz
    rng = np.random.default_rng(3)
    f = rng.standard_normal(shape) * 100.0
    ramp = np.broadcast_to((cc(nz) * h)[:, None, None], shape)
    ref = ramp + fft_solve(f, h, "DNN")
    p = oracle.poisson(shape, h)
    u, cyc, rel, _ = p.solve(f)
    assert rel < 1e-12
    assert oracle.rel_l2(u, ref) < 1e-12


def test_helmholtz_all_dirichlet_matches_fft_solver():
    nz, ny, nx = 16, 16, 24
    h = 1.0 / 16
    rng = np.random.default_rng(4)
    f = np.abs(rng.standard_normal((nz, ny, nx)))
    for kappa in (10.0, 100.0, 1000.0):
        ref = fft_solve(f, h, "DDD", alpha=kappa**2)
        p = oracle.helmholtz((nz, ny, nx), h, kappa)
        u, _, rel, _ = p.solve(f)
        assert oracle.rel_l2(u, ref) < 1e-12, kappa


# ------------------------------------------------ variable permittivity, mask


def _axis_problem(axis, eps1d, g0, g1, extra=3):
    """Layered problem along one axis (0 = z, 1 = y, 2 = x): eps varies with
    the cell index on that axis, Dirichlet g0/g1 on its two faces, Neumann on
    the others, no charge."""
    n = len(eps1d)
    shape = [extra + 1, extra + 2, extra + 3]
    shape[axis] = n
    shp = [1, 1, 1]
    shp[axis] = n
    eps = np.broadcast_to(np.asarray(eps1d, dtype=np.float64).reshape(shp), shape).copy()
    kind = [1] * 6
    val = [0.0] * 6
    face = {0: 4, 1: 2, 2: 0}[axis]
    kind[face] = kind[face + 1] = 0
    val[face], val[face + 1] = g0, g1
    return tuple(shape), shp, eps, kind, val


def _layered_exact(eps1d, h, g0, g1):
    inv = 1.0 / np.asarray(eps1d, dtype=np.float64)
    J = (g1 - g0) / (h * inv.sum())
    return g0 + J * h * (np.concatenate([[0.0], np.cumsum(inv)[:-1]]) + 0.5 * inv)


def test_golden_layered_capacitor_4cell():
    """Hand-derived fixture (tests/golden/layered_capacitor_4cell.txt)."""
    rows = {}
    with open(os.path.join(GOLDEN, "layered_capacitor_4cell.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            rows[key] = np.array([float(v) for v in vals])
    for axis in (0, 1, 2):
        shape, shp, eps, kind, val = _axis_problem(axis, rows["eps"], 0.0, 1.0)
        p = oracle.Problem(shape, 0.25, beta=eps, bc_kind=kind, bc_value=val)
        u, _, rel, _ = p.solve(np.zeros(shape))
        got = np.moveaxis(u, axis, 0).reshape(4, -1)
        for col in got.T:
            np.testing.assert_allclose(col, rows["phi"], rtol=0, atol=1e-13)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_layered_dielectric_exact(axis):
    """Piecewise-constant permittivity per cell along one axis: the harmonic
    face mean makes the discrete flux exact, so the discrete potential equals
    the continuous piecewise-linear solution at cell centres."""
    rng = np.random.default_rng(10 + axis)
    n = 16
    h = 1.0 / n
    eps1d = rng.uniform(1.0, 8.0, n)
    shape, shp, eps, kind, val = _axis_problem(axis, eps1d, 0.3, 1.7)
    p = oracle.Problem(shape, h, beta=eps, bc_kind=kind, bc_value=val)
    u, _, rel, _ = p.solve(np.zeros(shape))
    exact = np.broadcast_to(_layered_exact(eps1d, h, 0.3, 1.7).reshape(shp), shape)
    np.testing.assert_allclose(u, exact, rtol=0, atol=1e-12)


def test_electrode_plane_exact():
    """Electrode cells filling z layers >= K, held at V: the potential is the
    layered solution from the grounded face (distance h/2 to the first centre)
    to the first electrode centre (distance h from the last free centre, with
    the free cell's permittivity).  The top face value must not leak in."""
    n, K, V = 16, 11, 2.5
    h = 1.0 / n
    rng = np.random.default_rng(7)
    eps1d = rng.uniform(1.0, 5.0, n)
    shape = (n, 6, 5)
    eps = np.broadcast_to(eps1d[:, None, None], shape).copy()
    mask = np.zeros(shape, dtype=np.uint8)
    mask[K:] = 1
    u0 = np.zeros(shape)
    u0[K:] = V
    p = oracle.Problem(shape, h, beta=eps, mask=mask, bc_kind=(1, 1, 1, 1, 0, 0),
                       bc_value=(0, 0, 0, 0, 0.0, 123.0))
    u, _, rel, _ = p.solve(np.zeros(shape), u0=u0)
    inv = 1.0 / eps1d[:K]
    res = h * (np.concatenate([[0.0], np.cumsum(inv)[:-1]]) + 0.5 * inv)
    total = h * (inv[:-1].sum() + 0.5 * inv[-1] + inv[-1])
    exact = V * res / total
    np.testing.assert_allclose(u[:K], np.broadcast_to(exact[:, None, None], (K, 6, 5)),
                               rtol=0, atol=1e-12)
    assert np.all(u[K:] == V)


# ------------------------------------------------------------------ order


def _mms_error(n, var_eps):
    """Manufactured solution u = sin(pi x) sin(pi y) sin(pi z), homogeneous
    Dirichlet; optionally eps = 1 + x/2 + y^2/4 + z^3/8 with the analytic
    right-hand side -div(eps grad u)."""
    h = 1.0 / n
    x = cc(n) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    s = np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)
    if not var_eps:
        f, eps = 3 * np.pi**2 * s, None
    else:
        eps = 1 + X / 2 + Y**2 / 4 + Z**3 / 8
        ux = np.pi * np.cos(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)
        uy = np.pi * np.sin(np.pi * X) * np.cos(np.pi * Y) * np.sin(np.pi * Z)
        uz = np.pi * np.sin(np.pi * X) * np.sin(np.pi * Y) * np.cos(np.pi * Z)
        f = eps * 3 * np.pi**2 * s - (0.5 * ux + (Y / 2) * uy + (3 * Z**2 / 8) * uz)
    p = oracle.Problem((n, n, n), h, beta=eps)
    u, _, rel, _ = p.solve(f)
    return np.sqrt(np.mean((u - s) ** 2))


@pytest.mark.parametrize("var_eps", [False, True])
def test_second_order_convergence(var_eps):
    """Sec. 2 items (ii)-(iii) promise second order: halving h cuts the error ~4x."""
    e16, e32 = _mms_error(16, var_eps), _mms_error(32, var_eps)
    assert 3.6 < e16 / e32 < 4.4, e16 / e32


def _gaussian_free_space(x, y, z, c, sig):
    """Potential of a Gaussian charge of unit Q/eps0 and width sig centred at c
    in free space (Eq. 2 with eps = eps0): erf(r / (sqrt(2) sig)) / (4 pi r),
    with its limit sqrt(2/pi) / (4 pi sig) at r = 0."""
    from scipy.special import erf

    r = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
    rs = np.where(r > 1e-12, r, 1.0)
    return np.where(r > 1e-12, erf(rs / (np.sqrt(2.0) * sig)) / (4 * np.pi * rs),
                    np.sqrt(2.0 / np.pi) / (4 * np.pi * sig))


def _gaussian_error(n, c=(0.47, 0.52, 0.5), sig=0.08):
    """RMS error of the oracle's solution of -lap phi = rho/eps0 for the
    Gaussian charge (sampled at cell centres) on the unit cube, with Dirichlet
    data from the free-space potential at every boundary face centre."""
    h = 1.0 / n
    t = cc(n) * h
    Z, Y, X = np.meshgrid(t, t, t, indexing="ij")
    r2 = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2
    f = np.exp(-r2 / (2 * sig * sig)) / ((2 * np.pi) ** 1.5 * sig**3)
    A, B = np.meshgrid(t, t, indexing="ij")  # A: slow index, B: fast index
    g = _gaussian_free_space
    faces = [g(x0, B, A, c, sig).ravel() for x0 in (0.0, 1.0)]   # -x, +x: index k*ny + j
    faces += [g(B, y0, A, c, sig).ravel() for y0 in (0.0, 1.0)]  # -y, +y: index k*nx + i
    faces += [g(B, A, z0, c, sig).ravel() for z0 in (0.0, 1.0)]  # -z, +z: index j*nx + i
    p = oracle.Problem((n, n, n), h, 0.0, None, None, (0,) * 6, (0.0,) * 6,
                       face_data=np.concatenate(faces))
    u, _, rel, _ = p.solve(f)
    assert rel < 1e-12
    return np.sqrt(np.mean((u - g(X, Y, Z, c, sig)) ** 2))


def test_gaussian_charge_closed_form_second_order():
    """The closed-form potential of a Gaussian charge in free space is
    approached at second order: the RMS error falls ~4x per halving of h
    (16 -> 32 -> 64 cells), and at 64^3 it is below 1e-4 of the peak
    potential (about 0.4).  A wrong lift, ghost distance or sign, or a
    dropped term in the face data, breaks the ratio or the size."""
    e = [_gaussian_error(n) for n in (16, 32, 64)]
    assert 3.8 < e[0] / e[1] < 4.3, e
    assert 3.8 < e[1] / e[2] < 4.3, e
    assert e[2] < 1e-4, e


# --------------------------------------------------- invariants, brute force


def _random_small(seed, alpha=0.0):
    rng = np.random.default_rng(seed)
    shape = (5, 6, 7)
    eps = rng.uniform(0.5, 6.0, shape)
    mask = (rng.random(shape) < 0.12).astype(np.uint8)
    mask[2, 3, 3] = 0
    u0 = np.where(mask, rng.uniform(-1, 2, shape), 0.0)
    kind = tuple(int(k) for k in rng.integers(0, 2, 6))
    kind = (0,) + kind[1:]  # at least one Dirichlet face
    val = tuple(float(v) for v in rng.uniform(-1, 1, 6))
    p = oracle.Problem(shape, 0.37, alpha=alpha, beta=eps, mask=mask, bc_kind=kind, bc_value=val)
    f = rng.standard_normal(shape)
    return p, f, u0, mask


def _assemble(p, mask):
    free = np.flatnonzero(mask.reshape(-1) == 0)
    M = np.zeros((free.size, free.size))
    for col, c in enumerate(free):
        e = np.zeros(p.shape)
        e.reshape(-1)[c] = 1.0
        M[:, col] = p.apply(e, homog=True).reshape(-1)[free]
    return M, free


@pytest.mark.parametrize("alpha", [0.0, 3.0])
def test_operator_symmetric_positive_definite(alpha):
    """The finite-volume operator is symmetric (each face flux enters its two
    cells with opposite signs) and positive definite."""
    p, f, u0, mask = _random_small(1, alpha)
    M, _ = _assemble(p, mask)
    assert np.abs(M - M.T).max() < 1e-12 * np.abs(M).max()
    assert np.linalg.eigvalsh(M).min() > 0


@pytest.mark.parametrize("seed", [1, 2])
def test_multigrid_matches_dense_solve(seed):
    """Brute force: the multigrid answer equals a dense solve of the assembled
    system (lifts from boundary and electrode values = minus L of the zero guess)."""
    p, f, u0, mask = _random_small(seed, alpha=0.5 * seed)
    M, free = _assemble(p, mask)
    b = (f - p.apply(u0, homog=False)).reshape(-1)[free]
    x = np.linalg.solve(M, b)
    u, cyc, rel, _ = p.solve(f, u0=u0)
    np.testing.assert_allclose(u.reshape(-1)[free], x, rtol=0, atol=1e-12 * np.abs(x).max())
    assert np.all(u[mask == 1] == u0[mask == 1])


def test_gauss_law_interior_fluxes_cancel():
    """Summing the operator over all free cells leaves only the zeroth-order
    term and the fluxes through Dirichlet faces and electrode faces."""
    n = 12
    h = 1.0 / n
    rng = np.random.default_rng(5)
    eps = rng.uniform(1.0, 4.0, (n, n, n))
    mask = np.zeros((n, n, n), dtype=np.uint8)
    mask[8:10, 5:7, 5:7] = 1
    u = rng.standard_normal((n, n, n))
    u[mask == 1] = 0.7
    kind, val = (1, 1, 1, 1, 0, 0), (0, 0, 0, 0, 0.2, 1.0)
    p = oracle.Problem((n, n, n), h, alpha=0.0, beta=eps, mask=mask, bc_kind=kind, bc_value=val)
    total = p.apply(u)[mask == 0].sum()
    flux = 0.0
    free = mask == 0
    flux += (2 * eps[0] * (u[0] - 0.2) / h**2)[free[0]].sum()
    flux += (2 * eps[-1] * (u[-1] - 1.0) / h**2)[free[-1]].sum()
    for ax in range(3):
        for sgn in (1, -1):
            nb = np.roll(mask, -sgn, axis=ax)
            sl = [slice(None)] * 3
            sl[ax] = slice(-1, None) if sgn == 1 else slice(0, 1)
            nb[tuple(sl)] = 0
            sel = free & (nb == 1)
            flux += (eps * (u - 0.7) / h**2)[sel].sum()
    assert abs(total - flux) < 1e-9 * abs(flux)


def test_convergence_factor_config1():
    """The oracle multigrid is a real multigrid: V(2,2) reduces the residual
    by at least ~7x per cycle on the Gaussian-blob gap problem."""
    from paper_1809_08857_gb300 import workloads as W

    n = 32
    rho = W.gaussian_blobs(n, 0)
    p = oracle.poisson((n, n, n), 1.0 / n)
    u, cyc, rel, hist = p.solve(rho / oracle.EPS0, tol=1e-11)
    factors = hist[1:] / hist[:-1]
    assert rel <= 1e-11
    assert np.median(factors) < 0.15


# --------------------------------------------------- multigrid step identities


def test_rbgs_zeroes_residual_of_updated_colour():
    """After a red half-sweep every red free cell satisfies its own equation
    exactly (red cells couple only to black ones)."""
    p, f, u0, mask = _random_small(3, alpha=1.0)
    rng = np.random.default_rng(9)
    u = np.where(mask, u0, rng.standard_normal(p.shape))
    for color in (0, 1):
        u2 = p.rbgs(f, u, color)
        r, _ = p.residual(f, u2)
        k, j, i = np.indices(p.shape)
        sel = (((i + j + k) & 1) == color) & (mask == 0)
        assert np.abs(r[sel]).max() < 1e-10 * np.abs(f).max()
        other = ((i + j + k) & 1) != color
        assert np.array_equal(u2[other], u[other])


def test_restrict_is_child_average():
    rng = np.random.default_rng(11)
    rf = rng.standard_normal((8, 6, 10))
    got = oracle.restrict(rf, (4, 3, 5))
    ref = rf.reshape(4, 2, 3, 2, 5, 2).mean(axis=(1, 3, 5))
    np.testing.assert_allclose(got, ref, atol=1e-15)


def test_prolong_reproduces_constants_and_linears():
    """Trilinear cell-centred prolongation: weights sum to one (constants are
    kept under Neumann reflection) and linear functions are exact away from
    the boundary."""
    cshape = (4, 5, 6)
    ec = np.full(cshape, 2.5)
    out = oracle.prolong_add(ec, None, (1,) * 6, np.zeros((8, 10, 12)))
    np.testing.assert_allclose(out, 2.5, atol=1e-14)
    Zc, Yc, Xc = np.meshgrid(cc(4) * 2, cc(5) * 2, cc(6) * 2, indexing="ij")
    lin_c = 0.3 * Xc - 0.7 * Yc + 1.1 * Zc
    Zf, Yf, Xf = np.meshgrid(cc(8), cc(10), cc(12), indexing="ij")
    lin_f = 0.3 * Xf - 0.7 * Yf + 1.1 * Zf
    out = oracle.prolong_add(lin_c, None, (1,) * 6, np.zeros((8, 10, 12)))
    np.testing.assert_allclose(out[1:-1, 1:-1, 1:-1], lin_f[1:-1, 1:-1, 1:-1], atol=1e-12)
    # homogeneous Dirichlet ghosts: a boundary fine cell next to a face sees
    # the reflected (negated) coarse value
    out = oracle.prolong_add(np.ones(cshape), None, (0,) * 6, np.zeros((8, 10, 12)))
    assert abs(out[4, 5, 0] - 0.5) < 1e-14  # 3/4 * 1 + 1/4 * (-1)


def test_coarsen_rule():
    """A coarse cell is an electrode iff at least 3 of its 8 children are;
    beta is the mean of the free children."""
    beta = np.arange(1, 65, dtype=np.float64).reshape(4, 4, 4)
    mask = np.zeros((4, 4, 4), dtype=np.uint8)
    mask[0:2, 0:2, 0:2] = 1          # 8 children
    mask[2:4, 2:4, 2:4] = 1
    mask[3, 3, 3] = 0                # 7 children
    mask[0, 2, 0] = mask[1, 3, 1] = 1  # coarse (0, 1, 0): 2 children
    mask[2, 0, 0] = mask[3, 1, 1] = mask[2, 1, 0] = 1  # coarse (1, 0, 0): 3 children
    bc, mc = oracle.coarsen(beta, mask, (4, 4, 4))
    assert mc[0, 0, 0] == 1 and mc[1, 1, 1] == 1 and mc[1, 0, 0] == 1
    assert mc[0, 1, 0] == 0 and mc[0, 0, 1] == 0
    assert bc[1, 1, 1] == beta[3, 3, 3]
    free = beta[0:2, 2:4, 0:2][mask[0:2, 2:4, 0:2] == 0]
    np.testing.assert_allclose(bc[0, 1, 0], free.mean())
    np.testing.assert_allclose(bc[0, 0, 1], beta[0:2, 0:2, 2:4].mean())


# ------------------------------------------------- per-face Dirichlet data


def _faces_of(fun, shape, h):
    """Packed face data of fun(x, y, z) at the boundary face centres."""
    nz, ny, nx = shape
    x, y, z = cc(nx) * h, cc(ny) * h, cc(nz) * h
    Zk, Yj = np.meshgrid(z, y, indexing="ij")
    Zk2, Xi = np.meshgrid(z, x, indexing="ij")
    Yj3, Xi3 = np.meshgrid(y, x, indexing="ij")
    parts = [fun(0.0, Yj, Zk), fun(nx * h, Yj, Zk),
             fun(Xi, 0.0, Zk2), fun(Xi, ny * h, Zk2),
             fun(Xi3, Yj3, 0.0), fun(Xi3, Yj3, nz * h)]
    return np.concatenate([np.broadcast_to(p, q.shape).reshape(-1)
                           for p, q in zip(parts, [Yj, Yj, Xi, Xi, Xi3, Xi3])])


@pytest.mark.parametrize("alpha,eps", [(0.0, 1.0), (0.0, 3.0), (50.0, 1.0)])
def test_face_data_reproduces_linear_potential(alpha, eps):
    """Dirichlet data given per boundary face cell (the sub-box boundary data
    of a refined patch): a linear potential is reproduced exactly at the cell
    centres (the 7-point stencil and the face ghost are exact for linears), so
    any transposed or shifted face index fails."""
    shape = (10, 12, 14)
    h = 0.07
    lin = lambda x, y, z: 0.3 + 1.1 * x - 2.3 * y + 0.7 * z
    fd = _faces_of(lin, shape, h)
    nz, ny, nx = shape
    Z, Y, X = np.meshgrid(cc(nz) * h, cc(ny) * h, cc(nx) * h, indexing="ij")
    exact = lin(X, Y, Z)
    p = oracle.Problem(shape, h, alpha=alpha, beta=np.full(shape, eps), face_data=fd)
    u, _, rel, _ = p.solve(alpha * exact)
    np.testing.assert_allclose(u, exact, rtol=0, atol=1e-12)


# ---------------------------------------------------------------- screened operator


def test_screened_operator_is_alpha_plus_poisson():
    """alpha u - div(beta grad u): alpha enters as alpha * I only (not weighted
    by beta or by the boundary terms), on top of the variable-coefficient
    operator pinned above; checked on a random field, random beta, mixed BCs
    and an electrode block."""
    rng = np.random.default_rng(21)
    shape = (6, 7, 8)
    h = 0.11
    beta = rng.uniform(0.5, 5.0, shape)
    mask = np.zeros(shape, dtype=np.uint8)
    mask[2:4, 3:5, 1:3] = 1
    kinds = (0, 1, 1, 0, 0, 1)
    u = rng.standard_normal(shape)
    a0 = oracle.Problem(shape, h, 0.0, beta, mask, kinds).apply(u, homog=True)
    a1 = oracle.Problem(shape, h, 7.5, beta, mask, kinds).apply(u, homog=True)
    free = mask == 0
    np.testing.assert_allclose((a1 - a0)[free], 7.5 * u[free], rtol=1e-12, atol=1e-9)


def test_screened_constant_solutions():
    """Neumann on every face: constant u = f / alpha whatever beta is (no flux
    through any face).  Dirichlet value g on every face and f = alpha g: u = g
    (the ghost 2g - u equals u)."""
    rng = np.random.default_rng(22)
    shape = (8, 10, 12)
    h = 1.0 / 12
    beta = rng.uniform(0.2, 8.0, shape)
    alpha = 3.7
    p = oracle.Problem(shape, h, alpha, beta, None, (1,) * 6)
    u, _, _, _ = p.solve(np.full(shape, alpha * 2.5))
    np.testing.assert_allclose(u, 2.5, rtol=1e-12)
    p = oracle.Problem(shape, h, alpha, beta, None, (0,) * 6, (-1.25,) * 6)
    u, _, _, _ = p.solve(np.full(shape, alpha * -1.25))
    np.testing.assert_allclose(u, -1.25, rtol=1e-12)


def test_screened_neumann_conserves():
    """Neumann on every face: the sum over cells of (alpha u - div(beta grad
    u)) equals alpha times the sum of u for any u (interior face fluxes
    cancel pairwise), so a diffusion factor (I - mu L) keeps the total."""
    rng = np.random.default_rng(23)
    shape = (9, 8, 7)
    h = 0.2
    beta = rng.uniform(0.1, 3.0, shape)
    u = rng.standard_normal(shape)
    au = oracle.Problem(shape, h, 2.0, beta, None, (1,) * 6).apply(u)
    assert abs(au.sum() - 2.0 * u.sum()) <= 1e-10 * np.abs(au).sum()


# ---------------------------------------------------------------- Robin (Marshak) faces


def robin_mode(n, h, a):
    """Lowest discrete eigenvector of the 1D cell-centred second difference
    with the Robin ghost u_g = g u_c, g = (1 - ah/2)/(1 + ah/2), on both ends:
    u_i = cos(theta (i + 1/2) + phi), found from the two end conditions
    (tan phi = -(ah/2) cot(theta/2) from the low end, a scalar root for theta
    from the high end).  Returns (u, lambda) with lambda = (2 - 2 cos theta)/h^2."""
    from scipy.optimize import brentq

    gam = (1 - a * h / 2) / (1 + a * h / 2)
    phi_of = lambda t: np.arctan(-(a * h / 2) / np.tan(t / 2))
    F = lambda t: (np.cos(t * (n + 0.5) + phi_of(t)) - gam * np.cos(t * (n - 0.5) + phi_of(t)))
    t = brentq(F, 1e-9, np.pi / n - 1e-12)
    u = np.cos(t * (np.arange(n) + 0.5) + phi_of(t))
    # the low-end condition holds by construction; check the high end too
    assert abs(np.cos(t * (n + 0.5) + phi_of(t)) - gam * u[-1]) < 1e-10
    return u, (2 - 2 * np.cos(t)) / h**2


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("a", [0.5, 7.0, 60.0])
def test_robin_eigenmode(axis, a):
    """A mode along one axis with Robin faces on that axis (Neumann on the
    others) is an eigenvector of the discrete operator with eigenvalue
    alpha + lambda; solving with f = (alpha + lambda) u returns u."""
    n = 16
    h = 1.0 / n
    u1, lam1 = robin_mode(n, h, a)
    shape = [6, 7, 8]
    shape[2 - axis] = n
    shape = tuple(shape)
    kinds = [1] * 6
    vals = [0.0] * 6
    kinds[2 * axis] = kinds[2 * axis + 1] = 2
    vals[2 * axis] = vals[2 * axis + 1] = a
    bshape = [1, 1, 1]
    bshape[2 - axis] = n
    u = np.broadcast_to(u1.reshape(bshape), shape).copy()
    alpha = 3.0
    p = oracle.Problem(shape, h, alpha, None, None, kinds, vals)
    got, _, rel, _ = p.solve((alpha + lam1) * u)
    np.testing.assert_allclose(got, u, rtol=0, atol=1e-11)


def test_robin_limits():
    """a = 0 is the Neumann face; a very large a is the homogeneous Dirichlet
    face (the ghost factor tends to -1)."""
    rng = np.random.default_rng(31)
    shape = (8, 8, 8)
    h = 1.0 / 8
    f = rng.standard_normal(shape)
    ref_n, _, _, _ = oracle.Problem(shape, h, 2.0, None, None, (1,) * 6).solve(f)
    got, _, _, _ = oracle.Problem(shape, h, 2.0, None, None, (2,) * 6, (0.0,) * 6).solve(f)
    np.testing.assert_allclose(got, ref_n, rtol=0, atol=1e-12)
    ref_d, _, _, _ = oracle.Problem(shape, h, 2.0, None, None, (0,) * 6).solve(f)
    got, _, _, _ = oracle.Problem(shape, h, 2.0, None, None, (2,) * 6, (1e14,) * 6).solve(f)
    assert oracle.rel_l2(got, ref_d) < 1e-11
